/*
 * tbmd.h -- C ABI of the GB300 (sm_103a) Fast-QMMD / SP2 density-matrix library.
 *
 * Implements the per-step hot path of optimization-free extended-Lagrangian
 * Born-Oppenheimer MD for orthogonal self-consistent-charge tight binding
 * (Niklasson & Cawkwell, "Fast method for quantum mechanical molecular
 * dynamics"): the Hamiltonian H[n] (App. D, Eq. DFTB_2 with S = I,
 * Eq. EL_Orth_c), the density matrix D = theta(mu0 I - H[n]) by SP2
 * purification (Sec. III.B, App. D.2) or the Fermi operator at T_e > 0
 * (Eq. EL_4c, Eq. DM_perp), Mulliken charges (App. D), forces and energy
 * (Eq. EL_Orth_a, Eq. Etot_Orth) and the XL-BOMD integration of R and of the
 * auxiliary charges n (velocity Verlet; Eq. Verl_n).
 *
 * Conventions
 *   - Plain C, every function returns int: TB_OK (0) or a negative TB_ERR_*.
 *     No C++ exception crosses the ABI.
 *   - Units: eV, Angstrom, amu, fs.  Velocities in A/fs.
 *   - Every array pointer is a DEVICE pointer owned by the caller unless a
 *     comment says otherwise.  Matrices are dense, row-major, symmetric,
 *     leading dimension = n, orbitals grouped by atom (O-like: s, px, py, pz;
 *     H-like: s).
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as
 *     void*; NULL = legacy default stream).  A call returns after enqueueing:
 *     the return value reports argument and launch errors only.  Convergence
 *     and numerical status are written to the device-side report structs,
 *     valid after the stream has been synchronised.
 *   - Entry points that need scratch memory take a caller-allocated device
 *     workspace and its size; the matching *_workspace_size query gives the
 *     minimum.  The library itself calls no cudaMalloc.
 *   - A context is bound to the device current when it was created; calls
 *     must be made with that device current.
 */
#ifndef TBMD_H
#define TBMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TB_OK                  0
#define TB_ERR_ARG            -1  /* invalid argument (null pointer, bad size, workspace too small) */
#define TB_ERR_NOT_CONVERGED  -2  /* iteration cap reached (report status only) */
#define TB_ERR_GAP            -3  /* no gap at N_occ: trace cannot reach N_occ (report status only) */
#define TB_ERR_OOM            -4  /* capacity or admission budget exceeded */
#define TB_ERR_TIMEOUT        -5  /* a device-side wait gave up after its time limit */
#define TB_ERR_CUDA           -6  /* a CUDA runtime call or launch failed */
#define TB_ERR_UNSUPPORTED    -7  /* option not supported on this device/build */

/* atom types */
#define TB_TYPE_O 0  /* s, px, py, pz */
#define TB_TYPE_H 1  /* s */

/* arithmetic of the purification GEMMs */
#define TB_PREC_FP64    0  /* FP64 FMA (the plain FP64 path) */
#define TB_PREC_TF32    1  /* tcgen05 kind::tf32, FP32 accumulate */
#define TB_PREC_TF32X3  2  /* tcgen05 kind::tf32 on hi/lo splits: hi*hi + hi*lo + lo*hi (squares in the
                              grouped, block-sparse and Fermi products also lo*lo, which keeps
                              their diagonal unbiased) */
#define TB_PREC_BF16    3  /* tcgen05 kind::f16 (bf16), FP32 accumulate */
#define TB_PREC_BF16X3  4  /* tcgen05 kind::f16 (bf16) on hi/lo splits */

typedef struct tb_ctx tb_ctx;

/* Model constants of the orthogonal SCC-TB recipe (App. D).  Hopping
 * V(r) = t_hop exp(-r/r_decay), Slater-Koster two-centre table with
 * ss-sigma = -V, sp-sigma = +V, pp-sigma = +V, pp-pi = -V; V and the pair
 * potential phi(r) = pair_a exp(-r/pair_rho) are replaced on [r1, rcut) by
 * the quintic tail of App. D.  gamma(r) = coulomb_k / sqrt(r^2 + (coulomb_k/
 * hubbard_u)^2) * w(r/gamma_cut), w(x) = (1-x)^4 (1+4x), summed over periodic
 * images (gamma_form 0), or the Ewald-summed Gaussian-charge gamma (gamma_form 1). */
typedef struct {
  double eps_s_O, eps_p_O, eps_s_H;   /* onsite energies */
  double t_hop, r_decay;              /* hopping magnitude and decay length */
  double hubbard_u, coulomb_k, gamma_cut;
  double r1, rcut;                    /* tail start, cut-off of h and phi */
  double n0_O, n0_H;                  /* valence electrons of the neutral atoms */
  double pair_a, pair_rho;            /* E_pair (pair_a = 0: off) */
  /* App. D radial form zeta(R) = A0 exp(A1 R + A2 R^2 + A3 R^3 + A4 R^4): A0 = t_hop (pair_a),
   * A1 = -1/r_decay (-1/pair_rho); these are A2..A4 of the bond integrals and of phi (0: plain
   * exponentials).  The App. D tail matches zeta, zeta', zeta'' at r1. */
  double zeta_a2, zeta_a3, zeta_a4;
  double pair_a2, pair_a3, pair_a4;
  /* gamma_form 0: the windowed gamma above.  1: long-range gamma of Gaussian charges,
   * gamma_ij = coulomb_k sum_T erf(|R_j - R_i + T|/c)/|R_j - R_i + T| over all periodic images T
   * (Ewald summation with a neutralising background), c = 2 coulomb_k/(hubbard_u sqrt(pi)) so
   * that the on-site term is U; gamma_cut is then unused.  ewald_alpha: Ewald splitting (1/A),
   * 0 = 6.5/max(box, 10 A).  The Ewald gamma costs O(N^2 (images + reciprocal vectors)) per build
   * and per force call. */
  int gamma_form;
  double ewald_alpha;
  /* Basis-set overlap between atoms (App. D.1; non-orthogonal formulation when overlap_s0 != 0):
   * S is the unit matrix on site and, between atoms, minus the Slater-Koster table above
   * evaluated with s(r) = overlap_s0 exp(-r/overlap_rs) (with the App. D tail on [r1, rcut)),
   * i.e. ss-sigma = +s, sp-sigma = -s, pp-sigma = -s, pp-pi = +s.  overlap_s0 = 0: S = I,
   * the orthogonal model (tb_build_H); otherwise use tb_build_HS, dm_nonorth,
   * mulliken_nonorth and tb_forces_nonorth (xlbomd_* switch to them by themselves). */
  double overlap_s0, overlap_rs;
} tb_params;

/* A periodic system.  types and orb_off are device arrays. */
typedef struct {
  int natoms;                 /* N >= 1 */
  int norb;                   /* n = orb_off[N] */
  const int32_t* types;       /* [N] TB_TYPE_O / TB_TYPE_H */
  const int32_t* orb_off;     /* [N+1] first orbital of atom i; orb_off[N] = n */
  double box;                 /* cubic box side (A) > 0 */
} tb_system;

/* Options of dm_sp2. */
typedef struct {
  int precision;        /* TB_PREC_* of the purification GEMMs */
  int max_iter;         /* cap on projections of the main phase, 1..120 */
  double tol;           /* stop when Tr X - Tr X^2 <= tol (FP64 path) */
  int refine_iters;     /* FP64 projections after a tensor-core phase, 0..4 */
  int rule;             /* 0: X^2 when |Tr X^2 - N| <= |2Tr X - Tr X^2 - N| (look-ahead), 1: X^2 when Tr X > N */
  int refine_mode;      /* 0: refinement products emulate FP64 exactly on the bf16 tensor cores
                           (integer slices, FP64 result; needs n <= 4096, else FP64 FMA is used);
                           1: FP64 FMA */
  double tau;           /* > 0: thresholded block-sparse SP2 (Sec. III.B): after X0 and after every
                           projection, 32 x 32 blocks with Frobenius norm < tau are set to zero;
                           tensor-core precisions only, n <= 131072, no refinement */
  int bsr_blocks_per_row; /* capacity of the block-sparse pattern in 128 x 128 blocks per block
                             row (0: all, never overflows); exceeding it reports TB_ERR_OOM */
} tb_sp2_opts;

/* Written on the device by dm_sp2 (caller-owned device memory). */
typedef struct {
  int status;           /* TB_OK, TB_ERR_NOT_CONVERGED, TB_ERR_GAP, TB_ERR_TIMEOUT */
  int iters;            /* projections of the main phase */
  int refine_iters;     /* FP64 refinement projections applied */
  int n;                /* matrix size */
  double eps_min, eps_max;  /* Gershgorin bounds of H */
  double trace;         /* Tr D */
  double idem_trace;    /* Tr D - Tr D^2 of the returned D */
  double idem_fro;      /* ||X^2 - X||_F of the input of the last FP64 projection, -1 if none */
  uint64_t branch_bits[2];  /* bit k: branch of main-phase projection k (1 = 2X - X^2) */
  uint64_t refine_bits;     /* bit k: branch of refinement projection k */
  int64_t block_products;   /* block-sparse path: 128 x 128 block products of the full products
                               X X over all projections (2 * 128^3 flops each; the kernel
                               computes the upper-triangle blocks, about half, and mirrors
                               them); 0 on the dense paths */
  int64_t blocks;           /* block-sparse path: stored 128 x 128 blocks of the returned D; else 0 */
} tb_sp2_report;

/* ---------------------------------------------------------------- context */

/* Create a context on the current device.  *ctx is owned by the caller and
 * released with tb_ctx_destroy.  Fails with TB_ERR_UNSUPPORTED when the
 * device is not sm_103 (the library contains sm_103a code only). */
int tb_ctx_create(tb_ctx** ctx);
int tb_ctx_destroy(tb_ctx* ctx);
/* Static description of a status code. */
const char* tb_status_string(int status);
/* Last error message recorded by the context (valid until the next call). */
const char* tb_ctx_last_error(const tb_ctx* ctx);

/* Launch timing (measurement support, no counterpart in the paper).  With
 * profiling on, dm_sp2 records CUDA events on its stream between the
 * purification launches of its main phase (phase 0) and of its FP64
 * refinement (phase 1).  tb_ctx_sp2_launch_times waits for the last event
 * and writes the duration (ms) of each launch of the last dm_sp2 call into
 * the HOST array ms[0..cap), *count = launches written.  Launches after the
 * device-side stop decision return at once and show as short entries.
 * Block-sparse path (tau > 0): phase 0 entry k is the whole projection k
 * (symbolic and numeric kernels); phase 1 holds events around the numeric
 * kernels, so its entry 2k is numeric kernel k and entry 2k+1 the symbolic
 * kernels of projection k+1.  At most 130 entries per phase are kept. */
int tb_ctx_set_profiling(tb_ctx* ctx, int enable);
int tb_ctx_sp2_launch_times(tb_ctx* ctx, int phase, float* ms, int cap, int* count);

/* Execution controls (no counterpart in the paper; for testing and tuning).
 * tb_ctx_set_grid_limit caps the CTAs of the persistent tensor-core grids
 * (dense projections, Fermi-expansion products, block-sparse products) at
 * max_ctas (0: one CTA per SM, the default).  A smaller grid makes every CTA
 * walk more tiles, so a small matrix runs the same multi-round schedule
 * (several tiles per CTA, reuse of the two TMEM accumulators, 64-column half
 * units in the last round) as a large one on the whole GPU; results are the
 * same up to the order of the FP64 trace sums.  TB_ERR_ARG for max_ctas < 0.
 * tb_ctx_set_wait_limit sets the time limit, in ns of the device's global
 * timer (1 .. 2e9; default 2e9), of the pipeline waits (data and accumulator
 * barriers) of the dense-projection and Fermi-product kernels.  A wait that
 * runs out makes the kernel stop its pipeline, wait (at the full 2 s limit)
 * for its own copies and MMAs in flight, free its TMEM and return; the call's
 * report then says TB_ERR_TIMEOUT and the context stays usable.  Both apply
 * to calls enqueued after them. */
int tb_ctx_set_grid_limit(tb_ctx* ctx, int max_ctas);
int tb_ctx_set_wait_limit(tb_ctx* ctx, unsigned long long ns);

/* Kernel form of dm_sp2's dense tensor-core projections (a4).  When the
 * padded size ld is a multiple of 256, a projection can run on CTA pairs:
 * clusters of two CTAs computing 256 x 256 tiles with one
 * tcgen05.mma.cta_group::2, which halves the operand bytes each SM loads per
 * flop; otherwise (and for every other tensor-core product) one CTA computes
 * a 128 x 128 tile.  TB_SP2_FORM_AUTO (the default) takes the pair form
 * where its tile schedule is predicted to finish first (on GB300: ld = 4096
 * and up), TB_SP2_FORM_SINGLE never, TB_SP2_FORM_PAIRS wherever ld allows.
 * Both forms compute the same products in the same order; results agree to
 * the order of the FP64 trace sums.  A grid limit (tb_ctx_set_grid_limit)
 * caps the pair form at max_ctas / 2 clusters.  TB_ERR_ARG for an unknown
 * form; applies to calls enqueued after it. */
#define TB_SP2_FORM_AUTO 0
#define TB_SP2_FORM_SINGLE 1
#define TB_SP2_FORM_PAIRS 2
int tb_ctx_set_sp2_form(tb_ctx* ctx, int form);
/* The form (TB_SP2_FORM_SINGLE or TB_SP2_FORM_PAIRS) and the CTAs of the
 * persistent grid of the dense tensor-core projection dm_sp2 launches for
 * size n under the context's current settings (host only; queries the
 * device's cluster occupancy once).  TB_ERR_ARG for n < 1 or a null pointer. */
int tb_ctx_sp2_form_of(tb_ctx* ctx, int n, int* form, int* ctas);

/* ----------------------------------------------------------- a1: H[n] build */

/* H[n] = h(R) + diag(sum_l gamma_il n_l) over every orbital of atom i
 * (App. D, Eq. DFTB_2 with S = I; Eq. EL_Orth_c).
 *   R      [N*3] positions (any image; minimum-image convention applied)
 *   n_aux  [N] auxiliary charges n (NULL: all zero)
 *   H      [n*n] output, fully overwritten
 *   gamma  [N*N] output: gamma_ij summed over periodic images, gamma_ii
 *          includes U and the self-image terms. */
int tb_build_H(tb_ctx* ctx, const tb_params* p, const tb_system* sys,
               const double* R, const double* n_aux, double* H, double* gamma,
               void* stream);

/* ------------------------------------------------- a2..a6: SP2 purification */

/* Minimum workspace bytes of dm_sp2 for an n x n matrix. */
int dm_sp2_workspace_size(int n, const tb_sp2_opts* opts, size_t* bytes);

/* D = theta(mu0 I - H) with Tr D = n_occ by the SP2 recursion (Sec. III.B):
 * X0 = (eps_max I - H)/(eps_max - eps_min) from Gershgorin bounds; repeat
 * X <- X^2 or 2X - X^2 (branch chosen by trace, opts->rule) until
 * Tr X - Tr X^2 <= tol, then opts->refine_iters FP64 projections when the main
 * phase ran on the tensor cores.  Traces are accumulated in FP64.
 *   H [n*n] input (FP64), D [n*n] output (FP64), report: device, may be NULL.
 * Branch and stop decisions are taken on the device: no host synchronisation
 * inside.  The workspace must not be shared by concurrent calls. */
int dm_sp2(tb_ctx* ctx, const double* H, int n, double n_occ, const tb_sp2_opts* opts,
           double* D, void* workspace, size_t workspace_bytes, tb_sp2_report* report,
           void* stream);

/* Allocation-free FP64 SP2 (no counterpart in the paper: a convenience of
 * this library).  Same result as dm_sp2 with opts->precision = TB_PREC_FP64,
 * for callers that cannot allocate device memory when they need D (an MD
 * engine that reserves all memory up front and forbids allocation inside its
 * time step, a plugin whose host application owns the CUDA allocator, code
 * that must avoid the device-wide synchronisation of cudaMalloc/cudaFree).
 * The scratch is a static device array inside the library, sized for
 * n <= TB_SP2_STATIC_MAX_N (about 4 MiB per GPU, held until the process
 * exits); larger n fails with TB_ERR_ARG, other precisions with
 * TB_ERR_UNSUPPORTED.  The first call on a device, made with that device
 * current, looks up the array's device address: make it before any stream
 * capture.  That address stays valid while the device's context lives (a
 * cudaDeviceReset while the library is in use invalidates it, like every
 * other device pointer).  Every call reuses the same array (its state is
 * cleared at the start of each call), so calls that overlap on the GPU race:
 * serialise them on one stream.  H, D, report as for dm_sp2. */
#define TB_SP2_STATIC_MAX_N 512
int dm_sp2_static(tb_ctx* ctx, const double* H, int n, double n_occ, const tb_sp2_opts* opts,
                  double* D, tb_sp2_report* report, void* stream);

/* ----------------------------------------- grouped SP2 (many small systems) */

/* Workspace for a batch of `count` systems of sizes n[i] (host array,
 * 1 <= n[i] <= 512). */
int dm_sp2_grouped_workspace_size(int count, const int* n, const tb_sp2_opts* opts, size_t* bytes);

/* Plan a batch: SP2 (Sec. III.B, as dm_sp2's tensor-core main phase, no
 * refinement) of `count` independent systems in one persistent launch.
 *   n, n_occ   host arrays [count]
 *   H, D       host arrays [count] of device pointers to n[i] x n[i] FP64 matrices
 *   reports    device array [count] of tb_sp2_report, or NULL
 * Copies the per-system descriptors into the workspace.  autotune selects the
 * launch form: 2 = one CTA per system, 128-wide tiles, one CTA per SM, the hi/lo
 * operands stored by each projection's epilogue; 3 = the FP32-staged form
 * (tf32x3 only, else TB_ERR_UNSUPPORTED): the same but loading only the FP32 X
 * and splitting it into hi/lo in shared memory, bitwise the result of form 2;
 * 0 = form 3 for tf32x3, else form 2; 4 or 8 (5: 2) = thread-block clusters of
 * that many CTAs per system (the CTAs split each projection's tiles; as many
 * clusters as fit at once); 1 = time every form (tile width 64 or 128 with all or
 * half the SMs, clusters of 2, 4 or 8, the FP32-staged form) on the batch itself and
 * keep the fastest (the batch is solved several times).  config_out of the run
 * call reports the FP32-staged form as tile width 0.
 * Synchronises `stream`.  One plan per context at a time: a new plan replaces
 * the previous one. */
int dm_sp2_grouped_plan(tb_ctx* ctx, int count, const int* n, const double* n_occ, const double* const* H,
                        double* const* D, tb_sp2_report* reports, const tb_sp2_opts* opts, int autotune,
                        void* workspace, size_t workspace_bytes, void* stream);

/* Run the planned batch: one memset and one kernel launch on `stream`, no
 * host synchronisation, so it can be captured in a CUDA graph.  The H
 * matrices may change between runs (the pointers may not).
 * *config_out (host, may be NULL) = cluster size * 10^7 + tile width * 10^4 +
 * grid size (cluster size 1: one CTA per system). */
int dm_sp2_grouped_run(tb_ctx* ctx, void* workspace, int* config_out, void* stream);

/* ------------------------------------------- a10: finite temperature solve */

/* Options of dm_fermi. */
typedef struct {
  int precision;      /* tensor-core precision of the products: TB_PREC_TF32 .. TB_PREC_BF16X3 */
  int m;              /* most doubling steps (0: 14) after the third-order start E0 = L - 4/3 L^3,
                         L = -beta/2^(m+2) (H - mu I) (relative error 2 z^4/15, z = beta |eps - mu| /
                         2^(m+1)); the device uses the fewest m >= 8 (or this m if smaller) with
                         beta (eps_max - eps_min + 80 kT + 2 eV) <= 2^(m+1) (Gershgorin bounds; the
                         start is defined for |z| <= 1) and reports it; if even this m is too small
                         the report's status is TB_ERR_ARG and D holds no result */
  int ns_iters;       /* steps per inverse of A = I + 4E^2: the quadratic start (one product)
                         and ns_iters - 1 Newton-Schulz steps (0: 3, residual <= 99^-4) */
  int mu_iters;       /* cap on chemical-potential updates (one expansion each), 1..40 */
  double trace_tol;   /* stop when |Tr D - N_occ| <= trace_tol (0: 1e-6 + 1e-9 N_occ) */
} tb_fermi_opts;

/* Written on the device by dm_fermi. */
typedef struct {
  int status;         /* TB_OK, TB_ERR_NOT_CONVERGED (trace not reached), TB_ERR_TIMEOUT */
  int mu_iters;       /* expansions performed */
  int m;              /* doubling steps per expansion used on the device */
  int n;
  double mu;          /* chemical potential of the returned D */
  double trace;       /* Tr D */
  double trace_dd;    /* Tr D(I - D) (= dTr D/dmu / beta) */
  double eps_min, eps_max;
} tb_fermi_report;


int dm_fermi_workspace_size(int n, const tb_fermi_opts* opts, size_t* bytes);

/* D = (exp(beta (H - mu I)) + 1)^-1, beta = 1/kT, with mu such that
 * Tr D = n_occ (Eq. EL_4c, Eq. DM_perp; canonical), by the GEMM-only
 * recursive Fermi-operator expansion: from X0 = f at beta/2^m (E0 = X0 - I/2 =
 * -tanh(beta (H - mu I)/2^(m+1))/2 to third order), m steps
 * X <- X^2 [X^2 + (I - X)^2]^-1, each doubling beta, carried out on
 * E = X - I/2 as E <- 2E (I + 4E^2)^-1 (inverse by Newton-Schulz).  mu: safeguarded steps inside a
 * bisection bracket, all on the device: Newton's step -dev/(beta t) (t = Tr[D(I - D)], dev = Tr D - N_occ),
 * or, where |dev| ~ t (mu in a gap), the balance of the electrons (t + dev)/2 above and the holes
 * (t - dev)/2 below mu.  After each expansion the
 * products E^2 and E^3 give D(I - D) and D(I - D)(I - 2D); the expansion is accepted and shifted
 * by u = beta dmu to second order, D + u D(I - D) + u^2/2 D(I - D)(I - 2D), with u from the trace
 * condition, whenever the remainder bound |u|^3/6 Tr[D(I - D)] (Frobenius) is below 1e-7 sqrt(n);
 * otherwise the Newton step starts another expansion.
 *   H [n*n], D [n*n] (FP64); mu: device double, in = initial guess (NaN: the
 *   spectral midpoint), out = chemical potential of D; report: device or NULL. */
int dm_fermi(tb_ctx* ctx, const double* H, int n, double n_occ, double kT, const tb_fermi_opts* opts,
             double* D, double* mu, void* workspace, size_t workspace_bytes, tb_fermi_report* report,
             void* stream);

/* Workspace bytes of dm_fermi_entropy for an n x n H (19 FP64 matrices of the
 * padded size plus small buffers). */
int dm_fermi_entropy_workspace_size(int n, size_t* bytes);

/* Electronic entropy without diagonalisation (row f1): S/k_B =
 * -2 sum_i [f_i ln f_i + (1 - f_i) ln(1 - f_i)] (Eq. Entropy, used as the
 * approximation of Eq. Ent_Approx), f_i the occupations of the Fermi matrix
 * f(beta (H - mu I)) (Eq. EL_4c) at the given mu (the one dm_fermi returns).
 * FP64 recursive expansion, GEMMs and traces only: with Y = beta (H - mu I),
 * L(y) = ln(1 + e^y) = -ln(1 - f) obeys L(2y) = 2L(y) - ln 2 + ln(1 + 4e^2)
 * (e = f - 1/2) along the doubling chain and s = L(y) - (1 - f) y per state,
 * so S/k_B = 2 (n ln 2 + 2^m (dL0 + <E_m, Y0>) + sum_k 2^(m-1-k) Tr ln(I + 4E_k^2));
 * the start at |y0| <= 1/8 uses Taylor series, each Tr ln(I + 4E_k^2) a degree-20
 * Chebyshev series, each inverse three Newton-Schulz steps (17 FP64 products
 * per doubling; m from Gershgorin bounds, <= 16).
 *   H [n*n] (FP64), mu: device double (read), kT > 0 (eV);
 *   D [n*n] output or NULL: the FP64 Fermi matrix of the recursion at mu;
 *   S: device double output or NULL (not both NULL): S/k_B, NaN when the
 *   spectrum needs more than 16 doublings at this kT.
 * Asynchronous on `stream`; the workspace must not be shared by concurrent
 * calls. */
int dm_fermi_entropy(tb_ctx* ctx, const double* H, int n, const double* mu, double kT, double* D, double* S,
                     void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------- f3: non-orthogonal formulation (App. D.1) */

/* H[n] and the overlap S of the non-orthogonal formulation (Eq. DFTB_2 with the
 * charges n, as in Eq. EL_Orth_c):
 *   H_ab = h_ab + S_ab (v_a + v_b)/2,  v_a = sum_l gamma_{i(a) l} n_l (orbital a on atom i).
 *   n_aux [N] or NULL (then H = h), H [n*n], S [n*n], gamma [N*N] outputs (fully
 *   overwritten); v [N] output (the per-atom v, needed by tb_forces_nonorth), may be
 *   NULL only when n_aux is.  With overlap_s0 = 0 it writes S = I and the H of tb_build_H. */
int tb_build_HS(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                const double* n_aux, double* H, double* S, double* gamma, double* v, void* stream);

/* Report of dm_nonorth (device memory): the congruence factor's Newton-Schulz iterations
 * and the final max |(Z Y)_ij - I_ij| (Y -> S^{1/2}, Z -> S^{-1/2}). */
typedef struct {
  int status;           /* TB_OK, TB_ERR_NOT_CONVERGED (Z not converged in 24 iterations) */
  int ns_iters;
  double ns_residual;
} tb_nonorth_report;

/* Density matrix in the non-orthogonal basis (Eqs. DM_perp, Congr):
 *   Z = S^{-1/2} (Z^T S Z = I) by the coupled Newton-Schulz iteration (GEMM only, FP64,
 *   stopped on the device at max |Z Y - I| <= 1e-13, or below 1e-9 once it stops halving);
 *   H_perp = Z^T H Z;  rho_perp = theta(mu0 I - H_perp) by dm_sp2 with opts `so` (kT = 0), or
 *   the Fermi-Dirac matrix by dm_fermi with `fo` and the device mu[4] (kT > 0; mu as for
 *   dm_fermi: in the first element, warm start and result);
 *   rho = Z rho_perp Z^T;  W = Z (H_perp rho_perp + rho_perp H_perp) Z^T / 2, the
 *   energy-weighted density matrix of the Pulay force (rho H rho at kT = 0).
 * The congruence products run as FP64 GEMMs on the FP64 units (GB300: ~1.2 TFLOP/s, about
 * 25 n^3-products per call).
 *   H, S [n*n] inputs; rho, W [n*n] outputs; sp2_report / fermi_report as for dm_sp2 /
 *   dm_fermi (may be NULL); report may be NULL.  Workspace from dm_nonorth_workspace_size
 *   (1024-byte aligned). */
int dm_nonorth_workspace_size(int n, double kT, const tb_sp2_opts* so, const tb_fermi_opts* fo, size_t* bytes);
int dm_nonorth(tb_ctx* ctx, const double* H, const double* S, int n, double n_occ, double kT,
               const tb_sp2_opts* so, const tb_fermi_opts* fo, double* mu, double* rho, double* W,
               void* workspace, size_t workspace_bytes, tb_sp2_report* sp2_report,
               tb_fermi_report* fermi_report, tb_nonorth_report* report, void* stream);

/* Mulliken net charges with the overlap: q_i = 2 sum_{a in i} (rho S)_aa - N0_i (App. D.1;
 * the charge whose derivative dq/dR|_rho = 2 diag(rho S_R) Eq. EL_Nonorth_a uses).
 *   rho, S [n*n], q [N] output. */
int mulliken_nonorth(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* rho,
                     const double* S, double* q, void* stream);

/* F = -dE/dR at fixed n and E = 2 Tr[h rho] + 1/2 (2q - n)^T gamma n + E_pair in the
 * non-orthogonal formulation (Eq. EL_Nonorth_a with n for q):
 *   F = -d/dR { Tr[2 rho h] + Tr[(V rho + rho V - 2 W) S] }|_{rho, W} - (q - n/2)^T dgamma/dR n
 *       - dE_pair/dR,  V = diag(v):
 * the Pulay term Tr[(S^-1 H rho + rho H S^-1) S_R] = 2 Tr[W S_R] and the term of
 * dq/dR|_rho.  rho, W from dm_nonorth; q from mulliken_nonorth; v from tb_build_HS;
 * F [N*3], energy [4] outputs as for tb_forces. */
int tb_forces_nonorth(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                      const double* rho, const double* W, const double* q, const double* n_aux,
                      const double* v, const double* gamma, double* F, double* energy, void* stream);

/* ------------------------------- a5 boundary: block-sparse (BSR) matrices (Sec. III.B) */

/* A symmetric n x n matrix stored as 128 x 128 FP64 blocks in block-sparse-row form: the
 * layout of the thresholded SP2 (linear scaling for spatially ordered systems).  Block
 * (I, J) (block row I, block column J) sits in slot s with row_ptr[I] <= s < row_ptr[I + 1]
 * and col[s] = J, columns ascending within a row; its element (r, c) is
 * val[s * 16384 + r * 128 + c] = M[128 I + r][128 J + c], zero beyond n.  All arrays are
 * device memory owned by the caller; cap is the capacity in blocks (val holds
 * cap * 16384 doubles).  A call that would need more than cap blocks writes TB_ERR_OOM to
 * *status (device int) and leaves the matrix incomplete. */
#define TB_BSR_BLOCK 128
typedef struct {
  int n;          /* order */
  int nsb;        /* block rows = (n + 127) / 128 */
  int cap;        /* capacity in blocks */
  int* row_ptr;   /* [nsb + 1] */
  int* col;       /* [cap] */
  double* val;    /* [cap * 16384] */
  int* status;    /* device int: TB_OK or TB_ERR_OOM */
} tb_bsr;

/* Scratch of the block-sparse model calls: per block row, the atoms whose orbitals it holds
 * and their bounding box, and the block pattern. */
int tb_bsr_model_workspace_size(int natoms, int norb, size_t* bytes);

/* H[n] (a1) in BSR.  The pattern holds block (I, J) when the bounding boxes of the atoms of
 * block rows I and J (periodic minimum image) come within the model's range
 * (max(rcut, gamma_cut)), so every atom pair within range lies in a stored block; with the
 * atoms in spatial (e.g. Morton) order a block row has O(1) blocks and the build is
 * O(N).  The windowed gamma only (gamma_form 0), orthogonal model only.
 *   n_aux [N] or NULL; H: BSR output (structure and values); v [N] output, the per-atom SCC
 *   potential sum_l gamma_il n_l (zero without n_aux), which tb_forces_bsr needs.  The
 *   workspace (tb_bsr_model_workspace_size) keeps the block-row atom ranges and boxes for
 *   mulliken_bsr and tb_forces_bsr of the same positions. */
int tb_build_H_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                   const double* n_aux, tb_bsr* H, double* v, void* workspace, size_t workspace_bytes,
                   void* stream);

/* D = theta(mu0 I - H) by the thresholded block-sparse SP2 (a5; Sec. III.B, opts.tau > 0, a
 * tensor-core precision) with BSR input and output: X0 from H's blocks, the final iterate's
 * blocks (FP32 master, stored as FP64) written to D with their structure.  n <= 131072.
 * Workspace from dm_sp2_workspace_size(n, opts). */
int dm_sp2_sparse(tb_ctx* ctx, const tb_bsr* H, double n_occ, const tb_sp2_opts* opts, tb_bsr* D,
                  void* workspace, size_t workspace_bytes, tb_sp2_report* report, void* stream);

/* Workspace bytes of dm_fermi_sparse: seven block-sparse matrices (the iterate E twice, the
 * start L and the factors of each doubling step) of blocks_per_row x ceil(n/128) blocks of
 * 128 x 128 (FP32 master and operand splits; blocks_per_row <= 0: every block) and the
 * symbolic arrays.  TB_ERR_UNSUPPORTED for n > 131072. */
int dm_fermi_sparse_workspace_size(int n, const tb_fermi_opts* opts, int blocks_per_row, size_t* bytes);

/* Linear-scaling finite-temperature density matrix (row f2): the Fermi operator
 * D = (exp(beta (H - mu I)) + 1)^-1 with Tr D = n_occ (Eq. EL_4c, Eq. DM_perp; canonical) by
 * the recursive Fermi-operator expansion of dm_fermi (the construction the paper cites for
 * linear scaling at T_e > 0 and leaves unimplemented, end of Sec. III.C) on thresholded
 * block-sparse products: the start L = beta/2^(m+2) (mu I - H) and every product of the
 * expansion drop the 32 x 32 blocks with Frobenius norm < tau (the block reading of
 * Sec. III.B's threshold); the affine steps I -+ 2E and 2I - W are exact.  Per doubling step
 * W = (I - 2E)(I + 2E), A = 2I - W, Z = (32 A^2 - 144 A + 210 I)/99, ns_iters - 1
 * Newton-Schulz steps Z <- Z (2I - A Z), E <- E + E (Z W); m as in dm_fermi (the fewest
 * >= 8 with beta (eps_max - eps_min + 80 kT + 2 eV) <= 2^(m+1), at most opts.m).  D = I/2 + E.
 * The chemical potential is chosen on the host between expansions (dm_fermi's rule: Newton,
 * the gap-tail balance, bisection), from Tr D = n/2 + Tr E and Tr D(I - D) = n/4 - ||E||_F^2,
 * which it reads back after each expansion: the call synchronises `stream` once per
 * expansion and cannot be captured in a graph (TB_ERR_UNSUPPORTED).  No canonical shift:
 * expansions repeat until |Tr D - n_occ| <= opts.trace_tol (0: 1e-6 + 1e-9 n_occ) or
 * opts.mu_iters (1..100) have run (report status TB_ERR_NOT_CONVERGED, D of the last one).
 *   H: BSR (n <= 131072; H.status TB_OK, else TB_ERR_OOM in the report); tau > 0; kT > 0;
 *   blocks_per_row: capacity of every iterate as in tb_sp2_opts.bsr_blocks_per_row, exceeded:
 *   report status TB_ERR_OOM and an empty D; D: BSR output (blocks FP32-accurate, stored as
 *   FP64; D.status TB_ERR_OOM when more than D.cap blocks); mu: device double, in = initial
 *   guess (NaN or outside the Gershgorin bracket: the spectral midpoint), out = the chemical
 *   potential of D (written when the status is TB_OK); report: device or NULL. */
int dm_fermi_sparse(tb_ctx* ctx, const tb_bsr* H, double n_occ, double kT, const tb_fermi_opts* opts,
                    double tau, int blocks_per_row, tb_bsr* D, double* mu, void* workspace,
                    size_t workspace_bytes, tb_fermi_report* report, void* stream);

/* Mulliken charges (a7) from a BSR D: q_i = 2 sum_{a in i} D_aa - N0_i. */
int mulliken_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const tb_bsr* D, double* q,
                 void* stream);

/* Forces and energy (a8) as tb_forces, with D in BSR: the atom pairs within range are found
 * through H's block pattern and the workspace of the tb_build_H_bsr call at the same R;
 * gamma is evaluated on the fly (v from tb_build_H_bsr), so no N x N array is needed.
 *   F [N*3], energy [4] outputs. */
int tb_forces_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R, const tb_bsr* H,
                  const tb_bsr* D, const double* q, const double* n_aux, const double* v, double* F,
                  double* energy, const void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------- a7: charges */

/* Mulliken net charges q_i = 2 sum_{a in i} D_aa - N0_i (App. D).
 *   D [n*n], q [N] output. */
int mulliken(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* D,
             double* q, void* stream);

/* ------------------------------------------------------ a8: forces, energy */

/* F = -dE/dR at fixed n and E = 2 Tr[hD] + 1/2 (2q - n)^T gamma n + E_pair
 * (Eq. EL_Orth_a, Eq. Etot_Orth; the population multiplying d gamma / dR is taken net of
 * the neutral-atom reference, which makes the energy and force of Eq. EL_Orth_a
 * consistent; at n = q E is the SCC-TB energy 2 Tr[hD] + 1/2 q^T gamma q + E_pair).
 *   R [N*3], D [n*n], q [N], n_aux [N], gamma [N*N] (from tb_build_H)
 *   F [N*3] output (eV/A); energy [4] output: E_pot, 2Tr[hD], E_scc, E_pair. */
int tb_forces(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
              const double* D, const double* q, const double* n_aux, const double* gamma,
              double* F, double* energy, void* stream);

/* -------------------------------------------------------- a9: XL-BOMD step */

#define TB_XL_KMAX 8

/* Modified Verlet with dissipation for n (Eq. Verl_n):
 * n_{t+dt} = 2n_t - n_{t-dt} + kappa (q_t - n_t) + alpha sum_{k=0}^{K} c_k n_{t-k dt}. */
typedef struct {
  double dt;                 /* fs */
  double kappa;              /* dt^2 w^2 after the rescaling factor */
  double alpha;
  int K;                     /* 1..TB_XL_KMAX */
  double c[TB_XL_KMAX + 1];
} tb_xl_params;

/* Device-resident MD state.  All arrays are device memory owned by the caller. */
typedef struct {
  tb_system sys;
  double n_occ;
  double* R;            /* [N*3] */
  double* v;            /* [N*3] A/fs */
  double* F;            /* [N*3] force at R (valid after xlbomd_init) */
  const double* mass;   /* [N] amu */
  double* n_hist;       /* [(K+1)*N] shift register: slot j (N doubles) holds n_{t-j} */
  double* q;            /* [N] Mulliken charges of the last D */
  double* H;            /* [n*n] */
  double* D;            /* [n*n] */
  double* gamma;        /* [N*N] */
  double* energies;     /* [8]: E_tot, E_pot, 2Tr[hD], E_scc, E_pair, KE, max|n-q|, steps
                           (at kT > 0 E_tot includes -T_e S when the entropy fields below are
                           set, else it is KE + E_pot) */
  tb_sp2_report* sp2_report;  /* may be NULL */
  void* workspace;      /* dm_sp2 workspace (dm_sp2_workspace_size(norb)), or the dm_fermi
                           workspace when kT > 0 */
  size_t workspace_bytes;
  int64_t step;         /* host count of steps enqueued by xlbomd_step (energies[7] is the
                           device count, which also advances in graph replays) */
  double kT;            /* electronic temperature (eV); > 0: D by dm_fermi (Eq. EL_4c), else SP2 */
  tb_fermi_opts fermi;  /* options of dm_fermi when kT > 0 */
  double* mu;           /* device double[4] (kT > 0): [0] the chemical potential passed to and
                           returned by dm_fermi, [1..3] the values of the last three steps
                           (NaN until known); each step starts dm_fermi from the quadratic
                           extrapolation 3 mu[1] - 3 mu[2] + mu[3] (linear or constant while
                           fewer are known) */
  tb_fermi_report* fermi_report;  /* device, may be NULL */
  void* entropy_workspace;    /* kT > 0: dm_fermi_entropy workspace, or NULL (no entropy term) */
  size_t entropy_workspace_bytes;
  double* entropy;            /* device double: S/k_B of the last D (with entropy_workspace);
                                 energies[0] is then E_tot = KE + E_pot - kT S (Eq. Etot) */
  /* non-orthogonal formulation (p->overlap_s0 != 0): D holds rho, and these are required */
  double* S;                  /* [n*n] overlap */
  double* W;                  /* [n*n] energy-weighted density matrix */
  double* vscc;               /* [N] v = gamma n, the per-atom SCC potential */
  void* nonorth_workspace;    /* dm_nonorth workspace (dm_nonorth_workspace_size) */
  size_t nonorth_workspace_bytes;
  tb_nonorth_report* nonorth_report;  /* device, may be NULL */
  /* block-sparse boundary (orthogonal, sp2 opts with tau > 0): when H_bsr is set the step
   * builds H in BSR, runs dm_sp2_sparse (kT = 0) or dm_fermi_sparse (kT > 0, with the fermi
   * options, sp2 opts' tau and bsr_blocks_per_row; no entropy term; the workspace from
   * dm_fermi_sparse_workspace_size) into D_bsr, and takes q, F, E from it; H, D and gamma
   * may then be NULL (no n x n or N x N array) */
  tb_bsr* H_bsr;
  tb_bsr* D_bsr;
  void* bsr_workspace;        /* tb_bsr_model_workspace_size */
  size_t bsr_workspace_bytes;
} tb_md_state;

/* Initial state (App. D.3): SCF-converge the charges with Anderson mixing
 * (max|q - n| <= scf_tol or scf_max_iter iterations; host-side mixing of
 * N-vectors, synchronises the stream), set the whole n history to q and
 * compute F and the energies.  *scf_iters_out (host) gets the iteration
 * count or -1 when the cap was reached (the state is still usable). */
int xlbomd_init(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_xl_params* xp,
                const tb_sp2_opts* so, double scf_tol, int scf_max_iter, int* scf_iters_out,
                void* stream);

/* One Fast-QMMD step (Eqs. EL_3ax, EL_3bx; App. D.3): half kick, drift,
 * n update (Eq. Verl_n), H[n] (tb_build_H), D (dm_sp2, or dm_fermi when
 * st->kT > 0), q (mulliken), F and E (tb_forces), half kick, kinetic energy.
 * Fully asynchronous, and every launch has the same arguments from step to
 * step: a step captured into a CUDA graph (stream capture) replays as the
 * next step each time the graph is launched.  Under capture, dm_fermi's
 * chemical-potential loop becomes a conditional (while) graph node. */
int xlbomd_step(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_xl_params* xp,
                const tb_sp2_opts* so, void* stream);

/* ---------------------------------------------- serving: continuous batching */

/* A request loop over many XL-BOMD trajectories of uneven size on one GPU.
 * The paper has no serving counterpart; each step it runs is xlbomd_step.
 *
 * Each admitted trajectory keeps its whole state resident in one device
 * allocation: R, v, F, the n history, q, H, D, gamma, mu and the workspace
 * of its density solve.  Trajectories are admitted in the order they were
 * added, while the sum of the admitted footprints (tb_server_footprint)
 * stays within hbm_budget.  The others wait, and are admitted when a retired
 * trajectory frees its memory.  Admission runs the initial SCF (xlbomd_init,
 * synchronous) and captures one step into a CUDA graph.
 *
 * Step requests are served in submission order with at most one step in
 * flight per trajectory, on up to max_slots CUDA streams.  A request is
 * launched (one graph launch) as soon as its trajectory is idle and a slot
 * is free, while other steps are still running, so steps of different
 * trajectories overlap on the device.  The runtime is single-threaded: call
 * it from one host thread.  Host times are seconds since tb_server_create,
 * from a steady clock. */
#define TB_SERVER_MAX_SLOTS 64

typedef struct tb_server tb_server;

typedef struct {
  int max_slots;        /* steps in flight at once, one stream each: 1..TB_SERVER_MAX_SLOTS */
  size_t hbm_budget;    /* device bytes the admitted trajectories may hold together
                           (0: 90% of the free memory at create) */
  double kT;            /* electronic temperature (eV): > 0 D by dm_fermi, 0 by dm_sp2 */
  tb_xl_params xl;      /* integration parameters of every trajectory */
  tb_sp2_opts sp2;      /* density options at kT = 0 */
  tb_fermi_opts fermi;  /* density options at kT > 0 */
  double scf_tol;       /* initial SCF: max|q - n| */
  int scf_max_iter;     /* initial SCF cap (>= 1) */
} tb_server_opts;

/* One finished step request. */
typedef struct {
  int64_t request;      /* id returned by tb_server_submit (or the replay index order) */
  int traj;             /* trajectory id */
  int status;           /* status of the step's density solve (TB_OK, TB_ERR_NOT_CONVERGED, ...) */
  int solver_iters;     /* SP2 projections (kT = 0) or Fermi-operator expansions (kT > 0) */
  int solver_m;         /* kT > 0: doubling steps per expansion (tb_fermi_report.m); else 0 */
  int64_t step;         /* the trajectory's step count after this step */
  double t_submit;      /* host time of the request (replay: its scheduled arrival) */
  double t_launch;      /* host time of the graph launch */
  double t_done;        /* host time at which the completion was observed */
  double gpu_ms;        /* device time between the step's start and end events on its stream */
  double energies[8];   /* tb_md_state energies after the step */
} tb_completion;

typedef struct {
  int trajectories, admitted, waiting, running, queued;
  size_t bytes_in_use, budget;
  int64_t submitted, completed;
} tb_server_counts;

int tb_server_create(tb_ctx* ctx, const tb_params* p, const tb_server_opts* opts, tb_server** out);
/* Waits for the steps in flight, then frees every resource of the server. */
int tb_server_destroy(tb_server* server);

/* Device bytes a trajectory of natoms atoms (host types[natoms]) holds. */
int tb_server_footprint(const tb_server* server, int natoms, const int32_t* types, size_t* bytes);

/* Register a trajectory (host arrays, copied: types[N], R0[N*3] A, v0[N*3]
 * A/fs, mass[N] amu, cubic box side, n_occ = N_e/2) and admit it at once if
 * its footprint fits.  *traj_out = its id.  TB_ERR_OOM when the footprint
 * alone exceeds the budget. */
int tb_server_add(tb_server* server, int natoms, const int32_t* types, double box, const double* R0,
                  const double* v0, const double* mass, double n_occ, int* traj_out);

/* Queue one step of trajectory traj; *request_out (may be NULL) = its id. */
int tb_server_submit(tb_server* server, int traj, int64_t* request_out);

/* One scheduling pass: collect finished steps into out[0..max_out), free
 * retired trajectories, admit waiting ones, launch queued requests.  wait != 0:
 * repeat until at least one completion or nothing is in flight. */
int tb_server_poll(tb_server* server, int wait, tb_completion* out, int max_out, int* n_out);

/* Retire a trajectory: its queued steps still run; then its memory is freed
 * and waiting trajectories are admitted.  No new requests are accepted. */
int tb_server_retire(tb_server* server, int traj);

/* Copy a trajectory's state to host memory (any pointer may be NULL):
 * R[N*3], v[N*3], q[N], n_t[N], energies[8].  The trajectory must be
 * admitted and idle. */
int tb_server_read(tb_server* server, int traj, double* R, double* v, double* q, double* n_t, double* energies);

int tb_server_stats(const tb_server* server, tb_server_counts* out);

/* Replay an arrival trace in real time: request i (trajectory traj[i]) is
 * submitted when arrival_s[i] seconds (non-decreasing) have passed since the
 * call; polls until all have finished and writes out[i] for request i, with
 * t_submit = the scheduled arrival.  Needs a server with nothing in flight. */
int tb_server_replay(tb_server* server, int count, const double* arrival_s, const int* traj,
                     tb_completion* out);

#ifdef __cplusplus
}
#endif

#endif /* TBMD_H */
