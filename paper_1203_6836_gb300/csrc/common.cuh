// Internal declarations shared by the CUDA translation units of libtbmd.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/tbmd.h"

#define TB_PROF_MAX 130
struct tb_ctx {
  int device;
  int sm_count;
  int cc_major, cc_minor;
  PFN_cuTensorMapEncodeTiled_v12000 encode_tiled;
  char last_error[512];
  // launch timing of the last dm_sp2 call (events recorded between the
  // purification launches on the caller's stream when profiling is on)
  int prof_on;
  int prof_created;
  cudaEvent_t ev[2][TB_PROF_MAX + 1];
  int prof_n[2];
  // host copy of the last grouped-SP2 plan and the workspace it lives in
  alignas(64) char plan_cache[4096];
  void* plan_ws;
  // side stream on which the body of a conditional (while) graph node is
  // captured (created on first use)
  cudaStream_t loop_stream;
  // cap on the CTAs of the persistent tensor-core grids (0: one per SM)
  int grid_limit;
  // time limit (ns) of the pipeline waits of the tensor-core kernels
  unsigned long long wait_ns;
  // kernel form of the dense tensor-core projection (TB_SP2_FORM_*) and the
  // co-resident clusters of its CTA-pair form (-1: not queried yet)
  int sp2_form;
  int pair_clusters;
  int oz_pair_clusters;  // the same for the emulated-FP64 product's pair form
};

// CTAs of a persistent grid over `units` work units: one per SM, at most
// `units`, at most the context's grid limit.
static inline int tb_persistent_grid(const tb_ctx* ctx, int units) {
  int g = ctx->sm_count;
  if (ctx->grid_limit > 0 && ctx->grid_limit < g) g = ctx->grid_limit;
  if (units < g) g = units;
  return g < 1 ? 1 : g;
}

// Record the profiling event `idx` of phase `ph` on stream s (no-op when off).
static inline void tb_prof_mark(tb_ctx* ctx, int ph, int idx, cudaStream_t s) {
  if (ctx->prof_on && idx <= TB_PROF_MAX) {
    cudaEventRecord(ctx->ev[ph][idx], s);
    if (idx + 1 > ctx->prof_n[ph]) ctx->prof_n[ph] = idx + 1;
  }
}

// A loop whose trip count the device decides.  When the caller's stream is
// being captured into a CUDA graph, tb_loop_begin adds a conditional (while)
// node at the capture point and captures the body, launched once on
// `body_stream`, into it; the body's last kernel clears the condition with
// cudaGraphSetConditional(handle, 0).  Otherwise the host unrolls the body up
// to its cap on the caller's stream and the kernels of the rounds after the
// device's stop decision return at once.  The kernels and their order are the
// same in both forms.
struct DevLoop {
  int graph;                          // 1: body captured into a while node
  cudaStream_t outer;                 // the caller's stream
  cudaStream_t body_stream;           // where the body is launched
  cudaGraphConditionalHandle handle;  // valid when graph == 1
  cudaGraphNode_t node;
};
int tb_loop_begin(tb_ctx* ctx, cudaStream_t s, DevLoop* L);
// Close the body capture (also on an error path: pass the error code, which
// is returned unchanged).
int tb_loop_end(tb_ctx* ctx, DevLoop* L, int rc);

// Record a formatted message in the context and return `code`.
int tb_fail(tb_ctx* ctx, int code, const char* fmt, ...);

#define TB_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return tb_fail((ctx), TB_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,           \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

#define TB_LAUNCH_CHECK(ctx)                                                       \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess)                                                         \
      return tb_fail((ctx), TB_ERR_CUDA, "kernel launch failed: %s (%s:%d)",       \
                     cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

static inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Raise a kernel's dynamic shared-memory limit once per device (function
// attributes belong to the device's context); *done is the caller's static
// bit mask of devices already set.
template <typename K>
int tb_smem_attr(tb_ctx* ctx, K kernel, int bytes, unsigned long long* done) {
  const unsigned long long bit = 1ull << (ctx->device & 63);
  if (*done & bit) return TB_OK;
  TB_CUDA_TRY(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  *done |= bit;
  return TB_OK;
}

// ----------------------------------------------------------------- model

// Device copy of the model constants with the App. D tail coefficients
// precomputed on the host (closed form, see model.cu).
struct ModelDev {
  double eps_s_O, eps_p_O, eps_s_H;
  double t_hop, inv_decay;
  double U, kc, a2, gcut;
  double r1, rcut;
  double n0_O, n0_H;
  double pair_a, inv_prho;
  double Bhop[6], Bpair[6];
  double zhop[3], zpair[3];  // A2..A4 of zeta(R) for the bond integrals and phi
  double range;  // reach of the image loops: max(rcut, gcut), or rcut with the Ewald gamma
  double box;
  int gamma_form;     // 0: windowed gamma, 1: Ewald-summed Gaussian charges
  double ealpha;      // Ewald splitting (1/A)
  double gwidth;      // Gaussian width c = 2k/(U sqrt(pi))
  double erange;      // real-space reach: max(6.6/alpha, 6.6 c)
  double gmax;        // reciprocal cut-off 13.2 alpha
  double s0, inv_srs; // overlap radial s(r) = s0 exp(-r inv_srs) (s0 = 0: S = I)
  double Bov[6];      // its App. D tail
};

int tb_model_from_params(tb_ctx* ctx, const tb_params* p, double box, ModelDev* m);

// ------------------------------------------------------------------- SP2

// Device-side state of one dm_sp2 call (lives in the workspace).
#define SP2_MAX_ITER 120
#define SP2_MAX_REFINE 4
struct SP2State {
  int done;          // main phase finished (converged or capped)
  int iters;         // projections applied in the main phase
  int status;        // TB_OK / TB_ERR_*
  int rdone;         // refinement finished
  int riters;        // refinement projections applied
  int err;           // device-side error code (timeouts)
  int capped;        // main phase stopped at its iteration cap
  int rcapped;       // refinement stopped at its iteration cap
  double emin, emax;
  double t1[SP2_MAX_ITER + 2];   // Tr X_k
  double t2[SP2_MAX_ITER + 2];   // ||X_k||_F^2
  double rt1[SP2_MAX_REFINE + 2], rt2[SP2_MAX_REFINE + 2];
  double idem_fro;               // ||X^2 - X||_F of the last FP64 projection input
  unsigned long long branch[2];
  unsigned long long rbranch;
  unsigned long long block_products;  // block-sparse path: executed 128^3 block products
  int kc[2];                     // main-phase projection index inside a while graph node
};

// Parameters of a purification step shared by the FP64 and tensor-core kernels.
struct SP2StepArgs {
  int n;          // true size
  int ld;         // padded leading dimension (multiple of the tile)
  double nocc;
  double tol;
  double floor;   // tensor-core phase: noise floor of Tr X - Tr X^2 (2 n u)
  int rule;
  int k;          // projection index within its phase
  int max_iter;   // phase cap
  int phase;      // 0 = main, 1 = FP64 refinement
  int nparts_in;  // number of trace partials written by the previous kernel
  SP2State* st;
  const double* parts_in;   // [nparts_in * 2]
  double* parts_out;        // [ntiles * 2]
  unsigned long long wait_ns;  // pipeline wait limit (0: the 2 s default)
  // Device-counted index (kc != nullptr): the launch reads k = kc[kpar] and
  // writes kc[kpar ^ 1] = k + 1 for the next launch, so a captured run of
  // launches of alternating parity can be replayed as the body of a while
  // graph node; with cond the launch clears the node's condition once the
  // phase has stopped, failed or reached its cap.
  int* kc;
  int kpar;
  int cond;
  cudaGraphConditionalHandle loop;
};

// Projection index of a step launch (see SP2StepArgs::kc); `over` is the
// phase's done-or-error flag as read at kernel entry.
__device__ __forceinline__ int sp2_step_index(const SP2StepArgs& a, int over) {
  if (!a.kc) return a.k;
  const int k = a.kc[a.kpar];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    a.kc[a.kpar ^ 1] = k + 1;
    if (a.cond && (over || k >= a.max_iter)) cudaGraphSetConditional(a.loop, 0);
  }
  return k;
}

// Tensor-core purification step (gemm_tc.cu).  X_in / X_out are FP32 masters
// (ld x ld); hi/lo operand arrays of the input are read through the tensor
// maps; the epilogue writes the FP32 master and the hi/lo operands of the
// output.
int sp2_tc_step(tb_ctx* ctx, int precision, const SP2StepArgs& a,
                const CUtensorMap* map_hi, const CUtensorMap* map_lo,
                const float* X_in, float* X_out, void* out_hi, void* out_lo,
                cudaStream_t stream);
int sp2_tc_num_tiles(int ld);
// CTAs of the persistent single-CTA tensor-core grids (<= sp2_tc_num_tiles).
int sp2_tc_num_parts(const tb_ctx* ctx, int ld);
// Clusters of the CTA-pair projection kernel dm_sp2 runs at this ld (0: the
// single-CTA form), and the trace partials (CTAs) of one projection.
int sp2_tc_pairs(tb_ctx* ctx, int ld);
int sp2_tc_step_parts(tb_ctx* ctx, int ld);
int sp2_tc_tile();
size_t sp2_tc_operand_bytes(int precision);  // bytes per element of one operand array

// Emulated-FP64 projection on the tensor cores (gemm_oz.cu): splits X_in
// (FP64, ld x ld) into bf16 slices, then X_out = X_in^2 or 2 X_in - X_in^2.
int sp2_oz_step(tb_ctx* ctx, const SP2StepArgs& a, const double* Xin, double* Xout, void* slices, int* exps,
                cudaStream_t s);
int sp2_oz_max_ld();
// Partials (CTAs) of one emulated-FP64 projection: one per upper-triangle
// tile, or the persistent grid of the CTA-pair form.
int sp2_oz_num_parts(tb_ctx* ctx, int ld);
size_t sp2_oz_slice_bytes(int ld);

// Generic tensor-core product out = alpha A B + beta E + gamma I of symmetric,
// commuting matrices (gemm_tc.cu); all matrices ld x ld, FP32 masters with
// operand splits; parts (2 doubles per CTA: Tr out, ||out||^2) optional.
struct GemmArgs {
  int n, ld;
  float alpha, beta, gamma;
  const float* E;
  float* out;
  void* ohi;
  void* olo;
  double* parts;
  const int* skip;
  int* err;
  unsigned long long wait_ns;  // pipeline wait limit (0: the 2 s default)
  int lolo;                    // split precisions: also the lo*lo MMA (squares A A)
};
int tc_gemm(tb_ctx* ctx, int precision, const GemmArgs& g, const CUtensorMap* ah, const CUtensorMap* al,
            const CUtensorMap* bh, const CUtensorMap* bl, cudaStream_t s);
int tc_split(tb_ctx* ctx, int precision, const float* X, size_t count, void* hi, void* lo, const int* skip,
             cudaStream_t s);

// Gershgorin partial bounds of the rows of H (sp2.cu).
int sp2_launch_bounds(tb_ctx* ctx, const double* H, int n, double* bparts, cudaStream_t s);

// Thresholded block-sparse SP2 (bsr.cu).
int dm_sp2_bsr_workspace(int n, const tb_sp2_opts* o, int nsm, size_t* bytes);
int dm_sp2_bsr(tb_ctx* ctx, const double* H, int n, double nocc, const tb_sp2_opts* o, double* D, void* ws,
               size_t ws_bytes, tb_sp2_report* rep, cudaStream_t s);

// Encode a 2D row-major tensor map over an ld x ld operand array (gemm_tc.cu):
// boxes of box_rows (64 or 128) rows of row_bytes (64 or 128) bytes, swizzled
// to the row width.  The projection and Fermi-product kernels read 128-row
// boxes of sp2_tc_row_bytes(); the emulated-FP64 product reads 128-byte rows,
// in 64-row boxes for the B operand of its CTA-pair form.
int sp2_tc_make_map(tb_ctx* ctx, int precision, const void* base, int ld, CUtensorMap* map, int row_bytes = 128,
                    int box_rows = 128);
int sp2_tc_row_bytes();

// ------------------------------------------------------------ utilities

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Deterministic sum of `np` partial pairs by one warp (fixed order): lane l
// adds partials l, l+32, ..., then a fixed butterfly.  Same result in every CTA.
__device__ __forceinline__ void warp_reduce_partials(const double* parts, int np, double* s0,
                                                     double* s1) {
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
  for (int i = lane; i < np; i += 32) {
    a += parts[2 * i];
    b += parts[2 * i + 1];
  }
  *s0 = warp_sum(a);
  *s1 = warp_sum(b);
}

// Decision of SP2 projection k from the traces of X_k (t1 = Tr X, t2 = Tr X^2).
// Returns 1 when the phase stops before projection k (setting *capped when
// the iteration cap was the reason), else 0 and sets *branch.
// FP64 phases stop when |Tr X - Tr X^2| <= tol.  The tensor-core phase,
// whose products carry a relative error u, stops once Tr X - Tr X^2 reaches
// its noise floor (a.floor = 2 n u, which negative values are also below)
// or has stayed within 4x of it for four projections; the FP64 refinement
// takes it from there.  A rise of Tr X - Tr X^2 alone is no stop signal:
// on small-gap spectra the HOMO or LUMO eigenvalue of X climbs from near 0
// across the middle over several projections, doubling it each time.
__device__ __forceinline__ int sp2_decide(const SP2StepArgs& a, double t1, double t2,
                                          const double* hist_t1, const double* hist_t2,
                                          bool tc_phase, int* branch, int* capped) {
  const double e = t1 - t2;
  *capped = 0;
  if (tc_phase) {
    if (e <= a.floor) return 1;
    if (a.k >= 3) {
      bool flat = e <= 4.0 * a.floor;
      for (int j = 1; j <= 3; ++j) flat = flat && (hist_t1[a.k - j] - hist_t2[a.k - j] <= 4.0 * a.floor);
      if (flat) return 1;
    }
  } else if (fabs(e) <= a.tol) {
    return 1;
  }
  if (a.k >= a.max_iter) {
    *capped = 1;
    return 1;
  }
  if (a.rule == 0)
    *branch = (fabs(t2 - a.nocc) <= fabs(2.0 * t1 - t2 - a.nocc)) ? 0 : 1;
  else
    *branch = (t1 > a.nocc) ? 0 : 1;
  return 0;
}

// Next chemical potential of the Fermi expansion after an expansion at mu
// (dev = Tr D - N_occ, t1 = Tr D(I - D), beta = 1/kT), inside the bisection
// bracket (lo, hi) already narrowed by this expansion's sign.  Newton's step
// -dev/(beta t1), except where |dev| ~ t1: then the partly occupied states
// sit in the tails of a gap (f(1-f) ~ f or 1-f), Newton moves mu by only ~kT
// per expansion, and the electrons above mu, a = (t1 + dev)/2, and the holes
// below it, b = (t1 - dev)/2, which move as a e^{beta dmu} and b e^{-beta dmu},
// balance at dmu = ln(b/a)/(2 beta).  With one tail below resolution the step
// shrinks the other towards the tolerance, by at most 8 kT.  A step that
// leaves the bracket bisects it.
__host__ __device__ inline double foe_next_mu(double mu, double dev, double t1, double beta, double tol, double lo,
                                              double hi) {
  double next = t1 > 1e-12 ? mu - dev / (beta * t1) : NAN;
  const double r = t1 > 0.0 ? fabs(dev) / t1 : INFINITY;
  if (r >= 0.5 && r <= 1.5) {
    const double a = 0.5 * (t1 + dev), b = 0.5 * (t1 - dev);
    if (a > 0.0 && b > 0.0 && fmin(a, b) > 1e-3 * fmax(a, b))
      next = mu + 0.5 * log(b / a) / beta;
    else
      next = mu - copysign(fmin(log(fabs(dev) / tol), 8.0), dev) / beta;
  }
  if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
  return next;
}
