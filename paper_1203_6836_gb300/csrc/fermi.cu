// Finite-temperature density matrix (row a10): the Fermi operator
// D = (exp(beta (H - mu I)) + 1)^-1 with Tr D = N_occ (Eq. EL_4c,
// Eq. DM_perp; canonical reading), by a GEMM-only recursive expansion.
//
// With y = 1/(1 + e^t), y^2 / (y^2 + (1 - y)^2) = 1/(1 + e^{2t}): one step of
// X <- X^2 [X^2 + (I - X)^2]^-1 doubles the inverse temperature.  Starting
// from X0 = f at beta/2^m, m steps give f at beta.  The steps are carried out
// on the deviation E = X - I/2, for which the same map reads
//   E <- 2 E (I + 4 E^2)^-1                        (tanh double-angle form)
// and f at beta/2^m is E0 = -tanh(Z)/2, Z = beta (H - mu I) / 2^{m+1}.  The
// start takes tanh to third order: with L = -Z/2,
//   E0 = L - 4/3 L^3                               (two products, L^2 and L L^2)
// whose relative error 2 z^4/15 the doubling steps do not amplify (tanh(2y)
// has a relative sensitivity (1 - t^2)/(1 + t^2) <= 1 to tanh(y) = t).  In
// FP64 on a 20 eV wide spectrum at kT = 0.1 eV it reaches the Fermi function
// to 2e-14 with m = 10 and 4e-12 with m = 8 (the linearised start E0 = L:
// 1e-8 and 2e-7), far below the products' FP32-level error, so m is set by
// the range of the start: both forms need |z| <= 1 (z - z^3/3 is monotone
// there), beta max|eps - mu| <= 2^{m+1}.  The bounds kernel takes, for the
// whole chemical-potential bracket [lo, hi], the smallest m >= kMinM with
// beta (hi - lo) <= 2^{m+1}; the host issues m_max doubling steps and the
// first m_max - m return at once (device flags), so one captured graph serves
// every spectrum width up to beta (hi - lo) = 2^{m_max + 1}.
// E is small while the early steps double it, so FP32-level products keep a
// relative accuracy there (errors add up over the m steps instead of being
// doubled m times as absolute errors of X would be).  Per step:
//   W = (I - 2E)(I + 2E) = I - 4E^2                (one product; spectrum in [0, 1])
//   A = 2I - W = I + 4E^2                          (elementwise; spectrum in [1, 2])
//   Z = A^-1: Z1 = (210 I - 144 A + 32 A^2) / 99    (one product A A with the
//             affine part in its epilogue), then Newton-Schulz Z <- Z (2I - A Z)
//   E <- E + E (Z W)                               (two products; = 2 E Z)
// The factored W and the update form keep the saturated states exact: where
// E is near +-1/2 one factor of W is near 0, so W and Z W are small there and
// carry small absolute errors, and E changes only by that small amount.  The
// plain forms A = I + 4E^2, E <- 2EZ left every saturated occupied state of
// a 2400-orbital gapped system 1.8e-7 above 1 on the GB300 tensor cores (the
// error of the last products, which the saturated states do not forget), 3e-4
// electrons in all, enough to drag mu across a 3 eV gap.
// Z1 is the quadratic p minimising max |1 - x p(x)| on [1, 2]: 1 - x p(x) is
// the Chebyshev polynomial T3(2x - 3) / T3(-3), so ||I - A Z1|| <= 1/99 and two
// Newton-Schulz steps leave ||I - A Z|| <= 99^-4 ~ 1e-8 (seven products per
// doubling step, where Z0 = 2/3 I needs four Newton-Schulz steps for 2e-8).
// All factors are functions of H, hence symmetric and commuting, so every
// product is a tensor-core GEMM with the second operand read by rows, and
// its result is symmetric: the product kernel computes the upper-triangle
// tiles and mirrors them, so every iterate is exactly symmetric (rounding
// errors would otherwise leave an antisymmetric part that the doubling
// steps amplify).
// D = I/2 + E on the n x n block.
// The chemical potential: safeguarded Newton steps on Tr D(mu) = N_occ with
// dTr D/dmu = beta Tr[D(I - D)] inside a bisection bracket, one full
// expansion per step; every decision is taken on the device.

#include "common.cuh"

#include <algorithm>
#include <math.h>

namespace {

constexpr int kTile = 128;
constexpr int kMaxMu = 40;
constexpr int kMaxM = 40;   // doubling steps issued at most
constexpr int kMinM = 8;    // doubling steps used at least
constexpr int kMats = 7;    // E0/E1 (the iterate, alternating), A, Z, T, Y, W
// Canonical shift: the last expansion is accepted and shifted by u = beta dmu
// to second order,
//   D(mu + dmu) = D + u D(I - D) + u^2/2 D(I - D)(I - 2D) + R,
// with D(I - D) = W/4 and D(I - D)(I - 2D) = -E W/2, W = (I - 2E)(I + 2E) (two
// products, W and E W, after every expansion), u the root of the trace condition
// Tr D + u Tr[D(I-D)] + u^2/2 Tr[D(I-D)(I-2D)] = N_occ near -(Tr D - N)/Tr[D(I-D)].
// The remainder involves the third derivative beta^3 f(1-f)(1-6f+6f^2), whose
// last factor is at most 1 in magnitude, so ||R||_F <= |u|^3/6 Tr[D(I - D)]
// (D(I - D) is positive semi-definite with eigenvalues <= 1/4).  The shift
// replaces another expansion when that bound is below kCorrFro sqrt(n) and
// |u| <= kCorrMax.
constexpr double kCorrFro = 1e-7;
constexpr double kCorrMax = 0.1;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct FoeState {
  double mu, lo, hi;
  double emin, emax;
  int done, iters, capped, err;
  int ran;     // 1: the last k_foe_mu evaluated an expansion (it was not skipped)
  int nocorr;  // 0: apply the canonical shift u to the last expansion
  double dmu;  // u / beta
  double u;
  double c;    // start scale beta / 2^{meff+2}
  int meff;    // doubling steps used
  int skipd[kMaxM];  // 1: doubling step k returns at once (k < m_max - meff, or done)
  double tr[kMaxMu + 1], trdd[kMaxMu + 1], mus[kMaxMu + 1];
};

struct Mat {
  float* m;
  void* hi;
  void* lo;
  CUtensorMap mh, ml;
};

// Gershgorin bounds, the bisection bracket, the first mu and the number of
// doubling steps: the start needs beta |eps - mu| <= 2^{m+1} for every
// eigenvalue and every mu of the bracket, so m is the smallest value >= kMinM
// with beta (hi - lo) <= 2^{m+1}; when even m_max does not reach, the expansion
// is not defined: TB_ERR_ARG, nothing runs.
__global__ void k_foe_bounds(const double* bparts, int nb, FoeState* st, const double* mu_in, double kT,
                             int m_max) {
  double a = INFINITY, b = -INFINITY;
  for (int i = threadIdx.x; i < nb; i += 32) {
    a = fmin(a, bparts[2 * i]);
    b = fmax(b, bparts[2 * i + 1]);
  }
  a = warp_min(a);
  b = warp_max(b);
  if (threadIdx.x == 0) {
    st->emin = a;
    st->emax = b;
    st->lo = a - 40.0 * kT - 1.0;
    st->hi = b + 40.0 * kT + 1.0;
    const double g = mu_in ? *mu_in : NAN;
    st->mu = (isfinite(g) && g > st->lo && g < st->hi) ? g : 0.5 * (a + b);
    st->nocorr = 1;
    const double z = (st->hi - st->lo) / kT;
    int m = kMinM < m_max ? kMinM : m_max;
    while (m < m_max && !(z <= ldexp(1.0, m + 1))) ++m;
    st->meff = m;
    st->c = 1.0 / (kT * ldexp(1.0, m + 2));
    const bool bad = !(z <= ldexp(1.0, m + 1));
    if (bad) {
      st->err = TB_ERR_ARG;
      st->done = 1;
    }
    for (int k = 0; k < kMaxM; ++k) st->skipd[k] = bad || k < m_max - m;
  }
}

// L = -c (H - mu I), c = beta / 2^{m+2} (m: the doubling steps used), on the
// n x n block, zero in the padding.
__global__ void __launch_bounds__(256) k_foe_x0(const double* __restrict__ H, int n, int ld, const FoeState* st,
                                                float* __restrict__ X) {
  if (st->done || st->err) return;
  const double mu = st->mu, c = st->c;
  const size_t total = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), col = (int)(e % ld);
    double x = 0.0;
    if (r < n && col < n) x = (r == col ? c * mu : 0.0) - c * H[(size_t)r * n + col];
    X[e] = (float)x;
  }
}

// After an expansion: Tr E and ||E||_F^2 from the last product's partials
// give Tr D = n/2 + Tr E and Tr D(I - D) = n/4 - ||E||_F^2; then the stop
// test and the next mu (one block, every quantity FP64).  The expansion index
// is the device count st->iters.  Inside a while graph node (cond != 0) the
// condition is cleared on every stop: converged, capped, or an error flag
// raised by a product of this expansion.
__global__ void k_foe_mu(FoeState* st, const double* parts, const double* partsw, const double* parts3, int np,
                         int n, double nocc, double beta, double tol, int max_it, cudaGraphConditionalHandle handle,
                         int cond) {
  if (st->done || st->err || st->iters >= max_it) {
    if (threadIdx.x == 0) {
      st->ran = 0;
      if (cond) cudaGraphSetConditional(handle, 0);
    }
    return;
  }
  double x = 0.0, y = 0.0, z = 0.0;
  for (int i = threadIdx.x; i < np; i += 32) {
    x += parts[2 * i];
    y += partsw[2 * i];
    z += parts3[2 * i];
  }
  x = warp_sum(x);  // Tr E
  y = warp_sum(y);  // Tr W
  z = warp_sum(z);  // Tr E W
  if (threadIdx.x != 0) return;
  const int it = st->iters;
  const double mu = st->mu;
  const double trd = 0.5 * n + x;
  const double t1 = 0.25 * y;    // Tr D(I - D)
  const double t2 = -0.5 * z;    // Tr D(I - D)(I - 2D)
  st->tr[it] = trd;
  st->trdd[it] = t1;
  st->mus[it] = mu;
  st->iters = it + 1;
  st->ran = 1;
  const double dev = trd - nocc;
  const double step = t1 > 1e-12 ? -dev / (beta * t1) : NAN;  // Newton step on mu
  double u = beta * step;
  for (int k = 0; k < 3 && isfinite(u); ++k) {  // root of dev + t1 u + t2 u^2/2 near the Newton step
    const double g = dev + u * (t1 + 0.5 * t2 * u), gp = t1 + t2 * u;
    if (!(gp > 0.0)) break;
    u -= g / gp;
  }
  const bool shift = isfinite(u) && fabs(u) <= kCorrMax &&
                     fabs(u) * u * u / 6.0 * t1 <= kCorrFro * sqrt((double)max(n, 1));
  if (shift) {
    // accept this expansion with the second-order shift to mu + u / beta
    st->done = 1;
    st->nocorr = 0;
    st->u = u;
    st->dmu = u / beta;
    st->tr[it] = trd + u * (t1 + 0.5 * t2 * u);
    st->mus[it] = mu + u / beta;
  } else if (fabs(dev) <= tol) {
    st->done = 1;
  } else if (it + 1 >= max_it) {
    st->done = 1;
    st->capped = 1;
  } else {
    if (dev < 0.0) st->lo = mu;
    else st->hi = mu;
    st->mu = foe_next_mu(mu, dev, t1, beta, tol, st->lo, st->hi);
  }
  if (st->done)
    for (int k = 0; k < kMaxM; ++k) st->skipd[k] = 1;
  if (cond && st->done) cudaGraphSetConditional(handle, 0);
}

// P = I + 2E and M = I - 2E on the n x n block (FP32 masters; zero in the
// padding, so W = M P is zero there too), skipped with the doubling step.
__global__ void __launch_bounds__(256) k_foe_pm(const int* skip, int n, int ld, const float* __restrict__ E,
                                                float* __restrict__ P, float* __restrict__ M) {
  if (*skip) return;
  const size_t total = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / ld, c = e % ld;
    const float id = (r == c && r < (size_t)n) ? 1.0f : 0.0f;
    const float x = 2.0f * E[e];
    P[e] = id + x;
    M[e] = id - x;
  }
}

// A = 2I - W (FP32 master), skipped with the doubling step.
__global__ void __launch_bounds__(256) k_foe_a(const int* skip, int ld, const float* __restrict__ W,
                                               float* __restrict__ A) {
  if (*skip) return;
  const size_t total = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    A[e] = ((e / ld) == (e % ld) ? 2.0f : 0.0f) - W[e];
}

// Word copy of one iterate array into the other iterate buffer (skipped once
// the expansion loop is done).
__global__ void __launch_bounds__(256) k_foe_copy(const FoeState* st, const uint32_t* __restrict__ src,
                                                  uint32_t* __restrict__ dst, size_t words) {
  if (st->done || st->err) return;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// Copy the last X of an expansion into the result buffer, only when that
// expansion ran (a converged outer loop skips the later ones).
__global__ void __launch_bounds__(256) k_foe_keep(const FoeState* st, size_t count, const float* __restrict__ src,
                                                  float* __restrict__ dst) {
  if (!st->ran || src == dst) return;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// E <- E + u W/4 - u^2/4 E W on the n x n block (D(I - D) = W/4,
// D(I - D)(I - 2D) = -E W/2), with T = W and U = E W from the product kernel;
// skipped unless the shift applies.
__global__ void __launch_bounds__(256) k_foe_correct(const FoeState* st, int n, int ld, const float* __restrict__ T,
                                                     const float* __restrict__ U, float* __restrict__ E) {
  if (st->nocorr) return;
  const float u = (float)st->u, h = 0.5f * u * u;
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), col = (int)(e % n);
    const size_t i = (size_t)r * ld + col;
    const float x = E[i];
    const float first = 0.25f * T[i];
    const float second = -0.5f * U[i];
    E[i] = fmaf(h, second, fmaf(u, first, x));
  }
}

__global__ void __launch_bounds__(256) k_foe_finalize(const FoeState* st, int n, int ld, const float* __restrict__ X,
                                                      double* __restrict__ D, double nocc, double tol,
                                                      double* mu_out, tb_fermi_report* rep) {
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    D[e] = (double)X[(size_t)r * ld + c] + (r == c ? 0.5 : 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int it = st->iters > 0 ? st->iters - 1 : 0;
    const double mu = st->mus[it];
    if (mu_out) *mu_out = mu;
    if (rep) {
      rep->status = st->err ? st->err : (fabs(st->tr[it] - nocc) <= tol ? TB_OK : TB_ERR_NOT_CONVERGED);
      rep->mu_iters = st->iters;
      rep->m = st->meff;
      rep->n = n;
      rep->mu = mu;
      rep->trace = st->tr[it];
      rep->trace_dd = st->trdd[it];
      rep->eps_min = st->emin;
      rep->eps_max = st->emax;
    }
  }
}

struct FoeLayout {
  int ld;
  size_t off_state, off_bparts, off_parts, off_parts3, off_partsw, off_mat[kMats][3], off_res, total;
  int nparts;
};

FoeLayout foe_layout(int n, int prec) {
  FoeLayout L{};
  L.ld = round_up(std::max(n, 1), kTile);
  L.nparts = (L.ld / kTile) * (L.ld / kTile);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 1023) / 1024 * 1024;
    return r;
  };
  const size_t nn = (size_t)L.ld * L.ld;
  const size_t eb = (prec == TB_PREC_TF32 || prec == TB_PREC_TF32X3) ? 4 : 2;
  const bool split = prec == TB_PREC_TF32X3 || prec == TB_PREC_BF16X3;
  L.off_state = take(sizeof(FoeState));
  L.off_bparts = take(sizeof(double) * 2 * ((n + 7) / 8));
  L.off_parts = take(sizeof(double) * 2 * (size_t)L.nparts);
  L.off_parts3 = take(sizeof(double) * 2 * (size_t)L.nparts);
  L.off_partsw = take(sizeof(double) * 2 * (size_t)L.nparts);
  for (int i = 0; i < kMats; ++i) {
    L.off_mat[i][0] = take(sizeof(float) * nn);
    L.off_mat[i][1] = take(eb * nn);
    L.off_mat[i][2] = split ? take(eb * nn) : 0;
  }
  L.off_res = take(sizeof(float) * nn);
  L.total = o;
  return L;
}

int valid_opts(const tb_fermi_opts* o) {
  return o && o->precision >= TB_PREC_TF32 && o->precision <= TB_PREC_BF16X3 && o->m >= 0 && o->m <= 40 &&
         o->ns_iters >= 0 && o->ns_iters <= 12 && o->mu_iters >= 1 && o->mu_iters <= kMaxMu;
}

}  // namespace

extern "C" int dm_fermi_workspace_size(int n, const tb_fermi_opts* o, size_t* bytes) {
  if (!bytes || n < 1 || !valid_opts(o)) return TB_ERR_ARG;
  *bytes = foe_layout(n, o->precision).total;
  return TB_OK;
}

extern "C" int dm_fermi(tb_ctx* ctx, const double* H, int n, double nocc, double kT, const tb_fermi_opts* o,
                        double* D, double* mu, void* ws, size_t ws_bytes, tb_fermi_report* rep, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !D || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_fermi");
  if (n < 1 || !(kT > 0.0) || !(nocc >= 0.0) || nocc > n) return tb_fail(ctx, TB_ERR_ARG, "bad n, kT or n_occ");
  if (!valid_opts(o)) return tb_fail(ctx, TB_ERR_ARG, "invalid tb_fermi_opts");
  const FoeLayout L = foe_layout(n, o->precision);
  if (ws_bytes < L.total) return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu", ws_bytes, L.total);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  char* base = static_cast<char*>(ws);
  FoeState* st = reinterpret_cast<FoeState*>(base + L.off_state);
  double* bparts = reinterpret_cast<double*>(base + L.off_bparts);
  double* parts = reinterpret_cast<double*>(base + L.off_parts);
  double* parts3 = reinterpret_cast<double*>(base + L.off_parts3);
  double* partsw = reinterpret_cast<double*>(base + L.off_partsw);
  Mat M[kMats];  // E (two, alternating), A, Z, T, Y, W
  for (int i = 0; i < kMats; ++i) {
    M[i].m = reinterpret_cast<float*>(base + L.off_mat[i][0]);
    M[i].hi = base + L.off_mat[i][1];
    M[i].lo = L.off_mat[i][2] ? base + L.off_mat[i][2] : nullptr;
    int rc = sp2_tc_make_map(ctx, o->precision, M[i].hi, L.ld, &M[i].mh, sp2_tc_row_bytes());
    if (rc) return rc;
    if (M[i].lo) {
      rc = sp2_tc_make_map(ctx, o->precision, M[i].lo, L.ld, &M[i].ml, sp2_tc_row_bytes());
      if (rc) return rc;
    } else {
      M[i].ml = M[i].mh;
    }
  }
  const double beta = 1.0 / kT;
  // at most m doubling steps (m = 14: beta (hi - lo) <= 32768); the device uses
  // the fewest that the bracket allows, at least kMinM
  const int m = o->m > 0 ? o->m : 14;
  const int ns = o->ns_iters > 0 ? o->ns_iters : 3;
  // default: 1e-6 electrons plus 1e-9 per electron pair, above the FP32 noise
  // of the trace (~3e-8 sqrt(n)) and tight enough for 1e-6 e charges
  const double tol = o->trace_tol > 0.0 ? o->trace_tol : 1e-6 + 1e-9 * nocc;
  const size_t nn = (size_t)L.ld * L.ld;
  const size_t eb = (o->precision == TB_PREC_TF32 || o->precision == TB_PREC_TF32X3) ? 4 : 2;
  int* skip = &st->done;
  int* errp = &st->err;
  float* res = reinterpret_cast<float*>(base + L.off_res);

  TB_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(FoeState), s));
  int rc = sp2_launch_bounds(ctx, H, n, bparts, s);
  if (rc) return rc;
  k_foe_bounds<<<1, 32, 0, s>>>(bparts, (n + 7) / 8, st, mu, kT, m);
  TB_LAUNCH_CHECK(ctx);

  // the chemical-potential loop: a while graph node under capture, else
  // mu_iters unrolled rounds that return at once after the stop decision
  DevLoop loop;
  if ((rc = tb_loop_begin(ctx, s, &loop))) return rc;
  cudaStream_t ls = loop.body_stream;
  const int rounds = loop.graph ? 1 : o->mu_iters;
  auto gemm = [&](Mat& A, Mat& B, Mat& out, float alpha, float betac, const float* E, float gamma,
                  double* prt, int* skp = nullptr) -> int {
    GemmArgs g{};
    g.n = n;
    g.ld = L.ld;
    g.alpha = alpha;
    g.beta = betac;
    g.gamma = gamma;
    g.E = E;
    g.out = out.m;
    g.ohi = out.hi;
    g.olo = out.lo;
    g.parts = prt;
    g.skip = skp ? skp : skip;
    g.err = errp;
    g.wait_ns = ctx->wait_ns;
    g.lolo = &A == &B;
    return tc_gemm(ctx, o->precision, g, &A.mh, &A.ml, &B.mh, &B.ml, ls);
  };
  Mat* xf = &M[0];  // final iterate, E^2 and E^3 after an expansion
  Mat* af = &M[1];
  Mat* zf = &M[2];
  auto expansion = [&]() -> int {
    int r;
    Mat* E[2] = {&M[0], &M[5]};
    Mat* A = &M[1];
    Mat* Z = &M[2];
    Mat* T = &M[3];
    Mat* Y = &M[4];
    k_foe_x0<<<1184, 256, 0, ls>>>(H, n, L.ld, st, Y->m);
    TB_LAUNCH_CHECK(ctx);
    if ((r = tc_split(ctx, o->precision, Y->m, nn, Y->hi, Y->lo, skip, ls))) return r;
    // E0 = L - 4/3 L L^2 in both iterate buffers: the first doubling step the
    // device runs may be any of the m issued ones
    if ((r = gemm(*Y, *Y, *A, 1.0f, 0.0f, nullptr, 0.0f, nullptr))) return r;
    if ((r = gemm(*Y, *A, *E[0], -4.0f / 3.0f, 1.0f, Y->m, 0.0f, nullptr))) return r;
    {
      const void* src[3] = {E[0]->m, E[0]->hi, E[0]->lo};
      void* dst[3] = {E[1]->m, E[1]->hi, E[1]->lo};
      const size_t words[3] = {nn, eb * nn / 4, eb * nn / 4};
      for (int i = 0; i < 3; ++i) {
        if (!src[i]) continue;
        k_foe_copy<<<1184, 256, 0, ls>>>(st, static_cast<const uint32_t*>(src[i]), static_cast<uint32_t*>(dst[i]),
                                         words[i]);
        TB_LAUNCH_CHECK(ctx);
      }
    }
    Mat* W = &M[6];
    // P = I + 2E, M = I - 2E (in T and Y, free at that point) with their splits,
    // then W = M P; skp: the step's skip flag (or the expansion's)
    auto factored_w = [&](Mat& Ein, int* skp, double* prt) -> int {
      k_foe_pm<<<1184, 256, 0, ls>>>(skp, n, L.ld, Ein.m, T->m, Y->m);
      TB_LAUNCH_CHECK(ctx);
      int q;
      if ((q = tc_split(ctx, o->precision, T->m, nn, T->hi, T->lo, skp, ls))) return q;
      if ((q = tc_split(ctx, o->precision, Y->m, nn, Y->hi, Y->lo, skp, ls))) return q;
      return gemm(*Y, *T, *W, 1.0f, 0.0f, nullptr, 0.0f, prt, skp);
    };
    for (int step = 0; step < m; ++step) {
      Mat* X = E[step & 1];
      Mat* Xn = E[(step + 1) & 1];
      int* sk = &st->skipd[step];  // leading steps beyond the device's m return at once
      // W = (I - 2E)(I + 2E), A = 2I - W
      if ((r = factored_w(*X, sk, nullptr))) return r;
      k_foe_a<<<1184, 256, 0, ls>>>(sk, L.ld, W->m, A->m);
      TB_LAUNCH_CHECK(ctx);
      if ((r = tc_split(ctx, o->precision, A->m, nn, A->hi, A->lo, sk, ls))) return r;
      // Z1 = (32 A A - 144 A + 210 I) / 99, then Newton-Schulz
      if ((r = gemm(*A, *A, *Z, 32.0f / 99.0f, -144.0f / 99.0f, A->m, 210.0f / 99.0f, nullptr, sk))) return r;
      for (int k = 1; k < ns; ++k) {
        if ((r = gemm(*A, *Z, *T, -1.0f, 0.0f, nullptr, 2.0f, nullptr, sk))) return r;  // T = 2I - A Z
        if ((r = gemm(*Z, *T, *Y, 1.0f, 0.0f, nullptr, 0.0f, nullptr, sk))) return r;   // Z <- Z T
        std::swap(Z, Y);
      }
      // E <- E + E (Z W) (= 2 E Z); trace partials of the last step.  The
      // product kernel writes exactly symmetric results with their splits
      const bool last = step == m - 1;
      if ((r = gemm(*Z, *W, *T, 1.0f, 0.0f, nullptr, 0.0f, nullptr, sk))) return r;
      if ((r = gemm(*X, *T, *Xn, 1.0f, 1.0f, X->m, 0.0f, last ? parts : nullptr, sk))) return r;
    }
    Mat* X = E[m & 1];
    // W and E W of the final E (with Tr W and Tr E W) for the canonical shift
    if ((r = factored_w(*X, skip, partsw))) return r;
    if ((r = gemm(*X, *W, *Z, 1.0f, 0.0f, nullptr, 0.0f, parts3))) return r;
    k_foe_mu<<<1, 32, 0, ls>>>(st, parts, partsw, parts3, sp2_tc_num_parts(ctx, L.ld), n, nocc, beta, tol,
                               o->mu_iters, loop.handle, loop.graph);
    TB_LAUNCH_CHECK(ctx);
    k_foe_keep<<<1184, 256, 0, ls>>>(st, nn, X->m, res);
    TB_LAUNCH_CHECK(ctx);
    xf = X;
    af = W;
    zf = Z;
    return TB_OK;
  };
  for (int it = 0; it < rounds && rc == TB_OK; ++it) rc = expansion();
  if ((rc = tb_loop_end(ctx, &loop, rc))) return rc;
  // canonical shift of the accepted expansion (its E, W and E W are still in
  // *xf, *af, *zf)
  {
    const int fb = std::min(1184, (int)(((size_t)n * n + 255) / 256));
    k_foe_correct<<<fb, 256, 0, s>>>(st, n, L.ld, af->m, zf->m, res);
    TB_LAUNCH_CHECK(ctx);
  }
  const int fb = std::min(1184, (int)(((size_t)n * n + 255) / 256));
  k_foe_finalize<<<fb, 256, 0, s>>>(st, n, L.ld, res, D, nocc, tol, mu, rep);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
