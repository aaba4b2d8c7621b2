// Non-orthogonal formulation (row f3, App. D.1): the congruence factor
// Z = S^{-1/2} (Z^T S Z = I, Eq. Congr), H_perp = Z^T H Z, the density matrix
// rho = Z rho_perp Z^T of rho_perp = theta(mu0 I - H_perp) (dm_sp2) or the
// Fermi-Dirac matrix (dm_fermi) (Eq. DM_perp), and the energy-weighted
// density matrix W = Z (H_perp rho_perp + rho_perp H_perp) Z^T / 2 of the
// Pulay force.
//
// Z by the coupled Newton-Schulz iteration (GEMM only): with c >= lambda_max(S)
// (Gershgorin), Y_0 = S/c, Z_0 = I and
//   T_k = (3 I - Z_k Y_k)/2,  Y_{k+1} = Y_k T_k,  Z_{k+1} = T_k Z_k,
// Y_k -> (S/c)^{1/2} and Z_k -> (S/c)^{-1/2}, quadratically once
// ||I - S/c|| < 1 (the eigenvalues of S/c lie in (0, 1]); Z = Z_k / sqrt(c).
// Since Z_k Y_k = 3 I - 2 T_k, the residual max |Z_k Y_k - I| = 2 max |I - T_k|
// comes from T_k without another product; the iteration stops on the device
// at 1e-13, or below 1e-9 once the residual no longer halves (the rounding
// floor of the FP64 products at large n); later launches of the fixed
// sequence return at once.
//
// All products are FP64 GEMMs on the FP64 units (no tensor-core FP64 on
// GB300): T x T output tiles, bounds-guarded for any n, row-major with
// stride n.

#include "common.cuh"

#include <algorithm>

namespace {

constexpr int kMaxNS = 24;     // Newton-Schulz iterations at most (about 12 reach 1e-13 for cond(S) = 100)
constexpr double kNSTol = 1e-13;
constexpr double kNSFloor = 1e-9;  // below it, a residual that no longer halves is the rounding floor
constexpr int kK = 16;         // GEMM k-step

struct NonorthState {
  double c;        // Gershgorin bound of S
  double res;      // last Newton-Schulz residual
  int done;        // the iteration has converged
  int iters;
  int err;
};

struct Layout {
  size_t off_state, off_mat, mat_bytes, off_inner, total;
  size_t inner_bytes;
};

constexpr int kMats = 7;  // Z, Y, T, P (scratch), H_perp, rho_perp, Q (scratch)

Layout make_layout(int n, size_t inner) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o += (b + 1023) / 1024 * 1024;
    return r;
  };
  L.off_state = take(sizeof(NonorthState));
  L.mat_bytes = (sizeof(double) * (size_t)n * n + 1023) / 1024 * 1024;
  L.off_mat = take(L.mat_bytes * kMats);
  L.inner_bytes = inner;
  L.off_inner = take(inner);
  L.total = o;
  return L;
}

// C = alpha A B + beta E + gamma I (E may be null), n x n row-major; skipped
// when *skip is set.  T x T tile per CTA, 256 threads with (T/16)^2 outputs.
template <int T>
__global__ void __launch_bounds__(256) k_gemm64(int n, double alpha, const double* __restrict__ A,
                                                const double* __restrict__ B, double beta,
                                                const double* __restrict__ E, double gamma,
                                                double* __restrict__ C, const int* skip) {
  constexpr int R = T / 16;
  __shared__ double As[kK][T + 1];
  __shared__ double Bs[kK][T + 1];
  if (skip && *skip) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * T, col0 = blockIdx.x * T;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < n; k0 += kK) {
    for (int e = threadIdx.x; e < T * kK; e += 256) {
      const int r = e / kK, kk = e % kK;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < n && gk < n) ? A[(size_t)gr * n + gk] : 0.0;
      const int kb = e / T, c = e % T;
      const int gkb = k0 + kb, gc = col0 + c;
      Bs[kb][c] = (gkb < n && gc < n) ? B[(size_t)gkb * n + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      double av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      if (r >= n || c >= n) continue;
      const size_t e = (size_t)r * n + c;
      double v = alpha * acc[i][j];
      if (E) v += beta * E[e];
      if (r == c) v += gamma;
      C[e] = v;
    }
}

int gemm(tb_ctx* ctx, int n, double alpha, const double* A, const double* B, double beta, const double* E,
         double gamma, double* C, const int* skip, cudaStream_t s) {
  if (n <= 512) {
    const dim3 g((n + 15) / 16, (n + 15) / 16);
    k_gemm64<16><<<g, 256, 0, s>>>(n, alpha, A, B, beta, E, gamma, C, skip);
  } else {
    const dim3 g((n + 63) / 64, (n + 63) / 64);
    k_gemm64<64><<<g, 256, 0, s>>>(n, alpha, A, B, beta, E, gamma, C, skip);
  }
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// c = max_i sum_j |S_ij| (one block), the state reset.
__global__ void k_ns_bound(const double* __restrict__ S, int n, NonorthState* st) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double r = 0.0;
    for (int j = 0; j < n; ++j) r += fabs(S[(size_t)i * n + j]);
    m = fmax(m, r);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) {
      st->c = m > 0.0 ? m : 1.0;
      st->res = INFINITY;
      st->done = 0;
      st->iters = 0;
      st->err = 0;
    }
  }
}

// Y = S / c, Z = I.
__global__ void k_ns_init(const double* __restrict__ S, int n, const NonorthState* st, double* __restrict__ Y,
                          double* __restrict__ Z) {
  const double inv = 1.0 / st->c;
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    Y[e] = S[e] * inv;
    Z[e] = (e / n == e % n) ? 1.0 : 0.0;
  }
}

// Residual of T_k: 2 max |I - T_k| (one block), then the stop decision.
__global__ void k_ns_check(const double* __restrict__ T, int n, NonorthState* st) {
  __shared__ double red[32];
  if (st->done) return;
  double m = 0.0;
  const size_t total = (size_t)n * n;
  for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
    const double d = (e / n == e % n) ? 1.0 - T[e] : -T[e];
    m = fmax(m, fabs(d));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) {
      const double r = 2.0 * m, prev = st->res;
      st->res = r;
      st->iters += 1;
      // converged, or stalled at the FP64 rounding floor of the products
      if (r <= kNSTol || (r <= kNSFloor && r >= 0.5 * prev)) st->done = 1;
    }
  }
}

// Z <- Z / sqrt(c) (the final factor), report.
__global__ void k_ns_finish(double* __restrict__ Z, int n, const NonorthState* st, tb_nonorth_report* rep) {
  const double f = 1.0 / sqrt(st->c);
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    Z[e] *= f;
  if (rep && blockIdx.x == 0 && threadIdx.x == 0) {
    rep->status = st->done ? TB_OK : TB_ERR_NOT_CONVERGED;
    rep->ns_iters = st->iters;
    rep->ns_residual = st->res;
  }
}

// W = (W' + W'^T) / 2 in place.
__global__ void k_symmetrize(double* __restrict__ W, int n) {
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / n, c = e % n;
    if (r < c) {
      const double a = W[e], b = W[c * n + r];
      const double m = 0.5 * (a + b);
      W[e] = m;
      W[c * n + r] = m;
    }
  }
}

// dst = src unless *skip.
__global__ void k_copy_unless(const double* __restrict__ src, double* __restrict__ dst, int n, const int* skip) {
  if (*skip) return;
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

size_t inner_bytes(int n, double kT, const tb_sp2_opts* so, const tb_fermi_opts* fo, int* rc) {
  size_t b = 0;
  *rc = kT > 0.0 ? dm_fermi_workspace_size(n, fo, &b) : dm_sp2_workspace_size(n, so, &b);
  return b;
}

}  // namespace

extern "C" int dm_nonorth_workspace_size(int n, double kT, const tb_sp2_opts* so, const tb_fermi_opts* fo,
                                         size_t* bytes) {
  if (n < 1 || !bytes || (kT > 0.0 ? !fo : !so)) return TB_ERR_ARG;
  int rc = TB_OK;
  const size_t inner = inner_bytes(n, kT, so, fo, &rc);
  if (rc) return rc;
  *bytes = make_layout(n, inner).total;
  return TB_OK;
}

extern "C" int dm_nonorth(tb_ctx* ctx, const double* H, const double* S, int n, double n_occ, double kT,
                          const tb_sp2_opts* so, const tb_fermi_opts* fo, double* mu, double* rho, double* W,
                          void* ws, size_t ws_bytes, tb_sp2_report* sp2_report, tb_fermi_report* fermi_report,
                          tb_nonorth_report* report, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !S || !rho || !W || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_nonorth");
  if (n < 1) return tb_fail(ctx, TB_ERR_ARG, "n = %d", n);
  if (kT > 0.0 ? (!fo || !mu) : !so) return tb_fail(ctx, TB_ERR_ARG, "dm_nonorth: missing solver options");
  int rc = TB_OK;
  const size_t inner = inner_bytes(n, kT, so, fo, &rc);
  if (rc) return tb_fail(ctx, rc, "dm_nonorth: inner workspace query failed");
  const Layout L = make_layout(n, inner);
  if (ws_bytes < L.total) return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu", ws_bytes, L.total);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  char* base = static_cast<char*>(ws);
  NonorthState* st = reinterpret_cast<NonorthState*>(base + L.off_state);
  double* M[kMats];
  for (int i = 0; i < kMats; ++i) M[i] = reinterpret_cast<double*>(base + L.off_mat + i * L.mat_bytes);
  double *Z = M[0], *Y = M[1], *T = M[2], *P = M[3], *Hp = M[4], *Dp = M[5], *Q = M[6];
  const int eb = std::min(1184, (int)(((size_t)n * n + 255) / 256));

  // Z = S^{-1/2} by coupled Newton-Schulz; each update goes through P and a copy,
  // so the current iterate stays in Z and Y whichever launch the stop skips
  k_ns_bound<<<1, 1024, 0, s>>>(S, n, st);
  TB_LAUNCH_CHECK(ctx);
  k_ns_init<<<eb, 256, 0, s>>>(S, n, st, Y, Z);
  TB_LAUNCH_CHECK(ctx);
  const int* skip = &st->done;
  for (int it = 0; it < kMaxNS; ++it) {
    if ((rc = gemm(ctx, n, -0.5, Z, Y, 0.0, nullptr, 1.5, T, skip, s))) return rc;  // T = 3/2 I - Z Y / 2
    k_ns_check<<<1, 1024, 0, s>>>(T, n, st);
    TB_LAUNCH_CHECK(ctx);
    if ((rc = gemm(ctx, n, 1.0, Y, T, 0.0, nullptr, 0.0, P, skip, s))) return rc;
    k_copy_unless<<<eb, 256, 0, s>>>(P, Y, n, skip);
    TB_LAUNCH_CHECK(ctx);
    if ((rc = gemm(ctx, n, 1.0, T, Z, 0.0, nullptr, 0.0, P, skip, s))) return rc;
    k_copy_unless<<<eb, 256, 0, s>>>(P, Z, n, skip);
    TB_LAUNCH_CHECK(ctx);
  }
  k_ns_finish<<<eb, 256, 0, s>>>(Z, n, st, report);
  TB_LAUNCH_CHECK(ctx);

  // H_perp = Z H Z (Z symmetric)
  if ((rc = gemm(ctx, n, 1.0, Z, H, 0.0, nullptr, 0.0, P, nullptr, s))) return rc;
  if ((rc = gemm(ctx, n, 1.0, P, Z, 0.0, nullptr, 0.0, Hp, nullptr, s))) return rc;
  k_symmetrize<<<eb, 256, 0, s>>>(Hp, n);
  TB_LAUNCH_CHECK(ctx);
  // rho_perp
  void* iws = base + L.off_inner;
  if (kT > 0.0)
    rc = dm_fermi(ctx, Hp, n, n_occ, kT, fo, Dp, mu, iws, L.inner_bytes, fermi_report, s);
  else
    rc = dm_sp2(ctx, Hp, n, n_occ, so, Dp, iws, L.inner_bytes, sp2_report, s);
  if (rc) return rc;
  // rho = Z rho_perp Z
  if ((rc = gemm(ctx, n, 1.0, Z, Dp, 0.0, nullptr, 0.0, P, nullptr, s))) return rc;
  if ((rc = gemm(ctx, n, 1.0, P, Z, 0.0, nullptr, 0.0, rho, nullptr, s))) return rc;
  k_symmetrize<<<eb, 256, 0, s>>>(rho, n);
  TB_LAUNCH_CHECK(ctx);
  // W = Z (H_perp rho_perp + rho_perp H_perp) Z / 2 = sym(Z H_perp rho_perp Z)
  if ((rc = gemm(ctx, n, 1.0, Hp, Dp, 0.0, nullptr, 0.0, Q, nullptr, s))) return rc;
  if ((rc = gemm(ctx, n, 1.0, Z, Q, 0.0, nullptr, 0.0, P, nullptr, s))) return rc;
  if ((rc = gemm(ctx, n, 1.0, P, Z, 0.0, nullptr, 0.0, W, nullptr, s))) return rc;
  k_symmetrize<<<eb, 256, 0, s>>>(W, n);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
