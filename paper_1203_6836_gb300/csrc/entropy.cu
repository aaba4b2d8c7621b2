// Electronic entropy at finite temperature without diagonalisation (the
// entropy term of Eq. Ent_Approx, S = -2 k_B sum_i [f_i ln f_i + (1 - f_i)
// ln(1 - f_i)], f_i the occupations of the Fermi matrix of Eq. EL_4c / DM_perp).
//
// Method (FP64 throughout, GEMMs and traces only).  With Y = beta (H - mu I)
// and the recursive expansion y_k = 2^k y_0, f_k = f(y_k), e_k = f_k - 1/2,
// the function L(y) = ln(1 + e^y) = -ln(1 - f(y)) obeys
//   L(2y) = 2 L(y) - ln 2 + ln(1 + 4 e^2),
// and per state s = L(y) - (1 - f) y, so
//   S / k_B = 2 (n ln 2 + 2^m (dL0 + <E_m, Y0>) + sum_k 2^(m-1-k) Tr ln A_k),
// A_k = I + 4 E_k^2, Y0 = Y / 2^m, dL0 = Tr L(Y0) - n ln 2 - Tr Y0 / 2.
//   * m: the fewest doublings with beta max|eps - mu| <= 2^m / 8 (Gershgorin
//     bounds), so the Taylor series of L and of e(y0) = -tanh(y0/2)/2 at
//     |y0| <= 1/8 reach FP64 accuracy with terms up to y0^8 and y0^7;
//   * each doubling: B = 2A - 3I = 8E^2 - I (spectrum in [-1, 1]), the
//     Chebyshev matrices T_0..T_10 of B, traces of T_0..T_20 from them
//     (Tr T_{10+j} = 2 <T_10, T_j>_F - Tr T_{10-j}), Tr ln A from the degree-20
//     Chebyshev series of ln(3/2 + x/2); A^-1 from the quadratic minimax start
//     (210 I - 144 A + 32 A^2)/99 (A^2 = (T_2 + 12B + 19I)/8 needs no product)
//     and three Newton-Schulz steps; E <- 2 E A^-1;
//   * the terms are of size beta |eps - mu| and cancel to the entropy, which is
//     why FP64 is used: 17 FP64 products per doubling.
// The Fermi matrix D = I/2 + E_m of the same recursion is an optional output.
//
// Device-side control: the host enqueues kMaxM doubling steps; those with
// index below kMaxM - m return at once.

#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kMaxM = 16;        // doubling steps enqueued
constexpr int kP = 10;           // Chebyshev matrices T_0..T_10
constexpr int kDeg = 2 * kP;     // degree of the log series
constexpr int kTile = 64;        // padding unit (and FP64 GEMM tile for ld > 512)
constexpr int kK = 16;           // FP64 GEMM k-step
constexpr int kDotBlocks = 148;  // partial sums of the Frobenius products
constexpr int kMaxDots = 24;

inline int round_up(int x, int q) { return (x + q - 1) / q * q; }

struct EntState {
  double lo, hi, mu, beta;
  int m;      // doubling steps used
  int err;    // TB_ERR_ARG: the spectrum needs more than kMaxM doublings
  double dl0;   // Tr L(Y0) - n ln 2 - Tr Y0 / 2
  double acc;   // sum_k 2^(m-1-k) Tr ln A_k
  double ey;    // <E_m, Y0>
  double S;     // S / k_B
  double tau[kDeg + 1];
};

struct EntLayout {
  int n, ld;
  size_t off_state, off_bparts, off_parts, off_mat, mat_bytes, total;
  // matrices: Y0, Y2, Y4, W, E0, E1, B, T2..T10, Z0, Z1, R
  static constexpr int kMats = 19;
};

EntLayout ent_layout(int n) {
  EntLayout L{};
  L.n = n;
  L.ld = round_up(std::max(n, 1), kTile);
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o += (b + 1023) / 1024 * 1024;
    return r;
  };
  L.off_state = take(sizeof(EntState));
  L.off_bparts = take(sizeof(double) * 2 * ((n + 7) / 8));
  L.off_parts = take(sizeof(double) * kMaxDots * kDotBlocks);
  L.mat_bytes = sizeof(double) * (size_t)L.ld * L.ld;
  L.off_mat = o;
  o += EntLayout::kMats * ((L.mat_bytes + 1023) / 1024 * 1024);
  L.total = o;
  return L;
}

// Doubling step `step` of kMaxM runs only when step >= kMaxM - m.
__device__ __forceinline__ bool ent_skip(const EntState* st, int step) {
  return st->err || step < kMaxM - st->m;
}

// Gershgorin bounds (from the row partials), mu, beta, m.
__global__ void k_ent_setup(const double* bparts, int nb, EntState* st, const double* mu, double kT) {
  double a = INFINITY, b = -INFINITY;
  for (int i = threadIdx.x; i < nb; i += 32) {
    a = fmin(a, bparts[2 * i]);
    b = fmax(b, bparts[2 * i + 1]);
  }
  a = warp_min(a);
  b = warp_max(b);
  if (threadIdx.x != 0) return;
  st->lo = a;
  st->hi = b;
  st->mu = *mu;
  st->beta = 1.0 / kT;
  st->acc = 0.0;
  st->dl0 = 0.0;
  st->ey = 0.0;
  st->S = NAN;
  st->err = 0;
  const double ymax = st->beta * fmax(b - st->mu, st->mu - a);
  int m = 0;
  while (m <= kMaxM && !(ymax <= ldexp(1.0, m) / 8.0)) ++m;
  if (m > kMaxM || !isfinite(ymax)) {
    st->err = TB_ERR_ARG;
    st->m = 0;
  } else {
    st->m = m;
  }
}

// Y0 = beta (H - mu I) / 2^m on the n x n block, zero in the padding.
__global__ void __launch_bounds__(256) k_ent_y0(const double* __restrict__ H, int n, int ld, const EntState* st,
                                                double* __restrict__ Y0) {
  if (st->err) return;
  const double s = ldexp(st->beta, -st->m), mu = st->mu;
  const size_t total = (size_t)ld * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    double y = 0.0;
    if (r < n && c < n) y = s * (H[(size_t)r * n + c] - (r == c ? mu : 0.0));
    Y0[e] = y;
  }
}

// C = alpha A B + beta E + gamma I (ld x ld, FP64), T x T output tile per
// CTA, 16 x 16 threads; skipped when the doubling step `step` is not used.
struct F64Gemm {
  const double* A;
  const double* B;
  const double* E;  // may be null
  double* C;
  int ld;
  double alpha, beta, gamma;
  const EntState* st;
  int step;  // kMaxM: always runs
};

template <int T>
__global__ void __launch_bounds__(256) k_f64_gemm(F64Gemm g) {
  constexpr int R = T / 16;
  __shared__ double As[kK][T + 1];
  __shared__ double Bs[kK][T + 1];
  if (g.step < kMaxM && ent_skip(g.st, g.step)) return;
  if (g.st->err) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * T, col0 = blockIdx.x * T;
  const int ld = g.ld;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < ld; k0 += kK) {
    for (int e = threadIdx.x; e < T * kK; e += 256) {
      const int r = e / kK, kk = e % kK;
      As[kk][r] = g.A[(size_t)(row0 + r) * ld + k0 + kk];
      const int kb = e / T, c = e % T;
      Bs[kb][c] = g.B[(size_t)(k0 + kb) * ld + col0 + c];
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
      const size_t idx = (size_t)r * ld + c;
      double y = g.alpha * acc[i][j];
      if (g.E) y = fma(g.beta, g.E[idx], y);
      if (r == c) y += g.gamma;
      g.C[idx] = y;
    }
}

// Elementwise combinations (each skipped like its doubling step).
//   mode 0: out = -I/4 + X/48 - Y/480 + 17 Z/80640      (the Taylor polynomial of E0 / Y0)
//   mode 1: out = (210 I - 72 (X + 3I) + 4 (Y + 12 X + 19 I)) / 99   (X = B, Y = T_2: Newton-Schulz start)
struct Elem {
  const double* X;
  const double* Y;
  const double* Z;
  double* out;
  int ld, mode;
  const EntState* st;
  int step;
};

__global__ void __launch_bounds__(256) k_ent_elem(Elem a) {
  if (a.step < kMaxM && ent_skip(a.st, a.step)) return;
  if (a.st->err) return;
  const size_t total = (size_t)a.ld * a.ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const bool diag = (e / a.ld) == (e % a.ld);
    const double id = diag ? 1.0 : 0.0;
    double v;
    if (a.mode == 0) v = -0.25 * id + a.X[e] / 48.0 - a.Y[e] / 480.0 + 17.0 * a.Z[e] / 80640.0;
    else v = (210.0 * id - 72.0 * (a.X[e] + 3.0 * id) + 4.0 * (a.Y[e] + 12.0 * a.X[e] + 19.0 * id)) / 99.0;
    a.out[e] = v;
  }
}

// Up to kMaxDots Frobenius products <X_d, Y_d> (Y_d = null: Tr X_d) over the
// ld x ld arrays; block b writes its partial of product d to parts[d * kDotBlocks + b].
struct Dots {
  const double* X[kMaxDots];
  const double* Y[kMaxDots];
  int nd, ld;
  double* parts;
  const EntState* st;
  int step;
};

__global__ void __launch_bounds__(256) k_ent_dots(Dots a) {
  if (a.step < kMaxM && ent_skip(a.st, a.step)) return;
  if (a.st->err) return;
  __shared__ double red[8];
  const size_t total = (size_t)a.ld * a.ld;
  const size_t chunk = (total + gridDim.x - 1) / gridDim.x;
  const size_t e0 = (size_t)blockIdx.x * chunk, e1 = e0 + chunk < total ? e0 + chunk : total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int d = 0; d < a.nd; ++d) {
    double s = 0.0;
    if (a.Y[d]) {
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s = fma(a.X[d][e], a.Y[d][e], s);
    } else {
      // diagonal elements r (ld + 1) inside [e0, e1)
      const size_t dstep = (size_t)a.ld + 1;
      const size_t r = (e0 + dstep - 1) / dstep;
      for (size_t e = (r + threadIdx.x) * dstep; e < e1; e += blockDim.x * dstep) s += a.X[d][e];
    }
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += red[w];
      a.parts[d * kDotBlocks + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// Fixed-order sum of the partials of product d.
__device__ double ent_sum(const double* parts, int d) {
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += parts[d * kDotBlocks + b];
  return s;
}

// Scalar bookkeeping (one thread).
//   mode 0 (start): products <Y0,Y0>, <Y2,Y2>, <Y2,Y4>, <Y4,Y4> -> dL0
//   mode 1 (doubling step): Tr T_1..T_10, <T_10, T_1..T_10> -> Tr ln A -> acc
//   mode 2 (end): <E, Y0> -> S
struct Scal {
  const double* parts;
  EntState* st;
  int mode, step, n, ld;
  double c[kDeg + 1];
};

__global__ void k_ent_scalar(Scal a) {
  EntState* st = a.st;
  if (st->err) return;
  if (a.mode == 1 && ent_skip(st, a.step)) return;
  if (a.mode == 0) {
    const double t2 = ent_sum(a.parts, 0), t4 = ent_sum(a.parts, 1), t6 = ent_sum(a.parts, 2),
                 t8 = ent_sum(a.parts, 3);
    st->dl0 = t2 / 8.0 - t4 / 192.0 + t6 / 2880.0 - 17.0 * t8 / 645120.0;
  } else if (a.mode == 1) {
    // Tr T_0 = ld: the padding states (E = 0, B = -I there) add ln A = ln 1 = 0
    // through the series
    double tau[kDeg + 1];
    tau[0] = a.ld;
    for (int j = 1; j <= kP; ++j) tau[j] = ent_sum(a.parts, j - 1);
    for (int j = 1; j <= kP; ++j) tau[kP + j] = 2.0 * ent_sum(a.parts, kP + j - 1) - tau[kP - j];
    double lnA = 0.0;
    for (int j = 0; j <= kDeg; ++j) {
      lnA = fma(a.c[j], tau[j], lnA);
      st->tau[j] = tau[j];
    }
    const int k = a.step - (kMaxM - st->m);  // index within the m steps used
    st->acc += ldexp(lnA, st->m - 1 - k);
  } else {
    st->ey = ent_sum(a.parts, 0);
    st->S = 2.0 * (a.n * 0.6931471805599453 + ldexp(st->dl0 + st->ey, st->m) + st->acc);
  }
}

// D = I/2 + E on the n x n block (optional output) and S / k_B (device double).
__global__ void __launch_bounds__(256) k_ent_out(const EntState* st, const double* __restrict__ E, int n, int ld,
                                                 double* __restrict__ D, double* S) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && S) *S = st->err ? NAN : st->S;
  if (!D) return;
  const size_t total = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    D[e] = st->err ? NAN : E[(size_t)r * ld + c] + (r == c ? 0.5 : 0.0);
  }
}

// Chebyshev coefficients of ln(3/2 + x/2) on [-1, 1] (interpolation at 64
// Chebyshev nodes, discrete cosine sums; the series converges as 5.83^-j).
void log_coeffs(double* c) {
  const int N = 64;
  for (int j = 0; j <= kDeg; ++j) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
      const double th = M_PI * (k + 0.5) / N;
      s += std::log(1.5 + 0.5 * std::cos(th)) * std::cos(j * th);
    }
    c[j] = 2.0 * s / N;
  }
  c[0] *= 0.5;
}

int launch_gemm(tb_ctx* ctx, const F64Gemm& g, cudaStream_t s) {
  if (g.ld <= 512) {
    const dim3 grid(g.ld / 16, g.ld / 16);
    k_f64_gemm<16><<<grid, 256, 0, s>>>(g);
  } else {
    const dim3 grid(g.ld / 64, g.ld / 64);
    k_f64_gemm<64><<<grid, 256, 0, s>>>(g);
  }
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

}  // namespace

extern "C" int dm_fermi_entropy_workspace_size(int n, size_t* bytes) {
  if (n < 1 || !bytes) return TB_ERR_ARG;
  *bytes = ent_layout(n).total;
  return TB_OK;
}

extern "C" int dm_fermi_entropy(tb_ctx* ctx, const double* H, int n, const double* mu, double kT, double* D,
                                double* S, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !mu || !ws || (!D && !S)) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_fermi_entropy");
  if (n < 1) return tb_fail(ctx, TB_ERR_ARG, "n = %d", n);
  if (!(kT > 0.0)) return tb_fail(ctx, TB_ERR_ARG, "kT = %g must be > 0", kT);
  const EntLayout L = ent_layout(n);
  if (ws_bytes < L.total) return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu", ws_bytes, L.total);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  char* base = static_cast<char*>(ws);
  EntState* st = reinterpret_cast<EntState*>(base + L.off_state);
  double* bparts = reinterpret_cast<double*>(base + L.off_bparts);
  double* parts = reinterpret_cast<double*>(base + L.off_parts);
  const size_t mstride = (L.mat_bytes + 1023) / 1024 * 1024;
  double* M[EntLayout::kMats];
  for (int i = 0; i < EntLayout::kMats; ++i) M[i] = reinterpret_cast<double*>(base + L.off_mat + i * mstride);
  double *Y0 = M[0], *Y2 = M[1], *Y4 = M[2], *W = M[3], *Ebuf[2] = {M[4], M[5]}, *B = M[6];
  double* T[kP + 1] = {nullptr, B, M[7], M[8], M[9], M[10], M[11], M[12], M[13], M[14], M[15]};
  double *Z[2] = {M[16], M[17]}, *R = M[18];
  const int ld = L.ld;
  const int eg = std::min(1184, (int)(((size_t)ld * ld + 255) / 256));

  int rc = sp2_launch_bounds(ctx, H, n, bparts, s);
  if (rc) return rc;
  k_ent_setup<<<1, 32, 0, s>>>(bparts, (n + 7) / 8, st, mu, kT);
  TB_LAUNCH_CHECK(ctx);
  k_ent_y0<<<eg, 256, 0, s>>>(H, n, ld, st, Y0);
  TB_LAUNCH_CHECK(ctx);
  auto gemm = [&](const double* A, const double* Bm, const double* E, double* C, double alpha, double beta,
                  double gamma, int step) {
    F64Gemm g{A, Bm, E, C, ld, alpha, beta, gamma, st, step};
    return launch_gemm(ctx, g, s);
  };
  auto elem = [&](const double* X, const double* Y, const double* Zm, double* out, int mode, int step) {
    Elem a{X, Y, Zm, out, ld, mode, st, step};
    k_ent_elem<<<eg, 256, 0, s>>>(a);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  };
  Scal sc{};
  sc.parts = parts;
  sc.st = st;
  sc.n = n;
  sc.ld = ld;
  log_coeffs(sc.c);

  // ---- start: dL0 and E0 = Y0 (-I/4 + Y2/48 - Y4/480 + 17 Y2 Y4/80640)
  if ((rc = gemm(Y0, Y0, nullptr, Y2, 1.0, 0.0, 0.0, kMaxM))) return rc;
  if ((rc = gemm(Y2, Y2, nullptr, Y4, 1.0, 0.0, 0.0, kMaxM))) return rc;
  {
    Dots d{};
    d.nd = 4;
    d.ld = ld;
    d.parts = parts;
    d.st = st;
    d.step = kMaxM;
    d.X[0] = Y0; d.Y[0] = Y0;
    d.X[1] = Y2; d.Y[1] = Y2;
    d.X[2] = Y2; d.Y[2] = Y4;
    d.X[3] = Y4; d.Y[3] = Y4;
    k_ent_dots<<<kDotBlocks, 256, 0, s>>>(d);
    TB_LAUNCH_CHECK(ctx);
    sc.mode = 0;
    sc.step = kMaxM;
    k_ent_scalar<<<1, 1, 0, s>>>(sc);
    TB_LAUNCH_CHECK(ctx);
  }
  if ((rc = gemm(Y2, Y4, nullptr, R, 1.0, 0.0, 0.0, kMaxM))) return rc;
  if ((rc = elem(Y2, Y4, R, W, 0, kMaxM))) return rc;
  if ((rc = gemm(Y0, W, nullptr, Ebuf[0], 1.0, 0.0, 0.0, kMaxM))) return rc;

  // ---- doublings: the first kMaxM - m return at once; E alternates between
  // the two buffers only in the steps that run, so both start as E0
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(Ebuf[1], Ebuf[0], L.mat_bytes, cudaMemcpyDeviceToDevice, s));
  for (int step = 0; step < kMaxM; ++step) {
    // the steps used are kMaxM - m .. kMaxM - 1; step parity decides the buffers,
    // and both buffers hold E0 before the first used step
    double* Ein = Ebuf[step & 1];
    double* Eout = Ebuf[(step + 1) & 1];
    if ((rc = gemm(Ein, Ein, nullptr, B, 8.0, 0.0, -1.0, step))) return rc;  // B = 8 E^2 - I
    if ((rc = gemm(B, B, nullptr, T[2], 2.0, 0.0, -1.0, step))) return rc;   // T_2 = 2 B^2 - I
    for (int j = 3; j <= kP; ++j)
      if ((rc = gemm(B, T[j - 1], T[j - 2], T[j], 2.0, -1.0, 0.0, step))) return rc;  // T_j = 2 B T_{j-1} - T_{j-2}
    {
      // products 0..9: Tr T_1..T_10; 10..19: <T_10, T_1..T_10>
      Dots d{};
      d.nd = 2 * kP;
      d.ld = ld;
      d.parts = parts;
      d.st = st;
      d.step = step;
      for (int j = 1; j <= kP; ++j) {
        d.X[j - 1] = T[j];
        d.Y[j - 1] = nullptr;
        d.X[kP + j - 1] = T[kP];
        d.Y[kP + j - 1] = T[j];
      }
      k_ent_dots<<<kDotBlocks, 256, 0, s>>>(d);
      TB_LAUNCH_CHECK(ctx);
    }
    sc.mode = 1;
    sc.step = step;
    k_ent_scalar<<<1, 1, 0, s>>>(sc);
    TB_LAUNCH_CHECK(ctx);
    // A^-1: Z = (210 I - 144 A + 32 A^2)/99 with A = (B + 3I)/2, A^2 = (T_2 + 12 B + 19 I)/8,
    // then Z <- Z (2I - A Z), A Z = (B Z + 3 Z)/2
    if ((rc = elem(B, T[2], nullptr, Z[0], 1, step))) return rc;
    for (int it = 0; it < 3; ++it) {
      if ((rc = gemm(B, Z[it & 1], Z[it & 1], R, -0.5, -1.5, 2.0, step))) return rc;  // R = 2I - A Z
      if ((rc = gemm(Z[it & 1], R, nullptr, Z[(it + 1) & 1], 1.0, 0.0, 0.0, step))) return rc;
    }
    if ((rc = gemm(Ein, Z[1], nullptr, Eout, 2.0, 0.0, 0.0, step))) return rc;  // E <- 2 E A^-1
  }
  // the last step used has index kMaxM - 1: its output is in Ebuf[kMaxM & 1]
  double* Em = Ebuf[kMaxM & 1];
  {
    Dots d{};
    d.nd = 1;
    d.ld = ld;
    d.parts = parts;
    d.st = st;
    d.step = kMaxM;
    d.X[0] = Em;
    d.Y[0] = Y0;
    k_ent_dots<<<kDotBlocks, 256, 0, s>>>(d);
    TB_LAUNCH_CHECK(ctx);
    sc.mode = 2;
    sc.step = kMaxM;
    k_ent_scalar<<<1, 1, 0, s>>>(sc);
    TB_LAUNCH_CHECK(ctx);
  }
  const int ob = D ? std::min(1184, (int)(((size_t)n * n + 255) / 256)) : 1;
  k_ent_out<<<ob, 256, 0, s>>>(st, Em, n, ld, D, S);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
