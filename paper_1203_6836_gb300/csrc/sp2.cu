// SP2 purification (rows a2, a3, a4 FP64 path, a6): D = theta(mu0 I - H).
//
// The recursive second-order spectral projection of Sec. III.B, with the
// reading: X0 = (eps_max I - H)/(eps_max - eps_min) from Gershgorin bounds;
// each projection replaces X by X^2 or by 2X - X^2, the branch chosen from
// Tr X and Tr X^2 = ||X||_F^2 (look-ahead rule: the projection whose trace
// lands closer to N_occ); stop when Tr X - Tr X^2 <= tol.
//
// Device-side control: step kernel k first reduces, in a fixed order, the
// trace partials written by the epilogue of kernel k-1, takes the
// stop/branch decision (identical in every CTA) and either returns at once
// or computes X_{k+1}.  Launched eagerly, the host enqueues max_iter + 1 step
// kernels; captured into a CUDA graph, the projections after the first are
// a while node that stops with the decision.  No host synchronisation
// happens inside dm_sp2.
//
// Precision paths: TB_PREC_FP64 runs every projection as an FP64 GEMM (16 x 16
// output tiles for ld <= 512, 64 x 64 above); the tensor-core paths
// (gemm_tc.cu) keep X as an FP32 master plus bf16/tf32 operand splits and
// hand the final iterate to `refine_iters` FP64 projections, computed exactly
// from integer slices on the bf16 tensor cores (gemm_oz.cu, ld <= 4096) or
// with FP64 FMAs.  Traces and their reductions are FP64 throughout.

#include "common.cuh"

#include <algorithm>
#include <atomic>

namespace {

constexpr int kF64Tile = 64;     // FP64 GEMM output tile (padding unit of the FP64 path)
constexpr int kF64K = 16;        // FP64 GEMM k-step
constexpr int kInitTile = 64;    // X0 / conversion tile
constexpr int kLoopUnroll = 16;  // projections per pass of the graph's while node (even)

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Output tile of the FP64 projection: GB300 runs FP64 at ~8 GFLOP/s per SM,
// so small matrices are cut into 16 x 16 tiles to spread one product over
// many SMs; from ld = 576 on, 64 x 64 tiles give enough CTAs.
inline int f64_tile(int ld) { return ld <= 512 ? 16 : kF64Tile; }

struct Layout {
  int n, ld, prec;
  size_t off_state, off_bparts, off_parts, off_f0, off_f1, off_m0, off_m1, off_h0, off_l0, off_h1,
      off_l1, off_slices, off_exps, total;
  int max_parts;
  bool oz;  // refinement by the emulated-FP64 tensor-core kernel
};

Layout make_layout(int n, int prec, int refine, int refine_mode = 1) {
  Layout L{};
  L.n = n;
  L.prec = prec;
  const bool tc = prec != TB_PREC_FP64;
  L.ld = round_up(std::max(n, 1), tc ? sp2_tc_tile() : kF64Tile);
  const int t_f64 = (L.ld / f64_tile(L.ld)) * (L.ld / f64_tile(L.ld));
  const int t_init = (L.ld / kInitTile) * (L.ld / kInitTile);
  const int t_tc = tc ? sp2_tc_num_tiles(L.ld) : 0;
  L.max_parts = std::max(std::max(t_f64, t_init), t_tc);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 1023) / 1024 * 1024;
    return r;
  };
  L.off_state = take(sizeof(SP2State));
  L.off_bparts = take(sizeof(double) * 2 * ((L.ld + 7) / 8));
  L.off_parts = take(sizeof(double) * 3 * 2 * (size_t)L.max_parts);
  const size_t nn = (size_t)L.ld * L.ld;
  const bool need_f64 = !tc || refine > 0;
  L.off_f0 = need_f64 ? take(sizeof(double) * nn) : 0;
  L.off_f1 = need_f64 ? take(sizeof(double) * nn) : 0;
  if (tc) {
    const size_t ob = sp2_tc_operand_bytes(prec);
    const bool split = prec == TB_PREC_TF32X3 || prec == TB_PREC_BF16X3;
    L.off_m0 = take(sizeof(float) * nn);
    L.off_m1 = take(sizeof(float) * nn);
    L.off_h0 = take(ob * nn);
    L.off_h1 = take(ob * nn);
    L.off_l0 = split ? take(ob * nn) : 0;
    L.off_l1 = split ? take(ob * nn) : 0;
    L.oz = refine > 0 && refine_mode == 0 && L.ld <= sp2_oz_max_ld();
    if (L.oz) {
      L.off_slices = take(sp2_oz_slice_bytes(L.ld));
      L.off_exps = take(sizeof(int) * (size_t)L.ld);
    }
  }
  L.total = o;
  return L;
}

// ----------------------------------------------------------- Gershgorin bounds

// Warp per row: c_i = H_ii, r_i = sum_{j != i} |H_ij|; per-block min(c - r),
// max(c + r) into bparts.
__global__ void __launch_bounds__(256) k_bounds(const double* __restrict__ H, int n,
                                                double* __restrict__ bparts) {
  __shared__ double smin[8], smax[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  double lo = INFINITY, hi = -INFINITY;
  if (row < n) {
    const double* Hr = H + (size_t)row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += (j == row) ? 0.0 : fabs(Hr[j]);
    s = warp_sum(s);
    const double c = Hr[row];
    lo = c - s;
    hi = c + s;
  }
  if (lane == 0) {
    smin[warp] = lo;
    smax[warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = smin[0], b = smax[0];
    for (int w = 1; w < 8; ++w) {
      a = fmin(a, smin[w]);
      b = fmax(b, smax[w]);
    }
    bparts[2 * blockIdx.x] = a;
    bparts[2 * blockIdx.x + 1] = b;
  }
}

// Every block reduces the bound partials (fixed order) and writes its tile
// of X0 = (emax I - H)/(emax - emin), zero outside n x n, plus the tile's
// trace partials (Tr X0, ||X0||_F^2).  Output: FP64 X (X64 != nullptr) or the
// FP32 master of the tensor-core path (its operand split follows in gemm_tc.cu).
__device__ __forceinline__ void block_sum3(double a, double b, double c, double* out) {
  __shared__ double sh[3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    sh[0][warp] = a;
    sh[1][warp] = b;
    sh[2][warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < nw; ++w) {
      x += sh[0][w];
      y += sh[1][w];
      z += sh[2][w];
    }
    out[0] = x;
    out[1] = y;
    out[2] = z;
  }
}

__global__ void __launch_bounds__(256) k_init_x(const double* __restrict__ H, int n, int ld,
                                                const double* __restrict__ bparts, int nbparts,
                                                SP2State* st, double* __restrict__ X64,
                                                float* __restrict__ X32, double* __restrict__ parts) {
  __shared__ double s_lo, s_hi;
  if (threadIdx.x < 32) {
    double a = INFINITY, b = -INFINITY;
    for (int i = threadIdx.x; i < nbparts; i += 32) {
      a = fmin(a, bparts[2 * i]);
      b = fmax(b, bparts[2 * i + 1]);
    }
    a = warp_min(a);
    b = warp_max(b);
    if (threadIdx.x == 0) {
      s_lo = a;
      s_hi = b;
    }
  }
  __syncthreads();
  const double emin = s_lo, emax = s_hi;
  double w = emax - emin;
  if (!(w > 0.0)) w = 1.0;  // H = c I: X0 = 0 (no gap; reported through the trace)
  const double inv = 1.0 / w;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    st->emin = emin;
    st->emax = emax;
  }
  const int r0 = blockIdx.y * kInitTile, c0 = blockIdx.x * kInitTile;
  double t1 = 0.0, t2 = 0.0;
  for (int e = threadIdx.x; e < kInitTile * kInitTile; e += blockDim.x) {
    const int r = r0 + e / kInitTile, c = c0 + e % kInitTile;
    double x = 0.0;
    if (r < n && c < n) x = ((r == c ? emax : 0.0) - H[(size_t)r * n + c]) * inv;
    if (X64) {
      X64[(size_t)r * ld + c] = x;
    } else {
      const float xf = (float)x;
      X32[(size_t)r * ld + c] = xf;
      x = (double)xf;
    }
    if (r == c) t1 += x;
    t2 += x * x;
  }
  block_sum3(t1, t2, 0.0, parts + 3 * (blockIdx.y * gridDim.x + blockIdx.x));
}

// ------------------------------------------------------------ FP64 GEMM step

// X_out = X_in^2 or 2 X_in - X_in^2 for one 64x64 output tile; 256 threads,
// each 4x4 outputs at rows ty + 16i, cols tx + 16j; k-step 16 through shared
// memory.  X is symmetric, so B = X is read row-major like A.
// T x T output tile per CTA, 16 x 16 threads, (T/16)^2 outputs per thread.
template <int T>
__global__ void __launch_bounds__(256) k_sp2_step_f64(const SP2StepArgs a_in, const double* __restrict__ X,
                                                      double* __restrict__ Y) {
  constexpr int R = T / 16;
  __shared__ double As[kF64K][T + 1];
  __shared__ double Bs[kF64K][T + 1];
  __shared__ double s_t[3];
  __shared__ int s_dec[3];
  SP2State* st = a_in.st;
  const int done = a_in.phase == 0 ? st->done : st->rdone;
  SP2StepArgs a = a_in;
  a.k = sp2_step_index(a_in, done || st->err);
  if (done || st->err) return;
  if (threadIdx.x < 32) {
    double t1, t2;
    {
      const int lane = threadIdx.x;
      double x = 0, y = 0, z = 0;
      for (int i = lane; i < a.nparts_in; i += 32) {
        x += a.parts_in[3 * i];
        y += a.parts_in[3 * i + 1];
        z += a.parts_in[3 * i + 2];
      }
      t1 = warp_sum(x);
      t2 = warp_sum(y);
      z = warp_sum(z);
      if (lane == 0) {
        s_t[0] = t1;
        s_t[1] = t2;
        s_t[2] = z;
        int br = 0, capped = 0;
        const double* h1 = a.phase == 0 ? st->t1 : st->rt1;
        const double* h2 = a.phase == 0 ? st->t2 : st->rt2;
        const int stop = sp2_decide(a, t1, t2, h1, h2, false, &br, &capped);
        s_dec[0] = stop;
        s_dec[1] = br;
        s_dec[2] = capped;
      }
    }
  }
  __syncthreads();
  const int stop = s_dec[0], br = s_dec[1];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    if (a.phase == 0) {
      st->t1[a.k] = s_t[0];
      st->t2[a.k] = s_t[1];
      if (stop) {
        st->iters = a.k;
        st->capped = s_dec[2];
        st->done = 1;
        if (a.cond) cudaGraphSetConditional(a.loop, 0);
      } else if (br) {
        st->branch[a.k >> 6] |= 1ull << (a.k & 63);
      }
    } else {
      st->rt1[a.k] = s_t[0];
      st->rt2[a.k] = s_t[1];
      if (a.k > 0) st->idem_fro = sqrt(s_t[2]);
      if (stop) {
        st->riters = a.k;
        st->rcapped = s_dec[2];
        st->rdone = 1;
      } else if (br) {
        st->rbranch |= 1ull << a.k;
      }
    }
  }
  if (stop) return;

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * T, col0 = blockIdx.x * T;
  const int ld = a.ld;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < ld; k0 += kF64K) {
    // T rows x 16 k of A (rows of X) and 16 k x T cols of B (rows of X)
    for (int e = threadIdx.x; e < T * kF64K; e += 256) {
      const int r = e / kF64K, kk = e % kF64K;
      As[kk][r] = X[(size_t)(row0 + r) * ld + k0 + kk];
      const int kb = e / T, c = e % T;
      Bs[kb][c] = X[(size_t)(k0 + kb) * ld + col0 + c];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kF64K; ++kk) {
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
  double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
      const double x = X[(size_t)r * ld + c];
      const double cxx = acc[i][j];
      const double y = br ? 2.0 * x - cxx : cxx;
      Y[(size_t)r * ld + c] = y;
      if (r == c) t1 += y;
      t2 += y * y;
      t3 += (cxx - x) * (cxx - x);
    }
  block_sum3(t1, t2, t3, a.parts_out + 3 * (blockIdx.y * gridDim.x + blockIdx.x));
}

void launch_f64(dim3 g, const SP2StepArgs& a, const double* X, double* Y, cudaStream_t s) {
  if (f64_tile(a.ld) == 16) k_sp2_step_f64<16><<<g, 256, 0, s>>>(a, X, Y);
  else k_sp2_step_f64<kF64Tile><<<g, 256, 0, s>>>(a, X, Y);
}

// FP32 master (buffer chosen by the main phase's iteration count) -> FP64,
// with trace partials: the start of the FP64 refinement.
__global__ void __launch_bounds__(256) k_to_f64(const SP2State* st, const float* __restrict__ M0,
                                                const float* __restrict__ M1, int ld,
                                                double* __restrict__ F, double* __restrict__ parts) {
  const float* M = (st->iters & 1) ? M1 : M0;
  const int r0 = blockIdx.y * kInitTile, c0 = blockIdx.x * kInitTile;
  double t1 = 0.0, t2 = 0.0;
  for (int e = threadIdx.x; e < kInitTile * kInitTile; e += blockDim.x) {
    const int r = r0 + e / kInitTile, c = c0 + e % kInitTile;
    const double x = (double)M[(size_t)r * ld + c];
    F[(size_t)r * ld + c] = x;
    if (r == c) t1 += x;
    t2 += x * x;
  }
  block_sum3(t1, t2, 0.0, parts + 3 * (blockIdx.y * gridDim.x + blockIdx.x));
}

// Copy the final iterate into D (n x n) and fill the report.
__global__ void __launch_bounds__(256) k_finalize(SP2State* st, int n, int ld, int mode,
                                                  const double* __restrict__ F0,
                                                  const double* __restrict__ F1,
                                                  const float* __restrict__ M0,
                                                  const float* __restrict__ M1,
                                                  double* __restrict__ D, double nocc,
                                                  tb_sp2_report* rep) {
  // mode 0: FP64 main phase; 1: FP64 refinement; 2: FP32 master, no refinement
  const size_t total = (size_t)n * n;
  const int sel = mode == 1 ? (st->riters & 1) : (st->iters & 1);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    double x;
    if (mode == 2)
      x = (double)(sel ? M1 : M0)[(size_t)r * ld + c];
    else
      x = (sel ? F1 : F0)[(size_t)r * ld + c];
    D[e] = x;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && rep) {
    double t1, t2;
    if (mode == 1) {
      t1 = st->rt1[st->riters];
      t2 = st->rt2[st->riters];
    } else {
      t1 = st->t1[st->iters];
      t2 = st->t2[st->iters];
    }
    // status: device error; an FP64 phase that hit its cap without reaching
    // |Tr X - Tr X^2| <= 1e-6 max(1, N_occ); a trace that missed N_occ
    // (no gap at the occupation)
    int status = TB_OK;
    const double e = t1 - t2;
    const bool capped = mode == 1 ? st->rcapped : (mode == 0 ? st->capped : 0);
    if (st->err) status = st->err;
    else if (capped && fabs(e) > 1e-6 * fmax(1.0, nocc)) status = TB_ERR_NOT_CONVERGED;
    else if (fabs(t1 - nocc) > 0.25) status = TB_ERR_GAP;
    rep->status = status;
    rep->iters = st->iters;
    rep->refine_iters = mode == 1 ? st->riters : 0;
    rep->n = n;
    rep->eps_min = st->emin;
    rep->eps_max = st->emax;
    rep->trace = t1;
    rep->idem_trace = e;
    rep->idem_fro = mode == 1 && st->riters > 0 ? st->idem_fro : -1.0;
    rep->branch_bits[0] = st->branch[0];
    rep->branch_bits[1] = st->branch[1];
    rep->refine_bits = st->rbranch;
    rep->block_products = 0;
    rep->blocks = 0;
  }
}

}  // namespace

int sp2_launch_bounds(tb_ctx* ctx, const double* H, int n, double* bparts, cudaStream_t s) {
  k_bounds<<<(n + 7) / 8, 256, 0, s>>>(H, n, bparts);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// The main phase's projections k = 0..max_iter.  Projection 0 (whose input
// partials come from the X0 kernel) is launched on `s` and seeds the device
// counter st->kc.  When `s` is being captured into a CUDA graph, the rest is
// one while node whose body is kLoopUnroll launches of alternating parity
// (1, 0, 1, ...): the launches read their index from the counter and clear
// the condition once the phase stops, so a replay runs the projections it
// needs plus at most kLoopUnroll - 1 launches that return at once.  (Each
// pass of a while node costs a few microseconds, more than an empty launch,
// so the body holds several projections.)  Otherwise the host unrolls
// k = 1..max_iter; the launches after the stop return at once.
// `launch(args, k, stream)` enqueues one projection whose buffers are those
// of parity k & 1.
template <class F>
int main_phase(tb_ctx* ctx, SP2StepArgs& a, int np_first, int np, double* const slot[2], cudaStream_t s,
               F&& launch) {
  a.k = 0;
  a.kc = a.st->kc;
  a.kpar = 0;
  a.cond = 0;
  a.nparts_in = np_first;
  a.parts_in = slot[0];
  a.parts_out = slot[1];
  tb_prof_mark(ctx, 0, 0, s);
  int rc = launch(a, 0, s);
  if (rc) return rc;
  tb_prof_mark(ctx, 0, 1, s);
  a.nparts_in = np;
  DevLoop loop;
  if ((rc = tb_loop_begin(ctx, s, &loop))) return rc;
  if (loop.graph) {
    a.cond = 1;
    a.loop = loop.handle;
    for (int u = 0; u < kLoopUnroll && !rc; ++u) {
      const int p = (u + 1) & 1;
      a.kpar = p;
      a.parts_in = slot[p];
      a.parts_out = slot[p ^ 1];
      rc = launch(a, p, loop.body_stream);
    }
    return tb_loop_end(ctx, &loop, rc);
  }
  a.kc = nullptr;
  for (int k = 1; k <= a.max_iter; ++k) {
    a.k = k;
    a.parts_in = slot[k & 1];
    a.parts_out = slot[(k + 1) & 1];
    if ((rc = launch(a, k, s))) return rc;
    tb_prof_mark(ctx, 0, k + 1, s);
  }
  return TB_OK;
}

extern "C" int dm_sp2_workspace_size(int n, const tb_sp2_opts* o, size_t* bytes) {
  if (!o || !bytes || n < 1) return TB_ERR_ARG;
  if (o->precision < TB_PREC_FP64 || o->precision > TB_PREC_BF16X3) return TB_ERR_ARG;
  if (o->tau > 0.0) return dm_sp2_bsr_workspace(n, o, 0, bytes);
  *bytes = make_layout(n, o->precision, o->refine_iters, o->refine_mode).total;
  return TB_OK;
}

extern "C" int dm_sp2(tb_ctx* ctx, const double* H, int n, double nocc, const tb_sp2_opts* o,
                      double* D, void* ws, size_t ws_bytes, tb_sp2_report* rep, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !D || !o || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_sp2");
  if (n < 1) return tb_fail(ctx, TB_ERR_ARG, "n = %d", n);
  if (o->precision < TB_PREC_FP64 || o->precision > TB_PREC_BF16X3)
    return tb_fail(ctx, TB_ERR_ARG, "unknown precision %d", o->precision);
  if (o->max_iter < 1 || o->max_iter > SP2_MAX_ITER)
    return tb_fail(ctx, TB_ERR_ARG, "max_iter %d outside 1..%d", o->max_iter, SP2_MAX_ITER);
  if (o->refine_iters < 0 || o->refine_iters > SP2_MAX_REFINE)
    return tb_fail(ctx, TB_ERR_ARG, "refine_iters %d outside 0..%d", o->refine_iters, SP2_MAX_REFINE);
  if (!(nocc >= 0.0) || nocc > n) return tb_fail(ctx, TB_ERR_ARG, "n_occ %g outside [0, n]", nocc);
  const bool tc = o->precision != TB_PREC_FP64;
  const int refine = tc ? o->refine_iters : 0;
  if (o->tau < 0.0) return tb_fail(ctx, TB_ERR_ARG, "tau %g < 0", o->tau);
  if (o->tau > 0.0) {
    if (!tc) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse SP2 (tau > 0) needs a tensor-core precision");
    if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0)
      return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
    return dm_sp2_bsr(ctx, H, n, nocc, o, D, ws, ws_bytes, rep, as_stream(stream));
  }
  if (o->refine_mode < 0 || o->refine_mode > 1)
    return tb_fail(ctx, TB_ERR_ARG, "refine_mode %d outside 0..1", o->refine_mode);
  const Layout L = make_layout(n, o->precision, refine, o->refine_mode);
  if (ws_bytes < L.total)
    return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu", ws_bytes, L.total);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0)
    return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  char* base = static_cast<char*>(ws);
  SP2State* st = reinterpret_cast<SP2State*>(base + L.off_state);
  double* bparts = reinterpret_cast<double*>(base + L.off_bparts);
  double* parts = reinterpret_cast<double*>(base + L.off_parts);
  double* slot[2] = {parts, parts + 3 * (size_t)L.max_parts};
  double* F0 = L.off_f0 ? reinterpret_cast<double*>(base + L.off_f0) : nullptr;
  double* F1 = L.off_f1 ? reinterpret_cast<double*>(base + L.off_f1) : nullptr;
  if (!tc) {
    F0 = reinterpret_cast<double*>(base + L.off_f0);
    F1 = reinterpret_cast<double*>(base + L.off_f1);
  }
  float* M[2] = {nullptr, nullptr};
  void* Hi[2] = {nullptr, nullptr};
  void* Lo[2] = {nullptr, nullptr};
  if (tc) {
    M[0] = reinterpret_cast<float*>(base + L.off_m0);
    M[1] = reinterpret_cast<float*>(base + L.off_m1);
    Hi[0] = base + L.off_h0;
    Hi[1] = base + L.off_h1;
    if (L.off_l0) {
      Lo[0] = base + L.off_l0;
      Lo[1] = base + L.off_l1;
    }
  }
  const int ld = L.ld;

  TB_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(SP2State), s));
  const int nb = (n + 7) / 8;
  k_bounds<<<nb, 256, 0, s>>>(H, n, bparts);
  TB_LAUNCH_CHECK(ctx);
  const dim3 g_init(ld / kInitTile, ld / kInitTile);
  const int np_init = g_init.x * g_init.y;
  k_init_x<<<g_init, 256, 0, s>>>(H, n, ld, bparts, nb, st, tc ? nullptr : F0, tc ? M[0] : nullptr,
                                  slot[0]);
  TB_LAUNCH_CHECK(ctx);

  SP2StepArgs a{};
  a.n = n;
  a.ld = ld;
  a.nocc = nocc;
  a.rule = o->rule;
  a.st = st;
  a.wait_ns = ctx->wait_ns;
  if (!tc) {
    a.tol = o->tol;
    a.max_iter = o->max_iter;
    a.phase = 0;
    const dim3 g(ld / f64_tile(ld), ld / f64_tile(ld));
    const int npf = (int)(g.x * g.y);
    const int rc = main_phase(ctx, a, np_init, npf, slot, s, [&](const SP2StepArgs& b, int k, cudaStream_t q) {
      launch_f64(g, b, (k & 1) ? F1 : F0, (k & 1) ? F0 : F1, q);
      TB_LAUNCH_CHECK(ctx);
      return TB_OK;
    });
    if (rc) return rc;
    const int fb = std::min(1184, (int)(((size_t)n * n + 255) / 256));
    k_finalize<<<fb, 256, 0, s>>>(st, n, ld, 0, F0, F1, nullptr, nullptr, D, nocc, rep);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  }

  // tensor-core main phase: split X0 into operands, then projections
  CUtensorMap mh[2], ml[2];
  for (int b = 0; b < 2; ++b) {
    int rc = sp2_tc_make_map(ctx, o->precision, Hi[b], ld, &mh[b], sp2_tc_row_bytes());
    if (rc) return rc;
    if (Lo[b]) {
      rc = sp2_tc_make_map(ctx, o->precision, Lo[b], ld, &ml[b], sp2_tc_row_bytes());
      if (rc) return rc;
    } else {
      ml[b] = mh[b];
    }
  }
  a.tol = o->tol;
  a.max_iter = o->max_iter;
  a.phase = 0;
  {
    // relative error of one product: ~2^-24 for hi/lo splits, 2^-11 (tf32),
    // 2^-8 (bf16)
    const double u = (o->precision == TB_PREC_TF32X3 || o->precision == TB_PREC_BF16X3) ? 0x1p-24
                     : o->precision == TB_PREC_TF32 ? 0x1p-11 : 0x1p-8;
    a.floor = 2.0 * n * u;
  }
  // k = -1 converts X0 to operands (the kernel's split-only mode)
  {
    SP2StepArgs c = a;
    c.k = -1;
    c.nparts_in = 0;
    int rc = sp2_tc_step(ctx, o->precision, c, nullptr, nullptr, M[0], M[0], Hi[0], Lo[0], s);
    if (rc) return rc;
  }
  const int ntc = sp2_tc_step_parts(ctx, ld);
  {
    const int rc = main_phase(ctx, a, np_init, ntc, slot, s, [&](const SP2StepArgs& b, int k, cudaStream_t q) {
      const int i = k & 1, j = (k + 1) & 1;
      return sp2_tc_step(ctx, o->precision, b, &mh[i], &ml[i], M[i], M[j], Hi[j], Lo[j], q);
    });
    if (rc) return rc;
  }
  a.kc = nullptr;
  a.cond = 0;
  const int fb = std::min(1184, (int)(((size_t)n * n + 255) / 256));
  if (refine == 0) {
    k_finalize<<<fb, 256, 0, s>>>(st, n, ld, 2, nullptr, nullptr, M[0], M[1], D, nocc, rep);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  }
  // FP64 refinement
  const dim3 gc(ld / kInitTile, ld / kInitTile);
  k_to_f64<<<gc, 256, 0, s>>>(st, M[0], M[1], ld, F0, slot[0]);
  TB_LAUNCH_CHECK(ctx);
  SP2StepArgs r = a;
  r.phase = 1;
  r.max_iter = refine;
  r.tol = o->tol;
  const dim3 g(ld / f64_tile(ld), ld / f64_tile(ld));
  const int np_ref = L.oz ? sp2_oz_num_parts(ctx, ld) : (int)(g.x * g.y);
  tb_prof_mark(ctx, 1, 0, s);
  for (int k = 0; k <= refine; ++k) {
    r.k = k;
    r.nparts_in = k == 0 ? (int)(gc.x * gc.y) : np_ref;
    r.parts_in = slot[k & 1];
    r.parts_out = slot[(k + 1) & 1];
    double* Fin = (k & 1) ? F1 : F0;
    double* Fout = (k & 1) ? F0 : F1;
    if (L.oz && k < refine) {
      int rc = sp2_oz_step(ctx, r, Fin, Fout, base + L.off_slices, reinterpret_cast<int*>(base + L.off_exps), s);
      if (rc) return rc;
    } else {
      // FP64 FMA projection (or, at k = refine, only the final decision)
      launch_f64(g, r, Fin, Fout, s);
      TB_LAUNCH_CHECK(ctx);
    }
    tb_prof_mark(ctx, 1, k + 1, s);
  }
  k_finalize<<<fb, 256, 0, s>>>(st, n, ld, 1, F0, F1, nullptr, nullptr, D, nocc, rep);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// --------------------------------------------------------------------------
// dm_sp2_static: the FP64 SP2 path without any caller workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// density matrix: an MD engine that reserves all device memory up front and
// forbids allocation inside its time step, a plugin running inside a host
// application that owns the CUDA allocator, or code that must not trigger
// the device-wide synchronisation cudaMalloc/cudaFree may cause.  For them
// the scratch of the FP64 path lives in this file-scope device array, sized
// for n <= TB_SP2_STATIC_MAX_N (about 4 MiB, held by every GPU that loads
// the library until the process exits).  The symbol's device address is
// looked up once per device, on the first call made with that device
// current; make that first call before any stream capture.  The address
// stays valid while the device's context lives: a cudaDeviceReset while the
// library is in use invalidates it, as it does every other device pointer.
// All calls share the array: the SP2 state is cleared at the start of every
// call, and calls that overlap on the GPU (other streams, other host threads)
// race.
// --------------------------------------------------------------------------

namespace {
constexpr size_t kStaticScratchBytes = (size_t)4 * 1024 * 1024 + 64 * 1024;
static __device__ __align__(256) unsigned char g_sp2_scratch[kStaticScratchBytes];
constexpr int kMaxDevices = 64;
// device address of the array, per device; atomic, so host threads making a
// first call on the same device at once store the same value without a race
std::atomic<void*> g_sp2_scratch_addr[kMaxDevices] = {};
}  // namespace

extern "C" int dm_sp2_static(tb_ctx* ctx, const double* H, int n, double nocc, const tb_sp2_opts* o,
                             double* D, tb_sp2_report* rep, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!o) return tb_fail(ctx, TB_ERR_ARG, "null options to dm_sp2_static");
  if (o->precision != TB_PREC_FP64)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "dm_sp2_static runs the FP64 path only (precision %d)", o->precision);
  if (n < 1 || n > TB_SP2_STATIC_MAX_N)
    return tb_fail(ctx, TB_ERR_ARG, "dm_sp2_static: n = %d outside 1..%d (its static scratch is sized for %d)", n,
                   TB_SP2_STATIC_MAX_N, TB_SP2_STATIC_MAX_N);
  int dev = 0;
  TB_CUDA_TRY(ctx, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "device %d out of range", dev);
  void* addr = g_sp2_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sp2_scratch);
    if (e != cudaSuccess || !p)
      return tb_fail(ctx, TB_ERR_CUDA, "cudaGetSymbolAddress of the static SP2 scratch failed: %s",
                     cudaGetErrorString(e));
    g_sp2_scratch_addr[dev].store(p, std::memory_order_release);
    addr = p;
  }
  // dm_sp2 wants a 1024-byte aligned workspace: start at the first such
  // address inside the array
  const uintptr_t base = reinterpret_cast<uintptr_t>(addr);
  const uintptr_t aligned = (base + 1023) & ~uintptr_t(1023);
  const size_t avail = kStaticScratchBytes - (size_t)(aligned - base);
  const Layout L = make_layout(n, TB_PREC_FP64, 0);
  if (L.total > avail)
    return tb_fail(ctx, TB_ERR_ARG, "dm_sp2_static: n = %d needs %zu scratch bytes, %zu available", n, L.total,
                   avail);
  return dm_sp2(ctx, H, n, nocc, o, D, reinterpret_cast<void*>(aligned), avail, rep, stream);
}
