// Tensor-core SP2 projection (row a4): X_{k+1} = X_k^2 or 2 X_k - X_k^2
// (Sec. III.B) as a tcgen05 GEMM on sm_103a.
//
// X_k is symmetric and so is X_k^2: only the nt(nt+1)/2 tiles (I <= J) of
// the upper triangle are computed, and the epilogue writes every
// off-diagonal tile twice, as (I, J) and transposed as (J, I).  Both
// operands are row blocks of X read K-major.  The grid is persistent (at
// most one CTA per SM); CTA b takes tiles b, b + G, b + 2G, ... of the
// row-major upper triangle.  Warp roles (192 threads):
//   warp 0   one thread issues TMA tile loads (128-byte swizzled K-slices)
//            into a ring of shared-memory stages that runs on across tiles,
//            completion tracked by mbarriers;
//   warp 1   allocates two TMEM accumulators (2 x 128 FP32 columns) and one
//            thread issues tcgen05.mma (kind::f16 with bf16 or kind::tf32)
//            into them alternately, so the next tile's MMAs overlap the
//            epilogue of the previous one;
//   warps 2-5 epilogue: tcgen05.ld the accumulator, apply the SP2 branch
//            using the FP32 master of X_k, write the FP32 master and the
//            operand splits of X_{k+1} (the transposed copy with one
//            coalesced 32-lane store per column), and accumulate the FP64
//            trace partials (Tr X, ||X||_F^2) per CTA; the X^2 branch reads
//            no FP32 master of X_k.
// Split precisions (x3) keep X ~ hi + lo in two operand arrays and
// accumulate hi*hi + hi*lo + lo*hi in the same FP32 accumulator.
//
// Every mbarrier wait gives up after 2 s of %globaltimer time, records
// TB_ERR_TIMEOUT in the SP2 state and unwinds (waiting, bounded, for its own
// copies and MMAs, then freeing TMEM) instead of hanging.

#include "common.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

namespace {

using namespace tcx;

constexpr int BM = 128, BN = 128;
constexpr int kThreads = 192;

// Shared-memory pipeline of the projection and Fermi-product kernels: each
// stage holds a K-slice of `row` bytes (one swizzle row: 32 tf32 or 64 bf16
// values at 128 bytes) of the A and B row blocks (and their lo splits), in
// 192 KB: three 64 KB stages for the split precisions.  (64-byte slices fit
// six stages but measured 18% slower per projection at n = 4096: twice the
// TMA requests of half a cache line each.)
// Shared-memory descriptor of a K-major tile with `row`-byte swizzle rows.
template <int ROW>
__device__ __forceinline__ uint64_t Pipe_sdesc(uint32_t saddr) {
  if constexpr (ROW == 64) return sdesc64(saddr);
  else return sdesc(saddr);
}

template <int P>
struct Pipe {
  using C = Prec<P>;
  static constexpr int row = 128;                       // bytes of one K-slice row
  static constexpr int bk = row / C::eb;                // K elements per stage
  static constexpr int tile = 128 * row;                // one 128-row tile
  static constexpr int stage_bytes = 2 * C::nop * tile;
  static constexpr int stages = (192 * 1024) / stage_bytes;
  static constexpr int smem_bytes = stages * stage_bytes + 1024;
};


// X0 (FP32 master) -> operand arrays, elementwise.
template <int P>
__global__ void __launch_bounds__(256) k_split(const float* __restrict__ X, int ld, void* hi, void* lo) {
  const size_t segs = (size_t)ld * ld / 32;
  for (size_t sidx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < segs;
       sidx += (size_t)gridDim.x * blockDim.x) {
    float y[32];
    const float4* src = reinterpret_cast<const float4*>(X + sidx * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = src[j];
      y[4 * j] = v.x;
      y[4 * j + 1] = v.y;
      y[4 * j + 2] = v.z;
      y[4 * j + 3] = v.w;
    }
    char* h = static_cast<char*>(hi) + sidx * 32 * Prec<P>::eb;
    char* l = lo ? static_cast<char*>(lo) + sidx * 32 * Prec<P>::eb : h;
    store_operands<P>(y, h, l);
  }
}

// Row-major upper-triangle tile t -> (I, J), I <= J, of an nt x nt tiling.
__device__ __forceinline__ void tri_tile(int t, int nt, int* I, int* J) {
  int i = 0;
  while (t >= nt - i) {
    t -= nt - i;
    ++i;
  }
  *I = i;
  *J = i + t;
}

// Work units of a persistent grid of G CTAs over T tiles: the tiles that
// would leave the last round less than half full are split into two
// 64-column halves, so that round is nearly full (T = 528 on 152 CTAs: three
// rounds of tiles, then 144 halves instead of 72 tiles).
struct Units {
  int T, full, U;  // tiles, units before the halves, all units
};
__device__ __forceinline__ Units make_units(int T, int G) {
  const int F = T / G, rem = T - F * G;
  const bool split = rem > 0 && 2 * rem <= G;
  return Units{T, split ? F * G : T, split ? F * G + 2 * rem : T};
}
// Unit u -> tile t and half (-1: the whole 128-column tile).
__device__ __forceinline__ void unit_tile(const Units& w, int u, int* t, int* half) {
  if (u < w.full) {
    *t = u;
    *half = -1;
  } else {
    *t = w.full + ((u - w.full) >> 1);
    *half = (u - w.full) & 1;
  }
}

// Epilogue of one output tile of a projection: rows m0 + [0, 128) (this
// thread: row m0 + row, TMEM lane row), columns n0 + [0, 32 nchunk) read from
// TMEM at `tcol` (lane offset included).  Applies the branch (X^2, or
// 2X - X^2 from the FP32 master of X_k), writes the FP32 master and operand
// splits of X_{k+1} (and, when `mirror`, the transposed copy with one
// coalesced 32-lane store per column), and adds Tr X_{k+1} (diagonal
// elements) and ||X_{k+1}||_F^2 (twice for a mirrored tile) to t1, t2.
template <int P>
__device__ __forceinline__ void sp2_epi_tile(const SP2StepArgs& a, int br, uint32_t tcol, int row, int m0, int n0,
                                             int nchunk, bool mirror, const float* __restrict__ Xin,
                                             float* __restrict__ Xout, void* __restrict__ ohi,
                                             void* __restrict__ olo, double& t1, double& t2) {
  using C = Prec<P>;
  const double w = mirror ? 2.0 : 1.0;  // the transposed copy counts too
  const size_t gr = (size_t)(m0 + row);
  const float* xin = Xin + gr * a.ld + n0;
  float* xout = Xout + gr * a.ld + n0;
  char* hrow = static_cast<char*>(ohi) + (gr * a.ld + n0) * C::eb;
  char* lrow = olo ? static_cast<char*>(olo) + (gr * a.ld + n0) * C::eb : hrow;
  // (the X^2 branch needs no X_k: its FP32 master is read only for 2X - X^2;
  // ||X^2 - X||_F is left to the FP64 refinement, which reports it)
  double u2 = 0.0;
#pragma unroll 1
  for (int c = 0; c < nchunk; ++c) {
    uint32_t v[32];
    tmem_ld32(tcol + 32 * c, v);
    float y[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) y[j] = __uint_as_float(v[j]);
    if (br) {
      const float4* xi = reinterpret_cast<const float4*>(xin + 32 * c);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 x4 = xi[j];
        y[4 * j] = fmaf(2.0f, x4.x, -y[4 * j]);
        y[4 * j + 1] = fmaf(2.0f, x4.y, -y[4 * j + 1]);
        y[4 * j + 2] = fmaf(2.0f, x4.z, -y[4 * j + 2]);
        y[4 * j + 3] = fmaf(2.0f, x4.w, -y[4 * j + 3]);
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) u2 = fma((double)y[j], (double)y[j], u2);
    if (!mirror) {
      // diagonal tile (or one of its halves): element j is on the diagonal
      // when m0 + row == n0 + 32c + j
      const int dc = m0 + row - n0 - 32 * c;
      if (dc >= 0 && dc < 32) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j == dc) t1 += (double)y[j];
      }
    }
    float4* xo = reinterpret_cast<float4*>(xout + 32 * c);
#pragma unroll
    for (int j = 0; j < 8; ++j) xo[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
    store_operands<P>(y, hrow + 32 * c * C::eb, lrow + 32 * c * C::eb);
    if (mirror) {
      // element (row, 32c + j) of tile (I, J) is element (32c + j, row) of
      // tile (J, I): for each j the 32 lanes write 32 consecutive values
      const size_t col0 = (size_t)n0 + 32 * c;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const size_t idx = (col0 + j) * a.ld + m0 + row;
        Xout[idx] = y[j];
        store_operand1<P>(y[j], ohi, olo ? olo : ohi, idx);
      }
    }
  }
  t2 += w * u2;
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    k_sp2_step_tc(const SP2StepArgs a_in, const __grid_constant__ CUtensorMap mh,
                  const __grid_constant__ CUtensorMap ml, const float* __restrict__ Xin,
                  float* __restrict__ Xout, void* __restrict__ ohi, void* __restrict__ olo) {
  using C = Prec<P>;
  using Q = Pipe<P>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[Q::stages], empty[Q::stages], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ double s_t[3];
  __shared__ int s_dec[3];
  __shared__ volatile int s_abort;
  __shared__ double s_red[4][3];

  SP2State* st = a_in.st;
  SP2StepArgs a = a_in;
  a.k = sp2_step_index(a_in, st->done || st->err);
  if (st->done || st->err) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // ---- decision for projection k from the partials of X_k (same in every CTA)
  if (warp == 0) {
    double x = 0, y = 0, z = 0;
    for (int i = lane; i < a.nparts_in; i += 32) {
      x += a.parts_in[3 * i];
      y += a.parts_in[3 * i + 1];
      z += a.parts_in[3 * i + 2];
    }
    x = warp_sum(x);
    y = warp_sum(y);
    z = warp_sum(z);
    if (lane == 0) {
      int br = 0, capped = 0;
      const int stop = sp2_decide(a, x, y, st->t1, st->t2, true, &br, &capped);
      s_t[0] = x;
      s_t[1] = y;
      s_t[2] = z;
      s_dec[0] = stop;
      s_dec[1] = br;
      s_dec[2] = capped;
    }
  }
  __syncthreads();
  const int stop = s_dec[0], br = s_dec[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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
  }
  if (stop) return;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt = a.ld / BM;
  const Units wu = make_units(nt * (nt + 1) / 2, gridDim.x);
  const unsigned long long wl = a.wait_ns ? a.wait_ns : kWaitNs;  // pipeline wait limit
  const int nk = a.ld / Q::bk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Q::stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&mdone, 1);
    s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_map(&mh);
    if (C::split) prefetch_map(&ml);
    int g = 0, issued = 0;
    for (int u = blockIdx.x; u < wu.U && !s_abort; u += gridDim.x) {
      int t, half, I, J;
      unit_tile(wu, u, &t, &half);
      tri_tile(t, nt, &I, &J);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % Q::stages;
        if (g >= Q::stages && !mbar_wait(&empty[s], ((g / Q::stages) - 1) & 1, &s_abort, wl)) break;
        uint8_t* base = smem + s * Q::stage_bytes;
        mbar_expect_tx(&full[s], Q::stage_bytes);
        tma_load_2d(base, &mh, &full[s], kb * Q::bk, I * BM);
        tma_load_2d(base + Q::tile, &mh, &full[s], kb * Q::bk, J * BN);
        if constexpr (C::split) {
          tma_load_2d(base + 2 * Q::tile, &ml, &full[s], kb * Q::bk, I * BM);
          tma_load_2d(base + 3 * Q::tile, &ml, &full[s], kb * Q::bk, J * BN);
        }
        issued = g + 1;
      }
    }
    if (s_abort) {
      // let every issued copy land before the CTA can exit
      for (int q = (issued > Q::stages ? issued - Q::stages : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % Q::stages], (q / Q::stages) & 1) && gtime() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t id128 = idesc(C::tf32 ? 2u : 1u);
    constexpr uint32_t id64 = idesc(C::tf32 ? 2u : 1u, 128, 64);
    int g = 0, it = 0;
    for (int u = blockIdx.x; u < wu.U && !s_abort; u += gridDim.x, ++it) {
      int t, half;
      unit_tile(wu, u, &t, &half);
      const uint32_t id = half < 0 ? id128 : id64;
      // a half unit multiplies by rows [64 half, 64 half + 64) of the B tile:
      // 64 rows into it, a whole number of 8-row swizzle atoms
      const uint32_t boff = half > 0 ? 64 * Q::row : 0;
      const int buf = it & 1;
      if (it >= 2 && !mbar_wait(&tempty[buf], ((it >> 1) - 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * BN;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % Q::stages;
        if (!mbar_wait(&full[s], (g / Q::stages) & 1, &s_abort, wl)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(smem + s * Q::stage_bytes);
#pragma unroll
        for (int ks = 0; ks < Q::bk / C::uk; ++ks) {
          const uint32_t koff = ks * 32;
          const uint64_t ah = Pipe_sdesc<Q::row>(base + koff);
          const uint64_t bh = Pipe_sdesc<Q::row>(base + Q::tile + boff + koff);
          umma<C::tf32>(d, ah, bh, id, (kb | ks) != 0);
          if constexpr (C::split) {
            umma<C::tf32>(d, ah, Pipe_sdesc<Q::row>(base + 3 * Q::tile + boff + koff), id, 1u);
            umma<C::tf32>(d, Pipe_sdesc<Q::row>(base + 2 * Q::tile + koff), bh, id, 1u);
          }
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&tfull[buf]);
    }
    // arrives once every MMA this thread issued has completed
    umma_commit(&mdone);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int it = 0;
    for (int u = blockIdx.x; u < wu.U; u += gridDim.x, ++it) {
      const int buf = it & 1;
      if (!mbar_wait_warp(&tfull[buf], (it >> 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      int t, half, I, J;
      unit_tile(wu, u, &t, &half);
      tri_tile(t, nt, &I, &J);
      const int m0 = I * BM, n0 = J * BN + (half > 0 ? 64 : 0);
      sp2_epi_tile<P>(a, br, tmem + (static_cast<uint32_t>(32 * q) << 16) + buf * BN, row, m0, n0,
                      half < 0 ? BN / 32 : 2, I != J, Xin, Xout, ohi, olo, t1, t2);
      tc_fence_before();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    t3 = warp_sum(t3);
    if (lane == 0) {
      s_red[q][0] = t1;
      s_red[q][1] = t2;
      s_red[q][2] = t3;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 64) {
    const int cta = blockIdx.x;
    a.parts_out[3 * cta] = s_red[0][0] + s_red[1][0] + s_red[2][0] + s_red[3][0];
    a.parts_out[3 * cta + 1] = s_red[0][1] + s_red[1][1] + s_red[2][1] + s_red[3][1];
    a.parts_out[3 * cta + 2] = s_red[0][2] + s_red[1][2] + s_red[2][2] + s_red[3][2];
    if (s_abort) atomicExch(&st->err, TB_ERR_TIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) {
      // wait (bounded) until every issued MMA has retired before TMEM is freed
      const unsigned long long t0 = gtime();
      while (!mbar_try(&mdone, 0) && gtime() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// CTA-pair form of the projection (ld a multiple of 256): a cluster of two
// CTAs computes one 256 x 256 tile (I2, J2), I2 <= J2, of the upper triangle
// with tcgen05.mma.cta_group::2 (M = N = 256).  CTA r of the pair loads the
// 128-row blocks 2 I2 + r (A) and 2 J2 + r (B) of X into its own shared
// memory; the even CTA's thread issues the MMAs, which read both CTAs'
// stages, and each CTA's epilogue turns its 128 accumulator rows into the
// 128 x 128 tiles (2 I2 + r, 2 J2) and (2 I2 + r, 2 J2 + 1) of X_{k+1}
// (the one below the diagonal of a diagonal 256-tile is left to its
// mirror).  Per SM this halves the operand bytes loaded and read by the
// tensor core per flop against the single-CTA form.  The tail of the
// schedule is split into 256 x 128 halves (N = 128: the even CTA supplies
// B rows [128 h, 128 h + 64) of the half, the odd CTA the next 64) when that
// fills the last round better.
//
// Pair protocol: the odd CTA's TMA copies complete on the even CTA's `full`
// barriers (which expect both CTAs' bytes); the MMA commits arrive on the
// `empty` / `tfull` / `mdone` barriers of both CTAs (multicast); both CTAs'
// epilogue warps arrive on the even CTA's `tempty`.  The stop/branch
// decision of the even CTA is taken by both before anything collective, and
// both CTAs run to the final cluster barrier on every path; all waits are
// bounded as in the single-CTA form.
constexpr int BN2 = 256;
constexpr unsigned long long kSettleNs = 1000000ull;  // 1 ms: copies in flight land well within it

template <int P>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_sp2_step_tc2(const SP2StepArgs a_in, const __grid_constant__ CUtensorMap mh,
                   const __grid_constant__ CUtensorMap ml, const float* __restrict__ Xin,
                   float* __restrict__ Xout, void* __restrict__ ohi, void* __restrict__ olo) {
  using C = Prec<P>;
  using Q = Pipe<P>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[Q::stages], empty[Q::stages], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ double s_t[3];
  __shared__ int s_dec[3];
  __shared__ uint32_t s_go;
  __shared__ volatile int s_abort;
  __shared__ double s_red[4][3];

  SP2State* st = a_in.st;
  SP2StepArgs a = a_in;
  const int over = st->done || st->err;
  a.k = sp2_step_index(a_in, over);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();

  // ---- decision for projection k (same partials in every CTA); no CTA
  // leaves before the pair has agreed on it
  if (warp == 0) {
    double x = 0, y = 0, z = 0;
    if (!over) {
      for (int i = lane; i < a.nparts_in; i += 32) {
        x += a.parts_in[3 * i];
        y += a.parts_in[3 * i + 1];
        z += a.parts_in[3 * i + 2];
      }
      x = warp_sum(x);
      y = warp_sum(y);
      z = warp_sum(z);
    }
    if (lane == 0) {
      int br = 0, capped = 0;
      const int stop = over ? 1 : sp2_decide(a, x, y, st->t1, st->t2, true, &br, &capped);
      s_t[0] = x;
      s_t[1] = y;
      s_t[2] = z;
      s_dec[0] = stop;
      s_dec[1] = br;
      s_dec[2] = capped;
    }
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < Q::stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);  // 4 epilogue warps x 2 CTAs
    }
    mbar_init(&mdone, 1);
    s_abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (!over && blockIdx.x == 0 && threadIdx.x == 0) {
    st->t1[a.k] = s_t[0];
    st->t2[a.k] = s_t[1];
    if (s_dec[0]) {
      st->iters = a.k;
      st->capped = s_dec[2];
      st->done = 1;
      if (a.cond) cudaGraphSetConditional(a.loop, 0);
    } else if (s_dec[1]) {
      st->branch[a.k >> 6] |= 1ull << (a.k & 63);
    }
  }
  if (threadIdx.x == 0) s_go = (s_dec[0] ? 0u : 1u) | (s_dec[1] ? 2u : 0u);
  cluster_sync();  // barrier inits and s_go visible to the peer
  if (rank != 0 && threadIdx.x == 0) s_go = ld_cluster_u32(mapa_rank(smem_u32(&s_go), 0));
  cluster_sync();  // the even CTA's decision read before anyone leaves
  if (!(s_go & 1u)) return;
  const int br = (s_go >> 1) & 1;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt2 = a.ld / BN2;
  const int ncl = gridDim.x >> 1, cl = blockIdx.x >> 1;
  const Units wu = make_units(nt2 * (nt2 + 1) / 2, ncl);
  const unsigned long long wl = a.wait_ns ? a.wait_ns : kWaitNs;  // pipeline wait limit
  const int nk = a.ld / Q::bk;
  if (warp == 1) tmem_alloc_pair(&tmem_base, 2 * BN2);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    prefetch_map(&mh);
    if (C::split) prefetch_map(&ml);
    const uint32_t full0 = mapa_rank(smem_u32(&full[0]), 0);  // the even CTA's barriers
    int g = 0, issued = 0;
    for (int u = cl; u < wu.U && !s_abort; u += ncl) {
      int t, half, I2, J2;
      unit_tile(wu, u, &t, &half);
      tri_tile(t, nt2, &I2, &J2);
      const int ya = (2 * I2 + (int)rank) * BM;
      const int yb = half < 0 ? (2 * J2 + (int)rank) * BM : J2 * BN2 + 128 * half + 64 * (int)rank;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % Q::stages;
        if (g >= Q::stages && !mbar_wait(&empty[s], ((g / Q::stages) - 1) & 1, &s_abort, wl)) break;
        uint8_t* base = smem + s * Q::stage_bytes;
        if (rank == 0) mbar_expect_tx(&full[s], 2 * Q::stage_bytes);
        const uint32_t fb = full0 + 8u * s;
        tma_load_2d_pair(base, &mh, fb, kb * Q::bk, ya);
        tma_load_2d_pair(base + Q::tile, &mh, fb, kb * Q::bk, yb);
        if constexpr (C::split) {
          tma_load_2d_pair(base + 2 * Q::tile, &ml, fb, kb * Q::bk, ya);
          tma_load_2d_pair(base + 3 * Q::tile, &ml, fb, kb * Q::bk, yb);
        }
        issued = g + 1;
      }
    }
    if (s_abort && rank == 0) {
      // let this CTA's copies land before the pair can exit; a stage the odd
      // CTA never filled does not complete, so each wait is cut at kSettleNs
      for (int q = (issued > Q::stages ? issued - Q::stages : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % Q::stages], (q / Q::stages) & 1) && gtime() - t0 < kSettleNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------------------ MMA issuer (even CTA)
    constexpr uint32_t idf = idesc(C::tf32 ? 2u : 1u, 256, 256);
    constexpr uint32_t idh = idesc(C::tf32 ? 2u : 1u, 256, 128);
    int g = 0, it = 0;
    for (int u = cl; u < wu.U && !s_abort; u += ncl, ++it) {
      int t, half;
      unit_tile(wu, u, &t, &half);
      const uint32_t id = half < 0 ? idf : idh;
      const int buf = it & 1;
      if (it >= 2 && !mbar_wait(&tempty[buf], ((it >> 1) - 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * BN2;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int s = g % Q::stages;
        if (!mbar_wait(&full[s], (g / Q::stages) & 1, &s_abort, wl)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(smem + s * Q::stage_bytes);
#pragma unroll
        for (int ks = 0; ks < Q::bk / C::uk; ++ks) {
          const uint32_t koff = ks * 32;
          const uint64_t ah = Pipe_sdesc<Q::row>(base + koff);
          const uint64_t bh = Pipe_sdesc<Q::row>(base + Q::tile + koff);
          umma_pair<C::tf32>(d, ah, bh, id, (kb | ks) != 0);
          if constexpr (C::split) {
            umma_pair<C::tf32>(d, ah, Pipe_sdesc<Q::row>(base + 3 * Q::tile + koff), id, 1u);
            umma_pair<C::tf32>(d, Pipe_sdesc<Q::row>(base + 2 * Q::tile + koff), bh, id, 1u);
          }
        }
        umma_commit_pair(&empty[s], 3);
      }
      umma_commit_pair(&tfull[buf], 3);
    }
    // arrives (in both CTAs) once every MMA of the pair has completed
    umma_commit_pair(&mdone, 3);
  } else if (warp >= 2) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    double t1 = 0.0, t2 = 0.0;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t tempty0 = mapa_rank(smem_u32(&tempty[0]), 0);
    int it = 0;
    for (int u = cl; u < wu.U; u += ncl, ++it) {
      const int buf = it & 1;
      if (!mbar_wait_warp(&tfull[buf], (it >> 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      int t, half, I2, J2;
      unit_tile(wu, u, &t, &half);
      tri_tile(t, nt2, &I2, &J2);
      const int I = 2 * I2 + (int)rank;
      for (int h = 0; h < (half < 0 ? 2 : 1); ++h) {
        const int J = half < 0 ? 2 * J2 + h : 2 * J2 + half;
        if (I > J) continue;  // below the diagonal: written as the mirror of (J, I)
        sp2_epi_tile<P>(a, br, tmem + (static_cast<uint32_t>(32 * q) << 16) + buf * BN2 + (half < 0 ? BM * h : 0),
                        row, I * BM, J * BM, BM / 32, I != J, Xin, Xout, ohi, olo, t1, t2);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(tempty0 + 8u * buf);
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if (lane == 0) {
      s_red[q][0] = t1;
      s_red[q][1] = t2;
      s_red[q][2] = 0.0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 64) {
    const int cta = blockIdx.x;
    a.parts_out[3 * cta] = s_red[0][0] + s_red[1][0] + s_red[2][0] + s_red[3][0];
    a.parts_out[3 * cta + 1] = s_red[0][1] + s_red[1][1] + s_red[2][1] + s_red[3][1];
    a.parts_out[3 * cta + 2] = 0.0;
    if (s_abort) atomicExch(&st->err, TB_ERR_TIMEOUT);
  }
  if (warp == 1 && lane == 0) {
    // every MMA of the pair retired (bounded) before the pair frees its TMEM
    const unsigned long long t0 = gtime();
    while (!mbar_try(&mdone, 0) && gtime() - t0 < kWaitNs) {
    }
    if (s_abort) {
      // an aborted pair may leave copies of the odd CTA in flight that no
      // barrier of its own tracks (their bytes complete on the even CTA's):
      // give them kSettleNs to land
      const unsigned long long t1 = gtime();
      while (gtime() - t1 < kSettleNs) {
      }
    }
  }
  __syncwarp();
  cluster_sync();  // neither CTA leaves while the other may still signal it
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, 2 * BN2);
  }
}

template <int P>
int launch_step(tb_ctx* ctx, const SP2StepArgs& a, const CUtensorMap* mh, const CUtensorMap* ml,
                const float* Xin, float* Xout, void* ohi, void* olo, cudaStream_t s) {
  using C = Prec<P>;
  if (a.k < 0) {
    // split X0 into operand arrays
    k_split<P><<<1184, 256, 0, s>>>(Xin, a.ld, ohi, olo);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  }
  const int pairs = sp2_tc_pairs(ctx, a.ld);
  if (pairs > 0) {
    static unsigned long long attr2_done = 0;
    if (int rc_attr = tb_smem_attr(ctx, k_sp2_step_tc2<P>, Pipe<P>::smem_bytes, &attr2_done)) return rc_attr;
    k_sp2_step_tc2<P><<<2 * pairs, kThreads, Pipe<P>::smem_bytes, s>>>(a, *mh, *ml, Xin, Xout, ohi, olo);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  }
  static unsigned long long attr_done = 0;
  if (int rc_attr = tb_smem_attr(ctx, k_sp2_step_tc<P>, Pipe<P>::smem_bytes, &attr_done)) return rc_attr;
  const int grid = sp2_tc_num_parts(ctx, a.ld);
  k_sp2_step_tc<P><<<grid, kThreads, Pipe<P>::smem_bytes, s>>>(a, *mh, *ml, Xin, Xout, ohi, olo);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// Rounds of a persistent schedule of T units on G CTAs (or clusters), the
// last round counted as half when it runs as 64-column (N = 128) halves.
double sched_rounds(int T, int G) {
  const int F = T / G, rem = T - F * G;
  if (rem == 0) return F;
  return 2 * rem <= G ? F + 0.5 : F + 1.0;
}

// Co-resident clusters of the CTA-pair kernel on this device (queried once).
int pair_capacity(tb_ctx* ctx) {
  if (ctx->pair_clusters >= 0) return ctx->pair_clusters;
  int n = 0;
  static unsigned long long attr_done = 0;
  if (tb_smem_attr(ctx, k_sp2_step_tc2<TB_PREC_TF32X3>, Pipe<TB_PREC_TF32X3>::smem_bytes, &attr_done) == TB_OK) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * ctx->sm_count);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = Pipe<TB_PREC_TF32X3>::smem_bytes;
    if (cudaOccupancyMaxActiveClusters(&n, k_sp2_step_tc2<TB_PREC_TF32X3>, &cfg) != cudaSuccess) n = 0;
  }
  (void)cudaGetLastError();
  ctx->pair_clusters = n;
  return n;
}

}  // namespace

// Per-SM throughput of the pair form relative to the single-CTA form, used
// to choose between them: measured on the 4096 x 4096 tf32x3 projection,
// 0.343 ms for 3.5 rounds of 128-tiles on 152 CTAs against 0.271 ms for 2
// rounds of 256-tiles on 76 pairs (two 128-tiles per SM each).
constexpr double kPairGain = 1.45;

int sp2_tc_pairs(tb_ctx* ctx, int ld) {
  if (ld % BN2 != 0 || ctx->sp2_form == TB_SP2_FORM_SINGLE) return 0;
  int C = pair_capacity(ctx);
  if (ctx->grid_limit > 0) C = std::min(C, ctx->grid_limit / 2);
  const int nt2 = ld / BN2, T2 = nt2 * (nt2 + 1) / 2;
  C = std::min(C, T2);
  if (C < 1) return 0;
  if (ctx->sp2_form == TB_SP2_FORM_PAIRS) return C;
  // automatic: pairs when their schedule, at kPairGain the per-SM rate,
  // finishes before the single-CTA schedule of the 128 x 128 tiles
  const int nt = ld / BM, T1 = nt * (nt + 1) / 2;
  const int G = tb_persistent_grid(ctx, T1);
  const double t_single = sched_rounds(T1, G);             // in 128-tile times
  const double t_pair = 2.0 * sched_rounds(T2, C) / kPairGain;  // a 256-tile is 2 per SM
  return t_pair < t_single ? C : 0;
}

extern "C" int tb_ctx_sp2_form_of(tb_ctx* ctx, int n, int* form, int* ctas) {
  if (!ctx || !form || !ctas) return TB_ERR_ARG;
  if (n < 1) return tb_fail(ctx, TB_ERR_ARG, "n = %d", n);
  const int ld = (n + BM - 1) / BM * BM;
  const int p = sp2_tc_pairs(ctx, ld);
  *form = p > 0 ? TB_SP2_FORM_PAIRS : TB_SP2_FORM_SINGLE;
  *ctas = sp2_tc_step_parts(ctx, ld);
  return TB_OK;
}

int sp2_tc_step_parts(tb_ctx* ctx, int ld) {
  const int p = sp2_tc_pairs(ctx, ld);
  return p > 0 ? 2 * p : sp2_tc_num_parts(ctx, ld);
}

int sp2_tc_tile() { return BM; }
int sp2_tc_num_tiles(int ld) { return (ld / BM) * (ld / BN); }
int sp2_tc_num_parts(const tb_ctx* ctx, int ld) {
  const int nt = ld / BM;
  return tb_persistent_grid(ctx, nt * (nt + 1) / 2);
}
size_t sp2_tc_operand_bytes(int precision) {
  return (precision == TB_PREC_TF32 || precision == TB_PREC_TF32X3) ? 4 : 2;
}

int sp2_tc_row_bytes() { return Pipe<TB_PREC_TF32X3>::row; }

int sp2_tc_make_map(tb_ctx* ctx, int precision, const void* base, int ld, CUtensorMap* map, int row_bytes,
                    int box_rows) {
  if (!ctx->encode_tiled) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
  if (row_bytes != 64 && row_bytes != 128) return tb_fail(ctx, TB_ERR_ARG, "tile row of %d bytes", row_bytes);
  if (box_rows != 64 && box_rows != 128) return tb_fail(ctx, TB_ERR_ARG, "tile of %d rows", box_rows);
  const bool tf = precision == TB_PREC_TF32 || precision == TB_PREC_TF32X3;
  const size_t eb = tf ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ld};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * eb)};
  const cuuint32_t box[2] = {(cuuint32_t)(row_bytes / eb), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode_tiled(map, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                 2, const_cast<void*>(base), dims, strides, box, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return tb_fail(ctx, TB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TB_OK;
}

int sp2_tc_step(tb_ctx* ctx, int precision, const SP2StepArgs& a, const CUtensorMap* mh,
                const CUtensorMap* ml, const float* Xin, float* Xout, void* ohi, void* olo,
                cudaStream_t s) {
  switch (precision) {
    case TB_PREC_TF32: return launch_step<TB_PREC_TF32>(ctx, a, mh, ml, Xin, Xout, ohi, olo, s);
    case TB_PREC_TF32X3: return launch_step<TB_PREC_TF32X3>(ctx, a, mh, ml, Xin, Xout, ohi, olo, s);
    case TB_PREC_BF16: return launch_step<TB_PREC_BF16>(ctx, a, mh, ml, Xin, Xout, ohi, olo, s);
    case TB_PREC_BF16X3: return launch_step<TB_PREC_BF16X3>(ctx, a, mh, ml, Xin, Xout, ohi, olo, s);
    default: return tb_fail(ctx, TB_ERR_ARG, "precision %d has no tensor-core path", precision);
  }
}

// --------------------------------------------------------------------------
// Generic product of two symmetric, mutually commuting matrices (functions of
// the same H) for the Fermi-operator expansion.  With the split precisions a
// square A A also takes the lo*lo term: its diagonal sum_k lo_ik^2 is never
// negative, so dropping it would bias every diagonal element low (by ~2^-22
// of it) and the trace of the expansion by ~1e-7 per orbital, enough to move
// mu within a gap.  Products of different matrices drop lo*lo (their
// rounding residues are uncorrelated).  The product computed is
//   out = alpha * (A B) + beta * E + gamma * I
// with A, B given as tensor-core operand splits (B symmetric, so its rows are
// read K-major), E an optional symmetric FP32 matrix.  A B is then symmetric:
// like the SP2 projection, a persistent grid computes the upper-triangle
// tiles into two alternating TMEM accumulators and writes each off-diagonal
// tile also transposed, so `out` is exactly symmetric.  Writes the FP32
// master and the operand splits of `out` and per-CTA FP64 partials
// (Tr out, ||out||_F^2).  Returns at once when *skip is non-zero
// (device-side early exit of a converged outer iteration).
// --------------------------------------------------------------------------

namespace {

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(GemmArgs g, const __grid_constant__ CUtensorMap ah, const __grid_constant__ CUtensorMap al,
              const __grid_constant__ CUtensorMap bh, const __grid_constant__ CUtensorMap bl) {
  using C = Prec<P>;
  using Q = Pipe<P>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[Q::stages], empty[Q::stages], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ double s_red[4][2];
  if (g.skip && *g.skip) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt = g.ld / BM;
  const int ntiles = nt * (nt + 1) / 2;
  const unsigned long long wl = g.wait_ns ? g.wait_ns : kWaitNs;  // pipeline wait limit
  const int nk = g.ld / Q::bk;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Q::stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&mdone, 1);
    s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (warp == 0 && lane == 0) {
    prefetch_map(&ah);
    prefetch_map(&bh);
    int gk = 0, issued = 0;
    for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x) {
      int I, J;
      tri_tile(t, nt, &I, &J);
      for (int kb = 0; kb < nk; ++kb, ++gk) {
        const int s = gk % Q::stages;
        if (gk >= Q::stages && !mbar_wait(&empty[s], ((gk / Q::stages) - 1) & 1, &s_abort, wl)) break;
        uint8_t* base = smem + s * Q::stage_bytes;
        mbar_expect_tx(&full[s], Q::stage_bytes);
        tma_load_2d(base, &ah, &full[s], kb * Q::bk, I * BM);
        tma_load_2d(base + Q::tile, &bh, &full[s], kb * Q::bk, J * BN);
        if constexpr (C::split) {
          tma_load_2d(base + 2 * Q::tile, &al, &full[s], kb * Q::bk, I * BM);
          tma_load_2d(base + 3 * Q::tile, &bl, &full[s], kb * Q::bk, J * BN);
        }
        issued = gk + 1;
      }
    }
    if (s_abort) {
      for (int q = (issued > Q::stages ? issued - Q::stages : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % Q::stages], (q / Q::stages) & 1) && gtime() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(C::tf32 ? 2u : 1u);
    int gk = 0, it = 0;
    for (int t = blockIdx.x; t < ntiles && !s_abort; t += gridDim.x, ++it) {
      const int buf = it & 1;
      if (it >= 2 && !mbar_wait(&tempty[buf], ((it >> 1) - 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * BN;
      for (int kb = 0; kb < nk; ++kb, ++gk) {
        const int s = gk % Q::stages;
        if (!mbar_wait(&full[s], (gk / Q::stages) & 1, &s_abort, wl)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(smem + s * Q::stage_bytes);
#pragma unroll
        for (int ks = 0; ks < Q::bk / C::uk; ++ks) {
          const uint32_t koff = ks * 32;
          const uint64_t a0 = Pipe_sdesc<Q::row>(base + koff), b0 = Pipe_sdesc<Q::row>(base + Q::tile + koff);
          umma<C::tf32>(d, a0, b0, id, (kb | ks) != 0);
          if constexpr (C::split) {
            const uint64_t a1 = Pipe_sdesc<Q::row>(base + 2 * Q::tile + koff);
            const uint64_t b1 = Pipe_sdesc<Q::row>(base + 3 * Q::tile + koff);
            umma<C::tf32>(d, a0, b1, id, 1u);
            umma<C::tf32>(d, a1, b0, id, 1u);
            if (g.lolo) umma<C::tf32>(d, a1, b1, id, 1u);
          }
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&tfull[buf]);
    }
    // arrives once every MMA this thread issued has completed
    umma_commit(&mdone);
  } else if (warp >= 2) {
    double t1 = 0.0, t2 = 0.0;
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int buf = it & 1;
      if (!mbar_wait_warp(&tfull[buf], (it >> 1) & 1, &s_abort, wl)) break;
      tc_fence_after();
      int I, J;
      tri_tile(t, nt, &I, &J);
      const int m0 = I * BM, n0 = J * BN;
      const bool mirror = I != J;
      const size_t gr = (size_t)(m0 + row);
      const float* erow = g.E ? g.E + gr * g.ld + n0 : nullptr;
      float* orow = g.out + gr * g.ld + n0;
      char* hrow = static_cast<char*>(g.ohi) + (gr * g.ld + n0) * C::eb;
      char* lrow = g.olo ? static_cast<char*>(g.olo) + (gr * g.ld + n0) * C::eb : hrow;
      double u2 = 0.0, u3 = 0.0, lower = 0.0;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + buf * BN + 32 * c, v);
        // E's row segment: eight 16-byte loads instead of 32 scalar ones
        float es[32];
        if (erow) {
          const float4* e4 = reinterpret_cast<const float4*>(erow + 32 * c);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 t = e4[j];
            es[4 * j] = t.x;
            es[4 * j + 1] = t.y;
            es[4 * j + 2] = t.z;
            es[4 * j + 3] = t.w;
          }
        }
        float y[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + 32 * c + j;
          float val = g.alpha * __uint_as_float(v[j]);
          if (erow) val = fmaf(g.beta, es[j], val);
          if (col == (int)gr && (int)gr < g.n) val += g.gamma;
          y[j] = val;
          u2 += (double)val * (double)val;
          if (col < (int)gr) lower += (double)val * (double)val;
          if (col == (int)gr) t1 += (double)val;
        }
        const size_t col0 = (size_t)n0 + 32 * c;
        if (mirror) {
          float4* xo = reinterpret_cast<float4*>(orow + 32 * c);
#pragma unroll
          for (int j = 0; j < 8; ++j) xo[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
          store_operands<P>(y, hrow + 32 * c * C::eb, lrow + 32 * c * C::eb);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const size_t idx = (col0 + j) * g.ld + gr;
            g.out[idx] = y[j];
            store_operand1<P>(y[j], g.ohi, g.olo ? g.olo : g.ohi, idx);
          }
        } else {
          // diagonal tile: its upper triangle (col >= row) is kept and
          // mirrored, so the tile is exactly symmetric too
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const size_t col = col0 + j;
            if (col < gr) continue;
            const size_t idx = gr * g.ld + col, tdx = col * g.ld + gr;
            g.out[idx] = y[j];
            store_operand1<P>(y[j], g.ohi, g.olo ? g.olo : g.ohi, idx);
            if (col > gr) {
              g.out[tdx] = y[j];
              store_operand1<P>(y[j], g.ohi, g.olo ? g.olo : g.ohi, tdx);
              u3 += (double)y[j] * (double)y[j];
            }
          }
        }
      }
      // off-diagonal tiles count twice; in a diagonal tile the kept upper
      // triangle counts twice off the diagonal (u3) and the lower one not at all
      t2 += mirror ? 2.0 * u2 : u2 + u3 - lower;
      tc_fence_before();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if (lane == 0) {
      s_red[q][0] = t1;
      s_red[q][1] = t2;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 64) {
    if (g.parts) {
      const int cta = blockIdx.x;
      g.parts[2 * cta] = s_red[0][0] + s_red[1][0] + s_red[2][0] + s_red[3][0];
      g.parts[2 * cta + 1] = s_red[0][1] + s_red[1][1] + s_red[2][1] + s_red[3][1];
    }
    if (s_abort && g.err) atomicExch(g.err, TB_ERR_TIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) {
      // wait (bounded) until every issued MMA has retired before TMEM is freed
      const unsigned long long t0 = gtime();
      while (!mbar_try(&mdone, 0) && gtime() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
    tmem_dealloc(tmem, 2 * BN);
  }
}

template <int P>
int launch_gemm(tb_ctx* ctx, const GemmArgs& g, const CUtensorMap* ah, const CUtensorMap* al,
                const CUtensorMap* bh, const CUtensorMap* bl, cudaStream_t s) {
  using C = Prec<P>;
  static unsigned long long attr_done = 0;
  if (int rc_attr = tb_smem_attr(ctx, k_gemm_tc<P>, Pipe<P>::smem_bytes, &attr_done)) return rc_attr;
  k_gemm_tc<P><<<sp2_tc_num_parts(ctx, g.ld), kThreads, Pipe<P>::smem_bytes, s>>>(g, *ah, *al, *bh, *bl);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

template <int P>
__global__ void __launch_bounds__(256) k_split_only(const float* __restrict__ X, size_t count, void* hi, void* lo,
                                                    const int* skip) {
  if (skip && *skip) return;
  const size_t segs = count / 32;
  for (size_t sidx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < segs;
       sidx += (size_t)gridDim.x * blockDim.x) {
    float y[32];
    const float4* src = reinterpret_cast<const float4*>(X + sidx * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 v = src[j];
      y[4 * j] = v.x;
      y[4 * j + 1] = v.y;
      y[4 * j + 2] = v.z;
      y[4 * j + 3] = v.w;
    }
    char* h = static_cast<char*>(hi) + sidx * 32 * Prec<P>::eb;
    char* l = lo ? static_cast<char*>(lo) + sidx * 32 * Prec<P>::eb : h;
    store_operands<P>(y, h, l);
  }
}

}  // namespace

int tc_gemm(tb_ctx* ctx, int precision, const GemmArgs& g, const CUtensorMap* ah, const CUtensorMap* al,
            const CUtensorMap* bh, const CUtensorMap* bl, cudaStream_t s) {
  switch (precision) {
    case TB_PREC_TF32: return launch_gemm<TB_PREC_TF32>(ctx, g, ah, al, bh, bl, s);
    case TB_PREC_TF32X3: return launch_gemm<TB_PREC_TF32X3>(ctx, g, ah, al, bh, bl, s);
    case TB_PREC_BF16: return launch_gemm<TB_PREC_BF16>(ctx, g, ah, al, bh, bl, s);
    case TB_PREC_BF16X3: return launch_gemm<TB_PREC_BF16X3>(ctx, g, ah, al, bh, bl, s);
    default: return tb_fail(ctx, TB_ERR_ARG, "precision %d has no tensor-core path", precision);
  }
}

int tc_split(tb_ctx* ctx, int precision, const float* X, size_t count, void* hi, void* lo, const int* skip,
             cudaStream_t s) {
  switch (precision) {
    case TB_PREC_TF32: k_split_only<TB_PREC_TF32><<<1184, 256, 0, s>>>(X, count, hi, lo, skip); break;
    case TB_PREC_TF32X3: k_split_only<TB_PREC_TF32X3><<<1184, 256, 0, s>>>(X, count, hi, lo, skip); break;
    case TB_PREC_BF16: k_split_only<TB_PREC_BF16><<<1184, 256, 0, s>>>(X, count, hi, lo, skip); break;
    case TB_PREC_BF16X3: k_split_only<TB_PREC_BF16X3><<<1184, 256, 0, s>>>(X, count, hi, lo, skip); break;
    default: return tb_fail(ctx, TB_ERR_ARG, "precision %d has no tensor-core path", precision);
  }
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
