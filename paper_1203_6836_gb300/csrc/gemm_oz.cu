// Emulated-FP64 SP2 projection on the tensor cores (row a6, refinement).
//
// The FP64 refinement projections X <- X^2 or 2X - X^2 (Sec. III.B, App. D.2)
// would run on GB300's FP64 units at ~1.2 TFLOP/s.  Instead the product is
// formed exactly from integer slices on the bf16 tensor cores, following the
// error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 2012) in the tensor-core form of Mukunoki et al. (ISC 2020):
//
//   row scaling  x_ij = 2^{e_i} r_ij, |r_ij| < 1/2 (e_i from the row maximum)
//   slicing      r = sum_{s=1..S} d_s 2^{-7s}, d_s integers with |d_s| <= 64,
//                each exact in bf16 (8 significant bits)
//   products     P_st = sum_k d_s(i,k) d_t(j,k): integers with |P| <= K 2^12,
//                exact in the FP32 accumulator for K <= 4096
//   sum          (X X)_ij = 2^{e_i + e_j} sum_{(s,t)} 2^{-7(s+t)} P_st,
//                recombined in int64 fixed point, then rounded once to FP64.
// With S = 6 the slices carry 42 bits of each row-scaled entry (41 below the
// row maximum).  The kept pairs are s + t <= 7 (21 products) and (4, 4): a
// dropped pair weighs <= 2^-56 |d_s d_t| <= 2^-44 of |x_i| |x_j| per term, and
// the dropped off-diagonal pairs (s, t), (t, s) enter with random signs, while
// a dropped diagonal pair (s, s) is always positive and would bias a diagonal
// entry of X X by ~K E[d^2] 2^{-14 s}: (4, 4) is kept for that reason (its
// product is rounded to the fixed point's last place, 2^-49), the first
// dropped one, (5, 5), biases by ~K 2^-62.  22 bf16 products replace one FP64
// GEMM (6-bit slices would need 7 slices and 28 products for the same bounds).

// Kernel layout: one CTA per 128 x 128 tile of the upper triangle (X^2 is
// symmetric; the epilogue also writes each off-diagonal tile transposed,
// one coalesced 32-lane store per column); warp 0 issues TMA loads
// of (slice s, row block m) and (slice t, row block n) tiles, warp 1 issues
// tcgen05.mma into a ring of four TMEM accumulators (512 columns), warps
// 2-9 drain each pair's accumulator into int64 registers (64 columns per
// thread) and finally apply the SP2 branch in FP64 with the trace partials.

#include "common.cuh"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace {

using namespace tcx;

constexpr int kS = 6;          // slices
constexpr int kBeta = 7;       // bits per slice
constexpr int kPairs = kS * (kS + 1) / 2 + 1;  // (s, t) with s + t <= kS + 1, then (4, 4)
constexpr int kTile = 128;
constexpr int kBK = 64;        // bf16 per 128-byte row
constexpr int kTileBytes = kTile * 128;
constexpr int kStages = 6;
constexpr int kStageBytes = 2 * kTileBytes;
constexpr int kSmem = kStages * kStageBytes + 1024;
constexpr int kThreads = 320;
constexpr int kNacc = 4;       // TMEM accumulators of 128 columns

struct SliceMaps {
  CUtensorMap m[kS];
};

__device__ __forceinline__ void pair_of(int p, int* s, int* t) {
  // (1,1..kS), (2,1..kS-1), ..., (kS,1), then (4,4)
  if (p == kPairs - 1) {
    *s = 4;
    *t = 4;
    return;
  }
  int ss = 1, rem = p;
  while (rem >= kS + 1 - ss) {
    rem -= kS + 1 - ss;
    ++ss;
  }
  *s = ss;
  *t = rem + 1;
}

// One warp per row: e_i from the row maximum, then the kS signed 7-bit
// digits of every entry of the row.  r = x 2^{-e} (|r| < 1/2) is scaled
// exactly and rounded once to the integer R = rint(r 2^{7 kS}) (|R| <= 2^41);
// the digits are R's balanced base-128 digits, peeled off from the least
// significant end in int64 arithmetic: d in [-64, 63] for s >= 2 and
// |d_1| <= 64 (2^41 + 2^34 < 64.5 2^35), all exact in bf16.  Four consecutive
// entries per lane per pass.
__global__ void __launch_bounds__(256) k_oz_split(const SP2State* st, const double* __restrict__ X, int ld,
                                                  __nv_bfloat16* __restrict__ slices, int* __restrict__ exps) {
  if (st->rdone || st->err) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= ld) return;
  const double* xr = X + (size_t)row * ld;
  double mx = 0.0;
  for (int j = 4 * lane; j < ld; j += 128) {
    const double2 u = *reinterpret_cast<const double2*>(xr + j);
    const double2 w = *reinterpret_cast<const double2*>(xr + j + 2);
    mx = fmax(mx, fmax(fmax(fabs(u.x), fabs(u.y)), fmax(fabs(w.x), fabs(w.y))));
  }
  mx = warp_max(mx);
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): |x| / 2^{e+1} < 1/2
    e = max(e + 1, -960);  // keeps 2^{42 - e} finite; such rows are below every digit
  }
  if (lane == 0) exps[row] = e;
  const size_t plane = (size_t)ld * ld;
  const double scale = ldexp(1.0, kBeta * kS - e);  // exact power of two
  for (int j = 4 * lane; j < ld; j += 128) {
    const double2 u = *reinterpret_cast<const double2*>(xr + j);
    const double2 w = *reinterpret_cast<const double2*>(xr + j + 2);
    long long R[4] = {__double2ll_rn(u.x * scale), __double2ll_rn(u.y * scale), __double2ll_rn(w.x * scale),
                      __double2ll_rn(w.y * scale)};
    unsigned short dg[kS][4];
#pragma unroll
    for (int s = kS - 1; s >= 1; --s) {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        const long long d = ((R[e4] + 64) & 127) - 64;  // balanced remainder in [-64, 63]
        R[e4] = (R[e4] - d) >> kBeta;                   // exact division by 128
        dg[s][e4] = __bfloat16_as_ushort(__float2bfloat16_rn((float)d));
      }
    }
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) dg[0][e4] = __bfloat16_as_ushort(__float2bfloat16_rn((float)R[e4]));
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      uint2 pk;
      pk.x = (uint32_t)dg[s][0] | ((uint32_t)dg[s][1] << 16);
      pk.y = (uint32_t)dg[s][2] | ((uint32_t)dg[s][3] << 16);
      *reinterpret_cast<uint2*>(slices + s * plane + (size_t)row * ld + j) = pk;
    }
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

__global__ void __launch_bounds__(kThreads, 1)
    k_sp2_step_oz(SP2StepArgs a, const __grid_constant__ SliceMaps maps, const int* __restrict__ exps,
                  const double* __restrict__ Xin, double* __restrict__ Xout) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], tfull[kNacc], tempty[kNacc];
  __shared__ uint32_t tmem_base;
  __shared__ double s_t[3];
  __shared__ int s_dec[3];
  __shared__ volatile int s_abort;
  __shared__ double s_red[8][3];

  SP2State* st = a.st;
  if (st->rdone || st->err) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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
      const int stop = sp2_decide(a, x, y, st->rt1, st->rt2, false, &br, &capped);
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
  if (stop) return;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // X X is symmetric: CTA b computes upper-triangle tile b and also writes it
  // transposed
  int tI, tJ;
  tri_tile(blockIdx.x, a.ld / kTile, &tI, &tJ);
  const int m0 = tI * kTile, n0 = tJ * kTile;
  const bool mirror = tI != tJ;
  const int nk = a.ld / kBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kNacc; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 8);
    }
    s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, kNacc * kTile);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    for (int i = 0; i < kS; ++i) prefetch_map(&maps.m[i]);
    int g = 0, issued = 0;
    for (int p = 0; p < kPairs && !s_abort; ++p) {
      int s, t;
      pair_of(p, &s, &t);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int stg = g % kStages;
        if (g >= kStages && !mbar_wait(&empty[stg], ((g / kStages) - 1) & 1, &s_abort)) break;
        uint8_t* base = smem + stg * kStageBytes;
        mbar_expect_tx(&full[stg], kStageBytes);
        tma_load_2d(base, &maps.m[s - 1], &full[stg], kb * kBK, m0);
        tma_load_2d(base + kTileBytes, &maps.m[t - 1], &full[stg], kb * kBK, n0);
        issued = g + 1;
      }
    }
    if (s_abort) {
      for (int q = (issued > kStages ? issued - kStages : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % kStages], (q / kStages) & 1) && gtime() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    constexpr uint32_t id = idesc(1u);
    int g = 0;
    for (int p = 0; p < kPairs && !s_abort; ++p) {
      const int acc = p % kNacc;
      if (p >= kNacc && !mbar_wait(&tempty[acc], ((p / kNacc) - 1) & 1, &s_abort)) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * kTile;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int stg = g % kStages;
        if (!mbar_wait(&full[stg], (g / kStages) & 1, &s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = smem_u32(smem + stg * kStageBytes);
#pragma unroll
        for (int ks = 0; ks < kBK / 16; ++ks) {
          umma<false>(d, sdesc(base + ks * 32), sdesc(base + kTileBytes + ks * 32), id, (kb | ks) != 0);
        }
        umma_commit(&empty[stg]);
      }
      umma_commit(&tfull[acc]);
      if (!ok) break;
    }
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;          // TMEM lane quarter
    const int h = (warp - 2) >> 2;   // column half
    const int row = 32 * q + lane;
    long long acc64[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) acc64[j] = 0;
    bool ok = true;
    for (int p = 0; p < kPairs && ok; ++p) {
      int s, t;
      pair_of(p, &s, &t);
      const int acc = p % kNacc;
      if (!mbar_wait_warp(&tfull[acc], (p / kNacc) & 1, &s_abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // fixed point 2^{-kBeta (kS + 1)}: P_st << 7 (7 - s - t); (4, 4) lies one
      // place below it and is scaled by 2^-7 in FP32 (exact) and rounded to
      // the nearest integer; every other P_st converts exactly
      const int shift = kBeta * (kS + 1 - s - t);
      const int lsh = shift > 0 ? shift : 0;
      const float fs = shift >= 0 ? 1.0f : 1.0f / (float)(1 << -shift);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        uint32_t v[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(32 * q) << 16) + acc * kTile + 64 * h + 16 * c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc64[16 * c + j] += __float2ll_rn(__uint_as_float(v[j]) * fs) << lsh;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc])) : "memory");
    }
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    if (ok) {
      const int gr = m0 + row;
      const int er = exps[gr];
      const double* xin = Xin + (size_t)gr * a.ld + n0 + 64 * h;
      double* xout = Xout + (size_t)gr * a.ld + n0 + 64 * h;
      const int* ec = exps + n0 + 64 * h;
      const double w = mirror ? 2.0 : 1.0;  // the transposed copy counts too
      double u2 = 0.0, u3 = 0.0;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const double cxx = ldexp((double)acc64[j], er + ec[j] - kBeta * (kS + 1));
        const double x = xin[j];
        const double y = br ? 2.0 * x - cxx : cxx;
        xout[j] = y;
        // element (gr, n0 + 64h + j) is also element (n0 + 64h + j, gr): for
        // each j the 32 lanes write 32 consecutive values
        if (mirror) Xout[(size_t)(n0 + 64 * h + j) * a.ld + gr] = y;
        if (gr == n0 + 64 * h + j) t1 += y;
        u2 += y * y;
        u3 += (cxx - x) * (cxx - x);
      }
      t2 = w * u2;
      t3 = w * u3;
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    t3 = warp_sum(t3);
    if (lane == 0) {
      s_red[warp - 2][0] = t1;
      s_red[warp - 2][1] = t2;
      s_red[warp - 2][2] = t3;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 64) {
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < 8; ++w) {
      x += s_red[w][0];
      y += s_red[w][1];
      z += s_red[w][2];
    }
    const int cta = blockIdx.x;
    a.parts_out[3 * cta] = x;
    a.parts_out[3 * cta + 1] = y;
    a.parts_out[3 * cta + 2] = z;
    if (s_abort) atomicExch(&st->err, TB_ERR_TIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    if (s_abort && lane == 0) {
      // every accumulator ring slot got a final commit from the issuer or is
      // idle: wait (bounded) for the last one before freeing TMEM
      for (int b = 0; b < kNacc; ++b) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&tfull[b], 0) && gtime() - t0 < kWaitNs) {
        }
      }
    }
    __syncwarp();
    tmem_dealloc(tmem, kNacc * kTile);
  }
}

// ------------------------------------------------------------------ CTA pairs
// The same product on clusters of two CTAs (ld a multiple of 256).  A work
// unit is a 256 x 128 block (I2, J) of the upper triangle, J >= 2 I2: the
// pair's tcgen05.mma.cta_group::2 (M = 256, N = 128) takes A rows from both
// CTAs (CTA r: row block 2 I2 + r) and B rows 64 per CTA (CTA r: rows
// 128 J + 64 r); CTA r accumulates the 128 x 128 tile (2 I2 + r, J) (none when
// that tile lies below the diagonal: it is the mirror of one above).  The 22
// slice pairs run as 12 batches of one or two pairs that share their A slice
// (s, t..t+1), so a k-slice stage holds one A tile (16 KB) and one or two B
// half tiles (8 KB each) for one or two MMAs: with the pair split, 16.7 KB of
// operands per 128 x 128 x 64 MMA per SM against 32 KB in the single-CTA form.
// TMEM holds two sets of two 128-column accumulators, alternating between
// batches, so the drain of one batch overlaps the next batch's MMAs.  The pair
// protocol (agreed decision, copies completing on the even CTA's barriers,
// multicast commits, final cluster barrier) is that of k_sp2_step_tc2.
constexpr int kBatches = 12;
__constant__ int c_batch_s[kBatches] = {1, 1, 1, 2, 2, 2, 3, 3, 4, 4, 5, 6};
__constant__ int c_batch_t[kBatches] = {1, 3, 5, 1, 3, 5, 1, 3, 1, 3, 1, 1};
__constant__ int c_batch_n[kBatches] = {2, 2, 2, 2, 2, 1, 2, 2, 2, 2, 2, 1};
constexpr int kHalfBytes = 64 * 128;                   // 64-row B tile
constexpr int kStage2 = kTileBytes + 2 * kHalfBytes;   // 32 KB
constexpr int kStages2 = 6;
constexpr int kSmem2 = kStages2 * kStage2 + 1024;
constexpr unsigned long long kSettleNs = 1000000ull;

struct SliceMaps2 {
  CUtensorMap a[kS];  // 128-row boxes
  CUtensorMap b[kS];  // 64-row boxes
};

// Unit u of the 256 x 128 upper-triangle units (row-major over I2, then J from 2 I2).
__device__ __forceinline__ void pair_unit(int u, int nt, int* I2, int* J) {
  int i = 0;
  while (u >= nt - 2 * i) {
    u -= nt - 2 * i;
    ++i;
  }
  *I2 = i;
  *J = 2 * i + u;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    k_sp2_step_oz2(const SP2StepArgs a, const __grid_constant__ SliceMaps2 maps, const int* __restrict__ exps,
                   const double* __restrict__ Xin, double* __restrict__ Xout) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages2], empty[kStages2], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ double s_t[3];
  __shared__ int s_dec[3];
  __shared__ uint32_t s_go;
  __shared__ volatile int s_abort;
  __shared__ double s_red[8][3];

  SP2State* st = a.st;
  const int over = st->rdone || st->err;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();

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
      const int stop = over ? 1 : sp2_decide(a, x, y, st->rt1, st->rt2, false, &br, &capped);
      s_t[0] = x;
      s_t[1] = y;
      s_t[2] = z;
      s_dec[0] = stop;
      s_dec[1] = br;
      s_dec[2] = capped;
    }
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < kStages2; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 16);  // 8 epilogue warps x 2 CTAs
    }
    mbar_init(&mdone, 1);
    s_abort = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (!over && blockIdx.x == 0 && threadIdx.x == 0) {
    st->rt1[a.k] = s_t[0];
    st->rt2[a.k] = s_t[1];
    if (a.k > 0) st->idem_fro = sqrt(s_t[2]);
    if (s_dec[0]) {
      st->riters = a.k;
      st->rcapped = s_dec[2];
      st->rdone = 1;
    } else if (s_dec[1]) {
      st->rbranch |= 1ull << a.k;
    }
  }
  if (threadIdx.x == 0) s_go = (s_dec[0] ? 0u : 1u) | (s_dec[1] ? 2u : 0u);
  cluster_sync();
  if (rank != 0 && threadIdx.x == 0) s_go = ld_cluster_u32(mapa_rank(smem_u32(&s_go), 0));
  cluster_sync();
  if (!(s_go & 1u)) return;
  const int br = (s_go >> 1) & 1;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nt = a.ld / kTile, nt2 = a.ld / (2 * kTile);
  const int U = nt * nt2 - nt2 * (nt2 - 1);  // sum over I2 of (nt - 2 I2)
  const int ncl = gridDim.x >> 1, cl = blockIdx.x >> 1;
  const int nk = a.ld / kBK;
  if (warp == 1) tmem_alloc_pair(&tmem_base, 4 * kTile);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    for (int i = 0; i < kS; ++i) {
      prefetch_map(&maps.a[i]);
      prefetch_map(&maps.b[i]);
    }
    const uint32_t full0 = mapa_rank(smem_u32(&full[0]), 0);
    int g = 0, issued = 0;
    for (int u = cl; u < U && !s_abort; u += ncl) {
      int I2, J;
      pair_unit(u, nt, &I2, &J);
      const int ya = (2 * I2 + (int)rank) * kTile, yb = J * kTile + 64 * (int)rank;
      for (int b = 0; b < kBatches && !s_abort; ++b) {
        const int sa = c_batch_s[b], tb = c_batch_t[b], nb = c_batch_n[b];
        const uint32_t bytes = kTileBytes + nb * kHalfBytes;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int stg = g % kStages2;
          if (g >= kStages2 && !mbar_wait(&empty[stg], ((g / kStages2) - 1) & 1, &s_abort, a.wait_ns ? a.wait_ns : kWaitNs)) break;
          uint8_t* base = smem + stg * kStage2;
          if (rank == 0) mbar_expect_tx(&full[stg], 2 * bytes);
          const uint32_t fb = full0 + 8u * stg;
          tma_load_2d_pair(base, &maps.a[sa - 1], fb, kb * kBK, ya);
          tma_load_2d_pair(base + kTileBytes, &maps.b[tb - 1], fb, kb * kBK, yb);
          if (nb > 1) tma_load_2d_pair(base + kTileBytes + kHalfBytes, &maps.b[tb], fb, kb * kBK, yb);
          issued = g + 1;
        }
      }
    }
    if (s_abort && rank == 0) {
      for (int q = (issued > kStages2 ? issued - kStages2 : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % kStages2], (q / kStages2) & 1) && gtime() - t0 < kSettleNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------------------------------------------------- MMA issuer (even CTA)
    constexpr uint32_t id = idesc(1u, 256, 128);
    const unsigned long long wl = a.wait_ns ? a.wait_ns : kWaitNs;
    int g = 0, gb = 0;
    for (int u = cl; u < U && !s_abort; u += ncl) {
      for (int b = 0; b < kBatches && !s_abort; ++b, ++gb) {
        const int nb = c_batch_n[b];
        const int set = gb & 1;
        if (gb >= 2 && !mbar_wait(&tempty[set], ((gb >> 1) - 1) & 1, &s_abort, wl)) break;
        tc_fence_after();
        const uint32_t d0 = tmem + 2 * set * kTile;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int stg = g % kStages2;
          if (!mbar_wait(&full[stg], (g / kStages2) & 1, &s_abort, wl)) break;
          tc_fence_after();
          const uint32_t base = smem_u32(smem + stg * kStage2);
#pragma unroll
          for (int ks = 0; ks < kBK / 16; ++ks) {
            const uint64_t ad = sdesc(base + ks * 32);
            umma_pair<false>(d0, ad, sdesc(base + kTileBytes + ks * 32), id, (kb | ks) != 0);
            if (nb > 1) umma_pair<false>(d0 + kTile, ad, sdesc(base + kTileBytes + kHalfBytes + ks * 32), id, (kb | ks) != 0);
          }
          umma_commit_pair(&empty[stg], 3);
        }
        umma_commit_pair(&tfull[set], 3);
      }
    }
    umma_commit_pair(&mdone, 3);
  } else if (warp >= 2) {
    // ---------------------------------------------------------- epilogue (both CTAs)
    const int q = warp & 3;          // TMEM lane quarter
    const int h = (warp - 2) >> 2;   // column half
    const int row = 32 * q + lane;
    const uint32_t tempty0 = mapa_rank(smem_u32(&tempty[0]), 0);
    const unsigned long long wl = a.wait_ns ? a.wait_ns : kWaitNs;
    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
    bool ok = true;
    int gb = 0;
    for (int u = cl; u < U && ok; u += ncl) {
      int I2, J;
      pair_unit(u, nt, &I2, &J);
      const int I = 2 * I2 + (int)rank;
      long long acc64[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) acc64[j] = 0;
      for (int b = 0; b < kBatches; ++b, ++gb) {
        const int set = gb & 1;
        if (!mbar_wait_warp(&tfull[set], (gb >> 1) & 1, &s_abort, wl)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int p = 0; p < c_batch_n[b]; ++p) {
          const int s = c_batch_s[b], t = c_batch_t[b] + p;
          // fixed point 2^{-kBeta (kS + 1)} as in the single-CTA form
          const int shift = kBeta * (kS + 1 - s - t);
          const int lsh = shift > 0 ? shift : 0;
          const float fs = shift >= 0 ? 1.0f : 1.0f / (float)(1 << -shift);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(32 * q) << 16) + (2 * set + p) * kTile + 64 * h + 16 * c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc64[16 * c + j] += __float2ll_rn(__uint_as_float(v[j]) * fs) << lsh;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(tempty0 + 8u * set);
      }
      if (!ok || I > J) continue;  // below the diagonal: written as the mirror of (J, I)
      const bool mirror = I != J;
      const int m0 = I * kTile, n0 = J * kTile;
      const int gr = m0 + row;
      const int er = exps[gr];
      const double* xin = Xin + (size_t)gr * a.ld + n0 + 64 * h;
      double* xout = Xout + (size_t)gr * a.ld + n0 + 64 * h;
      const int* ec = exps + n0 + 64 * h;
      const double w = mirror ? 2.0 : 1.0;  // the transposed copy counts too
      double u2 = 0.0, u3 = 0.0;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const double cxx = ldexp((double)acc64[j], er + ec[j] - kBeta * (kS + 1));
        const double x = xin[j];
        const double y = br ? 2.0 * x - cxx : cxx;
        xout[j] = y;
        if (mirror) Xout[(size_t)(n0 + 64 * h + j) * a.ld + gr] = y;
        if (gr == n0 + 64 * h + j) t1 += y;
        u2 += y * y;
        u3 += (cxx - x) * (cxx - x);
      }
      t2 += w * u2;
      t3 += w * u3;
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    t3 = warp_sum(t3);
    if (lane == 0) {
      s_red[warp - 2][0] = t1;
      s_red[warp - 2][1] = t2;
      s_red[warp - 2][2] = t3;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 64) {
    double x = 0, y = 0, z = 0;
    for (int w = 0; w < 8; ++w) {
      x += s_red[w][0];
      y += s_red[w][1];
      z += s_red[w][2];
    }
    const int cta = blockIdx.x;
    a.parts_out[3 * cta] = x;
    a.parts_out[3 * cta + 1] = y;
    a.parts_out[3 * cta + 2] = z;
    if (s_abort) atomicExch(&st->err, TB_ERR_TIMEOUT);
  }
  if (warp == 1 && lane == 0) {
    const unsigned long long t0 = gtime();
    while (!mbar_try(&mdone, 0) && gtime() - t0 < kWaitNs) {
    }
    if (s_abort) {
      const unsigned long long t1 = gtime();
      while (gtime() - t1 < kSettleNs) {
      }
    }
  }
  __syncwarp();
  cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, 4 * kTile);
  }
}

int oz_pair_capacity(tb_ctx* ctx) {
  if (ctx->oz_pair_clusters >= 0) return ctx->oz_pair_clusters;
  int n = 0;
  static unsigned long long attr_done = 0;
  if (tb_smem_attr(ctx, k_sp2_step_oz2, kSmem2, &attr_done) == TB_OK) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * ctx->sm_count);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmem2;
    if (cudaOccupancyMaxActiveClusters(&n, k_sp2_step_oz2, &cfg) != cudaSuccess) n = 0;
  }
  (void)cudaGetLastError();
  ctx->oz_pair_clusters = n;
  return n;
}

// Clusters of the pair form for this ld (0: the single-CTA form).  The pair
// form moves half the operand bytes per MMA at the same tile count per SM, so
// it is taken wherever ld allows unless the single form is forced.
int oz_pairs(tb_ctx* ctx, int ld) {
  if (ld % (2 * kTile) != 0 || ctx->sp2_form == TB_SP2_FORM_SINGLE) return 0;
  int C = oz_pair_capacity(ctx);
  if (ctx->grid_limit > 0) C = std::min(C, ctx->grid_limit / 2);
  const int nt = ld / kTile, nt2 = ld / (2 * kTile);
  const int U = nt * nt2 - nt2 * (nt2 - 1);
  C = std::min(C, U);
  return C > 0 ? C : 0;
}

}  // namespace

int sp2_oz_max_ld() { return 4096; }
int sp2_oz_num_parts(tb_ctx* ctx, int ld) {
  const int p = oz_pairs(ctx, ld);
  if (p > 0) return 2 * p;
  const int nt = ld / kTile;
  return nt * (nt + 1) / 2;
}
size_t sp2_oz_slice_bytes(int ld) { return (size_t)kS * ld * ld * sizeof(__nv_bfloat16); }

int sp2_oz_step(tb_ctx* ctx, const SP2StepArgs& a, const double* Xin, double* Xout, void* slices, int* exps,
                cudaStream_t s) {
  if (a.ld > 4096 || a.ld % kTile) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "emulated FP64 needs ld <= 4096");
  static unsigned long long attr_done = 0;
  if (int rc_attr = tb_smem_attr(ctx, k_sp2_step_oz, kSmem, &attr_done)) return rc_attr;
  k_oz_split<<<(a.ld * 32 + 255) / 256, 256, 0, s>>>(a.st, Xin, a.ld, static_cast<__nv_bfloat16*>(slices), exps);
  TB_LAUNCH_CHECK(ctx);
  const size_t plane = (size_t)a.ld * a.ld * sizeof(__nv_bfloat16);
  const int pairs = oz_pairs(ctx, a.ld);
  if (pairs > 0) {
    static unsigned long long attr2_done = 0;
    if (int rc_attr = tb_smem_attr(ctx, k_sp2_step_oz2, kSmem2, &attr2_done)) return rc_attr;
    SliceMaps2 m2;
    for (int i = 0; i < kS; ++i) {
      int rc = sp2_tc_make_map(ctx, TB_PREC_BF16, static_cast<char*>(slices) + i * plane, a.ld, &m2.a[i], 128, 128);
      if (rc) return rc;
      rc = sp2_tc_make_map(ctx, TB_PREC_BF16, static_cast<char*>(slices) + i * plane, a.ld, &m2.b[i], 128, 64);
      if (rc) return rc;
    }
    k_sp2_step_oz2<<<2 * pairs, kThreads, kSmem2, s>>>(a, m2, exps, Xin, Xout);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  }
  SliceMaps maps;
  for (int i = 0; i < kS; ++i) {
    int rc = sp2_tc_make_map(ctx, TB_PREC_BF16, static_cast<char*>(slices) + i * plane, a.ld, &maps.m[i]);
    if (rc) return rc;
  }
  const int nt = a.ld / kTile;
  k_sp2_step_oz<<<nt * (nt + 1) / 2, kThreads, kSmem, s>>>(a, maps, exps, Xin, Xout);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
