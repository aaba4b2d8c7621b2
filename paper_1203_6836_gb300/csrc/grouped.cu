// Many independent SP2 problems in one persistent launch (SP2 of Sec. III.B
// applied to a batch of systems of uneven size).
//
// Each CTA takes whole systems from a device queue (largest first) and runs
// every step of the SP2 recursion for its system without leaving the kernel:
// Gershgorin bounds, X0, then the projections X <- X^2 or 2X - X^2 as tcgen05
// tiles (TMA -> shared memory -> TMEM, warp-specialised as in the dense
// kernel), the FP64 trace reductions and the stop/branch decisions (all in
// the CTA), and finally D.  With square tiles (BN = 128) only the upper
// triangle of the symmetric X^2 is computed and each off-diagonal tile is
// also written transposed.  Between two projections the CTA synchronises and
// fences its global writes for the async proxy, so the next projection's TMA
// loads see them.  All systems' X live in one stacked array (system s owns
// rows [row_off_s, row_off_s + ld_s) and columns [0, ld_s)), so four tensor
// maps per ping-pong buffer cover the batch.
//
// The plan call copies the per-system descriptors to the device once and
// autotunes the launch (tile width BN in {64, 128}, the persistent grid, the
// cluster and FP32-staged forms)
// by timing each candidate on the batch itself; the run call is a memset of
// the queue counter and one kernel launch, so it can be captured into a CUDA
// graph.

#include "common.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <numeric>
#include <vector>

namespace {

using namespace tcx;

constexpr int BM = 128;
constexpr int kThreads = 192;
constexpr int kThreadsFs = 320;  // FP32-staged form: four converter warps more
constexpr int kMaxLd = 512;

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct GDesc {
  const double* H;
  double* D;
  tb_sp2_report* rep;
  int n, ld, row_off, pad;
  double nocc;
};

struct GArgs {
  int count, max_iter, rule, cols;  // cols: stacked width
  double tol_floor_u;               // relative product error u (floor = 2 n u)
  const GDesc* desc;
  int* queue;
  float* M[2];
  void* Hi[2];
  void* Lo[2];
  int* err;
};

template <int P, int BN>
struct GCfg {
  using C = Prec<P>;
  static constexpr int a_bytes = BM * 128;
  static constexpr int b_bytes = BN * 128;
  static constexpr int stage_bytes = (a_bytes + b_bytes) * C::nop;
  static constexpr int stages = (200 * 1024) / stage_bytes;
  static constexpr int smem = stages * stage_bytes + 1024;
};

__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
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

// FS (tf32x3, BN = 128): the FP32-staged form.  TMA loads the FP32 masters
// of X_k only; four converter warps split each stage into hi and lo in shared
// memory, in place (the split is elementwise, so the 128B swizzle is kept),
// and the epilogue writes only the FP32 master of X_{k+1}.  The operands are
// bitwise those of the stored-split form, at half the operand bytes and a
// third of the epilogue's stores.
template <int P, int BN, bool FS>
__global__ void __launch_bounds__(FS ? kThreadsFs : kThreads, 1)
    k_sp2_grouped(GArgs ga, const __grid_constant__ CUtensorMap ah0, const __grid_constant__ CUtensorMap al0,
                  const __grid_constant__ CUtensorMap bh0, const __grid_constant__ CUtensorMap bl0,
                  const __grid_constant__ CUtensorMap ah1, const __grid_constant__ CUtensorMap al1,
                  const __grid_constant__ CUtensorMap bh1, const __grid_constant__ CUtensorMap bl1) {
  using C = Prec<P>;
  using G = GCfg<P, BN>;
  constexpr bool kSym = BN == BM;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[G::stages], empty[G::stages], tfull[2], tempty[2], conv[G::stages];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ int s_sys, s_stop, s_br;
  __shared__ double s_red[kThreadsFs / 32][3];
  __shared__ double s_t1, s_t2, s_lo, s_hi;
  __shared__ double s_hist[2][SP2_MAX_ITER + 2];
  __shared__ unsigned long long s_branch[2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    for (int s = 0; s < G::stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2 * BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  // pipeline counters persist across tiles, projections and systems
  int g_prod = 0, g_mma = 0, t_mma = 0, t_epi = 0, g_conv = 0;
  constexpr int kWarps = (FS ? kThreadsFs : kThreads) / 32;

  while (true) {
    if (threadIdx.x == 0) s_sys = atomicAdd(ga.queue, 1);
    __syncthreads();
    const int sys = s_sys;
    if (sys >= ga.count || s_abort) break;
    const GDesc d = ga.desc[sys];
    const int n = d.n, ld = d.ld, ro = d.row_off;
    // square tiles (BN = BM): only the upper triangle of the symmetric X^2 is
    // computed and mirrored; otherwise every tile
    const int nt_m = ld / BM, nt_n = ld / BN;
    const int ntiles = kSym ? nt_m * (nt_m + 1) / 2 : nt_m * nt_n;
    const int nk = ld / C::bk;

    // ---- Gershgorin bounds (warp per row)
    double lo = INFINITY, hi = -INFINITY;
    for (int r = warp; r < n; r += kWarps) {
      double sabs = 0.0;
      for (int c = lane; c < n; c += 32) sabs += (c == r) ? 0.0 : fabs(d.H[(size_t)r * n + c]);
      sabs = warp_sum(sabs);
      const double hd = d.H[(size_t)r * n + r];
      lo = fmin(lo, hd - sabs);
      hi = fmax(hi, hd + sabs);
    }
    if (lane == 0) {
      s_red[warp][0] = lo;
      s_red[warp][1] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = s_red[0][0], b = s_red[0][1];
      for (int w = 1; w < kWarps; ++w) {
        a = fmin(a, s_red[w][0]);
        b = fmax(b, s_red[w][1]);
      }
      s_lo = a;
      s_hi = b;
      s_branch[0] = s_branch[1] = 0ull;
    }
    __syncthreads();
    // ---- X0 into buffer 0, trace partials
    {
      const double emin = s_lo, emax = s_hi;
      double w = emax - emin;
      if (!(w > 0.0)) w = 1.0;
      const double inv = 1.0 / w;
      const float invf = (float)inv, emaxf = (float)emax;
      double t1 = 0.0, t2 = 0.0;
      for (int seg = threadIdx.x; seg < ld * (ld / 32); seg += kWarps * 32) {
        const int r = seg / (ld / 32), c0 = 32 * (seg % (ld / 32));
        float y[32];
        float s2 = 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + j;
          float x = 0.0f;
          // FP32 arithmetic (one rounding of H): |error| ~ 1e-7 |H| / w, the size
          // of the FP32 rounding of X0 itself
          if (r < n && c < n) x = ((r == c ? emaxf : 0.0f) - (float)d.H[(size_t)r * n + c]) * invf;
          y[j] = x;
          s2 = fmaf(x, x, s2);
          if (r == c) t1 += (double)x;
        }
        t2 += (double)s2;
        const size_t e0 = (size_t)(ro + r) * ga.cols + c0;
        float4* dst = reinterpret_cast<float4*>(ga.M[0] + e0);
#pragma unroll
        for (int j = 0; j < 8; ++j) dst[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
        if constexpr (!FS) {
          char* h = static_cast<char*>(ga.Hi[0]) + e0 * C::eb;
          char* l = ga.Lo[0] ? static_cast<char*>(ga.Lo[0]) + e0 * C::eb : h;
          store_operands<P>(y, h, l);
        }
      }
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      if (lane == 0) {
        s_red[warp][0] = t1;
        s_red[warp][1] = t2;
      }
      fence_async_global();
      __syncthreads();
    }
    const double floor_e = 2.0 * n * ga.tol_floor_u;
    int k = 0;
    for (;; ++k) {
      // ---- decision for projection k (every thread the same)
      if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
          t1 += s_red[w][0];
          t2 += s_red[w][1];
        }
        s_hist[0][k] = t1;
        s_hist[1][k] = t2;
        s_t1 = t1;
        s_t2 = t2;
        const double e = t1 - t2;
        int stop = 0;
        if (e <= floor_e) stop = 1;
        if (!stop && k >= 3) {
          bool flat = e <= 4.0 * floor_e;
          for (int j = 1; j <= 3; ++j) flat = flat && (s_hist[0][k - j] - s_hist[1][k - j] <= 4.0 * floor_e);
          if (flat) stop = 1;
        }
        if (k >= ga.max_iter) stop = 2;
        int br = 0;
        if (!stop) {
          br = ga.rule == 0 ? (fabs(t2 - d.nocc) <= fabs(2.0 * t1 - t2 - d.nocc) ? 0 : 1) : (t1 > d.nocc ? 0 : 1);
          if (br) s_branch[k >> 6] |= 1ull << (k & 63);
        }
        s_stop = stop;
        s_br = br;
      }
      __syncthreads();
      if (s_stop || s_abort) break;
      for (int w = threadIdx.x; w < kWarps; w += kWarps * 32) s_red[w][0] = s_red[w][1] = 0.0;
      const int br = s_br;
      const int ib = k & 1, ob = (k + 1) & 1;
      __syncthreads();
      if (warp == 0 && lane == 0) {
        const CUtensorMap* mah = ib ? &ah1 : &ah0;
        const CUtensorMap* mal = ib ? &al1 : &al0;
        const CUtensorMap* mbh = ib ? &bh1 : &bh0;
        const CUtensorMap* mbl = ib ? &bl1 : &bl0;
        for (int t = 0; t < ntiles && !s_abort; ++t) {
          int m0 = (t / nt_n) * BM, n0 = (t % nt_n) * BN;
          if constexpr (kSym) {
            int I, J;
            tri_tile(t, nt_m, &I, &J);
            m0 = I * BM;
            n0 = J * BN;
          }
          for (int kb = 0; kb < nk; ++kb, ++g_prod) {
            const int s = g_prod % G::stages;
            if (g_prod >= G::stages && !mbar_wait(&empty[s], ((g_prod / G::stages) - 1) & 1, &s_abort)) break;
            uint8_t* base = smem + s * G::stage_bytes;
            // FS: the FP32 masters only, into the hi positions
            mbar_expect_tx(&full[s], FS ? G::a_bytes + G::b_bytes : G::stage_bytes);
            tma_load_2d(base, mah, &full[s], kb * C::bk, ro + m0);
            tma_load_2d(base + G::a_bytes, mbh, &full[s], kb * C::bk, ro + n0);
            if constexpr (C::split && !FS) {
              tma_load_2d(base + G::a_bytes + G::b_bytes, mal, &full[s], kb * C::bk, ro + m0);
              tma_load_2d(base + 2 * G::a_bytes + G::b_bytes, mbl, &full[s], kb * C::bk, ro + n0);
            }
          }
        }
      } else if (warp == 1 && lane == 0) {
        constexpr uint32_t id = idesc(C::tf32 ? 2u : 1u, BM, BN);
        for (int t = 0; t < ntiles && !s_abort; ++t, ++t_mma) {
          const int acc = t_mma & 1;
          if (t_mma >= 2 && !mbar_wait(&tempty[acc], ((t_mma >> 1) - 1) & 1, &s_abort)) break;
          tc_fence_after();
          const uint32_t dt = tmem + acc * BN;
          for (int kb = 0; kb < nk; ++kb, ++g_mma) {
            const int s = g_mma % G::stages;
            if (!mbar_wait(FS ? &conv[s] : &full[s], (g_mma / G::stages) & 1, &s_abort)) break;
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * G::stage_bytes);
#pragma unroll
            for (int ks = 0; ks < C::bk / C::uk; ++ks) {
              const uint32_t koff = ks * 32;
              const uint64_t a0 = sdesc(base + koff), b0 = sdesc(base + G::a_bytes + koff);
              umma<C::tf32>(dt, a0, b0, id, (kb | ks) != 0);
              if constexpr (C::split) {
                const uint64_t a1 = sdesc(base + G::a_bytes + G::b_bytes + koff);
                const uint64_t b1 = sdesc(base + 2 * G::a_bytes + G::b_bytes + koff);
                umma<C::tf32>(dt, a0, b1, id, 1u);
                umma<C::tf32>(dt, a1, b0, id, 1u);
                umma<C::tf32>(dt, a1, b1, id, 1u);  // lo*lo: X X is a square (unbiased diagonal)
              }
            }
            umma_commit(&empty[s]);
          }
          umma_commit(&tfull[acc]);
        }
      } else if (FS && warp >= 6) {
        // converters: each stage's FP32 tiles of A and B (16 KB each, the hi
        // positions) become hi in place and lo at +32 KB, 16 float4 a thread
        const int ct = threadIdx.x - 192;
        for (int t = 0; t < ntiles && !s_abort; ++t) {
          for (int kb = 0; kb < nk; ++kb, ++g_conv) {
            const int s = g_conv % G::stages;
            if (!mbar_wait_warp(&full[s], (g_conv / G::stages) & 1, &s_abort)) break;
            float4* stage = reinterpret_cast<float4*>(smem + s * G::stage_bytes);
            constexpr int kHalf = (G::a_bytes + G::b_bytes) / 16;  // float4 of A and B
#pragma unroll 4
            for (int i = ct; i < kHalf; i += 128) {
              const float4 x = stage[i];
              const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
              stage[i] = h;
              stage[i + kHalf] = make_float4(to_tf32(x.x - h.x), to_tf32(x.y - h.y), to_tf32(x.z - h.z),
                                             to_tf32(x.w - h.w));
            }
            // the generic-proxy stores must be visible to the tensor core's reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&conv[s])) : "memory");
          }
        }
      } else if (warp >= 2) {
        const int q = warp & 3;
        const int row = 32 * q + lane;
        double t1 = 0.0, t2 = 0.0;
        for (int t = 0; t < ntiles; ++t, ++t_epi) {
          const int acc = t_epi & 1;
          if (!mbar_wait_warp(&tfull[acc], (t_epi >> 1) & 1, &s_abort)) break;
          tc_fence_after();
          int m0 = (t / nt_n) * BM, n0 = (t % nt_n) * BN;
          if constexpr (kSym) {
            int I, J;
            tri_tile(t, nt_m, &I, &J);
            m0 = I * BM;
            n0 = J * BN;
          }
          const bool mirror = kSym && m0 != n0;
          const size_t grow = (size_t)(ro + m0 + row);
          double u2 = 0.0;
          const float* xin = ga.M[ib] + grow * ga.cols + n0;
          float* xout = ga.M[ob] + grow * ga.cols + n0;
          char* hrow = static_cast<char*>(ga.Hi[ob]) + (grow * ga.cols + n0) * C::eb;
          char* lrow = ga.Lo[ob] ? static_cast<char*>(ga.Lo[ob]) + (grow * ga.cols + n0) * C::eb : hrow;
#pragma unroll 1
          for (int c = 0; c < BN / 32; ++c) {
            uint32_t v[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + acc * BN + 32 * c, v);
            // X_k's row segment: eight 16-byte loads instead of 32 scalar ones
            float xs[32];
            {
              const float4* x4 = reinterpret_cast<const float4*>(xin + 32 * c);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 t = x4[j];
                xs[4 * j] = t.x;
                xs[4 * j + 1] = t.y;
                xs[4 * j + 2] = t.z;
                xs[4 * j + 3] = t.w;
              }
            }
            float y[32];
            float c2 = 0.0f;  // chunk sum in FP32, accumulated in FP64 (GB300 FP64 is slow)
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float cxx = __uint_as_float(v[j]);
              const float x = xs[j];
              y[j] = br ? fmaf(2.0f, x, -cxx) : cxx;
              c2 = fmaf(y[j], y[j], c2);
              if (m0 + row == n0 + 32 * c + j) t1 += (double)y[j];
            }
            u2 += (double)c2;
            float4* xo = reinterpret_cast<float4*>(xout + 32 * c);
#pragma unroll
            for (int j = 0; j < 8; ++j) xo[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
            if constexpr (!FS) store_operands<P>(y, hrow + 32 * c * C::eb, lrow + 32 * c * C::eb);
            if (mirror) {
              // element (m0 + row, n0 + 32c + j) is also (n0 + 32c + j, m0 + row):
              // for each j the 32 lanes write 32 consecutive values
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const size_t idx = (size_t)(ro + n0 + 32 * c + j) * ga.cols + m0 + row;
                ga.M[ob][idx] = y[j];
                if constexpr (!FS) store_operand1<P>(y[j], ga.Hi[ob], ga.Lo[ob] ? ga.Lo[ob] : ga.Hi[ob], idx);
              }
            }
          }
          t2 += mirror ? 2.0 * u2 : u2;
          tc_fence_before();
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc])) : "memory");
        }
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        if (lane == 0) {
          s_red[warp][0] = t1;
          s_red[warp][1] = t2;
        }
        fence_async_global();
      }
      __syncthreads();
    }
    // ---- D from the final iterate (buffer k % 2), report
    {
      const float* X = ga.M[k & 1];
      for (int r = warp; r < n; r += kWarps)
        for (int c = lane; c < n; c += 32) d.D[(size_t)r * n + c] = (double)X[(size_t)(ro + r) * ga.cols + c];
      if (threadIdx.x == 0 && d.rep) {
        tb_sp2_report* rp = d.rep;
        const double e = s_t1 - s_t2;
        rp->status = s_abort ? TB_ERR_TIMEOUT : (fabs(s_t1 - d.nocc) > 0.25 ? TB_ERR_GAP : TB_OK);
        rp->iters = k;
        rp->refine_iters = 0;
        rp->n = n;
        rp->eps_min = s_lo;
        rp->eps_max = s_hi;
        rp->trace = s_t1;
        rp->idem_trace = e;
        rp->idem_fro = -1.0;
        rp->branch_bits[0] = s_branch[0];
        rp->branch_bits[1] = s_branch[1];
        rp->refine_bits = 0;
        rp->block_products = 0;
        rp->blocks = 0;
      }
      __syncthreads();
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_abort && ga.err) atomicExch(ga.err, TB_ERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    if (s_abort && lane == 0) {
      for (int b = 0; b < 2; ++b) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&tfull[b], 0) && gtime() - t0 < kWaitNs) {
        }
      }
    }
    __syncwarp();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// ---------------------------------------------------------------------------
// Cluster form: a thread-block cluster of CS CTAs (one per SM) runs one system
// at a time.  The CTAs split the rows of the Gershgorin bounds, of X0 and of
// D, and the upper-triangle 128 x 128 tiles of every projection (tile t goes
// to CTA t mod CS); their FP64 partials meet in CTA 0's shared memory
// (distributed shared memory), and a cluster barrier (release/acquire)
// separates the projections, after which every CTA takes the same decision
// from the same partials in the same order.  Fewer systems are in flight at
// once than with one CTA per system, so their working sets stay in L2.
// Every CTA of a cluster passes the same sequence of cluster barriers: the
// decisions are cluster-uniform, and a bounded wait that gives up marks the
// CTA's partials, which stops all of them together.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Generic pointer to the same shared variable in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T* cluster_map(T* p, uint32_t rank) {
  uint64_t in = reinterpret_cast<uint64_t>(p), out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(in), "r"(rank));
  return reinterpret_cast<T*>(out);
}

template <int P, int CS>
__global__ void __launch_bounds__(kThreads, 1)
    k_sp2_grouped_cl(GArgs ga, const __grid_constant__ CUtensorMap ah0, const __grid_constant__ CUtensorMap al0,
                     const __grid_constant__ CUtensorMap ah1, const __grid_constant__ CUtensorMap al1) {
  using C = Prec<P>;
  using G = GCfg<P, BM>;
  constexpr int BN = BM;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[G::stages], empty[G::stages], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ int s_sys;
  __shared__ double s_red[8][3];
  // partials of every CTA, valid in CTA 0: [parity][rank] = (t1, t2, abort)
  __shared__ double s_part[2][CS][3];
  __shared__ double s_bnd[CS][2];
  __shared__ double s_hist[2][SP2_MAX_ITER + 2];
  __shared__ unsigned long long s_branch[2];
  __shared__ double s_t1, s_t2, s_lo, s_hi;
  __shared__ int s_stop, s_br;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    for (int s = 0; s < G::stages; ++s) {
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
  int g_prod = 0, g_mma = 0, t_mma = 0, t_epi = 0;
  double* part0 = cluster_map(&s_part[0][0][0], 0);  // CTA 0's partials
  double* bnd0 = cluster_map(&s_bnd[0][0], 0);
  cluster_sync();  // every CTA of the cluster is running

  bool quit = false;
  while (!quit) {
    if (rank == 0 && threadIdx.x == 0) {
      const int sys = atomicAdd(ga.queue, 1);
      for (int r = 0; r < CS; ++r) *cluster_map(&s_sys, (uint32_t)r) = sys;
    }
    cluster_sync();
    const int sys = s_sys;
    if (sys >= ga.count) break;
    const GDesc d = ga.desc[sys];
    const int n = d.n, ld = d.ld, ro = d.row_off;
    const int nt = ld / BM;
    const int ntiles = nt * (nt + 1) / 2;
    const int nk = ld / C::bk;

    // ---- Gershgorin bounds: rows rank, rank + CS, ... (warp per row)
    {
      double lo = INFINITY, hi = -INFINITY;
      for (int r = (int)rank + CS * warp; r < n; r += CS * (kThreads / 32)) {
        double sabs = 0.0;
        for (int c = lane; c < n; c += 32) sabs += (c == r) ? 0.0 : fabs(d.H[(size_t)r * n + c]);
        sabs = warp_sum(sabs);
        const double hd = d.H[(size_t)r * n + r];
        lo = fmin(lo, hd - sabs);
        hi = fmax(hi, hd + sabs);
      }
      if (lane == 0) {
        s_red[warp][0] = lo;
        s_red[warp][1] = hi;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = s_red[0][0], b = s_red[0][1];
        for (int w = 1; w < kThreads / 32; ++w) {
          a = fmin(a, s_red[w][0]);
          b = fmax(b, s_red[w][1]);
        }
        bnd0[2 * rank] = a;
        bnd0[2 * rank + 1] = b;
      }
      cluster_sync();
      if (threadIdx.x == 0) {
        double a = bnd0[0], b = bnd0[1];
        for (int r = 1; r < CS; ++r) {
          a = fmin(a, bnd0[2 * r]);
          b = fmax(b, bnd0[2 * r + 1]);
        }
        s_lo = a;
        s_hi = b;
        s_branch[0] = s_branch[1] = 0ull;
      }
      __syncthreads();
    }
    // ---- X0 into buffer 0: row segments of 32 split over the cluster
    {
      const double emin = s_lo, emax = s_hi;
      double w = emax - emin;
      if (!(w > 0.0)) w = 1.0;
      const double inv = 1.0 / w;
      const float invf = (float)inv, emaxf = (float)emax;
      double t1 = 0.0, t2 = 0.0;
      const int segs = ld * (ld / 32);
      for (int seg = (int)rank * kThreads + threadIdx.x; seg < segs; seg += CS * kThreads) {
        const int r = seg / (ld / 32), c0 = 32 * (seg % (ld / 32));
        float y[32];
        float s2 = 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = c0 + j;
          float x = 0.0f;
          // FP32 arithmetic (one rounding of H): |error| ~ 1e-7 |H| / w, the size
          // of the FP32 rounding of X0 itself
          if (r < n && c < n) x = ((r == c ? emaxf : 0.0f) - (float)d.H[(size_t)r * n + c]) * invf;
          y[j] = x;
          s2 = fmaf(x, x, s2);
          if (r == c) t1 += (double)x;
        }
        t2 += (double)s2;
        const size_t e0 = (size_t)(ro + r) * ga.cols + c0;
        float4* dst = reinterpret_cast<float4*>(ga.M[0] + e0);
#pragma unroll
        for (int j = 0; j < 8; ++j) dst[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
        char* h = static_cast<char*>(ga.Hi[0]) + e0 * C::eb;
        char* l = ga.Lo[0] ? static_cast<char*>(ga.Lo[0]) + e0 * C::eb : h;
        store_operands<P>(y, h, l);
      }
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      if (lane == 0) {
        s_red[warp][0] = t1;
        s_red[warp][1] = t2;
      }
      fence_async_global();
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w2 = 0; w2 < kThreads / 32; ++w2) {
          a += s_red[w2][0];
          b += s_red[w2][1];
        }
        part0[3 * rank] = a;
        part0[3 * rank + 1] = b;
        part0[3 * rank + 2] = 0.0;
      }
      cluster_sync();
      fence_async_global();
    }
    const double floor_e = 2.0 * n * ga.tol_floor_u;
    int k = 0;
    for (;; ++k) {
      // ---- decision for projection k from the cluster's partials (parity k)
      if (threadIdx.x == 0) {
        const double* pk = part0 + (k & 1) * CS * 3;
        double t1 = 0.0, t2 = 0.0, ab = 0.0;
        for (int r = 0; r < CS; ++r) {
          t1 += pk[3 * r];
          t2 += pk[3 * r + 1];
          ab += pk[3 * r + 2];
        }
        s_hist[0][k] = t1;
        s_hist[1][k] = t2;
        s_t1 = t1;
        s_t2 = t2;
        const double e = t1 - t2;
        int stop = 0;
        if (e <= floor_e) stop = 1;
        if (!stop && k >= 3) {
          bool flat = e <= 4.0 * floor_e;
          for (int j = 1; j <= 3; ++j) flat = flat && (s_hist[0][k - j] - s_hist[1][k - j] <= 4.0 * floor_e);
          if (flat) stop = 1;
        }
        if (k >= ga.max_iter) stop = 2;
        if (ab != 0.0) stop = 3;
        int br = 0;
        if (!stop) {
          br = ga.rule == 0 ? (fabs(t2 - d.nocc) <= fabs(2.0 * t1 - t2 - d.nocc) ? 0 : 1) : (t1 > d.nocc ? 0 : 1);
          if (br) s_branch[k >> 6] |= 1ull << (k & 63);
        }
        s_stop = stop;
        s_br = br;
      }
      __syncthreads();
      if (s_stop) break;
      const int br = s_br;
      const int ib = k & 1, ob = (k + 1) & 1;
      if (warp == 0 && lane == 0) {
        const CUtensorMap* mah = ib ? &ah1 : &ah0;
        const CUtensorMap* mal = ib ? &al1 : &al0;
        for (int t = (int)rank; t < ntiles && !s_abort; t += CS) {
          int I, J;
          tri_tile(t, nt, &I, &J);
          for (int kb = 0; kb < nk; ++kb, ++g_prod) {
            const int s = g_prod % G::stages;
            if (g_prod >= G::stages && !mbar_wait(&empty[s], ((g_prod / G::stages) - 1) & 1, &s_abort)) break;
            uint8_t* base = smem + s * G::stage_bytes;
            mbar_expect_tx(&full[s], G::stage_bytes);
            tma_load_2d(base, mah, &full[s], kb * C::bk, ro + I * BM);
            tma_load_2d(base + G::a_bytes, mah, &full[s], kb * C::bk, ro + J * BN);
            if constexpr (C::split) {
              tma_load_2d(base + G::a_bytes + G::b_bytes, mal, &full[s], kb * C::bk, ro + I * BM);
              tma_load_2d(base + 2 * G::a_bytes + G::b_bytes, mal, &full[s], kb * C::bk, ro + J * BN);
            }
          }
        }
      } else if (warp == 1 && lane == 0) {
        constexpr uint32_t id = idesc(C::tf32 ? 2u : 1u, BM, BN);
        for (int t = (int)rank; t < ntiles && !s_abort; t += CS, ++t_mma) {
          const int acc = t_mma & 1;
          if (t_mma >= 2 && !mbar_wait(&tempty[acc], ((t_mma >> 1) - 1) & 1, &s_abort)) break;
          tc_fence_after();
          const uint32_t dt = tmem + acc * BN;
          for (int kb = 0; kb < nk; ++kb, ++g_mma) {
            const int s = g_mma % G::stages;
            if (!mbar_wait(&full[s], (g_mma / G::stages) & 1, &s_abort)) break;
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * G::stage_bytes);
#pragma unroll
            for (int ks = 0; ks < C::bk / C::uk; ++ks) {
              const uint32_t koff = ks * 32;
              const uint64_t a0 = sdesc(base + koff), b0 = sdesc(base + G::a_bytes + koff);
              umma<C::tf32>(dt, a0, b0, id, (kb | ks) != 0);
              if constexpr (C::split) {
                const uint64_t a1 = sdesc(base + G::a_bytes + G::b_bytes + koff);
                const uint64_t b1 = sdesc(base + 2 * G::a_bytes + G::b_bytes + koff);
                umma<C::tf32>(dt, a0, b1, id, 1u);
                umma<C::tf32>(dt, a1, b0, id, 1u);
                umma<C::tf32>(dt, a1, b1, id, 1u);  // lo*lo: X X is a square (unbiased diagonal)
              }
            }
            umma_commit(&empty[s]);
          }
          umma_commit(&tfull[acc]);
        }
      } else if (warp >= 2) {
        const int q = warp & 3;
        const int row = 32 * q + lane;
        double t1 = 0.0, t2 = 0.0;
        for (int t = (int)rank; t < ntiles; t += CS, ++t_epi) {
          const int acc = t_epi & 1;
          if (!mbar_wait_warp(&tfull[acc], (t_epi >> 1) & 1, &s_abort)) break;
          tc_fence_after();
          int I, J;
          tri_tile(t, nt, &I, &J);
          const int m0 = I * BM, n0 = J * BN;
          const bool mirror = m0 != n0;
          const size_t grow = (size_t)(ro + m0 + row);
          const float* xin = ga.M[ib] + grow * ga.cols + n0;
          float* xout = ga.M[ob] + grow * ga.cols + n0;
          char* hrow = static_cast<char*>(ga.Hi[ob]) + (grow * ga.cols + n0) * C::eb;
          char* lrow = ga.Lo[ob] ? static_cast<char*>(ga.Lo[ob]) + (grow * ga.cols + n0) * C::eb : hrow;
          double u2 = 0.0;
#pragma unroll 1
          for (int c = 0; c < BN / 32; ++c) {
            uint32_t v[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + acc * BN + 32 * c, v);
            // X_k's row segment: eight 16-byte loads instead of 32 scalar ones
            float xs[32];
            {
              const float4* x4 = reinterpret_cast<const float4*>(xin + 32 * c);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float4 t = x4[j];
                xs[4 * j] = t.x;
                xs[4 * j + 1] = t.y;
                xs[4 * j + 2] = t.z;
                xs[4 * j + 3] = t.w;
              }
            }
            float y[32];
            float c2 = 0.0f;  // chunk sum in FP32, accumulated in FP64 (GB300 FP64 is slow)
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float cxx = __uint_as_float(v[j]);
              const float x = xs[j];
              y[j] = br ? fmaf(2.0f, x, -cxx) : cxx;
              c2 = fmaf(y[j], y[j], c2);
              if (m0 + row == n0 + 32 * c + j) t1 += (double)y[j];
            }
            u2 += (double)c2;
            float4* xo = reinterpret_cast<float4*>(xout + 32 * c);
#pragma unroll
            for (int j = 0; j < 8; ++j) xo[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
            store_operands<P>(y, hrow + 32 * c * C::eb, lrow + 32 * c * C::eb);
            if (mirror) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const size_t idx = (size_t)(ro + n0 + 32 * c + j) * ga.cols + m0 + row;
                ga.M[ob][idx] = y[j];
                store_operand1<P>(y[j], ga.Hi[ob], ga.Lo[ob] ? ga.Lo[ob] : ga.Hi[ob], idx);
              }
            }
          }
          t2 += mirror ? 2.0 * u2 : u2;
          tc_fence_before();
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[acc])) : "memory");
        }
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        if (lane == 0) {
          s_red[warp][0] = t1;
          s_red[warp][1] = t2;
        }
        fence_async_global();
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w2 = 2; w2 < kThreads / 32; ++w2) {
          a += s_red[w2][0];
          b += s_red[w2][1];
        }
        double* pn = part0 + ob * CS * 3;
        pn[3 * rank] = a;
        pn[3 * rank + 1] = b;
        pn[3 * rank + 2] = s_abort ? 1.0 : 0.0;
      }
      cluster_sync();
      fence_async_global();
    }
    // ---- D from the final iterate (buffer k % 2): rows split over the cluster
    {
      const float* X = ga.M[k & 1];
      for (int r = (int)rank + CS * warp; r < n; r += CS * (kThreads / 32))
        for (int c = lane; c < n; c += 32) d.D[(size_t)r * n + c] = (double)X[(size_t)(ro + r) * ga.cols + c];
      if (rank == 0 && threadIdx.x == 0 && d.rep) {
        tb_sp2_report* rp = d.rep;
        rp->status = s_stop == 3 ? TB_ERR_TIMEOUT : (fabs(s_t1 - d.nocc) > 0.25 ? TB_ERR_GAP : TB_OK);
        rp->iters = k;
        rp->refine_iters = 0;
        rp->n = n;
        rp->eps_min = s_lo;
        rp->eps_max = s_hi;
        rp->trace = s_t1;
        rp->idem_trace = s_t1 - s_t2;
        rp->idem_fro = -1.0;
        rp->branch_bits[0] = s_branch[0];
        rp->branch_bits[1] = s_branch[1];
        rp->refine_bits = 0;
        rp->block_products = 0;
        rp->blocks = 0;
      }
      if (s_stop == 3) quit = true;  // cluster-uniform: every CTA saw the same partials
    }
    __syncthreads();
  }
  cluster_sync();  // no CTA leaves while another may still address its shared memory
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_abort && ga.err) atomicExch(ga.err, TB_ERR_TIMEOUT);
  if (warp == 1) {
    tc_fence_after();
    if (lane == 0) {
      umma_commit(&mdone);
      const unsigned long long t0 = gtime();
      while (!mbar_try(&mdone, 0) && gtime() - t0 < kWaitNs) {
      }
    }
    __syncwarp();
    tmem_dealloc(tmem, 2 * BN);
  }
}

// Plan header kept at the start of the workspace.
struct Plan {
  int count, precision, rule, max_iter;
  int rows, cols;
  int bn, grid, cs;  // cs > 1: cluster form with cs CTAs per system; bn = 0: the FP32-staged form (tf32x3)
  double u;
  size_t off_desc, off_queue, off_err, off_m[2], off_hi[2], off_lo[2], total;
  CUtensorMap ah[2], al[2], bh[2], bl[2];  // bh/bl for the chosen bn
  CUtensorMap bh64[2], bl64[2], bh128[2], bl128[2];
  CUtensorMap am[2];  // FP32 masters, 128-row boxes (FP32-staged form)
};

static_assert(sizeof(Plan) <= sizeof(((tb_ctx*)nullptr)->plan_cache), "plan cache too small");

size_t layout(int count, const int* n, int prec, Plan* p) {
  int rows = 0, cols = 0;
  for (int i = 0; i < count; ++i) {
    const int ld = round_up(std::max(n[i], 1), BM);
    rows += ld;
    cols = std::max(cols, ld);
  }
  p->rows = rows;
  p->cols = cols;
  size_t o = (sizeof(Plan) + 1023) / 1024 * 1024;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 1023) / 1024 * 1024;
    return r;
  };
  const size_t eb = (prec == TB_PREC_TF32 || prec == TB_PREC_TF32X3) ? 4 : 2;
  const bool split = prec == TB_PREC_TF32X3 || prec == TB_PREC_BF16X3;
  const size_t cells = (size_t)rows * cols;
  p->off_desc = take(sizeof(GDesc) * (size_t)count);
  p->off_queue = take(sizeof(int) * 4);
  p->off_err = take(sizeof(int) * 4);
  for (int b = 0; b < 2; ++b) {
    p->off_m[b] = take(sizeof(float) * cells);
    p->off_hi[b] = take(eb * cells);
    p->off_lo[b] = split ? take(eb * cells) : 0;
  }
  p->total = o;
  return o;
}

int make_map(tb_ctx* ctx, int prec, const void* base, int rows, int cols, int box_rows, CUtensorMap* map) {
  const bool tf = prec == TB_PREC_TF32 || prec == TB_PREC_TF32X3;
  const size_t eb = tf ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(cols * eb)};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode_tiled(map, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                 const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return tb_fail(ctx, TB_ERR_CUDA, "cuTensorMapEncodeTiled (grouped) failed (%d)", (int)r);
  return TB_OK;
}

GArgs make_args(const Plan& p, char* base) {
  GArgs ga{};
  ga.count = p.count;
  ga.max_iter = p.max_iter;
  ga.rule = p.rule;
  ga.cols = p.cols;
  ga.tol_floor_u = p.u;
  ga.desc = reinterpret_cast<const GDesc*>(base + p.off_desc);
  ga.queue = reinterpret_cast<int*>(base + p.off_queue);
  ga.err = reinterpret_cast<int*>(base + p.off_err);
  for (int b = 0; b < 2; ++b) {
    ga.M[b] = reinterpret_cast<float*>(base + p.off_m[b]);
    ga.Hi[b] = base + p.off_hi[b];
    ga.Lo[b] = p.off_lo[b] ? base + p.off_lo[b] : nullptr;
  }
  return ga;
}

template <int P, int BN, bool FS = false>
int launch(tb_ctx* ctx, const Plan& p, char* base, int grid, cudaStream_t s) {
  using G = GCfg<P, BN>;
  static unsigned long long attr_done = 0;
  if (int rc_attr = tb_smem_attr(ctx, k_sp2_grouped<P, BN, FS>, G::smem, &attr_done)) return rc_attr;
  const GArgs ga = make_args(p, base);
  TB_CUDA_TRY(ctx, cudaMemsetAsync(ga.queue, 0, sizeof(int), s));
  if constexpr (FS) {
    // A and B are row panels of the FP32 masters (BN = BM: one map per buffer)
    k_sp2_grouped<P, BN, true><<<grid, kThreadsFs, G::smem, s>>>(ga, p.am[0], p.am[0], p.am[0], p.am[0], p.am[1],
                                                                 p.am[1], p.am[1], p.am[1]);
  } else {
    const CUtensorMap* bh = BN == 64 ? p.bh64 : p.bh128;
    const CUtensorMap* bl = BN == 64 ? p.bl64 : p.bl128;
    k_sp2_grouped<P, BN, false><<<grid, kThreads, G::smem, s>>>(ga, p.ah[0], p.al[0], bh[0], bl[0], p.ah[1],
                                                                p.al[1], bh[1], bl[1]);
  }
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// Cluster form: as many clusters of CS CTAs as can be resident at once.
template <int P, int CS>
int launch_cl(tb_ctx* ctx, const Plan& p, char* base, cudaStream_t s, int* grid_out) {
  using G = GCfg<P, BM>;
  static unsigned long long attr_done = 0;
  if (int rc_attr = tb_smem_attr(ctx, k_sp2_grouped_cl<P, CS>, G::smem, &attr_done)) return rc_attr;
  const GArgs ga = make_args(p, base);
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = G::smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(std::max(CS, ctx->sm_count / CS * CS));
  int nclusters = 0;
  TB_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&nclusters, k_sp2_grouped_cl<P, CS>, &cfg));
  if (nclusters < 1) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "no cluster of %d CTAs fits", CS);
  cfg.gridDim = dim3(nclusters * CS);
  if (grid_out) *grid_out = nclusters * CS;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(ga.queue, 0, sizeof(int), s));
  TB_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, k_sp2_grouped_cl<P, CS>, ga, p.ah[0], p.al[0], p.ah[1], p.al[1]));
  return TB_OK;
}

template <int P>
int launch_cl_p(tb_ctx* ctx, const Plan& p, char* base, int cs, cudaStream_t s, int* grid_out) {
  switch (cs) {
    case 2: return launch_cl<P, 2>(ctx, p, base, s, grid_out);
    case 4: return launch_cl<P, 4>(ctx, p, base, s, grid_out);
    case 8: return launch_cl<P, 8>(ctx, p, base, s, grid_out);
    default: return tb_fail(ctx, TB_ERR_ARG, "cluster size %d (2, 4 or 8)", cs);
  }
}

int launch_cl_any(tb_ctx* ctx, const Plan& p, char* base, int cs, cudaStream_t s, int* grid_out) {
  switch (p.precision) {
    case TB_PREC_TF32: return launch_cl_p<TB_PREC_TF32>(ctx, p, base, cs, s, grid_out);
    case TB_PREC_TF32X3: return launch_cl_p<TB_PREC_TF32X3>(ctx, p, base, cs, s, grid_out);
    case TB_PREC_BF16: return launch_cl_p<TB_PREC_BF16>(ctx, p, base, cs, s, grid_out);
    case TB_PREC_BF16X3: return launch_cl_p<TB_PREC_BF16X3>(ctx, p, base, cs, s, grid_out);
    default: return tb_fail(ctx, TB_ERR_UNSUPPORTED, "grouped SP2 needs a tensor-core precision");
  }
}

int launch_any(tb_ctx* ctx, const Plan& p, char* base, int bn, int grid, cudaStream_t s) {
  const bool b64 = bn == 64;
  if (bn == 0) {
    if (p.precision != TB_PREC_TF32X3) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "the FP32-staged form is tf32x3 only");
    return launch<TB_PREC_TF32X3, 128, true>(ctx, p, base, grid, s);
  }
  switch (p.precision) {
    case TB_PREC_TF32: return b64 ? launch<TB_PREC_TF32, 64>(ctx, p, base, grid, s) : launch<TB_PREC_TF32, 128>(ctx, p, base, grid, s);
    case TB_PREC_TF32X3: return b64 ? launch<TB_PREC_TF32X3, 64>(ctx, p, base, grid, s) : launch<TB_PREC_TF32X3, 128>(ctx, p, base, grid, s);
    case TB_PREC_BF16: return b64 ? launch<TB_PREC_BF16, 64>(ctx, p, base, grid, s) : launch<TB_PREC_BF16, 128>(ctx, p, base, grid, s);
    case TB_PREC_BF16X3: return b64 ? launch<TB_PREC_BF16X3, 64>(ctx, p, base, grid, s) : launch<TB_PREC_BF16X3, 128>(ctx, p, base, grid, s);
    default: return tb_fail(ctx, TB_ERR_UNSUPPORTED, "grouped SP2 needs a tensor-core precision");
  }
}

}  // namespace

extern "C" int dm_sp2_grouped_workspace_size(int count, const int* n, const tb_sp2_opts* o, size_t* bytes) {
  if (count < 1 || !n || !o || !bytes) return TB_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > kMaxLd) return TB_ERR_ARG;
  Plan p{};
  *bytes = layout(count, n, o->precision, &p);
  return TB_OK;
}

extern "C" int dm_sp2_grouped_plan(tb_ctx* ctx, int count, const int* n, const double* nocc,
                                   const double* const* H, double* const* D, tb_sp2_report* reports,
                                   const tb_sp2_opts* o, int autotune, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (count < 1 || !n || !nocc || !H || !D || !o || !ws)
    return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_sp2_grouped_plan");
  if (o->precision == TB_PREC_FP64 || o->precision > TB_PREC_BF16X3)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "grouped SP2 needs a tensor-core precision");
  if (o->max_iter < 1 || o->max_iter > SP2_MAX_ITER) return tb_fail(ctx, TB_ERR_ARG, "max_iter outside 1..%d", SP2_MAX_ITER);
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > kMaxLd || !H[i] || !D[i] || !(nocc[i] >= 0.0) || nocc[i] > n[i])
      return tb_fail(ctx, TB_ERR_ARG, "system %d: n = %d (1..%d), n_occ = %g", i, n[i], kMaxLd, nocc[i]);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  if (autotune < 0 || autotune > 8 || autotune == 6 || autotune == 7)
    return tb_fail(ctx, TB_ERR_ARG, "autotune %d is not a launch form (0..5, 8)", autotune);
  Plan p{};
  const size_t need = layout(count, n, o->precision, &p);
  if (ws_bytes < need) return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu", ws_bytes, need);
  cudaStream_t s = as_stream(stream);
  char* base = static_cast<char*>(ws);
  p.count = count;
  p.precision = o->precision;
  p.rule = o->rule;
  p.max_iter = o->max_iter;
  p.u = (o->precision == TB_PREC_TF32X3 || o->precision == TB_PREC_BF16X3) ? 0x1p-24
        : o->precision == TB_PREC_TF32 ? 0x1p-11 : 0x1p-8;
  // descriptors, largest system first (longest-processing-time order)
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<GDesc> desc(count);
  int row = 0;
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    GDesc d{};
    d.H = H[i];
    d.D = D[i];
    d.rep = reports ? reports + i : nullptr;
    d.n = n[i];
    d.ld = round_up(n[i], BM);
    d.row_off = row;
    d.nocc = nocc[i];
    row += d.ld;
    desc[j] = d;
  }
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(base + p.off_desc, desc.data(), sizeof(GDesc) * count, cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx, cudaMemsetAsync(base + p.off_err, 0, sizeof(int) * 4, s));
  // the stacked operand arrays start zeroed: padding columns beyond a
  // system's ld are never read, and its padding inside ld is written by X0
  for (int b = 0; b < 2; ++b) {
    int rc = make_map(ctx, p.precision, base + p.off_hi[b], p.rows, p.cols, BM, &p.ah[b]);
    if (rc) return rc;
    rc = make_map(ctx, p.precision, base + p.off_hi[b], p.rows, p.cols, 64, &p.bh64[b]);
    if (rc) return rc;
    rc = make_map(ctx, p.precision, base + p.off_hi[b], p.rows, p.cols, 128, &p.bh128[b]);
    if (rc) return rc;
    if (p.off_lo[b]) {
      rc = make_map(ctx, p.precision, base + p.off_lo[b], p.rows, p.cols, BM, &p.al[b]);
      if (rc) return rc;
      rc = make_map(ctx, p.precision, base + p.off_lo[b], p.rows, p.cols, 64, &p.bl64[b]);
      if (rc) return rc;
      rc = make_map(ctx, p.precision, base + p.off_lo[b], p.rows, p.cols, 128, &p.bl128[b]);
      if (rc) return rc;
    } else {
      p.al[b] = p.ah[b];
      p.bl64[b] = p.bh64[b];
      p.bl128[b] = p.bh128[b];
    }
  }
  for (int b = 0; b < 2; ++b)
    if (p.precision == TB_PREC_TF32X3) {
      const int rc = make_map(ctx, p.precision, base + p.off_m[b], p.rows, p.cols, BM, &p.am[b]);
      if (rc) return rc;
    }
  p.bn = 128;
  p.grid = std::max(1, ctx->sm_count);
  p.cs = 1;
  if (autotune == 0 && p.precision == TB_PREC_TF32X3) {
    p.bn = 0;  // the FP32-staged form: bitwise the stored-split form's result, faster
  } else if (autotune == 3) {
    if (p.precision != TB_PREC_TF32X3) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "the FP32-staged form is tf32x3 only");
    p.bn = 0;
  } else if (autotune == 4 || autotune == 8 || autotune == 5) {
    p.cs = autotune == 5 ? 2 : autotune;
    int rc = launch_cl_any(ctx, p, base, p.cs, s, &p.grid);  // sizes the grid (and warms up)
    if (rc) return rc;
  } else if (autotune == 1) {
    // time every candidate on the batch itself and keep the fastest: one CTA
    // per system with 128- or 64-wide tiles and a full or half grid,
    // clusters of 2, 4 or 8 CTAs per system, or (tf32x3) the FP32-staged form
    struct Cand {
      int bn, grid, cs;
    };
    const Cand cands[8] = {{128, ctx->sm_count, 1}, {128, std::max(1, ctx->sm_count / 2), 1},
                           {64, ctx->sm_count, 1},  {64, std::max(1, ctx->sm_count / 2), 1},
                           {128, 0, 2},             {128, 0, 4},
                           {128, 0, 8},             {0, ctx->sm_count, 1}};
    cudaEvent_t e0, e1;
    TB_CUDA_TRY(ctx, cudaEventCreate(&e0));
    TB_CUDA_TRY(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    for (const Cand& c : cands) {
      int grid = c.grid;
      auto run = [&]() {
        return c.cs > 1 ? launch_cl_any(ctx, p, base, c.cs, s, &grid) : launch_any(ctx, p, base, c.bn, c.grid, s);
      };
      if (c.bn == 0 && p.precision != TB_PREC_TF32X3) continue;
      int rc = run();  // warm-up
      if (rc == TB_ERR_UNSUPPORTED) continue;  // no cluster of that size fits
      if (rc) return rc;
      TB_CUDA_TRY(ctx, cudaEventRecord(e0, s));
      rc = run();
      if (rc) return rc;
      TB_CUDA_TRY(ctx, cudaEventRecord(e1, s));
      TB_CUDA_TRY(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      TB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        p.bn = c.bn;
        p.grid = grid;
        p.cs = c.cs;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(base, &p, sizeof(Plan), cudaMemcpyHostToDevice, s));
  TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  // a host copy of the plan lives in the context for the run call
  std::copy(reinterpret_cast<const char*>(&p), reinterpret_cast<const char*>(&p) + sizeof(Plan), ctx->plan_cache);
  ctx->plan_ws = ws;
  return TB_OK;
}

extern "C" int dm_sp2_grouped_run(tb_ctx* ctx, void* ws, int* bn_out, void* stream) {
  if (!ctx || !ws) return TB_ERR_ARG;
  if (ctx->plan_ws != ws) return tb_fail(ctx, TB_ERR_ARG, "workspace has no plan in this context");
  Plan p;
  std::copy(ctx->plan_cache, ctx->plan_cache + sizeof(Plan), reinterpret_cast<char*>(&p));
  if (bn_out) *bn_out = p.cs * 10000000 + p.bn * 10000 + p.grid;
  if (p.cs > 1) return launch_cl_any(ctx, p, static_cast<char*>(ws), p.cs, as_stream(stream), nullptr);
  return launch_any(ctx, p, static_cast<char*>(ws), p.bn, p.grid, as_stream(stream));
}
