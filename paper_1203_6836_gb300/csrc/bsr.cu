// Thresholded block-sparse SP2 (row a5): the linear-scaling form of the
// purification (Sec. III.B, Table I tau > 0 rows).
//
// Reading: after X0 and after every projection, every 32 x 32 block of X whose
// Frobenius norm is below tau is set to zero (the paper drops elements below
// tau; the 32 x 32 block rule is the block-sparse reading).
//
// GB300 layout: X is stored as 128 x 128 super-blocks (one tcgen05 tile) in a
// block-sparse-row structure, ping-ponged between two buffers.  A super-block
// is stored when at least one of its sixteen 32 x 32 sub-blocks survives the
// drop rule; dropped sub-blocks inside a stored super-block hold zeros, so the
// arithmetic is the same as dropping 32 x 32 blocks.  For n <= 131072 there are
// at most 1024 super-rows and each row's pattern is a 1024-bit bitmap.
//
// Per projection (all on the device, no host synchronisation):
//   decide  reduce the trace partials of X_k, take the stop/branch decision
//           (every CTA the same), build each row's bitmaps of stored and live
//           (not all-zero) super-blocks;
//   symbolic  candidates of row I = OR of the live bitmaps of its live
//           columns; scans give the output slots; each upper output block
//           (I <= J; X^2 and its pattern are symmetric) gets the list of common
//           K (live in both rows I and J) as pairs of source slots; the upper
//           blocks are listed in (band of 8 block rows, column, row) order;
//   numeric  a persistent tcgen05 kernel walks that list: TMA loads the (I,K)
//           and (J,K) tiles of every pair into shared memory (tf32x3: the FP32
//           blocks, split into hi and lo there by four converter warps; other
//           precisions: their stored splits), the MMA accumulates in TMEM
//           (double-buffered between blocks), the epilogue applies the branch
//           (X^2 or 2X - X^2), zeroes every 32 x 32 sub-block with ||.||_F <
//           tau (one warp owns a 32-row band, so a sub-block norm is a warp
//           reduction), writes block (I,J) and, transposed, its mirror (J,I),
//           and accumulates FP64 trace partials.
// The final iterate is written to the dense FP64 D or, with BSR input and
// output (dm_sp2_sparse), to a BSR D.
//
// The same engine computes C = alpha A B + gamma S + delta I for two
// different symmetric, commuting matrices (the candidate pattern is that of
// A B and B A together, so it is symmetric; the diagonal blocks keep their
// upper triangle and mirror it), which is what the block-sparse Fermi
// expansion (dm_fermi_sparse, row f2) is built from, with exact affine steps
// alpha X + delta I on X's pattern.

#include "common.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

using namespace tcx;

constexpr int SB = 128;            // super-block side (tcgen05 tile)
constexpr int MW = 32;             // bitmap words per row (1024 super-rows: n <= 131072)
constexpr int kMaxNsb = MW * 32;
constexpr int kThreads = 192;      // numeric kernel: TMA, MMA, 4 epilogue warps
// tf32x3 keeps only the FP32 master of every block: the numeric kernel loads the
// masters and four converter warps split them into hi and lo in shared memory
// (the same rounding the stored splits had, so the products are bitwise those
// of stored splits), at half the operand bytes and a third of the stores
template <int P>
constexpr bool kStaged = P == TB_PREC_TF32X3;
template <int P>
constexpr int kNumThreads = kStaged<P> ? 320 : kThreads;
constexpr int kTiles = SB * SB;    // elements per super-block
constexpr int kMaxGrid = 256;      // cap of the persistent numeric grid (which is also at most the SM count)
constexpr int kBand = 8;           // block rows whose outputs the numeric kernel walks together

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Buf {
  int* row_ptr;      // [nsb + 1]
  int* col;          // [cap]
  int* nz;           // [cap] live flag (some sub-block kept)
  uint32_t* stored;  // [nsb * MW]
  uint32_t* live;    // [nsb * MW]
  float* val;        // [cap * kTiles] FP32 master
  void* hi;          // [cap * kTiles] stored operand splits (null with kStaged)
  void* lo;
};

struct Sym {
  uint32_t* cand;    // [nsb * MW]
  int* cnt;          // [nsb]
  int* out_row;      // [cap]
  int* old_idx;      // [cap]
  int* pcnt;         // [cap]
  int* pair_ptr;     // [cap + 1]
  int2* pairs;       // [pcap]
  int* scal;         // [4]: blocks of the new pattern, pairs, upper blocks
  int* order;        // [cap] upper output blocks in the numeric kernel's order
  uint16_t* flags;   // [nsb * nsb] X0 sub-block keep masks
};

struct Args {
  int n, ld, nsb, cap, pcap;
  int mw;                 // bitmap words in use: ceil(nsb / 32)
  double nocc, tau2, floor, tol;
  int rule, k, max_iter;
  SP2State* st;
  const double* parts_in;
  int nparts_in;
  double* parts_out;
  // start X0 = x0_s (x0_e I - H); x0_s = 0: the SP2 start from the Gershgorin
  // bounds in st (e = eps_max, s = 1/(eps_max - eps_min))
  double x0_e, x0_s;
  int keep_diag;          // every pattern stores the diagonal blocks
  int same_ab;            // the product's operands are one matrix
};

// Epilogue of a product C = alpha A B + gamma S + delta I: (alpha, gamma) =
// (a1, g1) when branch is set and bit k of the SP2 branch record is, else
// (a0, g0); delta on the diagonal of the n x n block.  lolo: also the lo x lo
// split product (squares, where it keeps the diagonal unbiased).
struct Epi {
  float a0, g0, a1, g1, d;
  int branch, lolo;
};

__device__ __forceinline__ int popc_below(const uint32_t* m, int bit) {
  int r = 0;
  for (int w = 0; w < (bit >> 5); ++w) r += __popc(m[w]);
  const uint32_t part = m[bit >> 5] & ((1u << (bit & 31)) - 1u);
  return r + __popc(part);
}

// Row of slot o of b: the last row whose start is <= o.
__device__ __forceinline__ int slot_row(const Buf& b, int nsb, int o) {
  int lo = 0, hi = nsb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (b.row_ptr[mid] <= o) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ init

// emin/emax from the Gershgorin partials (one block).
__global__ void k_bsr_bounds(const double* bparts, int nb, SP2State* st) {
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
  }
}

// (e, s) of the start X0 = s (e I - H).
__device__ __forceinline__ void x0_affine(const Args& a, double* e, double* s) {
  if (a.x0_s != 0.0) {
    *e = a.x0_e;
    *s = a.x0_s;
    return;
  }
  const double emin = a.st->emin, emax = a.st->emax;
  double w = emax - emin;
  if (!(w > 0.0)) w = 1.0;
  *e = emax;
  *s = 1.0 / w;
}

__device__ __forceinline__ double x0_val(const double* H, int n, int r, int c, double emax, double inv) {
  if (r >= n || c >= n) return 0.0;
  return ((r == c ? emax : 0.0) - H[(size_t)r * n + c]) * inv;
}

// Per-lane partial sums of squares of the 16 32 x 32 sub-blocks of a 128 x 128
// block x(r, c) (256 threads: warp w takes rows w + 8k, lane l the columns
// 32 c + l, so every row segment is one coalesced load; row w + 8k lies in
// sub-block row k / 4).
template <class X>
__device__ __forceinline__ void block_partials(X x, double (&acc)[16]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int r = warp + 8 * k;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const double v = x(r, 32 * cc + lane);
      acc[(k >> 2) * 4 + cc] = fma(v, v, acc[(k >> 2) * 4 + cc]);
    }
  }
}

// Keep mask of super-block (I, J) of X0 = s (e I - H) from the partial sums
// (block_partials) of e I - H over its upper twin (min(I,J), max(I,J)): a
// warp sum per sub-block, the eight warps combined in a fixed order, times
// scale2 = s^2, kept where ||.||_F >= tau (one FMA per element: GB300's FP64
// rate is low); below the
// diagonal the twin's mask transposed, so that the pattern is exactly
// symmetric (the products compute upper blocks and mirror them).  Called by
// every thread of the block; the mask is valid in thread 0.
__device__ uint16_t keep_mask(const Args& a, int I, int J, const double (&acc)[16], double scale2) {
  __shared__ double wsum[8][16];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const double v = warp_sum(acc[s]);
    if (lane == 0) wsum[warp][s] = v;
  }
  __syncthreads();
  uint16_t f = 0;
  if (threadIdx.x == 0)
    for (int s = 0; s < 16; ++s) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += wsum[w][s];
      t *= scale2;
      if (t >= a.tau2 && t > 0.0) f |= (uint16_t)(1u << (I <= J ? s : (s & 3) * 4 + (s >> 2)));
    }
  __syncthreads();  // wsum is reused by the next block of a grid-stride loop
  return f;
}

// One block per super-block (I, J) of X0 = s (e I - H): its keep mask.
__global__ void __launch_bounds__(256) k_bsr_init_flags(const double* __restrict__ H, Args a, Sym sy) {
  const int I = blockIdx.y, J = blockIdx.x;
  const int I0 = min(I, J), J0 = max(I, J);
  double emax, inv;
  x0_affine(a, &emax, &inv);
  double acc[16];
  block_partials([&](int r, int c) { return x0_val(H, a.n, I0 * SB + r, J0 * SB + c, emax, 1.0); }, acc);
  const uint16_t f = keep_mask(a, I, J, acc, inv * inv);
  if (threadIdx.x == 0) sy.flags[(size_t)I * a.nsb + J] = f;
}

// Row I of X0: live bitmap of its kept super-blocks; stored = live (and the
// diagonal block with keep_diag); count of stored blocks.
__global__ void k_bsr_init_rows(Args a, Sym sy, Buf b) {
  const int I = blockIdx.x;
  __shared__ uint32_t m[MW];
  if (threadIdx.x < MW) m[threadIdx.x] = 0u;
  __syncthreads();
  for (int J = threadIdx.x; J < a.nsb; J += blockDim.x)
    if (sy.flags[(size_t)I * a.nsb + J]) atomicOr(&m[J >> 5], 1u << (J & 31));
  __syncthreads();
  if (threadIdx.x < MW) {
    const uint32_t diag = (a.keep_diag && (I >> 5) == (int)threadIdx.x) ? 1u << (I & 31) : 0u;
    b.stored[I * MW + threadIdx.x] = m[threadIdx.x] | diag;
    b.live[I * MW + threadIdx.x] = m[threadIdx.x];
    m[threadIdx.x] |= diag;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < MW; ++w) c += __popc(m[w]);
    sy.cnt[I] = c;
  }
}

// Exclusive scan of cnt[0..nsb) into row_ptr (one block); total into scal[0].
// One warp: lane l scans rows [l * per, (l + 1) * per) after an exclusive
// warp scan of the lanes' sums.
__global__ void k_bsr_scan_rows(Args a, Sym sy, int* row_ptr) {
  if (a.st->done || a.st->err) return;
  const int lane = threadIdx.x & 31, per = (a.nsb + 31) / 32;
  const int lo = min(a.nsb, lane * per), hi = min(a.nsb, lo + per);
  int mine = 0;
  for (int i = lo; i < hi; ++i) mine += sy.cnt[i];
  int incl = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  int run = incl - mine;
  for (int i = lo; i < hi; ++i) {
    row_ptr[i] = run;
    run += sy.cnt[i];
  }
  if (lane == 31) {
    row_ptr[a.nsb] = incl;
    sy.scal[0] = incl;
    if (incl > a.cap) atomicExch(&a.st->err, TB_ERR_OOM);
  }
}

// Fill the X0 blocks of row I (one block per row): values with dropped
// sub-blocks zeroed, operand splits, trace partials of the row.
template <int P>
__global__ void __launch_bounds__(256) k_bsr_init_fill(const double* __restrict__ H, Args a, Sym sy, Buf b) {
  if (a.st->err) return;
  const int I = blockIdx.x;
  double emax, inv;
  x0_affine(a, &emax, &inv);
  double t1 = 0.0, t2 = 0.0;
  int o = b.row_ptr[I];
  for (int J = 0; J < a.nsb; ++J) {
    const uint16_t f = sy.flags[(size_t)I * a.nsb + J];
    if (!f && !(a.keep_diag && J == I)) continue;
    if (threadIdx.x == 0) {
      b.col[o] = J;
      b.nz[o] = f != 0;
    }
    // 128 rows x 4 segments of 32: 512 segments over 256 threads
    for (int seg = threadIdx.x; seg < SB * 4; seg += blockDim.x) {
      const int r = seg >> 2, cs = seg & 3;
      const bool keep = (f >> ((r >> 5) * 4 + cs)) & 1;
      float y[32];
      for (int j = 0; j < 32; ++j) {
        const double x = keep ? x0_val(H, a.n, I * SB + r, J * SB + 32 * cs + j, emax, inv) : 0.0;
        y[j] = (float)x;
        const double xf = (double)y[j];
        t2 += xf * xf;
        if (I == J && r == 32 * cs + j) t1 += xf;
      }
      const size_t e0 = (size_t)o * kTiles + (size_t)r * SB + 32 * cs;
      float* dst = b.val + e0;
      for (int j = 0; j < 32; ++j) dst[j] = y[j];
      if constexpr (!kStaged<P>) {
        char* h = static_cast<char*>(b.hi) + e0 * Prec<P>::eb;
        char* l = b.lo ? static_cast<char*>(b.lo) + e0 * Prec<P>::eb : h;
        store_operands<P>(y, h, l);
      }
    }
    ++o;
  }
  __shared__ double s1[8], s2[8];
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = t1;
    s2[threadIdx.x >> 5] = t2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      x += s1[q];
      y += s2[q];
    }
    a.parts_out[3 * I] = x;
    a.parts_out[3 * I + 1] = y;
    a.parts_out[3 * I + 2] = 0.0;
  }
}

// ---- BSR input (dm_sp2_sparse): H given as 128 x 128 FP64 blocks

// Slot of block (I, J) in a BSR row (binary search over its sorted columns), or -1.
__device__ __forceinline__ int bsr_find(const int* __restrict__ row_ptr, const int* __restrict__ col, int I, int J) {
  int lo = row_ptr[I], hi = row_ptr[I + 1] - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = col[mid];
    if (c == J) return mid;
    if (c < J) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// Gershgorin partials of block row I (one block of 256 threads): warp w
// takes rows w + 8k of every block of the row, lane l the columns 32 c + l, so
// each block is read as 64 independent coalesced loads a lane, and the row
// sums stay in registers until one warp sum per row; min(H_ii - r_i) and
// max(H_ii + r_i) over the rows go into bparts[2 I].
__global__ void __launch_bounds__(256) k_bsr_bounds_in(tb_bsr H, double* __restrict__ bparts) {
  __shared__ double smin[8], smax[8];
  const int I = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (*H.status != TB_OK) {  // an incomplete H (k_bsr_status_in fails the call)
    if (threadIdx.x == 0) bparts[2 * I] = bparts[2 * I + 1] = 0.0;
    return;
  }
  double rad[16], dia[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) rad[k] = dia[k] = 0.0;
  for (int o = H.row_ptr[I]; o < H.row_ptr[I + 1]; ++o) {
    const double* blk = H.val + (size_t)o * kTiles;
    const bool dblk = H.col[o] == I;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int r = warp + 8 * k;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const double x = blk[(size_t)r * SB + 32 * cc + lane];
        if (dblk && 32 * cc + lane == r) dia[k] += x;
        else rad[k] += fabs(x);
      }
    }
  }
  double lo = INFINITY, hi = -INFINITY;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const double rs = warp_sum(rad[k]), c = warp_sum(dia[k]);  // one lane holds the diagonal element
    if (I * SB + warp + 8 * k < H.n) {
      lo = fmin(lo, c - rs);
      hi = fmax(hi, c + rs);
    }
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
    bparts[2 * I] = a;
    bparts[2 * I + 1] = b;
  }
}

// e delta - h at element (r, c) of block (I, J) (zero outside the n x n matrix).
__device__ __forceinline__ double x0_unscaled(const double* blk, int I, int J, int n, int r, int c, double e) {
  const int gr = I * SB + r, gc = J * SB + c;
  if (gr >= n || gc >= n) return 0.0;
  const double h = blk ? blk[(size_t)r * SB + c] : 0.0;
  return gr == gc ? e - h : -h;
}

__device__ __forceinline__ double x0_blk(const double* blk, int I, int J, int n, int r, int c, double emax,
                                         double inv) {
  const int gr = I * SB + r, gc = J * SB + c;
  if (gr >= n || gc >= n) return 0.0;
  const double h = blk ? blk[(size_t)r * SB + c] : 0.0;
  return ((gr == gc ? emax : 0.0) - h) * inv;
}

// As k_bsr_init_flags, from the blocks of a BSR H (an absent block of H is
// zero in X0 off the diagonal).
// An H whose build overflowed its capacity fails the call (TB_ERR_OOM).
__global__ void k_bsr_status_in(const int* Hstatus, SP2State* st) {
  if (*Hstatus != TB_OK) st->err = TB_ERR_OOM;
}

// Row of slot o of a BSR matrix: the last row whose start is <= o.
__device__ __forceinline__ int bsr_row_of(const int* __restrict__ row_ptr, int nsb, int o) {
  int lo = 0, hi = nsb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (row_ptr[mid] <= o) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Keep masks of X0 from a BSR H, one block per stored block of H (grid-stride;
// the masks start zeroed, and a block H does not store is zero in X0 off the
// diagonal); k_bsr_init_flags_diag covers diagonal blocks H does not store.
__global__ void __launch_bounds__(256) k_bsr_init_flags_in(tb_bsr H, Args a, Sym sy) {
  if (*H.status != TB_OK) return;  // the call fails through k_bsr_status_in
  const int nblk = min(H.row_ptr[H.nsb], H.cap);
  double emax, inv;
  x0_affine(a, &emax, &inv);
  for (int o = blockIdx.x; o < nblk; o += gridDim.x) {
    const int I = bsr_row_of(H.row_ptr, H.nsb, o), J = H.col[o];
    const int I0 = min(I, J), J0 = max(I, J);
    const int slot = I <= J ? o : bsr_find(H.row_ptr, H.col, I0, J0);
    const double* blk = slot >= 0 ? H.val + (size_t)slot * kTiles : nullptr;
    double acc[16];
    block_partials([&](int r, int c) { return x0_unscaled(blk, I0, J0, a.n, r, c, emax); }, acc);
    const uint16_t f = keep_mask(a, I, J, acc, inv * inv);
    if (threadIdx.x == 0) sy.flags[(size_t)I * a.nsb + J] = f;
  }
}

__global__ void __launch_bounds__(256) k_bsr_init_flags_diag(tb_bsr H, Args a, Sym sy) {
  const int I = blockIdx.x;
  if (*H.status != TB_OK || bsr_find(H.row_ptr, H.col, I, I) >= 0) return;
  double emax, inv;
  x0_affine(a, &emax, &inv);
  double acc[16];
  block_partials([&](int r, int c) { return x0_unscaled(nullptr, I, I, a.n, r, c, emax); }, acc);
  const uint16_t f = keep_mask(a, I, I, acc, inv * inv);
  if (threadIdx.x == 0) sy.flags[(size_t)I * a.nsb + I] = f;
}

// As k_bsr_init_fill, from the blocks of a BSR H.
template <int P>
__global__ void __launch_bounds__(256) k_bsr_init_fill_in(tb_bsr H, Args a, Sym sy, Buf b) {
  if (a.st->err) return;
  const int I = blockIdx.x;
  double emax, inv;
  x0_affine(a, &emax, &inv);
  double t1 = 0.0, t2 = 0.0;
  int o = b.row_ptr[I];
  for (int J = 0; J < a.nsb; ++J) {
    const uint16_t f = sy.flags[(size_t)I * a.nsb + J];
    if (!f && !(a.keep_diag && J == I)) continue;
    const int slot = bsr_find(H.row_ptr, H.col, I, J);
    const double* blk = slot >= 0 ? H.val + (size_t)slot * kTiles : nullptr;
    if (threadIdx.x == 0) {
      b.col[o] = J;
      b.nz[o] = f != 0;
    }
    for (int seg = threadIdx.x; seg < SB * 4; seg += blockDim.x) {
      const int r = seg >> 2, cs = seg & 3;
      const bool keep = (f >> ((r >> 5) * 4 + cs)) & 1;
      float y[32];
      for (int j = 0; j < 32; ++j) {
        const double x = keep ? x0_blk(blk, I, J, a.n, r, 32 * cs + j, emax, inv) : 0.0;
        y[j] = (float)x;
        const double xf = (double)y[j];
        t2 += xf * xf;
        if (I == J && r == 32 * cs + j) t1 += xf;
      }
      const size_t e0 = (size_t)o * kTiles + (size_t)r * SB + 32 * cs;
      float* dst = b.val + e0;
      for (int j = 0; j < 32; ++j) dst[j] = y[j];
      if constexpr (!kStaged<P>) {
        char* hp = static_cast<char*>(b.hi) + e0 * Prec<P>::eb;
        char* lp = b.lo ? static_cast<char*>(b.lo) + e0 * Prec<P>::eb : hp;
        store_operands<P>(y, hp, lp);
      }
    }
    ++o;
  }
  __shared__ double s1[8], s2[8];
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = t1;
    s2[threadIdx.x >> 5] = t2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      x += s1[q];
      y += s2[q];
    }
    a.parts_out[3 * I] = x;
    a.parts_out[3 * I + 1] = y;
    a.parts_out[3 * I + 2] = 0.0;
  }
}

// ------------------------------------------------------- per projection

// Bitmaps of row I of b: stored blocks and live (not all-zero) blocks; ms and
// ml are zeroed shared arrays of the calling block.
__device__ void row_bitmaps(const Buf& b, int I, uint32_t* ms, uint32_t* ml) {
  for (int o = b.row_ptr[I] + threadIdx.x; o < b.row_ptr[I + 1]; o += blockDim.x) {
    const int J = b.col[o];
    atomicOr(&ms[J >> 5], 1u << (J & 31));
    if (b.nz[o]) atomicOr(&ml[J >> 5], 1u << (J & 31));
  }
  __syncthreads();
  if (threadIdx.x < MW) {
    b.stored[I * MW + threadIdx.x] = ms[threadIdx.x];
    b.live[I * MW + threadIdx.x] = ml[threadIdx.x];
  }
}

// Decision for projection k (every block the same) and the bitmaps of row I
// of X_k: stored blocks and live (not all-zero) blocks.
__global__ void k_bsr_decide(Args a, Buf b) {
  __shared__ int s_stop;
  __shared__ uint32_t ms[MW], ml[MW];
  SP2State* st = a.st;
  if (st->done || st->err) return;
  if (threadIdx.x < 32) {
    double x = 0, y = 0;
    for (int i = threadIdx.x; i < a.nparts_in; i += 32) {
      x += a.parts_in[3 * i];
      y += a.parts_in[3 * i + 1];
    }
    x = warp_sum(x);
    y = warp_sum(y);
    if (threadIdx.x == 0) {
      SP2StepArgs d{};
      d.nocc = a.nocc;
      d.tol = a.tol;
      d.floor = a.floor;
      d.rule = a.rule;
      d.k = a.k;
      d.max_iter = a.max_iter;
      int br = 0, capped = 0;
      const int stop = sp2_decide(d, x, y, st->t1, st->t2, true, &br, &capped);
      s_stop = stop;
      if (blockIdx.x == 0) {
        st->t1[a.k] = x;
        st->t2[a.k] = y;
        if (stop) {
          st->iters = a.k;
          st->capped = capped;
          st->done = 1;
        } else if (br) {
          st->branch[a.k >> 6] |= 1ull << (a.k & 63);
        }
      }
    }
  }
  if (threadIdx.x < MW) {
    ms[threadIdx.x] = 0u;
    ml[threadIdx.x] = 0u;
  }
  __syncthreads();
  if (s_stop) return;
  row_bitmaps(b, blockIdx.x, ms, ml);
}

// Bitmaps of stored and live blocks of every row of a product's output.
__global__ void k_bsr_bitmaps(Args a, Buf b) {
  __shared__ uint32_t ms[MW], ml[MW];
  if (a.st->done || a.st->err) return;
  if (threadIdx.x < MW) {
    ms[threadIdx.x] = 0u;
    ml[threadIdx.x] = 0u;
  }
  __syncthreads();
  row_bitmaps(b, blockIdx.x, ms, ml);
}

// Candidate columns of row I of A B: the OR of B's live rows over A's live
// columns of row I; unless A and B are one matrix also the same with A and B
// exchanged (the pattern of B A = (A B)^T), so that the pattern is symmetric
// as the upper-block computation with mirrors needs; S's live blocks; the
// diagonal block with keep_diag.  A and B are symmetric (rows = columns).
__global__ void k_bsr_cand(Args a, Buf A, Buf B, Buf S, Sym sy) {
  __shared__ uint32_t c[MW];
  if (a.st->done || a.st->err) return;
  const int I = blockIdx.x;
  if (threadIdx.x < MW) c[threadIdx.x] = 0u;
  __syncthreads();
  for (int side = 0; side < (a.same_ab ? 1 : 2); ++side) {
    const uint32_t* li = (side ? B.live : A.live) + I * MW;
    const uint32_t* rows = side ? A.live : B.live;
    for (int K = threadIdx.x; K < a.nsb; K += blockDim.x)
      if ((li[K >> 5] >> (K & 31)) & 1u)
        for (int w = 0; w < a.mw; ++w) {
          const uint32_t v = rows[K * MW + w];
          if (v) atomicOr(&c[w], v);
        }
  }
  __syncthreads();
  if (threadIdx.x < MW) {
    uint32_t v = c[threadIdx.x];
    if (S.live) v |= S.live[I * MW + threadIdx.x];
    if (a.keep_diag && (I >> 5) == (int)threadIdx.x) v |= 1u << (I & 31);
    sy.cand[I * MW + threadIdx.x] = v;
    c[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < MW; ++w) s += __popc(c[w]);
    sy.cnt[I] = s;
  }
}

// Output blocks of row I: column, slot of S_IJ (or -1), pair count.
__global__ void k_bsr_fill_out(Args a, Buf A, Buf B, Buf S, Buf bn, Sym sy) {
  if (a.st->done || a.st->err) return;
  const int I = blockIdx.x;
  const uint32_t* ci = sy.cand + I * MW;
  const uint32_t* si = S.stored ? S.stored + I * MW : nullptr;
  const uint32_t* li = A.live + I * MW;
  for (int J = threadIdx.x; J < a.nsb; J += blockDim.x) {
    if (!((ci[J >> 5] >> (J & 31)) & 1u)) continue;
    const int o = bn.row_ptr[I] + popc_below(ci, J);
    bn.col[o] = J;
    bn.nz[o] = 0;
    sy.out_row[o] = I;
    sy.old_idx[o] = (si && ((si[J >> 5] >> (J & 31)) & 1u)) ? S.row_ptr[I] + popc_below(si, J) : -1;
    int pc = 0;
    const uint32_t* lj = B.live + J * MW;
    if (J >= I)  // the product is symmetric: blocks below the diagonal are written as mirrors
      for (int w = 0; w < a.mw; ++w) pc += __popc(li[w] & lj[w]);
    sy.pcnt[o] = pc;
  }
}

// Exclusive scan of the pair counts of all output blocks (one block).
__global__ void __launch_bounds__(1024) k_bsr_scan_pairs(Args a, Sym sy) {
  __shared__ int part[1024];
  if (a.st->done || a.st->err) return;
  const int nb = sy.scal[0];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += sy.pcnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int v = part[t];
      part[t] = acc;
      acc += v;
    }
    sy.scal[1] = acc;
    sy.pair_ptr[nb] = acc;
    a.st->block_products += (unsigned long long)acc;
    if (acc > a.pcap) atomicExch(&a.st->err, TB_ERR_OOM);
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int i = lo; i < hi; ++i) {
    sy.pair_ptr[i] = run;
    run += sy.pcnt[i];
  }
}

// Pairs (slot of A_IK, slot of B_JK) of every upper output block (I, J):
// (A B)_IJ = sum_K A_IK B_JK^T for a symmetric B.
__global__ void k_bsr_pairs(Args a, Buf A, Buf B, Buf bn, Sym sy) {
  if (a.st->done || a.st->err) return;
  const int nb = sy.scal[0];
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < nb; o += gridDim.x * blockDim.x) {
    const int I = sy.out_row[o], J = bn.col[o];
    if (J < I) continue;
    const uint32_t* li = A.live + I * MW;
    const uint32_t* lj = B.live + J * MW;
    const uint32_t* si = A.stored + I * MW;
    const uint32_t* sj = B.stored + J * MW;
    int p = sy.pair_ptr[o];
    // the mirrored block (J, I) of the full product has as many block products
    if (J > I) atomicAdd(&a.st->block_products, (unsigned long long)sy.pcnt[o]);
    for (int w = 0; w < a.mw; ++w) {
      uint32_t m = li[w] & lj[w];
      while (m) {
        const int K = 32 * w + __ffs(m) - 1;
        m &= m - 1u;
        sy.pairs[p++] = make_int2(A.row_ptr[I] + popc_below(si, K), B.row_ptr[J] + popc_below(sj, K));
      }
    }
  }
}

// Upper output blocks (I <= J) in (band of kBand block rows, column J, row I)
// order.  The persistent numeric kernel takes them in this order, so the CTAs
// working at the same time cover a few columns of one band: they share the
// (I, K) tiles of the band's rows and the (J, K) tiles of those columns in L2
// instead of each streaming its own.  One block; one warp per band.
__global__ void __launch_bounds__(1024) k_bsr_order(Args a, Buf bn, Sym sy) {
  __shared__ int s_off[kMaxNsb / kBand + 1];
  if (a.st->done || a.st->err) return;
  const int nbands = (a.nsb + kBand - 1) / kBand;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int b = warp; b < nbands; b += nw) {
    int c = 0;
    for (int I = b * kBand; I < min(a.nsb, (b + 1) * kBand); ++I) {
      if (lane < MW) {
        uint32_t m = sy.cand[I * MW + lane];
        const int lo = I - 32 * lane;  // keep bits J >= I
        if (lo >= 32) m = 0u;
        else if (lo > 0) m &= ~((1u << lo) - 1u);
        c += __popc(m);
      }
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) s_off[b] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < nbands; ++b) {
      const int v = s_off[b];
      s_off[b] = acc;
      acc += v;
    }
    sy.scal[2] = acc;
  }
  __syncthreads();
  for (int b = warp; b < nbands; b += nw) {
    int pos = s_off[b];
    const int I0 = b * kBand;
    const int I = I0 + lane;
    // only the columns J >= I0 that some row of the band holds (the OR of the
    // band's candidate words), in increasing order
    for (int w = I0 >> 5; w < a.mw; ++w) {
      uint32_t any = 0u;
      for (int r = 0; r < kBand && I0 + r < a.nsb; ++r) any |= sy.cand[(I0 + r) * MW + w];
      if (w == (I0 >> 5)) any &= ~((1u << (I0 & 31)) - 1u);
      while (any) {
        const int J = 32 * w + __ffs(any) - 1;
        any &= any - 1u;
        const bool has = lane < kBand && I < a.nsb && I <= J && ((sy.cand[I * MW + w] >> (J & 31)) & 1u);
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (has) sy.order[pos + __popc(m & ((1u << lane) - 1u))] = bn.row_ptr[I] + popc_below(sy.cand + I * MW, J);
        pos += __popc(m);
      }
    }
  }
}

// Persistent numeric projection.
template <int P>
__global__ void __launch_bounds__(kNumThreads<P>, 1)
    k_bsr_step_tc(Args a, const __grid_constant__ CUtensorMap ah, const __grid_constant__ CUtensorMap al,
                  const __grid_constant__ CUtensorMap bh, const __grid_constant__ CUtensorMap bl, Buf S, Buf bn,
                  Sym sy, Epi ep) {
  using C = Prec<P>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[C::stages], empty[C::stages], tfull[2], tempty[2], mdone, conv[C::stages];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ double s_red[4][3];
  __shared__ float s_sym[4][32][33];  // per epilogue warp: one 32 x 32 diagonal sub-block
  SP2State* st = a.st;
  if (st->done || st->err) return;
  const int br = ep.branch ? (int)((st->branch[a.k >> 6] >> (a.k & 63)) & 1ull) : 0;
  const float alpha = br ? ep.a1 : ep.a0, gamma = br ? ep.g1 : ep.g0;
  const int nu = sy.scal[2];  // upper output blocks, walked in sy.order
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&conv[s], 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(&mdone, 1);
    s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2 * SB);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  constexpr int chunks = SB / C::bk;  // k-steps of one super-block

  if (warp == 0 && lane == 0) {
    prefetch_map(&ah);
    prefetch_map(&bh);
    if (C::split) {
      prefetch_map(&al);
      prefetch_map(&bl);
    }
    int g = 0, issued = 0;
    for (int u = blockIdx.x; u < nu && !s_abort; u += gridDim.x) {
      const int o = sy.order[u];
      const int p0 = sy.pair_ptr[o], p1 = sy.pair_ptr[o + 1];
      for (int p = p0; p < p1 && !s_abort; ++p) {
        const int2 pr = sy.pairs[p];
        for (int c = 0; c < chunks; ++c, ++g) {
          const int s = g % C::stages;
          if (g >= C::stages && !mbar_wait(&empty[s], ((g / C::stages) - 1) & 1, &s_abort)) break;
          uint8_t* base = smem + s * C::stage_bytes;
          // staged: the FP32 masters into the hi positions only
          mbar_expect_tx(&full[s], kStaged<P> ? 2 * 128 * 128 : C::stage_bytes);
          tma_load_2d(base, &ah, &full[s], c * C::bk, pr.x * SB);
          tma_load_2d(base + 128 * 128, &bh, &full[s], c * C::bk, pr.y * SB);
          if constexpr (C::split && !kStaged<P>) {
            tma_load_2d(base + 2 * 128 * 128, &al, &full[s], c * C::bk, pr.x * SB);
            tma_load_2d(base + 3 * 128 * 128, &bl, &full[s], c * C::bk, pr.y * SB);
          }
          issued = g + 1;
        }
      }
    }
    if (s_abort) {
      for (int q = (issued > C::stages ? issued - C::stages : 0); q < issued; ++q) {
        const unsigned long long t0 = gtime();
        while (!mbar_try(&full[q % C::stages], (q / C::stages) & 1) && gtime() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t id = idesc(C::tf32 ? 2u : 1u);
    int g = 0, it = 0;
    for (int u = blockIdx.x; u < nu && !s_abort; u += gridDim.x) {
      const int o = sy.order[u];
      const int buf = it & 1;
      if (it >= 2 && !mbar_wait(&tempty[buf], ((it >> 1) - 1) & 1, &s_abort)) break;
      tc_fence_after();
      const uint32_t d = tmem + buf * SB;
      const int p0 = sy.pair_ptr[o], p1 = sy.pair_ptr[o + 1];
      bool first = true;
      for (int p = p0; p < p1 && !s_abort; ++p) {
        for (int c = 0; c < chunks; ++c, ++g) {
          const int s = g % C::stages;
          if (!mbar_wait(kStaged<P> ? &conv[s] : &full[s], (g / C::stages) & 1, &s_abort)) break;
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * C::stage_bytes);
#pragma unroll
          for (int ks = 0; ks < C::bk / C::uk; ++ks) {
            const uint32_t koff = ks * 32;
            const uint64_t dah = sdesc(base + koff), dbh = sdesc(base + 128 * 128 + koff);
            umma<C::tf32>(d, dah, dbh, id, first ? 0u : 1u);
            first = false;
            if constexpr (C::split) {
              const uint64_t dal = sdesc(base + 2 * 128 * 128 + koff), dbl = sdesc(base + 3 * 128 * 128 + koff);
              umma<C::tf32>(d, dah, dbl, id, 1u);
              umma<C::tf32>(d, dal, dbh, id, 1u);
              // lo x lo: in a square it keeps the diagonal blocks' sums of squares unbiased
              if (ep.lolo) umma<C::tf32>(d, dal, dbl, id, 1u);
            }
          }
          umma_commit(&empty[s]);
        }
      }
      umma_commit(&tfull[buf]);
      ++it;
    }
    // arrives once every MMA this thread issued has completed
    umma_commit(&mdone);
  } else if (kStaged<P> && warp >= 6) {
    // converters: each stage's FP32 tiles of A and B (16 KB each, the hi
    // positions) become hi in place and lo at +32 KB, 16 float4 a thread
    const int ct = threadIdx.x - 192;
    constexpr int kHalf = 2 * 128 * 128 / 16;  // float4 of A and B
    int g = 0;
    for (int u = blockIdx.x; u < nu && !s_abort; u += gridDim.x) {
      const int o = sy.order[u];
      const int npc = (sy.pair_ptr[o + 1] - sy.pair_ptr[o]) * chunks;
      for (int i = 0; i < npc && !s_abort; ++i, ++g) {
        const int s = g % C::stages;
        if (!mbar_wait_warp(&full[s], (g / C::stages) & 1, &s_abort)) break;
        float4* stage = reinterpret_cast<float4*>(smem + s * C::stage_bytes);
#pragma unroll 4
        for (int e = ct; e < kHalf; e += 128) {
          const float4 x = stage[e];
          const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
          stage[e] = h;
          stage[e + kHalf] = make_float4(to_tf32(x.x - h.x), to_tf32(x.y - h.y), to_tf32(x.z - h.z),
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
    int it = 0;
    for (int u = blockIdx.x; u < nu; u += gridDim.x) {
      const int o = sy.order[u];
      const int buf = it & 1;
      ++it;
      if (!mbar_wait_warp(&tfull[buf], ((it - 1) >> 1) & 1, &s_abort)) break;
      tc_fence_after();
      const bool has = sy.pair_ptr[o + 1] > sy.pair_ptr[o];
      const int I = sy.out_row[o], J = bn.col[o];
      const bool mirror = J > I;
      // slot of the transposed block (J, I) in the new pattern
      const int om = mirror ? bn.row_ptr[J] + popc_below(sy.cand + J * MW, I) : o;
      float* xmir = bn.val + (size_t)om * kTiles;
      const int oi = sy.old_idx[o];
      const float* xold = oi >= 0 ? S.val + (size_t)oi * kTiles + (size_t)row * SB : nullptr;
      float* xnew = bn.val + (size_t)o * kTiles + (size_t)row * SB;
      // stored splits (not with kStaged)
      char* hrow = kStaged<P> ? nullptr : static_cast<char*>(bn.hi) + ((size_t)o * kTiles + (size_t)row * SB) * C::eb;
      char* lrow = bn.lo ? static_cast<char*>(bn.lo) + ((size_t)o * kTiles + (size_t)row * SB) * C::eb : hrow;
      int kept = 0;
      // a diagonal block of a product of two matrices is not exactly symmetric
      // in rounding (A B against B A): its upper triangle is kept and mirrored
      const bool symd = I == J && !a.same_ab;
#pragma unroll 1
      for (int c = 0; c < 4; ++c) {
        if (symd && c < q) continue;  // written as the mirror of sub-block (c, q)
        uint32_t v[32];
        if (has) {
          tmem_ld32(tmem + (static_cast<uint32_t>(32 * q) << 16) + buf * SB + 32 * c, v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        // S's row segment: eight 16-byte loads (a scalar load per element would
        // touch 32 rows' lines per warp instruction 32 times over)
        float xs[32];
        if (xold) {
          const float4* x4 = reinterpret_cast<const float4*>(xold + 32 * c);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 t = x4[j];
            xs[4 * j] = t.x;
            xs[4 * j + 1] = t.y;
            xs[4 * j + 2] = t.z;
            xs[4 * j + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) xs[j] = 0.0f;
        }
        float y[32];
        double ss = 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float cxx = __uint_as_float(v[j]);
          y[j] = fmaf(gamma, xs[j], alpha * cxx);
          if (ep.d != 0.0f && I == J && row == 32 * c + j && I * SB + row < a.n) y[j] += ep.d;
        }
        if (symd && c == q) {
          // the 32 x 32 diagonal sub-block: element (l, j) with j < l from lane j
#pragma unroll
          for (int j = 0; j < 32; ++j) s_sym[q][lane][j] = y[j];
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < lane) y[j] = s_sym[q][j][lane];
          __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) ss += (double)y[j] * (double)y[j];
        ss = warp_sum(ss);  // squared Frobenius norm of sub-block (q, c)
        const bool keep = ss >= a.tau2 && ss > 0.0;
        if (!keep) {
#pragma unroll
          for (int j = 0; j < 32; ++j) y[j] = 0.0f;
        } else {
          kept = 1;
        }
        double u2 = 0.0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          u2 += (double)y[j] * (double)y[j];
          if (I == J && row == 32 * c + j) t1 += (double)y[j];
        }
        const bool twice = mirror || (symd && c > q);
        t2 += twice ? 2.0 * u2 : u2;
        {
          // the 32 x 32 sub-tile through shared memory (lane l holds row l), so
          // that each warp store writes one row's 128 contiguous bytes
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j) s_sym[q][lane][j] = y[j];
          __syncwarp();
          float* rows = xnew - (size_t)lane * SB + 32 * c;  // row 32 q of the block, column 32 c
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) rows[(size_t)rr * SB + lane] = s_sym[q][rr][lane];
          __syncwarp();
        }
        if constexpr (!kStaged<P>) store_operands<P>(y, hrow + 32 * c * C::eb, lrow + 32 * c * C::eb);
        if (twice) {
          // element (row, 32c + j) of block (I, J) is element (32c + j, row) of
          // block (J, I) (of this block itself for symd): for each j the 32
          // lanes write 32 consecutive values
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const size_t e = (size_t)(32 * c + j) * SB + row;
            xmir[e] = y[j];
            if constexpr (!kStaged<P>) store_operand1<P>(y[j], bn.hi, bn.lo ? bn.lo : bn.hi, (size_t)om * kTiles + e);
          }
        }
      }
      tc_fence_before();
      if (lane == 0) {
        // the block is live when any of its 32-row bands kept a sub-block
        // (nz[o] was zeroed when the output pattern was built)
        if (kept) {
          atomicOr(&bn.nz[o], 1);
          if (mirror) atomicOr(&bn.nz[om], 1);
        }
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
      }
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
    a.parts_out[3 * blockIdx.x] = s_red[0][0] + s_red[1][0] + s_red[2][0] + s_red[3][0];
    a.parts_out[3 * blockIdx.x + 1] = s_red[0][1] + s_red[1][1] + s_red[2][1] + s_red[3][1];
    a.parts_out[3 * blockIdx.x + 2] = 0.0;
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
    tmem_dealloc(tmem, 2 * SB);
  }
}

// Final iterate (buffer chosen by the iteration count) -> dense FP64 D.
__global__ void k_bsr_to_dense(const SP2State* st, Args a, Buf b0, Buf b1, Sym sy0, Sym sy1, double* D) {
  if (st->err) return;  // D stays zero; the report carries the error
  const Buf& b = (st->iters & 1) ? b1 : b0;
  const int nblk = min(b.row_ptr[a.nsb], a.cap);
  for (int o = blockIdx.x; o < nblk; o += gridDim.x) {
    const int I = slot_row(b, a.nsb, o), J = b.col[o];
    for (int e = threadIdx.x; e < kTiles; e += blockDim.x) {
      const int r = I * SB + e / SB, c = J * SB + e % SB;
      if (r < a.n && c < a.n) D[(size_t)r * a.n + c] = (double)b.val[(size_t)o * kTiles + e];
    }
  }
}

// out = alpha X + delta I on X's pattern (X stores every diagonal block when
// delta != 0): values, operand splits, live flags and bitmaps.  Exact up to
// the FP32 rounding of the values; nothing is dropped.
template <int P>
__global__ void __launch_bounds__(256) k_bsr_affine(Args a, Buf X, Buf out, float alpha, float delta) {
  if (a.st->done || a.st->err) return;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int i = tid; i <= a.nsb; i += nth) out.row_ptr[i] = X.row_ptr[i];
  for (int i = tid; i < a.nsb * MW; i += nth) {
    const int I = i / MW, w = i % MW;
    out.stored[i] = X.stored[i];
    out.live[i] = X.live[i] | ((delta != 0.0f && (I >> 5) == w) ? 1u << (I & 31) : 0u);
  }
  const int nblk = X.row_ptr[a.nsb];
  for (int o = blockIdx.x; o < nblk; o += gridDim.x) {
    const int I = slot_row(X, a.nsb, o), J = X.col[o];
    const bool diag = I == J && delta != 0.0f;
    if (threadIdx.x == 0) {
      out.col[o] = J;
      out.nz[o] = X.nz[o] | (diag ? 1 : 0);
    }
    for (int seg = threadIdx.x; seg < SB * 4; seg += blockDim.x) {
      const int r = seg >> 2, cs = seg & 3;
      const size_t e0 = (size_t)o * kTiles + (size_t)r * SB + 32 * cs;
      float y[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        y[j] = alpha * X.val[e0 + j];
        if (diag && r == 32 * cs + j && I * SB + r < a.n) y[j] += delta;
      }
      float* dst = out.val + e0;
#pragma unroll
      for (int j = 0; j < 32; ++j) dst[j] = y[j];
      if constexpr (!kStaged<P>) {
        char* hp = static_cast<char*>(out.hi) + e0 * Prec<P>::eb;
        char* lp = out.lo ? static_cast<char*>(out.lo) + e0 * Prec<P>::eb : hp;
        store_operands<P>(y, hp, lp);
      }
    }
  }
}

// Final iterate -> BSR D (structure and FP64 values, plus dshift on the
// diagonal of the n x n block); TB_ERR_OOM in D.status when it holds more
// blocks than D.cap.  sel < 0: the SP2 iterate (buffer by the iteration
// count), else buffer sel.
__global__ void k_bsr_to_bsr(const SP2State* st, Args a, Buf b0, Buf b1, int sel, double dshift, tb_bsr D) {
  const Buf& b = (sel < 0 ? (st->iters & 1) : sel) ? b1 : b0;
  // after an error the iterate may never have been written: no blocks
  const int nblk = st->err ? 0 : min(b.row_ptr[a.nsb], a.cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) *D.status = nblk > D.cap ? TB_ERR_OOM : TB_OK;
  if (nblk > D.cap || st->err) {
    // an empty matrix: no row holds a block
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= a.nsb; i += gridDim.x * blockDim.x) D.row_ptr[i] = 0;
    return;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= a.nsb; i += gridDim.x * blockDim.x)
    D.row_ptr[i] = b.row_ptr[i];
  for (int o = blockIdx.x; o < nblk; o += gridDim.x) {
    const int J = b.col[o];
    if (threadIdx.x == 0) D.col[o] = J;
    const int I = dshift != 0.0 ? slot_row(b, a.nsb, o) : -1;
    const float* src = b.val + (size_t)o * kTiles;
    double* dst = D.val + (size_t)o * kTiles;
    for (int e = threadIdx.x; e < kTiles; e += blockDim.x) {
      const int r = e / SB;
      const bool dg = I == J && r == e % SB && I * SB + r < a.n;
      dst[e] = (double)src[e] + (dg ? dshift : 0.0);
    }
  }
}

__global__ void k_bsr_report(SP2State* st, Args a, Buf b0, Buf b1, tb_sp2_report* rep, int* nblk_out) {
  const Buf& b = (st->iters & 1) ? b1 : b0;
  if (nblk_out) *nblk_out = min(b.row_ptr[a.nsb], a.cap);
  if (!rep) return;
  const double t1 = st->t1[st->iters], t2 = st->t2[st->iters];
  int status = TB_OK;
  if (st->err) status = st->err;
  else if (fabs(t1 - a.nocc) > 0.25) status = TB_ERR_GAP;
  rep->status = status;
  rep->iters = st->iters;
  rep->refine_iters = 0;
  rep->n = a.n;
  rep->eps_min = st->emin;
  rep->eps_max = st->emax;
  rep->trace = t1;
  rep->idem_trace = t1 - t2;
  rep->idem_fro = -1.0;
  rep->branch_bits[0] = st->branch[0];
  rep->branch_bits[1] = st->branch[1];
  rep->refine_bits = 0;
  rep->block_products = (long long)st->block_products;
  rep->blocks = min(b.row_ptr[a.nsb], a.cap);
}

constexpr int kMaxBufs = 7;  // matrices of the Fermi expansion (SP2: two)

struct BsrLayout {
  int n, ld, nsb, cap, pcap, nbuf;
  bool staged;  // tf32x3: FP32 masters only, no stored operand splits
  size_t off_state, off_bparts, off_parts, off_scal, off_flags, off_cand, off_cnt, off_outrow, off_oldidx,
      off_pcnt, off_pptr, off_pairs, off_order;
  size_t off_rp[kMaxBufs], off_col[kMaxBufs], off_nz[kMaxBufs], off_st[kMaxBufs], off_lv[kMaxBufs],
      off_val[kMaxBufs], off_hi[kMaxBufs], off_lo[kMaxBufs];
  size_t total;
  int nparts;
};

// Workspace of nbuf block-sparse matrices of bpr blocks per block row on
// average (0: every block) and the shared symbolic arrays.
BsrLayout bsr_layout(int n, int prec, int bpr, int nbuf) {
  BsrLayout L{};
  L.n = n;
  L.ld = round_up(std::max(n, 1), SB);
  L.nsb = L.ld / SB;
  L.nbuf = nbuf;
  const int per_row = (bpr <= 0 || bpr > L.nsb) ? L.nsb : bpr;
  L.cap = L.nsb * per_row;
  L.pcap = L.cap * per_row;
  L.nparts = std::max(L.nsb, kMaxGrid);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o += (bytes + 1023) / 1024 * 1024;
    return r;
  };
  const size_t eb = (prec == TB_PREC_TF32 || prec == TB_PREC_TF32X3) ? 4 : 2;
  const bool split = prec == TB_PREC_TF32X3 || prec == TB_PREC_BF16X3;
  L.staged = prec == TB_PREC_TF32X3;
  L.off_state = take(sizeof(SP2State));
  L.off_bparts = take(sizeof(double) * 2 * std::max((n + 7) / 8, L.nsb));
  L.off_parts = take(sizeof(double) * 3 * 2 * L.nparts);
  L.off_scal = take(sizeof(int) * 4);
  L.off_flags = take(sizeof(uint16_t) * (size_t)L.nsb * L.nsb);
  L.off_cand = take(sizeof(uint32_t) * MW * L.nsb);
  L.off_cnt = take(sizeof(int) * L.nsb);
  L.off_outrow = take(sizeof(int) * L.cap);
  L.off_oldidx = take(sizeof(int) * L.cap);
  L.off_pcnt = take(sizeof(int) * L.cap);
  L.off_pptr = take(sizeof(int) * (L.cap + 1));
  L.off_pairs = take(sizeof(int2) * (size_t)L.pcap);
  L.off_order = take(sizeof(int) * L.cap);
  for (int b = 0; b < nbuf; ++b) {
    L.off_rp[b] = take(sizeof(int) * (L.nsb + 1));
    L.off_col[b] = take(sizeof(int) * L.cap);
    L.off_nz[b] = take(sizeof(int) * L.cap);
    L.off_st[b] = take(sizeof(uint32_t) * MW * L.nsb);
    L.off_lv[b] = take(sizeof(uint32_t) * MW * L.nsb);
    L.off_val[b] = take(sizeof(float) * (size_t)L.cap * kTiles);
    L.off_hi[b] = L.staged ? 0 : take(eb * (size_t)L.cap * kTiles);
    L.off_lo[b] = (split && !L.staged) ? take(eb * (size_t)L.cap * kTiles) : 0;
  }
  L.total = o;
  return L;
}

int make_block_map(tb_ctx* ctx, int prec, const void* base, int rows, CUtensorMap* map) {
  const bool tf = prec == TB_PREC_TF32 || prec == TB_PREC_TF32X3;
  const size_t eb = tf ? 4 : 2;
  const cuuint64_t dims[2] = {(cuuint64_t)SB, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(SB * eb)};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / eb), 128};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode_tiled(map, tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                 const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return tb_fail(ctx, TB_ERR_CUDA, "cuTensorMapEncodeTiled (blocks) failed (%d)", (int)r);
  return TB_OK;
}

// One block-sparse matrix of the workspace and the tensor maps of its operands.
struct Mat {
  Buf b;
  CUtensorMap mh, ml;
};

// The workspace bound to its parts.
struct Engine {
  BsrLayout L;
  SP2State* st;
  double* bparts;
  double* parts;  // two slots of 3 * nparts
  Sym sy;
  Mat m[kMaxBufs];
};

int bind_engine(tb_ctx* ctx, int prec, const BsrLayout& L, void* ws, Engine* e) {
  char* base = static_cast<char*>(ws);
  e->L = L;
  e->st = reinterpret_cast<SP2State*>(base + L.off_state);
  e->bparts = reinterpret_cast<double*>(base + L.off_bparts);
  e->parts = reinterpret_cast<double*>(base + L.off_parts);
  Sym& sy = e->sy;
  sy.cand = reinterpret_cast<uint32_t*>(base + L.off_cand);
  sy.cnt = reinterpret_cast<int*>(base + L.off_cnt);
  sy.out_row = reinterpret_cast<int*>(base + L.off_outrow);
  sy.old_idx = reinterpret_cast<int*>(base + L.off_oldidx);
  sy.pcnt = reinterpret_cast<int*>(base + L.off_pcnt);
  sy.pair_ptr = reinterpret_cast<int*>(base + L.off_pptr);
  sy.pairs = reinterpret_cast<int2*>(base + L.off_pairs);
  sy.scal = reinterpret_cast<int*>(base + L.off_scal);
  sy.order = reinterpret_cast<int*>(base + L.off_order);
  sy.flags = reinterpret_cast<uint16_t*>(base + L.off_flags);
  for (int i = 0; i < L.nbuf; ++i) {
    Buf& b = e->m[i].b;
    b.row_ptr = reinterpret_cast<int*>(base + L.off_rp[i]);
    b.col = reinterpret_cast<int*>(base + L.off_col[i]);
    b.nz = reinterpret_cast<int*>(base + L.off_nz[i]);
    b.stored = reinterpret_cast<uint32_t*>(base + L.off_st[i]);
    b.live = reinterpret_cast<uint32_t*>(base + L.off_lv[i]);
    b.val = reinterpret_cast<float*>(base + L.off_val[i]);
    b.hi = L.staged ? nullptr : base + L.off_hi[i];
    b.lo = L.off_lo[i] ? base + L.off_lo[i] : nullptr;
    // staged: the numeric kernel reads the FP32 masters (tf32 tiles of the same shape)
    int rc = make_block_map(ctx, prec, L.staged ? static_cast<void*>(b.val) : b.hi, L.cap * SB, &e->m[i].mh);
    if (rc) return rc;
    if (b.lo) {
      if ((rc = make_block_map(ctx, prec, b.lo, L.cap * SB, &e->m[i].ml))) return rc;
    } else {
      e->m[i].ml = e->m[i].mh;
    }
  }
  return TB_OK;
}

Args engine_args(const Engine& e, double tau) {
  Args a{};
  a.n = e.L.n;
  a.ld = e.L.ld;
  a.nsb = e.L.nsb;
  a.mw = (e.L.nsb + 31) / 32;
  a.cap = e.L.cap;
  a.pcap = e.L.pcap;
  a.tau2 = tau * tau;
  a.st = e.st;
  return a;
}

// X0 = s (e I - H) into out, with the drop, from a dense H (Hb null) or a BSR
// H; trace partials per block row into a.parts_out.
template <int P>
int launch_start(tb_ctx* ctx, Engine& e, const Args& a, const double* H, const tb_bsr* Hb, Mat& out,
                 cudaStream_t s) {
  const int nsb = e.L.nsb;
  if (Hb) {
    TB_CUDA_TRY(ctx, cudaMemsetAsync(e.sy.flags, 0, sizeof(uint16_t) * (size_t)nsb * nsb, s));
    k_bsr_init_flags_in<<<std::max(1, std::min(Hb->cap, 8192)), 256, 0, s>>>(*Hb, a, e.sy);
    TB_LAUNCH_CHECK(ctx);
    k_bsr_init_flags_diag<<<nsb, 256, 0, s>>>(*Hb, a, e.sy);
  } else {
    k_bsr_init_flags<<<dim3(nsb, nsb), 256, 0, s>>>(H, a, e.sy);
  }
  TB_LAUNCH_CHECK(ctx);
  k_bsr_init_rows<<<nsb, 256, 0, s>>>(a, e.sy, out.b);
  TB_LAUNCH_CHECK(ctx);
  k_bsr_scan_rows<<<1, 32, 0, s>>>(a, e.sy, out.b.row_ptr);
  TB_LAUNCH_CHECK(ctx);
  if (Hb) k_bsr_init_fill_in<P><<<nsb, 256, 0, s>>>(*Hb, a, e.sy, out.b);
  else k_bsr_init_fill<P><<<nsb, 256, 0, s>>>(H, a, e.sy, out.b);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// out = alpha A B + gamma S + delta I (S may be null), thresholded: the
// symbolic phase, then the persistent numeric kernel (trace partials per CTA
// into a.parts_out).  A and B are symmetric and their bitmaps current; out
// is none of A, B, S.  prof_k >= 0 marks the numeric launch for profiling.
template <int P>
int launch_product(tb_ctx* ctx, Engine& e, Args a, const Mat& A, const Mat& B, const Mat* S, Mat& out, Epi ep,
                   int grid, cudaStream_t s, int prof_k = -1) {
  a.same_ab = &A == &B;
  const Buf none{};
  const Buf& Sb = S ? S->b : none;
  const int nsb = e.L.nsb;
  k_bsr_cand<<<nsb, 256, 0, s>>>(a, A.b, B.b, Sb, e.sy);
  k_bsr_scan_rows<<<1, 32, 0, s>>>(a, e.sy, out.b.row_ptr);
  k_bsr_fill_out<<<nsb, 256, 0, s>>>(a, A.b, B.b, Sb, out.b, e.sy);
  k_bsr_scan_pairs<<<1, 1024, 0, s>>>(a, e.sy);
  k_bsr_pairs<<<std::max(1, std::min(e.L.cap, 4096) / 128 + 1), 128, 0, s>>>(a, A.b, B.b, out.b, e.sy);
  k_bsr_order<<<1, 1024, 0, s>>>(a, out.b, e.sy);
  TB_LAUNCH_CHECK(ctx);
  if (prof_k >= 0) tb_prof_mark(ctx, 1, 2 * prof_k, s);
  k_bsr_step_tc<P><<<grid, kNumThreads<P>, Prec<P>::smem_bytes, s>>>(a, A.mh, A.ml, B.mh, B.ml, Sb, out.b, e.sy, ep);
  TB_LAUNCH_CHECK(ctx);
  if (prof_k >= 0) tb_prof_mark(ctx, 1, 2 * prof_k + 1, s);
  return TB_OK;
}

template <int P>
int prepare_numeric(tb_ctx* ctx, int* grid) {
  static unsigned long long attr_done = 0;
  if (int rc = tb_smem_attr(ctx, k_bsr_step_tc<P>, Prec<P>::smem_bytes, &attr_done)) return rc;
  *grid = tb_persistent_grid(ctx, kMaxGrid);
  return TB_OK;
}

// H dense (Hb null) or BSR (Hb); D dense or BSR (Db).
template <int P>
int run_bsr(tb_ctx* ctx, const double* H, const tb_bsr* Hb, int n, double nocc, const tb_sp2_opts* o, double* D,
            tb_bsr* Db, void* ws, size_t ws_bytes, tb_sp2_report* rep, cudaStream_t s) {
  const BsrLayout L = bsr_layout(n, o->precision, o->bsr_blocks_per_row, 2);
  if (ws_bytes < L.total)
    return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu (block-sparse)", ws_bytes, L.total);
  Engine e;
  int rc = bind_engine(ctx, o->precision, L, ws, &e);
  if (rc) return rc;
  SP2State* st = e.st;
  double* slot[2] = {e.parts, e.parts + 3 * (size_t)L.nparts};
  Args a = engine_args(e, o->tau);
  a.nocc = nocc;
  a.tol = o->tol;
  a.rule = o->rule;
  a.max_iter = o->max_iter;
  {
    const double u = (o->precision == TB_PREC_TF32X3 || o->precision == TB_PREC_BF16X3) ? 0x1p-24
                     : o->precision == TB_PREC_TF32 ? 0x1p-11 : 0x1p-8;
    a.floor = 2.0 * n * u;
  }
  ctx->prof_n[0] = ctx->prof_n[1] = 0;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(SP2State), s));
  if (Hb) {
    k_bsr_status_in<<<1, 1, 0, s>>>(Hb->status, st);
    TB_LAUNCH_CHECK(ctx);
    k_bsr_bounds_in<<<L.nsb, 256, 0, s>>>(*Hb, e.bparts);
    TB_LAUNCH_CHECK(ctx);
    k_bsr_bounds<<<1, 32, 0, s>>>(e.bparts, L.nsb, st);
  } else {
    const int nb = (n + 7) / 8;
    if ((rc = sp2_launch_bounds(ctx, H, n, e.bparts, s))) return rc;
    k_bsr_bounds<<<1, 32, 0, s>>>(e.bparts, nb, st);
  }
  TB_LAUNCH_CHECK(ctx);
  a.parts_out = slot[0];
  if ((rc = launch_start<P>(ctx, e, a, H, Hb, e.m[0], s))) return rc;

  int grid = 0;
  if ((rc = prepare_numeric<P>(ctx, &grid))) return rc;
  // X^2 (branch 0) or 2X - X^2 (branch 1), the lo x lo product of a square
  const Epi sp2_epi{1.0f, 0.0f, -1.0f, 2.0f, 0.0f, 1, 1};
  tb_prof_mark(ctx, 0, 0, s);
  for (int k = 0; k <= o->max_iter; ++k) {
    a.k = k;
    a.parts_in = slot[k & 1];
    a.nparts_in = k == 0 ? L.nsb : grid;
    a.parts_out = slot[(k + 1) & 1];
    Mat& bo = e.m[k & 1];
    Mat& bn = e.m[(k + 1) & 1];
    k_bsr_decide<<<L.nsb, 128, 0, s>>>(a, bo.b);
    if ((rc = launch_product<P>(ctx, e, a, bo, bo, &bo, bn, sp2_epi, grid, s, k))) return rc;
    tb_prof_mark(ctx, 0, k + 1, s);
  }
  if (Db) {
    k_bsr_to_bsr<<<std::min(4096, std::max(1, L.cap)), 256, 0, s>>>(st, a, e.m[0].b, e.m[1].b, -1, 0.0, *Db);
  } else {
    TB_CUDA_TRY(ctx, cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, s));
    k_bsr_to_dense<<<std::min(4096, std::max(1, L.cap)), 256, 0, s>>>(st, a, e.m[0].b, e.m[1].b, e.sy, e.sy, D);
  }
  TB_LAUNCH_CHECK(ctx);
  k_bsr_report<<<1, 1, 0, s>>>(st, a, e.m[0].b, e.m[1].b, rep, nullptr);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// ------------------------------------------------ block-sparse Fermi expansion

constexpr int kFoeBufs = 7;  // E (two, alternating), Y, A, Z, T, W
constexpr int kFoeMinM = 8;

__global__ void k_bsr_fail(SP2State* st, int code) { st->err = code; }

__global__ void k_bsr_fermi_report(tb_fermi_report* rep, double* mu_out, int status, int iters, int m, int n,
                                   double mu, double trace, double trace_dd, double emin, double emax) {
  if (mu_out && status == TB_OK) *mu_out = mu;
  if (!rep) return;
  rep->status = status;
  rep->mu_iters = iters;
  rep->m = m;
  rep->n = n;
  rep->mu = mu;
  rep->trace = trace;
  rep->trace_dd = trace_dd;
  rep->eps_min = emin;
  rep->eps_max = emax;
}

// The recursive Fermi-operator expansion of dm_fermi on thresholded
// block-sparse products (every product and the start drop 32 x 32 blocks
// with Frobenius norm < tau; the affine steps are exact), the chemical
// potential by the host: one expansion per step, two traces read back.
template <int P>
int run_bsr_fermi(tb_ctx* ctx, const tb_bsr* Hb, int n, double nocc, double kT, const tb_fermi_opts* o,
                  double tau, int bpr, tb_bsr* Db, double* mu_dev, void* ws, size_t ws_bytes,
                  tb_fermi_report* rep, cudaStream_t s) {
  const BsrLayout L = bsr_layout(n, o->precision, bpr, kFoeBufs);
  if (ws_bytes < L.total)
    return tb_fail(ctx, TB_ERR_ARG, "workspace %zu bytes < required %zu (block-sparse)", ws_bytes, L.total);
  Engine e;
  int rc = bind_engine(ctx, o->precision, L, ws, &e);
  if (rc) return rc;
  SP2State* st = e.st;
  Args a = engine_args(e, tau);
  a.keep_diag = 1;
  a.parts_out = e.parts;
  const int m_max = o->m > 0 ? o->m : 14;
  const int ns = o->ns_iters > 0 ? o->ns_iters : 3;
  const double tol = o->trace_tol > 0.0 ? o->trace_tol : 1e-6 + 1e-9 * nocc;
  const double beta = 1.0 / kT;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(st, 0, sizeof(SP2State), s));
  k_bsr_status_in<<<1, 1, 0, s>>>(Hb->status, st);
  k_bsr_bounds_in<<<L.nsb, 256, 0, s>>>(*Hb, e.bparts);
  k_bsr_bounds<<<1, 32, 0, s>>>(e.bparts, L.nsb, st);
  TB_LAUNCH_CHECK(ctx);
  SP2State hs;
  double mu0 = NAN;
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(&hs, st, sizeof(SP2State), cudaMemcpyDeviceToHost, s));
  if (mu_dev) TB_CUDA_TRY(ctx, cudaMemcpyAsync(&mu0, mu_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  const double emin = hs.emin, emax = hs.emax;
  double lo = emin - 40.0 * kT - 1.0, hi = emax + 40.0 * kT + 1.0;
  int m = std::min(kFoeMinM, m_max);
  while (m < m_max && !(beta * (hi - lo) <= std::ldexp(1.0, m + 1))) ++m;
  double mu = (std::isfinite(mu0) && mu0 > lo && mu0 < hi) ? mu0 : 0.5 * (emin + emax);
  int status = hs.err ? hs.err : TB_ERR_NOT_CONVERGED;
  if (!hs.err && !(beta * (hi - lo) <= std::ldexp(1.0, m + 1))) status = TB_ERR_ARG;  // start undefined
  int grid = 0;
  if ((rc = prepare_numeric<P>(ctx, &grid))) return rc;
  std::vector<double> hp(3 * (size_t)grid);
  Mat* E[2] = {&e.m[0], &e.m[1]};
  Mat* Y = &e.m[2];
  Mat* A = &e.m[3];
  Mat* Z = &e.m[4];
  Mat* T = &e.m[5];
  Mat* W = &e.m[6];
  auto affine = [&](const Mat& X, Mat& out, float alpha, float delta) -> int {
    k_bsr_affine<P><<<std::min(4096, std::max(1, L.cap)), 256, 0, s>>>(a, X.b, out.b, alpha, delta);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  };
  auto product = [&](const Mat& X1, const Mat& X2, const Mat* S, Mat& out, Epi ep) -> int {
    int r = launch_product<P>(ctx, e, a, X1, X2, S, out, ep, grid, s);
    if (r) return r;
    k_bsr_bitmaps<<<L.nsb, 128, 0, s>>>(a, out.b);
    TB_LAUNCH_CHECK(ctx);
    return TB_OK;
  };
  const Epi plain{1.0f, 0.0f, 1.0f, 0.0f, 0.0f, 0, 0};
  auto with = [](float alpha, float gamma, float delta, int lolo) { return Epi{alpha, gamma, alpha, gamma, delta, 0, lolo}; };
  int it = 0, fin = 0;
  double trd = NAN, t1 = NAN;
  for (it = 1; status == TB_ERR_NOT_CONVERGED && it <= o->mu_iters; ++it) {
    // L = beta/2^(m+2) (mu I - H), then E0 = L - 4/3 L L^2
    a.x0_e = mu;
    a.x0_s = beta / std::ldexp(1.0, m + 2);
    if ((rc = launch_start<P>(ctx, e, a, nullptr, Hb, *Y, s))) return rc;
    a.x0_s = 0.0;
    if ((rc = product(*Y, *Y, nullptr, *A, with(1.0f, 0.0f, 0.0f, 1)))) return rc;
    if ((rc = product(*Y, *A, Y, *E[0], with(-4.0f / 3.0f, 1.0f, 0.0f, 0)))) return rc;
    int cur = 0;
    for (int step = 0; step < m; ++step) {
      Mat* Zc = Z;
      Mat* Yc = Y;
      // W = (I - 2E)(I + 2E), A = 2I - W
      if ((rc = affine(*E[cur], *T, -2.0f, 1.0f)) || (rc = affine(*E[cur], *Y, 2.0f, 1.0f))) return rc;
      if ((rc = product(*T, *Y, nullptr, *W, plain))) return rc;
      if ((rc = affine(*W, *A, -1.0f, 2.0f))) return rc;
      // Z1 = (32 A A - 144 A + 210 I) / 99, then Newton-Schulz Z <- Z (2I - A Z)
      if ((rc = product(*A, *A, A, *Zc, with(32.0f / 99.0f, -144.0f / 99.0f, 210.0f / 99.0f, 1)))) return rc;
      for (int k = 1; k < ns; ++k) {
        if ((rc = product(*A, *Zc, nullptr, *T, with(-1.0f, 0.0f, 2.0f, 0)))) return rc;
        if ((rc = product(*Zc, *T, nullptr, *Yc, plain))) return rc;
        std::swap(Zc, Yc);
      }
      // E <- E + E (Z W): the last product's partials are Tr E and ||E||_F^2
      if ((rc = product(*Zc, *W, nullptr, *T, plain))) return rc;
      if ((rc = product(*E[cur], *T, E[cur], *E[1 - cur], with(1.0f, 1.0f, 0.0f, 0)))) return rc;
      cur = 1 - cur;
    }
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(hp.data(), e.parts, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(&hs, st, sizeof(SP2State), cudaMemcpyDeviceToHost, s));
    TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hs.err) {
      status = hs.err;
      break;
    }
    double tr = 0.0, fro = 0.0;
    for (int i = 0; i < grid; ++i) {
      tr += hp[3 * i];
      fro += hp[3 * i + 1];
    }
    fin = cur;
    trd = 0.5 * n + tr;
    t1 = 0.25 * n - fro;  // Tr D(I - D) = n/4 - ||E||_F^2
    const double dev = trd - nocc;
    if (fabs(dev) <= tol) {
      status = TB_OK;
      break;
    }
    if (it == o->mu_iters) break;
    if (dev < 0.0) lo = mu;
    else hi = mu;
    mu = foe_next_mu(mu, dev, t1, beta, tol, lo, hi);
  }
  it = std::min(it, o->mu_iters);
  // D = I/2 + E; after an error (the state's flag, raised here for one the
  // host found) an empty matrix
  if (status != TB_OK && status != TB_ERR_NOT_CONVERGED) k_bsr_fail<<<1, 1, 0, s>>>(st, status);
  k_bsr_to_bsr<<<std::min(4096, std::max(1, L.cap)), 256, 0, s>>>(st, a, E[0]->b, E[1]->b, fin, 0.5, *Db);
  TB_LAUNCH_CHECK(ctx);
  k_bsr_fermi_report<<<1, 1, 0, s>>>(rep, mu_dev, status, it, m, n, mu, trd, t1, emin, emax);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

}  // namespace

int dm_sp2_bsr_workspace(int n, const tb_sp2_opts* o, int nsm, size_t* bytes) {
  if (n > kMaxNsb * SB) return TB_ERR_UNSUPPORTED;
  (void)nsm;
  *bytes = bsr_layout(n, o->precision, o->bsr_blocks_per_row, 2).total;
  return TB_OK;
}

int dm_sp2_bsr(tb_ctx* ctx, const double* H, int n, double nocc, const tb_sp2_opts* o, double* D, void* ws,
               size_t ws_bytes, tb_sp2_report* rep, cudaStream_t s) {
  if (n > kMaxNsb * SB) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse SP2 supports n <= %d", kMaxNsb * SB);
  switch (o->precision) {
    case TB_PREC_TF32: return run_bsr<TB_PREC_TF32>(ctx, H, nullptr, n, nocc, o, D, nullptr, ws, ws_bytes, rep, s);
    case TB_PREC_TF32X3: return run_bsr<TB_PREC_TF32X3>(ctx, H, nullptr, n, nocc, o, D, nullptr, ws, ws_bytes, rep, s);
    case TB_PREC_BF16: return run_bsr<TB_PREC_BF16>(ctx, H, nullptr, n, nocc, o, D, nullptr, ws, ws_bytes, rep, s);
    case TB_PREC_BF16X3: return run_bsr<TB_PREC_BF16X3>(ctx, H, nullptr, n, nocc, o, D, nullptr, ws, ws_bytes, rep, s);
    default: return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse SP2 needs a tensor-core precision");
  }
}

extern "C" int dm_sp2_sparse(tb_ctx* ctx, const tb_bsr* H, double nocc, const tb_sp2_opts* o, tb_bsr* D, void* ws,
                             size_t ws_bytes, tb_sp2_report* rep, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !D || !o || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_sp2_sparse");
  const int n = H->n;
  if (n < 1 || D->n != n || H->nsb != (n + SB - 1) / SB || D->nsb != H->nsb)
    return tb_fail(ctx, TB_ERR_ARG, "dm_sp2_sparse: inconsistent BSR sizes");
  if (!H->row_ptr || !H->col || !H->val || !D->row_ptr || !D->col || !D->val || !D->status)
    return tb_fail(ctx, TB_ERR_ARG, "dm_sp2_sparse: null BSR array");
  if (!(o->tau > 0.0)) return tb_fail(ctx, TB_ERR_ARG, "dm_sp2_sparse needs tau > 0");
  if (n > kMaxNsb * SB) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse SP2 supports n <= %d", kMaxNsb * SB);
  if (!(nocc >= 0.0) || nocc > n) return tb_fail(ctx, TB_ERR_ARG, "n_occ %g outside [0, n]", nocc);
  if (o->max_iter < 1 || o->max_iter > SP2_MAX_ITER)
    return tb_fail(ctx, TB_ERR_ARG, "max_iter %d outside 1..%d", o->max_iter, SP2_MAX_ITER);
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  switch (o->precision) {
    case TB_PREC_TF32: return run_bsr<TB_PREC_TF32>(ctx, nullptr, H, n, nocc, o, nullptr, D, ws, ws_bytes, rep, s);
    case TB_PREC_TF32X3: return run_bsr<TB_PREC_TF32X3>(ctx, nullptr, H, n, nocc, o, nullptr, D, ws, ws_bytes, rep, s);
    case TB_PREC_BF16: return run_bsr<TB_PREC_BF16>(ctx, nullptr, H, n, nocc, o, nullptr, D, ws, ws_bytes, rep, s);
    case TB_PREC_BF16X3: return run_bsr<TB_PREC_BF16X3>(ctx, nullptr, H, n, nocc, o, nullptr, D, ws, ws_bytes, rep, s);
    default: return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse SP2 needs a tensor-core precision");
  }
}

extern "C" int dm_fermi_sparse_workspace_size(int n, const tb_fermi_opts* o, int blocks_per_row, size_t* bytes) {
  if (n < 1 || !o || !bytes) return TB_ERR_ARG;
  if (n > kMaxNsb * SB) return TB_ERR_UNSUPPORTED;
  *bytes = bsr_layout(n, o->precision, blocks_per_row, kFoeBufs).total;
  return TB_OK;
}

extern "C" int dm_fermi_sparse(tb_ctx* ctx, const tb_bsr* H, double nocc, double kT, const tb_fermi_opts* o,
                               double tau, int blocks_per_row, tb_bsr* D, double* mu, void* ws, size_t ws_bytes,
                               tb_fermi_report* rep, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  if (!H || !D || !o || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to dm_fermi_sparse");
  const int n = H->n;
  if (n < 1 || D->n != n || H->nsb != (n + SB - 1) / SB || D->nsb != H->nsb)
    return tb_fail(ctx, TB_ERR_ARG, "dm_fermi_sparse: inconsistent BSR sizes");
  if (!H->row_ptr || !H->col || !H->val || !H->status || !D->row_ptr || !D->col || !D->val || !D->status)
    return tb_fail(ctx, TB_ERR_ARG, "dm_fermi_sparse: null BSR array");
  if (!(tau > 0.0)) return tb_fail(ctx, TB_ERR_ARG, "dm_fermi_sparse needs tau > 0");
  if (!(kT > 0.0)) return tb_fail(ctx, TB_ERR_ARG, "dm_fermi_sparse needs kT > 0");
  if (n > kMaxNsb * SB) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse expansion supports n <= %d", kMaxNsb * SB);
  if (!(nocc >= 0.0) || nocc > n) return tb_fail(ctx, TB_ERR_ARG, "n_occ %g outside [0, n]", nocc);
  if (o->mu_iters < 1 || o->mu_iters > 100) return tb_fail(ctx, TB_ERR_ARG, "mu_iters %d outside 1..100", o->mu_iters);
  if (o->m < 0 || o->m > 30 || o->ns_iters < 0 || o->ns_iters > 8)
    return tb_fail(ctx, TB_ERR_ARG, "dm_fermi_sparse: m or ns_iters out of range");
  if ((reinterpret_cast<uintptr_t>(ws) & 1023) != 0) return tb_fail(ctx, TB_ERR_ARG, "workspace must be 1024-byte aligned");
  cudaStream_t s = as_stream(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TB_CUDA_TRY(ctx, cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "dm_fermi_sparse reads traces on the host: not capturable");
  switch (o->precision) {
    case TB_PREC_TF32:
      return run_bsr_fermi<TB_PREC_TF32>(ctx, H, n, nocc, kT, o, tau, blocks_per_row, D, mu, ws, ws_bytes, rep, s);
    case TB_PREC_TF32X3:
      return run_bsr_fermi<TB_PREC_TF32X3>(ctx, H, n, nocc, kT, o, tau, blocks_per_row, D, mu, ws, ws_bytes, rep, s);
    case TB_PREC_BF16:
      return run_bsr_fermi<TB_PREC_BF16>(ctx, H, n, nocc, kT, o, tau, blocks_per_row, D, mu, ws, ws_bytes, rep, s);
    case TB_PREC_BF16X3:
      return run_bsr_fermi<TB_PREC_BF16X3>(ctx, H, n, nocc, kT, o, tau, blocks_per_row, D, mu, ws, ws_bytes, rep, s);
    default: return tb_fail(ctx, TB_ERR_UNSUPPORTED, "block-sparse expansion needs a tensor-core precision");
  }
}
