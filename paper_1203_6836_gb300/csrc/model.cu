// Orthogonal SCC tight-binding model on the GPU: H[n] build (a1), Mulliken
// charges (a7), forces and energy (a8).
//
//   H[n]_{ia,jb} = h_{ia,jb}(R) + delta_ij delta_ab sum_l gamma_il n_l
//       (App. D, Eq. DFTB_2 with S = I; Eq. EL_Orth_c)
//   q_i = 2 sum_{a in i} D_aa - N0_i                         (App. D)
//   E = 2 Tr[hD] + 1/2 (2q - n)^T gamma n + E_pair,  F = -dE/dR at fixed n
//       (Eq. EL_Orth_a, Eq. Etot_Orth; the D-derivative terms vanish for
//        D = theta(mu0 - H[n]) at fixed N_occ)
//
// Hopping: Slater-Koster two-centre table with ss-sigma = -V, sp-sigma = +V,
// pp-sigma = +V, pp-pi = -V sharing V(r) = zeta(r) = t exp(P(r)),
// P(r) = -r/r_decay + a2 r^2 + a3 r^3 + a4 r^4 (App. D's radial form); V and
// the pair potential (same form) are replaced on [r1, rcut) by the quintic
// tail of App. D.  gamma(r) = k/sqrt(r^2 + (k/U)^2) * (1-x)^4 (1+4x),
// x = r/gamma_cut (gamma_form 0), or the Ewald sum over all images of the
// Gaussian-charge interaction k erf(r/c)/r (gamma_form 1, k_gamma_ewald).
//
// Layout: H and D dense row-major n x n (FP64), orbitals grouped by atom;
// gamma dense N x N.  Pair work is done once per ordered or unordered atom
// pair by one thread or warp, so no atomics touch H; neighbours are found by
// a minimum-image screen in FP32 followed by an exact FP64 image loop.

#include "common.cuh"

#include <math.h>

// --------------------------------------------------------------------------
// host: tail coefficients (closed form of the six App. D conditions)
// --------------------------------------------------------------------------

// t(x) = B0 + B1 x + ... + B5 x^5 on x = R - r1 in [0, D], D = rcut - r1, with
// t, t', t'' equal to (f0, f1, f2) at x = 0 and zero at x = D.  B0..B2 follow
// directly; with y_k = B_k D^k the three end conditions read
//   y3 + y4 + y5 = -P0, 3y3 + 4y4 + 5y5 = -P1 D, 6y3 + 12y4 + 20y5 = -P2 D^2
// (P0, P1, P2 the value, slope and curvature of B0 + B1 x + B2 x^2 at D),
// solved by elimination below.
static void tail_closed_form(double f0, double f1, double f2, double r1, double rc, double B[6]) {
  const double D = rc - r1;
  B[0] = f0;
  B[1] = f1;
  B[2] = 0.5 * f2;
  const double P0 = B[0] + B[1] * D + B[2] * D * D;
  const double P1 = B[1] + 2.0 * B[2] * D;
  const double P2 = 2.0 * B[2];
  const double a = 3.0 * P0 - P1 * D;           // y4 + 2 y5
  const double b = 6.0 * P0 - P2 * D * D;       // 6 y4 + 14 y5
  const double y5 = 0.5 * (b - 6.0 * a);
  const double y4 = a - 2.0 * y5;
  const double y3 = -P0 - y4 - y5;
  B[3] = y3 / (D * D * D);
  B[4] = y4 / (D * D * D * D);
  B[5] = y5 / (D * D * D * D * D);
}

int tb_model_from_params(tb_ctx* ctx, const tb_params* p, double box, ModelDev* m) {
  if (!p) return tb_fail(ctx, TB_ERR_ARG, "null tb_params");
  if (!(p->rcut > p->r1) || !(p->r1 > 0) || !(p->r_decay > 0) || !(p->gamma_cut > 0) ||
      !(p->hubbard_u > 0) || !(box > 0) || (p->pair_a != 0.0 && !(p->pair_rho > 0)))
    return tb_fail(ctx, TB_ERR_ARG, "invalid model parameters");
  m->eps_s_O = p->eps_s_O;
  m->eps_p_O = p->eps_p_O;
  m->eps_s_H = p->eps_s_H;
  m->t_hop = p->t_hop;
  m->inv_decay = 1.0 / p->r_decay;
  m->U = p->hubbard_u;
  m->kc = p->coulomb_k;
  m->a2 = (p->coulomb_k / p->hubbard_u) * (p->coulomb_k / p->hubbard_u);
  m->gcut = p->gamma_cut;
  m->r1 = p->r1;
  m->rcut = p->rcut;
  m->n0_O = p->n0_O;
  m->n0_H = p->n0_H;
  m->pair_a = p->pair_a;
  m->inv_prho = p->pair_a != 0.0 ? 1.0 / p->pair_rho : 0.0;
  m->zhop[0] = p->zeta_a2;
  m->zhop[1] = p->zeta_a3;
  m->zhop[2] = p->zeta_a4;
  m->zpair[0] = p->pair_a2;
  m->zpair[1] = p->pair_a3;
  m->zpair[2] = p->pair_a4;
  // zeta, zeta', zeta'' at r1 for the tail: zeta' = P' zeta, zeta'' = (P'' + P'^2) zeta
  auto zeta3 = [&](double A0, double a1, const double* a, double r, double* f) {
    const double P = r * (a1 + r * (a[0] + r * (a[1] + r * a[2])));
    const double dP = a1 + r * (2.0 * a[0] + r * (3.0 * a[1] + r * 4.0 * a[2]));
    const double d2P = 2.0 * a[0] + r * (6.0 * a[1] + r * 12.0 * a[2]);
    const double v = A0 * exp(P);
    f[0] = v;
    f[1] = dP * v;
    f[2] = (d2P + dP * dP) * v;
  };
  double f[3];
  zeta3(p->t_hop, -m->inv_decay, m->zhop, p->r1, f);
  tail_closed_form(f[0], f[1], f[2], p->r1, p->rcut, m->Bhop);
  zeta3(p->pair_a, -m->inv_prho, m->zpair, p->r1, f);
  tail_closed_form(f[0], f[1], f[2], p->r1, p->rcut, m->Bpair);
  if (p->gamma_form != 0 && p->gamma_form != 1) return tb_fail(ctx, TB_ERR_ARG, "gamma_form %d", p->gamma_form);
  if (!(p->ewald_alpha >= 0.0)) return tb_fail(ctx, TB_ERR_ARG, "ewald_alpha %g < 0", p->ewald_alpha);
  m->gamma_form = p->gamma_form;
  m->range = p->gamma_form == 0 ? fmax(p->rcut, p->gamma_cut) : p->rcut;
  m->box = box;
  m->ealpha = p->ewald_alpha > 0.0 ? p->ewald_alpha : 6.5 / fmax(box, 10.0);
  m->gwidth = 2.0 * p->coulomb_k / (p->hubbard_u * sqrt(M_PI));
  m->erange = fmax(6.6 / m->ealpha, 6.6 * m->gwidth);
  m->gmax = 13.2 * m->ealpha;
  if (p->overlap_s0 != 0.0 && !(p->overlap_rs > 0.0))
    return tb_fail(ctx, TB_ERR_ARG, "overlap_rs %g must be > 0", p->overlap_rs);
  m->s0 = p->overlap_s0;
  m->inv_srs = p->overlap_s0 != 0.0 ? 1.0 / p->overlap_rs : 0.0;
  const double zero3[3] = {0.0, 0.0, 0.0};
  zeta3(p->overlap_s0, -m->inv_srs, zero3, p->r1, f);
  tail_closed_form(f[0], f[1], f[2], p->r1, p->rcut, m->Bov);
  return TB_OK;
}

// --------------------------------------------------------------------------
// device: radial functions
// --------------------------------------------------------------------------

__device__ __forceinline__ void tail_eval(const double* B, double x, double* f, double* df) {
  *f = B[0] + x * (B[1] + x * (B[2] + x * (B[3] + x * (B[4] + x * B[5]))));
  *df = B[1] + x * (2.0 * B[2] + x * (3.0 * B[3] + x * (4.0 * B[4] + x * 5.0 * B[5])));
}

// zeta(r) = A0 exp(P(r)), P(r) = a1 r + a2 r^2 + a3 r^3 + a4 r^4, and zeta'.
__device__ __forceinline__ void zeta(double A0, double a1, const double* a, double r, double* f, double* df) {
  const double P = r * (a1 + r * (a[0] + r * (a[1] + r * a[2])));
  const double dP = a1 + r * (2.0 * a[0] + r * (3.0 * a[1] + r * 4.0 * a[2]));
  const double v = A0 * exp(P);
  *f = v;
  *df = dP * v;
}

// V(r) and V'(r) of the hopping with its tail.
__device__ __forceinline__ void hop_radial(const ModelDev& m, double r, double* V, double* dV) {
  if (r < m.r1) {
    zeta(m.t_hop, -m.inv_decay, m.zhop, r, V, dV);
  } else if (r < m.rcut) {
    tail_eval(m.Bhop, r - m.r1, V, dV);
  } else {
    *V = 0.0;
    *dV = 0.0;
  }
}

// s(r) and s'(r) of the overlap with its tail.
__device__ __forceinline__ void ovl_radial(const ModelDev& m, double r, double* sv, double* dsv) {
  const double zero3[3] = {0.0, 0.0, 0.0};
  if (r < m.r1) {
    zeta(m.s0, -m.inv_srs, zero3, r, sv, dsv);
  } else if (r < m.rcut) {
    tail_eval(m.Bov, r - m.r1, sv, dsv);
  } else {
    *sv = 0.0;
    *dsv = 0.0;
  }
}

__device__ __forceinline__ void pair_radial(const ModelDev& m, double r, double* f, double* df) {
  if (m.pair_a == 0.0 || r >= m.rcut) {
    *f = 0.0;
    *df = 0.0;
  } else if (r < m.r1) {
    zeta(m.pair_a, -m.inv_prho, m.zpair, r, f, df);
  } else {
    tail_eval(m.Bpair, r - m.r1, f, df);
  }
}

__device__ __forceinline__ void gamma_radial(const ModelDev& m, double r, double* g, double* dg) {
  if (r >= m.gcut) {
    *g = 0.0;
    *dg = 0.0;
    return;
  }
  const double x = r / m.gcut, om = 1.0 - x;
  const double om3 = om * om * om;
  const double w = om3 * om * (1.0 + 4.0 * x);
  const double dw = (-4.0 * om3 * (1.0 + 4.0 * x) + 4.0 * om3 * om) / m.gcut;
  const double s = rsqrt(r * r + m.a2);
  const double ko = m.kc * s;
  const double dko = -m.kc * r * s * s * s;
  *g = ko * w;
  *dg = dko * w + ko * dw;
}

__device__ __forceinline__ int norb_of(int t) { return t == TB_TYPE_O ? 4 : 1; }

// Minimum-image displacement d = Rb - Ra in FP64.
__device__ __forceinline__ void min_image(const double* Ra, const double* Rb, double L,
                                          double d[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double x = Rb[c] - Ra[c];
    d[c] = x - L * rint(x / L);
  }
}

// FP32 screen: false when no periodic image of b lies within `range` of a.
// The minimum-image distance bounds every image distance from below; the
// margin covers FP32 rounding of coordinates up to ~1e4 A.
__device__ __forceinline__ bool screen_f32(const double* Ra, const double* Rb, float L,
                                           float range) {
  float r2 = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float x = (float)Rb[c] - (float)Ra[c];
    x -= L * rintf(x / L);
    r2 += x * x;
  }
  const float lim = range + 0.01f;
  return r2 < lim * lim;
}

// Image range along one axis: all k with |d + k L| < range.
__device__ __forceinline__ void image_range(double d, double L, double range, int* lo, int* hi) {
  *lo = (int)ceil((-range - d) / L);
  *hi = (int)floor((range - d) / L);
}

// --------------------------------------------------------------------------
// a1: H build
// --------------------------------------------------------------------------

// Slater-Koster block B (na x nb, row stride 4) for displacement d (a -> b).
__device__ __forceinline__ void sk_block(int ta, int tb, const double l[3], double V,
                                         double B[4][4]) {
  B[0][0] = -V;  // ss-sigma
  if (tb == TB_TYPE_O) {
#pragma unroll
    for (int c = 0; c < 3; ++c) B[0][1 + c] = l[c] * V;  // s_a - p_b
  }
  if (ta == TB_TYPE_O) {
#pragma unroll
    for (int c = 0; c < 3; ++c) B[1 + c][0] = -l[c] * V;  // p_a - s_b
  }
  if (ta == TB_TYPE_O && tb == TB_TYPE_O) {
    // l_c l_e (Vpp_sigma - Vpp_pi) + delta_ce Vpp_pi = 2V l_c l_e - V delta_ce
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int e = 0; e < 3; ++e) B[1 + c][1 + e] = 2.0 * V * l[c] * l[e] - (c == e ? V : 0.0);
  }
}

// One thread per unordered atom pair (i <= j): accumulate the hopping block
// and gamma over all periodic images, write both (i,j) and (j,i) blocks.
__global__ void __launch_bounds__(256) k_build_pairs(ModelDev m, int N, const int32_t* __restrict__ types,
                                                     const int32_t* __restrict__ offs,
                                                     const double* __restrict__ R,
                                                     double* __restrict__ H, int n,
                                                     double* __restrict__ G, double* __restrict__ S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (i >= N || j >= N || j < i) return;
  const double* Ri = R + 3 * i;
  const double* Rj = R + 3 * j;
  const int ti = types[i], tj = types[j];
  const int ni = norb_of(ti), nj = norb_of(tj);
  const int oi = offs[i], oj = offs[j];
  double B[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) B[a][b] = 0.0;
  double Bs[4][4];  // overlap block (S): unit on site, minus the table with s(r) between atoms
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) Bs[a][b] = (i == j && a == b) ? 1.0 : 0.0;
  const bool ovl = S != nullptr && m.s0 != 0.0;
  double gsum = (i == j) ? m.U : 0.0;
  if (S && i == j)
    for (int a = 0; a < ni; ++a) S[(size_t)(oi + a) * n + (oi + a)] = 1.0;
  // H, gamma (and S) were zeroed: pairs with no image in range write nothing
  // (gamma's window and h's tail both end at the cut-off)
  if (!(screen_f32(Ri, Rj, (float)m.box, (float)m.range) || i == j)) return;
  {
    double d0[3];
    min_image(Ri, Rj, m.box, d0);
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.range, &lo[c], &hi[c]);
    for (int kx = lo[0]; kx <= hi[0]; ++kx)
      for (int ky = lo[1]; ky <= hi[1]; ++ky)
        for (int kz = lo[2]; kz <= hi[2]; ++kz) {
          if (i == j && kx == 0 && ky == 0 && kz == 0) continue;
          const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
          const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          const double r = sqrt(r2);
          if (r >= m.range) continue;
          if (m.gamma_form == 0) {
            double g, dg;
            gamma_radial(m, r, &g, &dg);
            gsum += g;
          }
          if (r < m.rcut) {
            double V, dV;
            hop_radial(m, r, &V, &dV);
            const double l[3] = {d[0] / r, d[1] / r, d[2] / r};
            double Bi[4][4];
            sk_block(ti, tj, l, V, Bi);
            for (int a = 0; a < ni; ++a)
              for (int b = 0; b < nj; ++b) B[a][b] += Bi[a][b];
            if (ovl) {
              double sv, dsv;
              ovl_radial(m, r, &sv, &dsv);
              sk_block(ti, tj, l, sv, Bi);
              for (int a = 0; a < ni; ++a)
                for (int b = 0; b < nj; ++b) Bs[a][b] -= Bi[a][b];
            }
          }
        }
  }
  if (i == j) {
    // onsite energies on the diagonal of the (i,i) block
    if (ti == TB_TYPE_O) {
      B[0][0] += m.eps_s_O;
      B[1][1] += m.eps_p_O;
      B[2][2] += m.eps_p_O;
      B[3][3] += m.eps_p_O;
    } else {
      B[0][0] += m.eps_s_H;
    }
  }
  for (int a = 0; a < ni; ++a)
    for (int b = 0; b < nj; ++b) {
      H[(size_t)(oi + a) * n + (oj + b)] = B[a][b];
      if (i != j) H[(size_t)(oj + b) * n + (oi + a)] = B[a][b];
    }
  G[(size_t)i * N + j] = gsum;
  if (i != j) G[(size_t)j * N + i] = gsum;
  if (ovl)
    for (int a = 0; a < ni; ++a)
      for (int b = 0; b < nj; ++b) {
        S[(size_t)(oi + a) * n + (oj + b)] = Bs[a][b];
        if (i != j) S[(size_t)(oj + b) * n + (oi + a)] = Bs[a][b];
      }
}

// --------------------------------------------------------------------------
// long-range gamma (gamma_form 1): Gaussian charges, Ewald summation
// --------------------------------------------------------------------------
//
// gamma_ij = k sum_T erf(|d + T|/c)/|d + T|, d = R_j - R_i, split as
//   k [ sum_T (erfc(alpha r) - erfc(r/c))/r                  (real space, r = |d + T|)
//     + (4 pi/V) sum_{G != 0} e^{-G^2/4 alpha^2} cos(G.d)/G^2 - pi/(alpha^2 V) ]
// and on the diagonal (T = 0 left out of the real-space sum) U - 2 k alpha/sqrt(pi)
// added.  The reciprocal vectors G = 2 pi/L (h, k, l), |G| <= 13.2 alpha, are
// generated block-wise into shared memory (one per thread, weights with the
// factor 2 of the half space h > 0 | h = 0, k > 0 | h = k = 0, l > 0).

constexpr int kGChunk = 128;

struct GChunk {
  double gx[kGChunk], gy[kGChunk], gz[kGChunk], a[kGChunk];
};

// Fill chunk c (kGChunk cube indices starting at c * kGChunk) of the half-space
// reciprocal vectors: the weight is zero outside the sphere or the half space.
__device__ __forceinline__ void g_chunk(const ModelDev& m, int hmax, long long c, GChunk* s) {
  const long long side = 2 * hmax + 1;
  const long long idx = c * kGChunk + threadIdx.x % kGChunk;
  double gx = 0.0, gy = 0.0, gz = 0.0, w = 0.0;
  if (idx < side * side * side) {
    const int h = (int)(idx / (side * side)) - hmax;
    const int k = (int)((idx / side) % side) - hmax;
    const int l = (int)(idx % side) - hmax;
    const bool half = h > 0 || (h == 0 && (k > 0 || (k == 0 && l > 0)));
    const double tp = 2.0 * M_PI / m.box;
    gx = tp * h;
    gy = tp * k;
    gz = tp * l;
    const double g2 = gx * gx + gy * gy + gz * gz;
    if (half && g2 <= m.gmax * m.gmax) {
      const double V = m.box * m.box * m.box;
      w = 2.0 * 4.0 * M_PI / V * exp(-g2 / (4.0 * m.ealpha * m.ealpha)) / g2;
    }
  }
  if (threadIdx.x < kGChunk) {
    s->gx[threadIdx.x] = gx;
    s->gy[threadIdx.x] = gy;
    s->gz[threadIdx.x] = gz;
    s->a[threadIdx.x] = w;
  }
}

__device__ __forceinline__ int g_hmax(const ModelDev& m) { return (int)ceil(m.gmax * m.box / (2.0 * M_PI)); }

// Real-space part of gamma_ij / k and its gradient, images with r < erange.
__device__ __forceinline__ void ewald_real(const ModelDev& m, const double d0[3], bool self, double* v,
                                           double g[3]) {
  int lo[3], hi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.erange, &lo[c], &hi[c]);
  const double a = m.ealpha, ic = 1.0 / m.gwidth;
  const double ka = 2.0 * a / sqrt(M_PI), kc = 2.0 * ic / sqrt(M_PI);
  for (int kx = lo[0]; kx <= hi[0]; ++kx)
    for (int ky = lo[1]; ky <= hi[1]; ++ky)
      for (int kz = lo[2]; kz <= hi[2]; ++kz) {
        if (self && kx == 0 && ky == 0 && kz == 0) continue;
        const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (r >= m.erange) continue;
        const double f = (erfc(a * r) - erfc(r * ic)) / r;
        const double df = (-ka * exp(-a * a * r * r) + kc * exp(-r * r * ic * ic) - f) / r;
        *v += f;
#pragma unroll
        for (int c = 0; c < 3; ++c) g[c] += df * d[c] / r;
      }
}

// One thread per unordered pair (i <= j): gamma_ij and gamma_ji.
__global__ void __launch_bounds__(kGChunk) k_gamma_ewald(ModelDev m, int N, const double* __restrict__ R,
                                                         double* __restrict__ G) {
  __shared__ GChunk s;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  const bool live = i < N && j < N && j >= i;
  double d0[3] = {0.0, 0.0, 0.0};
  if (live) min_image(R + 3 * i, R + 3 * j, m.box, d0);
  double v = 0.0, gr[3] = {0.0, 0.0, 0.0};
  if (live) ewald_real(m, d0, i == j, &v, gr);
  const int hmax = g_hmax(m);
  const long long side = 2 * hmax + 1, chunks = (side * side * side + kGChunk - 1) / kGChunk;
  double rec = 0.0;
  for (long long c = 0; c < chunks; ++c) {
    __syncthreads();
    g_chunk(m, hmax, c, &s);
    __syncthreads();
    if (live)
      for (int t = 0; t < kGChunk; ++t)
        if (s.a[t] != 0.0) rec = fma(s.a[t], cos(s.gx[t] * d0[0] + s.gy[t] * d0[1] + s.gz[t] * d0[2]), rec);
  }
  if (!live) return;
  const double V = m.box * m.box * m.box;
  double gam = m.kc * (v + rec - M_PI / (m.ealpha * m.ealpha * V));
  if (i == j) gam += m.U - m.kc * 2.0 * m.ealpha / sqrt(M_PI);
  G[(size_t)i * N + j] = gam;
  if (i != j) G[(size_t)j * N + i] = gam;
}

// SCC forces of the long-range gamma: F_a += sum_{b != a} 1/2 (w_a n_b + w_b n_a)
// d gamma_ab / d d_ab (w = 2q - n, d = R_b - R_a).  One warp per atom a (8 per
// block, the reciprocal vectors shared by the block).
__global__ void __launch_bounds__(256) k_forces_ewald(ModelDev m, int N, const double* __restrict__ R,
                                                      const double* __restrict__ q,
                                                      const double* __restrict__ n_aux,
                                                      double* __restrict__ F) {
  __shared__ GChunk s;
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool live = a < N;
  const double wa = live ? 2.0 * q[a] - n_aux[a] : 0.0, na = live ? n_aux[a] : 0.0;
  double f[3] = {0.0, 0.0, 0.0};
  const int hmax = g_hmax(m);
  const long long side = 2 * hmax + 1, chunks = (side * side * side + kGChunk - 1) / kGChunk;
  // real space first (no shared memory), then the reciprocal part chunk by chunk
  if (live)
    for (int b = lane; b < N; b += 32) {
      if (b == a) continue;
      double d0[3], v = 0.0, g[3] = {0.0, 0.0, 0.0};
      min_image(R + 3 * a, R + 3 * b, m.box, d0);
      ewald_real(m, d0, false, &v, g);
      const double c = 0.5 * (wa * n_aux[b] + (2.0 * q[b] - n_aux[b]) * na) * m.kc;
#pragma unroll
      for (int k = 0; k < 3; ++k) f[k] += c * g[k];
    }
  for (long long ch = 0; ch < chunks; ++ch) {
    __syncthreads();
    if (threadIdx.x < kGChunk) g_chunk(m, hmax, ch, &s);
    __syncthreads();
    if (!live) continue;
    for (int b = lane; b < N; b += 32) {
      if (b == a) continue;
      double d0[3];
      min_image(R + 3 * a, R + 3 * b, m.box, d0);
      const double c = 0.5 * (wa * n_aux[b] + (2.0 * q[b] - n_aux[b]) * na) * m.kc;
      for (int t = 0; t < kGChunk; ++t) {
        if (s.a[t] == 0.0) continue;
        const double sn = sin(s.gx[t] * d0[0] + s.gy[t] * d0[1] + s.gz[t] * d0[2]);
        const double w = -c * s.a[t] * sn;
        f[0] += w * s.gx[t];
        f[1] += w * s.gy[t];
        f[2] += w * s.gz[t];
      }
    }
  }
  if (!live) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = warp_sum(f[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) F[3 * a + k] += f[k];
}

// SCC shift: one warp per atom i, shift_i = sum_l gamma_il n_l added to the
// diagonal of every orbital of atom i.
__global__ void __launch_bounds__(256) k_add_shift(int N, const int32_t* __restrict__ offs,
                                                   const double* __restrict__ G,
                                                   const double* __restrict__ n_aux,
                                                   double* __restrict__ H, int n) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N) return;
  const double* Gi = G + (size_t)warp * N;
  double s = 0.0;
  for (int l = lane; l < N; l += 32) s += Gi[l] * n_aux[l];
  s = warp_sum(s);
  if (lane == 0) {
    for (int a = offs[warp]; a < offs[warp + 1]; ++a) H[(size_t)a * n + a] += s;
  }
}

static int check_system(tb_ctx* ctx, const tb_system* sys) {
  if (!sys) return tb_fail(ctx, TB_ERR_ARG, "null tb_system");
  if (sys->natoms < 1 || sys->norb < 1 || !sys->types || !sys->orb_off || !(sys->box > 0))
    return tb_fail(ctx, TB_ERR_ARG, "invalid tb_system (natoms %d, norb %d, box %g)", sys->natoms,
                   sys->norb, sys->box);
  if (sys->natoms > 65535) return tb_fail(ctx, TB_ERR_ARG, "natoms > 65535 not supported");
  return TB_OK;
}

extern "C" int tb_build_H(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                          const double* n_aux, double* H, double* gamma, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !H || !gamma) return tb_fail(ctx, TB_ERR_ARG, "null R/H/gamma");
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  if (m.s0 != 0.0) return tb_fail(ctx, TB_ERR_ARG, "overlap_s0 != 0: the non-orthogonal H needs tb_build_HS");
  cudaStream_t s = as_stream(stream);
  const int N = sys->natoms, n = sys->norb;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(H, 0, sizeof(double) * (size_t)n * n, s));
  TB_CUDA_TRY(ctx, cudaMemsetAsync(gamma, 0, sizeof(double) * (size_t)N * N, s));
  dim3 grid((N + 255) / 256, N);
  k_build_pairs<<<grid, 256, 0, s>>>(m, N, sys->types, sys->orb_off, R, H, n, gamma, nullptr);
  TB_LAUNCH_CHECK(ctx);
  if (m.gamma_form == 1) {
    k_gamma_ewald<<<dim3((N + kGChunk - 1) / kGChunk, N), kGChunk, 0, s>>>(m, N, R, gamma);
    TB_LAUNCH_CHECK(ctx);
  }
  if (n_aux) {
    k_add_shift<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, sys->orb_off, gamma, n_aux, H, n);
    TB_LAUNCH_CHECK(ctx);
  }
  return TB_OK;
}

// v_i = sum_l gamma_il n_l, one warp per atom.
__global__ void __launch_bounds__(256) k_scc_potential(int N, const double* __restrict__ G,
                                                       const double* __restrict__ n_aux, double* __restrict__ v) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N) return;
  const double* Gi = G + (size_t)warp * N;
  double s = 0.0;
  for (int l = lane; l < N; l += 32) s += Gi[l] * n_aux[l];
  s = warp_sum(s);
  if (lane == 0) v[warp] = s;
}

// H_ab += S_ab (v_i(a) + v_j(b)) / 2 for the orbital rows of atom i = blockIdx.y
// (Eq. DFTB_2): each thread of the row block walks the columns, the column's atom
// found by bisection in the orbital offsets.
__global__ void __launch_bounds__(256) k_add_shift_nonorth(int N, const int32_t* __restrict__ offs,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ S,
                                                           double* __restrict__ H, int n) {
  const int i = blockIdx.y;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  int lo = 0, hi = N - 1;  // atom j with offs[j] <= b < offs[j + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const double vj = v[lo], vi = v[i];
  for (int a = offs[i]; a < offs[i + 1]; ++a) {
    const size_t e = (size_t)a * n + b;
    const double sab = S[e];
    if (sab != 0.0) H[e] += 0.5 * sab * (vi + vj);
  }
}

extern "C" int tb_build_HS(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                           const double* n_aux, double* H, double* S, double* gamma, double* v, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !H || !S || !gamma) return tb_fail(ctx, TB_ERR_ARG, "null R/H/S/gamma");
  if (n_aux && !v) return tb_fail(ctx, TB_ERR_ARG, "tb_build_HS with n_aux needs v");
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  const int N = sys->natoms, n = sys->norb;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(H, 0, sizeof(double) * (size_t)n * n, s));
  TB_CUDA_TRY(ctx, cudaMemsetAsync(S, 0, sizeof(double) * (size_t)n * n, s));
  TB_CUDA_TRY(ctx, cudaMemsetAsync(gamma, 0, sizeof(double) * (size_t)N * N, s));
  dim3 grid((N + 255) / 256, N);
  k_build_pairs<<<grid, 256, 0, s>>>(m, N, sys->types, sys->orb_off, R, H, n, gamma, S);
  TB_LAUNCH_CHECK(ctx);
  if (m.gamma_form == 1) {
    k_gamma_ewald<<<dim3((N + kGChunk - 1) / kGChunk, N), kGChunk, 0, s>>>(m, N, R, gamma);
    TB_LAUNCH_CHECK(ctx);
  }
  if (n_aux) {
    k_scc_potential<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, gamma, n_aux, v);
    TB_LAUNCH_CHECK(ctx);
    k_add_shift_nonorth<<<dim3((n + 255) / 256, N), 256, 0, s>>>(N, sys->orb_off, v, S, H, n);
    TB_LAUNCH_CHECK(ctx);
  }
  return TB_OK;
}

// --------------------------------------------------------------------------
// a7: Mulliken charges
// --------------------------------------------------------------------------

__global__ void k_mulliken(int N, const int32_t* __restrict__ types, const int32_t* __restrict__ offs,
                           const double* __restrict__ D, int n, double n0_O, double n0_H,
                           double* __restrict__ q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double pop = 0.0;
  for (int a = offs[i]; a < offs[i + 1]; ++a) pop += D[(size_t)a * n + a];
  q[i] = 2.0 * pop - (types[i] == TB_TYPE_O ? n0_O : n0_H);
}

// q_i = 2 sum_{a in i} (rho S)_aa - N0_i: one warp per atom, lanes over the
// columns of the rows of rho and S (S symmetric: (rho S)_aa = rho_a. . S_a.).
__global__ void __launch_bounds__(256) k_mulliken_nonorth(int N, const int32_t* __restrict__ types,
                                                          const int32_t* __restrict__ offs,
                                                          const double* __restrict__ rho,
                                                          const double* __restrict__ S, int n, double n0_O,
                                                          double n0_H, double* __restrict__ q) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N) return;
  double pop = 0.0;
  for (int a = offs[i]; a < offs[i + 1]; ++a) {
    const double* ra = rho + (size_t)a * n;
    const double* sa = S + (size_t)a * n;
    for (int b = lane; b < n; b += 32) pop += ra[b] * sa[b];
  }
  pop = warp_sum(pop);
  if (lane == 0) q[i] = 2.0 * pop - (types[i] == TB_TYPE_O ? n0_O : n0_H);
}

extern "C" int mulliken_nonorth(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* rho,
                                const double* S, double* q, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!p || !rho || !S || !q) return tb_fail(ctx, TB_ERR_ARG, "null argument to mulliken_nonorth");
  const int N = sys->natoms;
  k_mulliken_nonorth<<<(N * 32 + 255) / 256, 256, 0, as_stream(stream)>>>(N, sys->types, sys->orb_off, rho, S,
                                                                          sys->norb, p->n0_O, p->n0_H, q);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

extern "C" int mulliken(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* D,
                        double* q, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!p || !D || !q) return tb_fail(ctx, TB_ERR_ARG, "null argument to mulliken");
  const int N = sys->natoms;
  k_mulliken<<<(N + 127) / 128, 128, 0, as_stream(stream)>>>(N, sys->types, sys->orb_off, D, sys->norb,
                                                              p->n0_O, p->n0_H, q);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

// --------------------------------------------------------------------------
// a8: forces and energy
// --------------------------------------------------------------------------

// For the (a, b) block of D and displacement d (a -> b, |d| = r, l = d/r):
//   Eblk = sum_ab D_ab B_ab(d),  g_k = sum_ab D_ab dB_ab/dd_k.
// With u = D_sp - D_ps (s of one atom with p of the other), P = D_pp,
// S = P + P^T:
//   Eblk = -V D_ss + V u.l + 2V l^T P l - V tr P
//   g = -V' D_ss l + V (u - (u.l) l)/r + V' (u.l) l
//       + 2V (S l - (l^T S l) l)/r + V' (l^T S l) l - V' tr(P) l
template <class Get>
__device__ __forceinline__ void band_pair_g(int ta, int tb, Get Dg, const double l[3], double r, double V,
                                            double dV, double* Eblk, double g[3]) {
  const double Dss = Dg(0, 0);
  double u[3] = {0.0, 0.0, 0.0};
  if (tb == TB_TYPE_O)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] += Dg(0, 1 + c);
  if (ta == TB_TYPE_O)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] -= Dg(1 + c, 0);
  const double ul = u[0] * l[0] + u[1] * l[1] + u[2] * l[2];
  double E = -V * Dss + V * ul;
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = -dV * Dss * l[k] + V * (u[k] - ul * l[k]) / r + dV * ul * l[k];
  if (ta == TB_TYPE_O && tb == TB_TYPE_O) {
    double P[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int e = 0; e < 3; ++e) P[c][e] = Dg(1 + c, 1 + e);
    const double trP = P[0][0] + P[1][1] + P[2][2];
    double Sl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      Sl[c] = (P[c][0] + P[0][c]) * l[0] + (P[c][1] + P[1][c]) * l[1] + (P[c][2] + P[2][c]) * l[2];
    const double lSl = l[0] * Sl[0] + l[1] * Sl[1] + l[2] * Sl[2];  // = 2 l^T P l
    E += V * lSl - V * trP;
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] += 2.0 * V * (Sl[k] - lSl * l[k]) / r + dV * lSl * l[k] - dV * trP * l[k];
  }
  *Eblk = E;
}

// The same for the (a, b) block of a dense row-major D.
__device__ __forceinline__ void band_pair(int ta, int tb, const double* __restrict__ D, int n,
                                          int oa, int ob, const double l[3], double r, double V,
                                          double dV, double* Eblk, double g[3]) {
  band_pair_g(ta, tb, [&](int x, int y) { return D[(size_t)(oa + x) * n + ob + y]; }, l, r, V, dV, Eblk, g);
}

// One warp per atom a; lanes sweep all atoms b and their images.
// F_a = dE/dd summed over pairs (d = R_b - R_a + T), since dd/dR_a = -1.
// Per-atom energy shares are reduced with FP64 atomics into energy[1..3].
template <bool OVL>
__global__ void __launch_bounds__(256) k_forces(ModelDev m, int N, const int32_t* __restrict__ types,
                                                const int32_t* __restrict__ offs,
                                                const double* __restrict__ R,
                                                const double* __restrict__ D, int n,
                                                const double* __restrict__ q,
                                                const double* __restrict__ n_aux,
                                                const double* __restrict__ G,
                                                double* __restrict__ F, double* __restrict__ energy,
                                                const double* __restrict__ W,
                                                const double* __restrict__ vscc) {
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (a >= N) return;
  const double* Ra = R + 3 * a;
  const int ta = types[a], oa = offs[a];
  const double wa = 2.0 * q[a] - n_aux[a];
  const double na = n_aux[a];
  double f[3] = {0.0, 0.0, 0.0};
  double e_band = 0.0, e_pair = 0.0, e_scc = 0.0;
  // Pass 1 (lanes over all b): the gamma-n sum and an FP32 screen; the atoms b
  // with an image in range are compacted into a shared-memory list.  Pass 2:
  // all 32 lanes work through the list (about 3 of every 32 atoms are in range
  // at 1 g/cc), each lane summing its entries in list order.
  constexpr int kNb = 512;
  __shared__ int s_nb_all[8][kNb];  // one list per warp (up to 256 threads)
  int* s_nb = s_nb_all[threadIdx.x >> 5];
  auto pair_terms = [&](int b) {
    const double* Rb = R + 3 * b;
    const int tb = types[b], ob = offs[b];
    const double wb = 2.0 * q[b] - n_aux[b];
    const double nb = n_aux[b];
    double d0[3];
    min_image(Ra, Rb, m.box, d0);
    int lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.range, &lo[c], &hi[c]);
    for (int kx = lo[0]; kx <= hi[0]; ++kx)
      for (int ky = lo[1]; ky <= hi[1]; ++ky)
        for (int kz = lo[2]; kz <= hi[2]; ++kz) {
          if (b == a && kx == 0 && ky == 0 && kz == 0) continue;
          const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
          const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          if (r >= m.range) continue;
          const double l[3] = {d[0] / r, d[1] / r, d[2] / r};
          if (r < m.rcut) {
            double V, dV;
            hop_radial(m, r, &V, &dV);
            double Eblk, g[3];
            band_pair(ta, tb, D, n, oa, ob, l, r, V, dV, &Eblk, g);
            if (b != a) {
              // unordered pair energy 4*Eblk, shared half per atom
              e_band += 2.0 * Eblk;
#pragma unroll
              for (int k = 0; k < 3; ++k) f[k] += 4.0 * g[k];
            } else {
              e_band += 2.0 * Eblk;  // self-image block of h_aa
            }
            if constexpr (OVL) if (b != a) {
              // overlap terms: Tr[(V rho + rho V - 2 W) S] over the blocks (a,b) and
              // (b,a); S's block is minus the table with s(r), and V is v_a, v_b on
              // the two atoms' orbitals
              double sv, dsv, Er, Ew, gr[3], gw[3];
              ovl_radial(m, r, &sv, &dsv);
              band_pair(ta, tb, D, n, oa, ob, l, r, sv, dsv, &Er, gr);
              band_pair(ta, tb, W, n, oa, ob, l, r, sv, dsv, &Ew, gw);
              const double vv = vscc[a] + vscc[b];
#pragma unroll
              for (int k = 0; k < 3; ++k) f[k] -= 2.0 * (vv * gr[k] - 2.0 * gw[k]);
            }
            double ph, dph;
            pair_radial(m, r, &ph, &dph);
            e_pair += 0.5 * ph;
            if (b != a)
#pragma unroll
              for (int k = 0; k < 3; ++k) f[k] += dph * l[k];
          }
          if (b != a && m.gamma_form == 0) {
            double gg, dgg;
            gamma_radial(m, r, &gg, &dgg);
            const double c = 0.5 * (wa * nb + wb * na) * dgg;
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] += c * l[k];
          }
        }
    };
  int cnt = 0;
  for (int b0 = 0; b0 < N; b0 += 32) {
    const int b = b0 + lane;
    bool hit = false;
    if (b < N) {
      e_scc += G[(size_t)a * N + b] * n_aux[b];
      hit = b == a || screen_f32(Ra, R + 3 * b, (float)m.box, (float)m.range);
    }
    const unsigned mk = __ballot_sync(0xffffffffu, hit);
    if (hit) s_nb[cnt + __popc(mk & ((1u << lane) - 1u))] = b;
    cnt += __popc(mk);
    if (cnt > kNb - 32 || b0 + 32 >= N) {
      __syncwarp();
      for (int e = lane; e < cnt; e += 32) pair_terms(s_nb[e]);
      __syncwarp();
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = warp_sum(f[k]);
  e_band = warp_sum(e_band);
  e_pair = warp_sum(e_pair);
  e_scc = warp_sum(e_scc);
  if (lane == 0) {
    // onsite part of 2 Tr[hD]
    if (ta == TB_TYPE_O) {
      e_band += 2.0 * (m.eps_s_O * D[(size_t)oa * n + oa] +
                       m.eps_p_O * (D[(size_t)(oa + 1) * n + oa + 1] + D[(size_t)(oa + 2) * n + oa + 2] +
                                    D[(size_t)(oa + 3) * n + oa + 3]));
    } else {
      e_band += 2.0 * m.eps_s_H * D[(size_t)oa * n + oa];
    }
    e_scc *= 0.5 * wa;
    F[3 * a + 0] = f[0];
    F[3 * a + 1] = f[1];
    F[3 * a + 2] = f[2];
    atomicAdd(&energy[1], e_band);
    atomicAdd(&energy[2], e_scc);
    atomicAdd(&energy[3], e_pair);
    atomicAdd(&energy[0], e_band + e_scc + e_pair);
  }
}

extern "C" int tb_forces(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                         const double* D, const double* q, const double* n_aux, const double* gamma,
                         double* F, double* energy, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !D || !q || !n_aux || !gamma || !F || !energy)
    return tb_fail(ctx, TB_ERR_ARG, "null argument to tb_forces");
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  if (m.s0 != 0.0) return tb_fail(ctx, TB_ERR_ARG, "overlap_s0 != 0: forces need tb_forces_nonorth");
  cudaStream_t s = as_stream(stream);
  TB_CUDA_TRY(ctx, cudaMemsetAsync(energy, 0, 4 * sizeof(double), s));
  const int N = sys->natoms;
  // one warp per atom, one warp per block: FP64 runs at ~8 GFLOP/s per SM on
  // GB300, so small systems spread their atoms over as many SMs as possible
  k_forces<false><<<N, 32, 0, s>>>(m, N, sys->types, sys->orb_off, R, D, sys->norb, q,
                                                  n_aux, gamma, F, energy, nullptr, nullptr);
  TB_LAUNCH_CHECK(ctx);
  if (m.gamma_form == 1) {
    k_forces_ewald<<<(N + 7) / 8, 256, 0, s>>>(m, N, R, q, n_aux, F);
    TB_LAUNCH_CHECK(ctx);
  }
  return TB_OK;
}

extern "C" int tb_forces_nonorth(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                                 const double* rho, const double* W, const double* q, const double* n_aux,
                                 const double* v, const double* gamma, double* F, double* energy, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !rho || !W || !q || !n_aux || !v || !gamma || !F || !energy)
    return tb_fail(ctx, TB_ERR_ARG, "null argument to tb_forces_nonorth");
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  TB_CUDA_TRY(ctx, cudaMemsetAsync(energy, 0, 4 * sizeof(double), s));
  const int N = sys->natoms;
  if (m.s0 != 0.0)
    k_forces<true><<<N, 32, 0, s>>>(m, N, sys->types, sys->orb_off, R, rho, sys->norb, q, n_aux, gamma, F,
                                    energy, W, v);
  else
    k_forces<false><<<N, 32, 0, s>>>(m, N, sys->types, sys->orb_off, R, rho, sys->norb, q, n_aux, gamma, F,
                                     energy, nullptr, nullptr);
  TB_LAUNCH_CHECK(ctx);
  if (m.gamma_form == 1) {
    k_forces_ewald<<<(N + 7) / 8, 256, 0, s>>>(m, N, R, q, n_aux, F);
    TB_LAUNCH_CHECK(ctx);
  }
  return TB_OK;
}

// --------------------------------------------------------------------------
// a5 boundary: H, Mulliken charges and forces with block-sparse (BSR) matrices
// --------------------------------------------------------------------------
//
// Block row I holds orbitals [128 I, 128 I + 128); its atoms are those with an
// orbital there (an atom's orbitals may straddle two block rows).  The pattern
// of H stores block (I, J) when the bounding boxes of the two rows' atoms come
// within the model's range under the periodic minimum image, so every atom
// pair within range lies in a stored block; the atom pairs of a block are
// found from the two atom ranges, and the neighbours of an atom from its block
// row's stored columns.

namespace {

constexpr int kBB = 128;  // BSR block side (TB_BSR_BLOCK)

struct BsrModelWs {
  int* atom_lo;      // [nsb]
  int* atom_hi;      // [nsb] (exclusive)
  double* bbox;      // [nsb * 6]: centre xyz, half-extent xyz
  uint8_t* flags;    // [nsb * nsb]
  int* cnt;          // [nsb]
};

size_t bsr_model_bytes(int N, int nsb, BsrModelWs* w, void* base) {
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t r = o;
    o += (b + 255) / 256 * 256;
    return r;
  };
  const size_t a = take(sizeof(int) * nsb), b = take(sizeof(int) * nsb), c = take(sizeof(double) * 6 * nsb),
               d = take((size_t)nsb * nsb), e = take(sizeof(int) * nsb);
  (void)N;
  if (w && base) {
    char* p = static_cast<char*>(base);
    w->atom_lo = reinterpret_cast<int*>(p + a);
    w->atom_hi = reinterpret_cast<int*>(p + b);
    w->bbox = reinterpret_cast<double*>(p + c);
    w->flags = reinterpret_cast<uint8_t*>(p + d);
    w->cnt = reinterpret_cast<int*>(p + e);
  }
  return o;
}

__device__ __forceinline__ int bsr_slot(const int* __restrict__ row_ptr, const int* __restrict__ col, int I, int J) {
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

// Element (r, c) of a BSR matrix (0 where no block is stored).
__device__ __forceinline__ double bsr_get(const tb_bsr& M, int r, int c) {
  const int s = bsr_slot(M.row_ptr, M.col, r / kBB, c / kBB);
  return s < 0 ? 0.0 : M.val[(size_t)s * kBB * kBB + (size_t)(r % kBB) * kBB + (c % kBB)];
}

// First atom with an orbital at or after orbital a: offs[i + 1] > a.
__device__ __forceinline__ int atom_from(const int32_t* offs, int N, int a) {
  int lo = 0, hi = N;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (offs[mid + 1] > a) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void k_blk_atoms(int N, int n, int nsb, const int32_t* __restrict__ offs, BsrModelWs w) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nsb) return;
  const int r0 = I * kBB, r1 = min(n, r0 + kBB);
  w.atom_lo[I] = atom_from(offs, N, r0);
  w.atom_hi[I] = atom_from(offs, N, r1);  // first atom starting at or after r1 ... below
  // atoms with an orbital in [r0, r1): offs[i + 1] > r0 and offs[i] < r1
  int hi = w.atom_hi[I];
  while (hi < N && offs[hi] < r1) ++hi;
  w.atom_hi[I] = hi;
}

// Bounding box of block row I's atoms in the minimum-image frame of its first atom.
__global__ void __launch_bounds__(128) k_blk_box(ModelDev m, const double* __restrict__ R, int nsb, BsrModelWs w) {
  __shared__ double red[6][4];
  const int I = blockIdx.x;
  const int lo = w.atom_lo[I], hi = w.atom_hi[I];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  const double* R0 = R + 3 * lo;
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double d[3];
    min_image(R0, R + 3 * i, m.box, d);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      mn[k] = fmin(mn[k], d[k]);
      mx[k] = fmax(mx[k], d[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mn[k] = warp_min(mn[k]);
    mx[k] = warp_max(mx[k]);
  }
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) {
      red[k][threadIdx.x >> 5] = mn[k];
      red[3 + k][threadIdx.x >> 5] = mx[k];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      const double a = fmin(fmin(red[k][0], red[k][1]), fmin(red[k][2], red[k][3]));
      const double b = fmax(fmax(red[3 + k][0], red[3 + k][1]), fmax(red[3 + k][2], red[3 + k][3]));
      const double ok = hi > lo;
      w.bbox[6 * I + k] = ok ? R0[k] + 0.5 * (a + b) : 0.0;
      w.bbox[6 * I + 3 + k] = ok ? 0.5 * (b - a) : 0.0;
    }
  }
}

// flags[I][J] = 1 when the boxes of rows I and J come within `range` (periodic
// minimum image per axis; an axis whose boxes and range span half the box or
// more is not used to exclude).
__global__ void k_blk_pattern(ModelDev m, int nsb, BsrModelWs w) {
  const int I = blockIdx.x;
  for (int J = threadIdx.x; J < nsb; J += blockDim.x) {
    double g2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      double dc = w.bbox[6 * J + k] - w.bbox[6 * I + k];
      dc -= m.box * rint(dc / m.box);
      const double hs = w.bbox[6 * I + 3 + k] + w.bbox[6 * J + 3 + k];
      if (hs + m.range >= 0.5 * m.box) continue;
      const double gap = fmax(0.0, fabs(dc) - hs);
      g2 += gap * gap;
    }
    w.flags[(size_t)I * nsb + J] = (I == J || g2 < m.range * m.range) ? 1 : 0;
  }
}

__global__ void k_blk_count(int nsb, BsrModelWs w) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nsb) return;
  int c = 0;
  for (int J = 0; J < nsb; ++J) c += w.flags[(size_t)I * nsb + J];
  w.cnt[I] = c;
}

// row_ptr by a serial scan, OOM status, then each row's columns in order.
__global__ void k_blk_scan(int nsb, BsrModelWs w, tb_bsr H) {
  if (threadIdx.x != 0) return;
  int s = 0;
  for (int I = 0; I < nsb; ++I) {
    H.row_ptr[I] = s;
    s += w.cnt[I];
  }
  H.row_ptr[nsb] = s;
  *H.status = s > H.cap ? TB_ERR_OOM : TB_OK;
}

__global__ void k_blk_cols(int nsb, BsrModelWs w, tb_bsr H) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nsb || *H.status != TB_OK) return;
  int o = H.row_ptr[I];
  for (int J = 0; J < nsb; ++J)
    if (w.flags[(size_t)I * nsb + J]) H.col[o++] = J;
}

// Whether block row J's atom box can come within m.range of the point x under
// the periodic images (k_blk_pattern's test with a box of zero extent), in
// FP32 with a 1e-3 A margin, so that it errs only towards visiting a block.
__device__ __forceinline__ bool box_in_range(const ModelDev& m, const BsrModelWs& w, int J, const float (&x)[3]) {
  const float box = (float)m.box, reach = (float)m.range + 1e-3f;
  float g2 = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float dc = (float)w.bbox[6 * J + k] - x[k];
    dc -= box * rintf(dc / box);
    const float hs = (float)w.bbox[6 * J + 3 + k];
    if (hs + reach >= 0.5f * box) continue;
    const float gap = fmaxf(0.0f, fabsf(dc) - hs);
    g2 += gap * gap;
  }
  return g2 < reach * reach;
}

// The h elements of stored block o (one CTA per block, grid-stride): every
// ordered atom pair (i, j) of the two rows, summed over the images within the
// cut-off, onsite energies for i == j; each element belongs to one pair.
__global__ void __launch_bounds__(256) k_h_blocks(ModelDev m, int N, const int32_t* __restrict__ types,
                                                  const int32_t* __restrict__ offs, const double* __restrict__ R,
                                                  BsrModelWs w, tb_bsr H) {
  __shared__ int s_near[kBB];  // a block row holds at most kBB atoms (each has an orbital in it)
  __shared__ int s_nnear;
  if (*H.status != TB_OK) return;
  const int nblk = H.row_ptr[H.nsb];
  for (int o = blockIdx.x; o < nblk; o += gridDim.x) {
    int lo = 0, hi = H.nsb;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (H.row_ptr[mid] <= o) lo = mid;
      else hi = mid;
    }
    const int I = lo, J = H.col[o];
    double* blk = H.val + (size_t)o * kBB * kBB;
    for (int e = threadIdx.x; e < kBB * kBB; e += blockDim.x) blk[e] = 0.0;
    __syncthreads();
    const int ilo = w.atom_lo[I], ihi = w.atom_hi[I], jlo = w.atom_lo[J], jhi = w.atom_hi[J];
    // the atoms of row block I within range of column block J's atom box (the
    // others only have zero elements in this block): one warp, ballots
    if (threadIdx.x < 32) {
      int cnt = 0;
      for (int base = ilo; base < ihi; base += 32) {
        const int i = base + (int)threadIdx.x;
        bool ok = false;
        if (i < ihi) {
          const float xf[3] = {(float)R[3 * i], (float)R[3 * i + 1], (float)R[3 * i + 2]};
          ok = box_in_range(m, w, J, xf);
        }
        const unsigned msk = __ballot_sync(0xffffffffu, ok);
        if (ok) s_near[cnt + __popc(msk & ((1u << threadIdx.x) - 1u))] = i;
        cnt += __popc(msk);
      }
      if (threadIdx.x == 0) s_nnear = cnt;
    }
    __syncthreads();
    const int nj = jhi - jlo, npair = s_nnear * nj;
    const int r0 = I * kBB, c0 = J * kBB;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
      const int i = s_near[p / nj], j = jlo + p % nj;
      const int ti = types[i], tj = types[j];
      const int ni = norb_of(ti), njo = norb_of(tj);
      const int oi = offs[i], oj = offs[j];
      double B[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) B[a][b] = 0.0;
      const double* Ri = R + 3 * i;
      const double* Rj = R + 3 * j;
      if (i == j || screen_f32(Ri, Rj, (float)m.box, (float)m.rcut)) {
        double d0[3];
        min_image(Ri, Rj, m.box, d0);
        int lo3[3], hi3[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.rcut, &lo3[c], &hi3[c]);
        for (int kx = lo3[0]; kx <= hi3[0]; ++kx)
          for (int ky = lo3[1]; ky <= hi3[1]; ++ky)
            for (int kz = lo3[2]; kz <= hi3[2]; ++kz) {
              if (i == j && kx == 0 && ky == 0 && kz == 0) continue;
              const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
              const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
              if (r >= m.rcut) continue;
              double V, dV;
              hop_radial(m, r, &V, &dV);
              const double l[3] = {d[0] / r, d[1] / r, d[2] / r};
              double Bi[4][4];
              sk_block(ti, tj, l, V, Bi);
              for (int a = 0; a < ni; ++a)
                for (int b = 0; b < njo; ++b) B[a][b] += Bi[a][b];
            }
      }
      if (i == j) {
        if (ti == TB_TYPE_O) {
          B[0][0] += m.eps_s_O;
          B[1][1] += m.eps_p_O;
          B[2][2] += m.eps_p_O;
          B[3][3] += m.eps_p_O;
        } else {
          B[0][0] += m.eps_s_H;
        }
      }
      for (int a = 0; a < ni; ++a) {
        const int r = oi + a - r0;
        if (r < 0 || r >= kBB) continue;
        for (int b = 0; b < njo; ++b) {
          const int c = oj + b - c0;
          if (c < 0 || c >= kBB) continue;
          blk[(size_t)r * kBB + c] = B[a][b];
        }
      }
    }
    __syncthreads();
  }
}

// Visit the atoms of the stored block columns of row I once each (consecutive
// block rows share at most their straddling atom): fn(j), skipping the blocks
// whose atom box lies beyond m.range of the point x (their atoms, the
// straddling one included, are out of range and contribute nothing).  The
// lanes test 32 blocks at a time.
template <class Fn>
__device__ __forceinline__ void for_neighbour_atoms(const tb_bsr& H, const BsrModelWs& w, const ModelDev& m, int I,
                                                    const double* x, int lane, Fn fn) {
  const float xf[3] = {(float)x[0], (float)x[1], (float)x[2]};
  const int s1 = H.row_ptr[I + 1];
  int next = 0;
  for (int s0 = H.row_ptr[I]; s0 < s1; s0 += 32) {
    const bool near = s0 + lane < s1 && box_in_range(m, w, H.col[s0 + lane], xf);
    const unsigned mask = __ballot_sync(0xffffffffu, near);
    const int cnt = min(32, s1 - s0);
    for (int t = 0; t < cnt; ++t) {
      const int J = H.col[s0 + t];
      const int lo = max(next, w.atom_lo[J]), hi = w.atom_hi[J];
      if ((mask >> t) & 1u)
        for (int j = lo + lane; j < hi; j += 32) fn(j);
      next = max(next, hi);
    }
  }
}

// v_i = sum_l gamma_il n_l over the atoms within range (windowed gamma, its
// on-site U and the self-images): one warp per atom.
__global__ void __launch_bounds__(256) k_v_bsr(ModelDev m, int N, const int32_t* __restrict__ offs,
                                               const double* __restrict__ R, const double* __restrict__ n_aux,
                                               tb_bsr H, BsrModelWs w, double* __restrict__ v) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= N || *H.status != TB_OK) return;  // an overflowed pattern has no columns to visit
  const double* Ri = R + 3 * i;
  double s = 0.0;
  for_neighbour_atoms(H, w, m, offs[i] / kBB, Ri, lane, [&](int j) {
    const double* Rj = R + 3 * j;
    if (j != i && !screen_f32(Ri, Rj, (float)m.box, (float)m.gcut)) return;
    double d0[3];
    min_image(Ri, Rj, m.box, d0);
    int lo3[3], hi3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.gcut, &lo3[c], &hi3[c]);
    double g = 0.0;
    for (int kx = lo3[0]; kx <= hi3[0]; ++kx)
      for (int ky = lo3[1]; ky <= hi3[1]; ++ky)
        for (int kz = lo3[2]; kz <= hi3[2]; ++kz) {
          if (j == i && kx == 0 && ky == 0 && kz == 0) continue;
          const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
          const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          if (r >= m.gcut) continue;
          double gg, dgg;
          gamma_radial(m, r, &gg, &dgg);
          g += gg;
        }
    s += g * n_aux[j];
  });
  s = warp_sum(s);
  if (lane == 0) v[i] = s + m.U * n_aux[i];
}

// H_aa += v_i on every orbital a of atom i.
__global__ void k_shift_bsr(int N, const int32_t* __restrict__ offs, const double* __restrict__ v, tb_bsr H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *H.status != TB_OK) return;
  for (int a = offs[i]; a < offs[i + 1]; ++a) {
    const int s = bsr_slot(H.row_ptr, H.col, a / kBB, a / kBB);
    if (s >= 0) H.val[(size_t)s * kBB * kBB + (size_t)(a % kBB) * (kBB + 1)] += v[i];
  }
}

__global__ void k_mulliken_bsr(int N, const int32_t* __restrict__ types, const int32_t* __restrict__ offs, tb_bsr D,
                               double n0_O, double n0_H, double* __restrict__ q) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *D.status != TB_OK) return;
  double pop = 0.0;
  for (int a = offs[i]; a < offs[i + 1]; ++a) pop += bsr_get(D, a, a);
  q[i] = 2.0 * pop - (types[i] == TB_TYPE_O ? n0_O : n0_H);
}

// As k_forces, with D read from BSR and the neighbours from H's pattern.
__global__ void __launch_bounds__(32) k_forces_bsr(ModelDev m, int N, const int32_t* __restrict__ types,
                                                   const int32_t* __restrict__ offs, const double* __restrict__ R,
                                                   tb_bsr H, tb_bsr D, BsrModelWs w, const double* __restrict__ q,
                                                   const double* __restrict__ n_aux, const double* __restrict__ v,
                                                   double* __restrict__ F, double* __restrict__ energy) {
  const int a = blockIdx.x;
  const int lane = threadIdx.x & 31;
  if (a >= N || *H.status != TB_OK || *D.status != TB_OK) return;
  const double* Ra = R + 3 * a;
  const int ta = types[a], oa = offs[a];
  const double wa = 2.0 * q[a] - n_aux[a];
  const double na = n_aux[a];
  double f[3] = {0.0, 0.0, 0.0};
  double e_band = 0.0, e_pair = 0.0;
  for_neighbour_atoms(H, w, m, oa / kBB, Ra, lane, [&](int b) {
    const double* Rb = R + 3 * b;
    if (b != a && !screen_f32(Ra, Rb, (float)m.box, (float)m.range)) return;
    const int tb = types[b], ob = offs[b];
    const double wb = 2.0 * q[b] - n_aux[b];
    const double nb = n_aux[b];
    double Dl[4][4];
    const int nra = norb_of(ta), nrb = norb_of(tb);
    for (int x = 0; x < 4; ++x)
      for (int y = 0; y < 4; ++y) Dl[x][y] = (x < nra && y < nrb) ? bsr_get(D, oa + x, ob + y) : 0.0;
    double d0[3];
    min_image(Ra, Rb, m.box, d0);
    int lo3[3], hi3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) image_range(d0[c], m.box, m.range, &lo3[c], &hi3[c]);
    for (int kx = lo3[0]; kx <= hi3[0]; ++kx)
      for (int ky = lo3[1]; ky <= hi3[1]; ++ky)
        for (int kz = lo3[2]; kz <= hi3[2]; ++kz) {
          if (b == a && kx == 0 && ky == 0 && kz == 0) continue;
          const double d[3] = {d0[0] + kx * m.box, d0[1] + ky * m.box, d0[2] + kz * m.box};
          const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          if (r >= m.range) continue;
          const double l[3] = {d[0] / r, d[1] / r, d[2] / r};
          if (r < m.rcut) {
            double V, dV, Eblk, g[3];
            hop_radial(m, r, &V, &dV);
            band_pair_g(ta, tb, [&](int x, int y) { return Dl[x][y]; }, l, r, V, dV, &Eblk, g);
            e_band += 2.0 * Eblk;
            if (b != a)
#pragma unroll
              for (int k = 0; k < 3; ++k) f[k] += 4.0 * g[k];
            double ph, dph;
            pair_radial(m, r, &ph, &dph);
            e_pair += 0.5 * ph;
            if (b != a)
#pragma unroll
              for (int k = 0; k < 3; ++k) f[k] += dph * l[k];
          }
          if (b != a) {
            double gg, dgg;
            gamma_radial(m, r, &gg, &dgg);
            const double c = 0.5 * (wa * nb + wb * na) * dgg;
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] += c * l[k];
          }
        }
  });
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = warp_sum(f[k]);
  e_band = warp_sum(e_band);
  e_pair = warp_sum(e_pair);
  if (lane == 0) {
    if (ta == TB_TYPE_O) {
      e_band += 2.0 * (m.eps_s_O * bsr_get(D, oa, oa) +
                       m.eps_p_O * (bsr_get(D, oa + 1, oa + 1) + bsr_get(D, oa + 2, oa + 2) + bsr_get(D, oa + 3, oa + 3)));
    } else {
      e_band += 2.0 * m.eps_s_H * bsr_get(D, oa, oa);
    }
    const double e_scc = 0.5 * wa * v[a];
    F[3 * a + 0] = f[0];
    F[3 * a + 1] = f[1];
    F[3 * a + 2] = f[2];
    atomicAdd(&energy[1], e_band);
    atomicAdd(&energy[2], e_scc);
    atomicAdd(&energy[3], e_pair);
    atomicAdd(&energy[0], e_band + e_scc + e_pair);
  }
}

int bsr_check(tb_ctx* ctx, const tb_bsr* M, int n, const char* what) {
  if (!M || !M->row_ptr || !M->col || !M->val || !M->status)
    return tb_fail(ctx, TB_ERR_ARG, "%s: null BSR array", what);
  if (M->n != n || M->nsb != (n + kBB - 1) / kBB || M->cap < 1)
    return tb_fail(ctx, TB_ERR_ARG, "%s: BSR sizes (n %d, nsb %d, cap %d) do not fit n = %d", what, M->n, M->nsb,
                   M->cap, n);
  return TB_OK;
}

}  // namespace

extern "C" int tb_bsr_model_workspace_size(int natoms, int norb, size_t* bytes) {
  if (natoms < 1 || norb < 1 || !bytes) return TB_ERR_ARG;
  *bytes = bsr_model_bytes(natoms, (norb + kBB - 1) / kBB, nullptr, nullptr);
  return TB_OK;
}

extern "C" int tb_build_H_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R,
                              const double* n_aux, tb_bsr* H, double* v, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !v || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to tb_build_H_bsr");
  if ((rc = bsr_check(ctx, H, sys->norb, "tb_build_H_bsr"))) return rc;
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  if (m.gamma_form != 0) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "tb_build_H_bsr needs the windowed gamma");
  if (m.s0 != 0.0) return tb_fail(ctx, TB_ERR_UNSUPPORTED, "tb_build_H_bsr: orthogonal model only");
  const int N = sys->natoms, n = sys->norb, nsb = H->nsb;
  BsrModelWs w;
  if (ws_bytes < bsr_model_bytes(N, nsb, &w, ws)) return tb_fail(ctx, TB_ERR_ARG, "tb_build_H_bsr: workspace too small");
  cudaStream_t s = as_stream(stream);
  k_blk_atoms<<<(nsb + 127) / 128, 128, 0, s>>>(N, n, nsb, sys->orb_off, w);
  TB_LAUNCH_CHECK(ctx);
  k_blk_box<<<nsb, 128, 0, s>>>(m, R, nsb, w);
  TB_LAUNCH_CHECK(ctx);
  k_blk_pattern<<<nsb, 256, 0, s>>>(m, nsb, w);
  TB_LAUNCH_CHECK(ctx);
  k_blk_count<<<(nsb + 127) / 128, 128, 0, s>>>(nsb, w);
  TB_LAUNCH_CHECK(ctx);
  k_blk_scan<<<1, 32, 0, s>>>(nsb, w, *H);
  TB_LAUNCH_CHECK(ctx);
  k_blk_cols<<<(nsb + 127) / 128, 128, 0, s>>>(nsb, w, *H);
  TB_LAUNCH_CHECK(ctx);
  k_h_blocks<<<std::min(H->cap, 4096), 256, 0, s>>>(m, N, sys->types, sys->orb_off, R, w, *H);
  TB_LAUNCH_CHECK(ctx);
  if (n_aux) {
    k_v_bsr<<<(N * 32 + 255) / 256, 256, 0, s>>>(m, N, sys->orb_off, R, n_aux, *H, w, v);
    TB_LAUNCH_CHECK(ctx);
    k_shift_bsr<<<(N + 127) / 128, 128, 0, s>>>(N, sys->orb_off, v, *H);
  } else {
    TB_CUDA_TRY(ctx, cudaMemsetAsync(v, 0, sizeof(double) * N, s));
  }
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

extern "C" int mulliken_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const tb_bsr* D, double* q,
                            void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!p || !q) return tb_fail(ctx, TB_ERR_ARG, "null argument to mulliken_bsr");
  if ((rc = bsr_check(ctx, D, sys->norb, "mulliken_bsr"))) return rc;
  const int N = sys->natoms;
  k_mulliken_bsr<<<(N + 127) / 128, 128, 0, as_stream(stream)>>>(N, sys->types, sys->orb_off, *D, p->n0_O, p->n0_H, q);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}

extern "C" int tb_forces_bsr(tb_ctx* ctx, const tb_params* p, const tb_system* sys, const double* R, const tb_bsr* H,
                             const tb_bsr* D, const double* q, const double* n_aux, const double* v, double* F,
                             double* energy, const void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_system(ctx, sys);
  if (rc) return rc;
  if (!R || !q || !n_aux || !v || !F || !energy || !ws) return tb_fail(ctx, TB_ERR_ARG, "null argument to tb_forces_bsr");
  if ((rc = bsr_check(ctx, H, sys->norb, "tb_forces_bsr (H)"))) return rc;
  if ((rc = bsr_check(ctx, D, sys->norb, "tb_forces_bsr (D)"))) return rc;
  ModelDev m;
  rc = tb_model_from_params(ctx, p, sys->box, &m);
  if (rc) return rc;
  if (m.gamma_form != 0 || m.s0 != 0.0)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "tb_forces_bsr: windowed gamma, orthogonal model only");
  const int N = sys->natoms;
  BsrModelWs w;
  if (ws_bytes < bsr_model_bytes(N, H->nsb, &w, const_cast<void*>(ws)))
    return tb_fail(ctx, TB_ERR_ARG, "tb_forces_bsr: workspace too small");
  cudaStream_t s = as_stream(stream);
  TB_CUDA_TRY(ctx, cudaMemsetAsync(energy, 0, 4 * sizeof(double), s));
  k_forces_bsr<<<N, 32, 0, s>>>(m, N, sys->types, sys->orb_off, R, *H, *D, w, q, n_aux, v, F, energy);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
