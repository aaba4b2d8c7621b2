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
// pp-sigma = +V, pp-pi = -V sharing V(r) = t exp(-r/r_decay); V and the pair
// potential are replaced on [r1, rcut) by the quintic tail of App. D.
// gamma(r) = k/sqrt(r^2 + (k/U)^2) * (1-x)^4 (1+4x), x = r/gamma_cut.
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
  {
    const double a = m->inv_decay, v = p->t_hop * exp(-p->r1 * a);
    tail_closed_form(v, -a * v, a * a * v, p->r1, p->rcut, m->Bhop);
  }
  {
    const double a = m->inv_prho, v = p->pair_a * exp(-p->r1 * a);
    tail_closed_form(v, -a * v, a * a * v, p->r1, p->rcut, m->Bpair);
  }
  m->range = fmax(p->rcut, p->gamma_cut);
  m->box = box;
  return TB_OK;
}

// --------------------------------------------------------------------------
// device: radial functions
// --------------------------------------------------------------------------

__device__ __forceinline__ void tail_eval(const double* B, double x, double* f, double* df) {
  *f = B[0] + x * (B[1] + x * (B[2] + x * (B[3] + x * (B[4] + x * B[5]))));
  *df = B[1] + x * (2.0 * B[2] + x * (3.0 * B[3] + x * (4.0 * B[4] + x * 5.0 * B[5])));
}

// V(r) and V'(r) of the hopping with its tail.
__device__ __forceinline__ void hop_radial(const ModelDev& m, double r, double* V, double* dV) {
  if (r < m.r1) {
    const double v = m.t_hop * exp(-r * m.inv_decay);
    *V = v;
    *dV = -m.inv_decay * v;
  } else if (r < m.rcut) {
    tail_eval(m.Bhop, r - m.r1, V, dV);
  } else {
    *V = 0.0;
    *dV = 0.0;
  }
}

__device__ __forceinline__ void pair_radial(const ModelDev& m, double r, double* f, double* df) {
  if (m.pair_a == 0.0 || r >= m.rcut) {
    *f = 0.0;
    *df = 0.0;
  } else if (r < m.r1) {
    const double v = m.pair_a * exp(-r * m.inv_prho);
    *f = v;
    *df = -m.inv_prho * v;
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
                                                     double* __restrict__ G) {
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
  double gsum = (i == j) ? m.U : 0.0;
  // H and gamma were zeroed: pairs with no image in range write nothing
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
          double g, dg;
          gamma_radial(m, r, &g, &dg);
          gsum += g;
          if (r < m.rcut) {
            double V, dV;
            hop_radial(m, r, &V, &dV);
            const double l[3] = {d[0] / r, d[1] / r, d[2] / r};
            double Bi[4][4];
            sk_block(ti, tj, l, V, Bi);
            for (int a = 0; a < ni; ++a)
              for (int b = 0; b < nj; ++b) B[a][b] += Bi[a][b];
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
  cudaStream_t s = as_stream(stream);
  const int N = sys->natoms, n = sys->norb;
  TB_CUDA_TRY(ctx, cudaMemsetAsync(H, 0, sizeof(double) * (size_t)n * n, s));
  TB_CUDA_TRY(ctx, cudaMemsetAsync(gamma, 0, sizeof(double) * (size_t)N * N, s));
  dim3 grid((N + 255) / 256, N);
  k_build_pairs<<<grid, 256, 0, s>>>(m, N, sys->types, sys->orb_off, R, H, n, gamma);
  TB_LAUNCH_CHECK(ctx);
  if (n_aux) {
    k_add_shift<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, sys->orb_off, gamma, n_aux, H, n);
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
__device__ __forceinline__ void band_pair(int ta, int tb, const double* __restrict__ D, int n,
                                          int oa, int ob, const double l[3], double r, double V,
                                          double dV, double* Eblk, double g[3]) {
  const double Dss = D[(size_t)oa * n + ob];
  double u[3] = {0.0, 0.0, 0.0};
  if (tb == TB_TYPE_O)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] += D[(size_t)oa * n + ob + 1 + c];
  if (ta == TB_TYPE_O)
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] -= D[(size_t)(oa + 1 + c) * n + ob];
  const double ul = u[0] * l[0] + u[1] * l[1] + u[2] * l[2];
  double E = -V * Dss + V * ul;
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = -dV * Dss * l[k] + V * (u[k] - ul * l[k]) / r + dV * ul * l[k];
  if (ta == TB_TYPE_O && tb == TB_TYPE_O) {
    double P[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int e = 0; e < 3; ++e) P[c][e] = D[(size_t)(oa + 1 + c) * n + ob + 1 + e];
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

// One warp per atom a; lanes sweep all atoms b and their images.
// F_a = dE/dd summed over pairs (d = R_b - R_a + T), since dd/dR_a = -1.
// Per-atom energy shares are reduced with FP64 atomics into energy[1..3].
__global__ void __launch_bounds__(256) k_forces(ModelDev m, int N, const int32_t* __restrict__ types,
                                                const int32_t* __restrict__ offs,
                                                const double* __restrict__ R,
                                                const double* __restrict__ D, int n,
                                                const double* __restrict__ q,
                                                const double* __restrict__ n_aux,
                                                const double* __restrict__ G,
                                                double* __restrict__ F, double* __restrict__ energy) {
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
  cudaStream_t s = as_stream(stream);
  TB_CUDA_TRY(ctx, cudaMemsetAsync(energy, 0, 4 * sizeof(double), s));
  const int N = sys->natoms;
  // one warp per atom, one warp per block: FP64 runs at ~8 GFLOP/s per SM on
  // GB300, so small systems spread their atoms over as many SMs as possible
  k_forces<<<N, 32, 0, s>>>(m, N, sys->types, sys->orb_off, R, D, sys->norb, q,
                                                  n_aux, gamma, F, energy);
  TB_LAUNCH_CHECK(ctx);
  return TB_OK;
}
