// XL-BOMD (Fast-QMMD) integration on device-resident state (row a9).
//
// Nuclei: velocity Verlet with F = -dE/dR at fixed n (App. D.3).
// Auxiliary charges: modified Verlet with dissipation, Eq. Verl_n,
//   n_{t+dt} = 2 n_t - n_{t-dt} + kappa (q_t - n_t) + alpha sum_{k=0}^{K} c_k n_{t-k dt},
// with the Mulliken charges q_t of D[n_t] in place of sigma_t (Eq. EL_Orth_b).
// The n history is a (K+1)-slot shift register, slot j = n_{t-j}: each step
// moves it down one slot on the device, so every launch of a step has the
// same arguments and a step can be captured once into a CUDA graph and
// replayed.  A step enqueues: half kick + drift, n update, H[n] build, D
// (SP2, or the Fermi operator at kT > 0), Mulliken, forces/energy, half kick
// + kinetic energy; nothing synchronises the host.
//
// Initialisation (App. D.3): SCF-converged charges to a high degree, then
// the whole history set to q.  The SCF loop runs the same device kernels
// and mixes the N-vector of charges on the host with Anderson/Pulay mixing.

#include "common.cuh"

#include <math.h>
#include <string.h>

#include <vector>

namespace {

constexpr double kEvAmuToAFs2 = 9.648533e-3;  // 1 eV/(A amu) in A/fs^2

__global__ void k_kick_drift(int N, double* __restrict__ v, const double* __restrict__ F,
                             const double* __restrict__ mass, double dt, double* __restrict__ R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double s = 0.5 * dt * kEvAmuToAFs2 / mass[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vv = v[3 * i + c] + s * F[3 * i + c];
    v[3 * i + c] = vv;
    R[3 * i + c] += dt * vv;
  }
}

// Eq. Verl_n on the shift register: thread i reads n_{t-j} (slot j) of its
// atom, shifts them down one slot and puts n_{t+dt} in slot 0.
__global__ void k_n_update(int N, double* __restrict__ hist, int K, const double* __restrict__ q, double kappa,
                           double alpha, tb_xl_params xp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double nv[TB_XL_KMAX + 1];
  for (int j = 0; j <= K; ++j) nv[j] = hist[(size_t)j * N + i];
  double diss = 0.0;
  for (int j = 0; j <= K; ++j) diss += xp.c[j] * nv[j];
  const double n_new = 2.0 * nv[0] - nv[1] + kappa * (q[i] - nv[0]) + alpha * diss;
  for (int j = K; j >= 1; --j) hist[(size_t)j * N + i] = nv[j - 1];
  hist[i] = n_new;
}

// Second half kick, kinetic energy, E_tot and max|n - q| in one block; the
// step counter E[7] is 0 after the initial state (kick = 0), +1 per step.
__global__ void __launch_bounds__(256) k_kick_energy(int N, double* __restrict__ v, const double* __restrict__ F,
                                                     const double* __restrict__ mass, double dt, int kick,
                                                     const double* __restrict__ n_cur,
                                                     const double* __restrict__ q, double* __restrict__ E,
                                                     const double* __restrict__ S, double kT) {
  __shared__ double s_ke[8], s_dq[8];
  double ke = 0.0, dq = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double s = 0.5 * dt * kEvAmuToAFs2 / mass[i];
    double v2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double vv = v[3 * i + c];
      if (kick) {
        vv += s * F[3 * i + c];
        v[3 * i + c] = vv;
      }
      v2 += vv * vv;
    }
    ke += 0.5 * mass[i] * v2 / kEvAmuToAFs2;
    dq = fmax(dq, fabs(n_cur[i] - q[i]));
  }
  ke = warp_sum(ke);
  dq = warp_max(dq);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_ke[w] = ke;
    s_dq[w] = dq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += s_ke[k];
      b = fmax(b, s_dq[k]);
    }
    E[5] = a;
    E[0] = a + E[1] - (S ? kT * S[0] : 0.0);  // Eq. Etot: - T_e S at finite temperature
    E[6] = b;
    E[7] = kick ? E[7] + 1.0 : 0.0;
  }
}

// mu[0] <- the start of this step's dm_fermi, extrapolated from the last
// steps' values mu[1..3] (quadratic 3 mu1 - 3 mu2 + mu3, linear 2 mu1 - mu2,
// or mu1, as far as they are known).
__global__ void k_mu_predict(double* mu) {
  const double a = mu[1], b = mu[2], c = mu[3];
  if (!isfinite(a)) return;
  mu[0] = !isfinite(b) ? a : !isfinite(c) ? 2.0 * a - b : 3.0 * a - 3.0 * b + c;
}
// mu[3] <- mu[2] <- mu[1] <- mu[0] after a step's dm_fermi.
__global__ void k_mu_shift(double* mu) {
  mu[3] = mu[2];
  mu[2] = mu[1];
  mu[1] = mu[0];
}

__global__ void k_fill_hist(int N, int S, const double* __restrict__ q, double* __restrict__ hist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int s = 0; s < S; ++s) hist[(size_t)s * N + i] = q[i];
}

int check_state(tb_ctx* ctx, const tb_md_state* st, const tb_xl_params* xp, const tb_sp2_opts* so) {
  if (!st || !xp || !so) return tb_fail(ctx, TB_ERR_ARG, "null state/params/options");
  if (xp->K < 1 || xp->K > TB_XL_KMAX) return tb_fail(ctx, TB_ERR_ARG, "K = %d outside 1..%d", xp->K, TB_XL_KMAX);
  const bool bsr = st->H_bsr != nullptr;
  if (!st->R || !st->v || !st->F || !st->mass || !st->n_hist || !st->q || !st->energies || !st->workspace ||
      (!bsr && (!st->H || !st->D || !st->gamma)))
    return tb_fail(ctx, TB_ERR_ARG, "null array in tb_md_state");
  if (bsr && (!st->D_bsr || !st->vscc || !st->bsr_workspace || !(so->tau > 0.0)))
    return tb_fail(ctx, TB_ERR_ARG, "the block-sparse state needs D_bsr, vscc, bsr_workspace and sp2 opts with tau > 0");
  if (bsr && st->kT > 0.0 && st->entropy_workspace)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "the entropy term is not available with the block-sparse state");
  if (!(xp->dt > 0)) return tb_fail(ctx, TB_ERR_ARG, "dt must be > 0");
  if (st->kT > 0.0 && !st->mu) return tb_fail(ctx, TB_ERR_ARG, "kT > 0 needs the device mu");
  return TB_OK;
}

// Non-orthogonal formulation (App. D.1) when the model has an overlap.
bool nonorth_on(const tb_params* p) { return p && p->overlap_s0 != 0.0; }

int check_nonorth(tb_ctx* ctx, const tb_params* p, const tb_md_state* st) {
  if (!nonorth_on(p)) return TB_OK;
  if (!st->S || !st->W || !st->vscc || !st->nonorth_workspace)
    return tb_fail(ctx, TB_ERR_ARG, "overlap_s0 != 0: tb_md_state needs S, W, vscc and the dm_nonorth workspace");
  if (st->kT > 0.0 && st->entropy_workspace)
    return tb_fail(ctx, TB_ERR_UNSUPPORTED, "the entropy term is not available in the non-orthogonal formulation");
  return TB_OK;
}

// H[n] (and S, v in the non-orthogonal formulation; v with the block-sparse state).
int build_H_any(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const double* n_aux, cudaStream_t s) {
  if (st->H_bsr)
    return tb_build_H_bsr(ctx, p, &st->sys, st->R, n_aux, st->H_bsr, st->vscc, st->bsr_workspace,
                          st->bsr_workspace_bytes, s);
  if (nonorth_on(p)) return tb_build_HS(ctx, p, &st->sys, st->R, n_aux, st->H, st->S, st->gamma, st->vscc, s);
  return tb_build_H(ctx, p, &st->sys, st->R, n_aux, st->H, st->gamma, s);
}

int charges_any(tb_ctx* ctx, const tb_params* p, tb_md_state* st, cudaStream_t s) {
  if (st->H_bsr) return mulliken_bsr(ctx, p, &st->sys, st->D_bsr, st->q, s);
  if (nonorth_on(p)) return mulliken_nonorth(ctx, p, &st->sys, st->D, st->S, st->q, s);
  return mulliken(ctx, p, &st->sys, st->D, st->q, s);
}

bool entropy_on(const tb_md_state* st) { return st->kT > 0.0 && st->entropy_workspace && st->entropy; }

// D from H: Fermi operator (dm_fermi, or dm_fermi_sparse with the block-sparse
// state; mu carried in st->mu) when kT > 0, else the T_e = 0 projector by SP2.
int density(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_sp2_opts* so, cudaStream_t s) {
  if (st->H_bsr && st->kT > 0.0)
    return dm_fermi_sparse(ctx, st->H_bsr, st->n_occ, st->kT, &st->fermi, so->tau, so->bsr_blocks_per_row,
                           st->D_bsr, st->mu, st->workspace, st->workspace_bytes, st->fermi_report, s);
  if (st->H_bsr)
    return dm_sp2_sparse(ctx, st->H_bsr, st->n_occ, so, st->D_bsr, st->workspace, st->workspace_bytes,
                         st->sp2_report, s);
  if (nonorth_on(p))
    return dm_nonorth(ctx, st->H, st->S, st->sys.norb, st->n_occ, st->kT, so, &st->fermi, st->mu, st->D, st->W,
                      st->nonorth_workspace, st->nonorth_workspace_bytes, st->sp2_report, st->fermi_report,
                      st->nonorth_report, s);
  if (st->kT > 0.0)
    return dm_fermi(ctx, st->H, st->sys.norb, st->n_occ, st->kT, &st->fermi, st->D, st->mu, st->workspace,
                    st->workspace_bytes, st->fermi_report, s);
  return dm_sp2(ctx, st->H, st->sys.norb, st->n_occ, so, st->D, st->workspace, st->workspace_bytes,
                st->sp2_report, s);
}

// H[n] -> D -> q -> F, E for the current positions and the given n.
int electronic_step(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_sp2_opts* so,
                    const double* n_aux, cudaStream_t s) {
  int rc = build_H_any(ctx, p, st, n_aux, s);
  if (rc) return rc;
  rc = density(ctx, p, st, so, s);
  if (rc) return rc;
  if (entropy_on(st)) {
    // T_e S at the mu of this D (st->mu[0]), Eq. Ent_Approx; E_tot only
    rc = dm_fermi_entropy(ctx, st->H, st->sys.norb, st->mu, st->kT, nullptr, st->entropy, st->entropy_workspace,
                          st->entropy_workspace_bytes, s);
    if (rc) return rc;
  }
  rc = charges_any(ctx, p, st, s);
  if (rc) return rc;
  if (st->H_bsr)
    return tb_forces_bsr(ctx, p, &st->sys, st->R, st->H_bsr, st->D_bsr, st->q, n_aux, st->vscc, st->F,
                         st->energies + 1, st->bsr_workspace, st->bsr_workspace_bytes, s);
  if (nonorth_on(p))
    return tb_forces_nonorth(ctx, p, &st->sys, st->R, st->D, st->W, st->q, n_aux, st->vscc, st->gamma, st->F,
                             st->energies + 1, s);
  return tb_forces(ctx, p, &st->sys, st->R, st->D, st->q, n_aux, st->gamma, st->F, st->energies + 1, s);
}

// Anderson / Pulay mixing of x (the charges n) with residual f = q - n:
// minimise ||f_k - dF g|| over g (normal equations, Gaussian elimination with
// partial pivoting and a small ridge), then x_new = x_k - dX g + beta (f_k - dF g).
void anderson(const std::vector<std::vector<double>>& xs, const std::vector<std::vector<double>>& fs,
              double beta, std::vector<double>& out) {
  const size_t N = xs.back().size();
  const int m = (int)xs.size() - 1;
  const std::vector<double>& xk = xs.back();
  const std::vector<double>& fk = fs.back();
  out.assign(N, 0.0);
  if (m <= 0) {
    for (size_t i = 0; i < N; ++i) out[i] = xk[i] + beta * fk[i];
    return;
  }
  std::vector<std::vector<double>> dF(m, std::vector<double>(N)), dX(m, std::vector<double>(N));
  for (int j = 0; j < m; ++j)
    for (size_t i = 0; i < N; ++i) {
      dF[j][i] = fs[j + 1][i] - fs[j][i];
      dX[j][i] = xs[j + 1][i] - xs[j][i];
    }
  std::vector<double> A(m * m), b(m), g(m);
  double diag_max = 0.0;
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (size_t i = 0; i < N; ++i) s += dF[r][i] * dF[c][i];
      A[r * m + c] = s;
    }
    double s = 0.0;
    for (size_t i = 0; i < N; ++i) s += dF[r][i] * fk[i];
    b[r] = s;
    diag_max = fmax(diag_max, A[r * m + r]);
  }
  for (int r = 0; r < m; ++r) A[r * m + r] += 1e-12 * diag_max + 1e-300;
  // Gaussian elimination with partial pivoting
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r * m + c]) > fabs(A[piv * m + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < m; ++k) {
        double t = A[c * m + k];
        A[c * m + k] = A[piv * m + k];
        A[piv * m + k] = t;
      }
      double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    const double d = A[c * m + c];
    if (d == 0.0) continue;
    for (int r = c + 1; r < m; ++r) {
      const double f = A[r * m + c] / d;
      for (int k = c; k < m; ++k) A[r * m + k] -= f * A[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < m; ++k) s -= A[r * m + k] * g[k];
    g[r] = A[r * m + r] != 0.0 ? s / A[r * m + r] : 0.0;
  }
  for (size_t i = 0; i < N; ++i) {
    double xb = xk[i], fb = fk[i];
    for (int j = 0; j < m; ++j) {
      xb -= dX[j][i] * g[j];
      fb -= dF[j][i] * g[j];
    }
    out[i] = xb + beta * fb;
  }
}

}  // namespace

extern "C" int xlbomd_init(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_xl_params* xp,
                           const tb_sp2_opts* so, double scf_tol, int scf_max_iter, int* scf_iters_out,
                           void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_state(ctx, st, xp, so);
  if (!rc) rc = check_nonorth(ctx, p, st);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  const int N = st->sys.natoms;
  const int S = xp->K + 1;
  // slot 0 is the working n during the SCF; the history is filled afterwards
  double* n_dev = st->n_hist;
  std::vector<double> n(N, 0.0), q(N), f(N), nn;
  std::vector<std::vector<double>> xs, fs;
  const int hist = 8;
  const double beta = 0.2;
  int iters = -1;
  for (int it = 0; it < scf_max_iter; ++it) {
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(n_dev, n.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
    rc = build_H_any(ctx, p, st, n_dev, s);
    if (rc) return rc;
    rc = density(ctx, p, st, so, s);
    if (rc) return rc;
    rc = charges_any(ctx, p, st, s);
    if (rc) return rc;
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(q.data(), st->q, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    double res = 0.0;
    for (int i = 0; i < N; ++i) {
      f[i] = q[i] - n[i];
      res = fmax(res, fabs(f[i]));
    }
    if (res <= scf_tol) {
      iters = it;
      break;
    }
    xs.push_back(n);
    fs.push_back(f);
    if ((int)xs.size() > hist) {
      xs.erase(xs.begin());
      fs.erase(fs.begin());
    }
    anderson(xs, fs, beta, nn);
    n = nn;
  }
  if (scf_iters_out) *scf_iters_out = iters;
  // the whole history is set to the last Mulliken charges (n = q)
  TB_CUDA_TRY(ctx, cudaMemcpyAsync(n_dev, q.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s));
  k_fill_hist<<<(N + 127) / 128, 128, 0, s>>>(N, S, n_dev, st->n_hist);
  TB_LAUNCH_CHECK(ctx);
  st->step = 0;
  rc = electronic_step(ctx, p, st, so, st->n_hist, s);
  if (rc) return rc;
  k_kick_energy<<<1, 256, 0, s>>>(N, st->v, st->F, st->mass, xp->dt, 0, st->n_hist, st->q, st->energies,
                                  entropy_on(st) ? st->entropy : nullptr, st->kT);
  TB_LAUNCH_CHECK(ctx);
  if (st->kT > 0.0) {
    const double nan3[3] = {NAN, NAN, NAN};
    TB_CUDA_TRY(ctx, cudaMemcpyAsync(st->mu + 1, nan3, sizeof(nan3), cudaMemcpyHostToDevice, s));
    k_mu_shift<<<1, 1, 0, s>>>(st->mu);  // mu[1] = the initial state's mu
    TB_LAUNCH_CHECK(ctx);
  }
  // the host vectors must outlive the async copies above
  TB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return TB_OK;
}

extern "C" int xlbomd_step(tb_ctx* ctx, const tb_params* p, tb_md_state* st, const tb_xl_params* xp,
                           const tb_sp2_opts* so, void* stream) {
  if (!ctx) return TB_ERR_ARG;
  int rc = check_state(ctx, st, xp, so);
  if (!rc) rc = check_nonorth(ctx, p, st);
  if (rc) return rc;
  cudaStream_t s = as_stream(stream);
  const int N = st->sys.natoms;
  const int nb = (N + 127) / 128;
  k_kick_drift<<<nb, 128, 0, s>>>(N, st->v, st->F, st->mass, xp->dt, st->R);
  TB_LAUNCH_CHECK(ctx);
  k_n_update<<<nb, 128, 0, s>>>(N, st->n_hist, xp->K, st->q, xp->kappa, xp->alpha, *xp);
  TB_LAUNCH_CHECK(ctx);
  if (st->kT > 0.0) {
    k_mu_predict<<<1, 1, 0, s>>>(st->mu);
    TB_LAUNCH_CHECK(ctx);
  }
  rc = electronic_step(ctx, p, st, so, st->n_hist, s);
  if (rc) return rc;
  if (st->kT > 0.0) {
    k_mu_shift<<<1, 1, 0, s>>>(st->mu);
    TB_LAUNCH_CHECK(ctx);
  }
  k_kick_energy<<<1, 256, 0, s>>>(N, st->v, st->F, st->mass, xp->dt, 1, st->n_hist, st->q, st->energies,
                                  entropy_on(st) ? st->entropy : nullptr, st->kT);
  TB_LAUNCH_CHECK(ctx);
  st->step += 1;
  return TB_OK;
}
