"""Non-orthogonal SCC tight binding (App. D.1): the overlap S, a congruence
factor Z with Z^T S Z = I (Eq. Congr), H_perp = Z^T H Z, the density matrix
rho = Z rho_perp Z^T (Eq. DM_perp), Mulliken charges with S, and the energy
and forces of Eq. EL_Nonorth_a with its Pulay and dq/dR|_rho terms.

Test infrastructure: imported only by tests/, the package's smoke check and
the benchmark's CPU baseline.  Plain FP64 NumPy/LAPACK, written from the
definitions; nothing here is shared with the CUDA path.

Readings (the paper states the equations for LATTE's parameters, which are
not available):
  * S: unit on-site blocks; between atoms the Slater-Koster table of the
    hopping (tb.sk_block) with the overlap radial s(r) = overlap_s0
    exp(-r / overlap_rs) (App. D's zeta form with A0 = overlap_s0,
    A1 = -1/overlap_rs, A2..A4 = 0) and the App. D tail between r1 and rcut,
    with the signs of an overlap: ss-sigma = +s, sp-sigma = -s,
    pp-sigma = -s, pp-pi = +s, i.e. minus the hopping table evaluated with s.
    overlap_s0 = 0 is the orthogonal model;
  * H[n] (Eq. DFTB_2 with q -> n, as in Eq. EL_Orth_c): V^ee is diagonal,
    V_aa = v_i(a) = sum_l gamma_{i(a) l} n_l, so
    H_ab = h_ab + S_ab (v_a + v_b) / 2;
  * Mulliken charges q_i = 2 sum_{a in i} (rho S)_aa - N0_i.  The paper
    writes the diagonal of rho_perp, but the charge derivative it uses in
    Eq. EL_Nonorth_a, dq_j/dR|_rho = 2 sum_a (rho S_R)_aa, is that of the
    Mulliken form, which is taken here;
  * energy: E = KE + 2 Tr[h rho] + 1/2 (2q - n)^T gamma n + E_pair (- T_e S_e
    at finite T), the orthogonal reading with Mulliken q.  Its rho-dependent
    part is 2 Tr[rho H[n]] (q^T gamma n = Tr[rho (S V + V S)]), so rho, the
    ground state (or Fermi-Dirac state) of H[n] in the metric S, makes it
    stationary at fixed n;
  * force at fixed n:
      F = -d/dR { Tr[2 rho h(R)] + Tr[(V rho + rho V - 2 W) S(R)] }|_{rho, W}
          - (q - n/2)^T (dgamma/dR) n - dE_pair/dR,
    W = (S^-1 H rho + rho H S^-1) / 2 the energy-weighted density matrix
    (rho H rho at T_e = 0).  The W term is Eq. EL_Nonorth_a's Pulay term
    Tr[(S^-1 H rho + rho H S^-1) S_R], the V rho + rho V term its
    q^T gamma dq/dR|_rho with n for q; with S = I it is the orthogonal force.
    Pinned by central differences of E at fixed n.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

from workloads.water import ModelParams
from . import density, observables, tb


def overlap_radial(p: ModelParams) -> tb.Radial:
    """s(r) = overlap_s0 exp(-r / overlap_rs) with the App. D tail."""
    return tb.zeta_radial(p.overlap_s0, (-1.0 / p.overlap_rs, 0.0, 0.0, 0.0), p.r1, p.rcut)


def is_nonorth(p: ModelParams) -> bool:
    return p.overlap_s0 != 0.0


def build_S(R: np.ndarray, types: np.ndarray, box: float, p: ModelParams, pairs=None) -> np.ndarray:
    """Overlap matrix: identity on site, minus the Slater-Koster blocks of the
    overlap radial between every atom and every periodic image within rcut."""
    offs = tb.orbital_offsets(types)
    n = int(offs[-1])
    S = np.eye(n)
    if not is_nonorth(p):
        return S
    Sr = overlap_radial(p)
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    for i, j, d in zip(*pairs):
        blk, _ = tb.sk_block(int(types[i]), int(types[j]), d, Sr)
        si, sj = slice(offs[i], offs[i + 1]), slice(offs[j], offs[j + 1])
        S[si, sj] -= blk
        if i != j:
            S[sj, si] -= blk.T
    return S


def orbital_shift(G: np.ndarray, types: np.ndarray, n_aux: np.ndarray) -> np.ndarray:
    """v_a = sum_l gamma_{i(a) l} n_l for every orbital a of atom i."""
    offs = tb.orbital_offsets(types)
    v_atom = G @ n_aux
    return np.repeat(v_atom, np.diff(offs))


def build_H(h: np.ndarray, S: np.ndarray, G: np.ndarray, types: np.ndarray, n_aux: np.ndarray) -> np.ndarray:
    """H[n] = h + (S V + V S)/2 with V = diag(v) (Eq. DFTB_2)."""
    v = orbital_shift(G, types, n_aux)
    return h + 0.5 * S * (v[:, None] + v[None, :])


def congruence_factor(S: np.ndarray, kind: str = "lowdin") -> np.ndarray:
    """Z with Z^T S Z = I (Eq. Congr): the symmetric S^{-1/2} ('lowdin') or the
    inverse transposed Cholesky factor ('cholesky', S = L L^T, Z = L^{-T})."""
    if kind == "lowdin":
        w, U = np.linalg.eigh(S)
        return (U / np.sqrt(w)) @ U.T
    L = np.linalg.cholesky(S)
    return scipy.linalg.solve_triangular(L, np.eye(S.shape[0]), lower=True).T


class NonorthState:
    """rho, rho_perp, W, H_perp, Z and the spectrum of one density-matrix solve."""

    def __init__(self, rho, rho_perp, W, Hp, Z, eps, occ, mu, gap):
        self.rho, self.rho_perp, self.W, self.Hp, self.Z = rho, rho_perp, W, Hp, Z
        self.eps, self.occ, self.mu, self.gap = eps, occ, mu, gap


def density_matrix(H: np.ndarray, S: np.ndarray, n_occ: float, kT: float = 0.0,
                   kind: str = "lowdin") -> NonorthState:
    """rho = Z rho_perp Z^T with rho_perp = theta(mu0 I - H_perp) (T_e = 0) or the
    Fermi-Dirac matrix at Tr rho_perp = N_occ (Eq. DM_perp), H_perp = Z^T H Z;
    W = Z (H_perp rho_perp + rho_perp H_perp) Z^T / 2."""
    Z = congruence_factor(S, kind)
    Hp = Z.T @ H @ Z
    Hp = 0.5 * (Hp + Hp.T)
    r = density.density_fermi(Hp, n_occ, kT) if kT > 0 else density.density_T0(Hp, int(round(n_occ)))
    Dp = r.D
    rho = Z @ Dp @ Z.T
    W = 0.5 * Z @ (Hp @ Dp + Dp @ Hp) @ Z.T
    return NonorthState(rho, Dp, W, Hp, Z, r.eps, r.occ, r.mu, r.gap)


def mulliken(rho: np.ndarray, S: np.ndarray, types: np.ndarray, p: ModelParams) -> np.ndarray:
    """q_i = 2 sum_{a in i} (rho S)_aa - N0_i."""
    offs = tb.orbital_offsets(types)
    d = np.einsum("ab,ba->a", rho, S)
    pop = np.array([2.0 * d[offs[i]:offs[i + 1]].sum() for i in range(len(types))])
    return pop - observables.neutral_electrons(types, p)


def energy_terms(R, types, box, p: ModelParams, rho, q, n_aux, pairs=None):
    """2 Tr[h rho], 1/2 (2q - n)^T gamma n, E_pair (the orthogonal form with the
    Mulliken q of the metric S)."""
    return observables.energy_terms(R, types, box, p, rho, q, n_aux, pairs=pairs)


def forces(R, types, box, p: ModelParams, rho, W, q, n_aux, pairs=None) -> np.ndarray:
    """F = -dE/dR at fixed n (module docstring), [N, 3] eV/A."""
    F = observables.forces(R, types, box, p, rho, q, n_aux, pairs=pairs)
    if not is_nonorth(p):
        return F
    N = R.shape[0]
    offs = tb.orbital_offsets(types)
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    G = tb.build_gamma(R, box, p, pairs)
    v = orbital_shift(G, types, n_aux)
    MS = v[:, None] * rho + rho * v[None, :] - 2.0 * W   # weight of S(R) in the energy
    Sr = overlap_radial(p)
    dE = np.zeros((N, 3))
    for i, j, d in zip(*pairs):
        if i == j:
            continue
        _, dblk = tb.sk_block(int(types[i]), int(types[j]), d, Sr)
        Mij = MS[offs[i]:offs[i + 1], offs[j]:offs[j + 1]]
        # S_ij = -blk and S_ji = -blk^T both depend on d; MS is symmetric
        g = -2.0 * np.einsum("ab,abk->k", Mij, dblk)
        dE[j] += g
        dE[i] -= g
    return F - dE


def electronic_state(R, types, box, p: ModelParams, n_aux, n_occ, kT: float = 0.0, pairs=None):
    """h, S, gamma, H[n], the density-matrix solve and the Mulliken charges."""
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    h = tb.build_h(R, types, box, p, pairs)
    S = build_S(R, types, box, p, pairs)
    G = tb.build_gamma(R, box, p, pairs)
    H = build_H(h, S, G, types, n_aux)
    st = density_matrix(H, S, n_occ, kT)
    q = mulliken(st.rho, S, types, p)
    return h, S, G, H, st, q


def potential_energy(R, types, box, p: ModelParams, n_aux, n_occ, kT: float = 0.0) -> float:
    """E_pot at fixed n: 2 Tr[h rho] + 1/2 (2q - n)^T gamma n + E_pair, minus
    T_e S_e of the occupations of rho_perp at T_e > 0."""
    _, _, _, _, st, q = electronic_state(R, types, box, p, n_aux, n_occ, kT)
    E = float(sum(energy_terms(R, types, box, p, st.rho, q, n_aux)))
    if kT > 0:
        E -= kT * density.entropy_kB(st.occ)
    return E


def scf(R, types, box, p: ModelParams, n_occ, tol: float = 1e-10, max_iter: int = 300, beta: float = 0.2,
        history: int = 8, kT: float = 0.0, strict: bool = True):
    """Self-consistent charges n = q[rho(H[n], S)] by Anderson mixing (as
    md.scf); returns (q, n, iterations or -1)."""
    from . import md
    pairs = tb.pair_images(R, box, tb.pair_range(p))
    n_aux = np.zeros(len(types))
    xs, fs = [], []
    for it in range(max_iter):
        _, _, _, _, _, q = electronic_state(R, types, box, p, n_aux, n_occ, kT, pairs)
        f = q - n_aux
        if np.max(np.abs(f)) <= tol:
            return q, n_aux, it
        xs.append(n_aux.copy())
        fs.append(f)
        xs, fs = xs[-history:], fs[-history:]
        n_aux = md.anderson_mix(xs, fs, beta)
    if strict:
        raise RuntimeError(f"SCF did not converge in {max_iter} iterations")
    return q, xs[-1], -1


def xlbomd(R0, types, box, p: ModelParams, xl, v0, masses, n_occ, nsteps: int, scf_tol: float = 1e-10,
           kT: float = 0.0, record_R: bool = False):
    """The Fast-QMMD trajectory of md.xlbomd in the non-orthogonal formulation
    (Eqs. EL_Nonorth_a, EL_Nonorth_b with the integrators of Eq. Verl_n):
    half kick, drift, n update, H[n] -> rho -> q, force, half kick; E_tot =
    KE + E_pot - T_e S_e with S_e from the occupations of rho_perp."""
    from . import md
    q0, _, _ = scf(R0, types, box, p, n_occ, tol=scf_tol, kT=kT)
    R, v = R0.copy(), v0.copy()
    n_hist = [q0.copy() for _ in range(xl.K + 1)]
    traj = md.Trajectory([], [], [], [], [], [], [], [])

    def solve(R, n_aux):
        pairs = tb.pair_images(R, box, tb.pair_range(p))
        _, _, _, _, st, q = electronic_state(R, types, box, p, n_aux, n_occ, kT, pairs)
        F = forces(R, types, box, p, st.rho, st.W, q, n_aux, pairs)
        Ep = float(sum(energy_terms(R, types, box, p, st.rho, q, n_aux, pairs)))
        TS = kT * density.entropy_kB(st.occ) if kT > 0 else 0.0
        return q, F, Ep, TS, st.gap

    def record(R, v, q, n_aux, F, Ep, TS, gap):
        KE = observables.kinetic_energy(v, masses)
        traj.E_tot.append(KE + Ep - TS)
        traj.TS.append(TS)
        traj.E_pot.append(Ep)
        traj.KE.append(KE)
        traj.q.append(q.copy())
        traj.n.append(n_aux.copy())
        traj.F.append(F.copy())
        traj.gap.append(gap)
        if record_R:
            traj.R.append(R.copy())

    q_t, F, Ep, TS, gap = solve(R, n_hist[0])
    record(R, v, q_t, n_hist[0], F, Ep, TS, gap)
    for _ in range(nsteps):
        v = md.velocity_verlet_kick(v, F, masses, xl.dt)
        R = R + xl.dt * v
        n_new = md.modified_verlet_n(n_hist, q_t, xl)
        n_hist = [n_new] + n_hist[:-1]
        q_t, F, Ep, TS, gap = solve(R, n_new)
        v = md.velocity_verlet_kick(v, F, masses, xl.dt)
        record(R, v, q_t, n_new, F, Ep, TS, gap)
    return traj
