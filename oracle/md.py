"""SCF initialisation, integrators and the XL-BOMD / BOMD drivers.

XL-BOMD (Fast-QMMD, Eqs. EL_3ax, EL_3bx in the orthogonal SCC form of
Eqs. EL_Orth_a, EL_Orth_b):
  nuclei: velocity Verlet with F = -dE/dR at fixed n (App. D.3);
  charges: the modified Verlet scheme with dissipation of Eq. Verl_n,
    n_{t+dt} = 2 n_t - n_{t-dt} + kappa (q_t - n_t) + alpha sum_{k=0}^{K} c_k n_{t-k dt},
  where q_t = q[D(H[n_t])] plays the role of sigma_t (Eq. EL_Orth_b).
Initialisation (App. D.3): the first state is SCF-converged to a high degree
and the whole n history is set to q.  Reading: Anderson (Pulay) mixing to
max |q - n| <= 1e-10.
BOMD reference: every step is SCF-converged (n = q), starting from the
previous step's charges.
At T_e > 0 the constant of motion is E_tot = KE + U - T_e S (Eq. Etot), with
S the entropy of Eq. Entropy evaluated on the occupation numbers, i.e. the
eigenvalues of D (the approximation of Eq. Ent_Approx at n != rho).
"""

from __future__ import annotations

import dataclasses

import numpy as np

from workloads.water import ModelParams, XLParams, EV_PER_AMU_A2_FS2
from . import tb, density, observables


@dataclasses.dataclass
class Frame:
    R: np.ndarray
    types: np.ndarray
    box: float
    n_aux: np.ndarray
    D: np.ndarray
    q: np.ndarray
    H: np.ndarray
    gap: float


def electronic_state(R, types, box, p: ModelParams, n_aux, n_occ, kT: float = 0.0,
                     pairs=None, solver: str = "eigh"):
    """H[n] -> D -> q for given positions and auxiliary charges."""
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    h = tb.build_h(R, types, box, p, pairs)
    G = tb.build_gamma(R, box, p, pairs)
    H = tb.build_H(h, G, types, n_aux)
    if kT > 0:
        res = density.density_fermi(H, n_occ, kT)
    elif solver == "sp2":
        s = density.sp2(H, n_occ)
        res = density.DensityResult(D=s.X, eps=np.array([]), mu=float("nan"), gap=float("nan"),
                                    occ=np.array([]))
    else:
        res = density.density_T0(H, int(round(n_occ)))
    q = observables.mulliken(res.D, types, p)
    return H, G, res, q, pairs


def anderson_mix(xs: list, fs: list, beta: float) -> np.ndarray:
    """Anderson / Pulay mixing: minimise ||f_k - dF g|| over g in the span of
    the residual differences, then x_new = (x_k - dX g) + beta (f_k - dF g)."""
    xk, fk = xs[-1], fs[-1]
    if len(xs) == 1:
        return xk + beta * fk
    dX = np.stack([xs[i + 1] - xs[i] for i in range(len(xs) - 1)], axis=1)
    dF = np.stack([fs[i + 1] - fs[i] for i in range(len(fs) - 1)], axis=1)
    g, *_ = np.linalg.lstsq(dF, fk, rcond=None)
    return (xk - dX @ g) + beta * (fk - dF @ g)


def scf(R, types, box, p: ModelParams, n_occ, n_start=None, tol: float = 1e-10,
        max_iter: int = 300, beta: float = 0.2, history: int = 8, kT: float = 0.0,
        strict: bool = True):
    """Self-consistent charges: iterate n -> q[D(H[n])] with Anderson mixing
    until max_i |q_i - n_i| <= tol.  Returns (q, Frame, iterations); when the
    iteration cap is reached it raises (strict) or returns the last iterate
    with iterations = -1."""
    pairs = tb.pair_images(R, box, tb.pair_range(p))
    n_aux = np.zeros(len(types)) if n_start is None else n_start.copy()
    xs, fs = [], []
    for it in range(max_iter):
        H, G, res, q, _ = electronic_state(R, types, box, p, n_aux, n_occ, kT, pairs)
        f = q - n_aux
        if np.max(np.abs(f)) <= tol:
            return q, Frame(R, types, box, n_aux, res.D, q, H, res.gap), it
        xs.append(n_aux.copy())
        fs.append(f)
        xs, fs = xs[-history:], fs[-history:]
        n_aux = anderson_mix(xs, fs, beta)
    if strict:
        raise RuntimeError(f"SCF did not converge in {max_iter} iterations "
                           f"(max |q-n| = {np.max(np.abs(f)):.3e})")
    return q, Frame(R, types, box, xs[-1], res.D, q, H, res.gap), -1


def velocity_verlet_kick(v, F, masses, dt):
    """v <- v + dt/2 F/M (F in eV/A, M in amu, v in A/fs)."""
    return v + 0.5 * dt * F / masses[:, None] * EV_PER_AMU_A2_FS2


def modified_verlet_n(n_hist: list, q_t: np.ndarray, xl: XLParams) -> np.ndarray:
    """Eq. Verl_n: n_hist[0] = n_t, n_hist[k] = n_{t-k dt} for k = 0..K."""
    n_t, n_tm1 = n_hist[0], n_hist[1]
    diss = sum(ck * n_hist[k] for k, ck in enumerate(xl.c))
    return 2.0 * n_t - n_tm1 + xl.kappa * (q_t - n_t) + xl.alpha * diss


@dataclasses.dataclass
class Trajectory:
    E_tot: list
    E_pot: list
    KE: list
    q: list
    n: list
    F: list
    R: list
    gap: list
    TS: list = dataclasses.field(default_factory=list)


def _TS(D: np.ndarray, kT: float) -> float:
    """T_e S (eV) from the eigenvalues of D (Eqs. Entropy, Ent_Approx); 0 at T_e = 0."""
    if kT <= 0.0:
        return 0.0
    return kT * density.entropy_kB(np.linalg.eigvalsh(D))


def xlbomd(R0, types, box, p: ModelParams, xl: XLParams, v0, masses, n_occ, nsteps: int,
           scf_tol: float = 1e-10, kT: float = 0.0, record_R: bool = False, scf_max_iter: int = 300,
           scf_strict: bool = True) -> Trajectory:
    """Fast-QMMD trajectory (module docstring).  Step order: half kick, drift,
    n update from (n history, q_t), H[n_{t+1}] -> D -> q_{t+1}, force, half kick.
    scf_strict=False starts from the last SCF iterate when the cap is reached."""
    q0, fr, _ = scf(R0, types, box, p, n_occ, tol=scf_tol, kT=kT, max_iter=scf_max_iter, strict=scf_strict)
    R, v = R0.copy(), v0.copy()
    n_hist = [q0.copy() for _ in range(xl.K + 1)]
    q_t = q0
    D = fr.D
    F = observables.forces(R, types, box, p, D, q_t, n_hist[0])
    traj = Trajectory([], [], [], [], [], [], [], [])

    def record(R, v, D, q, n_aux, F, gap):
        Ep = observables.potential_energy(R, types, box, p, D, q, n_aux)
        KE = observables.kinetic_energy(v, masses)
        TS = _TS(D, kT)
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

    record(R, v, D, q_t, n_hist[0], F, fr.gap)
    for _ in range(nsteps):
        v = velocity_verlet_kick(v, F, masses, xl.dt)
        R = R + xl.dt * v
        n_new = modified_verlet_n(n_hist, q_t, xl)
        n_hist = [n_new] + n_hist[:-1]
        _, _, res, q_t, pairs = electronic_state(R, types, box, p, n_new, n_occ, kT)
        F = observables.forces(R, types, box, p, res.D, q_t, n_new, pairs)
        v = velocity_verlet_kick(v, F, masses, xl.dt)
        record(R, v, res.D, q_t, n_new, F, res.gap)
    return traj


def bomd(R0, types, box, p: ModelParams, dt: float, v0, masses, n_occ, nsteps: int,
         scf_tol: float = 1e-10, record_R: bool = False) -> Trajectory:
    """Born-Oppenheimer MD: SCF-converged charges at every step (n = q)."""
    q, fr, _ = scf(R0, types, box, p, n_occ, tol=scf_tol)
    R, v = R0.copy(), v0.copy()
    F = observables.forces(R, types, box, p, fr.D, q, q)
    traj = Trajectory([], [], [], [], [], [], [], [])

    def record(R, v, D, q, F, gap):
        Ep = observables.potential_energy(R, types, box, p, D, q, q)
        KE = observables.kinetic_energy(v, masses)
        traj.E_tot.append(KE + Ep)
        traj.E_pot.append(Ep)
        traj.KE.append(KE)
        traj.q.append(q.copy())
        traj.n.append(q.copy())
        traj.F.append(F.copy())
        traj.gap.append(gap)
        if record_R:
            traj.R.append(R.copy())

    record(R, v, fr.D, q, F, fr.gap)
    for _ in range(nsteps):
        v = velocity_verlet_kick(v, F, masses, dt)
        R = R + dt * v
        q, fr, _ = scf(R, types, box, p, n_occ, n_start=q, tol=scf_tol)
        F = observables.forces(R, types, box, p, fr.D, q, q)
        v = velocity_verlet_kick(v, F, masses, dt)
        record(R, v, fr.D, q, F, fr.gap)
    return traj


def energy_drift(E: list, dt_fs: float, natoms: int) -> tuple[float, float]:
    """(sigma, drift): standard deviation of E_tot about its mean (eV) and the
    slope of a least-squares line through E_tot per atom (eV/atom/ps), the two
    measures of Table II."""
    E = np.asarray(E)
    t_ps = np.arange(len(E)) * dt_fs * 1e-3
    slope = np.polyfit(t_ps, E, 1)[0] if len(E) > 1 else 0.0
    return float(np.std(E)), float(slope / natoms)
