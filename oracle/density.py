"""Density matrices: diagonalisation (the plain definition) and the SP2 recursion.

At T_e = 0 the density matrix is the step function of the Hamiltonian,
D = theta(mu0 I - H) (App. D.2, with H = H[n]): the projector on
the N_occ lowest eigenvectors, doubly occupied (so Tr D = N_occ = N_e/2).  At
T_e > 0 it is the Fermi operator D = (exp(beta (H - mu0 I)) + 1)^-1 of
Eq. EL_4c / Eq. DM_perp, with mu0 fixed by Tr D = N_occ (canonical reading).

SP2 (the recursive second-order spectral projection of Sec. III.B): the paper
defers its details to the cited SP2 work.  Reading used here and on the GPU:
  X0 = (eps_max I - H)/(eps_max - eps_min) with Gershgorin bounds;
  at each step compute Tr X and Tr X^2 (= ||X||_F^2 for symmetric X); stop when
  Tr X - Tr X^2 <= tol; otherwise take X <- X^2 when
  |Tr X^2 - N_occ| <= |2 Tr X - Tr X^2 - N_occ| and X <- 2X - X^2 otherwise
  (the projection whose trace lands closer to N_occ; ties go to X^2).
The thresholded variant drops, after X0 and after every projection, every
bs x bs block whose Frobenius norm is below tau (Sec. III.B applies the
threshold elementwise after each projection; the block rule is the
block-sparse reading).

The recursive Fermi-operator expansion (the finite-temperature construction
the paper cites for linear scaling at T_e > 0, end of Sec. III.C, left
unimplemented there): with f(t) = 1/(1 + e^t), f(t)^2 / (f(t)^2 + (1 -
f(t))^2) = f(2t), so m steps X <- X^2 [X^2 + (I - X)^2]^-1 take the Fermi
operator at beta / 2^m to the one at beta.  Reading used here and on the
GPU: the steps act on E = X - I/2, for which the map is E <- 2E (I + 4E^2)^-1,
starting from E0 = L - 4/3 L^3, L = -beta (H - mu I) / 2^(m+2) (tanh to third
order at beta / 2^m), and each step is written with products only:
  W = (I - 2E)(I + 2E),  A = 2I - W,
  Z = (32 A^2 - 144 A + 210 I) / 99, then ns - 1 Newton-Schulz steps
      T = 2I - A Z, Z <- Z T,
  E <- E + E (Z W).
m is the smallest value >= 8 with beta (hi - lo) <= 2^(m+1) over the
chemical-potential bracket [lo, hi] (the start needs |beta (eps - mu)| <=
2^(m+1)).  D = I/2 + E.  The thresholded variant drops every bs x bs block
with Frobenius norm below tau after L and after every product (the affine
steps P, Q, A are exact and drop nothing).
"""

from __future__ import annotations

import dataclasses

import numpy as np
from scipy.special import expit


@dataclasses.dataclass
class DensityResult:
    D: np.ndarray
    eps: np.ndarray        # eigenvalues, ascending
    mu: float              # chemical potential (mid-gap at T_e = 0)
    gap: float             # eps[N_occ] - eps[N_occ-1] (T_e = 0), else nan
    occ: np.ndarray        # occupations f_i (0/1 at T_e = 0)


def density_T0(H: np.ndarray, n_occ: int) -> DensityResult:
    """D = sum_{i <= N_occ} c_i c_i^T from the eigenvectors of H (LAPACK eigh)."""
    n_occ = int(round(n_occ))
    eps, C = np.linalg.eigh(H)
    Cocc = C[:, :n_occ]
    D = Cocc @ Cocc.T
    n = H.shape[0]
    gap = float(eps[n_occ] - eps[n_occ - 1]) if 0 < n_occ < n else float("inf")
    mu = 0.5 * float(eps[n_occ] + eps[n_occ - 1]) if 0 < n_occ < n else float("nan")
    occ = np.zeros(n)
    occ[:n_occ] = 1.0
    return DensityResult(D=D, eps=eps, mu=mu, gap=gap, occ=occ)


def fermi_occupations(eps: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """f_i = [exp((eps_i - mu)/kT) + 1]^-1 (computed as a logistic to avoid overflow)."""
    return expit(-(eps - mu) / kT)


def density_fermi(H: np.ndarray, n_occ: float, kT: float, tol: float = 1e-13,
                  max_iter: int = 400) -> DensityResult:
    """D = C f(eps) C^T with mu found by bisection so that sum_i f_i = N_occ."""
    eps, C = np.linalg.eigh(H)
    lo, hi = eps[0] - 60.0 * kT - 1.0, eps[-1] + 60.0 * kT + 1.0
    mu = 0.5 * (lo + hi)
    for _ in range(max_iter):
        mu = 0.5 * (lo + hi)
        s = fermi_occupations(eps, mu, kT).sum()
        if abs(s - n_occ) <= tol * max(1.0, n_occ):
            break
        if s > n_occ:
            hi = mu
        else:
            lo = mu
    f = fermi_occupations(eps, mu, kT)
    D = (C * f) @ C.T
    return DensityResult(D=D, eps=eps, mu=float(mu), gap=float("nan"), occ=f)


def entropy_kB(occ: np.ndarray) -> float:
    """S / k_B = -2 sum_i [f ln f + (1 - f) ln(1 - f)] (Eq. Entropy), with 0 ln 0 = 0."""
    f = np.clip(occ, 0.0, 1.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(f > 0, f * np.log(f), 0.0)
        b = np.where(f < 1, (1 - f) * np.log1p(-f), 0.0)
    return float(-2.0 * np.sum(a + b))


def gershgorin(H: np.ndarray) -> tuple[float, float]:
    """Gershgorin bounds: min_i (H_ii - R_i), max_i (H_ii + R_i), R_i = sum_{j!=i} |H_ij|."""
    d = np.diag(H)
    r = np.abs(H).sum(axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


@dataclasses.dataclass
class SP2Result:
    X: np.ndarray
    iters: int                 # number of projections applied
    branches: list             # 0 = X^2, 1 = 2X - X^2
    converged: bool
    idem: float                # final Tr X - Tr X^2
    eps_min: float
    eps_max: float
    idem_history: list
    pre_drop_norms: np.ndarray = None  # tau > 0: bs x bs block norms of the last iterate before its drop


def block_norms(X: np.ndarray, bs: int) -> np.ndarray:
    """Frobenius norm of every bs x bs block of X (ragged edge blocks are smaller)."""
    n = X.shape[0]
    nb = (n + bs - 1) // bs
    out = np.zeros((nb, nb))
    for I in range(nb):
        for J in range(nb):
            blk = X[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs]
            out[I, J] = np.sqrt(np.sum(blk * blk))
    return out


def _drop_blocks(X: np.ndarray, bs: int, tau: float) -> tuple[np.ndarray, np.ndarray]:
    """Zero every bs x bs block of X whose Frobenius norm is below tau; also
    returns the block norms before the drop."""
    norms = block_norms(X, bs)
    Y = X.copy()
    for I, J in zip(*np.nonzero(norms < tau)):
        Y[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = 0.0
    return Y, norms


def sp2(H: np.ndarray, n_occ: float, tol: float = 1e-10, max_iter: int = 100,
        rule: str = "lookahead", tau: float = 0.0, bs: int = 32) -> SP2Result:
    """SP2 recursion in FP64 (reading in the module docstring).  rule="simple"
    uses the alternative branch X^2 if Tr X > N_occ else 2X - X^2.  tau > 0
    applies the bs x bs block-Frobenius drop after X0 and after every
    projection."""
    emin, emax = gershgorin(H)
    n = H.shape[0]
    X = (emax * np.eye(n) - H) / (emax - emin)
    norms = None
    if tau > 0:
        X, norms = _drop_blocks(X, bs, tau)
    branches, hist = [], []
    converged = False
    idem = float("nan")
    for _ in range(max_iter + 1):
        t1 = float(np.trace(X))
        t2 = float(np.sum(X * X))
        idem = t1 - t2
        hist.append(idem)
        if idem <= tol:
            converged = True
            break
        if len(branches) == max_iter:
            break
        if rule == "lookahead":
            b = 0 if abs(t2 - n_occ) <= abs(2.0 * t1 - t2 - n_occ) else 1
        else:
            b = 0 if t1 > n_occ else 1
        X2 = X @ X
        X = X2 if b == 0 else 2.0 * X - X2
        if tau > 0:
            X, norms = _drop_blocks(X, bs, tau)
        branches.append(b)
    return SP2Result(X=X, iters=len(branches), branches=branches, converged=converged,
                     idem=idem, eps_min=emin, eps_max=emax, idem_history=hist, pre_drop_norms=norms)


@dataclasses.dataclass
class FermiExpansionResult:
    D: np.ndarray
    mu: float
    m: int                     # doubling steps
    expansions: int            # chemical-potential iterations (one expansion each)
    trace: float               # Tr D
    converged: bool
    pre_drop_norms: np.ndarray = None  # tau > 0: bs x bs block norms of the final E before its drop


def fermi_expansion(H: np.ndarray, n_occ: float, kT: float, tau: float = 0.0, bs: int = 32,
                    m_max: int = 14, ns_iters: int = 3, trace_tol: float = 1e-10,
                    mu_iters: int = 80) -> FermiExpansionResult:
    """The recursive Fermi-operator expansion in FP64 (reading in the module
    docstring), with mu such that Tr D = N_occ to trace_tol: bisection on the
    bracket [eps_min - 40 kT - 1, eps_max + 40 kT + 1] (Gershgorin), taking
    Newton's step -dev / (beta Tr D(I - D)) when it stays inside the bracket
    (Tr D(I - D) = n/4 - ||E||_F^2)."""
    n = H.shape[0]
    beta = 1.0 / kT
    I = np.eye(n)
    emin, emax = gershgorin(H)
    lo, hi = emin - 40.0 * kT - 1.0, emax + 40.0 * kT + 1.0
    m = min(8, m_max)
    while m < m_max and not beta * (hi - lo) <= 2.0 ** (m + 1):
        m += 1

    def drop(X):
        return _drop_blocks(X, bs, tau) if tau > 0 else (X, None)

    def expansion(mu):
        L, _ = drop(-beta / 2.0 ** (m + 2) * (H - mu * I))
        L2, _ = drop(L @ L)
        E, norms = drop(L - 4.0 / 3.0 * (L @ L2))
        for _ in range(m):
            W, _ = drop((I - 2.0 * E) @ (I + 2.0 * E))
            A = 2.0 * I - W
            Z, _ = drop((32.0 * (A @ A) - 144.0 * A + 210.0 * I) / 99.0)
            for _ in range(ns_iters - 1):
                T, _ = drop(2.0 * I - A @ Z)
                Z, _ = drop(Z @ T)
            V, _ = drop(Z @ W)
            E, norms = drop(E + E @ V)
        return E, norms

    mu = 0.5 * (emin + emax)
    E, norms, it, converged = None, None, 0, False
    for it in range(1, mu_iters + 1):
        E, norms = expansion(mu)
        dev = 0.5 * n + float(np.trace(E)) - n_occ
        if abs(dev) <= trace_tol:
            converged = True
            break
        if dev > 0:
            hi = mu
        else:
            lo = mu
        t1 = 0.25 * n - float(np.sum(E * E))
        nxt = mu - dev / (beta * t1) if t1 > 1e-14 else float("nan")
        mu = nxt if lo < nxt < hi else 0.5 * (lo + hi)
    D = 0.5 * I + E
    return FermiExpansionResult(D=D, mu=float(mu), m=m, expansions=it, trace=float(np.trace(D)),
                                converged=converged, pre_drop_norms=norms)


def idempotency_fro(X: np.ndarray) -> float:
    """||X^2 - X||_F."""
    return float(np.linalg.norm(X @ X - X))


def commutator_fro(H: np.ndarray, D: np.ndarray) -> float:
    """||[H, D]||_F = ||HD - DH||_F."""
    return float(np.linalg.norm(H @ D - D @ H))
