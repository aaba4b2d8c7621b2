"""Orthogonal self-consistent-charge tight-binding model (App. D, S = I).

H[n]_{ia,jb} = h_{ia,jb}(R) + delta_ij delta_ab sum_l gamma_il n_l
(Eq. DFTB_2 with S = I and the Mulliken charges q replaced by the dynamical
charges n, as in Eq. EL_Orth_c).

Readings of what the paper leaves open (the paper uses LATTE parameters that
are not given):
  * hopping: Slater-Koster two-centre form whose four bond integrals share
    the radial function V(r) = t exp(-r/r_decay): ss-sigma = -V,
    sp-sigma = +V, pp-sigma = +V, pp-pi = -V;
  * gamma_ij = sum over periodic images of g(|R_j - R_i + T|) with
    g(r) = k/sqrt(r^2 + (k/U)^2) * w(r/rg), w(x) = (1-x)^4 (1+4x) for x < 1
    and 0 beyond.  g equals the Hubbard U on site and decays like 1/R inside
    its range (App. D).  The window w is Wendland's compactly supported
    positive-definite function, so g (a product of two positive-definite
    radial kernels) keeps gamma positive definite and the SCC functional
    convex, which the optimization-free dynamics requires (Sec. II.C).  The
    App. D tail is not used for gamma: the paper applies it to h, S and phi;
  * the radial functions of h and of the pair potential phi are replaced for
    r1 <= R < rcut by the quintic tail t(R) of App. D, whose coefficients
    B0..B5 match f, f', f'' at r1 and vanish with two derivatives at rcut;
    beyond rcut they are zero;
  * the radial form of the bond integrals and of phi is App. D's
    zeta(R) = A0 exp(A1 R + A2 R^2 + A3 R^3 + A4 R^4), with A0 = t_hop
    (pair_a), A1 = -1/r_decay (-1/pair_rho) and A2..A4 = zeta_a2..a4
    (pair_a2..a4), all zero by default (a plain exponential);
  * gamma_form = 1 replaces the windowed gamma by Gaussian charges of width
    c = 2k/(U sqrt(pi)) (so that gamma_ii = U on site), whose interaction
    k erf(r/c)/r decays like k/R and is summed over all periodic images by
    Ewald's method with a neutralising background (the long-range gamma; the
    paper only fixes the 1/R decay and the on-site U).
"""

from __future__ import annotations

import numpy as np

from workloads.water import TYPE_O, TYPE_H, ModelParams

NORB = {TYPE_O: 4, TYPE_H: 1}


# --------------------------------------------------------------------------
# cut-off tail (App. D, equation for t(R))
# --------------------------------------------------------------------------

def tail_coeffs(f0: float, f1: float, f2: float, r1: float, rc: float) -> np.ndarray:
    """B0..B5 of t(R) = B0 + dR(B1 + dR(B2 + dR(B3 + dR(B4 + dR B5)))), dR = R - r1,
    from the six conditions of App. D: t, t', t'' equal f, f', f'' at r1 and
    vanish at rc.  Solved as the plain 6x6 linear system."""
    D = rc - r1
    A = np.array([
        [1, 0, 0, 0, 0, 0],
        [0, 1, 0, 0, 0, 0],
        [0, 0, 2, 0, 0, 0],
        [1, D, D**2, D**3, D**4, D**5],
        [0, 1, 2 * D, 3 * D**2, 4 * D**3, 5 * D**4],
        [0, 0, 2, 6 * D, 12 * D**2, 20 * D**3],
    ], dtype=np.float64)
    b = np.array([f0, f1, f2, 0.0, 0.0, 0.0])
    return np.linalg.solve(A, b)


def tail_eval(B: np.ndarray, dR: float) -> tuple[float, float]:
    """t(R) and t'(R) at dR = R - r1."""
    t = 0.0
    for c in B[::-1]:
        t = t * dR + c
    dt = 0.0
    for k in range(5, 0, -1):
        dt = dt * dR + k * B[k]
    return t, dt


class Radial:
    """A radial function with its App. D cut-off tail: f for R < r1, the
    quintic t(R) for r1 <= R < rc, zero beyond."""

    def __init__(self, f, df, d2f, r1: float, rc: float):
        self.f, self.df, self.r1, self.rc = f, df, r1, rc
        self.B = tail_coeffs(f(r1), df(r1), d2f(r1), r1, rc)

    def __call__(self, r: float) -> tuple[float, float]:
        """(value, derivative) at distance r."""
        if r < self.r1:
            return self.f(r), self.df(r)
        if r < self.rc:
            return tail_eval(self.B, r - self.r1)
        return 0.0, 0.0


def zeta_radial(A0: float, A: tuple, r1: float, rc: float) -> Radial:
    """zeta(R) = A0 exp(A1 R + A2 R^2 + A3 R^3 + A4 R^4) (App. D) with its tail;
    A = (A1, A2, A3, A4).  zeta' = P' zeta, zeta'' = (P'' + P'^2) zeta with
    P the polynomial in the exponent."""
    a1, a2, a3, a4 = A

    def P(r):
        return r * (a1 + r * (a2 + r * (a3 + r * a4)))

    def dP(r):
        return a1 + r * (2 * a2 + r * (3 * a3 + r * 4 * a4))

    def d2P(r):
        return 2 * a2 + r * (6 * a3 + r * 12 * a4)

    return Radial(lambda r: A0 * np.exp(P(r)),
                  lambda r: A0 * dP(r) * np.exp(P(r)),
                  lambda r: A0 * (d2P(r) + dP(r) ** 2) * np.exp(P(r)), r1, rc)


def hopping_radial(p: ModelParams) -> Radial:
    """V(r) = zeta(r) with A0 = t, A1 = -1/r_decay, and its tail."""
    return zeta_radial(p.t_hop, (-1.0 / p.r_decay, p.zeta_a2, p.zeta_a3, p.zeta_a4), p.r1, p.rcut)


class GammaRadial:
    """g(r) = k / sqrt(r^2 + (k/U)^2) * w(r/rg), w(x) = (1-x)^4 (1+4x) on [0, 1);
    g(0) = U."""

    def __init__(self, p: ModelParams):
        self.k, self.a2, self.rg = p.coulomb_k, (p.coulomb_k / p.hubbard_u) ** 2, p.gamma_cut

    def __call__(self, r: float) -> tuple[float, float]:
        if r >= self.rg:
            return 0.0, 0.0
        x = r / self.rg
        w = (1 - x) ** 4 * (1 + 4 * x)
        dw = (-4 * (1 - x) ** 3 * (1 + 4 * x) + 4 * (1 - x) ** 4) / self.rg
        ko = self.k / np.sqrt(r * r + self.a2)
        dko = -self.k * r / (r * r + self.a2) ** 1.5
        return ko * w, dko * w + ko * dw


def gamma_radial(p: ModelParams) -> GammaRadial:
    return GammaRadial(p)


def pair_radial(p: ModelParams) -> Radial:
    """phi(r) = zeta(r) with A0 = pair_a, A1 = -1/pair_rho, and its tail (the
    short-range repulsion of E_pair)."""
    a1 = -1.0 / p.pair_rho if p.pair_a != 0.0 else 0.0
    return zeta_radial(p.pair_a, (a1, p.pair_a2, p.pair_a3, p.pair_a4), p.r1, p.rcut)


# --------------------------------------------------------------------------
# orbitals and neighbours
# --------------------------------------------------------------------------

def pair_range(p: ModelParams) -> float:
    """Largest short-range interaction: hopping, pair potential and (windowed) gamma."""
    return max(p.rcut, p.gamma_cut) if p.gamma_form == 0 else p.rcut


def orbital_offsets(types: np.ndarray) -> np.ndarray:
    """offs[i] = first orbital of atom i, offs[N] = n; orbitals grouped by atom
    (O: s, px, py, pz; H: s)."""
    counts = np.array([NORB[int(t)] for t in types], dtype=np.int64)
    offs = np.zeros(len(types) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    return offs


def onsite_energies(types: np.ndarray, p: ModelParams) -> np.ndarray:
    e = []
    for t in types:
        e.extend([p.eps_s_O, p.eps_p_O, p.eps_p_O, p.eps_p_O] if t == TYPE_O else [p.eps_s_H])
    return np.array(e, dtype=np.float64)


def pair_images(R: np.ndarray, box: float, rc: float):
    """All (i, j, d) with d = R_j - R_i + T for lattice vectors T = box*(k1,k2,k3)
    and |d| < rc: pairs i < j with any T, and i == j with T != 0.  The
    displacement is first reduced to the minimum image, then shifted by the
    images that can still fall inside rc."""
    N = R.shape[0]
    nimg = int(np.ceil(rc / box + 0.5))
    rng = np.arange(-nimg, nimg + 1)
    shifts = np.array([(a, b, c) for a in rng for b in rng for c in rng], dtype=np.float64) * box
    out_i, out_j, out_d = [], [], []
    for i in range(N):
        d0 = R[i:] - R[i]
        d0 = d0 - box * np.round(d0 / box)
        d = d0[:, None, :] + shifts[None, :, :]          # [N-i, S, 3]
        r2 = np.einsum("jsk,jsk->js", d, d)
        mask = r2 < rc * rc
        mask[0] &= r2[0] > 1e-12                          # i == j: drop T = 0
        jj, ss = np.nonzero(mask)
        out_i.append(np.full(jj.shape, i))
        out_j.append(jj + i)
        out_d.append(d[jj, ss])
    return (np.concatenate(out_i), np.concatenate(out_j),
            np.concatenate(out_d).reshape(-1, 3))


# --------------------------------------------------------------------------
# Slater-Koster blocks
# --------------------------------------------------------------------------

def sk_block(ta: int, tb: int, d: np.ndarray, Vr: Radial):
    """Hopping block between the orbitals of an atom of type ta and one of type
    tb displaced by d (from a to b), and its derivative with respect to d.

    Two-centre Slater-Koster table with direction cosines l = d/|d|:
      <s|s> = Vss, <s|p_c> = l_c Vsp, <p_c|s> = -l_c Vsp,
      <p_c|p_e> = l_c l_e Vpp_sigma + (delta_ce - l_c l_e) Vpp_pi,
    with Vss = -V, Vsp = +V, Vpp_sigma = +V, Vpp_pi = -V.
    Returns (block [na, nb], dblock [na, nb, 3])."""
    r = float(np.sqrt(d @ d))
    V, dV = Vr(r)
    l = d / r
    dl = (np.eye(3) - np.outer(l, l)) / r        # dl[c, k] = d l_c / d d_k
    Vss, dVss = -V, -dV
    Vsp, dVsp = V, dV
    Vps, dVps = V, dV        # pp-sigma
    Vpi, dVpi = -V, -dV      # pp-pi

    def s_s():
        return np.array([[Vss]]), (dVss * l)[None, None, :]

    def s_p():
        blk = (l * Vsp)[None, :]                                  # [1, 3]
        dblk = (dl * Vsp + np.outer(l, l) * dVsp)[None, :, :]     # [1, 3, 3]
        return blk, dblk

    def p_p():
        ll = np.outer(l, l)
        blk = ll * (Vps - Vpi) + np.eye(3) * Vpi
        dll = np.einsum("ck,e->cek", dl, l) + np.einsum("c,ek->cek", l, dl)
        dblk = (dll * (Vps - Vpi) + ll[:, :, None] * (dVps - dVpi) * l[None, None, :]
                + np.eye(3)[:, :, None] * dVpi * l[None, None, :])
        return blk, dblk

    na, nb = NORB[ta], NORB[tb]
    blk = np.zeros((na, nb))
    dblk = np.zeros((na, nb, 3))
    b, db = s_s()
    blk[0, 0], dblk[0, 0] = b[0, 0], db[0, 0]
    if nb == 4:
        b, db = s_p()
        blk[0, 1:], dblk[0, 1:] = b[0], db[0]
    if na == 4:
        b, db = s_p()
        blk[1:, 0], dblk[1:, 0] = -b[0], -db[0]
    if na == 4 and nb == 4:
        b, db = p_p()
        blk[1:, 1:], dblk[1:, 1:] = b, db
    return blk, dblk


# --------------------------------------------------------------------------
# h(R), gamma(R), H[n]
# --------------------------------------------------------------------------

def build_h(R: np.ndarray, types: np.ndarray, box: float, p: ModelParams,
            pairs=None) -> np.ndarray:
    """Charge-independent Hamiltonian h(R): onsite energies on the diagonal,
    Slater-Koster blocks between every atom and every periodic image of every
    other atom (and of itself) within rcut."""
    offs = orbital_offsets(types)
    n = int(offs[-1])
    h = np.diag(onsite_energies(types, p))
    Vr = hopping_radial(p)
    if pairs is None:
        pairs = pair_images(R, box, pair_range(p))
    for i, j, d in zip(*pairs):
        blk, _ = sk_block(int(types[i]), int(types[j]), d, Vr)
        si, sj = slice(offs[i], offs[i + 1]), slice(offs[j], offs[j + 1])
        h[si, sj] += blk
        if i != j:
            h[sj, si] += blk.T
    return h


def build_gamma(R: np.ndarray, box: float, p: ModelParams, pairs=None) -> np.ndarray:
    """gamma_ij = sum over images T of g(|R_j - R_i + T|), including the
    on-site g(0) = U on the diagonal (gamma_form 0), or the Ewald-summed
    Gaussian-charge gamma (gamma_form 1)."""
    if p.gamma_form == 1:
        return gamma_ewald(R, box, p)
    N = R.shape[0]
    gr = gamma_radial(p)
    G = np.eye(N) * p.hubbard_u
    if pairs is None:
        pairs = pair_images(R, box, pair_range(p))
    for i, j, d in zip(*pairs):
        g, _ = gr(float(np.sqrt(d @ d)))
        G[i, j] += g
        if i != j:
            G[j, i] += g
    return G


def build_H(h: np.ndarray, G: np.ndarray, types: np.ndarray, n_aux: np.ndarray) -> np.ndarray:
    """H[n] = h + diag(sum_l gamma_il n_l) on every orbital of atom i
    (Eq. DFTB_2 with S = I; Eq. EL_Orth_c)."""
    offs = orbital_offsets(types)
    shift = G @ n_aux
    H = h.copy()
    for i in range(len(types)):
        for a in range(offs[i], offs[i + 1]):
            H[a, a] += shift[i]
    return H


def pair_energy(R: np.ndarray, box: float, p: ModelParams, pairs=None) -> float:
    """E_pair = sum over pairs (and self-images, counted once per pair of
    opposite images) of phi(r)."""
    if p.pair_a == 0.0:
        return 0.0
    pr = pair_radial(p)
    if pairs is None:
        pairs = pair_images(R, box, pair_range(p))
    E = 0.0
    for i, j, d in zip(*pairs):
        phi, _ = pr(float(np.sqrt(d @ d)))
        E += phi if i != j else 0.5 * phi
    return E


# --------------------------------------------------------------------------
# long-range gamma: Gaussian charges, Ewald summation
# --------------------------------------------------------------------------

def gaussian_width(p: ModelParams) -> float:
    """c with k erf(r/c)/r -> U at r -> 0: c = 2k / (U sqrt(pi))."""
    return 2.0 * p.coulomb_k / (p.hubbard_u * np.sqrt(np.pi))


def ewald_alpha(box: float, alpha: float = 0.0) -> float:
    """Splitting parameter (1/A): the given one, else 6.5 / max(box, 10 A), so
    the real-space sum needs images up to about max(box, 10 A)."""
    return alpha if alpha > 0.0 else 6.5 / max(box, 10.0)


def _lattice(box: float, rmax: float) -> np.ndarray:
    m = int(np.ceil(rmax / box)) + 1
    r = np.arange(-m, m + 1)
    return np.array([(a, b, c) for a in r for b in r for c in r], dtype=np.float64) * box


def _reciprocal(box: float, alpha: float):
    """G != 0 with exp(-G^2/(4 alpha^2)) above 1e-19 and their weights
    A_G = (4 pi / V) exp(-G^2/(4 alpha^2)) / G^2."""
    gmax = 2.0 * alpha * 6.6
    m = int(np.ceil(gmax * box / (2 * np.pi)))
    r = np.arange(-m, m + 1)
    G = np.array([(a, b, c) for a in r for b in r for c in r if (a, b, c) != (0, 0, 0)],
                 dtype=np.float64) * (2 * np.pi / box)
    G2 = np.einsum("gk,gk->g", G, G)
    keep = G2 <= gmax * gmax
    G, G2 = G[keep], G2[keep]
    A = 4.0 * np.pi / box**3 * np.exp(-G2 / (4.0 * alpha * alpha)) / G2
    return G, A


def ewald_psi(d: np.ndarray, box: float, alpha: float, self_term: bool = False):
    """Potential of a unit point charge and all its periodic images in a
    neutralising background, at displacements d [M, 3] (Ewald's split):
      psi(d) = sum_L erfc(alpha |d + L|)/|d + L|
               + (4 pi / V) sum_{G != 0} exp(-G^2/4 alpha^2) cos(G.d) / G^2 - pi/(alpha^2 V).
    self_term: d = 0 and the L = 0 term left out, which adds -2 alpha/sqrt(pi).
    Returns (psi [M], grad [M, 3])."""
    from scipy.special import erfc
    d = np.atleast_2d(d)
    L = _lattice(box, 6.6 / alpha)
    G, A = _reciprocal(box, alpha)
    psi = np.zeros(len(d))
    grad = np.zeros((len(d), 3))
    for m, dm in enumerate(d):
        x = dm[None, :] + L
        r = np.sqrt(np.einsum("lk,lk->l", x, x))
        ok = r > 1e-12
        x, r = x[ok], r[ok]
        f = erfc(alpha * r) / r
        df = (-2.0 * alpha / np.sqrt(np.pi) * np.exp(-(alpha * r) ** 2) - f) / r
        psi[m] = np.sum(f)
        grad[m] = np.sum((df / r)[:, None] * x, axis=0)
        gd = G @ dm
        psi[m] += np.sum(A * np.cos(gd))
        grad[m] -= np.sum((A * np.sin(gd))[:, None] * G, axis=0)
    psi -= np.pi / (alpha * alpha * box**3)
    if self_term:
        psi -= 2.0 * alpha / np.sqrt(np.pi)
    return psi, grad


def _gauss_short(d: np.ndarray, box: float, c: float, self_term: bool = False):
    """sum_L erfc(|d + L|/c)/|d + L| over all images (L = 0 left out at d = 0),
    and its gradient."""
    from scipy.special import erfc
    d = np.atleast_2d(d)
    L = _lattice(box, 6.6 * c)
    out = np.zeros(len(d))
    grad = np.zeros((len(d), 3))
    for m, dm in enumerate(d):
        x = dm[None, :] + L
        r = np.sqrt(np.einsum("lk,lk->l", x, x))
        ok = r > 1e-12
        x, r = x[ok], r[ok]
        f = erfc(r / c) / r
        df = (-2.0 / (c * np.sqrt(np.pi)) * np.exp(-(r / c) ** 2) - f) / r
        out[m] = np.sum(f)
        grad[m] = np.sum((df / r)[:, None] * x, axis=0)
    return out, grad


def gamma_ewald(R: np.ndarray, box: float, p: ModelParams, with_grad: bool = False):
    """gamma_ij = k sum_L erf(|d + L|/c)/|d + L|, d = R_j - R_i, over all images
    (Ewald, neutralising background) = k [psi(d) - sum_L erfc(|d + L|/c)/|d + L|];
    on the diagonal the L = 0 term is its on-site limit 2k/(c sqrt(pi)) = U.
    with_grad: also dgamma[i, j] = d gamma_ij / d d (antisymmetric in i, j)."""
    N = R.shape[0]
    k, c = p.coulomb_k, gaussian_width(p)
    alpha = ewald_alpha(box, p.ewald_alpha)
    G = np.zeros((N, N))
    dG = np.zeros((N, N, 3))
    iu, ju = np.triu_indices(N, 1)
    d = R[ju] - R[iu]
    psi, gpsi = ewald_psi(d, box, alpha)
    sr, gsr = _gauss_short(d, box, c)
    G[iu, ju] = G[ju, iu] = k * (psi - sr)
    dG[iu, ju] = k * (gpsi - gsr)
    dG[ju, iu] = -dG[iu, ju]
    psi0, _ = ewald_psi(np.zeros((1, 3)), box, alpha, self_term=True)
    s0, _ = _gauss_short(np.zeros((1, 3)), box, c)
    G[np.arange(N), np.arange(N)] = p.hubbard_u + k * (psi0[0] - s0[0])
    return (G, dG) if with_grad else G
