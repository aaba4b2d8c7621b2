"""Mulliken charges, energy and forces of the orthogonal T_e = 0 scheme.

Mulliken net charges (App. D): q_i = 2 sum_{a in i} (D_aa - D0_aa) = 2 sum_{a in i}
D_aa - N0_i, with N0_i the valence electrons of the neutral atom (6 for O,
1 for H); positive q means excess electrons.

Energy and force (Eq. EL_Orth_a, Eq. Etot_Orth).  Reading: the conserved
quantity of the force of Eq. EL_Orth_a is taken as
    E = KE + 2 Tr[h D] + 1/2 (2q - n)^T gamma n + E_pair,
the Harris-Foulkes-like form of App. C applied to the SCC energy, and
    F = -dE/dR at fixed n = -2 Tr[D dh/dR] - 1/2 (2q - n)^T (dgamma/dR) n - dE_pair/dR.
This equals Eq. EL_Orth_a when the population 2 sum_a D_aa that multiplies the
gamma derivative inside Tr[D H_R] is taken net of the neutral-atom reference,
and it reduces at n = q to the SCC-TB energy 2 Tr[hD] + 1/2 q^T gamma q.
The D-derivative terms vanish because D = theta(mu0 - H[n]) at fixed N_occ
(Tr[H dD] = 0 for a gapped projector).
"""

from __future__ import annotations

import numpy as np

from workloads.water import TYPE_O, ModelParams, EV_PER_AMU_A2_FS2
from . import tb


def neutral_electrons(types: np.ndarray, p: ModelParams) -> np.ndarray:
    return np.where(types == TYPE_O, p.n0_O, p.n0_H).astype(np.float64)


def mulliken(D: np.ndarray, types: np.ndarray, p: ModelParams) -> np.ndarray:
    """q_i = 2 sum_{a in i} D_aa - N0_i."""
    offs = tb.orbital_offsets(types)
    d = np.diag(D)
    pop = np.array([2.0 * d[offs[i]:offs[i + 1]].sum() for i in range(len(types))])
    return pop - neutral_electrons(types, p)


def kinetic_energy(v: np.ndarray, masses: np.ndarray) -> float:
    """1/2 sum M v^2 in eV (v in A/fs, M in amu)."""
    return float(0.5 * np.sum(masses[:, None] * v * v) / EV_PER_AMU_A2_FS2)


def energy_terms(R, types, box, p: ModelParams, D, q, n_aux, G=None, pairs=None):
    """Potential-energy terms (eV): 2 Tr[hD], 1/2 (2q - n)^T gamma n, E_pair."""
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    h = tb.build_h(R, types, box, p, pairs)
    if G is None:
        G = tb.build_gamma(R, box, p, pairs)
    e_band = 2.0 * float(np.sum(h * D))
    e_scc = 0.5 * float((2.0 * q - n_aux) @ G @ n_aux)
    e_pair = tb.pair_energy(R, box, p, pairs)
    return e_band, e_scc, e_pair


def potential_energy(R, types, box, p, D, q, n_aux, pairs=None) -> float:
    return float(sum(energy_terms(R, types, box, p, D, q, n_aux, pairs=pairs)))


def forces(R, types, box, p: ModelParams, D, q, n_aux, pairs=None) -> np.ndarray:
    """F = -dE/dR at fixed n and fixed D (see module docstring), [N, 3] eV/A."""
    N = R.shape[0]
    offs = tb.orbital_offsets(types)
    if pairs is None:
        pairs = tb.pair_images(R, box, tb.pair_range(p))
    Vr = tb.hopping_radial(p)
    gr = tb.gamma_radial(p)
    pr = tb.pair_radial(p)
    w = 2.0 * q - n_aux
    dE = np.zeros((N, 3))
    ewald = p.gamma_form == 1
    if ewald:
        # every pair interacts through the long-range gamma
        _, dG = tb.gamma_ewald(R, box, p, with_grad=True)
        for i in range(N):
            for j in range(i + 1, N):
                g = 0.5 * (w[i] * n_aux[j] + w[j] * n_aux[i]) * dG[i, j]
                dE[j] += g
                dE[i] -= g
    for i, j, d in zip(*pairs):
        if i == j:
            continue  # a self-image term depends on the box only
        r = float(np.sqrt(d @ d))
        u = d / r
        _, dblk = tb.sk_block(int(types[i]), int(types[j]), d, Vr)
        Dij = D[offs[i]:offs[i + 1], offs[j]:offs[j + 1]]
        # 2 Tr[hD]: block (i,j) and its transpose (j,i) both depend on d
        g_band = 4.0 * np.einsum("ab,abk->k", Dij, dblk)
        dg = 0.0 if ewald else gr(r)[1]
        g_scc = 0.5 * (w[i] * n_aux[j] + w[j] * n_aux[i]) * dg * u
        _, dphi = pr(r)
        g_pair = dphi * u
        g = g_band + g_scc + g_pair           # dE/dd, with dd/dR_j = +1, dd/dR_i = -1
        dE[j] += g
        dE[i] -= g
    return -dE
