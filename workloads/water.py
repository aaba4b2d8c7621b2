"""Water-like synthetic systems for the orthogonal SCC tight-binding model.

The paper's own workloads (liquid methane, polyethene, HNCO, naphthalene with
LATTE parameters; Sec. III) are not available, so seeded synthetic
"water-like" systems stand in for them: heavy O-like atoms carrying an sp
basis (s, px, py, pz) and light H-like atoms carrying one s orbital, placed
at random in a periodic cube.  Everything here is input generation: no
Hamiltonian, density matrix, charge or force is computed in this module.

Units: eV, Angstrom, amu, fs, K.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

TYPE_O = 0  # sp basis: s, px, py, pz
TYPE_H = 1  # s basis

AMU_G = 1.66054  # 1 amu in units of 1e-24 g, so L^3[A^3] = m[amu]*AMU_G/rho[g/cc]
KB_EV = 8.617333262e-5  # Boltzmann constant, eV/K
EV_PER_AMU_A2_FS2 = 9.648533e-3  # 1 eV/(A amu) expressed in A/fs^2


@dataclasses.dataclass(frozen=True)
class ModelParams:
    """Constants of the orthogonal water-like SCC-TB recipe.

    Onsite energies: O-s -20 eV, O-p -12 eV, H-s -7 eV.  Hopping magnitude
    t*exp(-r/r_decay) with t = 3 eV and r_decay = 0.5 A, smoothly cut between
    r1 and rcut by the quintic tail of App. D.  Hubbard U = 10 eV sets the
    on-site value of gamma; coulomb_k is e^2/(4 pi eps0) in eV*A and
    gamma_cut the range of gamma's compactly supported window.  Neutral
    atoms carry n0_O = 6 and n0_H = 1 valence electrons.  The short-range
    repulsive pair potential of E_pair is pair_a*exp(-r/pair_rho) with the
    App. D tail; pair_a = 24 eV, pair_rho = 0.3 A put an isolated H2O-like
    molecule of this model in equilibrium at r_OH = 0.96 A (pair_a = 0
    switches E_pair off).
    """

    eps_s_O: float = -20.0
    eps_p_O: float = -12.0
    eps_s_H: float = -7.0
    t_hop: float = 3.0
    r_decay: float = 0.5
    hubbard_u: float = 10.0
    coulomb_k: float = 14.399645
    gamma_cut: float = 6.0
    r1: float = 5.0
    rcut: float = 6.0
    n0_O: float = 6.0
    n0_H: float = 1.0
    mass_O: float = 16.0
    mass_H: float = 1.0
    pair_a: float = 24.0
    pair_rho: float = 0.3
    # radial form zeta(R) = A0 exp(A1 R + A2 R^2 + A3 R^3 + A4 R^4) of App. D:
    # A0 = t_hop (pair_a), A1 = -1/r_decay (-1/pair_rho); A2..A4 below
    zeta_a2: float = 0.0
    zeta_a3: float = 0.0
    zeta_a4: float = 0.0
    pair_a2: float = 0.0
    pair_a3: float = 0.0
    pair_a4: float = 0.0
    # gamma: 0 = the windowed short-range form, 1 = Gaussian charges of width
    # set by U with the long-range 1/R tail summed by Ewald (ewald_alpha: the
    # Ewald splitting in 1/A, 0 = chosen from the box)
    gamma_form: int = 0
    ewald_alpha: float = 0.0
    # basis-set overlap between atoms (App. D.1): radial s(r) = overlap_s0
    # exp(-r / overlap_rs) in the Slater-Koster table, the App. D tail between
    # r1 and rcut; overlap_s0 = 0 is the orthogonal model (S = I)
    overlap_s0: float = 0.0
    overlap_rs: float = 0.4


@dataclasses.dataclass(frozen=True)
class XLParams:
    """Integration constants for the auxiliary charges (Eq. Verl_n).

    K = 5 dissipation coefficients c_k and alpha, and kappa0 = dt^2 w^2, are
    the K = 5 values of the modified Verlet scheme with dissipation the paper
    cites for Eq. Verl_n (they are not printed in the paper itself).  The
    paper rescales kappa0 by a positive factor <= 1 (1/2 in all its examples
    but one, 3/4 in that one): kappa = kappa_scale * kappa0.
    """

    dt: float = 0.25
    kappa_scale: float = 0.5
    kappa0: float = 1.82
    alpha: float = 0.018
    c: tuple = (-6.0, 14.0, -8.0, -3.0, 4.0, -1.0)

    @property
    def kappa(self) -> float:
        return self.kappa_scale * self.kappa0

    @property
    def K(self) -> int:
        return len(self.c) - 1


@dataclasses.dataclass
class WaterSystem:
    R: np.ndarray       # [N, 3] float64 positions (A), inside [0, box)
    types: np.ndarray   # [N] int32, TYPE_O or TYPE_H
    box: float          # cubic box side (A)
    seed: int

    @property
    def natoms(self) -> int:
        return int(self.types.shape[0])

    @property
    def n_O(self) -> int:
        return int(np.count_nonzero(self.types == TYPE_O))

    @property
    def n_H(self) -> int:
        return int(np.count_nonzero(self.types == TYPE_H))

    @property
    def norb(self) -> int:
        return 4 * self.n_O + self.n_H

    def n_electrons(self, p: ModelParams = ModelParams()) -> float:
        return p.n0_O * self.n_O + p.n0_H * self.n_H

    def n_occ(self, p: ModelParams = ModelParams()) -> float:
        return 0.5 * self.n_electrons(p)

    def masses(self, p: ModelParams = ModelParams()) -> np.ndarray:
        return np.where(self.types == TYPE_O, p.mass_O, p.mass_H).astype(np.float64)


def atom_counts(natoms: int, p: ModelParams = ModelParams()) -> tuple[int, int]:
    """O/H split of an N-atom water-like system: N_O = floor(N/3), N_H = N - N_O,
    with N_O decremented while the electron count is odd."""
    n_O = natoms // 3
    n_H = natoms - n_O
    while (p.n0_O * n_O + p.n0_H * n_H) % 2 == 1 and n_O > 0:
        n_O -= 1
        n_H += 1
    return n_O, n_H


def box_from_density(n_O: int, n_H: int, density: float, p: ModelParams = ModelParams()) -> float:
    """Cube side (A) holding the given atoms at `density` g/cc."""
    mass = n_O * p.mass_O + n_H * p.mass_H
    return (mass * AMU_G / density) ** (1.0 / 3.0)


def _place_random(natoms: int, box: float, rng: np.random.Generator, min_sep: float,
                  max_tries: int = 100000) -> np.ndarray:
    """Random sequential placement: candidates drawn as (x, y, z) uniform in
    [0, box)^3, rejected when closer than `min_sep` (minimum image) to any
    earlier atom.  A cell grid only speeds up the rejection test."""
    ncell = max(1, int(math.floor(box / min_sep)))
    if ncell < 3:
        ncell = 1
    csize = box / ncell
    cells: dict[tuple[int, int, int], list[int]] = {}
    R = np.empty((natoms, 3), dtype=np.float64)
    ms2 = min_sep * min_sep
    for i in range(natoms):
        for _ in range(max_tries):
            x = rng.random(3) * box
            ok = True
            if ncell == 1:
                if i > 0:
                    d = R[:i] - x
                    d -= box * np.round(d / box)
                    ok = bool(np.all(np.einsum("ij,ij->i", d, d) >= ms2))
            else:
                c = tuple(int(v) % ncell for v in np.floor(x / csize))
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            key = ((c[0] + dx) % ncell, (c[1] + dy) % ncell, (c[2] + dz) % ncell)
                            for j in cells.get(key, ()):
                                d = R[j] - x
                                d -= box * np.round(d / box)
                                if float(d @ d) < ms2:
                                    ok = False
                                    break
                            if not ok:
                                break
                        if not ok:
                            break
                    if not ok:
                        break
            if ok:
                R[i] = x
                if ncell > 1:
                    cells.setdefault(c, []).append(i)
                break
        else:
            raise RuntimeError(f"could not place atom {i} of {natoms} in box {box:.3f} A")
    return R


def _morton_order(R: np.ndarray, box: float, cell: float = 3.0) -> np.ndarray:
    """Permutation sorting atoms by the Morton (Z-order) code of their cell,
    so that atoms close in space get close orbital indices."""
    ncell = max(1, int(box // cell))
    ijk = np.minimum((R / box * ncell).astype(np.int64), ncell - 1)
    code = np.zeros(R.shape[0], dtype=np.int64)
    for bit in range(21):
        for ax in range(3):
            code |= ((ijk[:, ax] >> bit) & 1) << (3 * bit + ax)
    return np.argsort(code, kind="stable")


def water_system(natoms: Optional[int] = None, *, n_O: Optional[int] = None,
                 n_H: Optional[int] = None, box: Optional[float] = None,
                 density: Optional[float] = None, seed: int = 0, min_sep: float = 0.9,
                 morton: bool = False, p: ModelParams = ModelParams()) -> WaterSystem:
    """A seeded water-like system.  The first N_O atoms are O-like and the rest
    H-like (before the optional Morton reordering).  Either `box` or
    `density` (g/cc) fixes the cube side."""
    if n_O is None or n_H is None:
        if natoms is None:
            raise ValueError("give natoms or (n_O, n_H)")
        n_O, n_H = atom_counts(natoms, p)
    if box is None:
        if density is None:
            raise ValueError("give box or density")
        box = box_from_density(n_O, n_H, density, p)
    rng = np.random.default_rng(seed)
    N = n_O + n_H
    R = _place_random(N, float(box), rng, min_sep)
    types = np.array([TYPE_O] * n_O + [TYPE_H] * n_H, dtype=np.int32)
    if morton:
        perm = _morton_order(R, float(box))
        R = R[perm].copy()
        types = types[perm].copy()
    return WaterSystem(R=R, types=types, box=float(box), seed=seed)


def thermal_velocities(masses: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Gaussian (Maxwell-Boltzmann) velocities in A/fs at `temperature` K with
    the centre-of-mass momentum removed."""
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(KB_EV * temperature / masses * EV_PER_AMU_A2_FS2)
    v = rng.standard_normal((masses.shape[0], 3)) * sigma[:, None]
    v -= (masses[:, None] * v).sum(axis=0) / masses.sum()
    return v


def random_gapped_matrix(n: int, n_occ: int, *, gap: float = 1.0, width: float = 20.0,
                         seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Dense symmetric test matrix H = Q diag(eps) Q^T with a known spectrum:
    n_occ eigenvalues spread below -gap/2 and the rest above +gap/2, within
    [-width/2, width/2].  Returns (H, eps) with eps sorted ascending."""
    rng = np.random.default_rng(seed)
    lo = -0.5 * width + rng.random(n_occ) * (0.5 * width - 0.5 * gap)
    hi = 0.5 * gap + rng.random(n - n_occ) * (0.5 * width - 0.5 * gap)
    eps = np.sort(np.concatenate([lo, hi]))
    if n_occ > 0:
        eps[n_occ - 1] = -0.5 * gap
    if n_occ < n:
        eps[n_occ] = 0.5 * gap
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    H = (Q * eps) @ Q.T
    H = 0.5 * (H + H.T)
    return H, eps


def batch_sizes(count: int = 512, lo: int = 16, hi: int = 256, seed: int = 4) -> np.ndarray:
    """Atom counts of the batched workload: uniform integers in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def serving_trajectories(count: int = 64, lo: int = 32, hi: int = 2048, rate: float = 2000.0,
                         n_requests: int = 2000, size_seed: int = 5, arrival_seed: int = 6):
    """Serving workload: trajectory atom counts log-uniform in [lo, hi] and
    Poisson request arrival times (s) at `rate` requests/s in total, each
    request naming a trajectory uniformly at random."""
    rs = np.random.default_rng(size_seed)
    sizes = np.floor(np.exp(rs.uniform(math.log(lo), math.log(hi + 1), size=count))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    ra = np.random.default_rng(arrival_seed)
    gaps = ra.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps)
    which = ra.integers(0, count, size=n_requests)
    return sizes, arrivals, which


def water_24_atoms() -> WaterSystem:
    """8 O + 16 H in a 6.5 A periodic cube, seed 0 (n = 48 orbitals)."""
    return water_system(n_O=8, n_H=16, box=6.5, seed=0)


def water_2048_atoms(seed: int = 0) -> WaterSystem:
    """2048 atoms (682 O + 1366 H, n = 4094 orbitals) at 1.0 g/cc."""
    return water_system(2048, density=1.0, seed=seed)


def water_16384_atoms_morton(seed: int = 0) -> WaterSystem:
    """16384 atoms (5460 O + 10924 H, n = 32764 orbitals) at 1.0 g/cc,
    Morton-ordered so that the density matrix is block sparse."""
    return water_system(16384, density=1.0, seed=seed, morton=True)


def molecular_liquid(n_mol: int, density: float = 1.0, seed: int = 0, bond: float = 0.96,
                     angle_deg: float = 104.5, jitter: float = 0.1, morton: bool = False,
                     p: ModelParams = ModelParams()) -> WaterSystem:
    """n_mol H2O-like molecules at `density` g/cc: O atoms on the first n_mol
    sites (row order) of the smallest cubic grid that holds them, Gaussian
    jitter, random orientations (O-H `bond` A, H-O-H `angle_deg`).  Atom
    order: all O, then the H pairs in molecule order, or Morton order of the
    positions with `morton`."""
    rng = np.random.default_rng(seed)
    box = box_from_density(n_mol, 2 * n_mol, density, p)
    m = 1
    while m ** 3 < n_mol:
        m += 1
    grid = (np.arange(m) + 0.5) / m * box
    th = math.radians(angle_deg)
    u1 = np.array([math.sin(th / 2), math.cos(th / 2), 0.0]) * bond
    u2 = np.array([-math.sin(th / 2), math.cos(th / 2), 0.0]) * bond
    Os, Hs = [], []
    for k in range(n_mol):
        x, y, z = grid[k // (m * m)], grid[(k // m) % m], grid[k % m]
        O = np.array([x, y, z]) + rng.normal(0.0, jitter, 3)
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        Os.append(O)
        Hs += [O + Q @ u1, O + Q @ u2]
    R = np.mod(np.array(Os + Hs), box)
    types = np.array([TYPE_O] * len(Os) + [TYPE_H] * len(Hs), dtype=np.int32)
    if morton:
        perm = _morton_order(R, float(box))
        R = R[perm].copy()
        types = types[perm].copy()
    return WaterSystem(R=R, types=types, box=float(box), seed=seed)


def molecular_water(m: int, box: float, seed: int = 0, bond: float = 0.96,
                    angle_deg: float = 104.5, jitter: float = 0.1) -> WaterSystem:
    """m^3 H2O-like molecules (O-H `bond` A, H-O-H `angle_deg`) with random
    orientations, their O atoms on an m x m x m grid in a `box` A cube,
    displaced by Gaussian jitter.  Atom order: all O, then the H pairs in
    molecule order."""
    rng = np.random.default_rng(seed)
    grid = (np.arange(m) + 0.5) / m * box
    th = math.radians(angle_deg)
    u1 = np.array([math.sin(th / 2), math.cos(th / 2), 0.0]) * bond
    u2 = np.array([-math.sin(th / 2), math.cos(th / 2), 0.0]) * bond
    Os, Hs = [], []
    for x in grid:
        for y in grid:
            for z in grid:
                O = np.array([x, y, z]) + rng.normal(0.0, jitter, 3)
                Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
                Os.append(O)
                Hs += [O + Q @ u1, O + Q @ u2]
    R = np.array(Os + Hs)
    types = np.array([TYPE_O] * len(Os) + [TYPE_H] * len(Hs), dtype=np.int32)
    return WaterSystem(R=R, types=types, box=float(box), seed=seed)


def gapped_params() -> ModelParams:
    """Constants of the gapped variant of the recipe, for T_e = 0 dynamics.

    With the default constants an isolated H2O-like molecule has a gap of
    only ~0.75 eV (hopping t(0.96 A) = 0.44 eV against U = 10 eV), and in any
    box of more than a few molecules the neighbours' Coulomb fields close it,
    so the T_e = 0 SCF has no fixed point and XL-BOMD diverges.  Here the
    O-H hopping is stronger and shorter ranged (t_hop = 20 eV, r_decay =
    0.4 A: 1.8 eV at the bond, 0.17 eV at 1.9 A, 0.02 eV at 2.8 A) and
    U = 6 eV; the isolated molecule's gap is 3.8 eV.  pair_a = 65.75 eV is
    the prefactor at which that molecule's O-H bond force vanishes at
    r_OH = 0.96 A (pair_rho = 0.3 A as in the default recipe)."""
    return dataclasses.replace(ModelParams(), t_hop=20.0, r_decay=0.4, hubbard_u=6.0, pair_a=65.75)


def nonorth_params() -> ModelParams:
    """The gapped recipe with a basis-set overlap: s(r) = 1.1 exp(-r / 0.4 A),
    0.10 at the O-H bond (the hopping there is 1.8 eV), 0.025 between the
    two H of a molecule; S is positive definite with eigenvalues in about
    [0.85, 1.2] for the molecular systems.  The overlap makes the bond
    repel, so pair_a = 24.14 eV is refitted for the isolated molecule's
    O-H bond force to vanish at 0.96 A (its gap is then 2.7 eV)."""
    return dataclasses.replace(gapped_params(), overlap_s0=1.1, overlap_rs=0.4, pair_a=24.14)


def gapped_vapour(n_mol: int = 682, seed: int = 0, morton: bool = False) -> WaterSystem:
    """n_mol H2O-like molecules at 0.1 g/cc (molecular_liquid), the system
    the gapped recipe (gapped_params) keeps gapped at T_e = 0: 682 molecules
    give 2046 atoms (n = 4092 orbitals) in a 58.85 A cube, O atoms ~6.5 A
    apart; 8 molecules give the 24-atom system."""
    return molecular_liquid(n_mol, 0.1, seed=seed, morton=morton)



def isolated_clusters(m: int, spacing: float = 16.0, seed: int = 0) -> WaterSystem:
    """m^3 rigid copies of one 8-molecule cluster (molecular_water(2, 8.0)),
    each under its own random rotation about the cluster's centroid, centred
    on an m x m x m lattice of `spacing` A in a periodic cube of m * spacing.
    Atoms are ordered cluster by cluster (8 O, then 16 H each).  The cluster
    reaches ~4.5 A from its centroid, so at 16 A spacing two clusters are at
    least 7 A apart: beyond a 6 A interaction range every cluster is
    isolated and all clusters have one spectrum."""
    base = molecular_water(2, 8.0, seed=1)
    c0 = base.R - base.R.mean(axis=0)
    rng = np.random.default_rng(seed)
    grid = (np.arange(m) + 0.5) * spacing
    Rs = []
    for x in grid:
        for y in grid:
            for z in grid:
                Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
                Rs.append(c0 @ Q.T + np.array([x, y, z]))
    R = np.concatenate(Rs)
    types = np.tile(base.types, m ** 3)
    return WaterSystem(R=R, types=types, box=float(m * spacing), seed=seed)
