"""Pins of the oracle's charges, forces and integrators: finite differences,
conservation laws, textbook integrator behaviour and the O(dt^2) agreement
with Born-Oppenheimer MD (Sec. IV)."""

import dataclasses

import numpy as np
import pytest

from workloads import (ModelParams, XLParams, TYPE_O, TYPE_H, water_24_atoms,
                       molecular_water, thermal_velocities)
from oracle import tb, density, observables, md

P = ModelParams()
# kappa rescaling for the molecular pin systems: their charge response has
# largest eigenvalue ~4.3, and the K = 5 recursion is stable for
# kappa (1 + lambda) below ~3.6, so kappa0 = 1.82 is rescaled by 0.15.
XL_PIN = dataclasses.replace(XLParams(), kappa_scale=0.15)


def _water_molecule(box=30.0, r=0.96):
    th = np.deg2rad(104.5)
    O = np.array([10.0, 10.0, 10.0])
    R = np.array([O, O + r * np.array([np.sin(th / 2), np.cos(th / 2), 0]),
                  O + r * np.array([-np.sin(th / 2), np.cos(th / 2), 0])])
    return R, np.array([TYPE_O, TYPE_H, TYPE_H], dtype=np.int32), box


def test_mulliken_neutrality():
    """Sum_i q_i = 2 Tr D - N_e = 0 when Tr D = N_occ."""
    s = water_24_atoms()
    h = tb.build_h(s.R, s.types, s.box, P)
    G = tb.build_gamma(s.R, s.box, P)
    H = tb.build_H(h, G, s.types, np.zeros(s.natoms))
    D = density.density_T0(H, int(s.n_occ(P))).D
    q = observables.mulliken(D, s.types, P)
    assert abs(q.sum()) < 1e-10
    # a hand count for one O and one H
    offs = tb.orbital_offsets(s.types)
    assert q[0] == pytest.approx(2 * np.trace(D[offs[0]:offs[1], offs[0]:offs[1]]) - 6.0)
    j = s.natoms - 1
    assert q[j] == pytest.approx(2 * D[offs[j], offs[j]] - 1.0)


@pytest.mark.parametrize("which", ["molecule", "random24"])
def test_forces_are_minus_energy_gradient_at_fixed_n(which):
    """F = -dE/dR at fixed n with D = theta(mu0 - H[n]) recomputed at every
    displaced geometry: central differences of the potential energy."""
    if which == "molecule":
        R, types, box = _water_molecule()
        n_aux = np.array([1.2, -0.5, -0.7])
        nocc = 4
    else:
        s = water_24_atoms()
        R, types, box = s.R, s.types, s.box
        n_aux = 0.3 * np.sin(np.arange(s.natoms))
        n_aux -= n_aux.mean()
        nocc = int(s.n_occ(P))

    def energy(Rx):
        H, G, res, q, pairs = md.electronic_state(Rx, types, box, P, n_aux, nocc)
        return observables.potential_energy(Rx, types, box, P, res.D, q, n_aux, pairs)

    H, G, res, q, pairs = md.electronic_state(R, types, box, P, n_aux, nocc)
    F = observables.forces(R, types, box, P, res.D, q, n_aux, pairs)
    h = 1e-5
    atoms = range(len(types)) if which == "molecule" else [0, 5, 9, 17]
    for a in atoms:
        for k in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[a, k] += h
            Rm[a, k] -= h
            fd = -(energy(Rp) - energy(Rm)) / (2 * h)
            assert F[a, k] == pytest.approx(fd, rel=2e-6, abs=2e-6)
    # no net force (translation invariance)
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-9)


@pytest.mark.parametrize("which,kT", [("molecule", 0.5), ("random24", 0.2)])
def test_finite_temperature_forces_are_minus_free_energy_gradient(which, kT):
    """At T_e > 0 the same force expression, evaluated on the Fermi-Dirac D,
    is -d(U - T_e S)/dR at fixed n: D makes U - T_e S stationary at fixed
    Tr D (Eqs. Etot, Entropy), so its response drops out of the derivative.
    Five-point central differences (h = 2e-4 A: truncation O(h^4), rounding
    ~1e-7 eV/A) of U - T_e S with D and mu recomputed at every displaced
    geometry; U alone differs by the entropy term's gradient."""
    if which == "molecule":
        R, types, box = _water_molecule()
        n_aux = np.array([1.2, -0.5, -0.7])
        nocc = 4.0
    else:
        s = water_24_atoms()
        R, types, box = s.R, s.types, s.box
        n_aux = 0.3 * np.sin(np.arange(s.natoms))
        n_aux -= n_aux.mean()
        nocc = s.n_occ(P)

    def energies(Rx):
        H, G, res, q, pairs = md.electronic_state(Rx, types, box, P, n_aux, nocc, kT=kT)
        U = observables.potential_energy(Rx, types, box, P, res.D, q, n_aux, pairs)
        return U, kT * density.entropy_kB(np.linalg.eigvalsh(res.D))

    H, G, res, q, pairs = md.electronic_state(R, types, box, P, n_aux, nocc, kT=kT)
    F = observables.forces(R, types, box, P, res.D, q, n_aux, pairs)
    h = 2e-4
    atoms = range(len(types)) if which == "molecule" else [0, 5, 9, 17]
    worst_u = 0.0
    for a in atoms:
        for k in range(3):
            U, TS = {}, {}
            for j in (-2, -1, 1, 2):
                Rx = R.copy()
                Rx[a, k] += j * h
                U[j], TS[j] = energies(Rx)

            def d5(f):
                return (-f[2] + 8.0 * f[1] - 8.0 * f[-1] + f[-2]) / (12.0 * h)

            fd = -(d5(U) - d5(TS))
            assert F[a, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
            worst_u = max(worst_u, abs(F[a, k] + d5(U)))
    assert worst_u > 0.1  # the entropy term's gradient (0.45 and 4 eV/A here) is not negligible


def test_energy_at_scf_is_the_scc_tb_energy():
    """At n = q: E = 2 Tr[hD] + 1/2 q^T gamma q (+ E_pair)."""
    R, types, box = _water_molecule()
    q, fr, it = md.scf(R, types, box, P, 4)
    assert it > 0
    h = tb.build_h(R, types, box, P)
    G = tb.build_gamma(R, box, P)
    E = observables.potential_energy(R, types, box, P, fr.D, q, q)
    assert E == pytest.approx(2 * np.sum(h * fr.D) + 0.5 * q @ G @ q + tb.pair_energy(R, box, P))


def test_velocity_verlet_harmonic_energy_error_is_second_order():
    """Velocity Verlet on a harmonic oscillator: the energy error is O(dt^2)."""
    k, m = 3.0, 2.0
    conv = 9.648533e-3

    def run(dt, T=40.0):
        x, v = np.array([[1.0, 0, 0]]), np.zeros((1, 3))
        F = -k * x
        E0 = 0.5 * k * 1.0
        err = 0.0
        for _ in range(int(round(T / dt))):
            v = md.velocity_verlet_kick(v, F, np.array([m]), dt)
            x = x + dt * v
            F = -k * x
            v = md.velocity_verlet_kick(v, F, np.array([m]), dt)
            E = 0.5 * k * float(np.sum(x * x)) + 0.5 * m * float(np.sum(v * v)) / conv
            err = max(err, abs(E - E0))
        return err

    e1, e2 = run(0.4), run(0.2)
    assert e1 / e2 == pytest.approx(4.0, rel=0.1)


def test_modified_verlet_fixed_point_and_decay():
    """sum c_k = 0, so a constant history n = q is a fixed point of Eq. Verl_n;
    a perturbation decays for kappa_eff below the K = 5 stability limit."""
    xl = XLParams()
    assert sum(xl.c) == 0.0
    q = np.array([0.3, -0.1, -0.2])
    hist = [q.copy() for _ in range(xl.K + 1)]
    assert np.allclose(md.modified_verlet_n(hist, q, xl), q, atol=1e-15)
    for kappa_eff in (0.5, 1.82, 3.0):
        x = dataclasses.replace(xl, kappa_scale=kappa_eff / xl.kappa0)
        hist = [np.array([1.0])] + [np.zeros(1) for _ in range(xl.K)]
        for _ in range(4000):
            hist = [md.modified_verlet_n(hist, np.zeros(1), x)] + hist[:-1]
        assert abs(hist[0][0]) < 1e-3
    x = dataclasses.replace(xl, kappa_scale=4.2 / xl.kappa0)
    hist = [np.array([1.0])] + [np.zeros(1) for _ in range(xl.K)]
    for _ in range(200):
        hist = [md.modified_verlet_n(hist, np.zeros(1), x)] + hist[:-1]
    assert abs(hist[0][0]) > 1e3


def test_xlbomd_conserves_energy_and_tracks_charges():
    """Fast-QMMD on a molecular pin system: E_tot fluctuates at the meV level
    without drift and n follows q (Fig. 2 idea)."""
    s = molecular_water(1, 12.0, seed=0)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100)
    tr = md.xlbomd(s.R, s.types, s.box, P, XL_PIN, v0, M, s.n_occ(P), 120)
    E = np.array(tr.E_tot)
    sigma, drift = md.energy_drift(E, XL_PIN.dt, s.natoms)
    assert np.max(np.abs(E - E[0])) < 5e-3
    assert abs(drift) < 0.05
    assert max(np.max(np.abs(a - b)) for a, b in zip(tr.n, tr.q)) < 0.05
    # the kinetic energy really changes (the molecule vibrates)
    assert np.ptp(tr.KE) > 10 * np.max(np.abs(E - E[0]))


def test_xlbomd_deviation_from_bomd_is_second_order_in_dt():
    """Sec. IV: charges and forces of Fast-QMMD deviate from BOMD as O(dt^2)."""
    s = molecular_water(1, 12.0, seed=0)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100)
    T = 8.0
    dev = []
    for dt in (0.2, 0.1):
        xl = dataclasses.replace(XL_PIN, dt=dt)
        nst = int(round(T / dt))
        a = md.xlbomd(s.R, s.types, s.box, P, xl, v0, M, s.n_occ(P), nst)
        b = md.bomd(s.R, s.types, s.box, P, dt, v0, M, s.n_occ(P), nst)
        dq = np.sqrt(np.mean([np.mean((x - y) ** 2) for x, y in zip(a.q, b.q)]))
        dev.append(dq)
    assert dev[0] / dev[1] == pytest.approx(4.0, rel=0.3)


def test_xlbomd_finite_temperature_entropy_term_restores_conservation():
    """Eqs. Etot, Entropy: at T_e > 0, KE + U alone is not conserved, while
    KE + U - T_e S (S from the occupation numbers, the eigenvalues of D) is.
    kT = 1.5 eV puts fractional occupations across the 1.75 eV gap of the
    molecule, so the entropy term is large and changes along the path."""
    s = molecular_water(1, 12.0, seed=0)
    M = s.masses(P)
    v0 = thermal_velocities(M, 600.0, seed=101)
    tr = md.xlbomd(s.R, s.types, s.box, P, XL_PIN, v0, M, s.n_occ(P), 80, kT=1.5)
    E = np.array(tr.E_tot)
    TS = np.array(tr.TS)
    E_no_S = E + TS
    assert np.min(TS) > 0.01
    assert np.max(np.abs(E - E[0])) < 0.05 * np.max(np.abs(E_no_S - E_no_S[0]))
    # the charges still follow q at T_e > 0
    assert max(np.max(np.abs(a - b)) for a, b in zip(tr.n, tr.q)) < 0.05


def test_energy_drift_measures_on_known_series():
    """Table II's two measures on series with a known answer: sigma is the
    standard deviation of E_tot about its mean (eV), drift the least-squares
    slope per atom in eV/atom/ps (time step in fs)."""
    from oracle.md import energy_drift
    N, dt, natoms = 401, 0.25, 10
    k = np.arange(N)
    # a pure line rising 1e-3 eV per step: slope 1e-3 eV / 0.25 fs = 4 eV/ps,
    # 0.4 eV/atom/ps; sigma of an evenly spaced line = step * sqrt((N^2 - 1)/12)
    sigma, drift = energy_drift(list(-12.5 + 1e-3 * k), dt, natoms)
    assert drift == pytest.approx(0.4, rel=1e-10)
    assert sigma == pytest.approx(1e-3 * np.sqrt((N * N - 1) / 12.0), rel=1e-10)
    # a palindromic fluctuation (E_k = E_{N-1-k}) has no slope; alternating
    # +-eps about the mean gives sigma = eps
    eps = 3e-6
    E = np.where((k % 4 == 0) | (k % 4 == 3), eps, -eps)[:400]
    sigma, drift = energy_drift(list(5.0 + E), dt, natoms)
    assert sigma == pytest.approx(eps, rel=1e-9)
    assert abs(drift) < 1e-12
    # both together: the slope is unchanged by the palindromic part
    sigma, drift = energy_drift(list(5.0 + E + 2e-4 * k[:400]), dt, natoms)
    assert drift == pytest.approx(2e-4 / 0.25e-3 / natoms, rel=1e-9)


def test_gapped_recipe_molecule_at_rest_and_gapped():
    """The gapped variant's constants (workloads.gapped_params) do what their
    docstring states: the isolated molecule's O-H bond force vanishes at
    r_OH = 0.96 A, it is stretched back from 1.0 A and pushed out from 0.92 A,
    and its SCF gap is ~3.8 eV."""
    from workloads import gapped_params
    G = gapped_params()
    fb = {}
    for r in (0.92, 0.96, 1.0):
        R, types, box = _water_molecule(r=r)
        q, fr, it = md.scf(R, types, box, G, 4.0, tol=1e-12)
        F = observables.forces(R, types, box, G, fr.D, q, fr.n_aux)
        u = (R[1] - R[0]) / np.linalg.norm(R[1] - R[0])
        fb[r] = float(F[1] @ u)
        if r == 0.96:
            assert fr.gap == pytest.approx(3.82, abs=0.02)
    assert abs(fb[0.96]) < 1e-3
    assert fb[0.92] > 0.3 and fb[1.0] < -0.3


def test_gapped_vapour_converges_and_conserves_energy_at_half_kappa0():
    """8 H2O-like molecules of the gapped recipe at 0.1 g/cc (24 atoms): the
    T_e = 0 SCF converges to 1e-10 e in a few tens of iterations, the gap stays
    open along 200 steps of 0.25 fs at the paper's kappa = kappa0 / 2, and
    E_tot fluctuates at the meV level without drift."""
    from workloads import gapped_params, gapped_vapour
    G = gapped_params()
    s = gapped_vapour(8)
    assert s.natoms == 24
    q, fr, it = md.scf(s.R, s.types, s.box, G, s.n_occ(G), tol=1e-10)
    assert 0 <= it < 60 and fr.gap > 2.0
    M = s.masses(G)
    v0 = thermal_velocities(M, 300.0, seed=100)
    tr = md.xlbomd(s.R, s.types, s.box, G, XLParams(), v0, M, s.n_occ(G), 200)
    sigma, drift = md.energy_drift(tr.E_tot, XLParams().dt, s.natoms)
    assert min(tr.gap) > 1.0
    assert sigma < 5e-3 and abs(drift) < 0.05
    assert max(np.max(np.abs(a - b)) for a, b in zip(tr.n, tr.q)) < 0.02


def test_isolated_clusters_geometry():
    """The isolated-cluster workload's claims: rigid copies (every cluster has
    the base cluster's interatomic distances), clusters more than 6 A (the
    model's interaction range) apart under the periodic images, and, for the
    oracle's h, no element between two clusters."""
    from workloads import isolated_clusters, gapped_params
    from oracle import tb
    s = isolated_clusters(3)
    nc, na = 27, 24
    C = s.R.reshape(nc, na, 3)
    d0 = np.linalg.norm(C[0][:, None] - C[0][None], axis=2)
    for c in range(1, nc):
        assert np.abs(np.linalg.norm(C[c][:, None] - C[c][None], axis=2) - d0).max() < 1e-12
    d = s.R[:, None, :] - s.R[None, :, :]
    d -= s.box * np.round(d / s.box)
    dist = np.linalg.norm(d, axis=2)
    cl = np.repeat(np.arange(nc), na)
    assert dist[cl[:, None] != cl[None, :]].min() > 6.0
    h = tb.build_h(s.R, s.types, s.box, gapped_params())
    oc = np.repeat(np.arange(nc), 48)
    assert np.count_nonzero(h[oc[:, None] != oc[None, :]]) == 0
