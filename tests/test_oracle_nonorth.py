"""Pins of the non-orthogonal oracle (App. D.1) against what fixes it
independently: the orthogonal model at S = I, the closed form of a
two-orbital bond with overlap, the generalized symmetric eigenproblem
H c = e S c (LAPACK), the independence of rho from the choice of Z,
generalized idempotency and charge neutrality, central differences of the
energy for the forces (T_e = 0 and the free energy at T_e > 0), and energy
conservation of the XL-BOMD trajectory."""

import dataclasses

import numpy as np
import pytest
import scipy.linalg

from workloads import (ModelParams, XLParams, TYPE_H, molecular_water, nonorth_params, thermal_velocities)
from oracle import density, md, nonorth, observables, tb

PN = nonorth_params()


def _system(seed=1):
    return molecular_water(2, 8.0, seed=seed)


def _state(s, p, n_aux, kT=0.0):
    return nonorth.electronic_state(s.R, s.types, s.box, p, n_aux, s.n_occ(p), kT)


def test_zero_overlap_is_the_orthogonal_model():
    s = _system()
    P0 = dataclasses.replace(PN, overlap_s0=0.0)
    rng = np.random.default_rng(0)
    n = rng.normal(0, 0.2, s.natoms)
    n -= n.mean()
    h, S, G, H, st, q = _state(s, P0, n)
    assert np.array_equal(S, np.eye(S.shape[0]))
    Ho = tb.build_H(h, G, s.types, n)
    assert np.abs(H - Ho).max() < 1e-13
    D = density.density_T0(Ho, int(s.n_occ(P0))).D
    assert np.abs(st.rho - D).max() < 1e-12
    Fo = observables.forces(s.R, s.types, s.box, P0, D, observables.mulliken(D, s.types, P0), n)
    F = nonorth.forces(s.R, s.types, s.box, P0, st.rho, st.W, q, n)
    assert np.abs(F - Fo).max() < 1e-10


def test_two_orbital_bond_closed_form():
    """Two H atoms r apart (one s orbital each, two electrons):
    H = [[e, -V], [-V, e]], S = [[1, s], [s, 1]] with V, s the hopping and
    overlap radials; the bonding state (e - V)/(1 + s) is doubly occupied,
    rho = [[1, 1], [1, 1]] / (2 (1 + s)), both Mulliken charges are 0 and
    2 Tr[h rho] = 2 (e - V)/(1 + s)."""
    r = 0.9
    R = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    types = np.array([TYPE_H, TYPE_H], dtype=np.int32)
    box = 30.0
    V, _ = tb.hopping_radial(PN)(r)
    sv, _ = nonorth.overlap_radial(PN)(r)
    e = PN.eps_s_H
    h = tb.build_h(R, types, box, PN)
    S = nonorth.build_S(R, types, box, PN)
    assert h[0, 1] == pytest.approx(-V, rel=1e-14) and S[0, 1] == pytest.approx(sv, rel=1e-14)
    st = nonorth.density_matrix(h, S, 1.0)
    assert np.abs(st.rho - np.full((2, 2), 1.0 / (2.0 * (1.0 + sv)))).max() < 1e-14
    assert st.eps[0] == pytest.approx((e - V) / (1.0 + sv), rel=1e-13)
    q = nonorth.mulliken(st.rho, S, types, PN)
    assert np.abs(q).max() < 1e-13
    assert 2.0 * np.sum(h * st.rho) == pytest.approx(2.0 * (e - V) / (1.0 + sv), rel=1e-13)


@pytest.mark.parametrize("kT", [0.0, 0.2])
def test_density_matrix_is_the_generalized_eigenproblem_and_independent_of_Z(kT):
    s = _system(2)
    rng = np.random.default_rng(3)
    n = rng.normal(0, 0.3, s.natoms)
    n -= n.mean()
    h, S, G, H, st, q = _state(s, PN, n, kT)
    e, C = scipy.linalg.eigh(H, S)
    nocc = s.n_occ(PN)
    if kT == 0.0:
        Cocc = C[:, :int(nocc)]
        rho_ref = Cocc @ Cocc.T
        W_ref = (Cocc * e[:int(nocc)]) @ Cocc.T
    else:
        f = density.fermi_occupations(e, st.mu, kT)
        rho_ref = (C * f) @ C.T
        W_ref = (C * (f * e)) @ C.T
    assert np.abs(st.rho - rho_ref).max() < 1e-11
    assert np.abs(st.W - W_ref).max() < 1e-10
    ch = nonorth.density_matrix(H, S, nocc, kT, kind="cholesky")
    assert np.abs(ch.rho - st.rho).max() < 1e-11
    Z = st.Z
    assert np.abs(Z.T @ S @ Z - np.eye(S.shape[0])).max() < 1e-12
    # generalized idempotency (T_e = 0), trace and neutrality
    if kT == 0.0:
        assert np.abs(st.rho @ S @ st.rho - st.rho).max() < 1e-11
        assert np.abs(st.W - st.rho @ H @ st.rho).max() < 1e-10
    assert np.trace(st.rho @ S) == pytest.approx(nocc, abs=1e-10)
    assert abs(q.sum()) < 1e-10


@pytest.mark.parametrize("kT", [0.0, 0.2])
def test_forces_are_minus_the_energy_gradient_at_fixed_n(kT):
    """Central differences of E_pot (T_e = 0) or E_pot - T_e S_e (T_e > 0) at
    fixed n, every coordinate of a 12-atom box, step 1e-5 A: the analytic
    force (band, overlap, gamma and pair terms) agrees to 1e-6 relative."""
    s = molecular_water(2, 8.0, seed=4)
    keep = np.r_[0:4, 8:16]        # 4 molecules: their O atoms and H pairs
    R, types = s.R[keep], s.types[keep]
    rng = np.random.default_rng(5)
    n = rng.normal(0, 0.2, len(types))
    n -= n.mean()
    nocc = (6.0 * 4 + 8) / 2
    _, S, _, _, st, q = nonorth.electronic_state(R, types, s.box, PN, n, nocc, kT)
    F = nonorth.forces(R, types, s.box, PN, st.rho, st.W, q, n)
    h = 1e-5
    Ffd = np.zeros_like(R)
    for a in range(R.shape[0]):
        for k in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[a, k] += h
            Rm[a, k] -= h
            Ffd[a, k] = -(nonorth.potential_energy(Rp, types, s.box, PN, n, nocc, kT)
                          - nonorth.potential_energy(Rm, types, s.box, PN, n, nocc, kT)) / (2 * h)
    scale = np.abs(F).max()
    assert np.abs(F - Ffd).max() < 1e-6 * scale
    # the overlap terms matter: without them the force is off
    Fo = observables.forces(R, types, s.box, PN, st.rho, q, n)
    assert np.abs(Fo - Ffd).max() > 1e-2 * scale


def test_xlbomd_conserves_energy_with_overlap():
    """Fast-QMMD in the non-orthogonal formulation on 8 H2O-like molecules
    (24 atoms): E_tot fluctuates at the meV level without drift over 100
    steps of 0.25 fs at kappa0 / 2, and n follows q."""
    s = _system(1)
    M = s.masses(PN)
    v0 = thermal_velocities(M, 300.0, seed=100)
    tr = nonorth.xlbomd(s.R, s.types, s.box, PN, XLParams(), v0, M, s.n_occ(PN), 100)
    E = np.array(tr.E_tot)
    sigma, drift = md.energy_drift(E, XLParams().dt, s.natoms)
    assert sigma < 1e-2 and abs(drift) < 0.05
    assert max(np.max(np.abs(a - b)) for a, b in zip(tr.n, tr.q)) < 0.05
    assert np.ptp(tr.KE) > 10 * sigma
