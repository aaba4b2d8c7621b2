"""Pins of the oracle's density matrices and SP2 recursion against closed
forms, textbook special cases and invariants."""

import numpy as np
import pytest

from workloads import random_gapped_matrix
from oracle import density


def test_two_level_closed_form():
    """2x2 H: D is the projector on the lower eigenvector,
    D = 1/2 [I - (H - Tr H/2 I) / sqrt(((a-a')/2)^2 + b^2)]."""
    a, ap, b = -1.3, 0.7, 0.45
    H = np.array([[a, b], [b, ap]])
    rad = np.sqrt(((a - ap) / 2) ** 2 + b * b)
    D_ref = 0.5 * (np.eye(2) - (H - 0.5 * (a + ap) * np.eye(2)) / rad)
    assert np.allclose(density.density_T0(H, 1).D, D_ref, atol=1e-14)
    s = density.sp2(H, 1, tol=1e-14)
    assert s.converged
    assert np.allclose(s.X, D_ref, atol=1e-12)


def test_diagonal_H_gives_step_function():
    e = np.array([3.0, -1.0, 0.5, -2.0, 7.0, 0.1])
    H = np.diag(e)
    D = density.density_T0(H, 3).D
    assert np.allclose(D, np.diag([0, 1, 0, 1, 0, 1.0]), atol=1e-15)
    s = density.sp2(H, 3, tol=1e-12)
    assert np.allclose(s.X, np.diag([0, 1, 0, 1, 0, 1.0]), atol=1e-10)


def test_six_site_ring_closed_form():
    """Nearest-neighbour ring, eps_k = -2t cos(2 pi k/6): the three lowest
    states (k = 0, +-1) are occupied (gap 2t) and
    D_ij = 1/6 sum_{k in {0, 1, -1}} cos(2 pi k (i - j)/6)."""
    t = 1.7
    n = 6
    H = np.zeros((n, n))
    for i in range(n):
        H[i, (i + 1) % n] = H[(i + 1) % n, i] = -t
    idx = np.arange(n)
    diff = idx[:, None] - idx[None, :]
    D_ref = sum(np.cos(2 * np.pi * k * diff / n) for k in (0, 1, -1)) / n
    res = density.density_T0(H, 3)
    assert res.gap == pytest.approx(2 * t)
    assert np.allclose(res.D, D_ref, atol=1e-14)
    s = density.sp2(H, 3, tol=1e-13)
    assert np.allclose(s.X, D_ref, atol=1e-11)


@pytest.mark.parametrize("n,nocc,seed", [(40, 13, 0), (128, 70, 1), (257, 100, 2)])
def test_sp2_matches_diagonalisation_and_invariants(n, nocc, seed):
    H, eps = random_gapped_matrix(n, nocc, gap=0.5, width=30.0, seed=seed)
    ref = density.density_T0(H, nocc)
    assert ref.gap == pytest.approx(0.5, rel=1e-8)
    for rule in ("lookahead", "simple"):
        s = density.sp2(H, nocc, tol=1e-11, rule=rule)
        assert s.converged
        assert np.linalg.norm(s.X - ref.D) / np.sqrt(n) < 1e-10
    D = ref.D
    assert np.trace(D) == pytest.approx(nocc, abs=1e-10)
    assert density.idempotency_fro(D) < 1e-12
    assert density.commutator_fro(H, D) < 1e-11


def test_sp2_branches_keep_trace_near_nocc():
    """The look-ahead branch drives Tr X to N_occ: at the end Tr X = N_occ."""
    H, _ = random_gapped_matrix(90, 33, gap=0.2, width=40.0, seed=9)
    s = density.sp2(H, 33, tol=1e-12)
    assert np.trace(s.X) == pytest.approx(33, abs=1e-9)
    assert set(s.branches) == {0, 1}
    # idempotency error decreases monotonically over the last iterations
    h = s.idem_history
    assert all(h[k + 1] < h[k] for k in range(len(h) - 6, len(h) - 1))


def test_gershgorin_bounds_contain_spectrum():
    H, eps = random_gapped_matrix(60, 20, seed=4)
    lo, hi = density.gershgorin(H)
    assert lo <= eps[0] and eps[-1] <= hi


def test_thresholded_sp2_tau_zero_is_dense_and_tau_drops_blocks():
    H, _ = random_gapped_matrix(96, 40, gap=1.0, width=20.0, seed=5)
    dense = density.sp2(H, 40, tol=1e-11)
    t0 = density.sp2(H, 40, tol=1e-11, tau=1e-300, bs=32)
    assert np.allclose(t0.X, dense.X, atol=1e-13)
    # a block-diagonal H with tiny couplings: tau removes the coupling blocks
    A, _ = random_gapped_matrix(32, 10, gap=1.0, seed=6)
    B, _ = random_gapped_matrix(32, 12, gap=1.0, seed=7)
    Hb = np.zeros((64, 64))
    Hb[:32, :32], Hb[32:, 32:] = A, B
    Hb[:32, 32:] = 1e-9
    Hb[32:, :32] = 1e-9
    t = density.sp2(Hb, 22, tol=1e-11, tau=1e-5, bs=32)
    assert np.all(t.X[:32, 32:] == 0.0)
    ref = density.density_T0(Hb, 22).D
    assert np.linalg.norm(t.X - ref) / 8 < 1e-6


def test_fermi_dirac_trace_limit_and_entropy():
    H, eps = random_gapped_matrix(50, 20, gap=1.0, width=10.0, seed=8)
    res = density.density_fermi(H, 20.0, 0.1)
    assert np.trace(res.D) == pytest.approx(20.0, abs=1e-10)
    assert np.allclose(res.D @ H, H @ res.D, atol=1e-10)
    # occupations are the Fermi function of the eigenvalues
    f = 1.0 / (np.exp((eps - res.mu) / 0.1) + 1.0)
    assert np.allclose(res.occ, f, atol=1e-12)
    # T -> 0 reproduces the step function for a gapped spectrum
    cold = density.density_fermi(H, 20.0, 1e-3)
    assert np.allclose(cold.D, density.density_T0(H, 20).D, atol=1e-12)
    # entropy: a half-filled level contributes 2 ln 2, filled/empty nothing
    assert density.entropy_kB(np.array([0.5])) == pytest.approx(2 * np.log(2))
    assert density.entropy_kB(np.array([0.0, 1.0])) == 0.0
