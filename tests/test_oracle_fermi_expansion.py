"""Pins of the oracle's recursive Fermi-operator expansion (density.fermi_expansion)
against what fixes it independently: the Fermi function of the eigenvalues
(LAPACK eigh, density_fermi), the scalar recursion on a diagonal H (the
logistic function itself), the trace condition, and the block-drop rule with
a case where dropping after the start changes the result."""

import numpy as np
import pytest

from oracle import density
from workloads import random_gapped_matrix


@pytest.mark.parametrize("kT", [0.1, 0.5])
@pytest.mark.parametrize("ns", [3, 4])
def test_expansion_is_the_fermi_operator(kT, ns):
    """200 x 200 with a 1 eV gap in a 20 eV spectrum, N_occ = 80.3 (mu in the
    gap's tail): three Newton-Schulz products per inverse leave ||I - AZ|| <=
    99^-4, four 99^-8; the third-order start is exact to 2 z^4 / 15 in z <=
    1/8."""
    H, _ = random_gapped_matrix(200, 80, seed=1)
    r = density.fermi_expansion(H, 80.3, kT, ns_iters=ns)
    ref = density.density_fermi(H, 80.3, kT)
    bound = 3e-9 if ns == 3 else 1e-10
    assert r.converged and r.m >= 8
    assert np.abs(r.D - ref.D).max() < bound
    assert abs(r.mu - ref.mu) < 1e3 * bound
    assert abs(np.trace(r.D) - 80.3) <= 1e-10


def test_diagonal_H_gives_the_logistic_function():
    e = np.linspace(-5.0, 5.0, 11)
    r = density.fermi_expansion(np.diag(e), 5.5, 0.3, ns_iters=4)
    f = 1.0 / (1.0 + np.exp((e - r.mu) / 0.3))
    assert np.abs(np.diag(r.D) - f).max() < 1e-10
    assert np.count_nonzero(r.D - np.diag(np.diag(r.D))) == 0
    assert abs(f.sum() - 5.5) < 1e-10


def test_m_follows_the_bracket():
    """beta (hi - lo) <= 2^(m+1) with hi - lo = Gershgorin width + 80 kT + 2."""
    H, _ = random_gapped_matrix(64, 20, seed=2)
    for kT, m in ((1.0, 8), (0.05, 9), (0.01, 12)):
        lo, hi = density.gershgorin(H)
        w = hi - lo + 80.0 * kT + 2.0
        r = density.fermi_expansion(H, 20.0, kT, mu_iters=1)
        assert r.m == max(8, int(np.ceil(np.log2(w / kT) - 1)))
        assert w / kT <= 2.0 ** (r.m + 1) and (r.m == 8 or w / kT > 2.0 ** r.m)


def test_threshold_drops_after_the_start():
    """Two identical 64-orbital systems coupled by one weak 32 x 32 block c:
    in L = -beta (H - mu I) / 2^(m+2) the coupling block's norm is below tau
    and is dropped, so the thresholded D has no coupling at all, while the
    exact D's coupling block is far above tau (dropping only the result would
    keep it).  Every 32 x 32 block of the thresholded E is either zero or has
    norm >= tau, and tau -> 0 gives the unthresholded expansion."""
    H1, _ = random_gapped_matrix(64, 24, seed=3, width=6.0)
    H = np.zeros((128, 128))
    H[:64, :64] = H1
    H[64:, 64:] = H1
    rng = np.random.default_rng(4)
    c = 5e-5 * rng.standard_normal((32, 32))
    H[:32, 64:96] = c
    H[64:96, :32] = c.T
    kT, tau = 0.3, 1e-5
    exact = density.fermi_expansion(H, 48.0, kT)
    thr = density.fermi_expansion(H, 48.0, kT, tau=tau)
    nrm = density.block_norms(exact.D, 32)
    assert nrm[0, 2] > 10 * tau
    assert np.count_nonzero(thr.D[:64, 64:]) == 0
    E = thr.D - 0.5 * np.eye(128)
    bn = density.block_norms(E, 32)
    assert np.all((bn == 0.0) | (bn >= tau))
    tiny = density.fermi_expansion(H, 48.0, kT, tau=1e-14)
    assert np.abs(tiny.D - exact.D).max() < 1e-12
