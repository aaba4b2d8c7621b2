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


# ---------------------------------------------------------------- drop rule
# Sec. III.B thresholds the iterate after each projection; the block-sparse
# reading drops every 32 x 32 block whose Frobenius norm is below tau, after
# X0 and after every projection.  The pins below separate that rule from its
# near neighbours: an element-max rule (drop a block when max |x| < tau), an
# element-wise rule (zero single elements below tau), a sum-of-|x| norm, a
# strict/non-strict comparison at tau, and a recursion that does not drop
# after X0.

def test_block_rule_is_the_frobenius_norm_of_the_block():
    tau = 1e-5
    bs = 32
    X = np.zeros((2 * bs, 2 * bs))
    # every element below tau, Frobenius norm 3.2 tau: kept whole
    X[:bs, bs:] = 0.1 * tau
    # one element 2 tau, the others 1e-3 tau: kept with its small elements
    X[bs:, :bs] = 1e-3 * tau
    X[bs + 3, 5] = 2.0 * tau
    # uniform blocks of norm 0.99 tau (dropped) and 1.01 tau (kept); their
    # sum of |x| (32 x 32 elements of 0.99 tau / 32) is about 32 tau
    X[:bs, :bs] = 0.99 * tau / bs
    X[bs:, bs:] = 1.01 * tau / bs
    Y, norms = density._drop_blocks(X, bs, tau)
    assert norms[0, 1] == pytest.approx(3.2 * tau, rel=1e-12)
    assert np.array_equal(Y[:bs, bs:], X[:bs, bs:])
    assert np.array_equal(Y[bs:, :bs], X[bs:, :bs])
    assert np.all(Y[:bs, :bs] == 0.0)
    assert np.array_equal(Y[bs:, bs:], X[bs:, bs:])
    # exactly tau is kept (drop only below tau)
    Z = np.zeros((bs, bs))
    Z[0, 0] = tau
    assert np.array_equal(density._drop_blocks(Z, bs, tau)[0], Z)


def test_block_rule_on_a_ragged_edge():
    """n = 40 with 32 x 32 blocks: the edge blocks are 32 x 8, 8 x 32, 8 x 8 and
    their norms are taken over the elements they hold."""
    tau = 1e-5
    X = np.zeros((40, 40))
    X[32:, 32:] = 0.2 * tau          # 8 x 8 of 0.2 tau: norm 1.6 tau, kept
    X[:32, 32:] = 0.01 * tau         # 32 x 8 of 0.01 tau: norm 0.16 tau, dropped
    X[32:, :32] = 0.01 * tau
    Y, norms = density._drop_blocks(X, 32, tau)
    assert norms.shape == (2, 2)
    assert norms[1, 1] == pytest.approx(1.6 * tau, rel=1e-12)
    assert np.array_equal(Y[32:, 32:], X[32:, 32:])
    assert np.all(Y[:32, 32:] == 0.0) and np.all(Y[32:, :32] == 0.0)


def test_threshold_is_applied_to_X0():
    """Two 64-orbital blocks coupled between the highest occupied state of one
    and the lowest empty state of the other (N_occ = 40), every coupling block
    of X0 below tau (largest 0.9 tau): dropped at X0, the coupling stays exactly
    zero.  The first projection (X^2) raises that coupling above tau (both
    states lie below the middle of the Gershgorin interval), so a recursion
    that only drops after projections keeps it and returns a coupled D."""
    tau, bs, nocc = 1e-5, 32, 40
    rng = np.random.default_rng(3)
    Qa = np.linalg.qr(rng.normal(size=(64, 64)))[0]
    Qb = np.linalg.qr(rng.normal(size=(64, 64)))[0]
    ea = np.sort(np.concatenate([rng.uniform(-2, -0.4, 32), rng.uniform(0.4, 2, 32)]))
    eb = np.sort(np.concatenate([rng.uniform(-2, -0.4, 32), rng.uniform(0.4, 2, 32)]))
    A, B = Qa @ np.diag(ea) @ Qa.T, Qb @ np.diag(eb) @ Qb.T
    levels = np.sort(np.concatenate([ea, eb]))
    mu = 0.5 * (levels[nocc - 1] + levels[nocc])
    ia, ib = np.nonzero(ea < mu)[0][-1], np.nonzero(eb > mu)[0][0]
    C = np.outer(Qa[:, ia], Qb[:, ib])

    def x0(scale):
        H = np.zeros((128, 128))
        H[:64, :64], H[64:, 64:] = A, B
        H[:64, 64:] = scale * C
        H[64:, :64] = H[:64, 64:].T
        lo, hi = density.gershgorin(H)
        return H, (hi * np.eye(128) - H) / (hi - lo)

    scale = 1.0
    for _ in range(4):  # the Gershgorin width moves with the coupling
        H, X0 = x0(scale)
        scale *= 0.9 * tau / density.block_norms(X0, bs)[:2, 2:].max()
    H, X0 = x0(scale)
    assert density.block_norms(X0, bs)[:2, 2:].max() == pytest.approx(0.9 * tau, rel=1e-6)
    s = density.sp2(H, nocc, tol=1e-10, tau=tau, bs=bs)
    assert s.converged
    assert np.all(s.X[:64, 64:] == 0.0)
    # negative control: the same recursion without the drop at X0
    X = X0
    assert density.block_norms(X0 @ X0, bs)[:2, 2:].max() > tau  # the first projection is X^2
    for _ in range(100):
        t1, t2 = np.trace(X), np.sum(X * X)
        if t1 - t2 <= 1e-10:
            break
        X2 = X @ X
        X = X2 if abs(t2 - nocc) <= abs(2 * t1 - t2 - nocc) else 2 * X - X2
        X = density._drop_blocks(X, bs, tau)[0]
    assert np.abs(X[:64, 64:]).max() > 1e-6
