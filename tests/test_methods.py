"""Pins of the numerical methods the GPU path uses where the paper gives no
recipe, checked in FP64 NumPy against exact definitions (no GPU):

* the recursive Fermi-operator expansion in deviation form against the
  Fermi function: m = 14 doublings from the linearised start, m = 10 and 8
  from the third-order start E0 = L - 4/3 L^3 (with a linearised m = 8 control);
* the second-order canonical shift of a Fermi density matrix and its
  remainder bound |u|^3/6 Tr[D(I - D)];
* the quadratic minimax start of the Newton-Schulz inverse of I + 4E^2 and
  the residual after two steps;
* the balanced base-128 digit split of the emulated-FP64 refinement: digit
  ranges, exact reconstruction, the sum of the 22 kept slice-pair products
  against the FP64 product, and the diagonal bias the kept pair (4, 4) removes.
"""

import numpy as np
import pytest

from oracle import density


def _random_h(n, seed, width=20.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    eps = np.sort(rng.uniform(-width / 2, width / 2, n))
    return (Q * eps) @ Q.T, eps, Q


def _fermi_matrix(eps, Q, mu, kT):
    f = density.fermi_occupations(eps, mu, kT)
    return (Q * f) @ Q.T


@pytest.mark.parametrize("kT", [0.1, 0.5])
def test_recursive_fermi_expansion_deviation_form(kT):
    """E0 = -beta/2^(m+2) (H - mu I); m times E <- 2E (I + 4E^2)^-1; D = I/2 + E
    equals the Fermi function at beta to 1e-8 with m = 14 (Eq. EL_4c)."""
    n, m = 60, 14
    H, eps, Q = _random_h(n, seed=1)
    mu = 0.3
    beta = 1.0 / kT
    E = -beta / 2.0 ** (m + 2) * (H - mu * np.eye(n))
    for _ in range(m):
        E = 2.0 * E @ np.linalg.inv(np.eye(n) + 4.0 * E @ E)
        E = 0.5 * (E + E.T)
    D = 0.5 * np.eye(n) + E
    ref = _fermi_matrix(eps, Q, mu, kT)
    assert np.abs(D - ref).max() < 1e-8
    # with two doublings the linearised start is visible: the check can fail
    E = -beta / 2.0 ** (2 + 2) * (H - mu * np.eye(n))
    for _ in range(2):
        E = 2.0 * E @ np.linalg.inv(np.eye(n) + 4.0 * E @ E)
    assert np.abs(0.5 * np.eye(n) + E - ref).max() > 1e-3


def _start3(H, mu, beta, m):
    """E0 = L - 4/3 L^3, L = -beta/2^(m+2) (H - mu I): -tanh(Z)/2 to third order."""
    L = -beta / 2.0 ** (m + 2) * (H - mu * np.eye(H.shape[0]))
    return L - 4.0 / 3.0 * L @ L @ L


@pytest.mark.parametrize("kT", [0.1, 0.5])
def test_fermi_expansion_third_order_start(kT):
    """From E0 = L - 4/3 L^3, m doublings give the Fermi function to ~1e-14
    at m = 10 and ~1e-11 at m = 8 (start error 2 z^4/15, not amplified by the
    doublings); the linearised start E0 = L misses by > 1e-7 at m = 8."""
    n = 60
    H, eps, Q = _random_h(n, seed=1)
    mu, beta = 0.3, 1.0 / kT
    ref = _fermi_matrix(eps, Q, mu, kT)
    I = np.eye(n)

    def expand(E, m):
        for _ in range(m):
            E = 2.0 * E @ np.linalg.inv(I + 4.0 * E @ E)
        return np.abs(0.5 * I + E - ref).max()

    assert expand(_start3(H, mu, beta, 10), 10) < 1e-12
    assert expand(_start3(H, mu, beta, 8), 8) < 1e-10
    assert expand(-beta / 2.0 ** 10 * (H - mu * I), 8) > 1e-7


def _z1(A):
    """Quadratic start Z1 = (210 I - 144 A + 32 A^2) / 99 for A with spectrum in [1, 2]."""
    n = A.shape[0]
    return (210.0 * np.eye(n) - 144.0 * A + 32.0 * A @ A) / 99.0


def test_newton_schulz_quadratic_start():
    """1 - x p(x) = T3(2x - 3) / T3(-3) on [1, 2]: |I - A Z1| <= 1/99, reached at the
    four Chebyshev extremal points x = 1, 1.25, 1.75, 2; two Newton-Schulz steps
    Z <- Z (2I - A Z) square the residual twice (99^-4); the linear start
    4/3 I - 4/9 A only reaches 1/9."""
    x = np.array([1.0, 1.25, 1.75, 2.0])
    assert np.allclose(np.abs(1.0 - x * np.diag(_z1(np.diag(x)))), 1.0 / 99.0, rtol=1e-12)
    rng = np.random.default_rng(6)
    n = 50
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([x, rng.uniform(1.0, 2.0, n - 4)])
    A = (Q * lam) @ Q.T
    I = np.eye(n)
    Z = _z1(A)
    assert np.linalg.norm(I - A @ Z, 2) <= 1.0 / 99.0 * (1 + 1e-9)
    assert np.linalg.norm(I - A @ Z, 2) >= 1.0 / 99.0 * (1 - 1e-6)
    for _ in range(2):
        Z = Z @ (2.0 * I - A @ Z)
    assert np.linalg.norm(I - A @ Z, 2) <= 99.0 ** -4 * (1 + 1e-6) + 1e-14
    Zl = 4.0 / 3.0 * I - 4.0 / 9.0 * A
    assert np.linalg.norm(I - A @ Zl, 2) == pytest.approx(1.0 / 9.0, rel=1e-9)


def test_fermi_expansion_with_newton_schulz_inverse():
    """The expansion from the third-order start with the inverse replaced by Z1
    and two Newton-Schulz steps (the products the tensor-core path forms, m = 10)
    still equals the Fermi function to 1e-8."""
    n, m, kT = 60, 10, 0.1
    H, eps, Q = _random_h(n, seed=7)
    mu = 0.1
    I = np.eye(n)
    E = _start3(H, mu, 1.0 / kT, m)
    for _ in range(m):
        A = I + 4.0 * E @ E
        Z = _z1(A)
        for _ in range(2):
            Z = Z @ (2.0 * I - A @ Z)
        E = 2.0 * E @ Z
    assert np.abs(0.5 * I + E - _fermi_matrix(eps, Q, mu, kT)).max() < 1e-8


@pytest.mark.parametrize("u", [1e-3, 1e-2, 5e-2])
def test_second_order_canonical_shift_and_its_bound(u):
    """D(mu + dmu) = D + u D(I-D) + u^2/2 D(I-D)(I-2D) + R, u = beta dmu, with
    ||R||_F <= |u|^3/6 Tr[D(I - D)]; the first-order form alone misses by O(u^2)."""
    n, kT = 80, 0.1
    H, eps, Q = _random_h(n, seed=2)
    mu = float(np.median(eps))
    beta = 1.0 / kT
    D = _fermi_matrix(eps, Q, mu, kT)
    D_true = _fermi_matrix(eps, Q, mu + u / beta, kT)
    E = D - 0.5 * np.eye(n)
    P1 = 0.25 * np.eye(n) - E @ E          # D(I - D)
    P2 = 2.0 * E @ E @ E - 0.5 * E         # D(I - D)(I - 2D)
    assert np.abs(P1 - D @ (np.eye(n) - D)).max() < 1e-12
    assert np.abs(P2 - D @ (np.eye(n) - D) @ (np.eye(n) - 2 * D)).max() < 1e-12
    D2 = D + u * P1 + 0.5 * u * u * P2
    R = np.linalg.norm(D_true - D2)
    bound = abs(u) ** 3 / 6.0 * np.trace(P1)
    assert R <= bound
    R1 = np.linalg.norm(D_true - (D + u * P1))
    assert R1 > 10 * R


def test_canonical_shift_solves_the_trace_condition():
    """u from dev + t1 u + t2 u^2 / 2 = 0 (Newton from -dev/t1) brings Tr D to
    N_occ to third order."""
    n, kT = 80, 0.1
    H, eps, Q = _random_h(n, seed=3)
    beta = 1.0 / kT
    nocc = 40.3
    mu_exact = density.density_fermi(H, nocc, kT).mu
    mu = mu_exact + 0.002  # a warm start off by 2 meV
    D = _fermi_matrix(eps, Q, mu, kT)
    E = D - 0.5 * np.eye(n)
    dev = np.trace(D) - nocc
    t1 = 0.25 * n - np.sum(E * E)
    t2 = 2.0 * np.trace(E @ E @ E) - 0.5 * np.trace(E)
    u = -dev / t1
    for _ in range(3):
        u -= (dev + u * (t1 + 0.5 * t2 * u)) / (t1 + t2 * u)
    D2 = D + u * (0.25 * np.eye(n) - E @ E) + 0.5 * u * u * (2 * E @ E @ E - 0.5 * E)
    assert abs(np.trace(D2) - nocc) < 1e-9
    assert abs(mu + u / beta - mu_exact) < 1e-7
    assert np.linalg.norm(D2 - _fermi_matrix(eps, Q, mu_exact, kT)) < abs(u) ** 3 / 6 * t1 + 1e-12


def _digits(r):
    """Balanced base-128 digits (6 of them) of rint(r 2^42), |r| < 1/2."""
    R = np.rint(r * 2.0 ** 42).astype(np.int64)
    d = np.zeros((6,) + R.shape, dtype=np.int64)
    for s in range(5, 0, -1):
        low = ((R + 64) & 127) - 64
        d[s] = low
        R = (R - low) >> 7
    d[0] = R
    return d


# (s, t), 0-based: s + t <= 5 (21 pairs), then the diagonal pair (3, 3)
_PAIRS = [(s, t) for s in range(6) for t in range(6) if s + t <= 5] + [(3, 3)]


def test_balanced_digit_split_is_exact_and_bounded():
    rng = np.random.default_rng(4)
    r = rng.uniform(-0.5, 0.5, 20000) * (1 - 1e-12)
    r[:4] = [0.0, 0.5 - 2.0 ** -50, -(0.5 - 2.0 ** -50), 2.0 ** -43]
    d = _digits(r)
    assert np.abs(d).max() <= 64 and d[1:].min() >= -64 and d[1:].max() <= 63
    rec = sum(d[s].astype(np.float64) * 2.0 ** (-7 * (s + 1)) for s in range(6))
    assert np.array_equal(rec, np.rint(r * 2.0 ** 42) / 2.0 ** 42)
    assert np.abs(rec - r).max() <= 2.0 ** -43
    # every digit is an integer exactly representable in bf16 (8 significant bits)
    assert np.abs(d).max() <= 256
    assert len(_PAIRS) == 22


def _row_scaled(X):
    """x = 2^e r with |r| < 1/2 per row (e = frexp exponent of the row maximum + 1)."""
    e = np.array([np.frexp(np.abs(row).max())[1] + 1 for row in X])
    return X / 2.0 ** e[:, None], e


def test_slice_pair_product_matches_fp64():
    """sum over the 22 kept pairs of 2^(-7(s+t)) P_st (P_st exact integer
    products) equals the FP64 product of the row-scaled matrices to ~2^-44 of
    the row scales; the integer products stay within 2^24 (exact in an FP32
    accumulator) for K <= 4096."""
    rng = np.random.default_rng(5)
    n = 96
    X = rng.standard_normal((n, n))
    X = 0.5 * (X + X.T)
    Rm, e = _row_scaled(X)
    assert np.abs(Rm).max() < 0.5
    d = _digits(Rm)
    acc = np.zeros((n, n))
    for s, t in _PAIRS:
        P = d[s] @ d[t].T
        assert np.abs(P).max() <= 64 * 64 * n
        acc += P.astype(np.float64) * 2.0 ** (-7 * (s + t + 2))
    prod = acc * 2.0 ** (e[:, None] + e[None, :])
    ref = X @ X
    scale = 2.0 ** (e[:, None] + e[None, :]) * n
    assert np.abs(prod - ref).max() / scale.max() < 2.0 ** -40
    assert 64 * 64 * 4096 <= 2 ** 24


def test_dropped_diagonal_pair_biases_the_diagonal():
    """A dropped diagonal pair (s, s) adds a positive sum of squares to every
    diagonal entry of X X: with (3, 3) (1-based (4, 4)) dropped the diagonal of
    a projector-like X (n = 512) is low by ~K E[d^2] 2^-56, while the
    off-diagonal pairs of the same weight only add noise; with (3, 3) kept the
    mean diagonal error is that noise, below 3 % of the bias."""
    rng = np.random.default_rng(8)
    n = 512
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = (Q[:, : n // 2]) @ Q[:, : n // 2].T
    Rm, e = _row_scaled(X)
    d = _digits(Rm)
    ref = X @ X
    scale = 2.0 ** (e[:, None] + e[None, :])

    def emulate(pairs):
        acc = np.zeros((n, n))
        for s, t in pairs:
            acc += (d[s] @ d[t].T).astype(np.float64) * 2.0 ** (-7 * (s + t + 2))
        return acc * scale

    full = emulate(_PAIRS)
    drop = emulate(_PAIRS[:-1])
    bias_drop = np.mean(np.diag(drop - ref) / np.diag(scale))
    bias_full = np.mean(np.diag(full - ref) / np.diag(scale))
    expect = n * np.mean(d[3].astype(np.float64) ** 2) * 2.0 ** -56
    assert bias_drop == pytest.approx(-expect, rel=0.2)
    assert abs(bias_full) < 0.03 * expect
