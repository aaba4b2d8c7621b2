"""Pins of the numerical methods the GPU path uses where the paper gives no
recipe, checked in FP64 NumPy against exact definitions (no GPU):

* the recursive Fermi-operator expansion in deviation form (m = 14 doublings
  from the linearised start) against the Fermi function;
* the second-order canonical shift of a Fermi density matrix and its
  remainder bound |u|^3/6 Tr[D(I - D)];
* the balanced base-64 digit split of the emulated-FP64 refinement: digit
  ranges, exact reconstruction, and the slice-pair sum with s + t <= 8
  against the FP64 product.
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


def _digits(x_row_scaled):
    """Balanced base-64 digits (7 of them) of rint(r 2^42), |r| < 1."""
    R = np.rint(x_row_scaled * 2.0 ** 42).astype(np.int64)
    d = np.zeros((7,) + R.shape, dtype=np.int64)
    for s in range(6, 0, -1):
        low = ((R + 32) & 63) - 32
        d[s] = low
        R = (R - low) >> 6
    d[0] = R
    return d


def test_balanced_digit_split_is_exact_and_bounded():
    rng = np.random.default_rng(4)
    r = rng.uniform(-1.0, 1.0, 20000) * (1 - 1e-12)
    r[:4] = [0.0, 1 - 2.0 ** -50, -(1 - 2.0 ** -50), 2.0 ** -43]
    d = _digits(r)
    assert np.abs(d[0]).max() <= 64 and np.abs(d[1:]).max() <= 32
    rec = sum(d[s].astype(np.float64) * 2.0 ** (-6 * (s + 1)) for s in range(7))
    assert np.array_equal(rec, np.rint(r * 2.0 ** 42) / 2.0 ** 42)
    assert np.abs(rec - r).max() <= 2.0 ** -43
    # every digit is an integer exactly representable in bf16 (8 significant bits)
    assert np.abs(d).max() <= 256


def test_slice_pair_product_matches_fp64():
    """sum over s + t <= 8 of 2^(-6(s+t)) P_st, P_st exact integer products,
    equals the FP64 product of the row-scaled matrices to ~2^-45 relative; the
    integer products stay below 2^24 (exact in an FP32 accumulator) for K <= 4096."""
    rng = np.random.default_rng(5)
    n = 96
    X = rng.standard_normal((n, n))
    X = 0.5 * (X + X.T)
    e = np.array([np.frexp(np.abs(row).max())[1] for row in X])
    Rm = X / 2.0 ** e[:, None]
    d = _digits(Rm)
    acc = np.zeros((n, n))
    for s in range(7):
        for t in range(7):
            if (s + 1) + (t + 1) <= 8:
                P = d[s] @ d[t].T
                assert np.abs(P).max() <= 64 * 64 * n
                acc += P.astype(np.float64) * 2.0 ** (-6 * (s + t + 2))
    prod = acc * 2.0 ** (e[:, None] + e[None, :])
    ref = X @ X
    scale = np.abs(X).max(axis=1)[:, None] * np.abs(X).max(axis=1)[None, :] * n
    assert np.abs(prod - ref).max() / scale.max() < 2.0 ** -40
    assert 64 * 64 * 4096 <= 2 ** 24
