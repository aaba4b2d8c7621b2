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


def _mu_search(eps, nocc, kT, mu, step_rule, iters=40, tol=1e-9):
    """Safeguarded chemical-potential search on exact Fermi occupations:
    the bracket starts 40 kT + 1 eV outside the spectrum; each step uses
    dev = sum f - N_occ and t = sum f(1 - f)."""
    beta = 1.0 / kT
    lo, hi = eps[0] - 40 * kT - 1, eps[-1] + 40 * kT + 1
    for it in range(iters):
        f = density.fermi_occupations(eps, mu, kT)
        dev, t = f.sum() - nocc, (f * (1 - f)).sum()
        if abs(dev) <= tol:
            return mu, it
        if dev < 0:
            lo = mu
        else:
            hi = mu
        nxt = mu - dev / (beta * t) if t > 1e-300 else np.nan
        r = abs(dev) / t if t > 0 else np.inf
        if step_rule == "two-tail" and 0.5 <= r <= 1.5:
            a, b = 0.5 * (t + dev), 0.5 * (t - dev)
            if a > 0 and b > 0 and min(a, b) > 1e-3 * max(a, b):
                nxt = mu + 0.5 * np.log(b / a) / beta
            else:
                nxt = mu - np.sign(dev) * min(np.log(abs(dev) / tol), 8.0) / beta
        if not (lo < nxt < hi):
            nxt = 0.5 * (lo + hi)
        mu = nxt
    return mu, iters


def test_two_tail_chemical_potential_step():
    """In a gap of 2.7 eV at kT = 0.1 eV, started 0.3 eV above the highest
    occupied level, Newton's step moves mu by about kT per expansion, while
    the tail steps (balance of the electron and hole tails, or one tail driven
    to the tolerance) land within it in a few; in dense spectra, where
    |dev| is far from Tr[D(I - D)], both rules take Newton's steps."""
    rng = np.random.default_rng(3)
    occ = np.sort(rng.uniform(-10, -1, 40))
    virt = np.sort(rng.uniform(1, 10, 60))
    eps = np.concatenate([occ, virt])
    mu_ref = 0.5 * (occ[-1] + virt[0])
    mu2, it2 = _mu_search(eps, 40.0, 0.1, occ[-1] + 0.3, "two-tail")
    mun, itn = _mu_search(eps, 40.0, 0.1, occ[-1] + 0.3, "newton")
    assert it2 <= 5 and itn >= 2 * it2 + 4
    f = density.fermi_occupations(eps, mu2, 0.1)
    assert abs(f.sum() - 40.0) <= 1e-9
    assert abs(mu2 - mu_ref) < 1.0  # any mu inside the gap carries the occupation
    eps_dense = np.sort(rng.uniform(-10, 10, 200))
    for rule in ("two-tail", "newton"):
        mu, it = _mu_search(eps_dense, 100.0, 0.5, 0.0, rule)
        f = density.fermi_occupations(eps_dense, mu, 0.5)
        assert abs(f.sum() - 100.0) <= 1e-9 and it <= 8


# ------------------------------------------------------------------ entropy
# Eq. Ent_Approx without diagonalisation.  Along the doubling chain of the
# expansion (y_k = 2^k y_0, f_k = f(y_k), e_k = f_k - 1/2) the function
# L(y) = ln(1 + e^y) = -ln(1 - f) obeys L(2y) = 2 L(y) - ln 2 + ln(1 + 4 e^2),
# and per state s(f) = -f ln f - (1 - f) ln(1 - f) = L(y) - (1 - f) y.  So
#   S/k_B = 2 (Tr L(Y) - Tr[(I - D) Y]),  Y = beta (H - mu I),
#   Tr L(Y) = n ln 2 + Tr Y/2 + 2^m dL0 + sum_k 2^(m-1-k) Tr ln(I + 4 E_k^2),
# with dL0 = Tr L(Y0) - n ln 2 - Tr Y0/2 from the Taylor series of L at
# |y0| <= 1/8 and Tr ln A (spectrum of A in [1, 2]) from its Chebyshev series
# of degree 20, whose traces come from T_0..T_10 and Frobenius products
# (Tr T_{10+j} = 2 <T_10, T_j> - Tr T_{10-j}).  All in FP64: the terms are of
# size beta |eps - mu| and cancel to the entropy, so FP32 products would not do.

def chebyshev_log_coeffs(deg=20, nodes=64):
    """Coefficients c_j of ln(3/2 + x/2) = sum_j c_j T_j(x) on [-1, 1] by
    interpolation at Chebyshev nodes (discrete cosine sums)."""
    th = np.pi * (np.arange(nodes) + 0.5) / nodes
    fx = np.log(1.5 + 0.5 * np.cos(th))
    c = np.array([2.0 / nodes * np.sum(fx * np.cos(j * th)) for j in range(deg + 1)])
    c[0] *= 0.5
    return c


def fermi_entropy_recursive(H, mu, kT, y0max=0.125, P=10):
    n = H.shape[0]
    beta = 1.0 / kT
    I = np.eye(n)
    lo, hi = density.gershgorin(H)
    ymax = beta * max(hi - mu, mu - lo)
    m = 0
    while ymax / 2.0 ** m > y0max:
        m += 1
    Y = beta * (H - mu * I)
    Y0 = Y / 2.0 ** m
    Y2 = Y0 @ Y0
    Y4 = Y2 @ Y2
    W = Y2 @ Y4
    dL0 = (np.sum(Y0 * Y0) / 8 - np.sum(Y2 * Y2) / 192 + np.sum(Y2 * Y4) / 2880
           - 17 * np.sum(Y4 * Y4) / 645120)
    E = Y0 @ (-I / 4 + Y2 / 48 - Y4 / 480 + 17 * W / 80640)   # -tanh(y0/2)/2 to y0^7
    c = chebyshev_log_coeffs(2 * P)
    acc = 0.0
    for k in range(m):
        B = 8 * (E @ E) - I                                   # 2A - 3I, A = I + 4E^2
        T = [I, B]
        for j in range(2, P + 1):
            T.append(2 * (B @ T[-1]) - T[-2])
        tau = np.zeros(2 * P + 1)
        for j in range(P + 1):
            tau[j] = np.trace(T[j])
        for j in range(P + 1, 2 * P + 1):
            tau[j] = 2 * np.sum(T[P] * T[j - P]) - tau[2 * P - j]
        acc += 2.0 ** (m - 1 - k) * np.dot(c, tau)
        # A^-1: quadratic minimax start from A = (B + 3I)/2, A^2 = (T2 + 12B + 19I)/8,
        # then three Newton-Schulz steps Z <- Z (2I - AZ)
        Z = (210 * I - 72 * (B + 3 * I) + 4 * (T[2] + 12 * B + 19 * I)) / 99
        for _ in range(3):
            Z = Z @ (2 * I - 0.5 * (B @ Z + 3 * Z))
        E = 2 * (E @ Z)
    D = 0.5 * I + E
    S = 2 * (n * np.log(2) - np.trace(Y) / 2 + 2.0 ** m * dL0 + acc + np.sum(D * Y))
    return S, D, m


def test_chebyshev_log_coefficients():
    c = chebyshev_log_coeffs()
    x = np.linspace(-1, 1, 1001)
    assert np.abs(np.polynomial.chebyshev.chebval(x, c) - np.log(1.5 + 0.5 * x)).max() < 1e-15


@pytest.mark.parametrize("n,seed,kT,width", [(40, 0, 0.1, 24.0), (90, 1, 0.5, 24.0), (150, 2, 0.1, 24.0),
                                              (60, 3, 1.5, 24.0), (120, 4, 0.05, 16.0)])
def test_recursive_fermi_entropy(n, seed, kT, width):
    """The recursion gives the eigenvalue entropy -2 sum [f ln f + (1-f) ln(1-f)]
    (Eq. Ent_Approx) to 2e-9 and the Fermi matrix to 1e-13 at the canonical mu,
    for spectra 16-24 eV wide at kT = 0.05-1.5 eV (m = 9..13 doublings)."""
    H, eps, Q = _random_h(n, seed, width)
    nocc = n // 2
    ref = density.density_fermi(H, nocc, kT)
    S_ref = density.entropy_kB(ref.occ)
    S, D, m = fermi_entropy_recursive(H, ref.mu, kT)
    assert 9 <= m <= 14
    assert abs(S - S_ref) < 2e-9 * max(1.0, S_ref)
    assert np.abs(D - ref.D).max() < 1e-13


def test_recursive_fermi_entropy_controls():
    """Negative controls: a Chebyshev series of degree 12 instead of 20, or a
    Taylor start at |y0| <= 3 (near the radius pi of the series) instead of
    1/8, miss the entropy by more than 1e-6."""
    H, eps, Q = _random_h(80, 7, 24.0)
    ref = density.density_fermi(H, 40, 0.1)
    S_ref = density.entropy_kB(ref.occ)
    S12, _, _ = fermi_entropy_recursive(H, ref.mu, 0.1, P=6)
    S3, _, _ = fermi_entropy_recursive(H, ref.mu, 0.1, y0max=3.0)
    assert abs(S12 - S_ref) > 1e-6 and abs(S3 - S_ref) > 1e-6
