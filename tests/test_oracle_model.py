"""Pins of the oracle's tight-binding model (App. D) against closed forms,
finite differences and invariants that do not reuse the oracle's formulas."""

import numpy as np
import pytest

from workloads import ModelParams, TYPE_O, TYPE_H, water_24_atoms
from oracle import tb

P = ModelParams()


def _fd(fun, x, h=1e-6):
    return (fun(x + h) - fun(x - h)) / (2 * h)


@pytest.mark.parametrize("radial", [tb.hopping_radial, tb.pair_radial])
def test_tail_matches_C2_at_r1_and_vanishes_at_rcut(radial):
    """App. D: t(R) matches value, first and second derivative of zeta at R1 and
    sets all three to zero at R_cut."""
    r = radial(P)
    val = lambda x: r(x)[0]
    r1, rc = P.r1, P.rcut
    e = 1e-7
    # value and slope are continuous at r1
    assert val(r1 - e) == pytest.approx(val(r1 + e), rel=1e-6)
    assert r(r1 - e)[1] == pytest.approx(r(r1 + e)[1], rel=1e-5)
    # second derivative continuous at r1 (one-sided central differences)
    h = 1e-4
    d2_left = (val(r1 - 2 * h) - 2 * val(r1 - h) + val(r1)) / h**2
    d2_right = (val(r1) - 2 * val(r1 + h) + val(r1 + 2 * h)) / h**2
    assert d2_left == pytest.approx(d2_right, rel=2e-3)
    # value, slope and curvature vanish at rc
    assert abs(val(rc - 1e-9)) < 1e-12 * max(1.0, abs(val(r1)))
    assert abs(r(rc - 1e-9)[1]) < 1e-9
    h = 1e-3
    d2_end = (val(rc - 2 * h) - 2 * val(rc - h) + val(rc)) / h**2
    assert abs(d2_end) < 2e-2 * abs(d2_left)
    assert r(rc + 0.1) == (0.0, 0.0)


@pytest.mark.parametrize("radial", [tb.hopping_radial, tb.pair_radial, tb.gamma_radial])
def test_radial_derivatives_match_finite_differences(radial):
    r = radial(P)
    for x in [0.3, 0.9, 1.7, 3.0, 4.99, 5.01, 5.5, 5.95]:
        assert r(x)[1] == pytest.approx(_fd(lambda y: r(y)[0], x), rel=1e-6, abs=1e-10)


def test_gamma_onsite_is_hubbard_u_and_decays_like_coulomb():
    g = tb.gamma_radial(P)
    assert g(0.0)[0] == pytest.approx(P.hubbard_u, rel=1e-15)
    # at r >> k/U (and well inside the window) g -> k/r times the window
    r = 0.6
    x = r / P.gamma_cut
    w = (1 - x) ** 4 * (1 + 4 * x)
    a = P.coulomb_k / P.hubbard_u
    assert g(r)[0] == pytest.approx(P.coulomb_k / np.hypot(r, a) * w)
    assert g(P.gamma_cut)[0] == 0.0


def test_gamma_matrix_positive_definite():
    """gamma is a product of positive-definite radial kernels, so the periodic
    gamma matrix is positive definite (the SCC functional is convex)."""
    s = water_24_atoms()
    G = tb.build_gamma(s.R, s.box, P)
    assert np.allclose(G, G.T)
    assert np.linalg.eigvalsh(G).min() > 0.5


def test_slater_koster_diatomic_along_z():
    """Closed-form two-centre blocks for a bond along +z (l = (0, 0, 1))."""
    r = 1.3
    V = P.t_hop * np.exp(-r / P.r_decay)
    Vr = tb.hopping_radial(P)
    blk, _ = tb.sk_block(TYPE_O, TYPE_O, np.array([0.0, 0.0, r]), Vr)
    expect = np.zeros((4, 4))
    expect[0, 0] = -V             # ss-sigma
    expect[0, 3] = V              # s -> pz: +l_z Vsp
    expect[3, 0] = -V             # pz -> s: -l_z Vsp
    expect[3, 3] = V              # pz pz: pp-sigma
    expect[1, 1] = expect[2, 2] = -V   # px px, py py: pp-pi
    assert np.allclose(blk, expect, atol=1e-15)
    blk, _ = tb.sk_block(TYPE_H, TYPE_O, np.array([0.0, 0.0, r]), Vr)
    assert np.allclose(blk, [[-V, 0, 0, V]])
    blk, _ = tb.sk_block(TYPE_O, TYPE_H, np.array([0.0, 0.0, r]), Vr)
    assert np.allclose(blk, [[-V], [0], [0], [-V]])


def test_slater_koster_reciprocity_and_derivative():
    """h_{a,b}(d) = h_{b,a}(-d)^T, and d(block)/dd matches finite differences."""
    Vr = tb.hopping_radial(P)
    rng = np.random.default_rng(3)
    for ta, tb_ in [(TYPE_O, TYPE_O), (TYPE_O, TYPE_H), (TYPE_H, TYPE_O), (TYPE_H, TYPE_H)]:
        d = rng.normal(size=3)
        d *= 1.4 / np.linalg.norm(d)
        b1, db = tb.sk_block(ta, tb_, d, Vr)
        b2, _ = tb.sk_block(tb_, ta, -d, Vr)
        assert np.allclose(b1, b2.T, atol=1e-15)
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            fd = (tb.sk_block(ta, tb_, d + e, Vr)[0] - tb.sk_block(ta, tb_, d - e, Vr)[0]) / 2e-6
            assert np.allclose(db[:, :, k], fd, rtol=1e-6, atol=1e-10)


def test_h_spectrum_invariant_under_rigid_rotation():
    """A wrong angular factor in the Slater-Koster table breaks rotational
    invariance of the spectrum of an isolated cluster."""
    rng = np.random.default_rng(1)
    R = rng.uniform(0, 3.0, size=(5, 3)) + 20.0
    types = np.array([TYPE_O, TYPE_O, TYPE_H, TYPE_H, TYPE_O], dtype=np.int32)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    R2 = (R - 21.5) @ Q.T + 21.5
    e1 = np.linalg.eigvalsh(tb.build_h(R, types, 100.0, P))
    e2 = np.linalg.eigvalsh(tb.build_h(R2, types, 100.0, P))
    assert np.allclose(e1, e2, atol=1e-12)


def test_H_is_h_plus_charge_shift_on_every_orbital_of_the_atom():
    s = water_24_atoms()
    h = tb.build_h(s.R, s.types, s.box, P)
    G = tb.build_gamma(s.R, s.box, P)
    assert np.allclose(h, h.T)
    n = np.linspace(-0.5, 0.5, s.natoms)
    H = tb.build_H(h, G, s.types, n)
    offs = tb.orbital_offsets(s.types)
    d = np.diag(H - h)
    for i in range(s.natoms):
        assert np.allclose(d[offs[i]:offs[i + 1]], sum(G[i, j] * n[j] for j in range(s.natoms)))
    assert np.allclose(H - np.diag(np.diag(H)), h - np.diag(np.diag(h)))


def test_periodic_images_small_box():
    """Two atoms in a box smaller than the cut-off see several images; the
    hopping matches an explicit sum over lattice translations."""
    box = 4.0
    R = np.array([[0.2, 0.3, 0.1], [1.1, 0.4, 0.3]])
    types = np.array([TYPE_H, TYPE_H], dtype=np.int32)
    h = tb.build_h(R, types, box, P)
    Vr = tb.hopping_radial(P)
    ref01 = 0.0
    ref00 = 0.0
    for a in range(-3, 4):
        for b in range(-3, 4):
            for c in range(-3, 4):
                T = box * np.array([a, b, c])
                r01 = np.linalg.norm(R[1] - R[0] + T)
                ref01 += -Vr(r01)[0]
                if (a, b, c) != (0, 0, 0):
                    ref00 += -Vr(np.linalg.norm(T))[0]
    assert h[0, 1] == pytest.approx(ref01, rel=1e-12)
    assert h[0, 0] == pytest.approx(P.eps_s_H + ref00, rel=1e-12)


# ---------------------------------------------------------------- long range
# The Ewald-summed Coulomb potential and the Gaussian-charge gamma, pinned by
# textbook lattice constants and closed-form limits.

def test_ewald_nacl_madelung_constant():
    """Rock salt (8 ions of charge +-1 in a cubic cell of side a): the Coulomb
    energy per ion pair is -M / r0 with r0 = a/2 and Madelung's constant
    M = 1.7475645946 (point charges; the background cancels for a neutral cell)."""
    a = 5.64
    na = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * a
    cl = na + np.array([.5, 0, 0]) * a
    R = np.vstack([na, cl])
    qv = np.array([1.0] * 4 + [-1.0] * 4)
    for alpha in (0.5, 0.9):
        E = 0.0
        for i in range(8):
            for j in range(8):
                if i == j:
                    psi, _ = tb.ewald_psi(np.zeros((1, 3)), a, alpha, self_term=True)
                else:
                    psi, _ = tb.ewald_psi((R[j] - R[i])[None, :], a, alpha)
                E += 0.5 * qv[i] * qv[j] * psi[0]
        assert E / 4 * (a / 2) == pytest.approx(-1.7475645946331822, rel=1e-10)


def test_ewald_simple_cubic_self_term_and_small_distance_limit():
    """A unit charge, its simple-cubic images and a neutralising background:
    the potential of the images at the charge is xi/L with xi = -2.837297479
    (the simple-cubic constant), and near the charge
    psi(d) = 1/d + xi/L + (2 pi / 3) d^2 / L^3 + O(d^4/L^5) (the background's
    uniform charge -1/V gives the d^2 term)."""
    L = 7.0
    xi = -2.837297479480620
    psi0, _ = tb.ewald_psi(np.zeros((1, 3)), L, 0.8, self_term=True)
    assert psi0[0] * L == pytest.approx(xi, rel=1e-10)
    res = []
    for s in (0.004, 0.002, 0.001):
        d = np.array([[2.0, 1.0, -1.5]]) * s * L
        r = np.linalg.norm(d)
        psi, _ = tb.ewald_psi(d, L, 0.8)
        res.append(psi[0] - (1 / r + xi / L + 2 * np.pi / 3 * r * r / L**3))
    # the remainder is fourth order: it drops 16-fold per halving of d
    assert res[0] / res[1] == pytest.approx(16.0, rel=0.03) and res[1] / res[2] == pytest.approx(16.0, rel=0.05)
    assert abs(res[2]) < 1e-10


def test_ewald_independent_of_the_split_and_gradient():
    rng = np.random.default_rng(3)
    box = 6.5
    d = rng.uniform(-4, 4, (5, 3))
    a, ga = tb.ewald_psi(d, box, 0.45)
    b, gb = tb.ewald_psi(d, box, 1.1)
    assert np.abs(a - b).max() < 1e-11 and np.abs(ga - gb).max() < 1e-11
    h = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (tb.ewald_psi(d + e, box, 0.7)[0] - tb.ewald_psi(d - e, box, 0.7)[0]) / (2 * h)
        assert np.abs(fd - ga[:, k]).max() < 1e-8


def test_gaussian_gamma_onsite_long_range_and_positive():
    """gamma_form = 1: gamma_ii = U + (images), gamma_ij -> k erf(r/c)/r + xi k/L
    for a pair far from its images (large box), Ewald split independent,
    positive definite on neutral charge vectors, gradient = finite differences."""
    import dataclasses
    P1 = dataclasses.replace(ModelParams(), gamma_form=1)
    from scipy.special import erf
    L = 60.0
    R = np.array([[0.0, 0.0, 0.0], [2.3, 1.1, -0.7]])
    G = tb.gamma_ewald(R, L, P1)
    c = tb.gaussian_width(P1)
    r = np.linalg.norm(R[1] - R[0])
    xi = -2.837297479480620
    k = P1.coulomb_k
    assert G[0, 1] == pytest.approx(k * erf(r / c) / r + k * xi / L + k * 2 * np.pi / 3 * r * r / L**3, abs=1e-6)
    assert G[0, 0] == pytest.approx(P1.hubbard_u + k * xi / L, abs=1e-9)
    s = water_24_atoms()
    Ga = tb.gamma_ewald(s.R, s.box, dataclasses.replace(P1, ewald_alpha=0.5))
    Gb, dG = tb.gamma_ewald(s.R, s.box, dataclasses.replace(P1, ewald_alpha=0.9), with_grad=True)
    assert np.abs(Ga - Gb).max() < 1e-10
    assert np.allclose(Gb, Gb.T, atol=1e-14)
    Pn = np.eye(24) - 1.0 / 24
    assert np.linalg.eigvalsh(Pn @ Gb @ Pn)[1:].min() > 0
    h = 1e-5
    i, j = 2, 7
    for kk in range(3):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[j, kk] += h
        Rm[j, kk] -= h
        fd = (tb.gamma_ewald(Rp, s.box, P1)[i, j] - tb.gamma_ewald(Rm, s.box, P1)[i, j]) / (2 * h)
        assert fd == pytest.approx(dG[i, j, kk], abs=1e-7)


def test_zeta_radial_form():
    """zeta(R) = A0 exp(A1 R + A2 R^2 + A3 R^3 + A4 R^4): with A2..A4 = 0 it is
    the plain exponential; with them nonzero its derivative is the finite
    difference of the value and the App. D tail joins it with two
    continuous derivatives at r1 and vanishes at rcut."""
    P = ModelParams()
    plain = tb.hopping_radial(P)
    for r in (0.8, 1.5, 3.0):
        assert plain(r)[0] == pytest.approx(P.t_hop * np.exp(-r / P.r_decay), rel=1e-14)
    z = tb.zeta_radial(3.0, (-2.0, 0.05, -0.01, 0.0005), P.r1, P.rcut)
    h = 1e-6
    for r in (1.0, 2.5, 4.5, 5.5):
        fd = (z(r + h)[0] - z(r - h)[0]) / (2 * h)
        assert fd == pytest.approx(z(r)[1], rel=1e-7)
    a, b = z(P.r1 - 1e-9), z(P.r1 + 1e-9)
    assert a[0] == pytest.approx(b[0], rel=1e-7) and a[1] == pytest.approx(b[1], rel=1e-6)
    d2 = lambda r: (z(r + 1e-6)[1] - z(r - 1e-6)[1]) / 2e-6
    assert d2(P.r1 - 3e-6) == pytest.approx(d2(P.r1 + 3e-6), rel=1e-4)
    assert z(P.rcut)[0] == 0.0 and abs(z(P.rcut - 1e-6)[0]) < 1e-12


def test_forces_are_minus_the_energy_gradient_with_long_range_gamma_and_zeta():
    """Central differences of the energy at fixed n and D, with the Ewald gamma
    and a nonzero zeta polynomial on both h and phi."""
    import dataclasses
    from oracle import observables, density
    P1 = dataclasses.replace(ModelParams(), gamma_form=1, zeta_a2=0.02, zeta_a3=-0.004, pair_a2=0.1)
    s = water_24_atoms()
    rng = np.random.default_rng(8)
    n = rng.normal(0, 0.2, 24)
    n -= n.mean()
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P1), tb.build_gamma(s.R, s.box, P1), s.types, n)
    D = density.density_T0(H, int(s.n_occ(P1))).D
    q = observables.mulliken(D, s.types, P1)
    F = observables.forces(s.R, s.types, s.box, P1, D, q, n)
    h = 1e-5
    for a, kk in ((0, 0), (5, 2), (17, 1)):
        Rp, Rm = s.R.copy(), s.R.copy()
        Rp[a, kk] += h
        Rm[a, kk] -= h
        Ep = observables.potential_energy(Rp, s.types, s.box, P1, D, q, n)
        Em = observables.potential_energy(Rm, s.types, s.box, P1, D, q, n)
        assert -(Ep - Em) / (2 * h) == pytest.approx(F[a, kk], rel=2e-6, abs=1e-7)
    assert np.abs(F.sum(axis=0)).max() < 1e-9
