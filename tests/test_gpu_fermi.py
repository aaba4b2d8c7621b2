"""dm_fermi (GEMM-only recursive Fermi-operator expansion, tensor cores) on
the GPU against the oracle's diagonalised Fermi-Dirac density matrix with
the canonical chemical potential (bisection to Tr D = N_occ).

Tolerance: the tf32x3 products carry ~2^-22 relative error; in the deviation
form E = X - I/2 those errors add up over the m (8..11 here) doubling steps instead
of being doubled m times, leaving ~1e-6 absolute error in D.  mu is compared
only where it is unique at this temperature (no wide gap around it)."""

import numpy as np
import pytest
import torch

from workloads import random_gapped_matrix, water_system, ModelParams, water_24_atoms
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import FermiSolver, fermi_opts, fermi_report_to_dict

pytestmark = pytest.mark.gpu
P = ModelParams()


def _run(ctx, H, nocc, kT, prec="tf32x3", warm_again=False):
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = FermiSolver(ctx, H.shape[0], fermi_opts(prec))
    s(Ht, nocc, kT, D)
    torch.cuda.synchronize()
    out = [(D.cpu().numpy(), fermi_report_to_dict(s.report))]
    if warm_again:
        s(Ht, nocc, kT, D)
        torch.cuda.synchronize()
        out.append((D.cpu().numpy(), fermi_report_to_dict(s.report)))
    return out


def _err(A, B):
    return np.linalg.norm(A - B) / np.sqrt(A.shape[0])


def _c1_H(seed=0):
    s = water_24_atoms()
    rng = np.random.default_rng(seed)
    na = rng.normal(0, 0.3, s.natoms)
    na -= na.mean()
    return tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types, na), s.n_occ(P)


@pytest.mark.parametrize("kT", [0.1, 0.5])
def test_fermi_matches_diagonalisation_small_gap(ctx, kT):
    H, nocc = _c1_H()
    ref = density.density_fermi(H, nocc, kT)
    (D, rep), (D2, rep2) = _run(ctx, H, nocc, kT, warm_again=True)
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 1e-6
    assert rep["mu"] == pytest.approx(ref.mu, abs=1e-5)
    assert abs(rep["trace"] - nocc) < 1e-5
    # a warm start from the previous mu converges in one expansion
    assert rep2["mu_iters"] == 1 and _err(D2, ref.D) < 1e-6


@pytest.mark.parametrize("prec,tol", [("tf32x3", 2e-6), ("bf16x3", 5e-6)])
def test_fermi_water_systems(ctx, prec, tol):
    w = water_system(300, density=1.0, seed=0)
    H = tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                   np.zeros(w.natoms))
    ref = density.density_fermi(H, w.n_occ(P), 0.1)
    (D, rep), = _run(ctx, H, w.n_occ(P), 0.1, prec)
    print(f"PARITY fermi {prec} water 300: dD={_err(D, ref.D):.3e}")
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < tol
    # D is a function of H: it commutes with H
    assert np.linalg.norm(H @ D - D @ H) / np.sqrt(H.shape[0]) < 100 * tol


def test_fermi_ragged_larger_system(ctx):
    w = water_system(1024, density=1.0, seed=1)
    H = tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                   np.zeros(w.natoms))
    ref = density.density_fermi(H, w.n_occ(P), 0.1)
    (D, rep), = _run(ctx, H, w.n_occ(P), 0.1)
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 2e-6
    assert rep["mu"] == pytest.approx(ref.mu, abs=1e-5)


def test_fermi_dense_random_spectrum(ctx):
    H, _ = random_gapped_matrix(500, 200, gap=0.5, width=20.0, seed=3)
    ref = density.density_fermi(H, 200.0, 0.1)
    (D, rep), = _run(ctx, H, 200.0, 0.1)
    print(f"PARITY fermi random 500: dD={_err(D, ref.D):.3e}")
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 2e-5


def test_fermi_low_temperature_limit_is_the_projector(ctx):
    """A gapped spectrum at kT << gap: the Fermi operator is the T = 0 projector."""
    H, _ = random_gapped_matrix(256, 100, gap=3.0, width=12.0, seed=8)
    proj = density.density_T0(H, 100).D
    (D, rep), = _run(ctx, H, 100.0, 0.05)
    assert _err(D, proj) < 5e-6


def test_fermi_spectrum_too_wide_for_the_doublings(ctx):
    """beta (eps_max - eps_min + 80 kT + 2 eV) > 2^(m+1) for the largest m
    allowed: the third-order start is not defined there, and the report says
    TB_ERR_ARG (no expansion runs)."""
    H, nocc = _c1_H()
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    kT = 0.011  # Gershgorin width 21.6 eV: beta (21.6 + 0.9 + 2) ~ 2230 > 2^11
    s = FermiSolver(ctx, H.shape[0], fermi_opts("tf32x3", m=10))
    s(Ht, nocc, kT, D)
    torch.cuda.synchronize()
    rep = fermi_report_to_dict(s.report)
    assert rep["status"] == tbmd.TB_ERR_ARG
    assert rep["mu_iters"] == 0


def test_fermi_uses_the_fewest_doublings_the_spectrum_allows(ctx):
    """The device takes the smallest m >= 8 with beta (hi - lo) <= 2^(m+1):
    8 for the 24-atom system at kT = 0.1 eV (beta (hi - lo) ~ 320), 11 at
    kT = 0.011 eV (~2230)."""
    H, nocc = _c1_H()
    (D, rep), = _run(ctx, H, nocc, 0.1)
    assert rep["m"] == 8 and rep["status"] == tbmd.TB_OK
    assert _err(D, density.density_fermi(H, nocc, 0.1).D) < 1e-6
    (D, rep), = _run(ctx, H, nocc, 0.011)
    assert rep["m"] == 11
    if rep["status"] == tbmd.TB_OK:
        assert _err(D, density.density_fermi(H, nocc, 0.011).D) < 1e-5
