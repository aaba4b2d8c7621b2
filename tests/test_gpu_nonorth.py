"""The non-orthogonal formulation (App. D.1) on the GPU against the oracle
(oracle/nonorth.py): S and H[n] (tb_build_HS), rho and W (dm_nonorth: the
Newton-Schulz congruence factor, H_perp = Z H Z, SP2 or the Fermi expansion
of H_perp, back-transformation), Mulliken charges with S, forces and energy
with the Pulay and dq/dR terms, and an XL-BOMD trajectory.

Tolerances.  S, H, gamma and v are the same FP64 sums in another order
(1e-12).  dm_nonorth with the FP64 SP2 path: Z converges to ~1e-13, every
congruence product is FP64, so rho and W agree with the generalized
eigenproblem to 1e-9 (the SP2 stop at 1e-11 per eigenvalue, carried through
two products with Z); with tf32x3 + 2 emulated-FP64 refinements of H_perp
the target 1e-6 (||drho||_F / sqrt(n)); at kT > 0 the tf32x3 Fermi
expansion's bound 2e-6.  Charges, forces and energy from the same rho and W
agree to FP64 rounding (1e-10 e, 1e-9 eV/A, 1e-9 eV).  The 20-step FP64
trajectory: positions 1e-9 A, charges 1e-8 e, E_tot 1e-8 eV, as for the
orthogonal trajectories."""

import numpy as np
import pytest
import torch

from workloads import XLParams, molecular_water, nonorth_params, gapped_vapour, thermal_velocities
from oracle import nonorth, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import (DeviceSystem, MDState, NonorthSolver, fermi_opts,
                                          nonorth_report_to_dict, report_to_dict, sp2_opts, xl_params)

pytestmark = pytest.mark.gpu
PN = nonorth_params()
TPN = tbmd.tb_params.from_model(PN)
f64 = dict(dtype=torch.float64, device="cuda")

SYSTEMS = {
    "8 molecules, 4 A apart": lambda: molecular_water(2, 8.0, seed=1),
    "27 molecules, vapour": lambda: gapped_vapour(27, seed=2),
    "64 molecules, 3.2 A apart": lambda: molecular_water(4, 12.8, seed=3),
}


def _charges(N, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    n = rng.normal(0, amp, N)
    return n - n.mean()


def _gpu_HS(ctx, s, n_aux):
    ds = DeviceSystem(s.R, s.types, s.box)
    n, N = ds.norb, ds.natoms
    H = torch.empty(n, n, **f64)
    S = torch.empty(n, n, **f64)
    G = torch.empty(N, N, **f64)
    v = torch.empty(N, **f64)
    tbmd.tb_build_HS(ctx, TPN, ds.sys, ds.R, torch.as_tensor(n_aux, device="cuda"), H, S, G, v)
    torch.cuda.synchronize()
    return ds, H, S, G, v


@pytest.mark.parametrize("system", list(SYSTEMS))
def test_build_HS_matches_oracle(ctx, system):
    s = SYSTEMS[system]()
    n_aux = _charges(s.natoms, 1)
    ds, H, S, G, v = _gpu_HS(ctx, s, n_aux)
    h = tb.build_h(s.R, s.types, s.box, PN)
    So = nonorth.build_S(s.R, s.types, s.box, PN)
    Go = tb.build_gamma(s.R, s.box, PN)
    Ho = nonorth.build_H(h, So, Go, s.types, n_aux)
    eS = float(np.abs(S.cpu().numpy() - So).max())
    eH = float(np.abs(H.cpu().numpy() - Ho).max())
    ev = float(np.abs(v.cpu().numpy() - Go @ n_aux).max())
    print(f"PARITY nonorth H,S {system}: max|dS| {eS:.2e} max|dH| {eH:.2e} max|dv| {ev:.2e}")
    assert eS < 1e-12 and eH < 1e-12 and ev < 1e-12
    # the orthogonal entry point refuses a model with an overlap
    with pytest.raises(tbmd.TBError):
        tbmd.tb_build_H(ctx, TPN, ds.sys, ds.R, None, H, G)


@pytest.mark.parametrize("system", list(SYSTEMS))
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_dm_nonorth_matches_the_generalized_eigenproblem(ctx, system, prec):
    s = SYSTEMS[system]()
    n_aux = _charges(s.natoms, 2)
    ds, H, S, G, v = _gpu_HS(ctx, s, n_aux)
    n = ds.norb
    rho = torch.empty(n, n, **f64)
    W = torch.empty(n, n, **f64)
    so = sp2_opts("fp64", tol=1e-11) if prec == "fp64" else sp2_opts("tf32x3", refine=2)
    sol = NonorthSolver(ctx, n, 0.0, sp2=so)
    sol(H, S, s.n_occ(PN), rho, W)
    torch.cuda.synchronize()
    ref = nonorth.density_matrix(H.cpu().numpy(), S.cpu().numpy(), s.n_occ(PN))
    rep = nonorth_report_to_dict(sol.report)
    srep = report_to_dict(sol.sp2_report)
    e_rho = np.linalg.norm(rho.cpu().numpy() - ref.rho) / np.sqrt(n)
    e_W = np.linalg.norm(W.cpu().numpy() - ref.W) / np.sqrt(n)
    print(f"PARITY dm_nonorth {prec} {system}: drho {e_rho:.2e} dW {e_W:.2e} (Newton-Schulz {rep['ns_iters']} "
          f"iterations, residual {rep['ns_residual']:.1e}; SP2 {srep['iters']}+{srep['refine_iters']}; "
          f"gap {ref.gap:.2f} eV)")
    assert rep["status"] == tbmd.TB_OK and srep["status"] == tbmd.TB_OK
    bound = 1e-9 if prec == "fp64" else 1e-6
    assert e_rho < bound and e_W < 30 * bound  # W carries |H| ~ 30 eV
    q = torch.empty(ds.natoms, **f64)
    tbmd.mulliken_nonorth(ctx, TPN, ds.sys, rho, S, q)
    torch.cuda.synchronize()
    qo = nonorth.mulliken(ref.rho, S.cpu().numpy(), s.types, PN)
    assert float(np.abs(q.cpu().numpy() - qo).max()) < (1e-9 if prec == "fp64" else 1e-5)
    assert abs(float(q.sum())) < 1e-8


def test_dm_nonorth_at_finite_temperature(ctx):
    s = SYSTEMS["27 molecules, vapour"]()
    n_aux = _charges(s.natoms, 4)
    ds, H, S, G, v = _gpu_HS(ctx, s, n_aux)
    n = ds.norb
    rho = torch.empty(n, n, **f64)
    W = torch.empty(n, n, **f64)
    sol = NonorthSolver(ctx, n, 0.2, fermi=fermi_opts("tf32x3"))
    sol(H, S, s.n_occ(PN), rho, W)
    torch.cuda.synchronize()
    ref = nonorth.density_matrix(H.cpu().numpy(), S.cpu().numpy(), s.n_occ(PN), kT=0.2)
    e_rho = np.linalg.norm(rho.cpu().numpy() - ref.rho) / np.sqrt(n)
    mu = float(sol.mu[0])
    print(f"PARITY dm_nonorth kT=0.2: drho {e_rho:.2e} mu {mu:.6f} (oracle {ref.mu:.6f})")
    assert e_rho < 2e-6
    assert np.trace(rho.cpu().numpy() @ S.cpu().numpy()) == pytest.approx(s.n_occ(PN), abs=1e-5)


@pytest.mark.parametrize("system", ["8 molecules, 4 A apart", "64 molecules, 3.2 A apart"])
def test_forces_and_energy_nonorth_match_oracle(ctx, system):
    """From the oracle's rho and W (so that only the force kernel is compared)."""
    s = SYSTEMS[system]()
    n_aux = _charges(s.natoms, 5)
    ds, H, S, G, v = _gpu_HS(ctx, s, n_aux)
    ref = nonorth.density_matrix(H.cpu().numpy(), S.cpu().numpy(), s.n_occ(PN))
    q = nonorth.mulliken(ref.rho, S.cpu().numpy(), s.types, PN)
    F = torch.empty(s.natoms, 3, **f64)
    E = torch.empty(4, **f64)
    tbmd.tb_forces_nonorth(ctx, TPN, ds.sys, ds.R, torch.as_tensor(ref.rho, device="cuda"),
                           torch.as_tensor(ref.W, device="cuda"), torch.as_tensor(q, device="cuda"),
                           torch.as_tensor(n_aux, device="cuda"), v, G, F, E)
    torch.cuda.synchronize()
    Fo = nonorth.forces(s.R, s.types, s.box, PN, ref.rho, ref.W, q, n_aux)
    Eo = nonorth.energy_terms(s.R, s.types, s.box, PN, ref.rho, q, n_aux)
    eF = float(np.abs(F.cpu().numpy() - Fo).max())
    print(f"PARITY nonorth forces {system}: max|dF| {eF:.2e} (max|F| {np.abs(Fo).max():.2f}) "
          f"dE {abs(E[0].item() - sum(Eo)):.2e}")
    assert eF < 1e-9 * max(1.0, np.abs(Fo).max())
    assert E[0].item() == pytest.approx(sum(Eo), abs=1e-9)


def test_xlbomd_nonorth_matches_oracle(ctx):
    """20 steps of 8 H2O-like molecules with the overlap (FP64 SP2 of H_perp)."""
    s = SYSTEMS["8 molecules, 4 A apart"]()
    XL = XLParams()
    M = s.masses(PN)
    v0 = thermal_velocities(M, 300.0, seed=100)
    ds = DeviceSystem(s.R, s.types, s.box)
    opts = sp2_opts("fp64", tol=1e-12, max_iter=120)
    st = MDState(ds, v0, M, s.n_occ(PN), XL.K, opts, nonorth=True)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    it = tbmd.xlbomd_init(ctx, TPN, st.st, xp, opts, 1e-10, 300)
    assert it >= 0
    o = nonorth.xlbomd(s.R, s.types, s.box, PN, XL, v0, M, s.n_occ(PN), 20, record_R=True)
    worst = [0.0, 0.0, 0.0]
    for k in range(21):
        if k:
            tbmd.xlbomd_step(ctx, TPN, st.st, xp, opts)
        torch.cuda.synchronize()
        worst = [max(worst[0], float(np.abs(st.R.cpu().numpy() - o.R[k]).max())),
                 max(worst[1], float(np.abs(st.q.cpu().numpy() - o.q[k]).max())),
                 max(worst[2], abs(st.energies[0].item() - o.E_tot[k]))]
    print(f"PARITY nonorth xlbomd: scf {it}, max|dR| {worst[0]:.2e} max|dq| {worst[1]:.2e} "
          f"max|dE_tot| {worst[2]:.2e}")
    assert worst[0] < 1e-9 and worst[1] < 1e-8 and worst[2] < 1e-8
