"""Long-range gamma (Ewald-summed Gaussian charges, gamma_form = 1) and the
zeta(R) radial form of App. D on the GPU against the oracle: gamma, H[n],
forces and energy, and a short XL-BOMD trajectory.

Tolerances: gamma and H are FP64 sums of the same terms in another order
(real-space images, reciprocal vectors) and agree to 1e-10 eV; forces to
1e-8 eV/A (relative 1e-9 of the largest), energies to 1e-8 eV."""

import dataclasses

import numpy as np
import pytest
import torch

from workloads import ModelParams, XLParams, molecular_water, thermal_velocities, water_24_atoms, water_system
from oracle import density, md, observables, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DeviceSystem, MDState, sp2_opts, xl_params

pytestmark = pytest.mark.gpu
PE = dataclasses.replace(ModelParams(), gamma_form=1, zeta_a2=0.02, zeta_a3=-0.004, pair_a2=0.1)


def _gpu_H(ctx, s, P, n_aux):
    TP = tbmd.tb_params.from_model(P)
    ds = DeviceSystem(s.R, s.types, s.box)
    f64 = dict(dtype=torch.float64, device="cuda")
    H = torch.empty(ds.norb, ds.norb, **f64)
    G = torch.empty(ds.natoms, ds.natoms, **f64)
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, torch.as_tensor(n_aux, device="cuda"), H, G)
    torch.cuda.synchronize()
    return ds, TP, H, G


@pytest.mark.parametrize("system,alpha", [("24 atoms", 0.0), ("24 atoms", 0.9), ("water 150", 0.0)])
def test_ewald_gamma_and_H_match_oracle(ctx, system, alpha):
    s = water_24_atoms() if system == "24 atoms" else water_system(150, density=1.0, seed=4)
    P = dataclasses.replace(PE, ewald_alpha=alpha)
    rng = np.random.default_rng(1)
    n = rng.normal(0, 0.2, s.natoms)
    n -= n.mean()
    ds, TP, H, G = _gpu_H(ctx, s, P, n)
    Go = tb.build_gamma(s.R, s.box, PE)  # the oracle's own split: the sum does not depend on it
    Ho = tb.build_H(tb.build_h(s.R, s.types, s.box, PE), Go, s.types, n)
    eG = float(np.abs(G.cpu().numpy() - Go).max())
    eH = float(np.abs(H.cpu().numpy() - Ho).max())
    print(f"PARITY ewald gamma {system} alpha={alpha}: max|dgamma| {eG:.2e} max|dH| {eH:.2e}")
    assert eG < 1e-10 and eH < 1e-10


def test_ewald_forces_and_energy_match_oracle(ctx):
    s = water_24_atoms()
    rng = np.random.default_rng(2)
    n = rng.normal(0, 0.2, s.natoms)
    n -= n.mean()
    ds, TP, H, G = _gpu_H(ctx, s, PE, n)
    Ho = tb.build_H(tb.build_h(s.R, s.types, s.box, PE), tb.build_gamma(s.R, s.box, PE), s.types, n)
    D = density.density_T0(Ho, int(s.n_occ(PE))).D
    q = observables.mulliken(D, s.types, PE)
    f64 = dict(dtype=torch.float64, device="cuda")
    F = torch.empty(s.natoms, 3, **f64)
    E = torch.empty(4, **f64)
    tbmd.tb_forces(ctx, TP, ds.sys, ds.R, torch.as_tensor(D, device="cuda"), torch.as_tensor(q, device="cuda"),
                   torch.as_tensor(n, device="cuda"), G, F, E)
    torch.cuda.synchronize()
    Fo = observables.forces(s.R, s.types, s.box, PE, D, q, n)
    Eo = observables.energy_terms(s.R, s.types, s.box, PE, D, q, n)
    eF = float(np.abs(F.cpu().numpy() - Fo).max())
    print(f"PARITY ewald forces: max|dF| {eF:.2e} (max|F| {np.abs(Fo).max():.2f}), "
          f"dE {abs(E[0].item() - sum(Eo)):.2e}")
    assert eF < 1e-8
    assert E[1].item() == pytest.approx(Eo[0], abs=1e-8)
    assert E[2].item() == pytest.approx(Eo[1], abs=1e-8)
    assert E[3].item() == pytest.approx(Eo[2], abs=1e-8)


def test_xlbomd_with_long_range_gamma_matches_oracle(ctx):
    """Ten steps of 8 H2O-like molecules (24 atoms) with the Ewald gamma and the zeta
    polynomial (T_e = 0, FP64 SP2): positions, charges and E_tot agree."""
    XL = dataclasses.replace(XLParams(), kappa_scale=0.15)
    m = molecular_water(2, 8.0, seed=1)
    M = m.masses(PE)
    v0 = thermal_velocities(M, 300.0, seed=101)
    TP = tbmd.tb_params.from_model(PE)
    ds = DeviceSystem(m.R, m.types, m.box)
    opts = sp2_opts("fp64", tol=1e-12, max_iter=120)
    st = MDState(ds, v0, M, m.n_occ(PE), XL.K, opts)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    o = md.xlbomd(m.R, m.types, m.box, PE, XL, v0, M, m.n_occ(PE), 10, record_R=True, scf_strict=False)
    worst = [0.0, 0.0, 0.0]
    for k in range(11):
        if k:
            tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
        torch.cuda.synchronize()
        worst = [max(worst[0], float(np.abs(st.R.cpu().numpy() - o.R[k]).max())),
                 max(worst[1], float(np.abs(st.q.cpu().numpy() - o.q[k]).max())),
                 max(worst[2], abs(st.energies[0].item() - o.E_tot[k]))]
    print(f"PARITY ewald xlbomd: max|dR| {worst[0]:.2e} max|dq| {worst[1]:.2e} max|dE_tot| {worst[2]:.2e}")
    assert worst[0] < 1e-9 and worst[1] < 1e-8 and worst[2] < 1e-8
