"""T_e = 0 XL-BOMD on the gapped recipe (workloads.gapped_params), whose SCF
converges: 100 steps of the 24-atom system against the oracle's trajectory,
and the thresholded block-sparse path against the dense path on the
2046-atom system (1/8 of the 16384-atom Morton system).

Tolerances.  24 atoms, FP64 SP2 stopped at |Tr X - Tr X^2| <= 1e-12 on both
sides: per step the GPU and the oracle differ by FP64 rounding (~1e-13 in
D); over 100 steps of 0.25 fs that difference is carried, not amplified
beyond ~10x (the trajectory is 25 fs, shorter than the vibrations' own
period), so positions are held to 1e-9 A, charges to 1e-8 e and E_tot to
1e-8 eV, as for the 10-step trajectories of the other MD tests.

2046 atoms: the dense path (tf32x3 products, two FP64-exact refinements)
gives D to ~1e-7 of the FP64 path.  The block-sparse path has no FP64
refinement: it stops when Tr X - Tr X^2 reaches the noise floor of its FP32
products, f = 2 n 2^-24 (4.9e-4 at n = 4092), so its Tr D is off N_occ by up
to ~f (plus the dropped blocks' share, far smaller at tau = 1e-5), held here
to 2 f.  A trace error d moves E_band = 2 Tr[hD] by at most 2 W d (W the
Gershgorin width of H) and the SCC energy by a like amount through the
charges, so E_tot of the two paths is held to B = 4 W f at every step
(0.043 eV here; measured 0.022 eV over 400 steps).  The offset varies with the step, so the
least-squares drift of the two E_tot series differs by at most 6 B / (N T)
for N atoms over a time T; sigma (E_tot's fluctuation, dominated by the
integration error of dt = 0.25 fs) agrees to 10 %."""

import numpy as np
import pytest
import torch

from workloads import XLParams, gapped_params, gapped_vapour, thermal_velocities
from oracle import md
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, DeviceSystem, MDState, report_to_dict, sp2_opts, xl_params

pytestmark = pytest.mark.gpu
P = gapped_params()
TP = tbmd.tb_params.from_model(P)
XL = XLParams()


def test_gapped_24_atoms_100_steps_match_oracle(ctx):
    s = gapped_vapour(8)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100)
    ds = DeviceSystem(s.R, s.types, s.box)
    opts = sp2_opts("fp64", tol=1e-12, max_iter=120)
    st = MDState(ds, v0, M, s.n_occ(P), XL.K, opts)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    it = tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    assert it >= 0
    o = md.xlbomd(s.R, s.types, s.box, P, XL, v0, M, s.n_occ(P), 100, record_R=True)
    worst = [0.0, 0.0, 0.0]
    E = []
    for k in range(101):
        if k:
            tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
        torch.cuda.synchronize()
        E.append(st.energies[0].item())
        worst = [max(worst[0], float(np.abs(st.R.cpu().numpy() - o.R[k]).max())),
                 max(worst[1], float(np.abs(st.q.cpu().numpy() - o.q[k]).max())),
                 max(worst[2], abs(E[-1] - o.E_tot[k]))]
    g = md.energy_drift(E, XL.dt, s.natoms)
    r = md.energy_drift(o.E_tot, XL.dt, s.natoms)
    print(f"PARITY gapped 24 atoms, 100 steps: scf {it}, max|dR| {worst[0]:.2e} max|dq| {worst[1]:.2e} "
          f"max|dE_tot| {worst[2]:.2e}; sigma {g[0]:.3e} / {r[0]:.3e} eV, drift {g[1]:.3e} / {r[1]:.3e}")
    assert report_to_dict(st.report)["status"] == tbmd.TB_OK
    assert worst[0] < 1e-9 and worst[1] < 1e-8 and worst[2] < 1e-8
    assert g[0] < 5e-3 and abs(g[1]) < 0.05


def test_gapped_2046_atoms_block_sparse_drift_matches_dense(ctx):
    s = gapped_vapour(682, seed=0, morton=True)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    steps = 400
    out = {}
    for label, o in (("sparse", sp2_opts("tf32x3", max_iter=60, tau=1e-5)),
                     ("dense", sp2_opts("tf32x3", max_iter=100, tol=1e-10, refine=2))):
        ds = DeviceSystem(s.R, s.types, s.box)
        st = MDState(ds, v0, M, s.n_occ(P), XL.K, o)
        it = tbmd.xlbomd_init(ctx, TP, st.st, xp, o, 1e-6, 200)
        Eb = torch.empty(steps + 1, dtype=torch.float64, device="cuda")
        Eb[0].copy_(st.energies[0])
        dq = torch.zeros((), dtype=torch.float64, device="cuda")
        for k in range(steps):
            tbmd.xlbomd_step(ctx, TP, st.st, xp, o)
            Eb[k + 1].copy_(st.energies[0])
            dq = torch.maximum(dq, st.energies[6])
        E = Eb.cpu().numpy()
        out[label] = (it, E, md.energy_drift(list(E), XL.dt, s.natoms), dq.item(),
                      report_to_dict(st.report))
        del st
    # both paths' D at the same H (R0, n = 0) against the FP64 path
    ds = DeviceSystem(s.R, s.types, s.box)
    n = ds.norb
    f64 = dict(dtype=torch.float64, device="cuda")
    H = torch.empty(n, n, **f64)
    G = torch.empty(s.natoms, s.natoms, **f64)
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, None, H, G)
    Ds = {}
    for label, o in (("sparse", sp2_opts("tf32x3", max_iter=60, tau=1e-5)),
                     ("dense", sp2_opts("tf32x3", max_iter=100, tol=1e-10, refine=2)),
                     ("fp64", sp2_opts("fp64", max_iter=100, tol=1e-11))):
        D = torch.empty_like(H)
        sol = DensitySolver(ctx, n, o)
        sol(H, s.n_occ(P), D)
        torch.cuda.synchronize()
        Ds[label] = (D, report_to_dict(sol.report))
    floor = 2.0 * n * 2.0 ** -24
    W = Ds["fp64"][1]["eps_max"] - Ds["fp64"][1]["eps_min"]
    e_dense = (Ds["dense"][0] - Ds["fp64"][0]).norm().item() / n ** 0.5
    tr_sparse = Ds["sparse"][1]["trace"] - s.n_occ(P)
    del Ds, H, G, D, sol
    (i_s, E_s, d_s, q_s, r_s), (i_d, E_d, d_d, q_d, r_d) = out["sparse"], out["dense"]
    dE = float(np.abs(E_s - E_d).max())
    B = 4.0 * W * floor
    T = steps * XL.dt * 1e-3
    print(f"PARITY gapped 2046 atoms, same H: dense vs FP64 ||dD||_F/sqrt(n) {e_dense:.2e}, block-sparse "
          f"Tr D - N {tr_sparse:.2e} (floor {floor:.2e})")
    print(f"PARITY gapped 2046 atoms, {steps} steps, block-sparse tau=1e-5 vs dense: scf {i_s}/{i_d}, "
          f"max|dE_tot| {dE:.2e} eV (bound {B:.2e}); sigma {d_s[0]:.3e} / {d_d[0]:.3e} eV, drift {d_s[1]:.3e} / "
          f"{d_d[1]:.3e} eV/atom/ps, max|n-q| {q_s:.2e} / {q_d:.2e}, D blocks {r_s['blocks']}")
    assert e_dense < 1e-6
    assert abs(tr_sparse) <= 2 * floor
    assert i_s >= 0 and i_d >= 0
    assert r_s["status"] == tbmd.TB_OK and r_d["status"] == tbmd.TB_OK
    assert dE <= B
    assert d_s[0] == pytest.approx(d_d[0], rel=0.1)
    assert abs(d_s[1] - d_d[1]) <= 6 * B / (s.natoms * T)
    assert q_s < 0.05 and q_d < 0.05
