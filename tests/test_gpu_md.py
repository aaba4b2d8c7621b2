"""xlbomd_init / xlbomd_step on the GPU against the oracle's XL-BOMD
trajectory from the same inputs (molecular pin system, FP64 SP2 on the GPU,
eigh in the oracle)."""

import dataclasses

import numpy as np
import pytest
import torch

from workloads import ModelParams, XLParams, molecular_water, thermal_velocities
from oracle import md
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DeviceSystem, MDState, sp2_opts, xl_params, report_to_dict

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)
XL = dataclasses.replace(XLParams(), kappa_scale=0.15)


def _gpu_traj(ctx, s, v0, nsteps, prec="fp64"):
    ds = DeviceSystem(s.R, s.types, s.box)
    opts = sp2_opts(prec, max_iter=100, tol=1e-12, refine=2)
    st = MDState(ds, v0, s.masses(P), s.n_occ(P), XL.K, opts)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    it = tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    out = {"E": [], "q": [], "n": [], "R": [], "it": it}

    def rec():
        torch.cuda.synchronize()
        out["E"].append(st.energies.cpu().numpy().copy())
        out["q"].append(st.q.cpu().numpy().copy())
        out["n"].append(st.n_current().cpu().numpy().copy())
        out["R"].append(st.R.cpu().numpy().copy())

    rec()
    for _ in range(nsteps):
        tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
        rec()
    out["report"] = report_to_dict(st.report)
    return out


@pytest.mark.parametrize("m,box", [(1, 12.0), (2, 8.0)])
def test_xlbomd_trajectory_matches_oracle(ctx, m, box):
    s = molecular_water(m, box, seed=0)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100)
    nsteps = 40
    g = _gpu_traj(ctx, s, v0, nsteps)
    assert g["it"] >= 0
    o = md.xlbomd(s.R, s.types, s.box, P, XL, v0, M, s.n_occ(P), nsteps, record_R=True)
    Eg = np.array([e[0] for e in g["E"]])
    Eo = np.array(o.E_tot)
    assert np.abs(Eg - Eo).max() < 1e-7
    for k in range(nsteps + 1):
        assert np.abs(g["q"][k] - o.q[k]).max() < 1e-7
        assert np.abs(g["n"][k] - o.n[k]).max() < 1e-7
        assert np.abs(g["R"][k] - o.R[k]).max() < 1e-8
    # energy conservation no worse than the oracle's
    dg = np.abs(Eg - Eg[0]).max()
    do = np.abs(Eo - Eo[0]).max()
    assert dg <= 1.1 * do + 1e-6
    # components: E_tot = E_pot + KE, E_pot = band + scc + pair
    e = g["E"][-1]
    assert e[0] == pytest.approx(e[1] + e[5], rel=1e-12)
    assert e[1] == pytest.approx(e[2] + e[3] + e[4], rel=1e-12)
    assert g["report"]["status"] == tbmd.TB_OK


def test_xlbomd_history_shift_register_matches_eq_verl_n(ctx):
    """After init the whole history equals q; one step applies Eq. Verl_n and
    moves the history down one slot."""
    s = molecular_water(1, 12.0, seed=1)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=7)
    ds = DeviceSystem(s.R, s.types, s.box)
    opts = sp2_opts("fp64", tol=1e-12)
    st = MDState(ds, v0, M, s.n_occ(P), XL.K, opts)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    torch.cuda.synchronize()
    h = st.n_hist.cpu().numpy()
    q0 = st.q.cpu().numpy()
    assert np.abs(h - q0[None, :]).max() < 1e-9
    tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
    torch.cuda.synchronize()
    n1 = st.n_current().cpu().numpy()
    # history = the SCF's last charges, q_t = charges of D[n_t] (equal to 1e-10)
    expect = md.modified_verlet_n([h[0]] * (XL.K + 1), q0, XL)
    assert np.abs(n1 - expect).max() < 1e-13
    h1 = st.n_hist.cpu().numpy()
    assert np.array_equal(h1[1:], h[:-1])
    assert st.energies[7].item() == 1.0
