"""Finite-temperature XL-BOMD steps through CUDA graphs and the serving
runtime (tb_server): continuous batching of step requests from trajectories
of uneven size, admission by device-memory footprint.

Parity: a finite-T trajectory (D by dm_fermi at kT = 0.1 eV, tf32x3
products) against the oracle's XL-BOMD with the diagonalised Fermi-Dirac
density matrix.  The FOE leaves ~1e-6 absolute error in D, so charges agree to
~1e-6 e per step and the positions, which feel them only through the forces,
much closer; the energy error is ~1e-6 eV per atom (2 Tr[hD] sums the D
error against h).  Alone vs in the mix: each trajectory's kernels see the same
inputs in the same order whatever else runs, so R, v, q and n are bitwise
equal; the energy sums use FP64 atomics, so they are compared to 1e-9 eV."""

import dataclasses

import numpy as np
import pytest
import torch

from workloads import ModelParams, XLParams, molecular_water, thermal_velocities
from oracle import md
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import (DeviceSystem, MDState, Server, fermi_opts, sp2_opts, xl_params)

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)
XL = dataclasses.replace(XLParams(), kappa_scale=0.15)
KT = 0.1


def _xp():
    return xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)


def _system(m, box, seed):
    s = molecular_water(m, box, seed=seed)
    M = s.masses(P)
    return s, M, thermal_velocities(M, 300.0, seed=100 + seed)


def _md_state(s, M, v0):
    ds = DeviceSystem(s.R, s.types, s.box)
    opts = sp2_opts("tf32x3", refine=3)
    return MDState(ds, v0, M, s.n_occ(P), XL.K, opts, kT=KT, fermi=fermi_opts()), opts


def test_finite_temperature_step_graph_replays_as_direct_steps(ctx):
    """One captured step (dm_fermi's mu loop as a while node) replayed k times
    gives the bitwise state of k direct xlbomd_step calls."""
    s, M, v0 = _system(2, 8.0, seed=0)
    xp = _xp()
    a, opts = _md_state(s, M, v0)
    b, _ = _md_state(s, M, v0)
    for st in (a, b):
        tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    k = 6
    for _ in range(k):
        tbmd.xlbomd_step(ctx, TP, a.st, xp, opts)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            tbmd.xlbomd_step(ctx, TP, b.st, xp, opts, stream=side)
    for _ in range(k):
        g.replay()
    torch.cuda.synchronize()
    for name in ("R", "v", "q", "n_hist", "mu"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name
    assert b.energies[7].item() == k
    assert abs(a.energies[1].item() - b.energies[1].item()) < 1e-9


def test_finite_temperature_trajectory_matches_oracle(ctx):
    s, M, v0 = _system(2, 8.0, seed=1)
    nsteps = 20
    st, opts = _md_state(s, M, v0)
    xp = _xp()
    tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-10, 300)
    o = md.xlbomd(s.R, s.types, s.box, P, XL, v0, M, s.n_occ(P), nsteps, kT=KT, record_R=True)
    worst = [0.0, 0.0, 0.0]
    for k in range(nsteps + 1):
        if k:
            tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
        torch.cuda.synchronize()
        worst = [max(worst[0], float(np.abs(st.q.cpu().numpy() - o.q[k]).max())),
                 max(worst[1], float(np.abs(st.R.cpu().numpy() - o.R[k]).max())),
                 max(worst[2], abs(st.energies[1].item() - o.E_pot[k]))]
        # the expansion's tf32x3 products leave q ~1e-7 from the oracle's
        # Fermi-Dirac charges (bounded here by 1e-5); the force difference that
        # causes (~ dq x 4 eV/A per e) moves an H atom by dF t^2 / 2M after 20
        # steps of 0.25 fs: 5e-7 A for dq = 1e-6
        assert np.abs(st.q.cpu().numpy() - o.q[k]).max() < 1e-5, k
        assert np.abs(st.R.cpu().numpy() - o.R[k]).max() < 5e-7, k
        assert st.energies[1].item() == pytest.approx(o.E_pot[k], abs=2e-6 * s.natoms)
    print(f"PARITY finite-T trajectory: dq max {worst[0]:.3e} dR max {worst[1]:.3e} dEpot max {worst[2]:.3e}")
    rep = tbmd.tb_fermi_report.from_buffer_copy(st.fermi_report.cpu().numpy().tobytes())
    assert rep.status == tbmd.TB_OK and rep.mu_iters >= 1


def _add(sv, s, M, v0):
    return sv.add(s.types, s.box, s.R, v0, M, s.n_occ(P))


MIX = [(1, 12.0, 0), (3, 9.0, 1), (2, 8.0, 2), (4, 12.0, 3), (1, 10.0, 4)]


def test_server_same_alone_and_in_the_mix(ctx):
    k = 5
    systems = [_system(*x) for x in MIX]
    mix = Server(ctx, TP, _xp(), kT=KT, max_slots=4)
    ids = [_add(mix, *x) for x in systems]
    for _ in range(k):  # interleaved requests: steps of different trajectories overlap
        for t in ids:
            mix.submit(t)
    done = mix.drain()
    assert len(done) == k * len(ids)
    assert all(c.status == tbmd.TB_OK for c in done)
    for t in ids:  # each trajectory's steps complete in order
        assert [c.step for c in done if c.traj == t] == list(range(1, k + 1))
    for j in (0, 1, 3):
        alone = Server(ctx, TP, _xp(), kT=KT, max_slots=1)
        t = _add(alone, *systems[j])
        for _ in range(k):
            alone.submit(t)
        alone.drain()
        x, y = alone.read(t), mix.read(ids[j])
        for name in ("R", "v", "q", "n"):
            assert np.array_equal(x[name], y[name]), (j, name)
        assert np.abs(x["E"] - y["E"]).max() < 1e-9
        alone.close()
    mix.close()


def test_server_trajectory_matches_oracle(ctx):
    s, M, v0 = systems = _system(2, 8.0, seed=1)
    nsteps = 10
    sv = Server(ctx, TP, _xp(), kT=KT, max_slots=2, scf_tol=1e-10, scf_max_iter=300)
    t = _add(sv, *systems)
    for _ in range(nsteps):
        sv.submit(t)
    E = [c.energies[1] for c in sorted(sv.drain(), key=lambda c: c.step)]
    o = md.xlbomd(s.R, s.types, s.box, P, XL, v0, M, s.n_occ(P), nsteps, kT=KT, record_R=True)
    r = sv.read(t)
    assert np.abs(r["q"] - o.q[-1]).max() < 1e-5
    assert np.abs(r["R"] - o.R[-1]).max() < 1e-7
    assert np.abs(np.array(E) - np.array(o.E_pot[1:])).max() < 2e-6 * s.natoms
    sv.close()


def test_server_admission_by_footprint(ctx):
    """A budget that holds two of three trajectories: the third waits until a
    retired one frees its memory, then runs its queued steps."""
    systems = [_system(*x) for x in MIX[:3]]
    probe = Server(ctx, TP, _xp(), kT=KT, max_slots=2, hbm_budget=1 << 40)
    fp = [probe.footprint(x[0].types) for x in systems]
    probe.close()
    budget = fp[0] + fp[1] + min(fp[2], fp[0]) // 2
    assert fp[2] > budget - fp[0] - fp[1]
    sv = Server(ctx, TP, _xp(), kT=KT, max_slots=2, hbm_budget=budget)
    ids = [_add(sv, *x) for x in systems]
    st = sv.stats()
    assert st["admitted"] == 2 and st["waiting"] == 1 and st["bytes_in_use"] == fp[0] + fp[1]
    for t in ids:
        for _ in range(2):
            sv.submit(t)
    first = []
    while sv.stats()["queued"] > 2 or sv.stats()["running"] > 0:
        first += sv.poll(wait=True)
        assert sv.stats()["bytes_in_use"] <= budget
    assert {c.traj for c in first} == {ids[0], ids[1]}
    assert sv.stats()["queued"] == 2  # the waiting trajectory's requests
    sv.retire(ids[0])
    rest = sv.drain()
    assert sorted(c.step for c in rest if c.traj == ids[2]) == [1, 2]
    st = sv.stats()
    assert st["waiting"] == 0 and st["bytes_in_use"] == fp[1] + fp[2] <= budget
    with pytest.raises(tbmd.TBError):
        sv.submit(ids[0])  # retired
    sv.close()


def test_server_replays_a_poisson_trace(ctx):
    systems = [_system(*x) for x in MIX[:4]]
    sv = Server(ctx, TP, _xp(), kT=KT, max_slots=4)
    ids = [_add(sv, *x) for x in systems]
    rng = np.random.default_rng(6)
    arrivals = np.cumsum(rng.exponential(1.0 / 2000.0, size=40))
    which = rng.integers(0, len(ids), size=40)
    out = sv.replay(arrivals, which)
    assert len(out) == 40
    per = {t: [] for t in ids}
    for i, c in enumerate(out):
        assert c.traj == which[i] and c.status == tbmd.TB_OK
        assert c.t_submit <= c.t_launch <= c.t_done and c.gpu_ms > 0.0
        per[c.traj].append(c.step)
    for t, steps in per.items():
        assert steps == list(range(1, len(steps) + 1))
    sv.close()


def test_server_requests_of_a_trajectory_that_cannot_be_admitted(ctx):
    """A budget that admits one of two trajectories, requests for both: drain
    returns the admitted one's steps and stops with the other's still queued
    (nothing running can free memory for it); a replay that names it is
    rejected instead of waiting forever; once the first retires, the second is
    admitted and its queued steps run."""
    systems = [_system(*x) for x in MIX[:2]]
    probe = Server(ctx, TP, _xp(), kT=KT, max_slots=2, hbm_budget=1 << 40)
    fp = [probe.footprint(x[0].types) for x in systems]
    probe.close()
    sv = Server(ctx, TP, _xp(), kT=KT, max_slots=2, hbm_budget=max(fp) + min(fp) // 2)
    ids = [_add(sv, *x) for x in systems]
    assert sv.stats()["admitted"] == 1 and sv.stats()["waiting"] == 1
    for t in ids:
        sv.submit(t)
        sv.submit(t)
    done = sv.drain()
    assert sorted(c.step for c in done) == [1, 2] and {c.traj for c in done} == {ids[0]}
    assert sv.stats()["queued"] == 2
    with pytest.raises(tbmd.TBError):
        sv.replay([0.0, 0.001], [ids[0], ids[1]])
    sv.retire(ids[0])
    rest = sv.drain()
    assert sorted(c.step for c in rest if c.traj == ids[1]) == [1, 2]
    assert all(c.status == tbmd.TB_OK for c in rest)
    sv.close()
