"""dm_sp2_grouped: many independent SP2 problems of uneven size in one
persistent launch, against the oracle's eigh density matrix of every system.

The grouped path runs the tensor-core phase only (tf32x3 products, FP32
storage, no FP64 refinement), so D is held to the accuracy that phase reaches
on these water-like systems (~1e-6 per sqrt(n); the dense path's own test
shows the same).  A system gives the bitwise same D alone and inside the
batch (one CTA owns it, same arithmetic in the same order), and the run call
replays inside a captured CUDA graph."""

import numpy as np
import pytest
import torch

from workloads import water_system, batch_sizes, ModelParams
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import Workspace, sp2_opts, report_to_dict

pytestmark = pytest.mark.gpu
P = ModelParams()


def _batch(count, seed=4):
    sizes = batch_sizes(count=count, lo=16, hi=256, seed=seed)
    Hs, nocc = [], []
    for i, N in enumerate(sizes):
        w = water_system(int(N), density=1.0, seed=1000 + i)
        Hs.append(tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                             np.zeros(w.natoms)))
        nocc.append(w.n_occ(P))
    return Hs, nocc


def _solve(ctx, Hs, nocc, autotune=False, prec="tf32x3"):
    opts = sp2_opts(prec, max_iter=100)
    n = [H.shape[0] for H in Hs]
    Ht = [torch.as_tensor(H, device="cuda") for H in Hs]
    Dt = [torch.empty_like(h) for h in Ht]
    rep = torch.zeros(len(Hs), ctypes_size(), dtype=torch.uint8, device="cuda")
    ws = Workspace(tbmd.dm_sp2_grouped_workspace_size(n, opts))
    tbmd.dm_sp2_grouped_plan(ctx, n, nocc, Ht, Dt, rep, opts, autotune, ws.ptr, ws.nbytes)
    cfg = tbmd.dm_sp2_grouped_run(ctx, ws.ptr)
    torch.cuda.synchronize()
    return Ht, Dt, rep, ws, cfg


def ctypes_size():
    import ctypes
    return ctypes.sizeof(tbmd.tb_sp2_report)


@pytest.mark.parametrize("mode", [1, 3, 4, 5, 8])
def test_grouped_batch_matches_eigh(ctx, mode):
    """mode 1: autotuned launch form; 3: the FP32-staged form; 4 / 8 / 5:
    clusters of 4 / 8 / 2 CTAs per system."""
    Hs, nocc = _batch(40)
    Ht, Dt, rep, ws, cfg = _solve(ctx, Hs, nocc, autotune=mode)
    cs, bn = cfg // 10 ** 7, (cfg // 10 ** 4) % 1000
    assert bn in (0, 64, 128) and cs in (1, 2, 4, 8)
    if mode == 3:
        assert bn == 0 and cs == 1
    elif mode > 1:
        assert cs == (2 if mode == 5 else mode)
    errs = []
    for i, H in enumerate(Hs):
        r = report_to_dict(rep[i])
        ref = density.density_T0(H, int(nocc[i]))
        err = np.linalg.norm(Dt[i].cpu().numpy() - ref.D) / np.sqrt(H.shape[0])
        errs.append(err)
        assert r["status"] == tbmd.TB_OK, (i, r)
        assert abs(r["trace"] - nocc[i]) < 5e-4
        assert err < 2e-5, (i, H.shape[0], err, ref.gap)
    print(f"PARITY grouped mode {mode}: dD max {max(errs):.3e} median {np.median(errs):.3e}")
    assert np.median(errs) < 3e-6


@pytest.mark.parametrize("mode", [0, 2, 4])
def test_grouped_same_alone_and_in_the_mix(ctx, mode):
    Hs, nocc = _batch(24, seed=9)
    _, Dall, _, _, _ = _solve(ctx, Hs, nocc, autotune=mode)
    for j in (0, 7, 23):
        _, Done, _, _, _ = _solve(ctx, [Hs[j]], [nocc[j]], autotune=mode)
        assert torch.equal(Done[0], Dall[j])


def test_fp32_staged_form_is_bitwise_the_stored_split_form(ctx):
    """The converter warps split the FP32 X in shared memory exactly as the
    stored-split form's epilogue splits it before storing (same rounding of
    the same FP32 values), and the MMAs, their order and the epilogue
    arithmetic are the same: D and every report are bitwise equal."""
    Hs, nocc = _batch(40, seed=5)
    _, D0, r0, _, cfg0 = _solve(ctx, Hs, nocc, autotune=2)
    _, D3, r3, _, cfg = _solve(ctx, Hs, nocc, autotune=3)
    assert (cfg0 // 10 ** 4) % 1000 == 128
    assert (cfg // 10 ** 4) % 1000 == 0
    for a, b in zip(D0, D3):
        assert torch.equal(a, b)
    assert torch.equal(r0, r3)


@pytest.mark.parametrize("mode", [0, 3, 8])
def test_grouped_run_replays_in_a_cuda_graph(ctx, mode):
    Hs, nocc = _batch(16, seed=11)
    Ht, Dt, rep, ws, cfg = _solve(ctx, Hs, nocc, autotune=mode)
    first = [d.clone() for d in Dt]
    for d in Dt:
        d.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            tbmd.dm_sp2_grouped_run(ctx, ws.ptr, stream=s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(first, Dt):
        assert torch.equal(a, b)
