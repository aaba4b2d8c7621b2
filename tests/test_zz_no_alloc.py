"""dm_sp2_static: the allocation-free FP64 SP2 entry point, for callers that
cannot allocate device memory when they need a density matrix (engines that
reserve all memory up front, plugins whose host owns the allocator, code
avoiding the synchronisation of cudaMalloc).  It must give what dm_sp2 gives
on the FP64 path, call after call, although every call reuses one static
scratch array.  This file is collected last on purpose."""

import numpy as np
import pytest
import torch

from workloads import random_gapped_matrix, water_system, ModelParams
from oracle import tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, sp2_opts, new_report, report_to_dict

pytestmark = pytest.mark.gpu


def _reference(ctx, H, nocc, opts):
    D = torch.empty_like(H)
    DensitySolver(ctx, H.shape[0], opts)(H, nocc, D)
    return D


def test_static_scratch_matches_dm_sp2_on_consecutive_calls(ctx):
    P = ModelParams()
    opts = sp2_opts("fp64", max_iter=100, tol=1e-11)
    w = water_system(150, density=1.0, seed=3)
    Hw = tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                    np.zeros(w.natoms))
    Hr, _ = random_gapped_matrix(511, 200, gap=0.5, width=30.0, seed=12)
    # n = 512: the largest size the static scratch holds (its largest layout)
    Hm, _ = random_gapped_matrix(tbmd.SP2_STATIC_MAX_N, 240, gap=0.5, width=30.0, seed=13)
    cases = [(torch.as_tensor(Hw, device="cuda"), w.n_occ(P)), (torch.as_tensor(Hr, device="cuda"), 200.0),
             (torch.as_tensor(Hm, device="cuda"), 240.0)]
    for H, nocc in cases + cases:          # two calls in a row, then again
        D = torch.full_like(H, float("nan"))
        rep = new_report()
        tbmd.dm_sp2_static(ctx, H, H.shape[0], nocc, opts, D, rep)
        Dref = _reference(ctx, H, nocc, opts)
        torch.cuda.synchronize()
        r = report_to_dict(rep)
        assert r["status"] == tbmd.TB_OK
        assert abs(r["trace"] - nocc) < 1e-9
        assert torch.isfinite(D).all()
        assert (D - Dref).abs().max().item() < 1e-12


def test_static_scratch_rejects_oversize_and_other_precisions(ctx):
    n = tbmd.SP2_STATIC_MAX_N + 1
    H = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    D = torch.empty_like(H)
    with pytest.raises(tbmd.TBError) as e:
        tbmd.dm_sp2_static(ctx, H, n, 10.0, sp2_opts("fp64"), D)
    assert e.value.code == tbmd.TB_ERR_ARG and "static scratch" in str(e.value)
    with pytest.raises(tbmd.TBError) as e:
        tbmd.dm_sp2_static(ctx, H[:64, :64].contiguous(), 64, 10.0, sp2_opts("tf32x3"), D)
    assert e.value.code == tbmd.TB_ERR_UNSUPPORTED
