"""The CTA-pair form of the dense tensor-core projection (tcgen05.mma
cta_group::2, 256 x 256 tiles) against the single-CTA form and the oracle.

dm_sp2 picks the pair form by itself only for ld = 4096 and up (the
full-size tests cover it there); here it is forced (tb_ctx_set_sp2_form) at
n = 1000 (ld = 1024: ten 256 x 256 tiles of the upper triangle, four of them
on the diagonal, with a ragged tail of 24 padded rows) and run on the whole
GPU, on four clusters (two rounds, the last as 256 x 128 halves) and on one
cluster (ten tiles in a row: both TMEM accumulators recycled).

Both forms issue the same MMAs over the same k-slices in the same order, so
the tensor-core iterates agree to the FP32 rounding of the accumulators and
the branch sequences are the same; after the FP64 refinement D of the two
forms agree to 1e-9.  Against eigh, tf32x3 meets the 1e-6 target; bf16x3
(hi + lo bf16 splits, ~2^-16 per product) is held to 5e-6 (1.5e-6 measured
at n = 1000 in both forms), as the bf16x3 Fermi products are."""

import numpy as np
import pytest
import torch

from workloads import ModelParams, random_gapped_matrix, water_system
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, report_to_dict, sp2_opts

pytestmark = pytest.mark.gpu
P = ModelParams()


def _water_H(natoms, seed):
    s = water_system(natoms, density=1.0, seed=seed)
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types,
                   np.zeros(s.natoms))
    return H, s.n_occ(P)


@pytest.fixture
def form(ctx):
    def set_form(f, limit=0):
        tbmd.tb_ctx_set_sp2_form(ctx, f)
        tbmd.tb_ctx_set_grid_limit(ctx, limit)
    yield set_form
    tbmd.tb_ctx_set_sp2_form(ctx, tbmd.TB_SP2_FORM_AUTO)
    tbmd.tb_ctx_set_grid_limit(ctx, 0)


def _solve(ctx, H, nocc, prec):
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = DensitySolver(ctx, H.shape[0], sp2_opts(prec, refine=2))
    s(Ht, nocc, D)
    torch.cuda.synchronize()
    return D.cpu().numpy(), report_to_dict(s.report)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("limit", [0, 8, 2])
def test_pair_form_matches_single_form_and_oracle(ctx, form, prec, limit):
    H, nocc = _water_H(502, 7)
    n = H.shape[0]
    assert n == 1000
    ref = density.density_T0(H, int(nocc))
    form(tbmd.TB_SP2_FORM_SINGLE, limit)
    D1, r1 = _solve(ctx, H, nocc, prec)
    form(tbmd.TB_SP2_FORM_PAIRS, limit)
    D2, r2 = _solve(ctx, H, nocc, prec)
    e1 = np.linalg.norm(D1 - ref.D) / np.sqrt(n)
    e2 = np.linalg.norm(D2 - ref.D) / np.sqrt(n)
    d12 = float(np.abs(D1 - D2).max())
    print(f"PARITY sp2 pairs {prec} n={n} grid limit {limit}: dD pair {e2:.3e} single {e1:.3e}, "
          f"max|D_pair - D_single| {d12:.3e} (bitwise {d12 == 0.0}), iters {r2['iters']}/{r1['iters']}")
    assert r1["status"] == r2["status"] == tbmd.TB_OK
    assert r2["branches"] == r1["branches"]
    assert d12 < 1e-9
    bound = 1e-6 if prec == "tf32x3" else 5e-6
    assert e2 < bound and e1 < bound
    assert abs(r2["trace"] - nocc) < 1e-8


def test_pair_form_on_a_random_spectrum(ctx, form):
    """A dense random H (Gershgorin bounds ~10x its spectrum) with n = 1024
    (no padding): the pair form against eigh, held like the single form's
    x3 paths on random matrices (2e-4, see test_gpu_sp2)."""
    H, _ = random_gapped_matrix(1024, 400, gap=0.5, width=20.0, seed=21)
    ref = density.density_T0(H, 400)
    form(tbmd.TB_SP2_FORM_PAIRS)
    D, r = _solve(ctx, H, 400.0, "tf32x3")
    e = np.linalg.norm(D - ref.D) / np.sqrt(1024)
    print(f"PARITY sp2 pairs random n=1024: dD={e:.3e} iters {r['iters']}")
    assert r["status"] == tbmd.TB_OK and e < 2e-4


def test_pair_form_timeout_unwinds(ctx, form):
    """A 1 ns pipeline wait limit on the pair form: the pair stops, both CTAs
    settle their copies, free the pair's TMEM and meet at the final cluster
    barrier; the report says TB_ERR_TIMEOUT and the next call succeeds."""
    H, _ = random_gapped_matrix(512, 200, gap=2.0, width=20.0, seed=12)
    ref = density.density_T0(H, 200)
    form(tbmd.TB_SP2_FORM_PAIRS)
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = DensitySolver(ctx, 512, sp2_opts("tf32", max_iter=100, refine=0))
    try:
        tbmd.tb_ctx_set_wait_limit(ctx, 1)
        s(Ht, 200.0, D)
        torch.cuda.synchronize()
        rep = report_to_dict(s.report)
    finally:
        tbmd.tb_ctx_set_wait_limit(ctx, 2_000_000_000)
    assert rep["status"] == tbmd.TB_ERR_TIMEOUT, rep
    s(Ht, 200.0, D)
    torch.cuda.synchronize()
    rep2 = report_to_dict(s.report)
    e = np.linalg.norm(D.cpu().numpy() - ref.D) / np.sqrt(512)
    print(f"PARITY pair timeout: first status {rep['status']}, then {rep2['status']} dD={e:.3e}")
    assert rep2["status"] == tbmd.TB_OK
    assert e < 5e-3


def test_form_knob_rejects_unknown_forms(ctx):
    with pytest.raises(tbmd.TBError):
        tbmd.tb_ctx_set_sp2_form(ctx, 3)
