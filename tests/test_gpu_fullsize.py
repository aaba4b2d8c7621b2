"""Parity at the sizes where the persistent tensor-core kernels run their
multi-round schedules, and the same schedules forced on small matrices.

The projection, Fermi-product and block-sparse kernels launch one CTA per SM
(152 on a GB300) and walk the upper-triangle 128 x 128 tiles (or block-sparse
output blocks) round-robin.  Below 152 tiles every CTA takes one tile, so the
paths that only run above it -- several tiles per CTA, the reuse of the two
TMEM accumulators after their first two tiles, the 64-column half units of a
last round that would be less than half full, and the emulated-FP64 product
at K = 4096 -- are checked here:

* the 2048-atom water-like system (n = 4094: 528 tiles, three rounds plus
  144 half units on 152 CTAs) with tf32x3 products and two FP64-exact
  refinement projections, against the eigh projector of the same H at the
  target ||dD||_F/sqrt(n) <= 1e-6 and |dq| <= 1e-6 e (Sec. III.B, App. D.2);
* the Fermi expansion on a 1200-atom system (n = 2400: 190 tiles);
* the thresholded block-sparse recursion on the Morton-ordered 2048-atom
  system (more than 152 upper super-blocks per product);
* smaller matrices with the grid capped (tb_ctx_set_grid_limit) at 1, 4, 7
  and 10 CTAs, which run 15 / 4 / 2 rounds and the half-unit split on 15
  tiles, compared with the uncapped grid and with eigh;
* the timeout unwind: with a 1 ns pipeline wait limit a projection gives up
  and the report says TB_ERR_TIMEOUT, and the next call on the same context
  with the default limit succeeds.

Each test prints its measured errors on a line starting with PARITY."""

import math

import numpy as np
import pytest
import torch

from workloads import ModelParams, random_gapped_matrix, water_2048_atoms, water_system
from oracle import density, observables, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import (DensitySolver, DeviceSystem, FermiSolver, fermi_opts,
                                          fermi_report_to_dict, report_to_dict, sp2_opts)

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)
SMS = 152


def _H(w):
    return tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                      np.zeros(w.natoms))


def _err(A, B):
    return float(np.linalg.norm(A - B) / np.sqrt(A.shape[0]))


def _upper_tiles(n):
    nt = (n + 127) // 128
    return nt * (nt + 1) // 2


def _sp2(ctx, H, nocc, opts):
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = DensitySolver(ctx, H.shape[0], opts)
    s(Ht, nocc, D)
    torch.cuda.synchronize()
    return D, report_to_dict(s.report)


@pytest.fixture(scope="module")
def water2048():
    w = water_2048_atoms()
    H = _H(w)
    ref = density.density_T0(H, int(w.n_occ(P)))
    return w, H, ref


def test_headline_system_tf32x3_with_emulated_fp64_refinement(ctx, water2048):
    w, H, ref = water2048
    n = H.shape[0]
    assert n == 4094 and _upper_tiles(n) == 528 > 3 * SMS
    assert ref.gap > 1e-3
    D, rep = _sp2(ctx, H, w.n_occ(P), sp2_opts("tf32x3", max_iter=100, tol=1e-10, refine=2, refine_mode="emulated"))
    assert rep["status"] == tbmd.TB_OK, rep
    assert rep["refine_iters"] == 2
    Dg = D.cpu().numpy()
    ds = DeviceSystem(w.R, w.types, w.box)
    q = torch.empty(w.natoms, dtype=torch.float64, device="cuda")
    tbmd.mulliken(ctx, TP, ds.sys, D, q)
    torch.cuda.synchronize()
    qo = observables.mulliken(ref.D, w.types, P)
    eD, eq = _err(Dg, ref.D), float(np.abs(q.cpu().numpy() - qo).max())
    h0 = tb.build_h(w.R, w.types, w.box, P)
    eband = abs(2 * np.sum(h0 * Dg) - 2 * np.sum(h0 * ref.D))
    print(f"PARITY dm_sp2 tf32x3+2oz n=4094: dD={eD:.3e} dq={eq:.3e} dEband={eband:.3e} eV "
          f"iters={rep['iters']}+{rep['refine_iters']} trace-N={rep['trace'] - w.n_occ(P):.2e}")
    assert eD <= 1e-6
    assert eq <= 1e-6
    assert abs(rep["trace"] - w.n_occ(P)) < 1e-6
    # D is a projector that commutes with H (idempotency restored by the refinement)
    assert abs(rep["idem_trace"]) < 1e-6


def test_fermi_expansion_above_one_round(ctx):
    w = water_system(1200, density=1.0, seed=3)
    H = _H(w)
    n = H.shape[0]
    assert _upper_tiles(n) > SMS
    nocc = w.n_occ(P)
    ref = density.density_fermi(H, nocc, 0.1)
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = FermiSolver(ctx, n, fermi_opts("tf32x3"))
    s(Ht, nocc, 0.1, D)
    torch.cuda.synchronize()
    rep = fermi_report_to_dict(s.report)
    Dg = D.cpu().numpy()
    eD = _err(Dg, ref.D)
    eq = float(np.abs(observables.mulliken(Dg, w.types, P) - observables.mulliken(ref.D, w.types, P)).max())
    # mu is unique only up to the gap it sits in: check the canonical condition
    # Tr f(H, mu) = N_occ at the returned mu with the oracle's eigenvalues
    ntr = float(density.fermi_occupations(ref.eps, rep["mu"], 0.1).sum())
    print(f"PARITY dm_fermi tf32x3 n={n}: dD={eD:.3e} dq={eq:.3e} mu-mu_ref={rep['mu'] - ref.mu:.2e} "
          f"N(mu)-N={ntr - nocc:.2e} m={rep['m']} expansions={rep['mu_iters']}")
    assert rep["status"] == tbmd.TB_OK, rep
    assert eD < 2e-6
    assert eq < 2e-6
    assert abs(ntr - nocc) <= 1e-6 + 1e-9 * nocc + 1e-6  # the default tolerance + the trace's FP32 noise


def test_block_sparse_above_one_round(ctx):
    w = water_system(2048, density=1.0, seed=0, morton=True)
    H = _H(w)
    n = H.shape[0]
    nocc = w.n_occ(P)
    tau = 1e-5
    D, rep = _sp2(ctx, H, nocc, sp2_opts("tf32x3", max_iter=100, tau=tau))
    o = density.sp2(H, nocc, tol=1e-9, tau=tau, bs=32)
    assert rep["status"] == tbmd.TB_OK, rep
    # stored 128 x 128 blocks of D (both triangles): the upper ones alone
    # exceed one per SM
    upper = (rep["blocks"] + (n + 127) // 128) // 2
    assert upper > SMS, rep["blocks"]
    Dg = D.cpu().numpy()
    eD = _err(Dg, o.X)
    mism, band = _pattern_mismatch(Dg, o, tau)
    print(f"PARITY dm_sp2 bsr tau=1e-5 n={n}: dD={eD:.3e} blocks={rep['blocks']} "
          f"pattern mismatches={mism} (band {band:.2e}) trace-N={rep['trace'] - nocc:.2e}")
    assert mism == 0
    assert eD < 3e-6


def _pattern_mismatch(Dg, o, tau, bs=32):
    """32 x 32 blocks that are zero on one side only, not counting blocks whose
    norm before the oracle's last drop lies within `band` of tau, where band
    is the largest block-norm difference between the two results (a drop
    decision can only differ where the two norms straddle tau)."""
    n = Dg.shape[0]
    nb = (n + bs - 1) // bs
    pad = np.zeros((nb * bs, nb * bs))
    pad[:n, :n] = Dg
    g = np.sqrt((pad.reshape(nb, bs, nb, bs) ** 2).sum(axis=(1, 3)))
    pad[:n, :n] = o.X
    r = np.sqrt((pad.reshape(nb, bs, nb, bs) ** 2).sum(axis=(1, 3)))
    pad[:n, :n] = Dg - o.X
    d = np.sqrt((pad.reshape(nb, bs, nb, bs) ** 2).sum(axis=(1, 3)))
    both = (g > 0) & (r > 0)
    band = float(d[both].max()) if both.any() else 0.0
    differ = (g == 0) != (r == 0)
    near = np.abs(o.pre_drop_norms - tau) <= band
    print(f"PARITY pattern: {int(differ.sum())} blocks differ in all, {int(near.sum())} of {near.size} "
          f"blocks lie within the band {band:.2e} of tau")
    return int((differ & ~near).sum()), band


@pytest.mark.parametrize("kind", ["tf32x3+refine", "fermi", "bsr"])
def test_guards_above_one_round(ctx, kind):
    """Every output element of D is written inside D at a ragged size whose
    tile grid exceeds one tile per SM (n = 2400: 190 upper tiles)."""
    w = water_system(1200, density=1.0, seed=4, morton=(kind == "bsr"))
    ds = DeviceSystem(w.R, w.types, w.box)
    n = ds.norb
    assert n % 128 != 0 and _upper_tiles(n) > SMS
    H = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Gm = torch.empty(ds.natoms, ds.natoms, dtype=torch.float64, device="cuda")
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, None, H, Gm)
    canary, g = 1.2345678e300, 64
    buf = torch.full((n * n + 2 * g,), canary, dtype=torch.float64, device="cuda")
    D = buf[g:g + n * n].view(n, n)
    nocc = w.n_occ(P)
    if kind == "fermi":
        FermiSolver(ctx, n, fermi_opts("tf32x3"))(H, nocc, 0.1, D)
    else:
        opts = sp2_opts("tf32x3", max_iter=100, refine=2) if kind != "bsr" else \
            sp2_opts("tf32x3", max_iter=100, tau=1e-5)
        DensitySolver(ctx, n, opts)(H, nocc, D)
    torch.cuda.synchronize()
    assert bool((buf[:g] == canary).all()) and bool((buf[g + n * n:] == canary).all())
    assert bool(torch.isfinite(D).all())
    # dm_fermi stops at |Tr D - N_occ| <= 1e-6 + 1e-9 N_occ (its default trace
    # tolerance); the thresholded recursion's trace moves with the dropped blocks
    bound = {"bsr": 1e-2, "fermi": 1e-6 + 1e-9 * nocc + 1e-6}.get(kind, 1e-5)
    assert abs(torch.trace(D).item() - nocc) <= bound


@pytest.fixture()
def grid_limit(ctx):
    def set_limit(g):
        tbmd.tb_ctx_set_grid_limit(ctx, g)
    yield set_limit
    tbmd.tb_ctx_set_grid_limit(ctx, 0)


@pytest.mark.parametrize("limit", [1, 4, 7, 10])
def test_capped_grid_runs_the_multi_round_schedule(ctx, grid_limit, limit):
    """n = 600 (ld = 640, 15 upper tiles).  1 CTA: 15 rounds through both
    TMEM accumulators; 4: 3 full rounds and 3 tiles; 7: 2 rounds and the last
    tile split into 2 halves; 10: 1 round and 5 tiles as 10 halves.  The tiles
    are the same products in the same order, so D is bitwise the uncapped
    result whenever the branch sequence is the same (the trace partials are
    summed in another grouping, which could only move a near tie)."""
    w = water_system(300, density=1.0, seed=0)
    H = _H(w)
    nocc = w.n_occ(P)
    ref = density.density_T0(H, int(nocc))
    opts = sp2_opts("tf32x3", max_iter=100, refine=2)
    D0, r0 = _sp2(ctx, H, nocc, opts)
    grid_limit(limit)
    D1, r1 = _sp2(ctx, H, nocc, opts)
    e = _err(D1.cpu().numpy(), ref.D)
    print(f"PARITY capped grid {limit}: dD={e:.3e} same branches={r0['branches'] == r1['branches']}")
    assert r1["status"] == tbmd.TB_OK
    assert e < 1e-6
    if r0["branches"] == r1["branches"] and r0["refine_branches"] == r1["refine_branches"]:
        assert torch.equal(D0, D1)


def test_capped_grid_fermi_and_block_sparse(ctx, grid_limit):
    w = water_system(300, density=1.0, seed=5)
    H = _H(w)
    nocc = w.n_occ(P)
    ref = density.density_fermi(H, nocc, 0.1)
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    grid_limit(7)
    s = FermiSolver(ctx, H.shape[0], fermi_opts("tf32x3"))
    s(Ht, nocc, 0.1, D)
    torch.cuda.synchronize()
    rep = fermi_report_to_dict(s.report)
    eF = _err(D.cpu().numpy(), ref.D)
    assert rep["status"] == tbmd.TB_OK and eF < 2e-6
    wm = water_system(600, density=1.0, seed=1, morton=True)
    Hm = _H(wm)
    grid_limit(5)
    Db, rb = _sp2(ctx, Hm, wm.n_occ(P), sp2_opts("tf32x3", max_iter=100, tau=1e-5))
    o = density.sp2(Hm, wm.n_occ(P), tol=1e-9, tau=1e-5, bs=32)
    eB = _err(Db.cpu().numpy(), o.X)
    mism, band = _pattern_mismatch(Db.cpu().numpy(), o, 1e-5)
    print(f"PARITY capped grid fermi(7): dD={eF:.3e}; bsr(5): dD={eB:.3e} mismatches={mism}")
    assert rb["status"] == tbmd.TB_OK and eB < 3e-6 and mism == 0


def test_timeout_unwinds_and_the_context_stays_usable(ctx):
    """A 1 ns limit on the pipeline waits: the first projection's epilogue
    cannot see its accumulator within it, so the kernel stops its pipeline,
    waits for its own copies and MMAs, frees TMEM and returns; every later
    launch of the call returns at once and the report says TB_ERR_TIMEOUT.
    With the default limit restored the same call on the same context and
    workspace succeeds."""
    H, _ = random_gapped_matrix(256, 100, gap=2.0, width=20.0, seed=12)
    ref = density.density_T0(H, 100)
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = DensitySolver(ctx, 256, sp2_opts("tf32", max_iter=100, refine=0))
    try:
        tbmd.tb_ctx_set_wait_limit(ctx, 1)
        s(Ht, 100.0, D)
        torch.cuda.synchronize()
        rep = report_to_dict(s.report)
    finally:
        tbmd.tb_ctx_set_wait_limit(ctx, 2_000_000_000)
    assert rep["status"] == tbmd.TB_ERR_TIMEOUT, rep
    s(Ht, 100.0, D)
    torch.cuda.synchronize()
    rep2 = report_to_dict(s.report)
    e = _err(D.cpu().numpy(), ref.D)
    print(f"PARITY timeout: first status {rep['status']}, then {rep2['status']} dD={e:.3e}")
    assert rep2["status"] == tbmd.TB_OK
    assert e < 5e-3
