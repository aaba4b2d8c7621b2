"""dm_sp2 on the GPU against the oracle's density matrices (eigh of the same
H, plain definition D = theta(mu0 I - H)) and its SP2 recursion.

Tolerances: the FP64 path stops at |Tr X - Tr X^2| <= 1e-11, which bounds
the distance to the projector by ~1e-11 per eigenvalue, so ||dD||_F/sqrt(n)
<= 1e-9 leaves room for rounding.

The tensor-core paths: an error e in the product of an early projection,
while the HOMO-LUMO separation of X is still delta (in units of the
Gershgorin width), rotates occupied into virtual states by ~e/delta, and the
FP64 refinement (which restores idempotency and the trace) cannot undo a
rotation.  On the water-like Hamiltonians (Gershgorin width ~15 eV,
gap 3.4 eV) the x3 splits (product error ~2^-22) are held to the target
||dD||_F/sqrt(n) <= 1e-6.  Dense random test matrices have Gershgorin bounds
~10x wider than their spectra, so the same splits are held to 2e-4 there,
and single-pass tf32 / bf16 (product error 2^-11 / 2^-8) to 5e-3 / 5e-2.
"""

import numpy as np
import pytest
import torch

from workloads import random_gapped_matrix, water_system, ModelParams, water_24_atoms
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, sp2_opts, report_to_dict

pytestmark = pytest.mark.gpu
P = ModelParams()


def _run(ctx, H: np.ndarray, nocc: float, prec="fp64", refine=2, tol=1e-11, max_iter=100, rule=0):
    n = H.shape[0]
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    solver = DensitySolver(ctx, n, sp2_opts(prec, max_iter=max_iter, tol=tol, refine=refine, rule=rule))
    solver(Ht, nocc, D)
    torch.cuda.synchronize()
    return D.cpu().numpy(), report_to_dict(solver.report)


def _err(D, Dref):
    return np.linalg.norm(D - Dref) / np.sqrt(D.shape[0])


def test_two_level_and_ring_closed_forms(ctx):
    a, ap, b = -1.3, 0.7, 0.45
    H = np.array([[a, b], [b, ap]])
    rad = np.sqrt(((a - ap) / 2) ** 2 + b * b)
    D_ref = 0.5 * (np.eye(2) - (H - 0.5 * (a + ap) * np.eye(2)) / rad)
    D, rep = _run(ctx, H, 1.0, tol=1e-14)
    assert rep["status"] == tbmd.TB_OK
    assert np.abs(D - D_ref).max() < 1e-12
    t = 1.7
    H = np.zeros((6, 6))
    for i in range(6):
        H[i, (i + 1) % 6] = H[(i + 1) % 6, i] = -t
    idx = np.arange(6)
    diff = idx[:, None] - idx[None, :]
    D_ref = sum(np.cos(2 * np.pi * k * diff / 6) for k in (0, 1, -1)) / 6
    D, rep = _run(ctx, H, 3.0, tol=1e-14)
    assert np.abs(D - D_ref).max() < 1e-11


def test_diagonal_and_edge_occupations(ctx):
    e = np.array([3.0, -1.0, 0.5, -2.0, 7.0, 0.1])
    D, rep = _run(ctx, np.diag(e), 3.0)
    assert np.abs(D - np.diag([0, 1, 0, 1, 0, 1.0])).max() < 1e-9
    H, _ = random_gapped_matrix(50, 20, seed=3)
    D, rep = _run(ctx, H, 0.0)
    assert np.abs(D).max() < 1e-9
    D, rep = _run(ctx, H, 50.0)
    assert np.abs(D - np.eye(50)).max() < 1e-9


@pytest.mark.parametrize("n,nocc,seed", [(37, 11, 0), (64, 40, 1), (130, 51, 2), (300, 120, 3), (513, 200, 4)])
def test_fp64_matches_eigh_and_oracle_recursion(ctx, n, nocc, seed):
    H, _ = random_gapped_matrix(n, nocc, gap=0.5, width=30.0, seed=seed)
    ref = density.density_T0(H, nocc)
    D, rep = _run(ctx, H, nocc, tol=1e-11)
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 1e-9
    assert abs(rep["trace"] - nocc) < 1e-9
    lo, hi = density.gershgorin(H)
    assert rep["eps_min"] == pytest.approx(lo, rel=1e-12)
    assert rep["eps_max"] == pytest.approx(hi, rel=1e-12)
    # same projections as the oracle's SP2 recursion
    o = density.sp2(H, nocc, tol=1e-11)
    assert rep["iters"] == o.iters
    assert rep["branches"] == o.branches


def test_fp64_simple_rule_and_not_converged_status(ctx):
    H, _ = random_gapped_matrix(90, 33, gap=0.3, width=20.0, seed=7)
    ref = density.density_T0(H, 33)
    D, rep = _run(ctx, H, 33, rule=1)
    assert _err(D, ref.D) < 1e-9
    o = density.sp2(H, 33, tol=1e-11, rule="simple")
    assert rep["branches"] == o.branches
    D, rep = _run(ctx, H, 33, max_iter=3)
    assert rep["status"] == tbmd.TB_ERR_NOT_CONVERGED
    assert rep["iters"] == 3


def test_fp64_water_hamiltonian(ctx):
    s = water_24_atoms()
    h = tb.build_h(s.R, s.types, s.box, P)
    G = tb.build_gamma(s.R, s.box, P)
    rng = np.random.default_rng(11)
    n_aux = rng.normal(0, 0.3, s.natoms)
    n_aux -= n_aux.mean()
    H = tb.build_H(h, G, s.types, n_aux)
    nocc = s.n_occ(P)
    ref = density.density_T0(H, int(nocc))
    D, rep = _run(ctx, H, nocc, tol=1e-12, max_iter=120)
    assert ref.gap > 1e-5
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 1e-8


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,nocc,seed", [(200, 70, 0), (600, 260, 1), (1000, 333, 2)])
def test_tensor_core_split_paths_dense_random(ctx, prec, n, nocc, seed):
    H, eps = random_gapped_matrix(n, nocc, gap=2.0, width=30.0, seed=seed)
    ref = density.density_T0(H, nocc)
    D, rep = _run(ctx, H, nocc, prec=prec, refine=3)
    lo, hi = density.gershgorin(H)
    print(f"PARITY sp2 {prec} random n={n}: dD={_err(D, ref.D):.3e} trace-N={rep['trace'] - nocc:.2e} "
          f"delta0={ref.gap / (hi - lo):.2e}")
    assert rep["status"] == tbmd.TB_OK, rep
    assert rep["refine_iters"] >= 2
    assert _err(D, ref.D) < 2e-4, (_err(D, ref.D), rep)
    assert abs(rep["trace"] - nocc) < 1e-5


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("bf16", 5e-2)])
def test_tensor_core_single_pass_paths(ctx, prec, tol):
    H, eps = random_gapped_matrix(384, 150, gap=2.0, width=30.0, seed=5)
    ref = density.density_T0(H, 150)
    D, rep = _run(ctx, H, 150, prec=prec, refine=4)
    assert _err(D, ref.D) < tol
    assert abs(rep["trace"] - 150) < 0.25


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("natoms", [300, 600])
def test_tensor_core_water_system_meets_target(ctx, prec, natoms):
    """Water-like systems with neutral charges (n = 600 / 1200: several
    128-tiles and a ragged tail) at the target 1e-6."""
    s = water_system(natoms, density=1.0, seed=0)
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types,
                   np.zeros(s.natoms))
    nocc = s.n_occ(P)
    ref = density.density_T0(H, int(nocc))
    D, rep = _run(ctx, H, nocc, prec=prec, refine=3)
    print(f"PARITY sp2 {prec} water {natoms}: dD={_err(D, ref.D):.3e} trace-N={rep['trace'] - nocc:.2e}")
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 1e-6
    assert abs(rep["trace"] - nocc) < 1e-6


@pytest.mark.parametrize("natoms", [300, 600])
def test_emulated_fp64_refinement_matches_fma_refinement(ctx, natoms):
    """The refinement projections on the tensor cores (exact integer slices,
    FP64 result) agree with FP64 FMA projections to far below the target:
    both start from the same tensor-core iterate and apply the same branches."""
    P_ = ModelParams()
    s = water_system(natoms, density=1.0, seed=1)
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P_), tb.build_gamma(s.R, s.box, P_), s.types,
                   np.zeros(s.natoms))
    nocc = s.n_occ(P_)
    ref = density.density_T0(H, int(nocc))
    out = {}
    for mode in ("emulated", "fp64"):
        n = H.shape[0]
        Ht = torch.as_tensor(H, device="cuda")
        D = torch.empty_like(Ht)
        solver = DensitySolver(ctx, n, sp2_opts("tf32x3", refine=3, refine_mode=mode))
        solver(Ht, nocc, D)
        torch.cuda.synchronize()
        out[mode] = (D.cpu().numpy(), report_to_dict(solver.report))
    (De, re_), (Df, rf) = out["emulated"], out["fp64"]
    assert re_["status"] == rf["status"] == tbmd.TB_OK
    # once X is idempotent to ~1e-10 the two branches are a near tie, so only
    # the first refinement branches must agree
    assert re_["refine_branches"][:2] == rf["refine_branches"][:2]
    assert np.abs(De - Df).max() < 1e-9
    assert abs(re_["trace"] - nocc) < 1e-8
    assert abs(re_["idem_trace"]) < 1e-8
    assert _err(De, ref.D) < 1e-6


@pytest.mark.parametrize("prec,natoms", [("fp64", 24), ("fp64", 150), ("tf32x3", 300)])
def test_graph_captured_sp2_replays_like_eager_calls(ctx, prec, natoms):
    """dm_sp2 captured into a CUDA graph runs its projections after the first
    as a while node that stops with the device-side decision.  Replays on
    Hamiltonians that need different numbers of projections give the same
    D and report, bit for bit, as eager calls on the same workspace; the
    number of projections varies with H, so the loop really stops on the
    device and not at a fixed unroll."""
    s = water_system(natoms, density=1.0, seed=3) if natoms != 24 else water_24_atoms()
    h = tb.build_h(s.R, s.types, s.box, P)
    g0 = tb.build_gamma(s.R, s.box, P)
    nocc = s.n_occ(P)
    rng = np.random.default_rng(5)
    Hs = []
    for amp in (0.0, 0.3):
        na = rng.normal(0, amp, s.natoms) if amp else np.zeros(s.natoms)
        na -= na.mean()
        Hs.append(tb.build_H(h, g0, s.types, na))
    n = Hs[0].shape[0]
    # a spectrum with a much smaller relative gap needs more projections
    Hs.append(random_gapped_matrix(n, int(nocc), gap=0.05, width=20.0, seed=11)[0])
    opts = sp2_opts(prec, tol=1e-11 if prec == "fp64" else 1e-10, refine=2)
    eager = []
    solver = DensitySolver(ctx, n, opts)
    for H in Hs:
        Ht = torch.as_tensor(H, device="cuda")
        D = torch.empty_like(Ht)
        solver(Ht, nocc, D)
        torch.cuda.synchronize()
        eager.append((D.clone(), report_to_dict(solver.report)))
    gs = DensitySolver(ctx, n, opts)
    Hin = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Dout = torch.empty_like(Hin)
    Hin.copy_(torch.as_tensor(Hs[0], device="cuda"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            gs(Hin, nocc, Dout, stream=side)
    torch.cuda.synchronize()
    iters = []
    for H, (De, re_) in zip(Hs, eager):
        Hin.copy_(torch.as_tensor(H, device="cuda"))
        Dout.zero_()
        g.replay()
        torch.cuda.synchronize()
        rg = report_to_dict(gs.report)
        iters.append(rg["iters"])
        assert rg == re_
        assert torch.equal(Dout, De)
        assert rg["status"] == tbmd.TB_OK
    print(f"PARITY sp2 graph {prec} n={n}: projections per replay {iters}, bitwise equal to eager")
    assert len(set(iters)) > 1
    del g
