"""Guard regions: every output of the path is written inside its bounds.

Each output array is carved out of a larger buffer whose leading and trailing
64 elements hold a canary value; after the calls the canaries must be intact and
the outputs finite.  The sizes are ragged (n = 300 is not a multiple of the
128-wide tensor-core tiles, N = 150 atoms), so the padded tails of the tiled
kernels are exercised."""

import math

import numpy as np
import pytest
import torch

from workloads import ModelParams, water_system
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, DeviceSystem, FermiSolver, fermi_opts, sp2_opts

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)
CANARY = 1.2345678e300
G = 64  # guard elements on each side (512 bytes: the view keeps the buffer's alignment)


def _guarded(*shape):
    count = math.prod(shape)
    buf = torch.full((count + 2 * G,), CANARY, dtype=torch.float64, device="cuda")
    return buf, buf[G:G + count].view(*shape)


def _check(buf, view, name):
    torch.cuda.synchronize()
    count = view.numel()
    assert bool((buf[:G] == CANARY).all()), f"{name}: write before the array"
    assert bool((buf[G + count:] == CANARY).all()), f"{name}: write after the array"
    assert bool(torch.isfinite(view).all()), f"{name}: non-finite output"


def _system():
    s = water_system(150, density=1.0, seed=7)
    ds = DeviceSystem(s.R, s.types, s.box)
    assert ds.norb % 128 != 0
    return s, ds


def test_model_kernels_write_inside_their_arrays(ctx):
    s, ds = _system()
    N, n = ds.natoms, ds.norb
    rng = np.random.default_rng(0)
    n_aux = torch.as_tensor(rng.normal(0, 0.3, N) - 0.0, device="cuda")
    hb, H = _guarded(n, n)
    gb, Gm = _guarded(N, N)
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, n_aux, H, Gm)
    _check(hb, H, "H")
    _check(gb, Gm, "gamma")
    A = rng.normal(0, 0.05, (n, n))
    D = torch.as_tensor(0.5 * (A + A.T) + 0.5 * np.eye(n), device="cuda")
    qb, q = _guarded(N)
    tbmd.mulliken(ctx, TP, ds.sys, D, q)
    _check(qb, q, "q")
    fb, F = _guarded(N, 3)
    eb, E = _guarded(4)
    tbmd.tb_forces(ctx, TP, ds.sys, ds.R, D, q, n_aux, Gm, F, E)
    _check(fb, F, "F")
    _check(eb, E, "energy")


@pytest.mark.parametrize("kind", ["fp64", "tf32x3+refine", "bsr", "fermi"])
def test_density_solvers_write_inside_D(ctx, kind):
    s, ds = _system()
    n = ds.norb
    H = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Gm = torch.empty(ds.natoms, ds.natoms, dtype=torch.float64, device="cuda")
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, None, H, Gm)
    db, D = _guarded(n, n)
    nocc = s.n_occ(P)
    if kind == "fermi":
        FermiSolver(ctx, n, fermi_opts("tf32x3"))(H, nocc, 0.1, D)
    else:
        opts = {"fp64": sp2_opts("fp64", max_iter=100, tol=1e-11),
                "tf32x3+refine": sp2_opts("tf32x3", max_iter=100, refine=2),
                "bsr": sp2_opts("tf32x3", max_iter=100, tau=1e-5)}[kind]
        DensitySolver(ctx, n, opts)(H, nocc, D)
    _check(db, D, f"D ({kind})")
    if kind != "bsr":  # the thresholded recursion's trace drifts by the dropped blocks (2e-4 here)
        assert abs(torch.trace(D).item() - nocc) < 1e-4
