"""Thresholded block-sparse SP2 on the GPU (dm_sp2 with tau > 0) against the
oracle's thresholded recursion (density.sp2 with tau, 32 x 32 blocks, FP64)
on the same Morton-ordered water-like Hamiltonians.

Both sides drop the same 32 x 32 blocks (compared exactly: the zero pattern
of D), and the surviving entries differ by the FP32 accuracy of the tf32x3
tensor-core products (~1e-6 per sqrt(n) here, no FP64 refinement in this
path); tau -> 0 reproduces the dense result."""

import numpy as np
import pytest
import torch

from workloads import random_gapped_matrix, water_system, ModelParams
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import DensitySolver, sp2_opts, report_to_dict

pytestmark = pytest.mark.gpu
P = ModelParams()


def _water_H(natoms, seed=0):
    w = water_system(natoms, density=1.0, seed=seed, morton=True)
    H = tb.build_H(tb.build_h(w.R, w.types, w.box, P), tb.build_gamma(w.R, w.box, P), w.types,
                   np.zeros(w.natoms))
    return H, w.n_occ(P)


def _run(ctx, H, nocc, tau, prec="tf32x3", bpr=0):
    Ht = torch.as_tensor(H, device="cuda")
    D = torch.empty_like(Ht)
    s = DensitySolver(ctx, H.shape[0], sp2_opts(prec, max_iter=100, tau=tau, blocks_per_row=bpr))
    s(Ht, nocc, D)
    torch.cuda.synchronize()
    return D.cpu().numpy(), report_to_dict(s.report)


def _err(A, B):
    return np.linalg.norm(A - B) / np.sqrt(A.shape[0])


@pytest.mark.parametrize("natoms,tau,tol", [(300, 1e-5, 3e-6), (600, 1e-5, 3e-6), (1024, 1e-5, 3e-6),
                                            (600, 1e-3, 1e-4), (1024, 1e-3, 1e-4)])
def test_thresholded_matches_oracle_recursion(ctx, natoms, tau, tol):
    H, nocc = _water_H(natoms)
    n = H.shape[0]
    D, rep = _run(ctx, H, nocc, tau)
    o = density.sp2(H, nocc, tol=1e-9, tau=tau, bs=32)
    assert rep["status"] == tbmd.TB_OK
    # the same 32 x 32 blocks are dropped on both sides
    nb = (n + 31) // 32
    pad = np.zeros((nb * 32, nb * 32))
    pad[:n, :n] = np.abs(D)
    zg = pad.reshape(nb, 32, nb, 32).max(axis=(1, 3)) == 0
    pad[:n, :n] = np.abs(o.X)
    zo = pad.reshape(nb, 32, nb, 32).max(axis=(1, 3)) == 0
    assert (zg == zo).mean() > 0.999
    assert _err(D, o.X) < tol
    assert abs(rep["trace"] - nocc) < 2e-3


def test_vanishing_tau_is_the_dense_result(ctx):
    H, nocc = _water_H(600, seed=2)
    ref = density.density_T0(H, int(nocc))
    D, rep = _run(ctx, H, nocc, 1e-300)
    assert rep["status"] == tbmd.TB_OK
    assert _err(D, ref.D) < 3e-6


def test_decoupled_blocks_stay_exactly_zero(ctx):
    """Two decoupled 160-orbital blocks (coupling 1e-9): the coupling blocks of
    X0 are below tau and every projection keeps them at exactly zero."""
    A, _ = random_gapped_matrix(160, 60, gap=2.0, width=20.0, seed=6)
    B, _ = random_gapped_matrix(160, 70, gap=2.0, width=20.0, seed=7)
    H = np.zeros((320, 320))
    H[:160, :160], H[160:, 160:] = A, B
    H[:160, 160:] = 1e-9
    H[160:, :160] = 1e-9
    D, rep = _run(ctx, H, 130.0, 1e-5)
    assert np.all(D[:160, 160:] == 0.0) and np.all(D[160:, :160] == 0.0)
    ref = density.density_T0(H, 130)
    assert _err(D, ref.D) < 1e-4


def test_capacity_overflow_is_reported(ctx):
    """A pattern cap of one 128 x 128 block per block row cannot hold X0 of a
    water system: the report says TB_ERR_OOM instead of writing out of bounds."""
    H, nocc = _water_H(300, seed=1)
    D, rep = _run(ctx, H, nocc, 1e-5, bpr=1)
    assert rep["status"] == tbmd.TB_ERR_OOM
