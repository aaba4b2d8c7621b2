"""The linear-scaling finite-temperature density matrix (row f2): the recursive
Fermi-operator expansion on thresholded block-sparse products
(dm_fermi_sparse) against the oracle.

Checks: with a tau far below every entry (1e-9) the expansion is the Fermi
operator of H (oracle density_fermi: eigh, mu by bisection) to the dense
expansion's bound (2e-6 = ||dD||_F / sqrt(n), the FP32-level products of the
tf32x3 recursion: ~60 products each with relative error ~2^-22 whose errors
add over the doubling steps), on systems with a ragged last block row and on
one with more than 152 upper blocks (the persistent numeric kernel's
multi-block loop); with tau = 1e-5 the oracle's thresholded expansion
(density.fermi_expansion: the same steps in FP64 with the same drop rule),
the zero patterns of the final E compared as for the thresholded SP2 (32 x 32
blocks differ only where the oracle's norm before its last drop lies within
the band of the two results' largest block difference around tau).  The
values: the GPU's intermediate products (W, Z, T, Z W) differ from the
oracle's by their FP32-level errors (~1e-6 absolute), so a block whose norm
lies within that band of tau is dropped by one side and kept by the other;
each such flip moves that product by less than tau in Frobenius norm, the
same kind of change the threshold itself makes.  Both results are therefore
thresholded expansions of H, and the bound is the threshold's own effect:
with eps_tau = ||D_oracle - D_exact||_F / sqrt(n), both ||D_gpu - D_oracle||
and ||D_gpu - D_exact|| (per sqrt(n)) stay below 2e-6 + 2 eps_tau; n > 32768 on isolated identical clusters (every cluster's block is the
cluster's own Fermi operator at the common mu, entries between clusters
exactly 0); a capacity overflow reported with an empty D."""

import numpy as np
import pytest
import torch

from workloads import (ModelParams, gapped_params, gapped_vapour, isolated_clusters, water_system)
from oracle import density, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import BsrMatrix, DeviceSystem, Workspace, fermi_opts, fermi_report_to_dict

pytestmark = pytest.mark.gpu
f64 = dict(dtype=torch.float64, device="cuda")


def _bsr_H(ctx, s, p, cap_per_row=None):
    tp = tbmd.tb_params.from_model(p)
    ds = DeviceSystem(s.R, s.types, s.box)
    n, N = ds.norb, ds.natoms
    nsb = (n + 127) // 128
    Hb = BsrMatrix(n, cap_per_row * nsb if cap_per_row else nsb * nsb)
    v = torch.zeros(N, **f64)
    ws = Workspace(tbmd.tb_bsr_model_workspace_size(N, n))
    tbmd.tb_build_H_bsr(ctx, tp, ds.sys, ds.R, None, Hb.mat, v, ws.ptr, ws.nbytes)
    torch.cuda.synchronize()
    assert int(Hb.status) == tbmd.TB_OK
    return ds, Hb


def _fermi(ctx, Hb, nocc, kT, tau, bpr=0, dcap=None, mu0=float("nan"), opts=None):
    n = Hb.n
    o = opts or fermi_opts("tf32x3")
    Db = BsrMatrix(n, dcap or Hb.nsb * Hb.nsb)
    ws = Workspace(tbmd.dm_fermi_sparse_workspace_size(n, o, bpr))
    mu = torch.full((1,), mu0, **f64)
    rep = torch.zeros(128, dtype=torch.uint8, device="cuda")
    tbmd.dm_fermi_sparse(ctx, Hb.mat, nocc, kT, o, tau, bpr, Db.mat, mu, ws.ptr, ws.nbytes, rep)
    torch.cuda.synchronize()
    return Db, float(mu[0]), fermi_report_to_dict(rep)


def _err(A, B):
    return float(np.linalg.norm(A - B) / np.sqrt(A.shape[0]))


SYSTEMS = {
    "water 300 atoms, 0.5 eV": (lambda: water_system(300, density=1.0, seed=1, morton=True), ModelParams(), 0.5),
    "gapped vapour 300 atoms, 0.2 eV": (lambda: gapped_vapour(100, seed=2, morton=True), gapped_params(), 0.2),
}


@pytest.mark.parametrize("system", list(SYSTEMS))
def test_small_tau_is_the_fermi_operator(ctx, system):
    mk, p, kT = SYSTEMS[system]
    s = mk()
    ds, Hb = _bsr_H(ctx, s, p)
    nocc = s.n_occ(p)
    Db, mu, r = _fermi(ctx, Hb, nocc, kT, 1e-9)
    ref = density.density_fermi(Hb.to_dense(), nocc, kT)
    D = Db.to_dense()
    e = _err(D, ref.D)
    print(f"PARITY dm_fermi_sparse tau=1e-9 {system}: dD {e:.2e}, mu {mu:.6f} (eigh {ref.mu:.6f}), "
          f"{r['mu_iters']} expansions of m={r['m']}, trace {r['trace']:.6f} of {nocc}, {Db.blocks()} blocks")
    assert r["status"] == tbmd.TB_OK and int(Db.status) == tbmd.TB_OK
    assert e < 2e-6
    assert abs(np.trace(D) - nocc) <= 1e-6 + 1e-9 * nocc + 1e-6
    assert np.abs(D - D.T).max() == 0.0


def _pattern_mismatch(Eg, o_D, norms, tau, bs=32):
    n = Eg.shape[0]
    nb = (n + bs - 1) // bs
    pad = np.zeros((nb * bs, nb * bs))

    def bn(X):
        pad[:] = 0.0
        pad[:n, :n] = X
        return np.sqrt((pad.reshape(nb, bs, nb, bs) ** 2).sum(axis=(1, 3)))

    g, r, d = bn(Eg), bn(o_D - 0.5 * np.eye(n)), bn(Eg - (o_D - 0.5 * np.eye(n)))
    both = (g > 0) & (r > 0)
    band = float(d[both].max()) if both.any() else 0.0
    differ = (g == 0) != (r == 0)
    near = np.abs(norms - tau) <= band
    return int((differ & ~near).sum()), int(differ.sum()), band


@pytest.mark.parametrize("system", list(SYSTEMS))
def test_thresholded_expansion_matches_the_oracle(ctx, system):
    mk, p, kT = SYSTEMS[system]
    s = mk()
    ds, Hb = _bsr_H(ctx, s, p)
    nocc = s.n_occ(p)
    tau = 1e-5
    Db, mu, r = _fermi(ctx, Hb, nocc, kT, tau)
    H = Hb.to_dense()
    o = density.fermi_expansion(H, nocc, kT, tau=tau, bs=32, trace_tol=1e-9)
    D = Db.to_dense()
    e = _err(D, o.D)
    mism, differ, band = _pattern_mismatch(D - 0.5 * np.eye(D.shape[0]), o.D, o.pre_drop_norms, tau)
    exact = density.density_fermi(H, nocc, kT)
    eps_tau = _err(o.D, exact.D)
    e_exact = _err(D, exact.D)
    print(f"PARITY dm_fermi_sparse tau=1e-5 {system}: dD {e:.2e} vs the oracle's expansion (m={o.m}, "
          f"{o.expansions} expansions; GPU m={r['m']}, {r['mu_iters']}), {differ} blocks differ in the zero "
          f"pattern, {mism} outside the band {band:.1e}; vs exact {e_exact:.2e}, the threshold's own effect "
          f"{eps_tau:.1e}")
    assert r["status"] == tbmd.TB_OK and o.converged and r["m"] == o.m
    assert e < 2e-6 + 2 * eps_tau and e_exact < 2e-6 + 2 * eps_tau and mism == 0
    assert np.abs(D - D.T).max() == 0.0


def test_more_than_one_round_of_upper_blocks(ctx):
    """gapped vapour, 2046 atoms (n = 4092, 528 upper blocks at tau = 1e-9)."""
    p = gapped_params()
    s = gapped_vapour(682, seed=0, morton=True)
    ds, Hb = _bsr_H(ctx, s, p)
    nocc = s.n_occ(p)
    Db, mu, r = _fermi(ctx, Hb, nocc, 0.2, 1e-9)
    ref = density.density_fermi(Hb.to_dense(), nocc, 0.2)
    e = _err(Db.to_dense(), ref.D)
    print(f"PARITY dm_fermi_sparse n={Hb.n}: dD {e:.2e}, {Db.blocks()} blocks, {r['mu_iters']} expansions")
    assert r["status"] == tbmd.TB_OK and e < 2e-6
    # warm start from the converged mu: one expansion
    Db2, mu2, r2 = _fermi(ctx, Hb, nocc, 0.2, 1e-9, mu0=mu)
    assert r2["status"] == tbmd.TB_OK and r2["mu_iters"] == 1
    assert np.abs(Db2.val.cpu().numpy() - Db.val.cpu().numpy()).max() < 1e-12


def test_beyond_32768_orbitals_on_isolated_clusters(ctx):
    """n = 105456: 13^3 rotated copies of one 8-molecule cluster 16 A apart
    (h block diagonal by cluster, every cluster the same spectrum), kT = 0.3
    eV: the common mu is the one at which each cluster holds its 32 electron
    pairs, so every cluster's block of D is that cluster's Fermi operator
    (oracle: eigh of the 48 x 48 cluster h).  Sampled clusters as in the
    thresholded SP2 test; bounds: the expansion's 2e-6 per entry scale (max
    |dD| < 1e-5), entries between clusters exactly 0.  mu itself is only
    fixed to within the gap (the trace hardly moves there), so it is printed,
    not compared."""
    p = gapped_params()
    s = isolated_clusters(13)
    nc, na, no = 13 ** 3, 24, 48
    ds, Hb = _bsr_H(ctx, s, p, cap_per_row=16)
    n = ds.norb
    nsb = Hb.nsb
    Db, mu, r = _fermi(ctx, Hb, s.n_occ(p), 0.3, 1e-9, bpr=8, dcap=8 * nsb)
    assert r["status"] == tbmd.TB_OK and int(Db.status) == tbmd.TB_OK
    rng = np.random.default_rng(7)
    picks = {0, nc - 1, 32768 // no, (n // 2) // no} | set(rng.choice(nc, 12, replace=False).tolist())
    worst, worst_out = 0.0, 0.0
    for c in sorted(picks):
        a, b = c * no, (c + 1) * no
        Rc, tc = s.R[c * na:(c + 1) * na], s.types[c * na:(c + 1) * na]
        ref = density.density_fermi(tb.build_h(Rc, tc, 1000.0, p), 32.0, 0.3)
        lo, hi = max(0, (a // 128 - 2) * 128), min(n, ((b - 1) // 128 + 3) * 128)
        W = Db.window(a, b, lo, hi)
        worst = max(worst, float(np.abs(W[:, a - lo:b - lo] - ref.D).max()))
        outer = np.concatenate([W[:, :a - lo], W[:, b - lo:]], axis=1)
        worst_out = max(worst_out, float(np.abs(outer).max()) if outer.size else 0.0)
    print(f"PARITY dm_fermi_sparse n={n}: {len(picks)} sampled clusters max|dD| {worst:.2e}, max|D| between "
          f"clusters {worst_out:.1e}, mu {mu:.5f} (cluster {ref.mu:.5f}), {Db.blocks()} D blocks, "
          f"{r['mu_iters']} expansions")
    assert worst < 1e-5 and worst_out == 0.0


def test_capacity_overflow_is_reported(ctx):
    p = ModelParams()
    s = water_system(300, density=1.0, seed=1, morton=True)
    ds, Hb = _bsr_H(ctx, s, p)
    Db, mu, r = _fermi(ctx, Hb, s.n_occ(p), 0.5, 1e-9, bpr=1)
    assert r["status"] == tbmd.TB_ERR_OOM
    assert Db.blocks() == 0


def test_bsr_state_at_finite_temperature_follows_the_dense_state(ctx):
    """10 XL-BOMD steps of the gapped 375-atom vapour at kT = 0.2 eV (no
    entropy term): the BSR state (dm_fermi_sparse, tau = 1e-9, no n x n
    array) against the dense state (dm_fermi).  Both solve Tr D = N_occ to
    the default trace tolerance with tf32x3 products, so their forces differ
    by the expansions' ~1e-6 errors; over 10 steps of 0.25 fs that moves no
    atom by more than 1e-6 A, and E_tot agrees to 1e-6 eV per atom."""
    from workloads import XLParams, thermal_velocities
    from paper_1203_6836_gb300.device import MDState, sp2_opts, xl_params
    PG = gapped_params()
    TPG = tbmd.tb_params.from_model(PG)
    s = gapped_vapour(125, seed=0, morton=True)
    XL = XLParams()
    M = s.masses(PG)
    v0 = thermal_velocities(M, 300.0, seed=100)
    opts = sp2_opts("tf32x3", max_iter=100, tau=1e-9)
    fo = fermi_opts("tf32x3")
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    out = {}
    for label in ("dense", "bsr"):
        ds = DeviceSystem(s.R, s.types, s.box)
        nsb = (ds.norb + 127) // 128
        st = MDState(ds, v0, M, s.n_occ(PG), XL.K, opts, kT=0.2, fermi=fo,
                     bsr_cap=(nsb * nsb, nsb * nsb) if label == "bsr" else None)
        it = tbmd.xlbomd_init(ctx, TPG, st.st, xp, opts, 1e-6, 200)
        E = [st.energies[0].item()]
        for _ in range(10):
            tbmd.xlbomd_step(ctx, TPG, st.st, xp, opts)
            E.append(st.energies[0].item())
        torch.cuda.synchronize()
        out[label] = (it, np.array(E), st.R.cpu().numpy(), float(st.mu[0]), st)
    (i_d, E_d, R_d, mu_d, st_d), (i_b, E_b, R_b, mu_b, st_b) = out["dense"], out["bsr"]
    dE = float(np.abs(E_d - E_b).max())
    dR = float(np.abs(R_d - R_b).max())
    print(f"PARITY bsr state kT=0.2 vs dense state, 10 steps: scf {i_b}/{i_d}, max|dE_tot| {dE:.2e} eV, "
          f"max|dR| {dR:.2e} A, mu {mu_b:.5f} / {mu_d:.5f}, D blocks {st_b.D_bsr.blocks()}")
    assert i_b >= 0 and i_d >= 0
    assert st_b.H is None and st_b.D is None and st_b.gamma is None
    assert dE < 1e-6 * s.natoms and dR < 1e-6
