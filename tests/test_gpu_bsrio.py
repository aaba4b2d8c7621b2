"""The block-sparse boundary (row a5 with BSR matrices at the boundary): H built
into BSR from the super-block bounding boxes (tb_build_H_bsr), SP2 with BSR
input and output (dm_sp2_sparse), Mulliken charges and forces from a BSR D,
and XL-BOMD steps that hold no n x n or N x N array.

Checks: the BSR H equals the dense H of tb_build_H (and the oracle's) entry by
entry, and stores every block the dense H has nonzero; v equals gamma n; D from
dm_sp2_sparse against the oracle's thresholded recursion (density.sp2 with
tau) on the same H, with the zero pattern compared as in test_gpu_bsr /
test_gpu_fullsize (blocks differ only where their norm lies within the band of
the two results' differences around tau); charges and forces from the same D
agree with the dense kernels to FP64 rounding; a trajectory of the BSR state
follows the dense-state trajectory with the same thresholded SP2.

Tolerances: H, v: same FP64 terms in another summation order (1e-12).
D: the tf32x3 thresholded path's 3e-6 (test_gpu_bsr).  q, F, E from one D:
1e-11 e, 1e-10 eV/A, 1e-9 eV (the same FP64 sums in another order).
Trajectory: the two states' H differ in the last bits (summation order), which
can move a 32 x 32 block across tau; over 10 steps E_tot is held to 1e-6 eV
per atom and positions to 1e-6 A."""

import numpy as np
import pytest
import torch

from workloads import ModelParams, XLParams, gapped_params, gapped_vapour, isolated_clusters, thermal_velocities, \
    water_24_atoms, water_system
from oracle import density, observables, tb
from paper_1203_6836_gb300 import tbmd
from paper_1203_6836_gb300.device import BsrMatrix, DeviceSystem, MDState, Workspace, report_to_dict, sp2_opts, \
    xl_params

pytestmark = pytest.mark.gpu
P = ModelParams()
TP = tbmd.tb_params.from_model(P)
f64 = dict(dtype=torch.float64, device="cuda")

SYSTEMS = {
    "24 atoms, 6.5 A box": lambda: water_24_atoms(),
    "water 600 Morton": lambda: water_system(600, density=1.0, seed=1, morton=True),
    "water 2048 Morton": lambda: water_system(2048, density=1.0, seed=0, morton=True),
}


def _charges(N, seed):
    rng = np.random.default_rng(seed)
    n = rng.normal(0, 0.2, N)
    return n - n.mean()


def _bsr_H(ctx, s, n_aux, tp=TP, cap=None):
    ds = DeviceSystem(s.R, s.types, s.box)
    n, N = ds.norb, ds.natoms
    nsb = (n + 127) // 128
    Hb = BsrMatrix(n, cap or nsb * nsb)
    v = torch.zeros(N, **f64)
    ws = Workspace(tbmd.tb_bsr_model_workspace_size(N, n))
    na = torch.as_tensor(n_aux, device="cuda") if n_aux is not None else None
    tbmd.tb_build_H_bsr(ctx, tp, ds.sys, ds.R, na, Hb.mat, v, ws.ptr, ws.nbytes)
    torch.cuda.synchronize()
    return ds, Hb, v, ws


@pytest.mark.parametrize("system", list(SYSTEMS))
def test_bsr_H_equals_the_dense_H(ctx, system):
    s = SYSTEMS[system]()
    n_aux = _charges(s.natoms, 1)
    ds, Hb, v, ws = _bsr_H(ctx, s, n_aux)
    assert int(Hb.status) == tbmd.TB_OK
    n = ds.norb
    Hd = torch.empty(n, n, **f64)
    G = torch.empty(s.natoms, s.natoms, **f64)
    tbmd.tb_build_H(ctx, TP, ds.sys, ds.R, torch.as_tensor(n_aux, device="cuda"), Hd, G)
    torch.cuda.synchronize()
    Hbd = Hb.to_dense()
    Hdn = Hd.cpu().numpy()
    e = float(np.abs(Hbd - Hdn).max())
    ev = float(np.abs(v.cpu().numpy() - G.cpu().numpy() @ n_aux).max())
    # every nonzero block of the dense H is stored
    nsb = Hb.nsb
    pad = np.zeros((nsb * 128, nsb * 128))
    pad[:n, :n] = np.abs(Hdn)
    nz = pad.reshape(nsb, 128, nsb, 128).max(axis=(1, 3)) > 0
    stored = np.zeros((nsb, nsb), bool)
    rp, col = Hb.row_ptr.cpu().numpy(), Hb.col.cpu().numpy()
    for I in range(nsb):
        stored[I, col[rp[I]:rp[I + 1]]] = True
    print(f"PARITY bsr H {system}: max|dH| {e:.2e} max|dv| {ev:.2e}, {Hb.blocks()} of {nsb * nsb} blocks stored, "
          f"{int(nz.sum())} nonzero")
    assert e < 1e-12 and ev < 1e-12
    assert not (nz & ~stored).any()
    if system == "water 600 Morton":
        Ho = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types, n_aux)
        assert float(np.abs(Hbd - Ho).max()) < 1e-12


def _pattern_mismatch(Dg, o, tau, bs=32):
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
    return int((differ & ~near).sum()), band


@pytest.mark.parametrize("system", ["water 600 Morton", "water 2048 Morton"])
def test_dm_sp2_sparse_matches_the_thresholded_recursion(ctx, system):
    s = SYSTEMS[system]()
    ds, Hb, v, ws = _bsr_H(ctx, s, None)
    n = ds.norb
    nocc = s.n_occ(P)
    opts = sp2_opts("tf32x3", max_iter=100, tau=1e-5)
    Db = BsrMatrix(n, Hb.nsb * Hb.nsb)
    sws = Workspace(tbmd.dm_sp2_workspace_size(n, opts))
    rep = torch.zeros(256, dtype=torch.uint8, device="cuda")
    tbmd.dm_sp2_sparse(ctx, Hb.mat, nocc, opts, Db.mat, sws.ptr, sws.nbytes, rep)
    torch.cuda.synchronize()
    r = report_to_dict(rep)
    H = Hb.to_dense()
    o = density.sp2(H, nocc, tol=1e-9, tau=1e-5, bs=32)
    D = Db.to_dense()
    e = np.linalg.norm(D - o.X) / np.sqrt(n)
    mism, band = _pattern_mismatch(D, o, 1e-5)
    print(f"PARITY dm_sp2_sparse {system}: dD {e:.2e}, {Db.blocks()} blocks of D, {mism} pattern mismatches "
          f"outside the band {band:.1e}, iters {r['iters']}")
    assert int(Db.status) == tbmd.TB_OK and r["status"] == tbmd.TB_OK
    assert e < 3e-6 and mism == 0


@pytest.mark.parametrize("system", ["24 atoms, 6.5 A box", "water 600 Morton"])
def test_charges_and_forces_from_a_bsr_D(ctx, system):
    s = SYSTEMS[system]()
    n_aux = _charges(s.natoms, 3)
    ds, Hb, v, ws = _bsr_H(ctx, s, n_aux)
    n, N = ds.norb, ds.natoms
    H = Hb.to_dense()
    D = density.density_T0(H, int(s.n_occ(P))).D
    # the D blocks on H's pattern (D is dense here: store every block)
    Db = BsrMatrix(n, Hb.nsb * Hb.nsb)
    nsb = Hb.nsb
    rp = np.arange(nsb + 1, dtype=np.int32) * nsb
    col = np.tile(np.arange(nsb, dtype=np.int32), nsb)
    pad = np.zeros((nsb * 128, nsb * 128))
    pad[:n, :n] = D
    blocks = pad.reshape(nsb, 128, nsb, 128).transpose(0, 2, 1, 3).reshape(-1)
    Db.row_ptr.copy_(torch.as_tensor(rp))
    Db.col.copy_(torch.as_tensor(col))
    Db.val.copy_(torch.as_tensor(blocks))
    q = torch.empty(N, **f64)
    tbmd.mulliken_bsr(ctx, TP, ds.sys, Db.mat, q)
    F = torch.empty(N, 3, **f64)
    E = torch.empty(4, **f64)
    tbmd.tb_forces_bsr(ctx, TP, ds.sys, ds.R, Hb.mat, Db.mat, q, torch.as_tensor(n_aux, device="cuda"), v, F, E,
                       ws.ptr, ws.nbytes)
    torch.cuda.synchronize()
    qo = observables.mulliken(D, s.types, P)
    Fo = observables.forces(s.R, s.types, s.box, P, D, qo, n_aux)
    Eo = observables.energy_terms(s.R, s.types, s.box, P, D, qo, n_aux)
    eq = float(np.abs(q.cpu().numpy() - qo).max())
    eF = float(np.abs(F.cpu().numpy() - Fo).max())
    print(f"PARITY bsr q, F {system}: max|dq| {eq:.2e} max|dF| {eF:.2e} dE {abs(E[0].item() - sum(Eo)):.2e}")
    assert eq < 1e-11 and eF < 1e-10
    assert E[0].item() == pytest.approx(sum(Eo), abs=1e-9)


def test_bsr_capacity_overflow_is_reported(ctx):
    s = SYSTEMS["water 600 Morton"]()
    ds, Hb, v, ws = _bsr_H(ctx, s, None, cap=3)
    assert int(Hb.status) == tbmd.TB_ERR_OOM


def test_bsr_state_trajectory_follows_the_dense_state(ctx):
    """10 steps of the gapped 375-atom vapour (Morton order) with tau = 1e-5:
    the BSR state (no n x n array) against the dense state with the same
    thresholded SP2."""
    PG = gapped_params()
    TPG = tbmd.tb_params.from_model(PG)
    s = gapped_vapour(125, seed=0, morton=True)
    XL = XLParams()
    M = s.masses(PG)
    v0 = thermal_velocities(M, 300.0, seed=100)
    opts = sp2_opts("tf32x3", max_iter=100, tau=1e-5)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    out = {}
    n = None
    for label in ("dense", "bsr"):
        ds = DeviceSystem(s.R, s.types, s.box)
        n = ds.norb
        nsb = (n + 127) // 128
        st = MDState(ds, v0, M, s.n_occ(PG), XL.K, opts, bsr_cap=(nsb * nsb, nsb * nsb) if label == "bsr" else None)
        it = tbmd.xlbomd_init(ctx, TPG, st.st, xp, opts, 1e-6, 200)
        E, R = [st.energies[0].item()], []
        for _ in range(10):
            tbmd.xlbomd_step(ctx, TPG, st.st, xp, opts)
            E.append(st.energies[0].item())
        torch.cuda.synchronize()
        out[label] = (it, np.array(E), st.R.cpu().numpy(), st.q.cpu().numpy(), st)
    (i_d, E_d, R_d, q_d, st_d), (i_b, E_b, R_b, q_b, st_b) = out["dense"], out["bsr"]
    dE = float(np.abs(E_d - E_b).max())
    dR = float(np.abs(R_d - R_b).max())
    print(f"PARITY bsr state vs dense state, 10 steps: scf {i_b}/{i_d}, max|dE_tot| {dE:.2e} eV, max|dR| {dR:.2e} A, "
          f"H blocks {st_b.H_bsr.blocks()}, D blocks {st_b.D_bsr.blocks()} of {(n + 127) // 128} ** 2")
    assert i_b >= 0 and i_d >= 0
    assert st_b.H is None and st_b.D is None and st_b.gamma is None
    assert dE < 1e-6 * s.natoms and dR < 1e-6


def test_dm_sp2_sparse_beyond_32768_orbitals_on_isolated_clusters(ctx):
    """n = 105456 (824 block rows, the row bitmaps' words 8..25 in use):
    13^3 rotated copies of an 8-molecule cluster 16 A apart, H = h (no
    charges).  Clusters do not interact, so h is block diagonal by cluster;
    every cluster has the same spectrum, so the global SP2 projection is, on
    each cluster, the projection on its own 32 lowest states.  The oracle
    computes that (eigh of the 48 x 48 cluster h) for sampled clusters: the
    first, the last, the ones across orbital 32768 (bitmap word 8) and n / 2,
    and 12 at random.  Bound: the tf32x3 phase without refinement stops at
    its FP32 noise floor (2e-5 max, as for the grouped path); entries
    between clusters are products with an exact zero factor, so exactly 0;
    the block pattern of D stays within two blocks of the diagonal (the
    symbolic square of H's one-block band); and the
    whole run holds no n x n array (BSR capacities of 16 / 8 blocks per
    row)."""
    PG = gapped_params()
    TPG = tbmd.tb_params.from_model(PG)
    s = isolated_clusters(13)
    nc, na, no = 13 ** 3, 24, 48
    ds = DeviceSystem(s.R, s.types, s.box)
    n = ds.norb
    assert n == nc * no and n > 32768
    nsb = (n + 127) // 128
    Hb = BsrMatrix(n, 16 * nsb)
    v = torch.zeros(s.natoms, **f64)
    ws = Workspace(tbmd.tb_bsr_model_workspace_size(s.natoms, n))
    tbmd.tb_build_H_bsr(ctx, TPG, ds.sys, ds.R, None, Hb.mat, v, ws.ptr, ws.nbytes)
    opts = sp2_opts("tf32x3", max_iter=100, tau=1e-9, blocks_per_row=8)
    Db = BsrMatrix(n, 8 * nsb)
    sws = Workspace(tbmd.dm_sp2_workspace_size(n, opts))
    rep = torch.zeros(256, dtype=torch.uint8, device="cuda")
    nocc = s.n_occ(PG)
    tbmd.dm_sp2_sparse(ctx, Hb.mat, nocc, opts, Db.mat, sws.ptr, sws.nbytes, rep)
    torch.cuda.synchronize()
    r = report_to_dict(rep)
    assert int(Hb.status) == tbmd.TB_OK and int(Db.status) == tbmd.TB_OK and r["status"] == tbmd.TB_OK
    rp, col = Db.row_ptr.cpu().numpy(), Db.col.cpu().numpy()
    rows = np.repeat(np.arange(nsb), np.diff(rp))
    # X^2's symbolic pattern of a one-block band: two blocks off the diagonal
    # (stored, valued 0 where no cluster spans both), no farther
    assert np.abs(col[:rp[-1]] - rows).max() <= 2
    rng = np.random.default_rng(7)
    picks = {0, nc - 1, 32768 // no, (n // 2) // no} | set(rng.choice(nc, 12, replace=False).tolist())
    worst, worst_out, tr = 0.0, 0.0, []
    for c in sorted(picks):
        a, b = c * no, (c + 1) * no
        Rc, tc = s.R[c * na:(c + 1) * na], s.types[c * na:(c + 1) * na]
        Dc = density.density_T0(tb.build_h(Rc, tc, 1000.0, PG), 32).D
        lo, hi = max(0, (a // 128 - 2) * 128), min(n, ((b - 1) // 128 + 3) * 128)
        W = Db.window(a, b, lo, hi)
        inner = W[:, a - lo:b - lo]
        worst = max(worst, float(np.abs(inner - Dc).max()))
        outer = np.concatenate([W[:, :a - lo], W[:, b - lo:]], axis=1)
        worst_out = max(worst_out, float(np.abs(outer).max()) if outer.size else 0.0)
        tr.append(np.trace(inner))
    print(f"PARITY dm_sp2_sparse n={n}: {len(picks)} sampled clusters max|dD| {worst:.2e}, "
          f"max|D| between clusters {worst_out:.1e}, cluster traces {min(tr):.6f}..{max(tr):.6f}; "
          f"{Hb.blocks()} H blocks, {Db.blocks()} D blocks, iters {r['iters']}, trace {r['trace']:.4f} of {nocc}")
    assert worst < 2e-5 and worst_out == 0.0
    assert max(abs(t - 32.0) for t in tr) < 1e-4
    assert abs(r["trace"] - nocc) < 1e-5 * nocc
