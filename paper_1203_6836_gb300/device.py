"""Device-side containers for calling libtbmd from PyTorch: torch owns the
memory, these helpers only lay out arrays and fill the C structs."""

from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import tbmd

NORB = {tbmd.TB_TYPE_O: 4, tbmd.TB_TYPE_H: 1}


def orbital_offsets(types: np.ndarray) -> np.ndarray:
    """First orbital of each atom (orbitals grouped by atom), length N + 1."""
    counts = np.where(np.asarray(types) == tbmd.TB_TYPE_O, 4, 1)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)


class DeviceSystem:
    """Atom types, orbital offsets and positions of one periodic system on a device."""

    def __init__(self, R: np.ndarray, types: np.ndarray, box: float, device="cuda"):
        self.device = torch.device(device)
        self.types = torch.as_tensor(np.asarray(types, dtype=np.int32), device=self.device)
        offs = orbital_offsets(types)
        self.orb_off = torch.as_tensor(offs, device=self.device)
        self.R = torch.as_tensor(np.asarray(R, dtype=np.float64), device=self.device).contiguous()
        self.natoms = int(len(types))
        self.norb = int(offs[-1])
        self.box = float(box)
        self.sys = tbmd.tb_system(natoms=self.natoms, norb=self.norb, types=self.types.data_ptr(),
                                  orb_off=self.orb_off.data_ptr(), box=self.box)


class Workspace:
    """A 1024-byte aligned device buffer carved out of a torch uint8 tensor."""

    def __init__(self, nbytes: int, device="cuda"):
        self.buf = torch.empty(int(nbytes) + 1024, dtype=torch.uint8, device=device)
        base = self.buf.data_ptr()
        self.ptr = (base + 1023) // 1024 * 1024
        self.nbytes = int(nbytes)


REFINE = {"emulated": 0, "fp64": 1}


def sp2_opts(precision: str = "fp64", max_iter: int = 100, tol: float = 1e-10, refine: int = 2,
             rule: int = 0, refine_mode: str = "emulated", tau: float = 0.0,
             blocks_per_row: int = 0) -> tbmd.tb_sp2_opts:
    """refine_mode: "emulated" (exact-slice FP64 emulation on the tensor cores) or "fp64" (FMA);
    tau > 0 selects the thresholded block-sparse path."""
    return tbmd.tb_sp2_opts(precision=tbmd.PREC[precision], max_iter=max_iter, tol=tol,
                            refine_iters=refine, rule=rule, refine_mode=REFINE[refine_mode], tau=tau,
                            bsr_blocks_per_row=blocks_per_row)


def xl_params(dt: float, kappa: float, alpha: float, c) -> tbmd.tb_xl_params:
    x = tbmd.tb_xl_params(dt=dt, kappa=kappa, alpha=alpha, K=len(c) - 1)
    for k, ck in enumerate(c):
        x.c[k] = float(ck)
    return x


def report_to_dict(buf: torch.Tensor) -> dict:
    """Decode a tb_sp2_report held in a device uint8 tensor."""
    raw = buf.detach().cpu().numpy().tobytes()
    r = tbmd.tb_sp2_report.from_buffer_copy(raw[:ctypes.sizeof(tbmd.tb_sp2_report)])
    return {"status": r.status, "iters": r.iters, "refine_iters": r.refine_iters, "n": r.n,
            "eps_min": r.eps_min, "eps_max": r.eps_max, "trace": r.trace, "idem_trace": r.idem_trace,
            "idem_fro": r.idem_fro, "block_products": r.block_products, "blocks": r.blocks,
            "branches": [(int(r.branch_bits[k >> 6]) >> (k & 63)) & 1 for k in range(r.iters)],
            "refine_branches": [(int(r.refine_bits) >> k) & 1 for k in range(r.refine_iters)]}


def new_report(device="cuda") -> torch.Tensor:
    return torch.zeros(ctypes.sizeof(tbmd.tb_sp2_report), dtype=torch.uint8, device=device)


class DensitySolver:
    """dm_sp2 with its workspace sized for n (reused across calls on one stream)."""

    def __init__(self, ctx: tbmd.Context, n: int, opts: tbmd.tb_sp2_opts, device="cuda"):
        self.ctx, self.n, self.opts = ctx, int(n), opts
        self.ws = Workspace(tbmd.dm_sp2_workspace_size(n, opts), device)
        self.report = new_report(device)

    def __call__(self, H: torch.Tensor, n_occ: float, D: torch.Tensor, stream=None):
        tbmd.dm_sp2(self.ctx, H, self.n, n_occ, self.opts, D, self.ws.ptr, self.ws.nbytes, self.report, stream)
        return D


class BsrMatrix:
    """A tb_bsr (128 x 128 FP64 blocks) with device arrays of `cap` blocks."""

    B = 128

    def __init__(self, n: int, cap: int, device="cuda"):
        nsb = (n + self.B - 1) // self.B
        self.n, self.nsb, self.cap = int(n), nsb, int(cap)
        self.row_ptr = torch.zeros(nsb + 1, dtype=torch.int32, device=device)
        self.col = torch.zeros(max(1, cap), dtype=torch.int32, device=device)
        self.val = torch.zeros(max(1, cap) * self.B * self.B, dtype=torch.float64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.mat = tbmd.tb_bsr(n=self.n, nsb=nsb, cap=self.cap, row_ptr=self.row_ptr.data_ptr(),
                               col=self.col.data_ptr(), val=self.val.data_ptr(), status=self.status.data_ptr())

    def blocks(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        """The matrix on the host (small systems, for checks)."""
        rp = self.row_ptr.cpu().numpy()
        col = self.col.cpu().numpy()
        val = self.val.cpu().numpy().reshape(-1, self.B, self.B)
        ld = self.nsb * self.B
        M = np.zeros((ld, ld))
        for I in range(self.nsb):
            for s in range(rp[I], rp[I + 1]):
                J = col[s]
                M[I * self.B:(I + 1) * self.B, J * self.B:(J + 1) * self.B] = val[s]
        return M[:self.n, :self.n]

    def window(self, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
        """Rows [r0, r1) x columns [c0, c1) on the host, gathered from the
        stored blocks that meet them (any n: for checks of a large matrix)."""
        B = self.B
        rp = self.row_ptr.cpu().numpy()
        col = self.col.cpu().numpy()
        I0, I1 = r0 // B, (r1 - 1) // B + 1
        J0, J1 = c0 // B, (c1 - 1) // B + 1
        slots, where = [], []
        for I in range(I0, I1):
            for s in range(rp[I], rp[I + 1]):
                if J0 <= col[s] < J1:
                    slots.append(s)
                    where.append((I - I0, col[s] - J0))
        W = np.zeros(((I1 - I0) * B, (J1 - J0) * B))
        if slots:
            idx = torch.as_tensor(slots, dtype=torch.long, device=self.val.device)
            blk = self.val.view(-1, B, B).index_select(0, idx).cpu().numpy()
            for (i, j), b in zip(where, blk):
                W[i * B:(i + 1) * B, j * B:(j + 1) * B] = b
        return W[r0 - I0 * B:r1 - I0 * B, c0 - J0 * B:c1 - J0 * B]


class MDState:
    """Device arrays of one XL-BOMD trajectory and its tb_md_state (T_e = 0 with
    SP2 options, or kT > 0 with Fermi-operator options)."""

    def __init__(self, ds: DeviceSystem, v0: np.ndarray, masses: np.ndarray, n_occ: float, K: int,
                 opts: tbmd.tb_sp2_opts, kT: float = 0.0, fermi: "tbmd.tb_fermi_opts" = None,
                 entropy: bool = False, nonorth: bool = False, bsr_cap: tuple = None):
        dev = ds.device
        N, n = ds.natoms, ds.norb
        f64 = dict(dtype=torch.float64, device=dev)
        self.ds = ds
        self.R = ds.R
        self.v = torch.as_tensor(np.asarray(v0, dtype=np.float64), device=dev).contiguous()
        self.F = torch.zeros(N, 3, **f64)
        self.mass = torch.as_tensor(np.asarray(masses, dtype=np.float64), device=dev)
        self.n_hist = torch.zeros(K + 1, N, **f64)
        self.q = torch.zeros(N, **f64)
        # bsr_cap = (blocks of H, blocks of D): the block-sparse state, no n x n or N x N array
        self.bsr = bsr_cap is not None
        if self.bsr:
            self.H = self.D = self.gamma = None
            self.H_bsr = BsrMatrix(n, bsr_cap[0], dev)
            self.D_bsr = BsrMatrix(n, bsr_cap[1], dev)
            self.bsr_ws = Workspace(tbmd.tb_bsr_model_workspace_size(N, n), dev)
        else:
            self.H = torch.zeros(n, n, **f64)
            self.D = torch.zeros(n, n, **f64)
            self.gamma = torch.zeros(N, N, **f64)
            self.H_bsr = self.D_bsr = self.bsr_ws = None
        self.energies = torch.zeros(8, **f64)
        self.report = new_report(dev)
        self.fermi_report = torch.zeros(ctypes.sizeof(tbmd.tb_fermi_report), dtype=torch.uint8, device=dev)
        self.mu = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
        if kT > 0.0:
            fermi = fermi or fermi_opts()
            if self.bsr:
                ws = tbmd.dm_fermi_sparse_workspace_size(n, fermi, opts.bsr_blocks_per_row)
            else:
                ws = tbmd.dm_fermi_workspace_size(n, fermi)
            self.ws = Workspace(ws, dev)
        else:
            fermi = tbmd.tb_fermi_opts()
            self.ws = Workspace(tbmd.dm_sp2_workspace_size(n, opts), dev)
        self.K = K
        # kT > 0 with entropy: E_tot (energies[0]) includes -kT S, S/k_B in self.entropy
        self.entropy = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        self.ent_ws = Workspace(tbmd.dm_fermi_entropy_workspace_size(n), dev) if (entropy and kT > 0.0) else None
        # the non-orthogonal formulation (a model with an overlap): S, W, v and dm_nonorth's
        # workspace, which holds the SP2 / Fermi workspace of H_perp
        self.nonorth_report = torch.zeros(ctypes.sizeof(tbmd.tb_nonorth_report), dtype=torch.uint8, device=dev)
        if nonorth:
            self.S = torch.zeros(n, n, **f64)
            self.W = torch.zeros(n, n, **f64)
            self.vscc = torch.zeros(N, **f64)
            self.no_ws = Workspace(tbmd.dm_nonorth_workspace_size(n, kT, opts, fermi), dev)
        else:
            self.S = self.W = self.no_ws = None
            self.vscc = torch.zeros(N, **f64) if self.bsr else None
        self.st = tbmd.tb_md_state(
            sys=ds.sys, n_occ=float(n_occ), R=self.R.data_ptr(), v=self.v.data_ptr(), F=self.F.data_ptr(),
            mass=self.mass.data_ptr(), n_hist=self.n_hist.data_ptr(), q=self.q.data_ptr(),
            H=self.H.data_ptr() if self.H is not None else None, D=self.D.data_ptr() if self.D is not None else None,
            gamma=self.gamma.data_ptr() if self.gamma is not None else None,
            energies=self.energies.data_ptr(), sp2_report=self.report.data_ptr(),
            workspace=self.ws.ptr, workspace_bytes=self.ws.nbytes, step=0, kT=float(kT), fermi=fermi,
            mu=self.mu.data_ptr(), fermi_report=self.fermi_report.data_ptr(),
            entropy_workspace=self.ent_ws.ptr if self.ent_ws else None,
            entropy_workspace_bytes=self.ent_ws.nbytes if self.ent_ws else 0,
            entropy=self.entropy.data_ptr() if self.ent_ws else None,
            S=self.S.data_ptr() if nonorth else None, W=self.W.data_ptr() if nonorth else None,
            vscc=self.vscc.data_ptr() if self.vscc is not None else None,
            nonorth_workspace=self.no_ws.ptr if nonorth else None,
            nonorth_workspace_bytes=self.no_ws.nbytes if nonorth else 0,
            nonorth_report=self.nonorth_report.data_ptr(),
            H_bsr=ctypes.addressof(self.H_bsr.mat) if self.bsr else None,
            D_bsr=ctypes.addressof(self.D_bsr.mat) if self.bsr else None,
            bsr_workspace=self.bsr_ws.ptr if self.bsr else None,
            bsr_workspace_bytes=self.bsr_ws.nbytes if self.bsr else 0)

    def n_current(self) -> torch.Tensor:
        return self.n_hist[0]


def fermi_opts(precision: str = "tf32x3", m: int = 14, ns_iters: int = 3, mu_iters: int = 30,
               trace_tol: float = 0.0) -> tbmd.tb_fermi_opts:
    return tbmd.tb_fermi_opts(precision=tbmd.PREC[precision], m=m, ns_iters=ns_iters, mu_iters=mu_iters,
                              trace_tol=trace_tol)


def fermi_report_to_dict(buf: torch.Tensor) -> dict:
    raw = buf.detach().cpu().numpy().tobytes()
    r = tbmd.tb_fermi_report.from_buffer_copy(raw[:ctypes.sizeof(tbmd.tb_fermi_report)])
    return {k: getattr(r, k) for k, _ in tbmd.tb_fermi_report._fields_}


class EntropySolver:
    """dm_fermi_entropy with its workspace sized for n: S/k_B (and optionally
    the FP64 Fermi matrix) of H at a given device mu."""

    def __init__(self, ctx: tbmd.Context, n: int, device="cuda"):
        self.ctx, self.n = ctx, int(n)
        self.ws = Workspace(tbmd.dm_fermi_entropy_workspace_size(n), device)
        self.S = torch.full((1,), float("nan"), dtype=torch.float64, device=device)

    def __call__(self, H: torch.Tensor, mu: torch.Tensor, kT: float, D: torch.Tensor = None, stream=None):
        tbmd.dm_fermi_entropy(self.ctx, H, self.n, mu, kT, D, self.S, self.ws.ptr, self.ws.nbytes, stream)
        return self.S


class FermiSolver:
    """dm_fermi with its workspace sized for n; mu is kept on the device and
    warm-starts the next call."""

    def __init__(self, ctx: tbmd.Context, n: int, opts: tbmd.tb_fermi_opts, device="cuda"):
        self.ctx, self.n, self.opts = ctx, int(n), opts
        self.ws = Workspace(tbmd.dm_fermi_workspace_size(n, opts), device)
        self.report = torch.zeros(ctypes.sizeof(tbmd.tb_fermi_report), dtype=torch.uint8, device=device)
        self.mu = torch.full((1,), float("nan"), dtype=torch.float64, device=device)

    def __call__(self, H: torch.Tensor, n_occ: float, kT: float, D: torch.Tensor, stream=None):
        tbmd.dm_fermi(self.ctx, H, self.n, n_occ, kT, self.opts, D, self.mu, self.ws.ptr, self.ws.nbytes,
                      self.report, stream)
        return D


class Server:
    """tb_server: continuous batching of XL-BOMD step requests (C++ runtime)."""

    def __init__(self, ctx: tbmd.Context, p: tbmd.tb_params, xl: tbmd.tb_xl_params, kT: float = 0.1,
                 max_slots: int = 16, hbm_budget: int = 0, sp2: "tbmd.tb_sp2_opts" = None,
                 fermi: "tbmd.tb_fermi_opts" = None, scf_tol: float = 1e-8, scf_max_iter: int = 200):
        self.ctx = ctx
        o = tbmd.tb_server_opts(max_slots=int(max_slots), hbm_budget=int(hbm_budget), kT=float(kT), xl=xl,
                                sp2=sp2 or sp2_opts("tf32x3", refine=3), fermi=fermi or fermi_opts(),
                                scf_tol=float(scf_tol), scf_max_iter=int(scf_max_iter))
        self.opts = o
        self.handle = tbmd.tb_server_create(ctx, p, o)
        self.natoms = []

    def footprint(self, types) -> int:
        return tbmd.tb_server_footprint(self.ctx, self.handle, types)

    def add(self, types, box, R0, v0, mass, n_occ) -> int:
        t = tbmd.tb_server_add(self.ctx, self.handle, types, box, R0, v0, mass, n_occ)
        self.natoms.append(len(types))
        return t

    def submit(self, traj: int) -> int:
        return tbmd.tb_server_submit(self.ctx, self.handle, traj)

    def poll(self, wait: bool = False, max_out: int = 64) -> list:
        return tbmd.tb_server_poll(self.ctx, self.handle, wait, max_out)

    def drain(self) -> list:
        """Poll until nothing is in flight and nothing queued can start; all
        completions.  Requests of trajectories still waiting for admission stay
        queued (nothing that runs can free memory for them): stats()["queued"]
        counts them."""
        out = []
        while True:
            out += self.poll(wait=True)
            if self.stats()["running"] == 0:
                # poll has dispatched whatever could start: nothing did
                out += self.poll(wait=False)
                return out

    def retire(self, traj: int):
        tbmd.tb_server_retire(self.ctx, self.handle, traj)

    def read(self, traj: int) -> dict:
        return tbmd.tb_server_read(self.ctx, self.handle, traj, self.natoms[traj])

    def stats(self) -> dict:
        return tbmd.tb_server_stats(self.ctx, self.handle)

    def replay(self, arrival_s, traj) -> list:
        return tbmd.tb_server_replay(self.ctx, self.handle, arrival_s, traj)

    def close(self):
        if self.handle:
            tbmd.tb_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nonorth_report_to_dict(buf: torch.Tensor) -> dict:
    raw = buf.detach().cpu().numpy().tobytes()
    r = tbmd.tb_nonorth_report.from_buffer_copy(raw[:ctypes.sizeof(tbmd.tb_nonorth_report)])
    return {k: getattr(r, k) for k, _ in tbmd.tb_nonorth_report._fields_}


class NonorthSolver:
    """dm_nonorth with its workspace sized for n: rho and W of (H, S)."""

    def __init__(self, ctx: tbmd.Context, n: int, kT: float = 0.0, sp2: "tbmd.tb_sp2_opts" = None,
                 fermi: "tbmd.tb_fermi_opts" = None, device="cuda"):
        self.ctx, self.n, self.kT = ctx, int(n), float(kT)
        self.sp2 = sp2 if sp2 is not None else sp2_opts("fp64")
        self.fermi = fermi if fermi is not None else fermi_opts()
        self.ws = Workspace(tbmd.dm_nonorth_workspace_size(n, kT, self.sp2, self.fermi), device)
        self.report = torch.zeros(ctypes.sizeof(tbmd.tb_nonorth_report), dtype=torch.uint8, device=device)
        self.sp2_report = new_report(device)
        self.fermi_report = torch.zeros(ctypes.sizeof(tbmd.tb_fermi_report), dtype=torch.uint8, device=device)
        self.mu = torch.full((4,), float("nan"), dtype=torch.float64, device=device)

    def __call__(self, H, S, n_occ: float, rho, W, stream=None):
        tbmd.dm_nonorth(self.ctx, H, S, self.n, n_occ, self.kT, self.sp2, self.fermi, self.mu, rho, W,
                        self.ws.ptr, self.ws.nbytes, self.sp2_report, self.fermi_report, self.report, stream)
        return rho
