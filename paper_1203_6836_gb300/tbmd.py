"""ctypes binding of libtbmd (include/tbmd.h): the same names, argument
marshalling only.  Every computation runs in the CUDA library; when the
library is missing the calls raise instead of falling back to anything.

Array arguments accept raw device addresses (int) or objects with a
`data_ptr()` method (torch CUDA tensors); `stream` accepts a cudaStream_t
address, a torch stream, or None for the current torch stream.
"""

from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtbmd.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "tbmd.h")

TB_OK = 0
TB_ERR_ARG = -1
TB_ERR_NOT_CONVERGED = -2
TB_ERR_GAP = -3
TB_ERR_OOM = -4
TB_ERR_TIMEOUT = -5
TB_ERR_CUDA = -6
TB_ERR_UNSUPPORTED = -7
TB_SP2_FORM_AUTO = 0
TB_SP2_FORM_SINGLE = 1
TB_SP2_FORM_PAIRS = 2

TB_TYPE_O = 0
TB_TYPE_H = 1

PREC = {"fp64": 0, "tf32": 1, "tf32x3": 2, "bf16": 3, "bf16x3": 4}
XL_KMAX = 8


class TBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class tb_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "eps_s_O", "eps_p_O", "eps_s_H", "t_hop", "r_decay", "hubbard_u", "coulomb_k",
        "gamma_cut", "r1", "rcut", "n0_O", "n0_H", "pair_a", "pair_rho",
        "zeta_a2", "zeta_a3", "zeta_a4", "pair_a2", "pair_a3", "pair_a4")] + [
        ("gamma_form", ctypes.c_int), ("ewald_alpha", ctypes.c_double),
        ("overlap_s0", ctypes.c_double), ("overlap_rs", ctypes.c_double)]

    @classmethod
    def from_model(cls, m) -> "tb_params":
        """Copy the attributes of the same names from a model-constants object."""
        return cls(**{n: (int if t is ctypes.c_int else float)(getattr(m, n)) for n, t in cls._fields_})


class tb_system(ctypes.Structure):
    _fields_ = [("natoms", ctypes.c_int), ("norb", ctypes.c_int),
                ("types", ctypes.c_void_p), ("orb_off", ctypes.c_void_p), ("box", ctypes.c_double)]


class tb_sp2_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("refine_iters", ctypes.c_int), ("rule", ctypes.c_int), ("refine_mode", ctypes.c_int),
                ("tau", ctypes.c_double), ("bsr_blocks_per_row", ctypes.c_int)]


class tb_sp2_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("n", ctypes.c_int), ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double),
                ("trace", ctypes.c_double), ("idem_trace", ctypes.c_double),
                ("idem_fro", ctypes.c_double), ("branch_bits", ctypes.c_uint64 * 2),
                ("refine_bits", ctypes.c_uint64), ("block_products", ctypes.c_int64), ("blocks", ctypes.c_int64)]


class tb_xl_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("kappa", ctypes.c_double), ("alpha", ctypes.c_double),
                ("K", ctypes.c_int), ("c", ctypes.c_double * (XL_KMAX + 1))]


class tb_fermi_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("m", ctypes.c_int), ("ns_iters", ctypes.c_int),
                ("mu_iters", ctypes.c_int), ("trace_tol", ctypes.c_double)]


class tb_fermi_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("mu_iters", ctypes.c_int), ("m", ctypes.c_int), ("n", ctypes.c_int),
                ("mu", ctypes.c_double), ("trace", ctypes.c_double), ("trace_dd", ctypes.c_double),
                ("eps_min", ctypes.c_double), ("eps_max", ctypes.c_double)]


class tb_bsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nsb", ctypes.c_int), ("cap", ctypes.c_int), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class tb_md_state(ctypes.Structure):
    _fields_ = [("sys", tb_system), ("n_occ", ctypes.c_double),
                ("R", ctypes.c_void_p), ("v", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("n_hist", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("H", ctypes.c_void_p), ("D", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("energies", ctypes.c_void_p), ("sp2_report", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("step", ctypes.c_int64), ("kT", ctypes.c_double), ("fermi", tb_fermi_opts),
                ("mu", ctypes.c_void_p), ("fermi_report", ctypes.c_void_p),
                ("entropy_workspace", ctypes.c_void_p), ("entropy_workspace_bytes", ctypes.c_size_t),
                ("entropy", ctypes.c_void_p),
                ("S", ctypes.c_void_p), ("W", ctypes.c_void_p), ("vscc", ctypes.c_void_p),
                ("nonorth_workspace", ctypes.c_void_p), ("nonorth_workspace_bytes", ctypes.c_size_t),
                ("nonorth_report", ctypes.c_void_p),
                ("H_bsr", ctypes.c_void_p), ("D_bsr", ctypes.c_void_p),
                ("bsr_workspace", ctypes.c_void_p), ("bsr_workspace_bytes", ctypes.c_size_t)]


class tb_nonorth_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ns_iters", ctypes.c_int), ("ns_residual", ctypes.c_double)]


class tb_server_opts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("hbm_budget", ctypes.c_size_t), ("kT", ctypes.c_double),
                ("xl", tb_xl_params), ("sp2", tb_sp2_opts), ("fermi", tb_fermi_opts),
                ("scf_tol", ctypes.c_double), ("scf_max_iter", ctypes.c_int)]


class tb_completion(ctypes.Structure):
    _fields_ = [("request", ctypes.c_int64), ("traj", ctypes.c_int), ("status", ctypes.c_int),
                ("solver_iters", ctypes.c_int), ("solver_m", ctypes.c_int), ("step", ctypes.c_int64), ("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double),
                ("t_done", ctypes.c_double), ("gpu_ms", ctypes.c_double), ("energies", ctypes.c_double * 8)]


class tb_server_counts(ctypes.Structure):
    _fields_ = [("trajectories", ctypes.c_int), ("admitted", ctypes.c_int), ("waiting", ctypes.c_int),
                ("running", ctypes.c_int), ("queued", ctypes.c_int), ("bytes_in_use", ctypes.c_size_t),
                ("budget", ctypes.c_size_t), ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "tb_ctx_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "tb_ctx_destroy": (ctypes.c_int, [_P]),
    "tb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tb_ctx_last_error": (ctypes.c_char_p, [_P]),
    "tb_ctx_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "tb_ctx_sp2_launch_times": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]),
    "tb_ctx_set_grid_limit": (ctypes.c_int, [_P, ctypes.c_int]),
    "tb_ctx_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_ulonglong]),
    "tb_ctx_set_sp2_form": (ctypes.c_int, [_P, ctypes.c_int]),
    "tb_bsr_model_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "tb_build_H_bsr": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P,
                                      ctypes.POINTER(tb_bsr), _P, _P, ctypes.c_size_t, _P]),
    "dm_sp2_sparse": (ctypes.c_int, [_P, ctypes.POINTER(tb_bsr), ctypes.c_double, ctypes.POINTER(tb_sp2_opts),
                                     ctypes.POINTER(tb_bsr), _P, ctypes.c_size_t, _P, _P]),
    "dm_fermi_sparse_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tb_fermi_opts), ctypes.c_int,
                                                      ctypes.POINTER(ctypes.c_size_t)]),
    "dm_fermi_sparse": (ctypes.c_int, [_P, ctypes.POINTER(tb_bsr), ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(tb_fermi_opts), ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(tb_bsr), _P, _P, ctypes.c_size_t, _P, _P]),
    "mulliken_bsr": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), ctypes.POINTER(tb_bsr),
                                    _P, _P]),
    "tb_forces_bsr": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P,
                                     ctypes.POINTER(tb_bsr), ctypes.POINTER(tb_bsr), _P, _P, _P, _P, _P, _P,
                                     ctypes.c_size_t, _P]),
    "tb_build_HS": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P, _P, _P,
                                   _P, _P]),
    "dm_nonorth_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.POINTER(tb_sp2_opts),
                                                 ctypes.POINTER(tb_fermi_opts), ctypes.POINTER(ctypes.c_size_t)]),
    "dm_nonorth": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(tb_sp2_opts), ctypes.POINTER(tb_fermi_opts), _P, _P, _P, _P,
                                  ctypes.c_size_t, _P, _P, _P, _P]),
    "mulliken_nonorth": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P, _P]),
    "tb_forces_nonorth": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P, _P,
                                         _P, _P, _P, _P, _P, _P]),
    "tb_ctx_sp2_form_of": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "tb_build_H": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P, _P, _P]),
    "dm_sp2_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tb_sp2_opts),
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "dm_sp2": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(tb_sp2_opts), _P, _P,
                              ctypes.c_size_t, _P, _P]),
    "dm_sp2_static": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(tb_sp2_opts), _P, _P,
                                     _P]),
    "dm_fermi_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(tb_fermi_opts),
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "dm_fermi": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(tb_fermi_opts), _P, _P, _P, ctypes.c_size_t, _P, _P]),
    "dm_fermi_entropy_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "dm_fermi_entropy": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_double, _P, _P, _P, ctypes.c_size_t,
                                        _P]),
    "dm_sp2_grouped_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                     ctypes.POINTER(tb_sp2_opts), ctypes.POINTER(ctypes.c_size_t)]),
    "dm_sp2_grouped_plan": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), _P, ctypes.POINTER(tb_sp2_opts),
                                           ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "dm_sp2_grouped_run": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "mulliken": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P]),
    "tb_forces": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_system), _P, _P, _P, _P, _P,
                                 _P, _P, _P]),
    "xlbomd_init": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_md_state),
                                   ctypes.POINTER(tb_xl_params), ctypes.POINTER(tb_sp2_opts), ctypes.c_double,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), _P]),
    "xlbomd_step": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_md_state),
                                   ctypes.POINTER(tb_xl_params), ctypes.POINTER(tb_sp2_opts), _P]),
    "tb_server_create": (ctypes.c_int, [_P, ctypes.POINTER(tb_params), ctypes.POINTER(tb_server_opts),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "tb_server_destroy": (ctypes.c_int, [_P]),
    "tb_server_footprint": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "tb_server_add": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_double, _D, _D,
                                     _D, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "tb_server_submit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "tb_server_poll": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(tb_completion), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "tb_server_retire": (ctypes.c_int, [_P, ctypes.c_int]),
    "tb_server_read": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D, _D, _D]),
    "tb_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(tb_server_counts)]),
    "tb_server_replay": (ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(tb_completion)]),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/tbmd.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|char\s*\*|const char\s*\*|size_t)\s*\**\s*"
                                 r"([A-Za-z_]\w*)\s*\(", txt, flags=re.M)))


def lib() -> ctypes.CDLL:
    """The loaded libtbmd.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1203_6836_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


class Context:
    """tb_ctx bound to the current CUDA device."""

    def __init__(self):
        h = ctypes.c_void_p()
        rc = lib().tb_ctx_create(ctypes.byref(h))
        if rc != TB_OK:
            raise TBError(rc, "tb_ctx_create: " + lib().tb_status_string(rc).decode())
        self.handle = h

    def check(self, rc: int, what: str) -> int:
        if rc != TB_OK:
            msg = lib().tb_ctx_last_error(self.handle).decode()
            raise TBError(rc, f"{what}: {msg or lib().tb_status_string(rc).decode()}")
        return rc

    def close(self):
        if self.handle:
            lib().tb_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tb_ctx_set_profiling(ctx: Context, enable: bool) -> int:
    return ctx.check(lib().tb_ctx_set_profiling(ctx.handle, int(bool(enable))), "tb_ctx_set_profiling")


def tb_ctx_sp2_launch_times(ctx: Context, phase: int, cap: int = 130) -> list[float]:
    buf = (ctypes.c_float * cap)()
    cnt = ctypes.c_int()
    ctx.check(lib().tb_ctx_sp2_launch_times(ctx.handle, int(phase), buf, cap, ctypes.byref(cnt)),
              "tb_ctx_sp2_launch_times")
    return [float(buf[i]) for i in range(cnt.value)]


def tb_ctx_set_grid_limit(ctx: Context, max_ctas: int) -> int:
    return ctx.check(lib().tb_ctx_set_grid_limit(ctx.handle, int(max_ctas)), "tb_ctx_set_grid_limit")


def tb_ctx_set_wait_limit(ctx: Context, ns: int) -> int:
    return ctx.check(lib().tb_ctx_set_wait_limit(ctx.handle, int(ns)), "tb_ctx_set_wait_limit")


def tb_ctx_set_sp2_form(ctx: Context, form: int) -> int:
    return ctx.check(lib().tb_ctx_set_sp2_form(ctx.handle, int(form)), "tb_ctx_set_sp2_form")


def tb_ctx_sp2_form_of(ctx: Context, n: int) -> tuple[int, int]:
    """(form, CTAs) of the dense tensor-core projection dm_sp2 launches for size n."""
    f, c = ctypes.c_int(), ctypes.c_int()
    ctx.check(lib().tb_ctx_sp2_form_of(ctx.handle, int(n), ctypes.byref(f), ctypes.byref(c)), "tb_ctx_sp2_form_of")
    return f.value, c.value


def tb_bsr_model_workspace_size(natoms: int, norb: int) -> int:
    b = ctypes.c_size_t()
    rc = lib().tb_bsr_model_workspace_size(int(natoms), int(norb), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "tb_bsr_model_workspace_size")
    return b.value


def tb_build_H_bsr(ctx: Context, p: tb_params, sys: tb_system, R, n_aux, H: tb_bsr, v, workspace,
                   workspace_bytes: int, stream=None) -> int:
    return ctx.check(lib().tb_build_H_bsr(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), _ptr(n_aux),
                                          ctypes.byref(H), _ptr(v), _ptr(workspace), int(workspace_bytes),
                                          _stream(stream)), "tb_build_H_bsr")


def dm_sp2_sparse(ctx: Context, H: tb_bsr, n_occ: float, opts: tb_sp2_opts, D: tb_bsr, workspace,
                  workspace_bytes: int, report=None, stream=None) -> int:
    return ctx.check(lib().dm_sp2_sparse(ctx.handle, ctypes.byref(H), float(n_occ), ctypes.byref(opts),
                                         ctypes.byref(D), _ptr(workspace), int(workspace_bytes), _ptr(report),
                                         _stream(stream)), "dm_sp2_sparse")


def dm_fermi_sparse_workspace_size(n: int, opts: "tb_fermi_opts", blocks_per_row: int) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_fermi_sparse_workspace_size(int(n), ctypes.byref(opts), int(blocks_per_row), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_fermi_sparse_workspace_size")
    return int(b.value)


def dm_fermi_sparse(ctx: Context, H: tb_bsr, n_occ: float, kT: float, opts: "tb_fermi_opts", tau: float,
                    blocks_per_row: int, D: tb_bsr, mu, workspace, workspace_bytes: int, report=None,
                    stream=None) -> int:
    return ctx.check(lib().dm_fermi_sparse(ctx.handle, ctypes.byref(H), float(n_occ), float(kT), ctypes.byref(opts),
                                           float(tau), int(blocks_per_row), ctypes.byref(D), _ptr(mu),
                                           _ptr(workspace), int(workspace_bytes), _ptr(report), _stream(stream)),
                     "dm_fermi_sparse")


def mulliken_bsr(ctx: Context, p: tb_params, sys: tb_system, D: tb_bsr, q, stream=None) -> int:
    return ctx.check(lib().mulliken_bsr(ctx.handle, ctypes.byref(p), ctypes.byref(sys), ctypes.byref(D), _ptr(q),
                                        _stream(stream)), "mulliken_bsr")


def tb_forces_bsr(ctx: Context, p: tb_params, sys: tb_system, R, H: tb_bsr, D: tb_bsr, q, n_aux, v, F, energy,
                  workspace, workspace_bytes: int, stream=None) -> int:
    return ctx.check(lib().tb_forces_bsr(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), ctypes.byref(H),
                                         ctypes.byref(D), _ptr(q), _ptr(n_aux), _ptr(v), _ptr(F), _ptr(energy),
                                         _ptr(workspace), int(workspace_bytes), _stream(stream)), "tb_forces_bsr")


def tb_build_HS(ctx: Context, p: tb_params, sys: tb_system, R, n_aux, H, S, gamma, v, stream=None) -> int:
    return ctx.check(lib().tb_build_HS(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), _ptr(n_aux),
                                       _ptr(H), _ptr(S), _ptr(gamma), _ptr(v), _stream(stream)), "tb_build_HS")


def dm_nonorth_workspace_size(n: int, kT: float, sp2: tb_sp2_opts = None, fermi: tb_fermi_opts = None) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_nonorth_workspace_size(int(n), float(kT), ctypes.byref(sp2) if sp2 is not None else None,
                                         ctypes.byref(fermi) if fermi is not None else None, ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_nonorth_workspace_size")
    return b.value


def dm_nonorth(ctx: Context, H, S, n: int, n_occ: float, kT: float, sp2: tb_sp2_opts, fermi: tb_fermi_opts, mu,
               rho, W, workspace, workspace_bytes: int, sp2_report=None, fermi_report=None, report=None,
               stream=None) -> int:
    return ctx.check(lib().dm_nonorth(ctx.handle, _ptr(H), _ptr(S), int(n), float(n_occ), float(kT),
                                      ctypes.byref(sp2) if sp2 is not None else None,
                                      ctypes.byref(fermi) if fermi is not None else None, _ptr(mu), _ptr(rho),
                                      _ptr(W), _ptr(workspace), int(workspace_bytes), _ptr(sp2_report),
                                      _ptr(fermi_report), _ptr(report), _stream(stream)), "dm_nonorth")


def mulliken_nonorth(ctx: Context, p: tb_params, sys: tb_system, rho, S, q, stream=None) -> int:
    return ctx.check(lib().mulliken_nonorth(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(rho), _ptr(S),
                                            _ptr(q), _stream(stream)), "mulliken_nonorth")


def tb_forces_nonorth(ctx: Context, p: tb_params, sys: tb_system, R, rho, W, q, n_aux, v, gamma, F, energy,
                      stream=None) -> int:
    return ctx.check(lib().tb_forces_nonorth(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), _ptr(rho),
                                             _ptr(W), _ptr(q), _ptr(n_aux), _ptr(v), _ptr(gamma), _ptr(F),
                                             _ptr(energy), _stream(stream)), "tb_forces_nonorth")


def tb_build_H(ctx: Context, p: tb_params, sys: tb_system, R, n_aux, H, gamma, stream=None) -> int:
    return ctx.check(lib().tb_build_H(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), _ptr(n_aux),
                                      _ptr(H), _ptr(gamma), _stream(stream)), "tb_build_H")


def dm_sp2_workspace_size(n: int, opts: tb_sp2_opts) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_sp2_workspace_size(int(n), ctypes.byref(opts), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_sp2_workspace_size")
    return int(b.value)


def dm_sp2(ctx: Context, H, n: int, n_occ: float, opts: tb_sp2_opts, D, workspace, workspace_bytes: int,
           report=None, stream=None) -> int:
    return ctx.check(lib().dm_sp2(ctx.handle, _ptr(H), int(n), float(n_occ), ctypes.byref(opts), _ptr(D),
                                  _ptr(workspace), int(workspace_bytes), _ptr(report), _stream(stream)),
                     "dm_sp2")


def dm_fermi_workspace_size(n: int, opts: tb_fermi_opts) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_fermi_workspace_size(int(n), ctypes.byref(opts), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_fermi_workspace_size")
    return int(b.value)


def dm_fermi(ctx: Context, H, n: int, n_occ: float, kT: float, opts: tb_fermi_opts, D, mu, workspace,
             workspace_bytes: int, report=None, stream=None) -> int:
    return ctx.check(lib().dm_fermi(ctx.handle, _ptr(H), int(n), float(n_occ), float(kT), ctypes.byref(opts),
                                    _ptr(D), _ptr(mu), _ptr(workspace), int(workspace_bytes), _ptr(report),
                                    _stream(stream)), "dm_fermi")


def dm_fermi_entropy_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_fermi_entropy_workspace_size(int(n), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_fermi_entropy_workspace_size")
    return int(b.value)


def dm_fermi_entropy(ctx: Context, H, n: int, mu, kT: float, D, S, workspace, workspace_bytes: int,
                     stream=None) -> int:
    return ctx.check(lib().dm_fermi_entropy(ctx.handle, _ptr(H), int(n), _ptr(mu), float(kT), _ptr(D), _ptr(S),
                                            _ptr(workspace), int(workspace_bytes), _stream(stream)),
                     "dm_fermi_entropy")


def _ints(v):
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def dm_sp2_grouped_workspace_size(n_list, opts: tb_sp2_opts) -> int:
    b = ctypes.c_size_t()
    rc = lib().dm_sp2_grouped_workspace_size(len(n_list), _ints(n_list), ctypes.byref(opts), ctypes.byref(b))
    if rc != TB_OK:
        raise TBError(rc, "dm_sp2_grouped_workspace_size")
    return int(b.value)


def dm_sp2_grouped_plan(ctx: Context, n_list, nocc_list, H_list, D_list, reports, opts: tb_sp2_opts,
                        autotune: int, workspace, workspace_bytes: int, stream=None) -> int:
    """autotune: 0 one CTA per system, 1 time every launch form, 4 / 8 clusters of that size."""
    cnt = len(n_list)
    nocc = (ctypes.c_double * cnt)(*[float(x) for x in nocc_list])
    hp = (ctypes.c_void_p * cnt)(*[_ptr(h) for h in H_list])
    dp = (ctypes.c_void_p * cnt)(*[_ptr(d) for d in D_list])
    return ctx.check(lib().dm_sp2_grouped_plan(ctx.handle, cnt, _ints(n_list), nocc, hp, dp, _ptr(reports),
                                               ctypes.byref(opts), int(autotune), _ptr(workspace),
                                               int(workspace_bytes), _stream(stream)), "dm_sp2_grouped_plan")


def dm_sp2_grouped_run(ctx: Context, workspace, stream=None) -> int:
    cfg = ctypes.c_int()
    ctx.check(lib().dm_sp2_grouped_run(ctx.handle, _ptr(workspace), ctypes.byref(cfg), _stream(stream)),
              "dm_sp2_grouped_run")
    return int(cfg.value)


SP2_STATIC_MAX_N = 512


def dm_sp2_static(ctx: Context, H, n: int, n_occ: float, opts: tb_sp2_opts, D, report=None, stream=None) -> int:
    """FP64 SP2 with the library's static scratch (no workspace argument)."""
    return ctx.check(lib().dm_sp2_static(ctx.handle, _ptr(H), int(n), float(n_occ), ctypes.byref(opts), _ptr(D),
                                         _ptr(report), _stream(stream)), "dm_sp2_static")


def mulliken(ctx: Context, p: tb_params, sys: tb_system, D, q, stream=None) -> int:
    return ctx.check(lib().mulliken(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(D), _ptr(q),
                                    _stream(stream)), "mulliken")


def tb_forces(ctx: Context, p: tb_params, sys: tb_system, R, D, q, n_aux, gamma, F, energy, stream=None) -> int:
    return ctx.check(lib().tb_forces(ctx.handle, ctypes.byref(p), ctypes.byref(sys), _ptr(R), _ptr(D), _ptr(q),
                                     _ptr(n_aux), _ptr(gamma), _ptr(F), _ptr(energy), _stream(stream)),
                     "tb_forces")


def xlbomd_init(ctx: Context, p: tb_params, st: tb_md_state, xp: tb_xl_params, so: tb_sp2_opts,
                scf_tol: float, scf_max_iter: int, stream=None) -> int:
    it = ctypes.c_int()
    ctx.check(lib().xlbomd_init(ctx.handle, ctypes.byref(p), ctypes.byref(st), ctypes.byref(xp),
                                ctypes.byref(so), float(scf_tol), int(scf_max_iter), ctypes.byref(it),
                                _stream(stream)), "xlbomd_init")
    return int(it.value)


def xlbomd_step(ctx: Context, p: tb_params, st: tb_md_state, xp: tb_xl_params, so: tb_sp2_opts,
                stream=None) -> int:
    return ctx.check(lib().xlbomd_step(ctx.handle, ctypes.byref(p), ctypes.byref(st), ctypes.byref(xp),
                                       ctypes.byref(so), _stream(stream)), "xlbomd_step")


# ------------------------------------------------------------------ serving

def _dptr(a):
    """Pointer to a C-contiguous float64 NumPy array (or None)."""
    return None if a is None else a.ctypes.data_as(_D)


def tb_server_create(ctx: Context, p: tb_params, opts: tb_server_opts) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    ctx.check(lib().tb_server_create(ctx.handle, ctypes.byref(p), ctypes.byref(opts), ctypes.byref(h)),
              "tb_server_create")
    return h


def tb_server_destroy(server) -> int:
    return lib().tb_server_destroy(server)


def tb_server_footprint(ctx: Context, server, types) -> int:
    import numpy as np
    t = np.ascontiguousarray(types, dtype=np.int32)
    b = ctypes.c_size_t()
    ctx.check(lib().tb_server_footprint(server, len(t), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        ctypes.byref(b)), "tb_server_footprint")
    return int(b.value)


def tb_server_add(ctx: Context, server, types, box: float, R0, v0, mass, n_occ: float) -> int:
    import numpy as np
    t = np.ascontiguousarray(types, dtype=np.int32)
    R = np.ascontiguousarray(R0, dtype=np.float64)
    v = np.ascontiguousarray(v0, dtype=np.float64)
    m = np.ascontiguousarray(mass, dtype=np.float64)
    out = ctypes.c_int()
    ctx.check(lib().tb_server_add(server, len(t), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(box),
                                  _dptr(R), _dptr(v), _dptr(m), float(n_occ), ctypes.byref(out)), "tb_server_add")
    return int(out.value)


def tb_server_submit(ctx: Context, server, traj: int) -> int:
    rid = ctypes.c_int64()
    ctx.check(lib().tb_server_submit(server, int(traj), ctypes.byref(rid)), "tb_server_submit")
    return int(rid.value)


def tb_server_poll(ctx: Context, server, wait: bool = False, max_out: int = 64) -> list:
    buf = (tb_completion * max_out)()
    n = ctypes.c_int()
    ctx.check(lib().tb_server_poll(server, int(bool(wait)), buf, max_out, ctypes.byref(n)), "tb_server_poll")
    return [buf[i] for i in range(n.value)]


def tb_server_retire(ctx: Context, server, traj: int) -> int:
    return ctx.check(lib().tb_server_retire(server, int(traj)), "tb_server_retire")


def tb_server_read(ctx: Context, server, traj: int, natoms: int) -> dict:
    import numpy as np
    R = np.zeros((natoms, 3))
    v = np.zeros((natoms, 3))
    q = np.zeros(natoms)
    n = np.zeros(natoms)
    E = np.zeros(8)
    ctx.check(lib().tb_server_read(server, int(traj), _dptr(R), _dptr(v), _dptr(q), _dptr(n), _dptr(E)),
              "tb_server_read")
    return {"R": R, "v": v, "q": q, "n": n, "E": E}


def tb_server_stats(ctx: Context, server) -> dict:
    c = tb_server_counts()
    ctx.check(lib().tb_server_stats(server, ctypes.byref(c)), "tb_server_stats")
    return {k: getattr(c, k) for k, _ in tb_server_counts._fields_}


def tb_server_replay(ctx: Context, server, arrival_s, traj) -> list:
    import numpy as np
    a = np.ascontiguousarray(arrival_s, dtype=np.float64)
    t = np.ascontiguousarray(traj, dtype=np.int32)
    out = (tb_completion * len(a))()
    ctx.check(lib().tb_server_replay(server, len(a), _dptr(a), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     out), "tb_server_replay")
    return list(out)
