"""The C ABI library builds for sm_103a and exports every function that
include/tbmd.h declares (no GPU needed: nothing is called)."""

import ctypes
import os

from paper_1203_6836_gb300 import build, tbmd


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = tbmd.header_functions()
    assert {"tb_ctx_create", "tb_build_H", "dm_sp2", "mulliken", "tb_forces", "xlbomd_step"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared in tbmd.h but not exported: {missing}"


def test_binding_covers_every_header_function():
    assert set(tbmd.header_functions()) <= set(tbmd._SIGS), set(tbmd.header_functions()) - set(tbmd._SIGS)


def test_status_strings_and_argument_errors_without_gpu():
    lib = tbmd.lib()
    assert lib.tb_status_string(tbmd.TB_ERR_ARG) == b"invalid argument"
    opts = tbmd.tb_sp2_opts(precision=0, max_iter=100, tol=1e-10, refine_iters=0, rule=0, refine_mode=1, tau=0.0,
                            bsr_blocks_per_row=0)
    assert lib.dm_sp2_workspace_size(0, ctypes.byref(opts), ctypes.byref(ctypes.c_size_t())) == tbmd.TB_ERR_ARG
    size = ctypes.c_size_t()
    assert lib.dm_sp2_workspace_size(4094, ctypes.byref(opts), ctypes.byref(size)) == tbmd.TB_OK
    assert size.value >= 2 * 8 * 4096 * 4096
    # a null context is rejected before anything touches the device
    assert lib.dm_sp2(None, None, 10, 5.0, ctypes.byref(opts), None, None, 0, None, None) == tbmd.TB_ERR_ARG
    # serving entry points reject a null server or context without touching the device
    so = tbmd.tb_server_opts(max_slots=4)
    out = ctypes.c_void_p()
    assert lib.tb_server_create(None, None, ctypes.byref(so), ctypes.byref(out)) == tbmd.TB_ERR_ARG
    n = ctypes.c_int()
    assert lib.tb_server_poll(None, 0, None, 0, ctypes.byref(n)) == tbmd.TB_ERR_ARG
    assert lib.tb_server_submit(None, 0, None) == tbmd.TB_ERR_ARG
    assert lib.tb_server_destroy(None) == tbmd.TB_OK
    assert ctypes.sizeof(tbmd.tb_completion) == 8 + 4 + 4 + 4 + 4 + 8 + 4 * 8 + 8 * 8


def test_fermi_options_and_layouts_without_gpu():
    """dm_fermi_workspace_size validates its options on the host; the workspace
    holds six matrices (the iterate's two buffers, A, Z, T, Y) with their tf32x3
    operand splits; the completion record carries the Fermi report's m at the
    offsets the server reads."""
    lib = tbmd.lib()
    size = ctypes.c_size_t()
    ok = tbmd.tb_fermi_opts(precision=tbmd.PREC["tf32x3"], m=14, ns_iters=3, mu_iters=30)
    assert lib.dm_fermi_workspace_size(4094, ctypes.byref(ok), ctypes.byref(size)) == tbmd.TB_OK
    assert size.value >= 6 * 12 * 4096 * 4096
    for bad in (dict(m=41), dict(ns_iters=13), dict(mu_iters=0), dict(mu_iters=41), dict(precision=99)):
        kw = dict(precision=tbmd.PREC["tf32x3"], m=14, ns_iters=3, mu_iters=30)
        kw.update(bad)
        o = tbmd.tb_fermi_opts(**kw)
        assert lib.dm_fermi_workspace_size(100, ctypes.byref(o), ctypes.byref(size)) == tbmd.TB_ERR_ARG, bad
    assert lib.dm_fermi_workspace_size(0, ctypes.byref(ok), ctypes.byref(size)) == tbmd.TB_ERR_ARG
    # the server copies the report's first ints: status, mu_iters, m
    assert tbmd.tb_fermi_report.status.offset == 0
    assert tbmd.tb_fermi_report.mu_iters.offset == 4
    assert tbmd.tb_fermi_report.m.offset == 8
    assert tbmd.tb_completion.solver_iters.offset == 16
    assert tbmd.tb_completion.solver_m.offset == 20
    assert tbmd.tb_completion.step.offset == 24



def test_block_sparse_workspaces_without_gpu():
    """The block-sparse SP2 and Fermi-expansion workspaces: n up to 131072
    (1024-bit row bitmaps), TB_ERR_UNSUPPORTED above; tf32x3 keeps only the
    FP32 master of each block (64 KB) where bf16x3 also stores two 32 KB
    operand splits; the expansion holds seven matrices where SP2 holds two;
    the capacity grows with the blocks per row."""
    lib = tbmd.lib()
    size = ctypes.c_size_t()

    def sp2(n, prec, bpr):
        o = tbmd.tb_sp2_opts(precision=tbmd.PREC[prec], max_iter=60, tol=1e-10, refine_iters=0, rule=0,
                             refine_mode=1, tau=1e-5, bsr_blocks_per_row=bpr)
        rc = lib.dm_sp2_workspace_size(n, ctypes.byref(o), ctypes.byref(size))
        return rc, size.value

    def foe(n, prec, bpr):
        o = tbmd.tb_fermi_opts(precision=tbmd.PREC[prec], m=14, ns_iters=3, mu_iters=30)
        rc = lib.dm_fermi_sparse_workspace_size(n, ctypes.byref(o), bpr, ctypes.byref(size))
        return rc, size.value

    assert sp2(131072, "tf32x3", 8)[0] == tbmd.TB_OK
    assert sp2(131073, "tf32x3", 8)[0] == tbmd.TB_ERR_UNSUPPORTED
    assert foe(131072, "tf32x3", 8)[0] == tbmd.TB_OK
    assert foe(131073, "tf32x3", 8)[0] == tbmd.TB_ERR_UNSUPPORTED
    assert foe(0, "tf32x3", 8)[0] == tbmd.TB_ERR_ARG
    nsb, bpr = 64, 16
    cap = nsb * bpr
    _, s_tf = sp2(nsb * 128, "tf32x3", bpr)
    _, s_bf = sp2(nsb * 128, "bf16x3", bpr)
    blk = 128 * 128
    assert s_tf >= 2 * cap * 4 * blk and s_tf < 2 * cap * 6 * blk  # FP32 masters, no splits
    assert s_bf - s_tf >= 2 * cap * 2 * 2 * blk - 2 * 1024  # bf16x3 adds hi and lo (2 B each)
    _, f_tf = foe(nsb * 128, "tf32x3", bpr)
    assert f_tf >= 7 * cap * 4 * blk and f_tf > 3 * s_tf
    assert foe(nsb * 128, "tf32x3", 2 * bpr)[1] > f_tf
