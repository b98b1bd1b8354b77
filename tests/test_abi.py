"""CPU-side checks of the C ABI: the shared library loads, exports every
symbol include/sla.h declares, and rejects bad arguments synchronously
(before any CUDA call, so these run without a GPU)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2601_13994_b300 import _lib as L
from paper_2601_13994_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def setup_module(module):
    B.build()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(sla_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert "sla_cg" in names and "sla_spmv" in names
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_status_strings():
    lib = L.lib()
    assert b"sm_103a" in lib.sla_version()
    for code, name in L.STATUS_NAMES.items():
        assert lib.sla_status_string(code).decode() == name
    assert lib.sla_status_string(12345) == b"UNKNOWN"


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "sla.h")).read()
    consts = dict(re.findall(r"#define (SLA_\w+) \(?(-?\d+)\)?", src))
    for k, v in consts.items():
        if hasattr(L, k):
            assert getattr(L, k) == int(v), k


def test_workspace_size_query():
    b1 = L.workspace_size(L.SLA_WS_CG, 1000, 5000)
    b2 = L.workspace_size(L.SLA_WS_CG, 2000, 5000)
    assert b1 % 256 == 0 and b2 > b1 >= 5 * 8 * 1000
    with pytest.raises(L.SlaError):
        L.workspace_size(999, 10, 10)
    with pytest.raises(L.SlaError):
        L.workspace_size(L.SLA_WS_CG, -1, 10)


def test_pipelined_flag_arguments_rejected_without_launch():
    """SLA_FLAG_CG_PIPELINED: only sla_cg and the CG adjoint accept it, never
    with the host loop or without the cooperative form, and sla_cg then
    needs the larger SLA_WS_CG_PIPELINED workspace (checked before any
    launch, so fake pointers serve)."""
    lib = L.lib()
    n = 1000
    wp = L.workspace_size(L.SLA_WS_CG_PIPELINED, n, 5000)
    wc = L.workspace_size(L.SLA_WS_CG, n, 5000)
    assert wp % 256 == 0 and wc % 256 == 0 and wp >= 8 * 8 * n
    # the CG workspace holds 5 n-vectors and the scaled values (nnz doubles)
    assert wc >= 8 * (5 * n + 5000)
    assert L.workspace_size(L.SLA_WS_ADJOINT, n, 5000) >= wp
    fake = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    A = L.SlaCsr(n, 5000, fake, fake)
    P = L.SLA_FLAG_CG_PIPELINED
    for extra in (L.SLA_FLAG_HOST_LOOP, L.SLA_FLAG_NO_COOP):
        o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, P | extra)
        assert lib.sla_cg(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                          ws, wp, None) == L.SLA_ERR_INVALID
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, P)
    assert lib.sla_cg(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                      ws, wp - 256, None) == L.SLA_ERR_WORKSPACE
    assert lib.sla_bicgstab(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                            ws, 1 << 30, None) == L.SLA_ERR_INVALID
    assert lib.sla_adjoint_backward(ctypes.byref(A), None, fake, fake, fake, ctypes.c_void_p(0x2000),
                                    ctypes.c_void_p(0x3000), L.SLA_ADJ_BICGSTAB, ctypes.byref(o), fake,
                                    ws, 1 << 30, None) == L.SLA_ERR_INVALID
    o8 = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 8)
    assert lib.sla_cg(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o8), fake,
                      ws, 1 << 30, None) == L.SLA_ERR_INVALID


def test_bad_arguments_rejected_without_launch():
    lib = L.lib()
    A = L.SlaCsr(10, 20, None, None)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    # null pattern pointers
    assert lib.sla_spmv(ctypes.byref(A), None, None, None, None) == L.SLA_ERR_INVALID
    assert lib.sla_cg(ctypes.byref(A), None, None, None, ctypes.byref(o), None, None, 0, None) == L.SLA_ERR_INVALID
    assert lib.sla_cg(None, None, None, None, None, None, None, 0, None) == L.SLA_ERR_INVALID
    # negative sizes
    A2 = L.SlaCsr(-1, 0, None, None)
    assert lib.sla_spmv(ctypes.byref(A2), None, None, None, None) == L.SLA_ERR_INVALID
    # bad options / workspace (fake but non-null pointers; rejected before use)
    fake = ctypes.c_void_p(0x1000)
    A3 = L.SlaCsr(10, 20, fake, fake)
    bad = L.SlaOpts(-1.0, 0.0, 100, 2, 1, 0, 0)
    assert lib.sla_cg(ctypes.byref(A3), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(bad), fake,
                      fake, 1 << 20, None) == L.SLA_ERR_INVALID
    o2 = L.SlaOpts(1e-8, 0.0, 100, 2, 7, 0, 0)
    assert lib.sla_cg(ctypes.byref(A3), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o2), fake,
                      ctypes.c_void_p(0x100000), 1 << 20, None) == L.SLA_ERR_INVALID
    o3 = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    # misaligned and undersized workspace
    assert lib.sla_cg(ctypes.byref(A3), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o3), fake,
                      ctypes.c_void_p(0x100010), 1 << 20, None) == L.SLA_ERR_WORKSPACE
    assert lib.sla_cg(ctypes.byref(A3), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o3), fake,
                      ctypes.c_void_p(0x100000), 16, None) == L.SLA_ERR_WORKSPACE
    # x aliasing b
    assert lib.sla_cg(ctypes.byref(A3), fake, fake, fake, ctypes.byref(o3), fake,
                      ctypes.c_void_p(0x100000), 1 << 20, None) == L.SLA_ERR_INVALID


def test_adjoint_rejects_aliased_outputs_without_launch():
    """lambda is written into grad_b before the gradient pass reads x, so
    grad_b aliasing x, or grad_val overlapping x or grad_b, is rejected
    before anything is enqueued (fake pointers: a launch would fault)."""
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 20, fake, fake)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    ws, big = ctypes.c_void_p(0x100000), ctypes.c_size_t(1 << 40)
    x, gx, gb, gv = 0x10000, 0x20000, 0x30000, 0x40000

    def call(x, gx, gb, gv):
        return lib.sla_adjoint_backward(ctypes.byref(A), None, fake, ctypes.c_void_p(x), ctypes.c_void_p(gx),
                                        ctypes.c_void_p(gb), ctypes.c_void_p(gv), L.SLA_ADJ_CG,
                                        ctypes.byref(o), fake, ws, big, None)
    assert call(x, gx, x, gv) == L.SLA_ERR_INVALID             # grad_b == x
    assert call(x, gx, gx, gv) == L.SLA_ERR_INVALID            # grad_b == grad_x
    assert call(x, gx, gb, x + 8 * 9) == L.SLA_ERR_INVALID     # grad_val overlaps x's last entry
    assert call(x, gx, gb, gb - 8 * 19) == L.SLA_ERR_INVALID   # grad_val's last entry is grad_b[0]
    # the multi-RHS adjoint applies the same rule over its k columns
    assert lib.sla_adjoint_backward_multi(ctypes.byref(A), fake, 4, ctypes.c_void_p(x), ctypes.c_void_p(gx),
                                          ctypes.c_void_p(gb), ctypes.c_void_p(x + 8 * 39), ctypes.byref(o),
                                          fake, ws, big, None) == L.SLA_ERR_INVALID


def test_batched_bicgstab_and_list_transpose_reject_bad_arguments_without_launch():
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 20, fake, fake)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    ws, big = ctypes.c_void_p(0x100000), ctypes.c_size_t(1 << 40)
    x = ctypes.c_void_p(0x2000)

    def shared(batch=4, opts=o, b=fake, xx=x, cfg=0, w=ws, nb=big):
        return lib.sla_bicgstab_batched_shared(ctypes.byref(A), batch, fake, b, xx, ctypes.byref(opts), fake,
                                               cfg, w, nb, None)
    assert shared(batch=-1) == L.SLA_ERR_INVALID
    assert shared(batch=0) == L.SLA_OK                                      # nothing to do
    assert shared(xx=fake) == L.SLA_ERR_INVALID                             # b == x
    assert shared(cfg=32) == L.SLA_ERR_INVALID                              # unknown config bit
    assert shared(cfg=4) == L.SLA_ERR_INVALID                               # unknown block size code
    flags = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, L.SLA_FLAG_HOST_LOOP)
    assert shared(opts=flags) == L.SLA_ERR_INVALID                          # flags not offered
    ggt = L.SlaOpts(1e-8, 0.0, 100, 2, L.SLA_PRECOND_GGT, 0, 0)
    assert shared(opts=ggt) == L.SLA_ERR_INVALID
    need = L.workspace_size(L.SLA_WS_BATCHED, 10, 20, 4)
    assert shared(nb=need - 1) == L.SLA_ERR_WORKSPACE
    assert shared(w=ctypes.c_void_p(0x100010)) == L.SLA_ERR_WORKSPACE
    assert lib.sla_bicgstab_batched_list(3, 10, 30, None, fake, fake, fake, fake, fake, x, None,
                                         ctypes.byref(o), fake, 0, ws, big, None) == L.SLA_ERR_INVALID
    assert lib.sla_bicgstab_batched_list(3, 10, 30, fake, fake, fake, fake, fake, fake, fake, None,
                                         ctypes.byref(o), fake, 0, ws, big, None) == L.SLA_ERR_INVALID
    for cfg in (64, 1 << 12, 1 << 4 | 1 << 7):                              # unknown list config bits
        assert lib.sla_bicgstab_batched_list(3, 10, 30, fake, fake, fake, fake, fake, fake, x, None,
                                             ctypes.byref(o), fake, cfg, ws, big, None) == L.SLA_ERR_INVALID
    assert shared(cfg=1 << 8) == L.SLA_ERR_INVALID                          # team bits: lists only
    # list transpose: empty list, null pointers, aliasing, workspace
    assert lib.sla_csr_list_transpose(0, 0, 0, None, None, None, None, None, None, None, None, 0,
                                      None) == L.SLA_OK
    assert lib.sla_csr_list_transpose(2, 10, 20, fake, fake, fake, fake, None, x, x, ws, big,
                                      None) == L.SLA_ERR_INVALID
    assert lib.sla_csr_list_transpose(2, 10, 20, fake, fake, fake, fake, fake, x, ctypes.c_void_p(0x3000),
                                      ws, big, None) == L.SLA_ERR_INVALID        # rowptrT == rowptr
    lt = L.workspace_size(L.SLA_WS_LIST_TRANSPOSE, 10, 20)
    assert lt >= L.workspace_size(L.SLA_WS_TRANSPOSE, 10, 20)
    assert lib.sla_csr_list_transpose(2, 10, 20, fake, fake, fake, fake, ctypes.c_void_p(0x4000), x,
                                      ctypes.c_void_p(0x3000), ws, lt - 1, None) == L.SLA_ERR_WORKSPACE
    # batched gather: overlapping output
    assert lib.sla_gather_values_batched(2, 20, fake, x, ctypes.c_void_p(0x2000 + 8 * 39), None) == L.SLA_ERR_INVALID
    assert lib.sla_gather_values_batched(-1, 20, fake, x, fake, None) == L.SLA_ERR_INVALID


def test_batched_adjoint_arguments_rejected_without_launch():
    """sla_adjoint_backward_batched_*: every rejection comes before the first
    enqueue (fake pointers: a launch would fault), including a BiCGStab
    config or option that the batched solver would refuse only after the
    values gather."""
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 20, fake, fake)
    AT = L.SlaCsrT(fake, fake, fake)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    ws, big = ctypes.c_void_p(0x100000), ctypes.c_size_t(1 << 40)
    x, gx, gb, gv = 0x10000, 0x20000, 0x30000, 0x40000       # 4 systems: 40 rows, 80 entries

    def shared(x=x, gx=gx, gb=gb, gv=gv, method=L.SLA_ADJ_CG, opts=o, at=None, cfg=0, w=ws, nb=big, batch=4):
        return lib.sla_adjoint_backward_batched_shared(
            ctypes.byref(A), None if at is None else ctypes.byref(at), batch, fake, ctypes.c_void_p(x),
            ctypes.c_void_p(gx), ctypes.c_void_p(gb), ctypes.c_void_p(gv), method, ctypes.byref(opts), fake,
            cfg, w, nb, None)
    assert shared(batch=0) == L.SLA_OK
    assert shared(batch=-1) == L.SLA_ERR_INVALID
    assert shared(method=7) == L.SLA_ERR_INVALID
    assert shared(opts=L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, L.SLA_FLAG_HOST_LOOP)) == L.SLA_ERR_INVALID
    assert shared(gb=x) == L.SLA_ERR_INVALID                    # grad_b == x
    assert shared(gb=gx + 8 * 39) == L.SLA_ERR_INVALID          # grad_b starts at grad_x's last entry
    assert shared(gv=x + 8 * 39) == L.SLA_ERR_INVALID           # grad_val overlaps x's last entry
    assert shared(gv=gb - 8 * 79) == L.SLA_ERR_INVALID          # grad_val's last entry is grad_b[0]
    need = L.workspace_size(L.SLA_WS_ADJOINT_BATCHED, 10, 20, 4)
    assert need >= L.workspace_size(L.SLA_WS_BATCHED, 10, 20, 4) + 8 * 80 and need % 256 == 0
    assert shared(nb=need - 1) == L.SLA_ERR_WORKSPACE
    assert shared(w=ctypes.c_void_p(0x100010)) == L.SLA_ERR_WORKSPACE
    bic = L.SLA_ADJ_BICGSTAB
    assert shared(method=bic) == L.SLA_ERR_INVALID              # no transpose
    assert shared(method=bic, at=AT, cfg=32) == L.SLA_ERR_INVALID        # team bits: lists only
    assert shared(method=bic, at=AT, cfg=4) == L.SLA_ERR_INVALID         # unknown block size code
    assert shared(method=bic, at=AT, opts=L.SlaOpts(-1.0, 0.0, 100, 2, 1, 0, 0)) == L.SLA_ERR_INVALID
    assert shared(method=bic, at=AT, opts=L.SlaOpts(1e-8, 0.0, 100, 2, L.SLA_PRECOND_GGT, 0, 0)) == \
        L.SLA_ERR_INVALID

    def lst(n_off=fake, rpt=fake, gb=gb, gv=gv, method=bic, cfg=0, nb=big):
        return lib.sla_adjoint_backward_batched_list(
            4, 10, 40, 80, n_off, fake, fake, fake, rpt, fake, fake, fake, ctypes.c_void_p(x),
            ctypes.c_void_p(gx), ctypes.c_void_p(gb), ctypes.c_void_p(gv), None, method, ctypes.byref(o), fake,
            cfg, ws, nb, None)
    assert lst(n_off=None) == L.SLA_ERR_INVALID
    assert lst(rpt=None) == L.SLA_ERR_INVALID                   # BiCGStab needs the transposes
    assert lst(cfg=64) == L.SLA_ERR_INVALID                     # unknown list config bit
    assert lst(gb=x + 8) == L.SLA_ERR_INVALID
    assert lst(gv=gb + 8 * 39) == L.SLA_ERR_INVALID
    assert lst(method=-1) == L.SLA_ERR_INVALID
    need_l = L.workspace_size(L.SLA_WS_ADJOINT_BATCHED, 40, 80, 1)
    assert need_l == need
    assert lst(nb=need_l - 1) == L.SLA_ERR_WORKSPACE


def test_multi_rhs_arguments_rejected_without_launch():
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 20, fake, fake)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, 1, 0, 0)
    big = ctypes.c_size_t(1 << 40)
    ws = ctypes.c_void_p(0x100000)
    # k out of range
    for k in (0, -1, L.SLA_MULTI_MAX_RHS + 1):
        assert lib.sla_cg_multi(ctypes.byref(A), fake, k, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                                ws, big, None) == L.SLA_ERR_INVALID
    # the factored preconditioner is not offered for several right-hand sides
    og = L.SlaOpts(1e-8, 0.0, 100, 2, 2, 0, 0)
    assert lib.sla_cg_multi(ctypes.byref(A), fake, 4, fake, ctypes.c_void_p(0x2000), ctypes.byref(og), fake,
                            ws, big, None) == L.SLA_ERR_INVALID
    # b aliasing x
    assert lib.sla_cg_multi(ctypes.byref(A), fake, 4, fake, fake, ctypes.byref(o), fake, ws, big,
                            None) == L.SLA_ERR_INVALID
    # workspace too small / misaligned
    need = L.workspace_size(L.SLA_WS_CG_MULTI, 10, 20, 4)
    assert lib.sla_cg_multi(ctypes.byref(A), fake, 4, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                            ws, need - 1, None) == L.SLA_ERR_WORKSPACE
    assert lib.sla_cg_multi(ctypes.byref(A), fake, 4, fake, ctypes.c_void_p(0x2000), ctypes.byref(o), fake,
                            ctypes.c_void_p(0x100010), big, None) == L.SLA_ERR_WORKSPACE
    # adjoint: grad_b aliasing x
    assert lib.sla_adjoint_backward_multi(ctypes.byref(A), fake, 4, fake, ctypes.c_void_p(0x3000), fake,
                                          ctypes.c_void_p(0x4000), ctypes.byref(o), fake, ws, big,
                                          None) == L.SLA_ERR_INVALID


def test_multi_rhs_workspace_grows_with_width():
    b1 = L.workspace_size(L.SLA_WS_CG_MULTI, 1000, 5000, 1)
    b16 = L.workspace_size(L.SLA_WS_CG_MULTI, 1000, 5000, 16)
    b13 = L.workspace_size(L.SLA_WS_CG_MULTI, 1000, 5000, 13)
    assert b16 == b13 > b1 and b16 >= 6 * 8 * 1000 * 16


def test_grid_barrier_selftest_rejects_bad_arguments_without_launch():
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    assert lib.sla_selftest_grid_barrier(4, -1, 1000, 1, None, None) == L.SLA_ERR_INVALID
    assert lib.sla_selftest_grid_barrier(0, -1, 1000, 1, fake, None) == L.SLA_ERR_INVALID
    assert lib.sla_selftest_grid_barrier(4, 4, 1000, 1, fake, None) == L.SLA_ERR_INVALID
    assert lib.sla_selftest_grid_barrier(4, -1, 0, 1, fake, None) == L.SLA_ERR_INVALID
    assert lib.sla_selftest_grid_barrier(4, -1, 1000, -1, fake, None) == L.SLA_ERR_INVALID


def test_spmv_scheme_rule_and_merge_argument_checks():
    lib = L.lib()
    # stencil-like: short rows -> row kernels; one dominant long row -> merge path
    assert lib.sla_spmv_scheme(1 << 20, 7 << 20, 7) == L.SLA_SPMV_ROWS
    assert lib.sla_spmv_scheme(100000, 300000, 100000) == L.SLA_SPMV_MERGE
    assert lib.sla_spmv_scheme(100000, 300000, 256) == L.SLA_SPMV_ROWS        # not above 256
    assert lib.sla_spmv_scheme(200000, 1431355, 4824) == L.SLA_SPMV_MERGE
    assert lib.sla_spmv_scheme(1 << 20, 5 << 20, 700) == L.SLA_SPMV_ROWS      # 6 Mi items: limit 768
    assert lib.sla_spmv_scheme(1 << 20, 5 << 20, 800) == L.SLA_SPMV_MERGE
    # above 4 Mi rows a long row goes to a warp: the limit is (n + nnz) / 256
    assert lib.sla_spmv_scheme(1 << 23, 7 << 23, 200000) == L.SLA_SPMV_ROWS
    assert lib.sla_spmv_scheme(1 << 23, 7 << 23, 300000) == L.SLA_SPMV_MERGE
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 20, fake, fake)
    assert lib.sla_spmv_merge(None, fake, fake, ctypes.c_void_p(0x2000), fake, 1 << 20, None) == L.SLA_ERR_INVALID
    assert lib.sla_spmv_merge(ctypes.byref(A), fake, fake, fake, fake, 1 << 20, None) == L.SLA_ERR_INVALID  # x == y
    assert lib.sla_spmv_merge(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), None, 0,
                              None) == L.SLA_ERR_WORKSPACE
    assert L.workspace_size(L.SLA_WS_SPMV_MERGE, 10, 20) >= 4 * 256


def test_column_colouring_is_a_distance2_colouring():
    """sla_colour_columns (host): columns sharing a row never share a colour,
    on the 2D/3D stencils, an FEM pattern and a random pattern with empty
    rows; the 5-point stencil needs at least 5 colours (a row has 5 columns);
    malformed patterns are rejected."""
    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rng = np.random.default_rng(0)
    rows = []
    for i in range(300):
        k = 0 if i % 17 == 0 else int(rng.integers(1, 12))
        rows.append(np.unique(rng.integers(0, 300, size=k)))
    rp_r = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int32)
    c_r = np.concatenate(rows).astype(np.int32)
    pats = [I.poisson2d(40)[:2], I.diffusion3d_random(9, 1)[:2], I.fem_p1_laplacian(30, 2)[:2], (rp_r, c_r)]
    for rp, c in pats:
        colour, k = sla.colour_columns(rp, c)
        n = len(rp) - 1
        assert colour.shape == (n,) and colour.min() >= 0 and colour.max() == k - 1
        maxlen = int(np.diff(rp).max())
        assert maxlen <= k <= maxlen * maxlen
        for i in range(n):
            cs = colour[c[rp[i]:rp[i + 1]]]
            assert np.unique(cs).size == cs.size
    assert sla.colour_columns(*I.poisson2d(40)[:2])[1] >= 5
    assert sla.colour_columns(np.zeros(1, np.int32), np.zeros(0, np.int32))[1] == 0
    lib = L.lib()
    k = ctypes.c_int32(0)
    out = np.empty(2, np.int32)
    bad_rp = np.array([0, 2, 1], np.int32)
    bad_c = np.array([0, 1], np.int32)
    assert lib.sla_colour_columns(2, bad_rp.ctypes.data_as(ctypes.c_void_p), bad_c.ctypes.data_as(ctypes.c_void_p),
                                  out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)) == L.SLA_ERR_INVALID
    rp2 = np.array([0, 1, 2], np.int32)
    c2 = np.array([0, 5], np.int32)
    assert lib.sla_colour_columns(2, rp2.ctypes.data_as(ctypes.c_void_p), c2.ctypes.data_as(ctypes.c_void_p),
                                  out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)) == L.SLA_ERR_INVALID


def test_eigsh_arguments_rejected_without_launch():
    """sla_eigsh / sla_eig_grad_values argument checks (before any launch)."""
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    n = 100
    A = L.SlaCsr(n, 300, fake, fake)
    need = L.workspace_size(L.SLA_WS_EIGSH, n, 300, 6)
    assert need >= 4 * 8 * n * 18
    with pytest.raises(L.SlaError):
        L.workspace_size(L.SLA_WS_EIGSH, n, 300, 9)
    ok = L.SlaOpts(1e-8, 0.0, 100, 0, 1, 0, 0)
    out = ctypes.c_void_p(0x2000)
    for k in (0, 9, n + 1):
        assert lib.sla_eigsh(ctypes.byref(A), fake, k, out, out, ctypes.byref(ok), fake, ws, need,
                             None) == L.SLA_ERR_INVALID
    for bad in (L.SlaOpts(0.0, 0.0, 100, 0, 1, 0, 0), L.SlaOpts(1e-8, 0.0, -1, 0, 1, 0, 0),
                L.SlaOpts(1e-8, 0.0, 100, 0, 2, 0, 0), L.SlaOpts(1e-8, 0.0, 100, 0, 1, 0, 1)):
        assert lib.sla_eigsh(ctypes.byref(A), fake, 6, out, out, ctypes.byref(bad), fake, ws, need,
                             None) == L.SLA_ERR_INVALID
    assert lib.sla_eigsh(ctypes.byref(A), fake, 6, out, out, ctypes.byref(ok), fake, ws, need - 256,
                         None) == L.SLA_ERR_WORKSPACE
    assert lib.sla_eigsh(ctypes.byref(A), fake, 6, None, out, ctypes.byref(ok), fake, ws, need,
                         None) == L.SLA_ERR_INVALID
    assert lib.sla_eig_grad_values(ctypes.byref(A), 0, fake, fake, fake, None) == L.SLA_ERR_INVALID
    assert lib.sla_eig_grad_values(ctypes.byref(A), 9, fake, fake, fake, None) == L.SLA_ERR_INVALID


def test_eig_vector_adjoint_arguments_rejected_without_launch():
    """sla_eig_vector_adjoint / sla_eig_vector_grad_values argument checks
    (before any launch) and the workspace kind's range."""
    lib = L.lib()
    fake = ctypes.c_void_p(0x1000)
    ws = ctypes.c_void_p(0x100000)
    n = 100
    A = L.SlaCsr(n, 300, fake, fake)
    need = L.workspace_size(L.SLA_WS_EIG_ADJOINT, n, 300, 6)
    assert need >= 3 * 8 * n * 6
    for kb in (0, 9):
        with pytest.raises(L.SlaError):
            L.workspace_size(L.SLA_WS_EIG_ADJOINT, n, 300, kb)
    ok = L.SlaOpts(1e-10, 0.0, 100, 0, 1, 0, 0)

    def call(k=6, opts=ok, lam=fake, V=fake, gV=fake, mu=fake, w=ws, nb=need):
        return lib.sla_eig_vector_adjoint(ctypes.byref(A), fake, k, lam, V, gV, mu, ctypes.byref(opts), fake,
                                          w, nb, None)
    for k in (0, 9, n + 1):
        assert call(k=k) == L.SLA_ERR_INVALID
    for bad in (L.SlaOpts(-1.0, 0.0, 100, 0, 1, 0, 0), L.SlaOpts(1e-8, -1.0, 100, 0, 1, 0, 0),
                L.SlaOpts(1e-8, 0.0, -1, 0, 1, 0, 0), L.SlaOpts(1e-8, 0.0, 100, 0, 2, 0, 0),
                L.SlaOpts(1e-8, 0.0, 100, 0, 1, 1, 0), L.SlaOpts(1e-8, 0.0, 100, 0, 1, 0, 1)):
        assert call(opts=bad) == L.SLA_ERR_INVALID
    for kw in ({"lam": None}, {"V": None}, {"gV": None}, {"mu": None}):
        assert call(**kw) == L.SLA_ERR_INVALID
    assert call(nb=need - 256) == L.SLA_ERR_WORKSPACE
    assert call(w=ctypes.c_void_p(0x100010)) == L.SLA_ERR_WORKSPACE
    for k, acc in ((0, 0), (9, 0), (6, 2)):
        assert lib.sla_eig_vector_grad_values(ctypes.byref(A), k, fake, fake, fake, acc,
                                              None) == L.SLA_ERR_INVALID


def test_normalize_bwd_rejects_bad_arguments_without_launch():
    """sla_ggt_normalize_bwd: mismatched sizes, null pointers and a dG that
    overlaps the forward's values are rejected before any launch (fake
    pointers: a launch would fault); dG == dGn is allowed."""
    lib = L.lib()
    lib.sla_ggt_normalize_bwd.restype = ctypes.c_int32
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(10, 28, fake, fake)
    G = L.SlaCsr(10, 19, fake, fake)
    GT = L.SlaCsrT(fake, fake, fake)
    g, d, o = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), ctypes.c_void_p(0x30000)

    def call(a=A, gg=G, gt=GT, gv=g, dgn=d, dg=o):
        return lib.sla_ggt_normalize_bwd(ctypes.byref(a), fake, ctypes.byref(gg), None if gt is None else ctypes.byref(gt),
                                         gv, dgn, dg, None)
    assert call(a=L.SlaCsr(11, 28, fake, fake)) == L.SLA_ERR_INVALID          # n differs
    assert call(gt=None) == L.SLA_ERR_INVALID
    assert call(dgn=None) == L.SLA_ERR_INVALID
    assert call(dg=ctypes.c_void_p(0x10000 + 8 * 18)) == L.SLA_ERR_INVALID     # dG overlaps g_val
    assert call(dg=ctypes.c_void_p(0x20000 + 8)) == L.SLA_ERR_INVALID          # dG partly overlaps dGn
    assert call(gg=L.SlaCsr(10, 0, fake, fake)) == L.SLA_OK                    # nothing to do
