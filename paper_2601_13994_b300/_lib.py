"""ctypes binding of ``libsla.so`` (the C ABI declared in include/sla.h).

Argument marshalling only: every entry point is called with raw device
pointers taken from torch tensors and the current CUDA stream.  There is no
fallback: if the shared library is missing the import of any solver raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsla.so")

SLA_OK = 0
SLA_NOT_CONVERGED = 1
SLA_BREAKDOWN = 2
SLA_NOT_SPD = 3
SLA_ERR_INVALID = -1
SLA_ERR_CUDA = -2
SLA_ERR_WORKSPACE = -3
SLA_ERR_TIMEOUT = -4

SLA_PRECOND_NONE = 0
SLA_PRECOND_JACOBI = 1
SLA_PRECOND_GGT = 2

SLA_FLAG_HOST_LOOP = 1
SLA_FLAG_NO_COOP = 2
SLA_FLAG_CG_PIPELINED = 4

SLA_WS_CG = 1
SLA_WS_BICGSTAB = 2
SLA_WS_ADJOINT = 3
SLA_WS_TRANSPOSE = 4
SLA_WS_COO = 5
SLA_WS_BATCHED = 6
SLA_WS_CG_GGT = 7
SLA_WS_CG_MULTI = 8
SLA_WS_SPMV_MERGE = 9
SLA_WS_CG_PIPELINED = 10
SLA_WS_EIGSH = 11
SLA_WS_EIG_ADJOINT = 12
SLA_WS_LIST_TRANSPOSE = 13
SLA_WS_ADJOINT_BATCHED = 14
SLA_EIG_MAX_K = 8
SLA_SPMV_ROWS = 0
SLA_SPMV_MERGE = 1
SLA_MP_DENSE_AUTO = 0
SLA_MP_DENSE_SIMT = 1
SLA_MP_DENSE_TC = 2
SLA_MULTI_MAX_RHS = 32

SLA_ADJ_CG = 0
SLA_ADJ_BICGSTAB = 1

SLA_NOALLOC_MAX_N = 393216

STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", 3: "NOT_SPD", -1: "ERR_INVALID",
                -2: "ERR_CUDA", -3: "ERR_WORKSPACE", -4: "ERR_TIMEOUT"}

INFO_BYTES = 24  # sla_info: int32 iters, int32 status, double rel_res, double true_rel_res


class SlaCsr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class SlaCsrT(ctypes.Structure):
    _fields_ = [("rowptr_t", ctypes.c_void_p), ("col_t", ctypes.c_void_p), ("perm_t", ctypes.c_void_p)]


class SlaOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("use_x0", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


class SlaError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__("%s returned %d (%s)" % (fn, code, STATUS_NAMES.get(code, "?")))
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libsla.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsla.so is not built (expected at %s); run "
                                   "`python -m paper_2601_13994_b300.build`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            L.sla_version.argtypes = []
            L.sla_version.restype = ctypes.c_char_p
            L.sla_status_string.argtypes = [i32]
            L.sla_status_string.restype = ctypes.c_char_p
            L.sla_workspace_size.argtypes = [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
            L.sla_workspace_size.restype = i32
            L.sla_csr_check.argtypes = [ctypes.POINTER(SlaCsr), P, P]
            L.sla_csr_check.restype = i32
            L.sla_spmv.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, P]
            L.sla_spmv.restype = i32
            L.sla_spmv_merge.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, P, ctypes.c_size_t, P]
            L.sla_spmv_merge.restype = i32
            L.sla_csr_row_stats.argtypes = [ctypes.POINTER(SlaCsr), P, P]
            L.sla_csr_row_stats.restype = i32
            L.sla_spmv_scheme.argtypes = [i32, ctypes.c_int64, i32]
            L.sla_spmv_scheme.restype = i32
            L.sla_cg.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, ctypes.POINTER(SlaOpts), P, P,
                                 ctypes.c_size_t, P]
            L.sla_cg.restype = i32
            L.sla_bicgstab.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, ctypes.POINTER(SlaOpts), P, P,
                                       ctypes.c_size_t, P]
            L.sla_bicgstab.restype = i32
            i64 = ctypes.c_int64
            L.sla_csr_transpose.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, P, ctypes.c_size_t, P]
            L.sla_csr_transpose.restype = i32
            L.sla_coo_to_csr.argtypes = [i32, i64, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_size_t, P]
            L.sla_coo_to_csr.restype = i32
            L.sla_segment_sum.argtypes = [i32, P, P, P, P, P]
            L.sla_segment_sum.restype = i32
            L.sla_gather_values.argtypes = [i64, P, P, P, P]
            L.sla_gather_values.restype = i32
            L.sla_colour_columns.argtypes = [i32, P, P, P, ctypes.POINTER(i32)]
            L.sla_colour_columns.restype = i32
            L.sla_eigsh.argtypes = [ctypes.POINTER(SlaCsr), P, i32, P, P, ctypes.POINTER(SlaOpts), P, P,
                                    ctypes.c_size_t, P]
            L.sla_eigsh.restype = i32
            L.sla_eig_grad_values.argtypes = [ctypes.POINTER(SlaCsr), i32, P, P, P, P]
            L.sla_eig_grad_values.restype = i32
            L.sla_eig_vector_adjoint.argtypes = [ctypes.POINTER(SlaCsr), P, i32, P, P, P, P,
                                                 ctypes.POINTER(SlaOpts), P, P, ctypes.c_size_t, P]
            L.sla_eig_vector_adjoint.restype = i32
            L.sla_eig_vector_grad_values.argtypes = [ctypes.POINTER(SlaCsr), i32, P, P, P, i32, P]
            L.sla_eig_vector_grad_values.restype = i32
            L.sla_grad_values.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, P]
            L.sla_grad_values.restype = i32
            L.sla_adjoint_backward.argtypes = [ctypes.POINTER(SlaCsr), ctypes.POINTER(SlaCsrT), P, P, P, P,
                                               P, i32, ctypes.POINTER(SlaOpts), P, P, ctypes.c_size_t, P]
            L.sla_adjoint_backward.restype = i32
            L.sla_cg_batched_shared.argtypes = [ctypes.POINTER(SlaCsr), i32, P, P, P, ctypes.POINTER(SlaOpts), P,
                                                i32, P, ctypes.c_size_t, P]
            L.sla_cg_batched_shared.restype = i32
            L.sla_cg_batched_list.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, P, ctypes.POINTER(SlaOpts), P,
                                              i32, P, ctypes.c_size_t, P]
            L.sla_cg_batched_list.restype = i32
            L.sla_grad_values_batched.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P]
            L.sla_grad_values_batched.restype = i32
            L.sla_bicgstab_batched_shared.argtypes = [ctypes.POINTER(SlaCsr), i32, P, P, P,
                                                      ctypes.POINTER(SlaOpts), P, i32, P, ctypes.c_size_t, P]
            L.sla_bicgstab_batched_shared.restype = i32
            L.sla_bicgstab_batched_list.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, P,
                                                    ctypes.POINTER(SlaOpts), P, i32, P, ctypes.c_size_t, P]
            L.sla_bicgstab_batched_list.restype = i32
            L.sla_csr_list_transpose.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, P, ctypes.c_size_t, P]
            L.sla_csr_list_transpose.restype = i32
            L.sla_gather_values_batched.argtypes = [i32, i64, P, P, P, P]
            L.sla_gather_values_batched.restype = i32
            L.sla_adjoint_backward_batched_shared.argtypes = [ctypes.POINTER(SlaCsr), ctypes.POINTER(SlaCsrT), i32,
                                                              P, P, P, P, P, i32, ctypes.POINTER(SlaOpts), P, i32,
                                                              P, ctypes.c_size_t, P]
            L.sla_adjoint_backward_batched_shared.restype = i32
            L.sla_adjoint_backward_batched_list.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P,
                                                            P, i32, ctypes.POINTER(SlaOpts), P, i32, P,
                                                            ctypes.c_size_t, P]
            L.sla_adjoint_backward_batched_list.restype = i32
            PP = ctypes.POINTER(ctypes.c_void_p)
            d = ctypes.c_double
            for name, args in (("sla_dist_halo_gather", [i64, P, P, P, P]),
                               ("sla_dist_halo_scatter", [i32, P, P, P, P, P, P]),
                               ("sla_dist_dots", [i32, P, i32, PP, PP, P, P, P, P]),
                               ("sla_dist_diag_inv", [i32, P, P, P, P, P, P, P]),
                               ("sla_dist_cg_start", [i32, P, P, P, P, P, P, P]),
                               ("sla_dist_cg_update", [i32, d, P, P, P, P, P, P, P]),
                               ("sla_dist_cg_direction", [i32, d, P, P, P]),
                               ("sla_dist_outer_values", [i32, P, P, P, P, P, P])):
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = i32
            L.sla_cg_ggt.argtypes = [ctypes.POINTER(SlaCsr), P, ctypes.POINTER(SlaCsr), P, ctypes.POINTER(SlaCsrT),
                                     P, P, ctypes.POINTER(SlaOpts), P, P, ctypes.c_size_t, P]
            L.sla_cg_ggt.restype = i32
            L.sla_cg_multi.argtypes = [ctypes.POINTER(SlaCsr), P, i32, P, P, ctypes.POINTER(SlaOpts), P, P,
                                       ctypes.c_size_t, P]
            L.sla_cg_multi.restype = i32
            L.sla_adjoint_backward_multi.argtypes = [ctypes.POINTER(SlaCsr), P, i32, P, P, P, P,
                                                     ctypes.POINTER(SlaOpts), P, P, ctypes.c_size_t, P]
            L.sla_adjoint_backward_multi.restype = i32
            L.sla_cg_noalloc.argtypes = [ctypes.POINTER(SlaCsr), P, P, P, ctypes.POINTER(SlaOpts), P, P]
            L.sla_cg_noalloc.restype = i32
            L.sla_selftest_grid_barrier.argtypes = [i32, i32, ctypes.c_int64, i32, P, P]
            L.sla_selftest_grid_barrier.restype = i32
            L.sla_fp64_probe.argtypes = [i32, i32, P, ctypes.POINTER(ctypes.c_int64), P]
            L.sla_fp64_probe.restype = i32
            _lib = L
    return _lib


def check(fn: str, code: int) -> int:
    if code < 0:
        raise SlaError(fn, code)
    return code


def workspace_size(kind: int, n: int, nnz: int, batch: int = 1) -> int:
    out = ctypes.c_size_t(0)
    check("sla_workspace_size", lib().sla_workspace_size(kind, n, nnz, batch, ctypes.byref(out)))
    return int(out.value)
