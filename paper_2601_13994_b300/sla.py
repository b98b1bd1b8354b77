"""User-level API over the C ABI: CSR matrices on a CUDA device, SpMV and
Krylov solves.  Every computation runs in the library's CUDA kernels; this
module only checks tensors, manages cached workspaces and passes pointers
and the current stream.

Mirrors the paper's problem statement ``x = A.solve(b)`` for a sparse A
given by its values on a sparsity pattern (App. B)."""
from __future__ import annotations

import ctypes
import json
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

__all__ = ["CSRMatrix", "SparseTensor", "SolveInfo", "spmv", "cg", "bicgstab", "solve", "adjoint_backward",
           "grad_values", "csr_transpose", "coo_to_csr", "segment_sum", "gather_values", "default_max_iter",
           "cg_multi", "adjoint_backward_multi", "solve_multi"]


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def fp64_peak_tflops(device: torch.device | str = "cuda", iters: int = 4096, blocks_per_sm: int = 8,
                     reps: int = 5) -> float:
    """Measured FP64 FMA throughput of the device (TFLOP/s): the library's
    probe kernel (independent FMA chains on every SM at full occupancy),
    timed with CUDA events on the current stream, best of `reps` after one
    warm-up launch."""
    dev = torch.device(device)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    flops = ctypes.c_int64(0)
    st = _stream_ptr(dev)
    L.check("sla_fp64_probe", L.lib().sla_fp64_probe(iters, blocks_per_sm, out.data_ptr(), ctypes.byref(flops), st))
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        L.check("sla_fp64_probe", L.lib().sla_fp64_probe(iters, blocks_per_sm, out.data_ptr(), ctypes.byref(flops),
                                                         st))
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return flops.value / (best / 1e3) / 1e12


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype, device, name: str, numel: int | None = None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if t.device != device:
        raise ValueError("%s is on %s, expected %s" % (name, t.device, device))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))


def default_max_iter(n: int) -> int:
    return int(min(max(10 * n, 100), 1_000_000))


class CSRMatrix:
    """Pattern of a square sparse matrix in CSR form (int32 indices) on one
    CUDA device.  Values are passed separately (float64 [nnz]) so that one
    pattern serves many value sets (batches, training steps)."""

    def __init__(self, rowptr: torch.Tensor, col: torch.Tensor, check: bool = True):
        self.device = rowptr.device
        if self.device.type != "cuda":
            raise ValueError("CSRMatrix lives on a CUDA device")
        _need(rowptr, torch.int32, self.device, "rowptr")
        _need(col, torch.int32, self.device, "col")
        self.rowptr = rowptr
        self.col = col
        self.n = rowptr.numel() - 1
        self.nnz = col.numel()
        if self.n < 0:
            raise ValueError("rowptr needs n+1 >= 1 entries")
        self._c = L.SlaCsr(self.n, self.nnz, rowptr.data_ptr(), col.data_ptr() if self.nnz else None)
        self._stats = None
        if check:
            self.validate()

    @classmethod
    def from_numpy(cls, rowptr, col, device="cuda", check: bool = True) -> "CSRMatrix":
        dev = torch.device(device)
        rp = torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.int32)).to(dev)
        c = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).to(dev)
        return cls(rp, c, check=check)

    def validate(self) -> None:
        """Checks the pattern and takes its row-length statistics (one host
        synchronisation for both)."""
        buf = torch.empty(3, dtype=torch.int32, device=self.device)
        st = _stream_ptr(self.device)
        L.check("sla_csr_check", L.lib().sla_csr_check(ctypes.byref(self._c), buf.data_ptr(), st))
        L.check("sla_csr_row_stats", L.lib().sla_csr_row_stats(ctypes.byref(self._c), buf[1:].data_ptr(), st))
        h = buf.cpu()
        if int(h[0]) != 1:
            raise ValueError("invalid CSR pattern (rowptr not monotone, rowptr[n] != nnz, column "
                             "out of range, or columns not strictly ascending in a row)")
        self._stats = (int(h[1]), int(h[2]))

    def row_stats(self) -> tuple:
        """(longest row, rows longer than 1024 entries), computed on the
        device once per pattern."""
        if self._stats is None:
            buf = torch.empty(2, dtype=torch.int32, device=self.device)
            L.check("sla_csr_row_stats", L.lib().sla_csr_row_stats(ctypes.byref(self._c), buf.data_ptr(),
                                                                  _stream_ptr(self.device)))
            h = buf.cpu()
            self._stats = (int(h[0]), int(h[1]))
        return self._stats

    @property
    def spmv_scheme(self) -> int:
        """L.SLA_SPMV_ROWS or L.SLA_SPMV_MERGE, from the row-length statistics."""
        return int(L.lib().sla_spmv_scheme(self.n, self.nnz, self.row_stats()[0]))

    @property
    def c(self) -> L.SlaCsr:
        return self._c


@dataclass
class SolveInfo:
    """Outcome of a solve, read from the device record(s) on first access."""
    raw: torch.Tensor  # uint8 [B, 24] on the device

    def _host(self):
        if not hasattr(self, "_cache"):
            h = self.raw.cpu().numpy()
            ints = h[:, :8].copy().view(np.int32).reshape(-1, 2)
            dbl = h[:, 8:].copy().view(np.float64).reshape(-1, 2)
            self._cache = (ints, dbl)
        return self._cache

    @property
    def iters(self):
        v = self._host()[0][:, 0]
        return int(v[0]) if v.shape[0] == 1 else v

    @property
    def status(self):
        v = self._host()[0][:, 1]
        return int(v[0]) if v.shape[0] == 1 else v

    @property
    def status_name(self):
        s = self.status
        if np.ndim(s) == 0:
            return L.STATUS_NAMES.get(int(s), "?")
        return [L.STATUS_NAMES.get(int(v), "?") for v in s]

    @property
    def rel_res(self):
        v = self._host()[1][:, 0]
        return float(v[0]) if v.shape[0] == 1 else v

    @property
    def true_rel_res(self):
        v = self._host()[1][:, 1]
        return float(v[0]) if v.shape[0] == 1 else v

    def as_dict(self):
        return {"iters": self.iters, "status": self.status, "status_name": self.status_name,
                "rel_res": self.rel_res, "true_rel_res": self.true_rel_res}


# Workspaces are cached per (device, kind, sizes) so that the library's
# graph cache (keyed by workspace address) is hit on repeated calls.
_ws_lock = threading.Lock()
_ws_cache: dict = {}


def workspace(kind: int, n: int, nnz: int, batch: int, device: torch.device) -> torch.Tensor:
    key = (device.index, kind, n, nnz, batch)
    with _ws_lock:
        t = _ws_cache.get(key)
        if t is None:
            nbytes = L.workspace_size(kind, n, nnz, batch)
            t = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
            if t.data_ptr() % 256:
                raise RuntimeError("workspace allocation is not 256-byte aligned")
            _ws_cache[key] = t
    return t


def clear_workspaces() -> None:
    with _ws_lock:
        _ws_cache.clear()


_SCHEMES = {"rows": L.SLA_SPMV_ROWS, "merge": L.SLA_SPMV_MERGE}


def spmv(A: CSRMatrix, val: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None,
         scheme: str = "auto") -> torch.Tensor:
    """y = A x (FP64).  scheme "auto" picks the row kernels (sla_spmv) or
    the merge-path kernel (sla_spmv_merge) from the pattern's row-length
    statistics (sla_spmv_scheme); "rows" / "merge" force one."""
    _need(val, torch.float64, A.device, "val", A.nnz)
    _need(x, torch.float64, A.device, "x", A.n)
    y = torch.empty(A.n, dtype=torch.float64, device=A.device) if out is None else out
    _need(y, torch.float64, A.device, "out", A.n)
    if scheme == "auto":
        kind = A.spmv_scheme
    elif scheme in _SCHEMES:
        kind = _SCHEMES[scheme]
    else:
        raise ValueError("scheme must be 'auto', 'rows' or 'merge'")
    if kind == L.SLA_SPMV_MERGE:
        ws = workspace(L.SLA_WS_SPMV_MERGE, A.n, A.nnz, 1, A.device)
        L.check("sla_spmv_merge", L.lib().sla_spmv_merge(ctypes.byref(A.c), _ptr(val), _ptr(x), _ptr(y),
                                                        ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))
    else:
        L.check("sla_spmv", L.lib().sla_spmv(ctypes.byref(A.c), _ptr(val), _ptr(x), _ptr(y),
                                            _stream_ptr(A.device)))
    return y


_PRECOND = {"none": L.SLA_PRECOND_NONE, "jacobi": L.SLA_PRECOND_JACOBI}


def _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, n, graph=True, cooperative=True,
          pipelined=False):
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    if precond not in _PRECOND:
        raise ValueError("precond must be one of %s" % sorted(_PRECOND))
    if pipelined and not (graph and cooperative):
        raise ValueError("pipelined=True runs as one cooperative launch: graph and cooperative must stay True")
    flags = ((0 if graph else L.SLA_FLAG_HOST_LOOP) | (0 if cooperative else L.SLA_FLAG_NO_COOP)
             | (L.SLA_FLAG_CG_PIPELINED if pipelined else 0))
    return L.SlaOpts(float(rtol), float(atol), mi, int(max_restarts), _PRECOND[precond], int(use_x0), flags)


def _krylov(fn_name: str, ws_kind: int, A: CSRMatrix, val, b, rtol, atol, max_iter, precond, x0,
            max_restarts, out, graph, cooperative=True, pipelined=False):
    _need(val, torch.float64, A.device, "val", A.nnz)
    _need(b, torch.float64, A.device, "b", A.n)
    if out is None:
        x = torch.empty(A.n, dtype=torch.float64, device=A.device)
    else:
        x = out
        _need(x, torch.float64, A.device, "out", A.n)
    use_x0 = 0
    if x0 is not None:
        _need(x0, torch.float64, A.device, "x0", A.n)
        if x0.data_ptr() != x.data_ptr():
            x.copy_(x0)
        use_x0 = 1
    info = torch.empty((1, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, A.n, graph, cooperative, pipelined)
    ws = workspace(ws_kind, A.n, A.nnz, 1, A.device)
    fn = getattr(L.lib(), fn_name)
    L.check(fn_name, fn(ctypes.byref(A.c), _ptr(val), _ptr(b), _ptr(x), ctypes.byref(o), info.data_ptr(),
                        ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))
    return x, SolveInfo(info)


def bicgstab(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
             max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
             max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True,
             cooperative: bool = True):
    """Right-preconditioned BiCGStab for nonsymmetric A.  Returns (x, SolveInfo).
    Up to 768 Ki rows one cooperative launch (``cooperative=False`` opts out)."""
    return _krylov("sla_bicgstab", L.SLA_WS_BICGSTAB, A, val, b, rtol, atol, max_iter, precond, x0,
                   max_restarts, out, graph, cooperative)


def cg(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
       max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
       max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True,
       cooperative: bool = True, pipelined: bool = False):
    """Preconditioned CG for SPD A (Algorithm 1, one process).  Returns
    (x, SolveInfo).  Up to 2.5 Mi rows the solve is one cooperative kernel
    launch (``cooperative=False`` opts out); otherwise, with ``graph=True``,
    it is one graph launch.  Nothing synchronises until the info is read;
    ``graph=False`` launches the per-phase kernels from a host loop
    (synchronising the stream).  ``pipelined=True``: the pipelined PCG of
    Ghysels and Vanroose (the three inner products of an iteration in one
    reduction, one grid barrier per iteration; App. C's roadmap for the
    reduction latency) as one cooperative launch at any size."""
    ws_kind = L.SLA_WS_CG_PIPELINED if pipelined else L.SLA_WS_CG
    return _krylov("sla_cg", ws_kind, A, val, b, rtol, atol, max_iter, precond, x0, max_restarts, out,
                   graph, cooperative, pipelined)


# ---------------------------------------------------------------------------
# Pattern utilities
# ---------------------------------------------------------------------------

def _scratch(kind: int, n: int, nnz: int, device: torch.device) -> torch.Tensor:
    nbytes = L.workspace_size(kind, n, nnz, 1)
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def csr_transpose(A: CSRMatrix):
    """CSR of A^T: (rowptrT, colT, permT) with valT = val[permT] (stable)."""
    dev = A.device
    rpT = torch.empty(A.n + 1, dtype=torch.int32, device=dev)
    cT = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
    pT = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
    ws = _scratch(L.SLA_WS_TRANSPOSE, A.n, A.nnz, dev)
    L.check("sla_csr_transpose", L.lib().sla_csr_transpose(ctypes.byref(A.c), rpT.data_ptr(), cT.data_ptr(),
                                                          pT.data_ptr(), ws.data_ptr(), ws.numel(),
                                                          _stream_ptr(dev)))
    return rpT, cT[:A.nnz], pT[:A.nnz]


def transpose_of(A: CSRMatrix):
    """Cached CSR of A^T for a pattern (computed on first use)."""
    t = getattr(A, "_transpose", None)
    if t is None:
        t = csr_transpose(A)
        A._transpose = t
        A._transpose_c = L.SlaCsrT(t[0].data_ptr(), t[1].data_ptr() if A.nnz else None,
                                   t[2].data_ptr() if A.nnz else None)
    return t


def colour_columns(rowptr, col):
    """Distance-2 colouring of a CSR pattern's columns (host arrays, the C
    library's greedy ``sla_colour_columns``): returns (colour int32 [n],
    number of colours).  Columns that share a row differ in colour."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    c = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    colour = np.empty(max(n, 1), dtype=np.int32)
    k = ctypes.c_int32(0)
    L.check("sla_colour_columns", L.lib().sla_colour_columns(
        n, rp.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p) if c.size else None,
        colour.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)))
    return colour[:n], int(k.value)


def gather_values(perm: torch.Tensor, val: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """out[k] = val[perm[k]]."""
    m = perm.numel()
    out = torch.empty(m, dtype=torch.float64, device=val.device) if out is None else out
    L.check("sla_gather_values", L.lib().sla_gather_values(m, perm.data_ptr(), val.data_ptr(),
                                                          out.data_ptr(), _stream_ptr(val.device)))
    return out


def coo_to_csr(n: int, row: torch.Tensor, col: torch.Tensor, val: torch.Tensor | None = None):
    """COO (int64 row/col, any order, duplicates) -> CSR pattern on the device.

    Returns (CSRMatrix, val_csr or None, perm, order, segptr): perm[e] is the
    CSR slot of COO entry e; (order, segptr) rebuild CSR values from new COO
    values with ``segment_sum``."""
    dev = row.device
    m = row.numel()
    row = row.to(torch.int64).contiguous()
    col = col.to(torch.int64).contiguous()
    v = torch.zeros(m, dtype=torch.float64, device=dev) if val is None else val.detach().contiguous()
    rowptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    col_out = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    val_out = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
    perm = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    order = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    segptr = torch.empty(m + 1, dtype=torch.int32, device=dev)
    nnz_out = torch.empty(1, dtype=torch.int32, device=dev)
    ws = _scratch(L.SLA_WS_COO, n, m, dev)
    L.check("sla_coo_to_csr", L.lib().sla_coo_to_csr(
        n, m, row.data_ptr(), col.data_ptr(), v.data_ptr(), rowptr.data_ptr(), col_out.data_ptr(),
        val_out.data_ptr(), perm.data_ptr(), order.data_ptr(), segptr.data_ptr(), nnz_out.data_ptr(),
        ws.data_ptr(), ws.numel(), _stream_ptr(dev)))
    nnz = int(nnz_out.item())
    if nnz < 0:
        raise ValueError("COO row/col index out of range [0, %d)" % n)
    A = CSRMatrix(rowptr, col_out[:nnz].clone(), check=False)
    return (A, None if val is None else val_out[:nnz].clone(), perm[:m], order[:m], segptr[:nnz + 1])


def segment_sum(segptr: torch.Tensor, idx: torch.Tensor, val: torch.Tensor) -> torch.Tensor:
    nseg = segptr.numel() - 1
    out = torch.empty(nseg, dtype=torch.float64, device=val.device)
    L.check("sla_segment_sum", L.lib().sla_segment_sum(nseg, segptr.data_ptr(), idx.data_ptr(),
                                                      val.data_ptr(), out.data_ptr(),
                                                      _stream_ptr(val.device)))
    return out


# ---------------------------------------------------------------------------
# Adjoint (Eq. 2-3) and the autograd bridge (Sec. 3.1, "Bridging backends")
# ---------------------------------------------------------------------------

def grad_values(A: CSRMatrix, lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """grad_val[k] = -lam[row(k)] * x[col(k)] (Eq. 3)."""
    g = torch.empty(A.nnz, dtype=torch.float64, device=A.device)
    L.check("sla_grad_values", L.lib().sla_grad_values(ctypes.byref(A.c), lam.data_ptr(), x.data_ptr(),
                                                      g.data_ptr(), _stream_ptr(A.device)))
    return g


_ADJ = {"cg": L.SLA_ADJ_CG, "bicgstab": L.SLA_ADJ_BICGSTAB}


def adjoint_backward(A: CSRMatrix, val: torch.Tensor, x: torch.Tensor, grad_x: torch.Tensor, *,
                     method: str = "cg", rtol: float = 1e-10, atol: float = 0.0,
                     max_iter: int | None = None, precond: str = "jacobi", max_restarts: int = 2,
                     graph: bool = True, cooperative: bool = True, pipelined: bool = False):
    """Solve A^T lambda = grad_x; returns (grad_b = lambda, grad_val, SolveInfo).
    ``pipelined=True`` (method "cg" only) solves with the pipelined PCG."""
    if pipelined and method != "cg":
        raise ValueError("pipelined=True is a CG variant (method='cg')")
    _need(val, torch.float64, A.device, "val", A.nnz)
    _need(x, torch.float64, A.device, "x", A.n)
    _need(grad_x, torch.float64, A.device, "grad_x", A.n)
    gb = torch.empty(A.n, dtype=torch.float64, device=A.device)
    gv = torch.empty(A.nnz, dtype=torch.float64, device=A.device)
    info = torch.empty((1, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _opts(rtol, atol, max_iter, max_restarts, precond, 0, A.n, graph, cooperative, pipelined)
    atp = None
    if method == "bicgstab":
        transpose_of(A)
        atp = ctypes.byref(A._transpose_c)
    ws = workspace(L.SLA_WS_ADJOINT, A.n, A.nnz, 1, A.device)
    L.check("sla_adjoint_backward", L.lib().sla_adjoint_backward(
        ctypes.byref(A.c), atp, val.data_ptr(), x.data_ptr(), grad_x.data_ptr(), gb.data_ptr(),
        gv.data_ptr(), _ADJ[method], ctypes.byref(o), info.data_ptr(), ws.data_ptr(), ws.numel(),
        _stream_ptr(A.device)))
    return gb, gv, SolveInfo(info)


class SolveError(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Eigenvalues (Sec. 3.2 "Eigenvalue problems", Eq. 4)
# ---------------------------------------------------------------------------

def eig_grad_values(A: CSRMatrix, V: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """Hellmann-Feynman gradient on the pattern (Eq. 4): out[e] = sum_i
    g_i V[row_e, i] V[col_e, i]; V [n, k] unit eigenvectors, g [k]."""
    k = V.shape[1]
    _need(V, torch.float64, A.device, "V", A.n * k)
    _need(g, torch.float64, A.device, "g", k)
    out = torch.empty(A.nnz, dtype=torch.float64, device=A.device)
    L.check("sla_eig_grad_values", L.lib().sla_eig_grad_values(
        ctypes.byref(A.c), k, V.data_ptr(), g.data_ptr(), out.data_ptr(), _stream_ptr(A.device)))
    return out


def eig_vector_adjoint(A: CSRMatrix, val: torch.Tensor, lam: torch.Tensor, V: torch.Tensor, gV: torch.Tensor, *,
                       rtol: float = 1e-10, atol: float = 0.0, max_iter: int | None = None,
                       precond: str = "jacobi"):
    """The deflated solve of Sec. 3.2 for each of the k pairs: mu [n, k],
    column j with (A - lam_j I) mu_j = (I - v_j v_j^T) gV_j, v_j^T mu_j = 0.
    Returns (mu, SolveInfo with k records)."""
    k = V.shape[1]
    _need(val, torch.float64, A.device, "val", A.nnz)
    for t, name, m in ((lam, "lambda", k), (V, "V", A.n * k), (gV, "gV", A.n * k)):
        _need(t, torch.float64, A.device, name, m)
    mu = torch.empty((A.n, k), dtype=torch.float64, device=A.device)
    mi = max_iter if max_iter is not None else 10 * A.n
    o = L.SlaOpts(float(rtol), float(atol), int(mi), 0, _PRECOND[precond], 0, 0)
    info = torch.empty((k, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    ws = workspace(L.SLA_WS_EIG_ADJOINT, A.n, A.nnz, k, A.device)
    L.check("sla_eig_vector_adjoint", L.lib().sla_eig_vector_adjoint(
        ctypes.byref(A.c), val.data_ptr(), k, lam.data_ptr(), V.data_ptr(), gV.data_ptr(), mu.data_ptr(),
        ctypes.byref(o), info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))
    return mu, SolveInfo(info)


def eig_vector_grad_values(A: CSRMatrix, mu: torch.Tensor, V: torch.Tensor, out: torch.Tensor | None = None):
    """Eigenvector part of dL/dA on the pattern: -sum_j mu[row_e, j]
    V[col_e, j], added to `out` when given."""
    k = V.shape[1]
    _need(V, torch.float64, A.device, "V", A.n * k)
    _need(mu, torch.float64, A.device, "mu", A.n * k)
    acc = out is not None
    if out is None:
        out = torch.empty(A.nnz, dtype=torch.float64, device=A.device)
    else:
        _need(out, torch.float64, A.device, "out", A.nnz)
    L.check("sla_eig_vector_grad_values", L.lib().sla_eig_vector_grad_values(
        ctypes.byref(A.c), k, mu.data_ptr(), V.data_ptr(), out.data_ptr(), int(acc), _stream_ptr(A.device)))
    return out


class _Eigsh(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, A, k, opts, box):
        _need(val, torch.float64, A.device, "val", A.nnz)
        lam = torch.empty(k, dtype=torch.float64, device=A.device)
        V = torch.empty((A.n, k), dtype=torch.float64, device=A.device)
        use_x0 = 0
        if opts["v0"] is not None:
            _need(opts["v0"], torch.float64, A.device, "v0", A.n * k)
            V.copy_(opts["v0"].reshape(A.n, k))
            use_x0 = 1
        mi = opts["max_iter"] if opts["max_iter"] is not None else 20000
        o = L.SlaOpts(float(opts["tol"]), 0.0, int(mi), 0, _PRECOND[opts["precond"]], use_x0, 0)
        info = torch.empty((1, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
        ws = workspace(L.SLA_WS_EIGSH, A.n, A.nnz, k, A.device)
        L.check("sla_eigsh", L.lib().sla_eigsh(ctypes.byref(A.c), val.detach().data_ptr(), k, lam.data_ptr(),
                                               V.data_ptr(), ctypes.byref(o), info.data_ptr(), ws.data_ptr(),
                                               ws.numel(), _stream_ptr(A.device)))
        box["info"] = SolveInfo(info)
        ctx.A = A
        ctx.opts = opts
        ctx.box = box
        ctx.save_for_backward(val, lam, V)
        return lam, V

    @staticmethod
    def backward(ctx, glam, gV):
        val, lam, V = ctx.saved_tensors
        if glam is None:
            glam = torch.zeros_like(lam)
        gval = eig_grad_values(ctx.A, V, glam.contiguous().to(torch.float64))
        if gV is not None and bool(gV.abs().max() > 0):
            mu, info = eig_vector_adjoint(ctx.A, val.detach(), lam, V, gV.contiguous().to(torch.float64),
                                          rtol=ctx.opts["adjoint_rtol"], precond=ctx.opts["precond"])
            ctx.box["adjoint_info"] = info
            st = np.atleast_1d(info.status)
            if (st != L.SLA_OK).any():
                raise SolveError("eigsh backward: the deflated eigenvector solve ended with %s"
                                 % info.status_name)
            eig_vector_grad_values(ctx.A, mu, V, out=gval)
        return gval, None, None, None, None


def eigsh(A: CSRMatrix, val: torch.Tensor, k: int = 6, *, tol: float = 1e-8, max_iter: int | None = None,
          precond: str = "jacobi", v0: torch.Tensor | None = None, strict: bool | None = True,
          adjoint_rtol: float = 1e-10):
    """The k smallest eigenpairs of SPD A by LOBPCG (Sec. 3.3; Knyazev 2001)
    with the Jacobi preconditioner (k <= 8; max_iter defaults to 20000
    iterations).  Returns (lambda [k] ascending, V [n, k] unit columns, each
    with its largest-magnitude entry positive, SolveInfo).  Both are
    differentiable w.r.t. val (simple eigenvalues): lambda by the
    Hellmann-Feynman gradient v_i v_j on the pattern (Eq. 4), V by one
    deflated solve per pair (sla_eig_vector_adjoint, to adjoint_rtol; a
    failed solve raises SolveError).  strict=True raises on a failed
    solve, False warns, None skips the check."""
    if not 1 <= k <= L.SLA_EIG_MAX_K:
        raise ValueError("k must be in 1..%d" % L.SLA_EIG_MAX_K)
    if precond not in _PRECOND:
        raise ValueError("precond must be one of %s" % sorted(_PRECOND))
    box = {}
    lam, V = _Eigsh.apply(val, A, int(k), {"tol": tol, "max_iter": max_iter, "precond": precond, "v0": v0,
                                           "adjoint_rtol": adjoint_rtol}, box)
    info = box["info"]
    if strict is not None:
        _check_info(info, "eigsh", strict)
    return lam, V, info


def _check_info(info: SolveInfo, what: str, strict: bool):
    if info.status != L.SLA_OK:
        msg = "%s: %s after %d iterations (rel_res %.3e)" % (what, info.status_name, info.iters, info.rel_res)
        if strict:
            raise SolveError(msg)
        import warnings
        warnings.warn(msg)


class SparseSolve(torch.autograd.Function):
    """x = A^{-1} b with the adjoint backward: forward runs the Krylov solve
    without recording anything, backward is one adjoint solve plus one
    O(nnz) pass, so the autograd graph holds one node whatever the iteration
    count (Sec. 3.1-3.2, Tab. 2)."""

    @staticmethod
    def forward(ctx, val, b, A, method, kw, strict):
        fn = cg if method == "cg" else bicgstab
        x, info = fn(A, val.detach(), b.detach(), **kw)
        if strict is not None:
            _check_info(info, "forward " + method, strict)
        ctx.save_for_backward(val, x)
        ctx.A, ctx.method, ctx.kw, ctx.strict = A, method, kw, strict
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        val, x = ctx.saved_tensors
        kw = {k: v for k, v in ctx.kw.items() if k not in ("x0", "out")}
        gb, gv, info = adjoint_backward(ctx.A, val.detach(), x, gx.contiguous().to(torch.float64),
                                        method=ctx.method, **kw)
        if ctx.strict is not None:
            _check_info(info, "adjoint " + ctx.method, ctx.strict)
        return gv, gb, None, None, None, None


def solve(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, method: str = "cg", strict: bool | None = True,
          **kw) -> torch.Tensor:
    """Differentiable x = A^{-1} b w.r.t. val (CSR order) and b.  method:
    "cg" (SPD A; the adjoint reuses A since A^T = A) or "bicgstab" (the
    adjoint runs on the cached CSR of A^T).  strict=True raises on a failed
    solve, False warns, None skips the check (no host synchronisation)."""
    if method not in _ADJ:
        raise ValueError("method must be 'cg' or 'bicgstab'")
    return SparseSolve.apply(val, b, A, method, kw, strict)


class _CooValues(torch.autograd.Function):
    """COO values -> CSR values on a fixed pattern (duplicates summed in COO
    order); backward gathers the CSR gradient back to every COO entry."""

    @staticmethod
    def forward(ctx, val, segptr, order, perm):
        ctx.perm = perm
        return segment_sum(segptr, order, val.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        return gather_values(ctx.perm, g.contiguous()), None, None, None


class SparseTensor:
    """The paper's SparseTensor(val, row, col, shape) (App. B) on one CUDA
    device: COO input (any order, duplicates summed), a CSR pattern built
    once, and differentiable ``solve`` / ``matvec``."""

    def __init__(self, val: torch.Tensor, row: torch.Tensor, col: torch.Tensor, shape):
        n, n2 = int(shape[-2]), int(shape[-1])
        if n != n2:
            raise ValueError("square matrices only")
        self.val = val
        self.shape = (n, n)
        self.A, _, self.perm, self.order, self.segptr = coo_to_csr(n, row, col)

    def csr_values(self) -> torch.Tensor:
        return _CooValues.apply(self.val, self.segptr, self.order, self.perm)

    def solve(self, b: torch.Tensor, method: str = "cg", **kw) -> torch.Tensor:
        return solve(self.A, self.csr_values(), b, method=method, **kw)

    def matvec(self, x: torch.Tensor) -> torch.Tensor:
        return spmv(self.A, self.csr_values().detach(), x.contiguous())

    def eigsh(self, k: int = 6, **kw):
        """The k smallest eigenpairs (LOBPCG); eigenvalues (Eq. 4) and
        eigenvectors (one deflated solve per pair) differentiable w.r.t. the
        COO values."""
        return eigsh(self.A, self.csr_values(), k, **kw)


# ---------------------------------------------------------------------------
# Batched solves in one persistent launch (shared pattern / distinct patterns)
# ---------------------------------------------------------------------------

# The batched CG's launch shapes the autotuner searches (sla_cg_batched_*
# config): 256/512/1024 threads per CTA (codes 1/2/3), vectors on chip or in
# global memory (bit 4 = 16), threads per row 2/4/8 (bits 8-9 = log2), systems
# per CTA 2/4 (bits 10-11 = log2); for lists also without the block teams for
# the large systems (bit 5 = 32; the other shape bits act on the single-CTA
# kernel, so they are searched with the teams off) and the teams on the
# pipelined PCG (bit 6 = 64).
TPR_SHIFT, SPC_SHIFT = 8, 10
BATCH_CONFIGS = ((1, 2, 3, 1 | 16, 2 | 16, 3 | 16)
                 + tuple(c | (t << TPR_SHIFT) for c in (1, 2, 3) for t in (1, 2, 3))
                 + tuple(c | (k << SPC_SHIFT) for c in (1, 2, 3) for k in (1, 2)))
LIST_CONFIGS = ((1, 2, 3, 1 | 16, 2 | 16, 64)
                + (1 | 32, 2 | 32, 3 | 32)
                + tuple(c | 32 | (t << TPR_SHIFT) for c in (2, 3) for t in (1, 2))
                + tuple(c | 32 | (1 << SPC_SHIFT) for c in (2, 3)))


def config_shape(config: int) -> dict:
    """The launch shape a batched-CG config word selects."""
    code = config & 15
    return {"threads_per_cta": {0: "auto", 1: 256, 2: 512, 3: 1024}.get(code, "?"),
            "vectors": "global" if config & 16 else "shared memory where they fit",
            "threads_per_row": 1 << ((config >> TPR_SHIFT) & 3),
            "systems_per_cta": 1 << ((config >> SPC_SHIFT) & 3),
            "block_teams": not (config & 32), "pipelined_teams": bool(config & 64)}


class CSRList:
    """Distinct square patterns concatenated on one device (SparseTensorList
    of Sec. 3.1): per-system row pointers back to back, local columns,
    offsets n_off / nnz_off, and a largest-first processing order."""

    def __init__(self, patterns, device="cuda"):
        dev = torch.device(device)
        ns = [len(rp) - 1 for rp, _ in patterns]
        nnzs = [int(rp[-1]) for rp, _ in patterns]
        self.batch = len(patterns)
        self.n_off_h = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.nnz_off_h = np.concatenate([[0], np.cumsum(nnzs)]).astype(np.int64)
        if self.n_off_h[-1] >= 2 ** 31 or self.nnz_off_h[-1] >= 2 ** 31:
            raise ValueError("batch too large for int32 offsets")
        self.n_max = max(ns) if ns else 0
        self.total_rows = int(self.n_off_h[-1])
        self.total_nnz = int(self.nnz_off_h[-1])
        rp_cat = np.concatenate([np.asarray(rp, np.int32) for rp, _ in patterns]) if patterns else np.zeros(0, np.int32)
        c_cat = np.concatenate([np.asarray(c, np.int32) for _, c in patterns]) if patterns else np.zeros(0, np.int32)
        self.rowptr = torch.from_numpy(rp_cat).to(dev)
        self.col = torch.from_numpy(c_cat).to(dev)
        self.n_off = torch.from_numpy(self.n_off_h.astype(np.int32)).to(dev)
        self.nnz_off = torch.from_numpy(self.nnz_off_h.astype(np.int32)).to(dev)
        self.order = torch.from_numpy(np.argsort(-np.asarray(nnzs), kind="stable").astype(np.int32)).to(dev)
        self.device = self.rowptr.device
        self._transpose = None

    def transpose(self):
        """(CSRList of the A_s^T, permT) with valT = val[permT] over the
        concatenated values (sla_csr_list_transpose; computed once)."""
        if self._transpose is None:
            T = object.__new__(CSRList)
            for k in ("batch", "n_off_h", "nnz_off_h", "n_max", "total_rows", "total_nnz", "n_off", "nnz_off",
                      "order", "device"):
                setattr(T, k, getattr(self, k))
            T.rowptr = torch.empty_like(self.rowptr)
            T.col = torch.empty(max(self.total_nnz, 1), dtype=torch.int32, device=self.device)
            permT = torch.empty(max(self.total_nnz, 1), dtype=torch.int32, device=self.device)
            ws = _scratch(L.SLA_WS_LIST_TRANSPOSE, self.total_rows, self.total_nnz, self.device)
            L.check("sla_csr_list_transpose", L.lib().sla_csr_list_transpose(
                self.batch, self.total_rows, self.total_nnz, self.n_off.data_ptr(), self.nnz_off.data_ptr(),
                self.rowptr.data_ptr(), self.col.data_ptr(), T.rowptr.data_ptr(), T.col.data_ptr(),
                permT.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(self.device)))
            T.col = T.col[:self.total_nnz]
            T._transpose = None
            self._transpose = (T, permT[:self.total_nnz])
        return self._transpose


_tune_cache: dict = {}
_tune_loaded = False


def _tune_file() -> str:
    """Where tuned launch shapes persist: $SLA_TUNE_CACHE, else
    ~/.cache/paper_2601_13994_b300/tune.json."""
    return os.environ.get("SLA_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2601_13994_b300", "tune.json")


def _device_tag() -> str:
    try:
        return torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    except Exception:  # no device: the tag only names the cache entries
        return "unknown"


def _tune_key_str(key) -> str:
    return "|".join([_device_tag()] + [str(k) for k in key])


def _load_tune_file():
    """Reads the persisted choices once per process (keys: device|kind|shape)."""
    global _tune_loaded
    if _tune_loaded:
        return
    _tune_loaded = True
    try:
        with open(_tune_file()) as f:
            saved = json.load(f)
    except (OSError, ValueError):
        return
    tag = _device_tag() + "|"
    for k, v in saved.items():
        if not k.startswith(tag) or not isinstance(v, int):
            continue
        parts = k[len(tag):].split("|")
        key = tuple(int(p) if p.lstrip("-").isdigit() else p for p in parts)
        _tune_cache.setdefault(key, v)


def _save_tune_choice(key, cfg: int):
    path = _tune_file()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        try:
            with open(path) as f:
                saved = json.load(f)
        except (OSError, ValueError):
            saved = {}
        saved[_tune_key_str(key)] = int(cfg)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(saved, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: the choice stays in this process


def _batched_opts(rtol, atol, max_iter, max_restarts, precond, use_x0, n):
    return _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, n, True)


def cg_batched(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
               max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
               max_restarts: int = 2, config: int | str = "auto", out: torch.Tensor | None = None):
    """B systems on one pattern: val [B, nnz], b [B, n] -> x [B, n], SolveInfo
    (B records).  One persistent launch; config "tune" runs the autotuner."""
    B = b.shape[0]
    _need(val, torch.float64, A.device, "val", B * A.nnz)
    _need(b, torch.float64, A.device, "b", B * A.n)
    x = torch.empty((B, A.n), dtype=torch.float64, device=A.device) if out is None else out
    use_x0 = 0
    if x0 is not None:
        x.copy_(x0)
        use_x0 = 1
    info = torch.empty((B, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, use_x0, A.n)
    ws = workspace(L.SLA_WS_BATCHED, A.n, A.nnz, B, A.device)

    def run(cfg):
        L.check("sla_cg_batched_shared", L.lib().sla_cg_batched_shared(
            ctypes.byref(A.c), B, val.data_ptr(), b.data_ptr(), x.data_ptr(), ctypes.byref(o), info.data_ptr(),
            cfg, ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))

    cfg = _resolve_config(config, ("shared", A.n, A.nnz, B), run, x, x0)
    run(cfg)
    return x, SolveInfo(info)


def cg_batched_list(P: CSRList, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
                    max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
                    max_restarts: int = 2, config: int | str = "auto", out: torch.Tensor | None = None):
    """Distinct patterns (concatenated values / right-hand sides) in one
    persistent launch; returns (x concatenated, SolveInfo with B records)."""
    _need(val, torch.float64, P.device, "val", P.total_nnz)
    _need(b, torch.float64, P.device, "b", P.total_rows)
    x = torch.empty(P.total_rows, dtype=torch.float64, device=P.device) if out is None else out
    use_x0 = 0
    if x0 is not None:
        x.copy_(x0)
        use_x0 = 1
    info = torch.empty((P.batch, L.INFO_BYTES), dtype=torch.uint8, device=P.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, use_x0, P.n_max)
    ws = workspace(L.SLA_WS_BATCHED, P.total_rows, P.total_nnz, 1, P.device)

    def run(cfg):
        L.check("sla_cg_batched_list", L.lib().sla_cg_batched_list(
            P.batch, P.n_max, P.total_rows, P.n_off.data_ptr(), P.nnz_off.data_ptr(), P.rowptr.data_ptr(),
            P.col.data_ptr(), val.data_ptr(), b.data_ptr(), x.data_ptr(),
            None if P.order is None else P.order.data_ptr(), ctypes.byref(o),
            info.data_ptr(), cfg, ws.data_ptr(), ws.numel(), _stream_ptr(P.device)))

    cfg = _resolve_config(config, ("list", P.n_max, P.total_rows, P.total_nnz, P.batch), run, x, x0,
                          LIST_CONFIGS)
    run(cfg)
    return x, SolveInfo(info)


# BiCGStab batches: 256/512/1024 threads, vectors on chip as far as they fit / in global
BICG_BATCH_CONFIGS = (1, 2, 3, 1 | 16, 2 | 16, 3 | 16)
# Lists: one CTA per system (bit 32), or block teams for the large systems:
# team size code << 8 (3, 2, 4, 6 blocks), entry threshold code << 10
# (32768, 16384, 65536, 131072 entries).
BICG_TEAM_SIZES, BICG_TEAM_MIN_NNZ = (3, 2, 4, 6), (32768, 16384, 65536, 131072)
BICG_LIST_CONFIGS = ((1 | 32, 2 | 32, 3 | 32, 1 | 16 | 32, 2 | 16 | 32, 3 | 16 | 32)
                     + tuple((t << 8) | (m << 10) for t in range(4) for m in range(3)))


def bicg_list_shape(config: int) -> dict:
    """The launch shape a batched-BiCGStab list config word selects."""
    if config & 32:
        return {"block_teams": False, "threads_per_cta": {0: "auto", 1: 256, 2: 512, 3: 1024}.get(config & 15, "?"),
                "vectors": "global" if config & 16 else "shared memory where they fit"}
    return {"block_teams": True, "team_blocks": BICG_TEAM_SIZES[(config >> 8) & 3],
            "team_min_nnz": BICG_TEAM_MIN_NNZ[(config >> 10) & 3], "threads_per_cta": 512, "vectors": "global"}


def bicgstab_batched(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10,
                     atol: float = 0.0, max_iter: int | None = None, precond: str = "jacobi",
                     x0: torch.Tensor | None = None, max_restarts: int = 2, config: int | str = "auto",
                     out: torch.Tensor | None = None):
    """B nonsymmetric systems on one pattern by BiCGStab: val [B, nnz], b
    [B, n] -> x [B, n], SolveInfo (B records).  One persistent launch;
    config "tune" runs the autotuner."""
    B = b.shape[0]
    _need(val, torch.float64, A.device, "val", B * A.nnz)
    _need(b, torch.float64, A.device, "b", B * A.n)
    x = torch.empty((B, A.n), dtype=torch.float64, device=A.device) if out is None else out
    use_x0 = 0
    if x0 is not None:
        x.copy_(x0)
        use_x0 = 1
    info = torch.empty((B, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, use_x0, A.n)
    ws = workspace(L.SLA_WS_BATCHED, A.n, A.nnz, B, A.device)

    def run(cfg):
        L.check("sla_bicgstab_batched_shared", L.lib().sla_bicgstab_batched_shared(
            ctypes.byref(A.c), B, val.data_ptr(), b.data_ptr(), x.data_ptr(), ctypes.byref(o), info.data_ptr(),
            cfg, ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))

    cfg = _resolve_config(config, ("bicg_shared", A.n, A.nnz, B), run, x, x0, BICG_BATCH_CONFIGS)
    run(cfg)
    return x, SolveInfo(info)


def bicgstab_batched_list(P: CSRList, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10,
                          atol: float = 0.0, max_iter: int | None = None, precond: str = "jacobi",
                          x0: torch.Tensor | None = None, max_restarts: int = 2, config: int | str = "auto",
                          out: torch.Tensor | None = None):
    """Distinct nonsymmetric patterns (concatenated values / right-hand
    sides) by BiCGStab in one launch (the large systems by teams of blocks
    unless config has bit 32; see BICG_LIST_CONFIGS); returns (x
    concatenated, SolveInfo with B records)."""
    _need(val, torch.float64, P.device, "val", P.total_nnz)
    _need(b, torch.float64, P.device, "b", P.total_rows)
    x = torch.empty(P.total_rows, dtype=torch.float64, device=P.device) if out is None else out
    use_x0 = 0
    if x0 is not None:
        x.copy_(x0)
        use_x0 = 1
    info = torch.empty((P.batch, L.INFO_BYTES), dtype=torch.uint8, device=P.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, use_x0, P.n_max)
    ws = workspace(L.SLA_WS_BATCHED, P.total_rows, P.total_nnz, 1, P.device)

    def run(cfg):
        L.check("sla_bicgstab_batched_list", L.lib().sla_bicgstab_batched_list(
            P.batch, P.n_max, P.total_rows, P.n_off.data_ptr(), P.nnz_off.data_ptr(), P.rowptr.data_ptr(),
            P.col.data_ptr(), val.data_ptr(), b.data_ptr(), x.data_ptr(),
            None if P.order is None else P.order.data_ptr(), ctypes.byref(o),
            info.data_ptr(), cfg, ws.data_ptr(), ws.numel(), _stream_ptr(P.device)))

    cfg = _resolve_config(config, ("bicg_list", P.n_max, P.total_rows, P.total_nnz, P.batch), run, x, x0,
                          BICG_LIST_CONFIGS)
    run(cfg)
    return x, SolveInfo(info)


def gather_values_batched(perm: torch.Tensor, val: torch.Tensor) -> torch.Tensor:
    """out[s, m] = val[s, perm[m]] for val [B, nnz] (the values of every
    A_s^T of a shared pattern, perm = permT of csr_transpose)."""
    B, nnz = val.shape
    out = torch.empty_like(val)
    L.check("sla_gather_values_batched", L.lib().sla_gather_values_batched(
        B, nnz, perm.data_ptr(), val.data_ptr(), out.data_ptr(), _stream_ptr(val.device)))
    return out


def _resolve_config(config, key, run, x, x0, candidates=BATCH_CONFIGS):
    """'auto': cached tuned choice if any, else the library's heuristic (0);
    'tune': time every kernel variant on this batch (two runs each, CUDA
    events) and cache the fastest under the batch's shape key."""
    if isinstance(config, int):
        return config
    _load_tune_file()
    if config == "auto":
        return _tune_cache.get(key, 0)
    if config != "tune":
        raise ValueError("config must be an int, 'auto' or 'tune'")
    best, best_t = 0, float("inf")
    for cfg in candidates:
        times = []
        for _ in range(2):
            if x0 is not None:
                x.copy_(x0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            run(cfg)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        if min(times) < best_t:
            best, best_t = cfg, min(times)
    _tune_cache[key] = best
    _save_tune_choice(key, best)
    return best


def tuned_configs() -> dict:
    return dict(_tune_cache)


def grad_values_batched_shared(A: CSRMatrix, lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    B = lam.shape[0]
    g = torch.empty((B, A.nnz), dtype=torch.float64, device=A.device)
    L.check("sla_grad_values_batched", L.lib().sla_grad_values_batched(
        B, 1, A.n, A.nnz, A.rowptr.data_ptr(), A.col.data_ptr(), None, None, lam.data_ptr(), x.data_ptr(),
        g.data_ptr(), _stream_ptr(A.device)))
    return g


def grad_values_batched_list(P: CSRList, lam: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    g = torch.empty(P.total_nnz, dtype=torch.float64, device=P.device)
    L.check("sla_grad_values_batched", L.lib().sla_grad_values_batched(
        P.batch, 0, P.n_max, 0, P.rowptr.data_ptr(), P.col.data_ptr(), P.n_off.data_ptr(), P.nnz_off.data_ptr(),
        lam.data_ptr(), x.data_ptr(), g.data_ptr(), _stream_ptr(P.device)))
    return g


def _adjoint_config(config, key) -> int:
    """Launch shape of a batched adjoint solve: an int as given; otherwise
    the choice tuned for the forward solve of the same shape, else 0."""
    if isinstance(config, int):
        return config
    if config not in ("auto", "tune"):
        raise ValueError("config must be an int, 'auto' or 'tune'")
    _load_tune_file()
    return _tune_cache.get(key, 0)


def adjoint_backward_batched(A: CSRMatrix, val: torch.Tensor, x: torch.Tensor, grad_x: torch.Tensor, *,
                             method: str = "cg", rtol: float = 1e-10, atol: float = 0.0,
                             max_iter: int | None = None, precond: str = "jacobi", max_restarts: int = 2,
                             config: int | str = "auto"):
    """Eq. 3 for every system of a shared-pattern batch in one call
    (sla_adjoint_backward_batched_shared): A_s^T lambda_s = grad_x[s] by one
    batched CG (symmetric A_s) or BiCGStab (on the CSR of A^T) launch, then
    the gradients of all systems.  val [B, nnz], x and grad_x [B, n];
    returns (grad_b = lambda [B, n], grad_val [B, nnz], SolveInfo with B
    records)."""
    if method not in _ADJ:
        raise ValueError("method must be 'cg' or 'bicgstab'")
    B = x.shape[0]
    _need(val, torch.float64, A.device, "val", B * A.nnz)
    _need(x, torch.float64, A.device, "x", B * A.n)
    _need(grad_x, torch.float64, A.device, "grad_x", B * A.n)
    gb = torch.empty((B, A.n), dtype=torch.float64, device=A.device)
    gv = torch.empty((B, A.nnz), dtype=torch.float64, device=A.device)
    info = torch.empty((B, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, 0, A.n)
    atp = None
    if method == "bicgstab":
        transpose_of(A)
        atp = ctypes.byref(A._transpose_c)
    cfg = _adjoint_config(config, ("shared" if method == "cg" else "bicg_shared", A.n, A.nnz, B))
    ws = workspace(L.SLA_WS_ADJOINT_BATCHED, A.n, A.nnz, B, A.device)
    L.check("sla_adjoint_backward_batched_shared", L.lib().sla_adjoint_backward_batched_shared(
        ctypes.byref(A.c), atp, B, val.data_ptr(), x.data_ptr(), grad_x.data_ptr(), gb.data_ptr(),
        gv.data_ptr(), _ADJ[method], ctypes.byref(o), info.data_ptr(), cfg, ws.data_ptr(), ws.numel(),
        _stream_ptr(A.device)))
    return gb, gv, SolveInfo(info)


def adjoint_backward_batched_list(P: CSRList, val: torch.Tensor, x: torch.Tensor, grad_x: torch.Tensor, *,
                                  method: str = "cg", rtol: float = 1e-10, atol: float = 0.0,
                                  max_iter: int | None = None, precond: str = "jacobi", max_restarts: int = 2,
                                  config: int | str = "auto"):
    """Eq. 3 for every system of a list of distinct patterns in one call
    (sla_adjoint_backward_batched_list; BiCGStab on the list's transposes
    from sla_csr_list_transpose).  val [total_nnz], x and grad_x
    [total_rows]; returns (grad_b = lambda, grad_val, SolveInfo with B
    records)."""
    if method not in _ADJ:
        raise ValueError("method must be 'cg' or 'bicgstab'")
    _need(val, torch.float64, P.device, "val", P.total_nnz)
    _need(x, torch.float64, P.device, "x", P.total_rows)
    _need(grad_x, torch.float64, P.device, "grad_x", P.total_rows)
    gb = torch.empty(P.total_rows, dtype=torch.float64, device=P.device)
    gv = torch.empty(max(P.total_nnz, 1), dtype=torch.float64, device=P.device)[:P.total_nnz]
    info = torch.empty((P.batch, L.INFO_BYTES), dtype=torch.uint8, device=P.device)
    o = _batched_opts(rtol, atol, max_iter, max_restarts, precond, 0, P.n_max)
    rpT = cT = permT = None
    if method == "bicgstab":
        PT, pT = P.transpose()
        rpT, cT, permT = PT.rowptr.data_ptr(), PT.col.data_ptr(), pT.data_ptr()
    key = ("list" if method == "cg" else "bicg_list", P.n_max, P.total_rows, P.total_nnz, P.batch)
    cfg = _adjoint_config(config, key)
    ws = workspace(L.SLA_WS_ADJOINT_BATCHED, P.total_rows, P.total_nnz, 1, P.device)
    L.check("sla_adjoint_backward_batched_list", L.lib().sla_adjoint_backward_batched_list(
        P.batch, P.n_max, P.total_rows, P.total_nnz, P.n_off.data_ptr(), P.nnz_off.data_ptr(),
        P.rowptr.data_ptr(), P.col.data_ptr(), rpT, cT, permT, val.data_ptr(), x.data_ptr(), grad_x.data_ptr(),
        gb.data_ptr(), gv.data_ptr(), None if P.order is None else P.order.data_ptr(), _ADJ[method],
        ctypes.byref(o), info.data_ptr(), cfg, ws.data_ptr(), ws.numel(), _stream_ptr(P.device)))
    return gb, gv, SolveInfo(info)


_BATCH_SOLVERS = {"cg": (lambda *a, **k: cg_batched(*a, **k)), "bicgstab": (lambda *a, **k: bicgstab_batched(*a, **k))}
_LIST_SOLVERS = {"cg": (lambda *a, **k: cg_batched_list(*a, **k)),
                 "bicgstab": (lambda *a, **k: bicgstab_batched_list(*a, **k))}


class BatchedSolve(torch.autograd.Function):
    """x[s] = A_s^{-1} b[s] for a batch on one shared pattern, with the
    adjoint backward (Eq. 3 per system) in one library call: one batched
    solve of A_s^T lambda_s = dL/dx_s for all systems (CG on A for SPD
    systems; BiCGStab on the shared CSR of A^T with every system's values
    gathered for nonsymmetric ones), then one gradient pass."""

    @staticmethod
    def forward(ctx, val, b, A, method, kw, strict):
        x, info = _BATCH_SOLVERS[method](A, val.detach().contiguous(), b.detach().contiguous(), **kw)
        if strict is not None:
            _check_batch(info, "batched forward", strict)
        ctx.save_for_backward(val, x)
        ctx.A, ctx.method, ctx.kw, ctx.strict = A, method, kw, strict
        return x

    @staticmethod
    def backward(ctx, gx):
        val, x = ctx.saved_tensors
        kw = {k: v for k, v in ctx.kw.items() if k not in ("x0", "out")}
        g = gx.contiguous().to(torch.float64)
        lam, gval, info = adjoint_backward_batched(ctx.A, val.detach().contiguous(), x, g, method=ctx.method, **kw)
        if ctx.strict is not None:
            _check_batch(info, "batched adjoint", ctx.strict)
        return gval.view(val.shape), lam, None, None, None, None


class BatchedListSolve(torch.autograd.Function):
    """Distinct patterns (the paper's SparseTensorList, Sec. 3.1 and Tab. 1):
    x_s = A_s^{-1} b_s for every system in one launch, each with its own
    gradient (Eq. 3): one batched solve of A_s^T lambda_s = dL/dx_s (CG on
    A_s, or BiCGStab on the list's transposes), then -lambda_s,i x_s,j on
    every pattern.  Values and right-hand sides are concatenated."""

    @staticmethod
    def forward(ctx, val, b, P, method, kw, strict):
        x, info = _LIST_SOLVERS[method](P, val.detach().contiguous(), b.detach().contiguous(), **kw)
        if strict is not None:
            _check_batch(info, "batched list forward", strict)
        ctx.save_for_backward(val, x)
        ctx.P, ctx.method, ctx.kw, ctx.strict = P, method, kw, strict
        return x

    @staticmethod
    def backward(ctx, gx):
        val, x = ctx.saved_tensors
        kw = {k: v for k, v in ctx.kw.items() if k not in ("x0", "out")}
        g = gx.contiguous().to(torch.float64)
        lam, gval, info = adjoint_backward_batched_list(ctx.P, val.detach().contiguous(), x, g,
                                                        method=ctx.method, **kw)
        if ctx.strict is not None:
            _check_batch(info, "batched list adjoint", ctx.strict)
        return gval, lam, None, None, None, None


def _check_batch(info: SolveInfo, what: str, strict: bool):
    st = np.atleast_1d(info.status)
    bad = np.nonzero(st != L.SLA_OK)[0]
    if bad.size:
        msg = "%s: %d of %d systems did not converge (first: system %d, %s)" % (
            what, bad.size, st.size, bad[0], L.STATUS_NAMES.get(int(st[bad[0]]), "?"))
        if strict:
            raise SolveError(msg)
        import warnings
        warnings.warn(msg)


def solve_batched(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, method: str = "cg",
                  strict: bool | None = True, **kw) -> torch.Tensor:
    """Differentiable batched solve on a shared pattern: val [B, nnz], b
    [B, n] -> x [B, n]; method "cg" (SPD) or "bicgstab" (nonsymmetric)."""
    if method not in _BATCH_SOLVERS:
        raise ValueError("method must be 'cg' or 'bicgstab'")
    return BatchedSolve.apply(val, b, A, method, kw, strict)


def solve_batched_list(P: CSRList, val: torch.Tensor, b: torch.Tensor, *, method: str = "cg",
                       strict: bool | None = True, **kw) -> torch.Tensor:
    """Differentiable solve of a list of distinct patterns (concatenated
    val [total_nnz], b [total_rows] -> x [total_rows]); every system gets
    its own gradient.  method "cg" (SPD) or "bicgstab" (nonsymmetric)."""
    if method not in _LIST_SOLVERS:
        raise ValueError("method must be 'cg' or 'bicgstab'")
    return BatchedListSolve.apply(val, b, P, method, kw, strict)


# ---------------------------------------------------------------------------
# Several right-hand sides sharing one matrix
# ---------------------------------------------------------------------------

def _rhs_block(t: torch.Tensor, A: CSRMatrix, name: str) -> int:
    _need(t, torch.float64, A.device, name)
    if t.dim() != 2 or t.shape[1] != A.n:
        raise ValueError("%s must be [k, n] with n = %d" % (name, A.n))
    k = t.shape[0]
    if not 1 <= k <= L.SLA_MULTI_MAX_RHS:
        raise ValueError("k = %d right-hand sides; 1 <= k <= %d" % (k, L.SLA_MULTI_MAX_RHS))
    return k


def cg_multi(A: CSRMatrix, val: torch.Tensor, B: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
             max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
             max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True):
    """A X = B for k <= 32 right-hand sides (rows of B [k, n]) sharing one SPD
    matrix: k independent PCG solves advanced together, A read once per
    iteration for all of them.  Returns (X [k, n], SolveInfo over k)."""
    _need(val, torch.float64, A.device, "val", A.nnz)
    k = _rhs_block(B, A, "B")
    X = torch.empty((k, A.n), dtype=torch.float64, device=A.device) if out is None else out
    _need(X, torch.float64, A.device, "out", k * A.n)
    use_x0 = 0
    if x0 is not None:
        _need(x0, torch.float64, A.device, "x0", k * A.n)
        if x0.data_ptr() != X.data_ptr():
            X.copy_(x0.view(k, A.n))
        use_x0 = 1
    info = torch.empty((k, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, A.n, graph)
    ws = workspace(L.SLA_WS_CG_MULTI, A.n, A.nnz, k, A.device)
    L.check("sla_cg_multi", L.lib().sla_cg_multi(ctypes.byref(A.c), _ptr(val), k, _ptr(B), _ptr(X),
                                                ctypes.byref(o), info.data_ptr(), ws.data_ptr(), ws.numel(),
                                                _stream_ptr(A.device)))
    return X, SolveInfo(info)


def adjoint_backward_multi(A: CSRMatrix, val: torch.Tensor, X: torch.Tensor, grad_X: torch.Tensor, *,
                           rtol: float = 1e-10, atol: float = 0.0, max_iter: int | None = None,
                           precond: str = "jacobi", max_restarts: int = 2, graph: bool = True):
    """Adjoint of cg_multi (symmetric A): A Lambda_j = grad_X_j; returns
    (grad_B = Lambda [k, n], grad_val [nnz] summed over the columns, SolveInfo)."""
    _need(val, torch.float64, A.device, "val", A.nnz)
    k = _rhs_block(X, A, "X")
    if _rhs_block(grad_X, A, "grad_X") != k:
        raise ValueError("grad_X must have the shape of X")
    gb = torch.empty((k, A.n), dtype=torch.float64, device=A.device)
    gv = torch.empty(A.nnz, dtype=torch.float64, device=A.device)
    info = torch.empty((k, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _opts(rtol, atol, max_iter, max_restarts, precond, 0, A.n, graph)
    ws = workspace(L.SLA_WS_CG_MULTI, A.n, A.nnz, k, A.device)
    L.check("sla_adjoint_backward_multi", L.lib().sla_adjoint_backward_multi(
        ctypes.byref(A.c), _ptr(val), k, _ptr(X), _ptr(grad_X), _ptr(gb), _ptr(gv), ctypes.byref(o),
        info.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))
    return gb, gv, SolveInfo(info)


class MultiSolve(torch.autograd.Function):
    """X = A^{-1} B for the rows of B [k, n], one SPD A: one multi-RHS PCG
    forward, one multi-RHS adjoint solve and one O(k nnz) gradient pass
    backward (Eq. 2-3 per column, the value gradients summed)."""

    @staticmethod
    def forward(ctx, val, B, A, kw, strict):
        X, info = cg_multi(A, val.detach(), B.detach().contiguous(), **kw)
        if strict is not None:
            _check_batch(info, "multi-RHS forward", strict)
        ctx.save_for_backward(val, X)
        ctx.A, ctx.kw, ctx.strict = A, kw, strict
        ctx.info = info
        return X

    @staticmethod
    def backward(ctx, gX):
        val, X = ctx.saved_tensors
        kw = {k: v for k, v in ctx.kw.items() if k not in ("x0", "out")}
        gb, gv, info = adjoint_backward_multi(ctx.A, val.detach(), X, gX.contiguous().to(torch.float64), **kw)
        if ctx.strict is not None:
            _check_batch(info, "multi-RHS adjoint", ctx.strict)
        return gv, gb, None, None, None


def solve_multi(A: CSRMatrix, val: torch.Tensor, B: torch.Tensor, *, strict: bool | None = True,
                **kw) -> torch.Tensor:
    """Differentiable X = A^{-1} B for B [k, n] (k <= 32 right-hand sides of
    one SPD matrix), w.r.t. val (CSR order) and B."""
    return MultiSolve.apply(val, B, A, kw, strict)


# ---------------------------------------------------------------------------
# CG with a factored preconditioner M^{-1} = G G^T
# ---------------------------------------------------------------------------

def cg_ggt(A: CSRMatrix, val: torch.Tensor, G: CSRMatrix, g_val: torch.Tensor, b: torch.Tensor, *,
           rtol: float = 1e-10, atol: float = 0.0, max_iter: int | None = None, x0: torch.Tensor | None = None,
           max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True,
           cooperative: bool = True):
    """PCG with z = G (G^T r), G lower triangular (CSR pattern G, values
    g_val).  The CSR of G^T is computed once per pattern and cached.  Up to
    1.5 Mi rows the solve is one cooperative kernel launch (``cooperative=False``
    opts out); otherwise one graph launch (``graph=False``: a host loop)."""
    _need(val, torch.float64, A.device, "val", A.nnz)
    _need(g_val, torch.float64, A.device, "g_val", G.nnz)
    _need(b, torch.float64, A.device, "b", A.n)
    if G.n != A.n:
        raise ValueError("G must be n x n")
    transpose_of(G)
    x = torch.empty(A.n, dtype=torch.float64, device=A.device) if out is None else out
    use_x0 = 0
    if x0 is not None:
        if x0.data_ptr() != x.data_ptr():
            x.copy_(x0)
        use_x0 = 1
    info = torch.empty((1, L.INFO_BYTES), dtype=torch.uint8, device=A.device)
    o = _opts(rtol, atol, max_iter, max_restarts, "jacobi", use_x0, A.n, graph, cooperative)
    ws = workspace(L.SLA_WS_CG_GGT, A.n, G.nnz, 1, A.device)
    L.check("sla_cg_ggt", L.lib().sla_cg_ggt(
        ctypes.byref(A.c), val.data_ptr(), ctypes.byref(G.c), g_val.data_ptr(), ctypes.byref(G._transpose_c),
        b.data_ptr(), x.data_ptr(), ctypes.byref(o), info.data_ptr(), ws.data_ptr(), ws.numel(),
        _stream_ptr(A.device)))
    return x, SolveInfo(info)
