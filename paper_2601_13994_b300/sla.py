"""User-level API over the C ABI: CSR matrices on a CUDA device, SpMV and
Krylov solves.  Every computation runs in the library's CUDA kernels; this
module only checks tensors, manages cached workspaces and passes pointers
and the current stream.

Mirrors the paper's problem statement ``x = A.solve(b)`` for a sparse A
given by its values on a sparsity pattern (App. B)."""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

__all__ = ["CSRMatrix", "SolveInfo", "spmv", "cg", "bicgstab", "default_max_iter"]


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


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
        if check:
            self.validate()

    @classmethod
    def from_numpy(cls, rowptr, col, device="cuda", check: bool = True) -> "CSRMatrix":
        dev = torch.device(device)
        rp = torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.int32)).to(dev)
        c = torch.from_numpy(np.ascontiguousarray(col, dtype=np.int32)).to(dev)
        return cls(rp, c, check=check)

    def validate(self) -> None:
        ok = torch.empty(1, dtype=torch.int32, device=self.device)
        L.check("sla_csr_check", L.lib().sla_csr_check(ctypes.byref(self._c), ok.data_ptr(),
                                                      _stream_ptr(self.device)))
        if int(ok.item()) != 1:
            raise ValueError("invalid CSR pattern (rowptr not monotone, rowptr[n] != nnz, column "
                             "out of range, or columns not strictly ascending in a row)")

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


def spmv(A: CSRMatrix, val: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """y = A x (FP64)."""
    _need(val, torch.float64, A.device, "val", A.nnz)
    _need(x, torch.float64, A.device, "x", A.n)
    y = torch.empty(A.n, dtype=torch.float64, device=A.device) if out is None else out
    _need(y, torch.float64, A.device, "out", A.n)
    L.check("sla_spmv", L.lib().sla_spmv(ctypes.byref(A.c), _ptr(val), _ptr(x), _ptr(y),
                                        _stream_ptr(A.device)))
    return y


_PRECOND = {"none": L.SLA_PRECOND_NONE, "jacobi": L.SLA_PRECOND_JACOBI}


def _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, n, graph=True):
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    if precond not in _PRECOND:
        raise ValueError("precond must be one of %s" % sorted(_PRECOND))
    return L.SlaOpts(float(rtol), float(atol), mi, int(max_restarts), _PRECOND[precond], int(use_x0),
                     0 if graph else L.SLA_FLAG_HOST_LOOP)


def _krylov(fn_name: str, ws_kind: int, A: CSRMatrix, val, b, rtol, atol, max_iter, precond, x0,
            max_restarts, out, graph):
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
    o = _opts(rtol, atol, max_iter, max_restarts, precond, use_x0, A.n, graph)
    ws = workspace(ws_kind, A.n, A.nnz, 1, A.device)
    fn = getattr(L.lib(), fn_name)
    L.check(fn_name, fn(ctypes.byref(A.c), _ptr(val), _ptr(b), _ptr(x), ctypes.byref(o), info.data_ptr(),
                        ws.data_ptr(), ws.numel(), _stream_ptr(A.device)))
    return x, SolveInfo(info)


def bicgstab(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
             max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
             max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True):
    """Right-preconditioned BiCGStab for nonsymmetric A.  Returns (x, SolveInfo)."""
    return _krylov("sla_bicgstab", L.SLA_WS_BICGSTAB, A, val, b, rtol, atol, max_iter, precond, x0,
                   max_restarts, out, graph)


def cg(A: CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10, atol: float = 0.0,
       max_iter: int | None = None, precond: str = "jacobi", x0: torch.Tensor | None = None,
       max_restarts: int = 2, out: torch.Tensor | None = None, graph: bool = True):
    """Preconditioned CG for SPD A (Algorithm 1, one process).  Returns
    (x, SolveInfo).  With ``graph=True`` the solve is one graph launch and
    nothing synchronises until the info is read; ``graph=False`` launches the
    same kernels from a host loop (synchronising the stream)."""
    return _krylov("sla_cg", L.SLA_WS_CG, A, val, b, rtol, atol, max_iter, precond, x0, max_restarts, out,
                   graph)
