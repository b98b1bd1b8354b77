"""The distributed layer of Sec. 3.3 -- row-block partition with halo
metadata, the halo exchange H before every SpMV (Eq. 5), its transpose H^T
in the backward pass (Eq. 6), all-reduced inner products, and the
distributed CG of Algorithm 1 (App. C) -- with its P partitions emulated on
one GPU.

Partition p owns a contiguous block of rows O_p and stores A[O_p, :] with
its columns renumbered into an extended local space: its |O_p| own entries,
then its halo H_p (the sorted global columns outside O_p that its rows
reference).  On one device the partitions' extended vectors lie back to
back; H is one gather (every partition's owned entries and the values its
halo receives from their owners), H^T one fixed-order gather-sum at the
owners (summation at the receive site), every all-reduce a fixed-order sum
over partitions of their local sums, and the local SpMVs of all partitions
one SpMV of the concatenated local matrices.  Every step runs in the
library's kernels (sla_dist_*, sla_spmv, sla_grad_values); this module
builds the partition metadata on the host (integer index work, once per
pattern) and sequences the steps.  Nothing is exchanged between GPUs: each
call of this library uses one GPU.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from . import sla

__all__ = ["partition_rows", "build_layout", "DistributedMatrix", "halo_exchange", "dist_spmv", "dist_cg",
           "dist_solve"]


def partition_rows(n: int, P: int, rowptr=None, balance: str = "rows") -> np.ndarray:
    """Contiguous row blocks (the paper's partition_simple): P + 1 offsets.
    balance "rows": equal row counts; "nnz": blocks of about equal stored
    entries (rowptr required)."""
    if not 1 <= P <= max(n, 1):
        raise ValueError("P must be in [1, n]")
    if balance == "rows":
        return np.round(np.linspace(0, n, P + 1)).astype(np.int64)
    if balance != "nnz" or rowptr is None:
        raise ValueError("balance is 'rows', or 'nnz' with rowptr")
    rp = np.asarray(rowptr, np.int64)
    targets = np.linspace(0, rp[-1], P + 1)
    off = np.searchsorted(rp, targets[1:-1], side="left")
    off = np.concatenate([[0], off, [n]]).astype(np.int64)
    off = np.maximum.accumulate(off)
    # every partition keeps at least one row
    for p in range(1, P + 1):
        off[p] = max(off[p], off[p - 1] + 1) if p < P else n
    for p in range(P - 1, 0, -1):
        off[p] = min(off[p], off[p + 1] - 1)
    return off


def build_layout(rowptr, col, row_off) -> dict:
    """Halo metadata of a row-block partition (host numpy):
      ext_off [P+1]  start of partition p's extended vector;
      n_own, n_halo [P];
      col_ext [nnz]  each entry's column in the extended space (ext_off[p] +
                     local index: own c - o_p, or |O_p| + rank of c in H_p);
      src [total_ext] the global index each extended entry holds;
      own_pos [n]    the extended position of owned entry i;
      hptr [n+1], hlist  for each global i, the extended positions of the
                     halo copies of i, ordered by partition then halo
                     position (H^T sums them in this order)."""
    rp = np.asarray(rowptr, np.int64)
    c = np.asarray(col, np.int64)
    off = np.asarray(row_off, np.int64)
    n, P = len(rp) - 1, len(off) - 1
    col_ext = np.empty(len(c), np.int64)
    n_own = np.diff(off)
    halos, ext_off = [], [0]
    for p in range(P):
        o0, o1 = off[p], off[p + 1]
        e0, e1 = rp[o0], rp[o1]
        cols = c[e0:e1]
        outside = (cols < o0) | (cols >= o1)
        halo = np.unique(cols[outside])
        local = np.where(outside, n_own[p] + np.searchsorted(halo, cols), cols - o0)
        col_ext[e0:e1] = ext_off[-1] + local
        halos.append(halo)
        ext_off.append(ext_off[-1] + n_own[p] + len(halo))
    ext_off = np.asarray(ext_off, np.int64)
    total_ext = int(ext_off[-1])
    src = np.empty(total_ext, np.int64)
    own_pos = np.empty(n, np.int64)
    is_halo = np.zeros(total_ext, bool)
    for p in range(P):
        o0, o1 = off[p], off[p + 1]
        a = ext_off[p]
        src[a:a + n_own[p]] = np.arange(o0, o1)
        own_pos[o0:o1] = np.arange(a, a + n_own[p])
        src[a + n_own[p]:ext_off[p + 1]] = halos[p]
        is_halo[a + n_own[p]:ext_off[p + 1]] = True
    hpos = np.nonzero(is_halo)[0]                    # ascending: by partition, then halo position
    order = np.argsort(src[hpos], kind="stable")     # grouped by owner index, order kept within
    hlist = hpos[order]
    hptr = np.zeros(n + 1, np.int64)
    np.add.at(hptr, src[hpos] + 1, 1)
    hptr = np.cumsum(hptr)
    return {"ext_off": ext_off, "n_own": n_own, "n_halo": np.array([len(h) for h in halos], np.int64),
            "col_ext": col_ext, "src": src, "own_pos": own_pos, "hptr": hptr, "hlist": hlist,
            "total_ext": total_ext}


def _i32(a, dev):
    a = np.asarray(a, np.int64)
    if a.size and (a.max() >= 2 ** 31 or a.min() < 0):
        raise ValueError("index out of int32 range")
    return torch.from_numpy(a.astype(np.int32)).to(dev)


class DistributedMatrix:
    """A square CSR pattern split into P row blocks with halo metadata
    (Sec. 3.3), every partition's data on one device."""

    def __init__(self, rowptr, col, P: int, device="cuda", balance: str = "rows"):
        rp = np.asarray(rowptr, np.int64)
        self.n, self.nnz, self.P = len(rp) - 1, int(rp[-1]), int(P)
        self.row_off_h = partition_rows(self.n, self.P, rp, balance)
        lay = build_layout(rp, col, self.row_off_h)
        self.layout = lay
        self.total_ext = lay["total_ext"]
        self.halo_sizes = lay["n_halo"].tolist()
        self.row_off = _i32(self.row_off_h, torch.device(device))
        dev = self.row_off.device  # with its index (cuda:0), as the tensors report it
        self.device = dev
        self.src = _i32(lay["src"], dev)
        self.own_pos = _i32(lay["own_pos"], dev)
        self.hptr = _i32(lay["hptr"], dev)
        self.hlist = _i32(lay["hlist"], dev)
        self.rowptr = _i32(rp, dev)
        self.col_ext = _i32(lay["col_ext"], dev)
        # the local matrices of all partitions: n rows, extended columns
        self.local = sla.CSRMatrix(self.rowptr, self.col_ext, check=False)
        self._local_t = None
        self._partial = torch.empty(8 * self.P * 3, dtype=torch.float64, device=dev)
        self._dots = torch.empty(3, dtype=torch.float64, device=dev)

    def local_transpose(self):
        """(CSR of A_local^T over total_ext rows, permT): the transposed
        local SpMV of Eq. 6 (the pattern padded with empty rows to a square
        total_ext x total_ext one, then sla_csr_transpose)."""
        if self._local_t is None:
            pad = torch.full((self.total_ext - self.n,), self.nnz, dtype=torch.int32, device=self.device)
            sq = sla.CSRMatrix(torch.cat([self.rowptr, pad]), self.col_ext, check=False)
            rpT, cT, pT = sla.csr_transpose(sq)
            self._local_t = (sla.CSRMatrix(rpT, cT, check=False), pT)
        return self._local_t

    def dots(self, pairs):
        """All-reduced inner products of up to 3 (a, b) pairs of [n] vectors:
        each partition's local sum, then the sum over partitions in order.
        Returns a host list of floats (the all-reduce hands every rank the
        totals)."""
        k = len(pairs)
        A = (ctypes.c_void_p * k)(*[a.data_ptr() for a, _ in pairs])
        B = (ctypes.c_void_p * k)(*[b.data_ptr() for _, b in pairs])
        L.check("sla_dist_dots", L.lib().sla_dist_dots(self.P, self.row_off.data_ptr(), k, A, B,
                                                        self._partial.data_ptr(), self._dots.data_ptr(), None,
                                                        sla._stream_ptr(self.device)))
        return self._dots[:k].tolist()


def _spmv_rect(A: sla.CSRMatrix, val: torch.Tensor, x: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """out = A x for the rectangular local matrices (A.n rows; x as long as
    the column space: total_ext for A_local, n for its transpose) through
    sla_spmv, which reads x at the column indices only."""
    L.check("sla_spmv", L.lib().sla_spmv(ctypes.byref(A.c), val.data_ptr(), x.data_ptr(), out.data_ptr(),
                                         sla._stream_ptr(A.device)))
    return out


def _halo_gather(DA: DistributedMatrix, x: torch.Tensor) -> torch.Tensor:
    x_ext = torch.empty(DA.total_ext, dtype=torch.float64, device=DA.device)
    L.check("sla_dist_halo_gather", L.lib().sla_dist_halo_gather(DA.total_ext, DA.src.data_ptr(), x.data_ptr(),
                                                                 x_ext.data_ptr(), sla._stream_ptr(DA.device)))
    return x_ext


def _halo_scatter(DA: DistributedMatrix, g_ext: torch.Tensor) -> torch.Tensor:
    g = torch.empty(DA.n, dtype=torch.float64, device=DA.device)
    L.check("sla_dist_halo_scatter", L.lib().sla_dist_halo_scatter(
        DA.n, DA.own_pos.data_ptr(), DA.hptr.data_ptr(), DA.hlist.data_ptr(), g_ext.data_ptr(), g.data_ptr(),
        sla._stream_ptr(DA.device)))
    return g


class HaloExchange(torch.autograd.Function):
    """x [n] (every partition's owned entries) -> x_ext [total_ext]: H;
    the backward is the transposed exchange H^T."""

    @staticmethod
    def forward(ctx, x, DA):
        sla._need(x, torch.float64, DA.device, "x", DA.n)
        ctx.DA = DA
        return _halo_gather(DA, x)

    @staticmethod
    def backward(ctx, g_ext):
        return _halo_scatter(ctx.DA, g_ext.contiguous()), None


class _LocalSpMV(torch.autograd.Function):
    """y = A_local x_ext on every partition (no communication); backward:
    d x_ext = A_local^T dy, d val[k] = dy[i] x_ext[col_ext k]."""

    @staticmethod
    def forward(ctx, val, x_ext, DA):
        ctx.save_for_backward(val, x_ext)
        ctx.DA = DA
        y = torch.empty(DA.n, dtype=torch.float64, device=DA.device)
        return _spmv_rect(DA.local, val.detach().contiguous(), x_ext.detach().contiguous(), y)

    @staticmethod
    def backward(ctx, gy):
        val, x_ext = ctx.saved_tensors
        DA = ctx.DA
        gy = gy.contiguous()
        g_val = g_x = None
        if ctx.needs_input_grad[0]:
            g_val = torch.empty(DA.nnz, dtype=torch.float64, device=DA.device)
            L.check("sla_dist_outer_values", L.lib().sla_dist_outer_values(
                DA.n, DA.rowptr.data_ptr(), DA.col_ext.data_ptr(), gy.data_ptr(), x_ext.data_ptr(),
                g_val.data_ptr(), sla._stream_ptr(DA.device)))
        if ctx.needs_input_grad[1]:
            AT, permT = DA.local_transpose()
            valT = sla.gather_values(permT, val.detach().contiguous())
            g_x = _spmv_rect(AT, valT, gy, torch.empty(DA.total_ext, dtype=torch.float64, device=DA.device))
        return g_val, g_x, None


def halo_exchange(DA: DistributedMatrix, x: torch.Tensor) -> torch.Tensor:
    """H(x), differentiable (backward H^T)."""
    return HaloExchange.apply(x, DA)


def dist_spmv(DA: DistributedMatrix, val: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """y_{O_p} = A_local H(x_{O_p}) on every partition (Eq. 5); its gradient
    with respect to x is H^T(A_local^T dL/dy) (Eq. 6)."""
    return _LocalSpMV.apply(val, HaloExchange.apply(x, DA), DA)


def dist_cg(DA: DistributedMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-10,
            atol: float = 0.0, max_iter: int | None = None, max_restarts: int = 2):
    """Distributed Jacobi-PCG, Algorithm 1 (App. C) with the library's
    readings: one halo exchange per iteration inside the SpMV and two
    all-reduces (p.q; then r.z with r.r in one); stop when ||r|| <=
    max(rtol ||b||, atol), recompute the true residual through the same
    distributed SpMV and restart from x if it is above twice the target (at
    most max_restarts times); x0 = 0; NOT_SPD on A_ii <= 0, p^T A p <= 0 or
    r^T z <= 0; BREAKDOWN on a non-finite scalar.  Returns (x, info dict)."""
    dev, n = DA.device, DA.n
    sla._need(val, torch.float64, dev, "val", DA.nnz)
    sla._need(b, torch.float64, dev, "b", n)
    lib, st = L.lib(), sla._stream_ptr(dev)
    mi = sla.default_max_iter(n) if max_iter is None else int(max_iter)
    f = lambda: torch.empty(n, dtype=torch.float64, device=dev)
    x, r, z, p, q, dinv = f(), f(), f(), f(), f(), f()
    x.zero_()
    bad = torch.zeros(1, dtype=torch.int32, device=dev)
    L.check("sla_dist_diag_inv", lib.sla_dist_diag_inv(n, DA.rowptr.data_ptr(), DA.col_ext.data_ptr(),
                                                       val.data_ptr(), DA.own_pos.data_ptr(), dinv.data_ptr(),
                                                       bad.data_ptr(), st))
    info = {"iters": 0, "status": L.SLA_NOT_CONVERGED, "rel_res": float("nan"), "true_rel_res": float("nan"),
            "partitions": DA.P, "halo_sizes": DA.halo_sizes, "restarts": 0}
    if int(bad.item()):
        info["status"] = L.SLA_NOT_SPD
        return x, info
    (bb,) = DA.dots([(b, b)])
    bnorm = bb ** 0.5
    if bnorm == 0.0:
        info.update(status=L.SLA_OK, rel_res=0.0, true_rel_res=0.0)
        return x, info
    thresh = max(rtol * bnorm, atol)

    def spmv_into(v, out):
        _spmv_rect(DA.local, val, _halo_gather(DA, v), out)

    it, status, rnorm = 0, L.SLA_NOT_CONVERGED, float("nan")
    for restart in range(max_restarts + 1):
        spmv_into(x, q)
        L.check("sla_dist_cg_start", lib.sla_dist_cg_start(n, b.data_ptr(), q.data_ptr(), dinv.data_ptr(),
                                                           r.data_ptr(), z.data_ptr(), p.data_ptr(), st))
        rz, rr = DA.dots([(r, z), (r, r)])
        rnorm = rr ** 0.5
        status = L.SLA_NOT_CONVERGED
        if not (np.isfinite(rz) and np.isfinite(rnorm)):
            status = L.SLA_BREAKDOWN
            break
        while not rnorm <= thresh and it < mi:
            spmv_into(p, q)                                   # halo exchange + local SpMV
            (pq,) = DA.dots([(p, q)])                         # all_reduce(p^T A p)
            if not np.isfinite(pq):
                status = L.SLA_BREAKDOWN
                break
            if not pq > 0.0:
                status = L.SLA_NOT_SPD
                break
            alpha = rz / pq
            L.check("sla_dist_cg_update", lib.sla_dist_cg_update(n, alpha, p.data_ptr(), q.data_ptr(),
                                                                 dinv.data_ptr(), x.data_ptr(), r.data_ptr(),
                                                                 z.data_ptr(), st))
            rz_new, rr = DA.dots([(r, z), (r, r)])            # all_reduce(r^T z, r^T r)
            rnorm = rr ** 0.5
            it += 1
            if not (np.isfinite(rz_new) and np.isfinite(rnorm)):
                status = L.SLA_BREAKDOWN
                break
            if rnorm <= thresh:
                status = L.SLA_OK
                break
            if not rz_new > 0.0:
                status = L.SLA_NOT_SPD
                break
            L.check("sla_dist_cg_direction", lib.sla_dist_cg_direction(n, rz_new / rz, z.data_ptr(),
                                                                       p.data_ptr(), st))
            rz = rz_new
        if rnorm <= thresh:
            status = L.SLA_OK
        if status != L.SLA_OK:
            break
        spmv_into(x, q)                                       # true residual
        L.check("sla_dist_cg_start", lib.sla_dist_cg_start(n, b.data_ptr(), q.data_ptr(), dinv.data_ptr(),
                                                           r.data_ptr(), z.data_ptr(), p.data_ptr(), st))
        (tt,) = DA.dots([(r, r)])
        if tt ** 0.5 <= 2.0 * thresh:
            break
        if restart == max_restarts:
            status = L.SLA_NOT_CONVERGED
            break
        info["restarts"] += 1
    spmv_into(x, q)
    L.check("sla_dist_cg_start", lib.sla_dist_cg_start(n, b.data_ptr(), q.data_ptr(), dinv.data_ptr(),
                                                       r.data_ptr(), z.data_ptr(), p.data_ptr(), st))
    (tt,) = DA.dots([(r, r)])
    info.update(iters=it, status=status, rel_res=rnorm / bnorm, true_rel_res=tt ** 0.5 / bnorm)
    return x, info


class DistSolve(torch.autograd.Function):
    """x = A^{-1} b by the distributed CG; backward (Sec. 3.3 with Eq. 3):
    one distributed adjoint solve A^T lambda = dL/dx on the same partition
    (A SPD: A^T = A), grad_b = lambda, and dL/dA_ij = -lambda_i x_j
    assembled on every partition's own entries from the halo values of x
    (no further communication)."""

    @staticmethod
    def forward(ctx, val, b, DA, kw, strict):
        x, info = dist_cg(DA, val.detach().contiguous(), b.detach().contiguous(), **kw)
        if strict and info["status"] != L.SLA_OK:
            raise sla.SolveError("distributed CG: %s after %d iterations" % (
                L.STATUS_NAMES.get(info["status"], "?"), info["iters"]))
        ctx.save_for_backward(val, x)
        ctx.DA, ctx.kw, ctx.strict = DA, kw, strict
        return x

    @staticmethod
    def backward(ctx, gx):
        val, x = ctx.saved_tensors
        DA = ctx.DA
        lam, info = dist_cg(DA, val.detach().contiguous(), gx.contiguous().to(torch.float64), **ctx.kw)
        if ctx.strict and info["status"] != L.SLA_OK:
            raise sla.SolveError("distributed adjoint CG: %s" % L.STATUS_NAMES.get(info["status"], "?"))
        x_ext = _halo_gather(DA, x)
        g_val = sla.grad_values(DA.local, lam, x_ext)
        return g_val, lam, None, None, None


def dist_solve(DA: DistributedMatrix, val: torch.Tensor, b: torch.Tensor, *, strict: bool = True,
               **kw) -> torch.Tensor:
    """Differentiable distributed SPD solve (forward distributed CG, one
    distributed adjoint solve backward)."""
    return DistSolve.apply(val, b, DA, kw, strict)
