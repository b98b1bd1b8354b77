"""FP64 CPU oracle for the sparse Krylov solve + adjoint path (arXiv 2601.13994).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference leg of ``bench.py`` may import this package.
It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``sla_oracle.c`` (plain single-threaded C, FP64,
sequential sums, compiled with -ffp-contract=off); this module only marshals
NumPy arrays through ctypes and loops over batches.  Pins that tie it to the
paper and to mathematics (dense LU, Poisson closed forms, finite
differences, brute force) live in ``tests/test_oracle_pins.py``.

Function map (paper passage each one follows):
  spmv              SpMV y = A x (the product inside Algorithm 1, step 3a)
  diag              Jacobi diagonal (Sec. 4.1, Tab. 3 caption)
  pcg               Algorithm 1 with P = 1, Jacobi / none / G G^T preconditioner
  pcg_pipelined     pipelined PCG (Ghysels-Vanroose), the merged-reduction CG
                    variant App. C names as the roadmap for reduction latency
  cg_fixed          exactly k unpreconditioned CG steps (Sec. 4.2, Tab. 7 setting)
  bicgstab          right-preconditioned BiCGStab (cited in Sec. 1 and 3.1)
  transpose         CSR of A^T for A^T lambda = dL/dx (Eq. 3)
  coo_to_csr        COO ingest of SparseTensor(val, row, col, shape) (App. B)
  grad_values       dL/dA_ij = -lambda_i x_j on the pattern (Eq. 3)
  adjoint_backward  A^T lambda = g, grad_b = lambda, grad_val (Eq. 2-3)
  pcg_omp           ``pcg`` (Jacobi / none) with its loops spread over the
                    host's cores by OpenMP (``sla_oracle_omp.c``): the
                    all-core CPU baseline; differs from ``pcg`` in the
                    summation order of the inner products only
Modules: ``oracle.mpnn`` (learned factor), ``oracle.inverse`` (Sec. 4.6
inverse problem), ``oracle.nonlinear`` (Newton solve and its adjoint
gradient, Sec. 3.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sla_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_SRC = os.path.join(_HERE, "sla_oracle_omp.c")
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_omp_lib = None

STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", 3: "NOT_SPD", -1: "INVALID"}


def build(force: bool = False) -> str:
    """Compile sla_oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off)
    and sla_oracle_omp.c into liboracle_omp.so (the same flags + -fopenmp)."""
    for src, lib, extra in ((_SRC, _LIB_PATH, []), (_OMP_SRC, _OMP_LIB_PATH, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", *extra,
                                   "-shared", "-fPIC", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
    return _LIB_PATH


def _load_omp():
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            # threads that wait at the end of a parallel loop sleep instead of
            # spinning (read when the OpenMP runtime loads): with a core taken
            # by another process, spinning threads slowed an 8-thread run of a
            # 64^3 system 10x; at the benchmark's sizes a loop runs for
            # milliseconds, so the wake-up costs nothing measurable
            os.environ.setdefault("OMP_WAIT_POLICY", "passive")
            build()
            lib = ctypes.CDLL(_OMP_LIB_PATH)
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            d = ctypes.c_double
            lib.or_omp_threads.argtypes = []
            lib.or_omp_threads.restype = ctypes.c_int
            lib.or_omp_spmv.argtypes = [i32, P, P, P, P, P]
            lib.or_omp_spmv.restype = None
            lib.or_omp_pcg.argtypes = [i32, P, P, P, P, P, d, d, i32, i32, i32, i32, i32, P, P]
            lib.or_omp_pcg.restype = ctypes.c_int
            _omp_lib = lib
    return _omp_lib


def omp_threads() -> int:
    """Threads the OpenMP oracle uses (OMP_NUM_THREADS, else the cores this
    process may run on)."""
    return int(_load_omp().or_omp_threads())


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            i64 = ctypes.c_int64
            d = ctypes.c_double
            lib.or_spmv.argtypes = [i32, P, P, P, P, P]
            lib.or_spmv.restype = None
            lib.or_diag.argtypes = [i32, P, P, P, P]
            lib.or_diag.restype = None
            lib.or_pcg.argtypes = [i32, P, P, P, P, P, d, d, i32, i32, i32, i32, P, P, P, P, P]
            lib.or_pcg.restype = ctypes.c_int
            lib.or_pcg_pipelined.argtypes = [i32, P, P, P, P, P, d, d, i32, i32, i32, i32, P, P]
            lib.or_pcg_pipelined.restype = ctypes.c_int
            lib.or_cg_fixed.argtypes = [i32, P, P, P, P, P, i32]
            lib.or_cg_fixed.restype = None
            lib.or_bicgstab.argtypes = [i32, P, P, P, P, P, d, d, i32, i32, i32, i32, P, P]
            lib.or_bicgstab.restype = ctypes.c_int
            lib.or_transpose.argtypes = [i32, P, P, P, P, P]
            lib.or_transpose.restype = None
            lib.or_coo_to_csr.argtypes = [i32, i64, P, P, P, P, P, P, P]
            lib.or_coo_to_csr.restype = i32
            lib.or_grad_values.argtypes = [i32, P, P, P, P, P]
            lib.or_grad_values.restype = None
            lib.or_adjoint_backward.argtypes = [i32, P, P, P, P, P, P, P, i32, d, d, i32, P, P]
            lib.or_adjoint_backward.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _info(info, res):
    return {"iters": int(info[0]), "status": int(info[1]), "status_name": STATUS.get(int(info[1]), "?"),
            "rel_res": float(res[0]), "true_rel_res": float(res[1])}


def spmv(rowptr, col, val, x):
    rowptr, col, val, x = _i32(rowptr), _i32(col), _f64(val), _f64(x)
    n = rowptr.shape[0] - 1
    y = np.empty(n)
    _load().or_spmv(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def diag(rowptr, col, val):
    rowptr, col, val = _i32(rowptr), _i32(col), _f64(val)
    n = rowptr.shape[0] - 1
    d = np.empty(n)
    _load().or_diag(n, _p(rowptr), _p(col), _p(val), _p(d))
    return d


_PRECOND = {"none": 0, "jacobi": 1, "ggt": 2}


def default_max_iter(n: int) -> int:
    return int(min(max(10 * n, 100), 1_000_000))


def pcg(rowptr, col, val, b, rtol=1e-10, atol=0.0, max_iter=None, precond="jacobi",
        x0=None, max_restarts=2, G=None):
    """Preconditioned CG (Algorithm 1, P = 1).  Returns (x, info)."""
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.shape[0] - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    info = np.zeros(2, np.int32)
    res = np.zeros(2)
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    gr = gc = gv = None
    if precond == "ggt":
        gr, gc, gv = _i32(G[0]), _i32(G[1]), _f64(G[2])
    _load().or_pcg(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), rtol, atol, mi, max_restarts,
                   0 if x0 is None else 1, _PRECOND[precond],
                   None if gr is None else _p(gr), None if gc is None else _p(gc),
                   None if gv is None else _p(gv), _p(info), _p(res))
    return x, _info(info, res)


def pcg_omp(rowptr, col, val, b, rtol=1e-10, atol=0.0, max_iter=None, precond="jacobi", x0=None,
            max_restarts=2, threads=None):
    """Jacobi (or unpreconditioned) PCG of ``pcg`` on the host's cores
    (OpenMP; ``threads`` None: every core this process may run on).
    Returns (x, info) with info["threads"] the thread count used."""
    if threads is None:
        threads = len(os.sched_getaffinity(0))
    if precond not in ("jacobi", "none"):
        raise ValueError("pcg_omp supports precond 'jacobi' or 'none'")
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.shape[0] - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    info = np.zeros(2, np.int32)
    res = np.zeros(2)
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    lib = _load_omp()
    lib.or_omp_pcg(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), rtol, atol, mi, max_restarts,
                   0 if x0 is None else 1, _PRECOND[precond], int(threads), _p(info), _p(res))
    out = _info(info, res)
    out["threads"] = int(lib.or_omp_threads())
    return x, out


def pcg_pipelined(rowptr, col, val, b, rtol=1e-10, atol=0.0, max_iter=None, precond="jacobi",
                  x0=None, max_restarts=2):
    """Pipelined PCG (one merged reduction per iteration; App. C roadmap).
    Same exits and restarts as pcg.  Returns (x, info)."""
    if precond not in ("none", "jacobi"):
        raise ValueError("pcg_pipelined: precond must be 'none' or 'jacobi'")
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.shape[0] - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    info = np.zeros(2, np.int32)
    res = np.zeros(2)
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    _load().or_pcg_pipelined(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), rtol, atol, mi,
                             max_restarts, 0 if x0 is None else 1, _PRECOND[precond], _p(info), _p(res))
    return x, _info(info, res)


def cg_fixed(rowptr, col, val, b, k):
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.shape[0] - 1
    x = np.zeros(n)
    _load().or_cg_fixed(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), int(k))
    return x


def bicgstab(rowptr, col, val, b, rtol=1e-10, atol=0.0, max_iter=None, precond="jacobi",
             x0=None, max_restarts=2):
    """Right-preconditioned BiCGStab.  Returns (x, info)."""
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = rowptr.shape[0] - 1
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    info = np.zeros(2, np.int32)
    res = np.zeros(2)
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    _load().or_bicgstab(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), rtol, atol, mi, max_restarts,
                        0 if x0 is None else 1, _PRECOND[precond], _p(info), _p(res))
    return x, _info(info, res)


def transpose(rowptr, col):
    """Stable CSR transpose: (rowptrT, colT, permT) with valT = val[permT]."""
    rowptr, col = _i32(rowptr), _i32(col)
    n = rowptr.shape[0] - 1
    nnz = int(rowptr[-1])
    rpT = np.empty(n + 1, np.int32)
    cT = np.empty(max(nnz, 1), np.int32)
    pT = np.empty(max(nnz, 1), np.int32)
    _load().or_transpose(n, _p(rowptr), _p(col), _p(rpT), _p(cT), _p(pT))
    return rpT, cT[:nnz], pT[:nnz]


def coo_to_csr(n, row, col, val):
    """COO (any order, duplicates allowed) -> (rowptr, col, val, perm)."""
    row = np.ascontiguousarray(row, dtype=np.int64)
    colin = np.ascontiguousarray(col, dtype=np.int64)
    val = _f64(val)
    m = row.shape[0]
    rp = np.empty(n + 1, np.int32)
    c = np.empty(max(m, 1), np.int32)
    v = np.empty(max(m, 1))
    perm = np.empty(max(m, 1), np.int32)
    nnz = _load().or_coo_to_csr(int(n), m, _p(row), _p(colin), _p(val), _p(rp), _p(c), _p(v), _p(perm))
    return rp, c[:nnz].copy(), v[:nnz].copy(), perm[:m].copy()


def grad_values(rowptr, col, lam, x):
    rowptr, col, lam, x = _i32(rowptr), _i32(col), _f64(lam), _f64(x)
    n = rowptr.shape[0] - 1
    g = np.empty(int(rowptr[-1]))
    _load().or_grad_values(n, _p(rowptr), _p(col), _p(lam), _p(x), _p(g))
    return g


def adjoint_backward(rowptr, col, val, x, g, method="cg", rtol=1e-10, atol=0.0, max_iter=None):
    """Eq. 2-3: solve A^T lambda = g; returns (grad_b = lambda, grad_val, info)."""
    rowptr, col, val, x, g = _i32(rowptr), _i32(col), _f64(val), _f64(x), _f64(g)
    n = rowptr.shape[0] - 1
    gb = np.zeros(n)
    gv = np.empty(int(rowptr[-1]))
    info = np.zeros(2, np.int32)
    res = np.zeros(2)
    mi = default_max_iter(n) if max_iter is None else int(max_iter)
    _load().or_adjoint_backward(n, _p(rowptr), _p(col), _p(val), _p(x), _p(g), _p(gb), _p(gv),
                                0 if method == "cg" else 1, rtol, atol, mi, _p(info), _p(res))
    return gb, gv, _info(info, res)
