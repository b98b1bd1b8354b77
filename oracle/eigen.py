"""FP64 CPU oracle of the eigenvalue path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s reference leg
may import this module; it shares no code with the CUDA library.

Sec. 3.2, "Eigenvalue problems": for symmetric A with A v = lambda v,
||v||_2 = 1 and lambda simple, the Hellmann-Feynman theorem gives
d lambda / d A_ij = v_i v_j (Eq. 4), evaluated on the sparsity pattern.
The library computes the k smallest eigenpairs iteratively (LOBPCG, the
eigensolver the paper names); what it converges to has a plain definition,
so the oracle is that definition: the k smallest eigenpairs of the dense
matrix by a symmetric eigensolver (a library routine used as one step),
and the gradient loop written out entry by entry.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla_dense


def dense(rowptr, col, val):
    n = len(rowptr) - 1
    M = np.zeros((n, n))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            M[i, col[k]] += val[k]
    return M


def smallest_eigenpairs(rowptr, col, val, k):
    """(lambda [k] ascending, V [n, k]) of the k smallest eigenpairs; each
    column of V has unit norm and its largest-magnitude entry positive."""
    M = dense(rowptr, col, val)
    lam, V = sla_dense.eigh(M, subset_by_index=[0, k - 1])
    for i in range(k):
        j = int(np.argmax(np.abs(V[:, i])))
        if V[j, i] < 0:
            V[:, i] = -V[:, i]
    return lam, V


def eigenvalue_grad_values(rowptr, col, V, g):
    """dL/dA_e = sum_i g_i V[row_e, i] V[col_e, i] on the pattern (Eq. 4
    with upstream gradients g_i = dL/dlambda_i)."""
    n = len(rowptr) - 1
    V = np.asarray(V, dtype=np.float64)
    out = np.empty(int(rowptr[-1]))
    for r in range(n):
        for e in range(rowptr[r], rowptr[r + 1]):
            s = 0.0
            for i in range(len(g)):
                s += g[i] * V[r, i] * V[col[e], i]
            out[e] = s
    return out
