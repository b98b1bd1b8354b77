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

Eigenvector gradients (Sec. 3.2: one extra deflated linear solve per
pair).  Eq. 4 is the master adjoint specialised to the constrained residual
F(v, lambda; A) = (A v - lambda v, (v^T v - 1) / 2).  Its Jacobian in
(v, lambda) is [[A - lambda I, -v], [v^T, 0]]; the adjoint system with the
transpose, for upstream gradients gv = dL/dv and glam = dL/dlambda, gives
(A - lambda I) mu = (I - v v^T) gv with v^T mu = 0 (the deflated solve) and
the multiplier s = v^T gv, and then dL/dA_ab = -mu_a v_b + glam v_a v_b.
The oracle solves the bordered system [[A - lambda I, v], [v^T, 0]]
[mu; s] = [(I - v v^T) gv; 0], nonsingular for a simple eigenvalue, by a
dense LU (a library routine used as one step).
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


def eigenvector_adjoint(rowptr, col, val, lam, V, gV):
    """mu [n, k]: column j solves (A - lam_j I) mu_j = (I - v_j v_j^T) gV_j
    with v_j^T mu_j = 0, by the dense bordered system above."""
    M = dense(rowptr, col, val)
    n = M.shape[0]
    V = np.asarray(V, dtype=np.float64).reshape(n, -1)
    gV = np.asarray(gV, dtype=np.float64).reshape(n, -1)
    k = V.shape[1]
    mu = np.zeros((n, k))
    for j in range(k):
        v = V[:, j]
        K = np.zeros((n + 1, n + 1))
        K[:n, :n] = M - lam[j] * np.eye(n)
        K[:n, n] = v
        K[n, :n] = v
        rhs = np.zeros(n + 1)
        rhs[:n] = gV[:, j] - v * (v @ gV[:, j])
        mu[:, j] = np.linalg.solve(K, rhs)[:n]
    return mu


def eigenvector_grad_values(rowptr, col, V, mu):
    """The eigenvector part of dL/dA on the pattern: out[e] =
    -sum_j mu[row_e, j] V[col_e, j]."""
    n = len(rowptr) - 1
    V = np.asarray(V, dtype=np.float64).reshape(n, -1)
    mu = np.asarray(mu, dtype=np.float64).reshape(n, -1)
    out = np.empty(int(rowptr[-1]))
    for r in range(n):
        for e in range(rowptr[r], rowptr[r + 1]):
            s = 0.0
            for j in range(V.shape[1]):
                s -= mu[r, j] * V[col[e], j]
            out[e] = s
    return out


def eigen_loss_grad(rowptr, col, val, k, glam, gV):
    """dL/dA on the pattern of L = sum_j glam_j lambda_j + sum_j gV_j^T v_j
    (the k smallest pairs, signs as in smallest_eigenpairs): the
    Hellmann-Feynman part plus the eigenvector part."""
    lam, V = smallest_eigenpairs(rowptr, col, val, k)
    mu = eigenvector_adjoint(rowptr, col, val, lam, V, gV)
    return (eigenvalue_grad_values(rowptr, col, V, np.asarray(glam, dtype=np.float64))
            + eigenvector_grad_values(rowptr, col, V, mu))
