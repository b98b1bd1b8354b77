"""FP64 CPU oracle of the inverse coefficient problem (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s reference leg
may import this module; it shares no code with the CUDA library.

Sec. 4.6 (inverse coefficient learning) with the parametrisation of the
scaled-up workload: cell-centred conductivity kappa = exp(theta) on N x N
cells, the five-point discretisation of -div(kappa grad u) with Dirichlet
ghosts, unscaled (h^2 times the operator):

* face between cells a and b:   c = (kappa_a + kappa_b) / 2
* boundary face of cell a:      c = kappa_a
* A_ii = sum of the 4 face coefficients of cell i, A_ij = -c_face.

Unknown i = p + N q (p along x); CSR rows keep ascending columns
(i-N, i-1, i, i+1, i+N).  For k right-hand sides B [k, n] and targets
X_t [k, n]:  loss = mean over (j, i) of (x_j,i - X_t j,i)^2, x_j = A^{-1} b_j.

The gradient w.r.t. theta is the adjoint of Eq. 2-3 per right-hand side
(lambda_j = A^{-1} dL/dx_j, dL/dA_ij = -sum_j lambda_j,i x_j,j), followed by
the chain rule through the face rule and exp, written out face by face.
"""
from __future__ import annotations

import numpy as np

from . import adjoint_backward, pcg


def assemble(theta):
    """(rowptr, col, val) of A(theta), plain loops over cells."""
    theta = np.asarray(theta, dtype=np.float64)
    N = theta.shape[0]
    kap = np.exp(theta)
    rowptr = [0]
    col, val = [], []
    for q in range(N):
        for p in range(N):
            i = p + N * q
            cw = 0.5 * (kap[q, p - 1] + kap[q, p]) if p > 0 else kap[q, p]
            ce = 0.5 * (kap[q, p + 1] + kap[q, p]) if p < N - 1 else kap[q, p]
            cs = 0.5 * (kap[q - 1, p] + kap[q, p]) if q > 0 else kap[q, p]
            cn = 0.5 * (kap[q + 1, p] + kap[q, p]) if q < N - 1 else kap[q, p]
            if q > 0:
                col.append(i - N)
                val.append(-cs)
            if p > 0:
                col.append(i - 1)
                val.append(-cw)
            col.append(i)
            val.append(cw + ce + cs + cn)
            if p < N - 1:
                col.append(i + 1)
                val.append(-ce)
            if q < N - 1:
                col.append(i + N)
                val.append(-cn)
            rowptr.append(len(col))
    return np.asarray(rowptr, np.int32), np.asarray(col, np.int32), np.asarray(val, np.float64)


def dense(rowptr, col, val):
    n = len(rowptr) - 1
    M = np.zeros((n, n))
    for i in range(n):
        for k in range(rowptr[i], rowptr[i + 1]):
            M[i, col[k]] += val[k]
    return M


def solve_dense(theta, B):
    """X [k, n] with A(theta) X_j = B_j by dense LU (small N only)."""
    M = dense(*assemble(theta))
    return np.linalg.solve(M, np.asarray(B, dtype=np.float64).T).T


def loss_dense(theta, B, Xt):
    X = solve_dense(theta, B)
    return float(np.mean((X - Xt) ** 2))


def entry_index(rowptr, col, i, j):
    for k in range(rowptr[i], rowptr[i + 1]):
        if col[k] == j:
            return k
    raise KeyError((i, j))


def chain_theta(theta, rowptr, col, grad_val):
    """dL/dtheta from dL/dval through the face rule and kappa = exp(theta)."""
    theta = np.asarray(theta, dtype=np.float64)
    N = theta.shape[0]
    kap = np.exp(theta)
    g = np.zeros_like(theta)
    for q in range(N):
        for p in range(N):
            a = p + N * q
            da = grad_val[entry_index(rowptr, col, a, a)]
            # boundary faces of cell a: c = kappa_a, enters A_aa only
            nb = (p == 0) + (p == N - 1) + (q == 0) + (q == N - 1)
            g[q, p] += nb * da * kap[q, p]
            # interior faces to the east and north (each face once)
            for (qq, pp) in ((q, p + 1), (q + 1, p)):
                if qq >= N or pp >= N:
                    continue
                b = pp + N * qq
                db = grad_val[entry_index(rowptr, col, b, b)]
                dab = grad_val[entry_index(rowptr, col, a, b)]
                dba = grad_val[entry_index(rowptr, col, b, a)]
                dc = da + db - dab - dba          # dL/dc of this face
                g[q, p] += dc * 0.5 * kap[q, p]
                g[qq, pp] += dc * 0.5 * kap[qq, pp]
    return g


def loss_and_grad(theta, B, Xt, rtol=1e-14):
    """(loss, dL/dtheta) with the oracle's CG forward and adjoint solves."""
    rp, c, v = assemble(theta)
    B = np.asarray(B, dtype=np.float64)
    Xt = np.asarray(Xt, dtype=np.float64)
    k, n = B.shape
    X = np.empty_like(B)
    for j in range(k):
        X[j], _ = pcg(rp, c, v, B[j], rtol=rtol)
    L = float(np.mean((X - Xt) ** 2))
    G = 2.0 * (X - Xt) / (k * n)
    gval = np.zeros(len(v))
    gB = np.empty_like(B)
    for j in range(k):
        gB[j], gv, _ = adjoint_backward(rp, c, v, X[j], G[j], method="cg", rtol=rtol)
        gval += gv
    return L, chain_theta(theta, rp, c, gval), gB
