"""FP64 CPU oracle of the nonlinear adjoint (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s reference leg
may import this module; it shares no code with the CUDA library.

Sec. 3.2, "Nonlinear systems": a residual F(u, theta) = 0 converged by
Newton to u*; the gradient of a loss L(u*) is one adjoint solve with the
Jacobian at the solution, J^T lambda = dL/du*, then
dL/dtheta = -(dF/dtheta)^T lambda (Eq. 2 with J in place of A).

The residual is the semilinear diffusion problem on the inverse problem's
N x N cells (kappa = exp(theta), the same unscaled five-point A(theta) as
``oracle.inverse.assemble``), with a cubic reaction:

    F(u, theta) = A(theta) u + h^2 (gamma u^3 - f),   h = 1 / (N + 1),

so J = A(theta) + 3 h^2 gamma diag(u^2) (SPD for gamma >= 0).  Newton starts
from u0 = 0 and stops when ||F(u)||_2 <= max(tol ||F(u0)||_2, atol); each
step solves J delta = -F by sparse LU.  Because F is linear in the entries
of A, dF_i/dA_ij = u_j and dL/dA_ij = -lambda_i u*_j; the chain to theta is
``oracle.inverse.chain_theta``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .inverse import assemble, chain_theta


def residual(theta, u, f, gamma):
    """F(u, theta) with A(theta) assembled by plain loops."""
    rp, c, v = assemble(theta)
    N = np.asarray(theta).shape[0]
    h2 = 1.0 / (N + 1) ** 2
    u = np.asarray(u, dtype=np.float64)
    n = len(rp) - 1
    F = np.empty(n)
    for i in range(n):
        s = 0.0
        for k in range(rp[i], rp[i + 1]):
            s += v[k] * u[c[k]]
        F[i] = s + h2 * (gamma * u[i] ** 3 - f[i])
    return F


def jacobian(theta, u, gamma):
    """(rowptr, col, val) of J = A(theta) + 3 h^2 gamma diag(u^2)."""
    rp, c, v = assemble(theta)
    N = np.asarray(theta).shape[0]
    h2 = 1.0 / (N + 1) ** 2
    v = v.copy()
    for i in range(len(rp) - 1):
        for k in range(rp[i], rp[i + 1]):
            if c[k] == i:
                v[k] += 3.0 * h2 * gamma * u[i] ** 2
    return rp, c, v


def newton(theta, f, gamma, tol=1e-12, atol=0.0, max_newton=30):
    """u* and the history of ||F(u_k)||_2 (u0 = 0)."""
    n = np.asarray(theta).size
    u = np.zeros(n)
    F = residual(theta, u, f, gamma)
    f0 = np.linalg.norm(F)
    hist = [f0]
    target = max(tol * f0, atol)
    for _ in range(max_newton):
        if hist[-1] <= target:
            break
        rp, c, v = jacobian(theta, u, gamma)
        J = sp.csr_matrix((v, c, rp), shape=(n, n)).tocsc()
        u = u + spla.spsolve(J, -F)
        F = residual(theta, u, f, gamma)
        hist.append(np.linalg.norm(F))
    return u, hist


def loss_and_grad(theta, f, gamma, u_target, tol=1e-13):
    """L = mean((u* - u_target)^2) and dL/dtheta by the adjoint."""
    theta = np.asarray(theta, dtype=np.float64)
    u, _ = newton(theta, f, gamma, tol=tol)
    n = u.size
    L = float(np.mean((u - u_target) ** 2))
    g = 2.0 * (u - u_target) / n
    rp, c, v = jacobian(theta, u, gamma)
    J = sp.csr_matrix((v, c, rp), shape=(n, n))
    lam = spla.spsolve(J.T.tocsc(), g)
    # dL/dA_ij = -lambda_i u_j on A's pattern (F is linear in A's entries)
    ra, ca, _ = assemble(theta)
    gval = np.empty(len(ca))
    for i in range(n):
        for k in range(ra[i], ra[i + 1]):
            gval[k] = -lam[i] * u[ca[k]]
    return L, chain_theta(theta, ra, ca, gval), u


def loss(theta, f, gamma, u_target, tol=1e-13):
    u, _ = newton(theta, f, gamma, tol=tol)
    return float(np.mean((u - u_target) ** 2))
