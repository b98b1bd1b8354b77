"""Nonlinear solves with the one-solve adjoint backward (Sec. 3.2,
"Nonlinear systems"; Tab. 5, "Nonlinear (5 Newton)").

A residual F(u, params) = 0, given as ordinary differentiable PyTorch code,
is converged by Newton to u*.  Each Newton step solves J delta = -F with the
library's Krylov solvers (``sla.cg`` for SPD Jacobians, ``sla.bicgstab``
otherwise) on a fixed CSR pattern that holds J's nonzeros.  J's values come
from the residual itself: with a distance-2 colouring of the pattern's
columns (``sla.colour_columns``) one Jacobian-vector product per colour --
forward-mode autograd, all colours batched -- yields every entry, which the
library's gather kernel writes in CSR order (Curtis-Powell-Reid).  The
backward pass is the paper's: one adjoint solve J(u*)^T lambda = dL/du*
(``sla.adjoint_backward``), then dL/dparams = -(dF/dparams)^T lambda, a
vector-Jacobian product of the residual.  It is exact once F(u*) ~ 0; an
early stop biases it, as the paper notes.

``SemilinearDiffusion`` is the synthetic workload: the inverse problem's
grid and face rule (kappa = exp(theta), unscaled five-point operator) with a
cubic reaction, F = A(theta) u + h^2 (gamma u^3 - f).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
from torch.func import jvp, vmap

from . import inputs as I
from . import sla

__all__ = ["SparseJacobian", "newton", "nonlinear_solve", "NewtonInfo", "SemilinearDiffusion"]


class SparseJacobian:
    """Values of dF/du on a CSR pattern from coloured Jacobian-vector
    products.  ``F`` maps u [n] to F(u) [n] (the other arguments bound)."""

    def __init__(self, A: sla.CSRMatrix, rowptr=None, col=None):
        self.A = A
        rp = np.asarray(rowptr if rowptr is not None else A.rowptr.cpu().numpy(), dtype=np.int32)
        c = np.asarray(col if col is not None else A.col.cpu().numpy(), dtype=np.int32)
        colour, self.ncolours = sla.colour_columns(rp, c)
        n = A.n
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
        idx = colour[c].astype(np.int64) * n + rows
        if idx.size and idx.max() >= 2 ** 31:
            raise ValueError("pattern too large for one coloured Jacobian (n x colours >= 2^31)")
        dev = A.device
        self.idx = torch.from_numpy(idx.astype(np.int32)).to(dev)
        seeds = np.zeros((self.ncolours, n))
        seeds[colour, np.arange(n)] = 1.0
        self.seeds = torch.from_numpy(seeds).to(dev)

    def values(self, F, u: torch.Tensor) -> torch.Tensor:
        """J's values in CSR order at u."""
        u = u.detach()
        Y = vmap(lambda t: jvp(F, (u,), (t,))[1])(self.seeds)
        return sla.gather_values(self.idx, Y.contiguous().reshape(-1))


@dataclass
class NewtonInfo:
    newton_iters: int
    krylov_iters: list
    residual_norms: list
    converged: bool


def newton(F, u0: torch.Tensor, jac: SparseJacobian, *, method: str = "cg", tol: float = 1e-10,
           atol: float = 0.0, max_newton: int = 30, lin_rtol: float = 1e-12, **solver_kw):
    """Newton's method for F(u) = 0 from u0: stop when ||F(u)||_2 <=
    max(tol ||F(u0)||_2, atol), or (not converged) when a step no longer
    lowers ||F|| -- the rounding floor of F's evaluation -- or after
    max_newton steps.  Each step's linear solve runs on the library's
    kernels.  Returns (u, NewtonInfo)."""
    solve = sla.cg if method == "cg" else sla.bicgstab
    u = u0.detach().clone()
    with torch.no_grad():
        Fu = F(u)
    norms = [float(Fu.norm())]
    target = max(tol * norms[0], atol)
    kits = []
    k = 0
    while norms[-1] > target and k < max_newton:
        vals = jac.values(F, u)
        delta, info = solve(jac.A, vals, (-Fu).contiguous(), rtol=lin_rtol, **solver_kw)
        if info.status != 0:
            raise sla.SolveError("Newton step %d: %s after %d iterations" % (k, info.status_name, info.iters))
        kits.append(info.iters)
        u = u + delta
        with torch.no_grad():
            Fu = F(u)
        norms.append(float(Fu.norm()))
        k += 1
        if norms[-1] >= norms[-2]:
            break
    return u, NewtonInfo(k, kits, norms, norms[-1] <= target)


class _NonlinearSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, u0, jac, opts, *params):
        p = [q.detach() for q in params]
        u, info = newton(lambda v: F(v, *p), u0, jac, **opts)
        jac.last_info = info
        ctx.F, ctx.jac, ctx.opts = F, jac, opts
        ctx.save_for_backward(u, *params)
        return u

    @staticmethod
    def backward(ctx, gu):
        u, *params = ctx.saved_tensors
        F, jac, opts = ctx.F, ctx.jac, ctx.opts
        p = [q.detach() for q in params]
        vals = jac.values(lambda v: F(v, *p), u)
        method = opts.get("method", "cg")
        rtol = opts.get("lin_rtol", 1e-12)
        # one adjoint solve J^T lambda = dL/du* (A^T = A for "cg")
        lam, _, info = sla.adjoint_backward(jac.A, vals, u, gu.contiguous().to(torch.float64),
                                            method=method, rtol=rtol)
        if info.status != 0:
            raise sla.SolveError("nonlinear adjoint: %s after %d iterations" % (info.status_name, info.iters))
        need = [q.requires_grad for q in params]
        grads = [None] * len(params)
        if any(need):
            with torch.enable_grad():
                pp = [q.detach().requires_grad_(r) for q, r in zip(params, need)]
                Fv = F(u.detach(), *pp)
                gs = torch.autograd.grad(Fv, [q for q, r in zip(pp, need) if r], grad_outputs=-lam)
            it = iter(gs)
            grads = [next(it) if r else None for r in need]
        return (None, None, None, None, *grads)


def nonlinear_solve(F, u0: torch.Tensor, params: tuple, jac: SparseJacobian, **opts) -> torch.Tensor:
    """u* with F(u*, *params) = 0, differentiable w.r.t. params (Sec. 3.2):
    Newton forward on the library's solvers, one adjoint solve backward.
    opts: method ("cg" | "bicgstab"), tol, atol, max_newton, lin_rtol.
    The Newton record of the last forward is ``jac.last_info``."""
    return _NonlinearSolve.apply(F, u0, jac, opts, *params)


class SemilinearDiffusion:
    """F(u, theta) = A(theta) u + h^2 (gamma u^3 - f) on N x N cells:
    A(theta) the unscaled five-point operator of -div(exp(theta) grad u)
    with the inverse problem's face rule (face = mean of the two cells'
    kappa, boundary face = the cell's kappa), h = 1/(N + 1).  theta is a
    smooth Gaussian random field (std 0.5), f = 1 + U[-1/2, 1/2] noise, and
    the target is u* at a second field."""

    def __init__(self, N: int = 512, gamma: float = 10.0, *, seed_theta: int = 5000, seed_target: int = 5001,
                 seed_f: int = 5002, sigma_cells: float = 8.0, std: float = 0.5, device="cuda"):
        self.N, self.n, self.gamma = N, N * N, float(gamma)
        self.h2 = 1.0 / (N + 1) ** 2
        dev = torch.device(device)
        self.device = dev
        rp, c, _ = I.poisson2d(N)
        self.rowptr, self.col = rp, c
        self.A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
        self.jac = SparseJacobian(self.A, rp, c)
        self.jac.last_info = None
        self.theta0 = torch.from_numpy(I.gaussian_random_field(N, seed_theta, sigma_cells, std)).to(dev)
        self.theta_t = torch.from_numpy(I.gaussian_random_field(N, seed_target, sigma_cells, std)).to(dev)
        rng = np.random.default_rng(seed_f)
        self.f = torch.from_numpy(1.0 + 0.5 * rng.uniform(-1.0, 1.0, self.n)).to(dev)

    def residual(self, u: torch.Tensor, theta: torch.Tensor) -> torch.Tensor:
        N = self.N
        kap = torch.exp(theta)
        U = u.view(N, N)
        mid_x = 0.5 * (kap[:, 1:] + kap[:, :-1])
        mid_y = 0.5 * (kap[1:, :] + kap[:-1, :])
        cw = torch.cat([kap[:, :1], mid_x], 1)
        ce = torch.cat([mid_x, kap[:, -1:]], 1)
        cs = torch.cat([kap[:1, :], mid_y], 0)
        cn = torch.cat([mid_y, kap[-1:, :]], 0)
        zc = torch.zeros(N, 1, dtype=u.dtype, device=u.device)
        zr = torch.zeros(1, N, dtype=u.dtype, device=u.device)
        Uw = torch.cat([zc, U[:, :-1]], 1)
        Ue = torch.cat([U[:, 1:], zc], 1)
        Us = torch.cat([zr, U[:-1, :]], 0)
        Un = torch.cat([U[1:, :], zr], 0)
        Au = (cw + ce + cs + cn) * U - cw * Uw - ce * Ue - cs * Us - cn * Un
        return Au.reshape(-1) + self.h2 * (self.gamma * u ** 3 - self.f)

    def solve(self, theta: torch.Tensor, **opts) -> torch.Tensor:
        u0 = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        return nonlinear_solve(self.residual, u0, (theta,), self.jac, **opts)

    def target(self, **opts) -> torch.Tensor:
        with torch.no_grad():
            return self.solve(self.theta_t, **opts)

    def loss(self, theta: torch.Tensor, u_target: torch.Tensor, **opts) -> torch.Tensor:
        u = self.solve(theta, **opts)
        return torch.mean((u - u_target) ** 2)
