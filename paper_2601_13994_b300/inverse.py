"""Differentiable inverse coefficient problem (Sec. 4.6), scaled up: learn a
cell-centred log-conductivity theta on an N x N grid from solutions of
-div(exp(theta) grad u) = b_j for a batch of right-hand sides.

The forward and backward solves are the library's multi-right-hand-side PCG
and its adjoint (sla_cg_multi / sla_adjoint_backward_multi behind
``sla.solve_multi``); the assembly of A's values from theta is ordinary
differentiable PyTorch code on the device, as the paper's user code
assembles its SparseTensor (Sec. 4.6):

* kappa = exp(theta), face coefficient between cells a, b = (kappa_a +
  kappa_b) / 2, boundary face of a cell = its kappa (Dirichlet ghosts);
* A_ii = sum of the cell's four face coefficients, A_ij = -c_face,
  unscaled (h^2 times the operator), on the 5-point pattern of the grid;
* loss = mean over the batch and the n unknowns of (x - x_target)^2, with
  x_target the solve at the true field.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs as I
from . import sla

__all__ = ["InverseProblem", "assemble_values"]


def _selection(N: int, device) -> torch.Tensor:
    """Flat indices into a [n, 5] (south, west, diag, east, north) table of
    the entries that exist, in CSR order (ascending columns per row)."""
    n = N * N
    q, p = np.divmod(np.arange(n), N)
    mask = np.stack([q > 0, p > 0, np.ones(n, bool), p < N - 1, q < N - 1], axis=1)
    return torch.from_numpy(np.flatnonzero(mask.reshape(-1))).to(device)


def assemble_values(theta: torch.Tensor, sel: torch.Tensor) -> torch.Tensor:
    """CSR values of A(theta) on the 5-point pattern (differentiable)."""
    kap = torch.exp(theta)
    mid_x = 0.5 * (kap[:, 1:] + kap[:, :-1])        # faces between columns p-1, p
    mid_y = 0.5 * (kap[1:, :] + kap[:-1, :])        # faces between rows q-1, q
    cw = torch.cat([kap[:, :1], mid_x], dim=1)
    ce = torch.cat([mid_x, kap[:, -1:]], dim=1)
    cs = torch.cat([kap[:1, :], mid_y], dim=0)
    cn = torch.cat([mid_y, kap[-1:, :]], dim=0)
    diag = cw + ce + cs + cn
    table = torch.stack([-cs, -cw, diag, -ce, -cn], dim=-1).reshape(-1)
    return table[sel]


class InverseProblem:
    """Synthetic instance: theta_true a smooth Gaussian random field
    (``inputs.gaussian_random_field``), k right-hand sides ~ U[-1, 1], and
    the target solutions at theta_true."""

    def __init__(self, N: int = 512, k: int = 16, *, seed_theta: int = 4000, seed_rhs: int = 4001,
                 sigma_cells: float = 8.0, std: float = 0.5, rtol: float = 1e-8,
                 target_rtol: float = 1e-10, device="cuda"):
        self.N, self.k, self.n = N, k, N * N
        self.device = torch.device(device)
        rp, c, _ = I.poisson2d(N)
        self.A = sla.CSRMatrix.from_numpy(rp, c, device=self.device)
        self.sel = _selection(N, self.device)
        self.rtol = rtol
        self.theta_true = torch.from_numpy(I.gaussian_random_field(N, seed_theta, sigma_cells, std)).to(self.device)
        self.B = torch.from_numpy(I.rhs_uniform(self.n, seed_rhs, batch=k)).to(self.device)
        with torch.no_grad():
            self.X_target = sla.solve_multi(self.A, self.values(self.theta_true), self.B, rtol=target_rtol)

    def values(self, theta: torch.Tensor) -> torch.Tensor:
        return assemble_values(theta, self.sel)

    def solve(self, theta: torch.Tensor, **kw) -> torch.Tensor:
        kw.setdefault("rtol", self.rtol)
        return sla.solve_multi(self.A, self.values(theta), self.B, **kw)

    def loss(self, theta: torch.Tensor, **kw) -> torch.Tensor:
        X = self.solve(theta, **kw)
        return ((X - self.X_target) ** 2).mean()

    def loss_and_grad(self, theta: torch.Tensor, **kw):
        th = theta.detach().clone().requires_grad_(True)
        L = self.loss(th, **kw)
        L.backward()
        return L.detach(), th.grad
