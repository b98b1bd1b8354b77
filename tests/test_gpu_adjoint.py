"""Adjoint backward (Eq. 2-3) on the GPU against the oracle gradient, the
dense formula, central finite differences (Sec. 4.3) and the closed form on
a Poisson eigenvector; plus the O(1)-node autograd bridge (Tab. 2)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6  # gradient relative error bar vs the oracle


def test_grad_values_bit_exact():
    rp, c, v = I.diffusion3d_random(17, 2)
    n = len(rp) - 1
    rng = np.random.default_rng(0)
    lam = rng.uniform(-1, 1, n)
    x = rng.uniform(-1, 1, n)
    g = sla.grad_values(csr(rp, c), to_dev(lam), to_dev(x)).cpu().numpy()
    assert np.array_equal(g, oracle.grad_values(rp, c, lam, x))


def test_config1_adjoint_matches_oracle():
    """Config 1: Poisson 64^2, b ~ U[-1,1], L = sum x^2; gradients w.r.t.
    values and b through the autograd Function vs the oracle's adjoint."""
    rp, c, v = I.poisson2d(64)
    b = I.rhs_uniform(4096, 0)
    A = csr(rp, c)
    vt = to_dev(v).requires_grad_(True)
    bt = to_dev(b).requires_grad_(True)
    x = sla.solve(A, vt, bt, rtol=1e-12)
    loss = (x * x).sum()
    loss.backward()
    xo, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    gb, gv, info = oracle.adjoint_backward(rp, c, v, xo, 2 * xo, rtol=1e-13)
    assert rel(x.detach().cpu().numpy(), xo) <= 1e-8
    assert rel(bt.grad.cpu().numpy(), gb) <= GRAD_TOL
    assert elementwise_rel(bt.grad.cpu().numpy(), gb) <= GRAD_TOL
    assert rel(vt.grad.cpu().numpy(), gv) <= GRAD_TOL
    assert elementwise_rel(vt.grad.cpu().numpy(), gv) <= GRAD_TOL


def test_autograd_graph_has_one_node():
    rp, c, v = I.diffusion2d_random(32, 1)
    A = csr(rp, c)
    vt = to_dev(v).requires_grad_(True)
    bt = to_dev(I.rhs_uniform(1024, 1)).requires_grad_(True)
    x = sla.solve(A, vt, bt)
    node = x.grad_fn
    assert type(node).__name__ == "SparseSolveBackward"
    # the solve node feeds straight from the two leaves: no per-iteration nodes
    nxt = [f for f, _ in node.next_functions if f is not None]
    assert all(type(f).__name__ == "AccumulateGrad" for f in nxt) and len(nxt) == 2


@pytest.mark.parametrize("kind", ["spd", "nonsym"])
def test_adjoint_vs_dense_formula(kind):
    if kind == "spd":
        rp, c, v = I.diffusion2d_random(20, 4)
        method = "cg"
    else:
        rp, c, v = I.convdiff3d(8, 5.0)
        method = "bicgstab"
    n = len(rp) - 1
    A = csr(rp, c)
    b = I.rhs_uniform(n, 3)
    g = I.rhs_uniform(n, 4)
    fn = sla.cg if method == "cg" else sla.bicgstab
    x, _ = fn(A, to_dev(v), to_dev(b), rtol=1e-13)
    gb, gv, info = sla.adjoint_backward(A, to_dev(v), x, to_dev(g), method=method, rtol=1e-13)
    torch.cuda.synchronize()
    assert info.status == 0
    D = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    D[rows, c] = v
    lam = np.linalg.solve(D.T, g)
    xs = np.linalg.solve(D, b)
    assert rel(gb.cpu().numpy(), lam) <= 1e-9
    assert rel(gv.cpu().numpy(), -lam[rows] * xs[c]) <= 1e-9
    gbo, gvo, _ = oracle.adjoint_backward(rp, c, v, xs, g, method=method, rtol=1e-13)
    assert rel(gv.cpu().numpy(), gvo) <= GRAD_TOL
    assert elementwise_rel(gv.cpu().numpy(), gvo) <= GRAD_TOL


@pytest.mark.parametrize("kind", ["spd", "nonsym"])
def test_central_finite_differences_32(kind):
    """Central FD (eps = 1e-5, Sec. 4.3) at 32 x 32 with tight inner solves,
    along random directions in the values and in b."""
    if kind == "spd":
        rp, c, v = I.diffusion2d_random(32, 7)
        method = "cg"
    else:
        rp, c, v = I.convdiff3d(10, 3.0)
        method = "bicgstab"
    n = len(rp) - 1
    A = csr(rp, c)
    w = to_dev(I.rhs_uniform(n, 9))
    b0 = I.rhs_uniform(n, 8)

    def L(vv, bb):
        x = sla.solve(A, vv, bb, method=method, rtol=1e-14, max_restarts=4)
        return (w * x * x).sum()

    vt = to_dev(v).requires_grad_(True)
    bt = to_dev(b0).requires_grad_(True)
    L(vt, bt).backward()
    rng = np.random.default_rng(1)
    eps = 1e-5
    for _ in range(3):
        dv = rng.standard_normal(len(v)); dv /= np.linalg.norm(dv)
        db = rng.standard_normal(n); db /= np.linalg.norm(db)
        with torch.no_grad():
            lp = float(L(to_dev(v + eps * dv * np.abs(v)), to_dev(b0 + eps * db)))
            lm = float(L(to_dev(v - eps * dv * np.abs(v)), to_dev(b0 - eps * db)))
        fd = (lp - lm) / (2 * eps)
        an = float((vt.grad.cpu().numpy() * dv * np.abs(v)).sum() + (bt.grad.cpu().numpy() * db).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_closed_form_eigenvector_gradient():
    N, j, k = 24, 3, 2
    rp, c, v = I.poisson2d(N)
    p = np.arange(1, N + 1)
    vec = np.outer(np.sin(k * np.pi * p / (N + 1)), np.sin(j * np.pi * p / (N + 1))).ravel()
    mu = 4 * math.sin(j * math.pi / (2 * (N + 1))) ** 2 + 4 * math.sin(k * math.pi / (2 * (N + 1))) ** 2
    A = csr(rp, c)
    vt = to_dev(v).requires_grad_(True)
    bt = to_dev(vec).requires_grad_(True)
    x = sla.solve(A, vt, bt, rtol=1e-14)
    (x * x).sum().backward()
    rows = np.repeat(np.arange(N * N), np.diff(rp))
    assert rel(bt.grad.cpu().numpy(), 2 * vec / mu ** 2) <= 1e-10
    assert rel(vt.grad.cpu().numpy(), -2 * vec[rows] * vec[c] / mu ** 3) <= 1e-10


def test_sparse_tensor_coo_api_gradients_in_coo_order():
    """SparseTensor(val, row, col, shape).solve(b) with shuffled COO input and
    a duplicated entry: gradients come back in the caller's COO order."""
    rp, c, v = I.diffusion2d_random(16, 5)
    n = 256
    rows = np.repeat(np.arange(n), np.diff(rp))
    perm = np.random.default_rng(3).permutation(len(c))
    row_coo = np.concatenate([rows[perm], [5]])
    col_coo = np.concatenate([c[perm], [5]]).astype(np.int64)
    val_coo = np.concatenate([v[perm], [0.25]])
    vt = to_dev(val_coo).requires_grad_(True)
    b = to_dev(I.rhs_uniform(n, 2)).requires_grad_(True)
    T = sla.SparseTensor(vt, to_dev(row_coo), to_dev(col_coo), (n, n))
    x = T.solve(b, rtol=1e-13)
    (x * x).sum().backward()
    # oracle: same COO -> CSR, solve, adjoint, map back through perm
    orp, oc, ov, operm = oracle.coo_to_csr(n, row_coo, col_coo, val_coo)
    xo, _ = oracle.pcg(orp, oc, ov, b.detach().cpu().numpy(), rtol=1e-13)
    gbo, gvo, _ = oracle.adjoint_backward(orp, oc, ov, xo, 2 * xo, rtol=1e-13)
    assert rel(x.detach().cpu().numpy(), xo) <= 1e-8
    assert rel(vt.grad.cpu().numpy(), gvo[operm]) <= GRAD_TOL
    assert elementwise_rel(vt.grad.cpu().numpy(), gvo[operm]) <= GRAD_TOL
    assert rel(b.grad.cpu().numpy(), gbo) <= GRAD_TOL
    assert elementwise_rel(b.grad.cpu().numpy(), gbo) <= GRAD_TOL


@pytest.mark.slow
def test_full_size_256_adjoint_properties():
    """Config size (3D 256^3, L = sum x^2): the adjoint solution satisfies
    ||A lambda - 2x|| <= 2 rtol ||2x|| (checked with an independent SpMV),
    and sampled value gradients equal -lambda_i x_j exactly (one product per
    entry, formed here on the host from the returned lambda and x)."""
    N = 256
    rp, c, v = I.diffusion3d_random(N, 1)
    b = I.rhs_uniform(N ** 3, 11)
    A = csr(rp, c)
    vt = to_dev(v)
    x, info = sla.cg(A, vt, to_dev(b), rtol=1e-10)
    g = 2.0 * x
    gb, gv, ia = sla.adjoint_backward(A, vt, x, g, rtol=1e-10)
    torch.cuda.synchronize()
    assert info.status == 0 and ia.status == 0
    res = sla.spmv(A, vt, gb) - g
    assert float(res.norm() / g.norm()) <= 2e-10
    rng = np.random.default_rng(5)
    ks = rng.integers(0, len(c), 4096)
    rows = np.searchsorted(rp, ks, side="right") - 1
    lam = gb.cpu().numpy()
    xh = x.cpu().numpy()
    gvh = gv.cpu().numpy()
    assert np.array_equal(gvh[ks], -lam[rows] * xh[c[ks]])
