"""The distributed layer (Sec. 3.3, Eqs. 5-6, Algorithm 1) with its
partitions emulated on one GPU: the halo exchange and its transpose against
their definitions, the distributed SpMV against the global one, the
distributed CG against the oracle's PCG, and its adjoint gradients against
the oracle's."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import distributed as D
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu


def test_halo_exchange_and_transpose_bit_exact():
    rp, c, v = I.diffusion3d_random(9, 4)
    n = len(rp) - 1
    DA = D.DistributedMatrix(rp, c, 5)
    lay = DA.layout
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n)
    g = rng.standard_normal(DA.total_ext)
    xe = D._halo_gather(DA, to_dev(x)).cpu().numpy()
    assert np.array_equal(xe, x[lay["src"]])
    gx = D._halo_scatter(DA, to_dev(g)).cpu().numpy()
    want = g[lay["own_pos"]].copy()
    for i in range(n):
        for t in range(lay["hptr"][i], lay["hptr"][i + 1]):
            want[i] += g[lay["hlist"][t]]
    assert np.array_equal(gx, want)


@pytest.mark.parametrize("P", [1, 3, 8])
def test_dist_spmv_equals_global_spmv_and_its_gradients(P):
    """y = A_local H(x) is the global product to the bit (same rows, same
    entry order); dL/dx = H^T(A_local^T dL/dy) (Eq. 6) equals A^T dL/dy,
    dL/dA_ij = dL/dy_i x_j."""
    rp, c, v = I.fem_p1_laplacian(14, 2)
    n = len(rp) - 1
    DA = D.DistributedMatrix(rp, c, P, balance="nnz")
    A = csr(rp, c)
    rng = np.random.default_rng(2)
    x = to_dev(rng.standard_normal(n)).requires_grad_(True)
    val = to_dev(v).requires_grad_(True)
    y = D.dist_spmv(DA, val, x)
    assert torch.equal(y.detach(), sla.spmv(A, to_dev(v), x.detach()))
    w = to_dev(rng.standard_normal(n))
    (w * y).sum().backward()
    Ad = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(Ad, (rows, c), v)
    wn = w.cpu().numpy()
    assert np.allclose(x.grad.cpu().numpy(), Ad.T @ wn, rtol=0, atol=1e-12)
    assert np.allclose(val.grad.cpu().numpy(), wn[rows] * x.detach().cpu().numpy()[c], rtol=0, atol=1e-14)


@pytest.mark.parametrize("gen,P", [("var3d", 1), ("var3d", 4), ("var3d", 7), ("fem", 5), ("poisson", 2)])
def test_dist_cg_matches_oracle(gen, P):
    if gen == "var3d":
        rp, c, v = I.diffusion3d_random(16, 3)
    elif gen == "fem":
        rp, c, v = I.fem_p1_laplacian(30, 6)
    else:
        rp, c, v = I.poisson2d(40)
    n = len(rp) - 1
    b = I.rhs_uniform(n, 8)
    DA = D.DistributedMatrix(rp, c, P)
    x, info = D.dist_cg(DA, to_dev(v), to_dev(b), rtol=1e-10)
    xo, io = oracle.pcg(rp, c, v, b, rtol=1e-13)
    _, io10 = oracle.pcg(rp, c, v, b, rtol=1e-10)
    assert info["status"] == 0 and io["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-8
    assert elementwise_rel(x.cpu().numpy(), xo) <= 1e-8
    assert abs(info["iters"] - io10["iters"]) <= max(2, io10["iters"] // 50)
    assert info["true_rel_res"] <= 2e-10
    assert len(info["halo_sizes"]) == P and (P == 1) == (sum(info["halo_sizes"]) == 0)


def test_dist_cg_edge_cases():
    rp, c, v = I.poisson2d(10)
    DA = D.DistributedMatrix(rp, c, 3)
    x, info = D.dist_cg(DA, to_dev(v), to_dev(np.zeros(100)))
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    v2 = v.copy()
    v2[(np.repeat(np.arange(100), np.diff(rp)) == 57) & (c == 57)] = -1.0
    _, info = D.dist_cg(DA, to_dev(v2), to_dev(np.ones(100)))
    _, io = oracle.pcg(rp, c, v2, np.ones(100))
    assert info["status"] == io["status"] == 3
    _, info = D.dist_cg(DA, to_dev(v), to_dev(I.rhs_uniform(100, 1)), rtol=1e-15, max_iter=4, max_restarts=0)
    assert info["status"] == 1 and info["iters"] == 4


@pytest.mark.parametrize("P", [2, 6])
def test_dist_solve_adjoint_matches_oracle(P):
    """Distributed CG forward, one distributed adjoint solve backward,
    -lambda_i x_j assembled on every partition's own entries."""
    rp, c, v = I.diffusion2d_random(24, 5)
    n = len(rp) - 1
    b = I.rhs_uniform(n, 9)
    DA = D.DistributedMatrix(rp, c, P)
    val = to_dev(v).requires_grad_(True)
    bt = to_dev(b).requires_grad_(True)
    x = D.dist_solve(DA, val, bt, rtol=1e-12)
    (x * x).sum().backward()
    xo, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    gb, gv, io = oracle.adjoint_backward(rp, c, v, xo, 2 * xo, rtol=1e-13)
    assert io["status"] == 0
    for got, want in ((bt.grad, gb), (val.grad, gv)):
        assert rel(got.cpu().numpy(), want) <= 1e-6
        assert elementwise_rel(got.cpu().numpy(), want) <= 1e-6
