"""Several right-hand sides sharing one matrix (sla_cg_multi and its adjoint)
and the inverse coefficient problem built on them (Sec. 4.6), against the
oracle: per-column solutions at relative residual 1e-10 within 1e-8 of the
oracle's tight solution, gradients within 1e-6, statuses and edge cases
identical to the single right-hand-side solver."""
import numpy as np
import pytest
import torch

import oracle
import oracle.inverse as OI
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from paper_2601_13994_b300.inverse import InverseProblem
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6


def run_multi(rp, c, v, B, **kw):
    A = csr(rp, c)
    X, info = sla.cg_multi(A, to_dev(v), to_dev(B), **kw)
    torch.cuda.synchronize()
    return X.cpu().numpy(), info


@pytest.mark.parametrize("k", [1, 3, 16, 32])
def test_multi_matches_oracle_per_column(k):
    rp, c, v = I.diffusion2d_random(40, 7)
    n = len(rp) - 1
    B = I.rhs_uniform(n, 30 + k, batch=k)
    X, info = run_multi(rp, c, v, B, rtol=1e-10)
    its = np.atleast_1d(info.iters)
    st = np.atleast_1d(info.status)
    trr = np.atleast_1d(info.true_rel_res)
    for j in range(k):
        xo, _ = oracle.pcg(rp, c, v, B[j], rtol=1e-13)
        _, io = oracle.pcg(rp, c, v, B[j], rtol=1e-10)
        assert st[j] == 0
        assert rel(X[j], xo) <= 1e-8
        assert abs(int(its[j]) - io["iters"]) <= max(2, io["iters"] // 50)
        assert trr[j] <= 2e-10


def test_multi_edge_cases():
    rp, c, v = I.diffusion2d_random(24, 3)
    n = len(rp) - 1
    A = csr(rp, c)
    vt = to_dev(v)
    # zero right-hand sides among nonzero ones: x = 0, 0 iterations, OK
    B = I.rhs_uniform(n, 9, batch=5)
    B[1] = 0.0
    B[4] = 0.0
    X, info = sla.cg_multi(A, vt, to_dev(B), rtol=1e-10)
    X = X.cpu().numpy()
    assert list(info.status) == [0] * 5
    assert info.iters[1] == 0 and info.iters[4] == 0
    assert np.all(X[1] == 0.0) and np.all(X[4] == 0.0)
    for j in (0, 2, 3):
        xo, _ = oracle.pcg(rp, c, v, B[j], rtol=1e-13)
        assert rel(X[j], xo) <= 1e-8
    # initial guess = solution: converged by the initial check
    X0 = torch.from_numpy(X).to("cuda")
    X2, info2 = sla.cg_multi(A, vt, to_dev(B), rtol=1e-8, x0=X0)
    assert list(info2.status) == [0] * 5 and max(info2.iters) <= 1
    # max_iter reached
    X3, info3 = sla.cg_multi(A, vt, to_dev(B[:2]), rtol=1e-14, max_iter=3, max_restarts=0)
    assert list(info3.status) == [1, 0] and list(info3.iters) == [3, 0]
    _, io = oracle.pcg(rp, c, v, B[0], rtol=1e-14, max_iter=3, max_restarts=0)
    assert io["status"] == 1 and io["iters"] == 3
    # non-positive diagonal with Jacobi: every column NOT_SPD
    v_bad = v.copy()
    d0 = [k for k in range(rp[5], rp[6]) if c[k] == 5][0]
    v_bad[d0] = 0.0
    _, info4 = sla.cg_multi(A, to_dev(v_bad), to_dev(B[:3]), rtol=1e-10)
    assert list(info4.status) == [3, 3, 3]
    # empty system
    A0 = sla.CSRMatrix(torch.zeros(1, dtype=torch.int32, device="cuda"),
                       torch.zeros(0, dtype=torch.int32, device="cuda"))
    X5, info5 = sla.cg_multi(A0, torch.zeros(0, dtype=torch.float64, device="cuda"),
                             torch.zeros((2, 0), dtype=torch.float64, device="cuda"))
    assert list(info5.status) == [0, 0]


def test_multi_unpreconditioned_and_host_loop_identical():
    rp, c, v = I.fem_p1_laplacian(30, 5)
    n = len(rp) - 1
    B = I.rhs_uniform(n, 12, batch=6)
    Xg, ig = run_multi(rp, c, v, B, rtol=1e-10, precond="none")
    Xh, ih = run_multi(rp, c, v, B, rtol=1e-10, precond="none", graph=False)
    assert np.array_equal(Xg, Xh)
    assert np.array_equal(np.atleast_1d(ig.iters), np.atleast_1d(ih.iters))
    for j in range(6):
        xo, _ = oracle.pcg(rp, c, v, B[j], rtol=1e-13, precond="none")
        assert rel(Xg[j], xo) <= 1e-8


def test_multi_adjoint_matches_oracle():
    rp, c, v = I.diffusion2d_random(32, 11)
    n = len(rp) - 1
    k = 5
    B = I.rhs_uniform(n, 40, batch=k)
    G = I.rhs_uniform(n, 41, batch=k)
    A = csr(rp, c)
    X, _ = sla.cg_multi(A, to_dev(v), to_dev(B), rtol=1e-13)
    gb, gv, info = sla.adjoint_backward_multi(A, to_dev(v), X, to_dev(G), rtol=1e-13)
    assert list(info.status) == [0] * k
    gb = gb.cpu().numpy()
    gv = gv.cpu().numpy()
    Xn = X.cpu().numpy()
    ref_gv = np.zeros(len(v))
    for j in range(k):
        lam, g1, _ = oracle.adjoint_backward(rp, c, v, Xn[j], G[j], method="cg", rtol=1e-13)
        assert rel(gb[j], lam) <= GRAD_TOL
        assert elementwise_rel(gb[j], lam) <= GRAD_TOL
        ref_gv += g1
    assert rel(gv, ref_gv) <= GRAD_TOL
    assert elementwise_rel(gv, ref_gv) <= GRAD_TOL
    # the gradient pass alone, from the same lambda and x, is the sum of the
    # per-column Eq. 3 products
    ref2 = sum(oracle.grad_values(rp, c, gb[j], Xn[j]) for j in range(k))
    assert rel(gv, ref2) <= 1e-14


def test_solve_multi_autograd_against_oracle():
    rp, c, v = I.diffusion2d_random(20, 2)
    n = len(rp) - 1
    k = 4
    B = I.rhs_uniform(n, 50, batch=k)
    W = I.rhs_uniform(n, 51, batch=k)
    A = csr(rp, c)
    vt = to_dev(v).requires_grad_(True)
    bt = to_dev(B).requires_grad_(True)
    X = sla.solve_multi(A, vt, bt, rtol=1e-13)
    (X * to_dev(W)).sum().backward()
    gv_ref = np.zeros(len(v))
    for j in range(k):
        xj, _ = oracle.pcg(rp, c, v, B[j], rtol=1e-14)
        lam, g1, _ = oracle.adjoint_backward(rp, c, v, xj, W[j], method="cg", rtol=1e-14)
        assert rel(bt.grad[j].cpu().numpy(), lam) <= GRAD_TOL
        assert elementwise_rel(bt.grad[j].cpu().numpy(), lam) <= GRAD_TOL
        gv_ref += g1
    assert rel(vt.grad.cpu().numpy(), gv_ref) <= GRAD_TOL
    assert elementwise_rel(vt.grad.cpu().numpy(), gv_ref) <= GRAD_TOL


def test_inverse_gradient_32_matches_oracle_and_fd():
    """Config: 2D inverse problem at 32 x 32, 16 right-hand sides; GPU loss
    and dL/dtheta (multi-RHS PCG + adjoint + autograd through the assembly)
    against the oracle's and against central differences of the dense-LU
    loss (eps = 1e-5)."""
    P = InverseProblem(32, 16, seed_theta=4010, seed_rhs=4011, target_rtol=1e-13)
    th0 = 0.8 * torch.from_numpy(I.gaussian_random_field(32, 4012)).to("cuda")
    L, g = P.loss_and_grad(th0, rtol=1e-13)
    th_np = th0.cpu().numpy()
    B = P.B.cpu().numpy()
    Xt = P.X_target.cpu().numpy()
    # the target itself against the oracle's dense solve at theta_true
    Xt_ref = OI.solve_dense(P.theta_true.cpu().numpy(), B)
    assert rel(Xt, Xt_ref) <= 1e-8
    Lo, go, _ = OI.loss_and_grad(th_np, B, Xt, rtol=1e-14)
    assert abs(float(L) - Lo) <= 1e-9 * Lo
    g = g.cpu().numpy()
    assert rel(g, go) <= GRAD_TOL
    assert elementwise_rel(g, go) <= GRAD_TOL
    rng = np.random.default_rng(3)
    eps = 1e-5
    for _ in range(3):
        d = rng.standard_normal(th_np.shape)
        fd = (OI.loss_dense(th_np + eps * d, B, Xt) - OI.loss_dense(th_np - eps * d, B, Xt)) / (2 * eps)
        assert abs(fd - float((g * d).sum())) <= GRAD_TOL * abs(fd)


@pytest.mark.slow
def test_inverse_full_size_512_16rhs():
    """Config size (512 x 512, 16 right-hand sides): every forward and
    adjoint column converges with a true residual within 2 rtol (checked
    here with an independent SpMV), and the gradient agrees with a central
    difference of the GPU loss along a smooth direction (a property that
    holds at any size)."""
    P = InverseProblem(512, 16)
    th0 = torch.zeros((512, 512), dtype=torch.float64, device="cuda")
    th = th0.clone().requires_grad_(True)
    X = P.solve(th, rtol=1e-10)
    vals = P.values(th0)
    for j in range(16):
        r = P.B[j] - sla.spmv(P.A, vals, X[j].detach().contiguous())
        assert float(r.norm() / P.B[j].norm()) <= 2e-10
    L = ((X - P.X_target) ** 2).mean()
    L.backward()
    g = th.grad
    d = torch.from_numpy(I.gaussian_random_field(512, 4099)).to("cuda")
    eps = 1e-4
    with torch.no_grad():
        lp = P.loss(th0 + eps * d, rtol=1e-12)
        lm = P.loss(th0 - eps * d, rtol=1e-12)
    fd = float((lp - lm) / (2 * eps))
    an = float((g * d).sum())
    assert abs(fd - an) <= 1e-5 * abs(fd)
