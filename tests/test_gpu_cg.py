"""Jacobi-PCG parity: GPU solutions against the oracle's solution (and dense
LU where small) on the same seeded inputs.  Bar: relative solution error
<= 1e-8 at relative residual 1e-10; statuses and edge cases identical."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, rel, sampled_errors, stored_oracle, to_dev

pytestmark = pytest.mark.gpu


def gpu_cg(rp, c, v, b, **kw):
    A = csr(rp, c)
    x, info = sla.cg(A, to_dev(v), to_dev(b), **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info.as_dict()


def exact(rp, c, v, b):
    return spl.spsolve(sp.csr_matrix((v, c, rp)).tocsc(), b)


def test_config1_poisson64_matches_oracle_and_lu():
    rp, c, v = I.poisson2d(64)
    b = I.rhs_uniform(4096, 0)
    x, info = gpu_cg(rp, c, v, b, rtol=1e-10)
    xo, io = oracle.pcg(rp, c, v, b, rtol=1e-10)
    xs = exact(rp, c, v, b)
    assert info["status"] == 0 and io["status"] == 0
    assert rel(x, xs) <= 1e-8
    assert rel(x, xo) <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2
    assert info["true_rel_res"] <= 2e-10
    assert abs(info["true_rel_res"] - io["true_rel_res"]) <= 1e-10


@pytest.mark.parametrize("N,seed", [(16, 1), (33, 2), (48, 3)])
def test_diffusion3d_matches_oracle(N, seed):
    rp, c, v = I.diffusion3d_random(N, seed)
    n = N ** 3
    b = I.rhs_uniform(n, seed + 100)
    x, info = gpu_cg(rp, c, v, b, rtol=1e-10)
    xo, io = oracle.pcg(rp, c, v, b, rtol=1e-13)
    assert info["status"] == 0
    assert rel(x, xo) <= 1e-8
    _, io10 = oracle.pcg(rp, c, v, b, rtol=1e-10)
    assert abs(info["iters"] - io10["iters"]) <= max(2, io10["iters"] // 50)


def test_fem_and_unpreconditioned():
    rp, c, v = I.fem_p1_laplacian(40, 8)
    n = len(rp) - 1
    b = I.rhs_uniform(n, 4)
    for pc in ("jacobi", "none"):
        x, info = gpu_cg(rp, c, v, b, rtol=1e-10, precond=pc)
        xo, io = oracle.pcg(rp, c, v, b, rtol=1e-10, precond=pc)
        assert info["status"] == 0 and io["status"] == 0
        assert rel(x, exact(rp, c, v, b)) <= 1e-8
        assert abs(info["iters"] - io["iters"]) <= max(2, io["iters"] // 50)


@pytest.mark.parametrize("coop", [True, False])
def test_edge_cases_match_oracle(coop):
    """b = 0 (with a discarded warm start), a negative diagonal, an
    indefinite system, iteration caps, NaN, a warm start at the solution,
    n = 1 and atol-only stopping, through the cooperative launch and through
    the graph of per-phase kernels (the path of the large systems)."""
    rp, c, v = I.poisson2d(6)
    n = 36
    # b = 0 (also with a warm start, which must be discarded)
    x, info = gpu_cg(rp, c, v, np.zeros(n), cooperative=coop)
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    A = csr(rp, c)
    x0 = to_dev(np.ones(n))
    xx, inf = sla.cg(A, to_dev(v), to_dev(np.zeros(n)), x0=x0, cooperative=coop)
    assert inf.status == 0 and not xx.cpu().numpy().any()
    # non-positive diagonal -> NOT_SPD, NaN residuals
    v2 = v.copy()
    v2[rp[3]:rp[4]][c[rp[3]:rp[4]] == 3] = -1.0
    _, info = gpu_cg(rp, c, v2, np.ones(n), cooperative=coop)
    _, io = oracle.pcg(rp, c, v2, np.ones(n))
    assert info["status_name"] == io["status_name"] == "NOT_SPD"
    assert np.isnan(info["rel_res"])
    # indefinite, positive diagonal -> p^T A p <= 0
    rpi = np.array([0, 2, 4], np.int32); ci = np.array([0, 1, 0, 1], np.int32)
    vi = np.array([1.0, 2.0, 2.0, 1.0])
    _, info = gpu_cg(rpi, ci, vi, np.array([1.0, -1.0]), cooperative=coop)
    assert info["status_name"] == "NOT_SPD"
    # iteration cap
    b = I.rhs_uniform(n, 0)
    _, info = gpu_cg(rp, c, v, b, rtol=1e-14, max_iter=2, cooperative=coop)
    _, io = oracle.pcg(rp, c, v, b, rtol=1e-14, max_iter=2)
    assert info["status_name"] == io["status_name"] == "NOT_CONVERGED" and info["iters"] == 2
    _, info = gpu_cg(rp, c, v, b, rtol=1e-14, max_iter=0, cooperative=coop)
    assert info["status_name"] == "NOT_CONVERGED" and info["iters"] == 0
    # NaN in b
    bn = b.copy(); bn[4] = np.nan
    _, info = gpu_cg(rp, c, v, bn, cooperative=coop)
    assert info["status_name"] == "BREAKDOWN"
    # warm start from the exact solution
    xs = exact(rp, c, v, b)
    x, inf = sla.cg(csr(rp, c), to_dev(v), to_dev(b), x0=to_dev(xs), rtol=1e-10, cooperative=coop)
    assert inf.status == 0 and inf.iters <= 1
    # n = 1 and atol-only stopping
    x, info = gpu_cg(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]), np.array([2.0]),
                     cooperative=coop)
    assert info["status"] == 0 and abs(x[0] - 0.5) < 1e-15
    x, info = gpu_cg(rp, c, v, b, rtol=0.0, atol=1e-6, cooperative=coop)
    _, io = oracle.pcg(rp, c, v, b, rtol=0.0, atol=1e-6)
    assert info["status"] == 0 and abs(info["iters"] - io["iters"]) <= 1


def test_deterministic_and_graph_reuse():
    rp, c, v = I.diffusion3d_random(24, 5)
    n = 24 ** 3
    A = csr(rp, c)
    vt = to_dev(v)
    b1 = to_dev(I.rhs_uniform(n, 1))
    b2 = to_dev(I.rhs_uniform(n, 2))
    xa, ia = sla.cg(A, vt, b1)
    xb, ib = sla.cg(A, vt, b2)
    xc, ic = sla.cg(A, vt, b1)
    torch.cuda.synchronize()
    assert torch.equal(xa, xc) and ia.iters == ic.iters
    xo, _ = oracle.pcg(rp, c, v, b2.cpu().numpy(), rtol=1e-13)
    assert rel(xb.cpu().numpy(), xo) <= 1e-8


@pytest.mark.slow
def test_full_size_diffusion3d_256_true_residual():
    """The bench workload (3D 7-point variable coefficients, 256^3, rtol 1e-8),
    in the bench's launch configuration: the residual b - A x is recomputed
    by the oracle's SpMV, and sampled rows are checked one by one."""
    N = 256
    rp, c, v = I.diffusion3d_random(N, 1)
    n = N ** 3
    b = I.rhs_uniform(n, 11)
    x, info = gpu_cg(rp, c, v, b, rtol=1e-8)
    assert info["status"] == 0
    r = b - oracle.spmv(rp, c, v, x)
    true_rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert true_rel <= 2e-8
    assert abs(true_rel - info["true_rel_res"]) <= 1e-3 * true_rel


@pytest.mark.slow
@pytest.mark.parametrize("N", [128, 256, 464])
def test_full_size_diffusion3d_matches_stored_oracle_solution(N):
    """The 3D variable-coefficient configurations at full size against the
    oracle's own solution (rtol 1e-12, stored at 256 sampled indices by
    tests/golden/make_golden.py), element by element on the sample.

    Solved at rtol 1e-11: the solution error is the residual times up to the
    condition number, which grows as N^2 (at 64^3 the sampled error is 13x
    the rtol), so rtol 1e-10 would not certify 1e-8 at 256^3 and beyond; the
    bar stays 1e-8 and the tolerance is tightened instead.  128^3 runs both
    in the cooperative launch (its default) and as the per-phase graph;
    256^3 and 464^3 take the graph with the TMA SpMV pipeline, the bench's
    configuration.  The rtol 1e-8 solve must also take the oracle's
    iteration count to within 2 %."""
    g = stored_oracle("oracle_diffusion3d_%d.json" % N)
    rp, c, v = I.diffusion3d_random(N, 1)
    n = N ** 3
    b = I.rhs_uniform(n, 11)
    A = csr(rp, c)
    vt, bt = to_dev(v), to_dev(b)
    del v
    modes = [{}, {"cooperative": False}] if N == 128 else [{}]
    for kw in modes:
        x, info = sla.cg(A, vt, bt, rtol=1e-11, **kw)
        torch.cuda.synchronize()
        assert info.status == 0, (kw, info.as_dict())
        emax, enorm = sampled_errors(x.cpu().numpy(), g)
        assert emax <= 1e-8 and enorm <= 1e-8, (kw, emax, enorm)
        del x
    x8, i8 = sla.cg(A, vt, bt, rtol=1e-8)
    torch.cuda.synchronize()
    io = g["pcg_rtol_1e-8"]["iters"]
    assert i8.status == 0 and abs(i8.iters - io) <= max(2, io // 50), (i8.iters, io)
    assert i8.true_rel_res <= 2e-8


def test_host_loop_mode_reproduces_graph_mode():
    """Same kernels, same grids: the host-driven loop must give the same bits
    as the graph (the per-phase kernels; cooperative=False, since this size
    would otherwise run as one cooperative launch)."""
    rp, c, v = I.diffusion3d_random(20, 9)
    n = 8000
    A = csr(rp, c)
    vt = to_dev(v)
    b = to_dev(I.rhs_uniform(n, 3))
    xg, ig = sla.cg(A, vt, b, rtol=1e-10, cooperative=False)
    xh, ih = sla.cg(A, vt, b, rtol=1e-10, graph=False)
    torch.cuda.synchronize()
    assert torch.equal(xg, xh) and ig.iters == ih.iters and ig.status == ih.status == 0
    # bounded run (iteration cap) in host-loop mode
    _, ic = sla.cg(A, vt, b, rtol=1e-14, max_iter=20, graph=False)
    assert ic.iters == 20 and ic.status_name == "NOT_CONVERGED"
