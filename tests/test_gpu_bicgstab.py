"""BiCGStab parity: GPU solutions of nonsymmetric systems against the
oracle's BiCGStab and dense/sparse LU on the same seeded inputs."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, rel, to_dev

pytestmark = pytest.mark.gpu


def gpu_bicg(rp, c, v, b, **kw):
    A = csr(rp, c)
    x, info = sla.bicgstab(A, to_dev(v), to_dev(b), **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info.as_dict()


def exact(rp, c, v, b):
    return spl.spsolve(sp.csr_matrix((v, c, rp)).tocsc(), b)


@pytest.mark.parametrize("N,pe", [(16, 10.0), (24, 1.0), (33, 10.0)])
def test_convdiff_matches_oracle_and_lu(N, pe):
    rp, c, v = I.convdiff3d(N, pe)
    b = I.rhs_uniform(N ** 3, N)
    x, info = gpu_bicg(rp, c, v, b, rtol=1e-10)
    xo, io = oracle.bicgstab(rp, c, v, b, rtol=1e-10)
    assert info["status"] == 0 and io["status"] == 0
    xs = exact(rp, c, v, b)
    assert rel(x, xs) <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= max(2, io["iters"] // 20)
    assert info["true_rel_res"] <= 2e-10


def test_spd_system_agrees_with_cg():
    rp, c, v = I.diffusion3d_random(20, 3)
    b = I.rhs_uniform(8000, 1)
    x, info = gpu_bicg(rp, c, v, b, rtol=1e-11)
    A = csr(rp, c)
    xc, ic = sla.cg(A, to_dev(v), to_dev(b), rtol=1e-11)
    assert info["status"] == 0 and ic.status == 0
    assert rel(x, xc.cpu().numpy()) <= 1e-8


def test_bicgstab_edge_cases_match_oracle():
    rp, c, v = I.convdiff3d(5)
    n = 125
    x, info = gpu_bicg(rp, c, v, np.zeros(n))
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    v0 = v.copy()
    v0[(c == 0) & (np.arange(len(c)) < rp[1])] = 0.0
    _, info = gpu_bicg(rp, c, v0, np.ones(n))
    _, io = oracle.bicgstab(rp, c, v0, np.ones(n))
    assert info["status"] == io["status"] == -1
    b = I.rhs_uniform(n, 1)
    _, info = gpu_bicg(rp, c, v, b, rtol=1e-15, max_iter=1)
    _, io = oracle.bicgstab(rp, c, v, b, rtol=1e-15, max_iter=1)
    assert info["status_name"] == io["status_name"] == "NOT_CONVERGED"
    assert info["iters"] == io["iters"] == 1
    bn = b.copy(); bn[0] = np.inf
    _, info = gpu_bicg(rp, c, v, bn)
    assert info["status_name"] == "BREAKDOWN"
    # unpreconditioned, and a warm start at the solution
    x, info = gpu_bicg(rp, c, v, b, rtol=1e-11, precond="none")
    xo, io = oracle.bicgstab(rp, c, v, b, rtol=1e-11, precond="none")
    assert info["status"] == 0 and rel(x, exact(rp, c, v, b)) <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 2
    xs = exact(rp, c, v, b)
    x, inf = sla.bicgstab(csr(rp, c), to_dev(v), to_dev(b), x0=to_dev(xs), rtol=1e-10)
    assert inf.status == 0 and inf.iters <= 1


def test_half_step_exit_and_host_loop():
    # an exactly diagonal system converges at the half step of iteration 1
    n = 1000
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    v = np.linspace(1.0, 3.0, n)
    b = I.rhs_uniform(n, 2)
    x, info = gpu_bicg(rp, c, v, b, rtol=1e-12)
    _, io = oracle.bicgstab(rp, c, v, b, rtol=1e-12)
    assert info["status"] == 0 and info["iters"] == io["iters"] == 1
    assert np.allclose(x, b / v, rtol=1e-14, atol=0)
    rp, c, v = I.convdiff3d(12, 5.0)
    b = to_dev(I.rhs_uniform(12 ** 3, 7))
    A = csr(rp, c)
    vt = to_dev(v)
    xg, ig = sla.bicgstab(A, vt, b, rtol=1e-10)
    xh, ih = sla.bicgstab(A, vt, b, rtol=1e-10, graph=False)
    torch.cuda.synchronize()
    assert torch.equal(xg, xh) and ig.iters == ih.iters


@pytest.mark.slow
def test_convdiff_128_full_size_true_residual():
    """3D convection-diffusion 128^3, Pe 10 (the nonsymmetric configuration),
    rtol 1e-8: residual recomputed by the oracle's SpMV."""
    N = 128
    rp, c, v = I.convdiff3d(N, 10.0)
    b = I.rhs_uniform(N ** 3, 5)
    x, info = gpu_bicg(rp, c, v, b, rtol=1e-8)
    assert info["status"] == 0
    r = b - oracle.spmv(rp, c, v, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 2e-8
