"""G G^T-preconditioned CG against the oracle's PCG with the same G."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, rel, to_dev

pytestmark = pytest.mark.gpu


def pattern_optimal_factor(rp, c, v):
    """Lower-triangular G on the pattern of tril(A) with G G^T ~ A^{-1}:
    column i solves A[P, P] y = e_i on P = {j >= i : A_ji != 0} and is scaled
    by 1/sqrt(y_i) (a factored sparse approximate inverse)."""
    n = len(rp) - 1
    A = sp.csr_matrix((v, c, rp), shape=(n, n))
    rows, cols, vals = [], [], []
    for i in range(n):
        js = c[rp[i]:rp[i + 1]]
        P = np.sort(js[js >= i])
        y = np.linalg.solve(A[P][:, P].toarray(), np.eye(len(P))[0])
        rows += list(P); cols += [i] * len(P); vals += list(y / np.sqrt(y[0]))
    G = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    G.sort_indices()
    return G.indptr.astype(np.int32), G.indices.astype(np.int32), G.data


def as_applied(G):
    """The factor as the solver applies it: values rounded to FP32."""
    return G[0], G[1], G[2].astype(np.float32).astype(np.float64)


def test_diagonal_factor_reproduces_jacobi():
    rp, c, v = I.diffusion2d_random(48, 2)
    n = len(rp) - 1
    d = v[c == np.repeat(np.arange(n), np.diff(rp))]
    Grp, Gc, Gv = np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), 1.0 / np.sqrt(d)
    b = to_dev(I.rhs_uniform(n, 1))
    A = csr(rp, c)
    x1, i1 = sla.cg_ggt(A, to_dev(v), csr(Grp, Gc), to_dev(Gv), b, rtol=1e-10)
    x2, i2 = sla.cg(A, to_dev(v), b, rtol=1e-10)
    torch.cuda.synchronize()
    assert i1.status == i2.status == 0 and abs(i1.iters - i2.iters) <= 2
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("mat", ["var2d", "var3d"])
def test_pattern_optimal_factor_matches_oracle(mat):
    rp, c, v = I.diffusion2d_random(40, 5, 1.5) if mat == "var2d" else I.diffusion3d_random(14, 6)
    n = len(rp) - 1
    G = pattern_optimal_factor(rp, c, v)
    b = I.rhs_uniform(n, 3)
    x, info = sla.cg_ggt(csr(rp, c), to_dev(v), csr(G[0], G[1]), to_dev(G[2]), to_dev(b), rtol=1e-10)
    torch.cuda.synchronize()
    xo, io = oracle.pcg(rp, c, v, b, rtol=1e-10, precond="ggt", G=as_applied(G))
    _, ij = oracle.pcg(rp, c, v, b, rtol=1e-10)
    assert info.status == io["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-8
    assert abs(info.iters - io["iters"]) <= 2
    assert io["iters"] < ij["iters"]            # the factor helps
    assert info.true_rel_res <= 2e-10


def test_ggt_edge_cases_and_host_loop():
    rp, c, v = I.diffusion2d_random(20, 8)
    n = len(rp) - 1
    G = pattern_optimal_factor(rp, c, v)
    A = csr(rp, c)
    Gm = csr(G[0], G[1])
    gv = to_dev(G[2])
    x, info = sla.cg_ggt(A, to_dev(v), Gm, gv, to_dev(np.zeros(n)))
    assert info.status == 0 and info.iters == 0 and not x.cpu().numpy().any()
    b = to_dev(I.rhs_uniform(n, 4))
    # graph and host loop run the same per-phase kernels: same bits
    xg, ig = sla.cg_ggt(A, to_dev(v), Gm, gv, b, rtol=1e-11, cooperative=False)
    xh, ih = sla.cg_ggt(A, to_dev(v), Gm, gv, b, rtol=1e-11, graph=False)
    torch.cuda.synchronize()
    assert torch.equal(xg, xh) and ig.iters == ih.iters
    # the cooperative launch: same method, other summation grid
    xc, ic = sla.cg_ggt(A, to_dev(v), Gm, gv, b, rtol=1e-11)
    xc2, ic2 = sla.cg_ggt(A, to_dev(v), Gm, gv, b, rtol=1e-11)
    torch.cuda.synchronize()
    assert torch.equal(xc, xc2) and ic.iters == ic2.iters
    assert ic.status == 0 and abs(ic.iters - ig.iters) <= 2
    assert float((xc - xg).norm() / xg.norm()) <= 1e-8
    for coop in (True, False):
        _, ic = sla.cg_ggt(A, to_dev(v), Gm, gv, b, rtol=1e-15, max_iter=3, cooperative=coop)
        assert ic.status_name == "NOT_CONVERGED" and ic.iters == 3
