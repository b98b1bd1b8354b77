"""The batched adjoint entry points (sla_adjoint_backward_batched_shared and
_list: Eq. 3 for every system of a batch, Sec. 3.1) called directly: each
system's lambda and -lambda_i x_j against the oracle's adjoint of that system
alone; bit for bit what the separate batched solve, values gather and
gradient pass give in the same launch shape; per-system statuses."""
import numpy as np
import scipy.sparse as sp
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu


def _weights(shape, seed):
    """A nonuniform dL/dx, so that no two systems share an adjoint right-hand side."""
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("method,precond", [("cg", "jacobi"), ("cg", "none"), ("bicgstab", "jacobi"),
                                            ("bicgstab", "none")])
def test_shared_pattern_matches_oracle_per_system(method, precond):
    B, N = 6, 20
    if method == "cg":
        rp, c, vals = I.batched_shared_2d(N, B, seed0=310, sigma=0.5)
    else:
        rp, c, vals = I.batched_convdiff_2d(N, B, seed0=330)
    n = N * N
    A = csr(rp, c)
    solve = oracle.pcg if method == "cg" else oracle.bicgstab
    xs = np.stack([solve(rp, c, vals[s], I.rhs_uniform(n, 40 + s), rtol=1e-13)[0] for s in range(B)])
    g = _weights((B, n), 7)
    gb, gv, info = sla.adjoint_backward_batched(A, to_dev(vals), to_dev(xs), to_dev(g), method=method,
                                                precond=precond, rtol=1e-12)
    torch.cuda.synchronize()
    assert (np.atleast_1d(info.status) == 0).all()
    assert gb.shape == (B, n) and gv.shape == (B, len(c))
    for s in range(B):
        ob, ov, io = oracle.adjoint_backward(rp, c, vals[s], xs[s], g[s], method=method, rtol=1e-13)
        assert io["status"] == 0
        for got, want in ((gb[s], ob), (gv[s], ov)):
            assert rel(got.cpu().numpy(), want) <= 1e-7, s
            assert elementwise_rel(got.cpu().numpy(), want) <= 1e-7, s


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_shared_pattern_bit_equal_to_separate_calls(method):
    """One call = the batched solve of A_s^T lambda = g (on the gathered
    values of A^T for BiCGStab) followed by the batched gradient pass, in the
    same launch shape: the same kernels, so the same bits."""
    B, N = 9, 24
    if method == "cg":
        rp, c, vals = I.batched_shared_2d(N, B, seed0=350, sigma=0.5)
    else:
        rp, c, vals = I.batched_convdiff_2d(N, B, seed0=370)
    A = csr(rp, c)
    v = to_dev(vals)
    x = to_dev(_weights((B, N * N), 3))
    g = to_dev(_weights((B, N * N), 4))
    cfgs = (0, 2, 3 | 16) if method == "cg" else (0, 1, 2 | 16)
    for cfg in cfgs:
        gb, gv, info = sla.adjoint_backward_batched(A, v, x, g, method=method, rtol=1e-11, config=cfg)
        if method == "cg":
            lam, i2 = sla.cg_batched(A, v, g, rtol=1e-11, config=cfg)
        else:
            rpT, cT, pT = sla.transpose_of(A)
            AT = sla.CSRMatrix(rpT, cT, check=False)
            lam, i2 = sla.bicgstab_batched(AT, sla.gather_values_batched(pT, v), g, rtol=1e-11, config=cfg)
        gv2 = sla.grad_values_batched_shared(A, lam, x)
        torch.cuda.synchronize()
        assert torch.equal(gb, lam) and torch.equal(gv, gv2), cfg
        assert np.array_equal(np.atleast_1d(info.iters), np.atleast_1d(i2.iters)), cfg
        assert (np.atleast_1d(info.status) == 0).all()


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_list_matches_oracle_and_separate_calls(method):
    """Distinct patterns, with and without the block teams for the large
    systems: each system against the oracle's adjoint, and bit for bit the
    separate list solve, values gather and gradient pass."""
    if method == "cg":
        mats = I.fem_list(6, seed0=2300, n_lo=200, n_hi=40000)
    else:
        mats = I.convdiff_list(6, seed0=640, n_lo=200, n_hi=40000)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([m[2] for m in mats])
    solve = oracle.pcg if method == "cg" else oracle.bicgstab
    xs = [solve(rp, c, vs, I.rhs_uniform(len(rp) - 1, 90 + s), rtol=1e-13)[0] for s, (rp, c, vs) in enumerate(mats)]
    g = _weights(P.total_rows, 11)
    v, x, gt = to_dev(vals), to_dev(np.concatenate(xs)), to_dev(g)
    no_teams = 32 if method == "cg" else 1 | 32
    for cfg in (0, no_teams):
        gb, gv, info = sla.adjoint_backward_batched_list(P, v, x, gt, method=method, rtol=1e-12, config=cfg)
        if method == "cg":
            lam, _ = sla.cg_batched_list(P, v, gt, rtol=1e-12, config=cfg)
        else:
            PT, permT = P.transpose()
            lam, _ = sla.bicgstab_batched_list(PT, sla.gather_values(permT, v), gt, rtol=1e-12, config=cfg)
        gv2 = sla.grad_values_batched_list(P, lam, x)
        torch.cuda.synchronize()
        assert torch.equal(gb, lam) and torch.equal(gv, gv2), cfg
        assert (np.atleast_1d(info.status) == 0).all(), cfg
        for s, (rp, c, vs) in enumerate(mats):
            r0, r1 = P.n_off_h[s], P.n_off_h[s + 1]
            e0, e1 = P.nnz_off_h[s], P.nnz_off_h[s + 1]
            ob, ov, io = oracle.adjoint_backward(rp, c, vs, xs[s], g[r0:r1], method=method, rtol=1e-13)
            assert io["status"] == 0
            for got, want in ((gb[r0:r1], ob), (gv[e0:e1], ov)):
                assert rel(got.cpu().numpy(), want) <= 1e-7, (cfg, s)
                assert elementwise_rel(got.cpu().numpy(), want) <= 1e-7, (cfg, s)


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_per_system_statuses(method):
    """A zero dL/dx gives lambda = 0 and a zero gradient in 0 iterations; an
    iteration cap gives NOT_CONVERGED in that system's record only (the
    records are per system, the others converge)."""
    B, N = 4, 16
    if method == "cg":
        rp, c, vals = I.batched_shared_2d(N, B, seed0=390, sigma=0.5)
    else:
        rp, c, vals = I.batched_convdiff_2d(N, B, seed0=410)
    A = csr(rp, c)
    g = _weights((B, N * N), 5)
    g[1] = 0.0
    x = to_dev(_weights((B, N * N), 6))
    gb, gv, info = sla.adjoint_backward_batched(A, to_dev(vals), x, to_dev(g), method=method, rtol=1e-10)
    torch.cuda.synchronize()
    st, its = np.atleast_1d(info.status), np.atleast_1d(info.iters)
    assert (st == 0).all() and its[1] == 0 and its[0] > 0
    assert not gb[1].any() and not gv[1].any()
    _, _, capped = sla.adjoint_backward_batched(A, to_dev(vals), x, to_dev(g), method=method, rtol=1e-15,
                                                max_iter=2, max_restarts=0)
    torch.cuda.synchronize()
    cs = np.atleast_1d(capped.status)
    assert cs[1] == 0 and all(sla.L.STATUS_NAMES[int(cs[s])] == "NOT_CONVERGED" for s in (0, 2, 3))


def _adjoint_residuals_ok(rp, c, v, lam, g, method, tol):
    """||A^T lambda - g|| <= tol ||g|| with the product taken on the CPU."""
    A = sp.csr_matrix((v, c, rp))
    At = A if method == "cg" else A.T.tocsr()
    return np.linalg.norm(At @ lam - g) <= tol * np.linalg.norm(g)


def _vs_oracle(rp, c, v, x, g, gb, gv, method):
    """One system's adjoint against the oracle's at rtol 1e-12 (the smooth
    dL/dx = 2x leaves some FEM systems short of 1e-13 in FP64)."""
    ob, ov, io = oracle.adjoint_backward(rp, c, v, x, g, method=method, rtol=1e-12)
    assert io["status"] == 0, io
    for got, want in ((gb, ob), (gv, ov)):
        assert rel(got, want) <= 1e-7
        assert elementwise_rel(got, want) <= 1e-7


@pytest.mark.slow
@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_full_size_shared_1024_systems_64(method):
    """The benchmark's shared-pattern batches (1024 systems on the 64 x 64
    five-point pattern: diffusion for CG, upwind convection-diffusion for
    BiCGStab, seeds 1000 + s) with L = sum x^2, adjoint rtol 1e-10: every
    system's adjoint residual on the CPU, 16 sampled systems against the
    oracle's adjoint element by element."""
    B, N = 1024, 64
    if method == "cg":
        rp, c, vals = I.batched_shared_2d(N, B, seed0=1000, sigma=0.5)
    else:
        rp, c, vals = I.batched_convdiff_2d(N, B, seed0=1000)
    A = csr(rp, c)
    vt = to_dev(vals)
    b = I.rhs_uniform(N * N, 7, batch=B)
    solve = sla.cg_batched if method == "cg" else sla.bicgstab_batched
    x, info = solve(A, vt, to_dev(b), rtol=1e-10)
    gb, gv, ainfo = sla.adjoint_backward_batched(A, vt, x, 2 * x, method=method, rtol=1e-10)
    torch.cuda.synchronize()
    assert (np.atleast_1d(info.status) == 0).all() and (np.atleast_1d(ainfo.status) == 0).all()
    xh, gbh, gvh = x.cpu().numpy(), gb.cpu().numpy(), gv.cpu().numpy()
    for s in range(B):
        assert _adjoint_residuals_ok(rp, c, vals[s], gbh[s], 2 * xh[s], method, 2e-10), s
    idx = sorted(set(np.random.default_rng(12).choice(B, 14, replace=False).tolist()) | {0, B - 1})
    for s in idx:
        _vs_oracle(rp, c, vals[s], xh[s], 2 * xh[s], gbh[s], gvh[s], method)


@pytest.mark.slow
@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_full_size_list_512(method):
    """The benchmark's distinct-pattern batches (512 FEM Laplacians, seeds
    2000 + s, for CG; 512 convection-diffusion rectangles, seeds 5000 + s,
    for BiCGStab; n log-uniform in [1e3, 5e4], the large systems on block
    teams) with L = sum x^2, adjoint rtol 1e-10: every adjoint residual on
    the CPU, 16 systems (the four largest among them) against the oracle's
    adjoint element by element."""
    if method == "cg":
        mats, seed_b = I.fem_list(512, seed0=2000), 3000
    else:
        mats, seed_b = I.convdiff_list(512, seed0=5000), 6000
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vt = to_dev(np.concatenate([v for _, _, v in mats]))
    bt = to_dev(np.concatenate([I.rhs_uniform(len(rp) - 1, seed_b + s) for s, (rp, _, _) in enumerate(mats)]))
    solve = sla.cg_batched_list if method == "cg" else sla.bicgstab_batched_list
    x, info = solve(P, vt, bt, rtol=1e-10)
    gb, gv, ainfo = sla.adjoint_backward_batched_list(P, vt, x, 2 * x, method=method, rtol=1e-10)
    torch.cuda.synchronize()
    assert (np.atleast_1d(info.status) == 0).all() and (np.atleast_1d(ainfo.status) == 0).all()
    xh, gbh, gvh = x.cpu().numpy(), gb.cpu().numpy(), gv.cpu().numpy()
    part = lambda a, off, s: a[off[s]:off[s + 1]]
    for s, (rp, c, v) in enumerate(mats):
        xs = part(xh, P.n_off_h, s)
        assert _adjoint_residuals_ok(rp, c, v, part(gbh, P.n_off_h, s), 2 * xs, method, 2e-10), s
    sizes = np.array([len(m[0]) for m in mats])
    idx = set(np.argsort(sizes)[-4:].tolist()) | set(np.random.default_rng(13).choice(len(mats), 12, replace=False).tolist())
    for s in sorted(idx):
        rp, c, v = mats[s]
        xs = part(xh, P.n_off_h, s)
        _vs_oracle(rp, c, v, xs, 2 * xs, part(gbh, P.n_off_h, s), part(gvh, P.nnz_off_h, s), method)
