"""Batched BiCGStab (one persistent launch; the nonsymmetric members of the
paper's batched SparseTensor and SparseTensorList, Sec. 3.1) against the
oracle's BiCGStab solved one system at a time; per-system statuses; kernel
variants; CUDA graph capture; the list transpose bit for bit against the
oracle's; and the differentiable batches (Eq. 3 per system) against the
oracle's adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu


# BiCGStab's iteration count is sensitive to rounding: on the 40 systems of
# the shared-pattern test, the oracle's own count moved by up to 9 % (88 ->
# 96) when b was perturbed by 1e-15 relative noise.  The GPU sums in another
# order, so its count is held to the oracle's within that spread (12 %, at
# least 3); the solution itself is held to 1e-8 element by element.
ITERS_TOL = 0.12


def _check_systems(rps, cs, vals, bs, xs, info, rtol, idx=None, iters_tol=ITERS_TOL):
    """Each system against the oracle: its solution x* (rtol 1e-13) element
    by element and in norm to 1e-8, its status, and its iteration count at
    the same rtol to within the rounding spread (ITERS_TOL)."""
    its = np.atleast_1d(info.iters)
    st = np.atleast_1d(info.status)
    idx = range(len(bs)) if idx is None else idx
    for s in idx:
        xo, io = oracle.bicgstab(rps[s], cs[s], vals[s], bs[s], rtol=1e-13)
        assert io["status"] == 0 and st[s] == 0, (s, st[s])
        assert elementwise_rel(xs[s], xo) <= 1e-8, s
        assert rel(xs[s], xo) <= 1e-8, s
        _, ir = oracle.bicgstab(rps[s], cs[s], vals[s], bs[s], rtol=rtol)
        assert abs(int(its[s]) - ir["iters"]) <= max(3, int(iters_tol * ir["iters"])), (s, its[s], ir["iters"])


def test_shared_pattern_matches_oracle_per_system():
    B, N = 40, 32
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=100)
    b = I.rhs_uniform(N * N, 5, batch=B)
    x, info = sla.bicgstab_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-10)
    torch.cuda.synchronize()
    _check_systems([rp] * B, [c] * B, vals, b, x.cpu().numpy(), info, 1e-10)
    assert len(set(np.atleast_1d(info.iters).tolist())) > 1   # each CTA stopped on its own
    tr = np.atleast_1d(info.true_rel_res)
    assert (tr <= 2e-10).all()


def test_unpreconditioned_and_warm_start():
    B, N = 6, 20
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=300)
    b = I.rhs_uniform(N * N, 6, batch=B)
    A = csr(rp, c)
    x, info = sla.bicgstab_batched(A, to_dev(vals), to_dev(b), rtol=1e-10, precond="none")
    torch.cuda.synchronize()
    for s in range(B):
        xo, io = oracle.bicgstab(rp, c, vals[s], b[s], rtol=1e-13, precond="none")
        assert np.atleast_1d(info.status)[s] == 0 and rel(x[s].cpu().numpy(), xo) <= 1e-8
    # warm start at the solution: converged with no iteration (recursive residual)
    xs = torch.stack([torch.from_numpy(oracle.bicgstab(rp, c, vals[s], b[s], rtol=1e-14)[0])
                      for s in range(B)]).cuda()
    x2, i2 = sla.bicgstab_batched(A, to_dev(vals), to_dev(b), rtol=1e-8, x0=xs)
    torch.cuda.synchronize()
    assert (np.atleast_1d(i2.iters) == 0).all() and (np.atleast_1d(i2.status) == 0).all()


def test_mixed_statuses_do_not_leak_between_systems():
    B, N = 6, 20
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=17)
    b = I.rhs_uniform(N * N, 1, batch=B)
    b[1] = 0.0                                       # zero right-hand side
    diag = np.nonzero(c == np.repeat(np.arange(N * N), np.diff(rp)))[0]
    vals[3, diag[10]] = 0.0                          # zero diagonal: invalid with Jacobi
    x, info = sla.bicgstab_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-10, max_iter=400,
                                   config=1)
    torch.cuda.synchronize()
    st = np.atleast_1d(info.status)
    its = np.atleast_1d(info.iters)
    assert st[1] == 0 and its[1] == 0 and not x[1].any()
    _, io = oracle.bicgstab(rp, c, vals[3], b[3], rtol=1e-10)
    assert st[3] == io["status"] == -1 and its[3] == 0 and np.isnan(np.atleast_1d(info.rel_res)[3])
    # an iteration cap on the others reproduces the oracle's NOT_CONVERGED
    xc, ic = sla.bicgstab_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-14, max_iter=5,
                                  max_restarts=0)
    torch.cuda.synchronize()
    for s in (0, 2, 4, 5):
        xo, io = oracle.bicgstab(rp, c, vals[s], b[s], rtol=1e-13)
        assert st[s] == 0 and rel(x[s].cpu().numpy(), xo) <= 1e-8
        _, io5 = oracle.bicgstab(rp, c, vals[s], b[s], rtol=1e-14, max_iter=5, max_restarts=0)
        assert np.atleast_1d(ic.status)[s] == io5["status"] == 1 and np.atleast_1d(ic.iters)[s] == 5


def test_all_kernel_variants_agree():
    B, N = 16, 24
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=3)
    b = to_dev(I.rhs_uniform(N * N, 2, batch=B))
    A = csr(rp, c)
    v = to_dev(vals)
    res = {}
    for cfg in sla.BICG_BATCH_CONFIGS:
        x, info = sla.bicgstab_batched(A, v, b, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        assert (np.atleast_1d(info.status) == 0).all()
        res[cfg] = (x.clone(), np.atleast_1d(info.iters).copy())
    for code in (1, 2, 3):
        # same block size: vectors on chip or in the workspace give the same bits
        assert torch.equal(res[code][0], res[code | 16][0])
        assert np.array_equal(res[code][1], res[code | 16][1])
        assert rel(res[code][0].cpu().numpy(), res[1][0].cpu().numpy()) <= 1e-9
    tuned = sla.bicgstab_batched(A, v, b, rtol=1e-10, config="tune")[0]
    assert any(k[0] == "bicg_shared" for k in sla.tuned_configs())
    assert rel(tuned.cpu().numpy(), res[1][0].cpu().numpy()) <= 1e-9
    with pytest.raises(sla.L.SlaError):
        sla.bicgstab_batched(A, v, b, rtol=1e-10, config=32)


def test_distinct_patterns_match_oracle():
    mats = I.convdiff_list(30, seed0=400, n_lo=100, n_hi=6000)
    mats.append(I.convdiff2d_random(90, 80, 9))      # 7200 rows: vectors partly off chip
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 50 + s) for s, (rp, _, _) in enumerate(mats)]
    x, info = sla.bicgstab_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-10)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    xs = [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
    _check_systems([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs, info, 1e-10)
    # one CTA per system, every vector in the workspace or on chip: the same bits
    x16, _ = sla.bicgstab_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-10, config=2 | 16 | 32)
    x2, _ = sla.bicgstab_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-10, config=2 | 32)
    torch.cuda.synchronize()
    assert torch.equal(x16, x2)


def test_list_block_teams_match_oracle():
    """The large systems of a list solved by teams of blocks of one
    cooperative launch (sums of the team's blocks in a fixed order), the
    small ones by single blocks of the same launch: every team size (2, 3,
    4, 6 blocks) and entry threshold against the oracle per system, and
    against one CTA per system."""
    mats = I.convdiff_list(24, seed0=700, n_lo=100, n_hi=3000)
    mats += [I.convdiff2d_random(200, 160, 11),   # 32000 rows, ~159 k entries: a team at every threshold
             I.convdiff2d_random(150, 120, 12),   # 18000 rows, ~90 k entries
             I.convdiff2d_random(100, 75, 13),    # 7500 rows, ~37 k entries
             I.convdiff2d_random(73, 71, 14)]     # 5183 rows (not a multiple of any team's threads)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = to_dev(np.concatenate([v for _, _, v in mats]))
    bs = [I.rhs_uniform(len(rp) - 1, 80 + s) for s, (rp, _, _) in enumerate(mats)]
    bt = to_dev(np.concatenate(bs))
    xo = [oracle.bicgstab(rp, c, v, b, rtol=1e-13)[0] for (rp, c, v), b in zip(mats, bs)]
    xc, ic = sla.bicgstab_batched_list(P, vals, bt, rtol=1e-10, config=3 | 32)
    torch.cuda.synchronize()
    xc = xc.cpu().numpy()
    for cfg in [(t << 8) | (m << 10) for t in range(4) for m in range(4)]:
        x, info = sla.bicgstab_batched_list(P, vals, bt, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        assert (np.atleast_1d(info.status) == 0).all(), (cfg, info.status)
        xh = x.cpu().numpy()
        for s in range(len(mats)):
            xs = xh[P.n_off_h[s]:P.n_off_h[s + 1]]
            assert elementwise_rel(xs, xo[s]) <= 1e-8, (cfg, s)
        # both meet rtol 1e-10 on their own; their solutions agree to the
        # same 1e-8 as each does with the oracle's x*
        assert rel(xh, xc) <= 1e-8, cfg
        if cfg == 0:
            _check_systems([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs,
                           [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))], info, 1e-10)
    shape = sla.bicg_list_shape(2 << 8 | 1 << 10)
    assert shape["block_teams"] and shape["team_blocks"] == 4 and shape["team_min_nnz"] == 16384
    assert not sla.bicg_list_shape(3 | 32)["block_teams"]


def test_graph_capture_and_replay():
    B, N = 8, 16
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=11)
    A = csr(rp, c)
    v = to_dev(vals)
    b_static = to_dev(I.rhs_uniform(N * N, 1, batch=B))
    x_static = torch.empty_like(b_static)
    sla.bicgstab_batched(A, v, b_static, rtol=1e-10, out=x_static)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sla.bicgstab_batched(A, v, b_static, rtol=1e-10, out=x_static)
    torch.cuda.current_stream().wait_stream(s)
    b_new = to_dev(I.rhs_uniform(N * N, 2, batch=B))
    b_static.copy_(b_new)
    g.replay()
    torch.cuda.synchronize()
    x_ref, _ = sla.bicgstab_batched(A, v, b_new, rtol=1e-10)
    torch.cuda.synchronize()
    assert torch.equal(x_static, x_ref)


def test_list_transpose_bit_exact_against_oracle():
    mats = I.convdiff_list(12, seed0=500, n_lo=50, n_hi=3000)
    mats.insert(3, (np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)))   # an empty system
    mats.append(I.fem_p1_laplacian(12, 3))
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    PT, permT = P.transpose()
    torch.cuda.synchronize()
    rpT = PT.rowptr.cpu().numpy()
    cT = PT.col.cpu().numpy()
    pT = permT.cpu().numpy()
    for s, (rp, c, _) in enumerate(mats):
        n0, e0, e1 = P.n_off_h[s], P.nnz_off_h[s], P.nnz_off_h[s + 1]
        orp, oc, op = oracle.transpose(rp, c)
        assert np.array_equal(rpT[n0 + s:P.n_off_h[s + 1] + s + 1], orp), s
        assert np.array_equal(cT[e0:e1], oc), s
        assert np.array_equal(pT[e0:e1] - e0, op), s


def test_batched_bicgstab_adjoint_matches_oracle():
    """solve_batched(method="bicgstab"): Eq. 3 per system through the shared
    CSR of A^T with every system's values gathered."""
    B, N = 5, 16
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=21)
    A = csr(rp, c)
    v = to_dev(vals).requires_grad_(True)
    b = to_dev(I.rhs_uniform(N * N, 3, batch=B)).requires_grad_(True)
    x = sla.solve_batched(A, v, b, method="bicgstab", rtol=1e-12)
    (x * x).sum().backward()
    for s in range(B):
        xo, _ = oracle.bicgstab(rp, c, vals[s], b[s].detach().cpu().numpy(), rtol=1e-13)
        gb, gv, io = oracle.adjoint_backward(rp, c, vals[s], xo, 2 * xo, method="bicgstab", rtol=1e-13)
        assert io["status"] == 0
        assert rel(x[s].detach().cpu().numpy(), xo) <= 1e-8
        for got, want in ((b.grad[s], gb), (v.grad[s], gv)):
            assert rel(got.cpu().numpy(), want) <= 1e-6
            assert elementwise_rel(got.cpu().numpy(), want) <= 1e-6


@pytest.mark.parametrize("method", ["cg", "bicgstab"])
def test_list_solve_gradients_per_system(method):
    """solve_batched_list: each system of a list gets its own Eq. 3 gradient
    (the paper's SparseTensorList with isolated per-element graphs)."""
    if method == "cg":
        mats = I.fem_list(7, seed0=2100, n_lo=200, n_hi=3000)
    else:
        mats = I.convdiff_list(7, seed0=600, n_lo=200, n_hi=3000)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([m[2] for m in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 70 + s) for s, (rp, _, _) in enumerate(mats)]
    v = to_dev(vals).requires_grad_(True)
    b = to_dev(np.concatenate(bs)).requires_grad_(True)
    x = sla.solve_batched_list(P, v, b, method=method, rtol=1e-12)
    w = to_dev(np.random.default_rng(1).standard_normal(P.total_rows))
    (w * x * x).sum().backward()   # a weighted loss, so every system's g differs
    solve = oracle.pcg if method == "cg" else oracle.bicgstab
    for s, (rp, c, vs) in enumerate(mats):
        r0, r1 = P.n_off_h[s], P.n_off_h[s + 1]
        e0, e1 = P.nnz_off_h[s], P.nnz_off_h[s + 1]
        xo, _ = solve(rp, c, vs, bs[s], rtol=1e-13)
        g = 2 * w[r0:r1].cpu().numpy() * xo
        gb, gv, io = oracle.adjoint_backward(rp, c, vs, xo, g, method=method, rtol=1e-13)
        assert io["status"] == 0
        assert rel(x[r0:r1].detach().cpu().numpy(), xo) <= 1e-8
        for got, want in ((b.grad[r0:r1], gb), (v.grad[e0:e1], gv)):
            assert rel(got.cpu().numpy(), want) <= 1e-6, s
            assert elementwise_rel(got.cpu().numpy(), want) <= 1e-6, s


@pytest.mark.slow
def test_full_size_shared_1024_systems_64():
    """1024 nonsymmetric systems on the 64 x 64 five-point pattern (faces
    exp(N(0, 0.5^2)), cell Peclet up to 10 in a random direction), rtol
    1e-8: every system's true residual by the oracle's SpMV; 16 sampled
    systems at rtol 1e-10 against the oracle's x*."""
    B, N = 1024, 64
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=1000)
    b = I.rhs_uniform(N * N, 7, batch=B)
    A = csr(rp, c)
    x, info = sla.bicgstab_batched(A, to_dev(vals), to_dev(b), rtol=1e-8)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    assert (np.atleast_1d(info.status) == 0).all()
    for s in range(B):
        r = b[s] - oracle.spmv(rp, c, vals[s], xh[s])
        assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b[s])
    x10, i10 = sla.bicgstab_batched(A, to_dev(vals), to_dev(b), rtol=1e-10)
    torch.cuda.synchronize()
    idx = sorted(set(np.random.default_rng(8).choice(B, 14, replace=False).tolist()) | {0, B - 1})
    _check_systems([rp] * B, [c] * B, vals, b, x10.cpu().numpy(), i10, 1e-10, idx=idx)


@pytest.mark.slow
def test_full_size_convdiff_list_512():
    """512 nonsymmetric systems with distinct patterns, n log-uniform in
    [1e3, 5e4], rtol 1e-8 in one launch: every residual by the oracle's
    SpMV; 16 systems (the four largest among them) at rtol 1e-10 against the
    oracle's x*."""
    mats = I.convdiff_list(512, seed0=5000)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 6000 + s) for s, (rp, _, _) in enumerate(mats)]
    bt = to_dev(np.concatenate(bs))
    x, info = sla.bicgstab_batched_list(P, to_dev(vals), bt, rtol=1e-8)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    assert (np.atleast_1d(info.status) == 0).all()
    for s, (rp, c, v) in enumerate(mats):
        xs = xh[P.n_off_h[s]:P.n_off_h[s + 1]]
        assert np.linalg.norm(bs[s] - oracle.spmv(rp, c, v, xs)) <= 2e-8 * np.linalg.norm(bs[s])
    x10, i10 = sla.bicgstab_batched_list(P, to_dev(vals), bt, rtol=1e-10)
    torch.cuda.synchronize()
    xh10 = x10.cpu().numpy()
    xs10 = [xh10[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
    sizes = np.array([len(m[0]) for m in mats])
    idx = set(np.argsort(sizes)[-4:].tolist()) | set(np.random.default_rng(9).choice(len(mats), 12, replace=False).tolist())
    _check_systems([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs10, i10, 1e-10,
                   idx=sorted(idx))
