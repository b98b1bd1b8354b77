"""Batched Jacobi-PCG (one persistent launch) against the oracle solved one
system at a time; per-system statuses; kernel variants; autotuner; CUDA
graph capture; batched adjoint gradients."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu


def _per_system_check(rp, c, vals, bs, x, info, rtol, iters_tol=2, idx=None):
    its = np.atleast_1d(info.iters)
    st = np.atleast_1d(info.status)
    idx = range(len(bs)) if idx is None else idx
    for s in idx:
        xo, io = oracle.pcg(rp[s], c[s], vals[s], bs[s], rtol=rtol)
        assert st[s] == io["status"] == 0, s
        assert rel(x[s], xo) <= 1e-8, s
        assert abs(int(its[s]) - io["iters"]) <= iters_tol, (s, its[s], io["iters"])


def _vs_oracle_xstar(rps, cs, vals, bs, xs, idx):
    """Sampled systems of a full-size batch solved at rtol 1e-10 against the
    oracle's solution at rtol 1e-13, element by element (max-norm relative
    to max |x*|) and in norm, both to 1e-8."""
    for s in idx:
        xo, io = oracle.pcg(rps[s], cs[s], vals[s], bs[s], rtol=1e-13)
        assert io["status"] == 0, s
        assert elementwise_rel(xs[s], xo) <= 1e-8, s
        assert rel(xs[s], xo) <= 1e-8, s


def test_shared_pattern_matches_oracle_per_system():
    B, N = 48, 32
    rp, c, vals = I.batched_shared_2d(N, B, seed0=1000, sigma=0.5)
    b = I.rhs_uniform(N * N, 5, batch=B)
    A = csr(rp, c)
    x, info = sla.cg_batched(A, to_dev(vals), to_dev(b), rtol=1e-10)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    _per_system_check([rp] * B, [c] * B, vals, b, xh, info, 1e-10)
    # systems converge after different iteration counts: each CTA stopped on its own
    assert len(set(np.atleast_1d(info.iters).tolist())) > 1


def test_mixed_statuses_do_not_leak_between_systems():
    B, N = 6, 20
    rp, c, vals = I.batched_shared_2d(N, B, seed0=7, sigma=0.5)
    b = I.rhs_uniform(N * N, 1, batch=B)
    b[1] = 0.0                                       # zero right-hand side
    diag = np.nonzero(c == np.repeat(np.arange(N * N), np.diff(rp)))[0]
    vals[3, diag[10]] = -1.0                         # non-positive diagonal
    x, info = sla.cg_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-10, max_iter=400)
    torch.cuda.synchronize()
    st = np.atleast_1d(info.status)
    its = np.atleast_1d(info.iters)
    assert st[1] == 0 and its[1] == 0 and not x[1].any()
    assert sla.L.STATUS_NAMES[int(st[3])] == "NOT_SPD"
    for s in (0, 2, 4, 5):
        xo, io = oracle.pcg(rp, c, vals[s], b[s], rtol=1e-10)
        assert st[s] == 0 and rel(x[s].cpu().numpy(), xo) <= 1e-8


def test_all_kernel_variants_agree():
    B, N = 16, 24
    rp, c, vals = I.batched_shared_2d(N, B, seed0=3, sigma=0.5)
    b = to_dev(I.rhs_uniform(N * N, 2, batch=B))
    A = csr(rp, c)
    v = to_dev(vals)
    res = {}
    for cfg in sla.BATCH_CONFIGS:
        x, info = sla.cg_batched(A, v, b, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        res[cfg] = (x.clone(), np.atleast_1d(info.iters).copy())
    for code in (1, 2, 3):
        # same block size: on-chip or global vectors give the same bits
        assert torch.equal(res[code][0], res[code | 16][0])
        assert np.array_equal(res[code][1], res[code | 16][1])
        assert rel(res[code][0].cpu().numpy(), res[1][0].cpu().numpy()) <= 1e-9
    tuned = sla.cg_batched(A, v, b, rtol=1e-10, config="tune")[0]
    assert any(k[0] == "shared" for k in sla.tuned_configs())
    assert rel(tuned.cpu().numpy(), res[1][0].cpu().numpy()) <= 1e-9


def test_launch_shapes_threads_per_row_and_systems_per_cta():
    """Every launch shape the autotuner searches solves every system to the
    oracle's tolerance.  Several systems per CTA run each system on a slice
    of NT / SPC threads with its own named barrier and the same reduction
    tree as a CTA of that size, so their bits equal that shape's (512
    threads as two slices = 256 threads); more threads per row change the
    summation order of each row only."""
    B, N = 18, 24
    rp, c, vals = I.batched_shared_2d(N, B, seed0=5, sigma=0.5)
    b = I.rhs_uniform(N * N, 4, batch=B)
    A = csr(rp, c)
    v, bt = to_dev(vals), to_dev(b)
    res = {}
    for cfg in sla.BATCH_CONFIGS:
        x, info = sla.cg_batched(A, v, bt, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        res[cfg] = (x.cpu().numpy(), np.atleast_1d(info.iters).copy(), np.atleast_1d(info.status).copy())
        assert (res[cfg][2] == 0).all(), (cfg, sla.config_shape(cfg))
    S = sla.SPC_SHIFT
    for cfg, same in (((2 | 1 << S), 1), ((3 | 1 << S), 2), ((3 | 2 << S), 1)):
        assert np.array_equal(res[cfg][0], res[same][0]) and np.array_equal(res[cfg][1], res[same][1]), cfg
    for cfg in sla.BATCH_CONFIGS:
        assert rel(res[cfg][0], res[1][0]) <= 1e-9, cfg
    x8, i8 = sla.cg_batched(A, v, bt, rtol=1e-10, config=1 | 3 << sla.TPR_SHIFT)   # 8 threads per row
    torch.cuda.synchronize()
    _per_system_check([rp] * B, [c] * B, vals, b, x8.cpu().numpy(), i8, 1e-10)
    with pytest.raises(sla.L.SlaError):   # systems per CTA with more than one thread per row
        sla.cg_batched(A, v, bt, rtol=1e-10, config=2 | 1 << S | 1 << sla.TPR_SHIFT)
    with pytest.raises(sla.L.SlaError):   # unknown bit
        sla.cg_batched(A, v, bt, rtol=1e-10, config=2 | 1 << 12)


@pytest.mark.parametrize("cfg", [2 | 1 << 10, 1 | 2 << 10, 3 | 2 << 8])
def test_mixed_statuses_with_launch_shapes(cfg):
    """A slice whose system ends at once (b = 0, a bad diagonal) takes the
    next system while its sibling slice is still iterating."""
    B, N = 9, 20
    rp, c, vals = I.batched_shared_2d(N, B, seed0=7, sigma=0.5)
    b = I.rhs_uniform(N * N, 1, batch=B)
    b[1] = 0.0
    diag = np.nonzero(c == np.repeat(np.arange(N * N), np.diff(rp)))[0]
    vals[3, diag[10]] = -1.0
    x, info = sla.cg_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-10, config=cfg)
    torch.cuda.synchronize()
    st = np.atleast_1d(info.status)
    assert st[1] == 0 and np.atleast_1d(info.iters)[1] == 0 and not x[1].any()
    assert sla.L.STATUS_NAMES[int(st[3])] == "NOT_SPD"
    for s in (0, 2, 4, 5, 6, 7, 8):
        xo, _ = oracle.pcg(rp, c, vals[s], b[s], rtol=1e-13)
        assert st[s] == 0 and rel(x[s].cpu().numpy(), xo) <= 1e-8, s


def test_list_launch_shapes_match_oracle():
    mats = I.fem_list(20, seed0=2200, n_lo=100, n_hi=3000)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 90 + s) for s, (rp, _, _) in enumerate(mats)]
    bt = to_dev(np.concatenate(bs))
    for cfg in sla.LIST_CONFIGS:
        x, info = sla.cg_batched_list(P, to_dev(vals), bt, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        xs = [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
        _per_system_check([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs, info,
                          1e-10, iters_tol=3, idx=[0, 7, 19])


def test_tuned_choice_persists(tmp_path, monkeypatch):
    """config='tune' writes its choice to the cache file; a new process (the
    in-memory cache cleared) reads it back for config='auto'."""
    monkeypatch.setenv("SLA_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(sla, "_tune_cache", {})
    monkeypatch.setattr(sla, "_tune_loaded", False)
    B, N = 8, 16
    rp, c, vals = I.batched_shared_2d(N, B, seed0=3, sigma=0.5)
    A = csr(rp, c)
    v, bt = to_dev(vals), to_dev(I.rhs_uniform(N * N, 2, batch=B))
    sla.cg_batched(A, v, bt, rtol=1e-10, config="tune")
    key = ("shared", N * N, int(rp[-1]), B)
    chosen = sla.tuned_configs()[key]
    assert chosen in sla.BATCH_CONFIGS and (tmp_path / "tune.json").exists()
    monkeypatch.setattr(sla, "_tune_cache", {})
    monkeypatch.setattr(sla, "_tune_loaded", False)
    assert sla._resolve_config("auto", key, None, None, None) == chosen


def test_distinct_patterns_match_oracle():
    mats = I.fem_list(30, seed0=2000, n_lo=100, n_hi=3000)
    mats.append(I.diffusion2d_random(80, 9))         # 6400 rows: vectors off chip
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 50 + s) for s, (rp, _, _) in enumerate(mats)]
    x, info = sla.cg_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-10)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    xs = [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
    _per_system_check([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs, info, 1e-10)


def test_distinct_patterns_with_block_teams():
    """Systems with at least 32768 entries are solved by teams of blocks of a
    cooperative launch, the rest by single blocks of the same launch; against
    the oracle, also with the team path off (config bit 32, one CTA per
    system in the persistent kernel) and without a processing order (a team
    that meets a small system turns into single blocks, which then also take
    large systems): every variant is deterministic."""
    mats = I.fem_list(12, seed0=2100, n_lo=200, n_hi=3000)
    mats.insert(3, I.diffusion2d_random(120, 31))     # 14400 rows, 71520 entries
    mats.append(I.diffusion3d_random(25, 32))         # 15625 rows, 105625 entries
    mats.insert(7, I.diffusion2d_random(130, 33))     # 16900 rows (zero right-hand side below)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    nnzs = [int(rp[-1]) for rp, _, _ in mats]
    assert sum(z >= 32768 for z in nnzs) == 3
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 70 + s) for s, (rp, _, _) in enumerate(mats)]
    bs[7][:] = 0.0
    bt = to_dev(np.concatenate(bs))
    outs = {}
    for name, cfg, order in (("teams", 0, P.order), ("no_teams", 2 | 32, P.order), ("unordered", 0, None)):
        P.order = order
        x, info = sla.cg_batched_list(P, to_dev(vals), bt, rtol=1e-10, config=cfg)
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        xs = [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
        st = np.atleast_1d(info.status)
        its = np.atleast_1d(info.iters)
        assert st[7] == 0 and its[7] == 0 and not xs[7].any()
        idx = [s for s in range(len(mats)) if s != 7]
        _per_system_check([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs, info, 1e-10,
                          iters_tol=3, idx=idx)
        outs[name] = xh
        x2, _ = sla.cg_batched_list(P, to_dev(vals), bt, rtol=1e-10, config=cfg)
        assert np.array_equal(x2.cpu().numpy(), xh), name


def test_distinct_patterns_pipelined_teams():
    """config bit 64: the systems with at least 32768 entries by teams on the
    pipelined PCG, per system against the oracle's pipelined PCG (solution
    and iteration count), the small ones by single blocks on the standard
    form, against the oracle's PCG; with and without a processing order
    (with fewer systems than teams, every team takes one system from the
    queue, so each large system is a team's either way), a zero right-hand
    side, and deterministic across repeats."""
    mats = I.fem_list(10, seed0=2200, n_lo=200, n_hi=3000)
    mats.insert(2, I.diffusion2d_random(120, 41))     # 71520 entries: a team system
    mats.append(I.diffusion3d_random(25, 42))         # 105625 entries: a team system
    mats.insert(5, I.fem_list(1, seed0=2299, n_lo=500, n_hi=600)[0])
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 90 + s) for s, (rp, _, _) in enumerate(mats)]
    bs[5][:] = 0.0
    bt = to_dev(np.concatenate(bs))
    for order in (P.order, None):
        P.order = order
        x, info = sla.cg_batched_list(P, to_dev(vals), bt, rtol=1e-10, config=64)
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        st, its = np.atleast_1d(info.status), np.atleast_1d(info.iters)
        assert st[5] == 0 and its[5] == 0 and not xh[P.n_off_h[5]:P.n_off_h[6]].any()
        for s, (rp, c, v) in enumerate(mats):
            if s == 5:
                continue
            xo, io = oracle.pcg_pipelined(rp, c, v, bs[s], rtol=1e-10)
            xs, js = oracle.pcg(rp, c, v, bs[s], rtol=1e-10)
            if int(rp[-1]) < 32768:
                xo, io = xs, js  # a single block: the standard form
            assert st[s] == io["status"] == 0, s
            assert rel(xh[P.n_off_h[s]:P.n_off_h[s + 1]], xo) <= 1e-8, s
            assert abs(int(its[s]) - io["iters"]) <= 2, (s, its[s], io["iters"])
        x2, _ = sla.cg_batched_list(P, to_dev(vals), bt, rtol=1e-10, config=64)
        assert np.array_equal(x2.cpu().numpy(), xh)


def test_graph_capture_and_replay():
    B, N = 8, 16
    rp, c, vals = I.batched_shared_2d(N, B, seed0=11, sigma=0.5)
    A = csr(rp, c)
    v = to_dev(vals)
    b_static = to_dev(I.rhs_uniform(N * N, 1, batch=B))
    x_static = torch.empty_like(b_static)
    sla.cg_batched(A, v, b_static, rtol=1e-10, out=x_static)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sla.cg_batched(A, v, b_static, rtol=1e-10, out=x_static)
    torch.cuda.current_stream().wait_stream(s)
    b_new = to_dev(I.rhs_uniform(N * N, 2, batch=B))
    b_static.copy_(b_new)
    g.replay()
    torch.cuda.synchronize()
    x_ref, _ = sla.cg_batched(A, v, b_new, rtol=1e-10)
    torch.cuda.synchronize()
    assert torch.equal(x_static, x_ref)


def _capture(fn):
    """Runs fn once outside, then captures it in a CUDA graph on a side stream."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    return g


def test_graph_capture_of_cooperative_launches():
    """The cooperative paths (the block-team batch, single-system CG, G G^T
    PCG and BiCGStab below their size limits) only enqueue work, so a CUDA
    graph captures them; replays with new right-hand sides give the bits of
    direct calls."""
    mats = I.fem_list(6, seed0=2300, n_lo=200, n_hi=2000)
    mats.append(I.diffusion2d_random(120, 41))        # a team system
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = to_dev(np.concatenate([v for _, _, v in mats]))
    b_static = to_dev(np.concatenate([I.rhs_uniform(len(rp) - 1, 90 + s) for s, (rp, _, _) in enumerate(mats)]))
    x_static = torch.empty_like(b_static)
    g = _capture(lambda: sla.cg_batched_list(P, vals, b_static, rtol=1e-10, out=x_static))
    b_new = to_dev(np.concatenate([I.rhs_uniform(len(rp) - 1, 190 + s) for s, (rp, _, _) in enumerate(mats)]))
    b_static.copy_(b_new)
    g.replay()
    torch.cuda.synchronize()
    x_ref, info = sla.cg_batched_list(P, vals, b_new, rtol=1e-10)
    torch.cuda.synchronize()
    assert (np.atleast_1d(info.status) == 0).all()
    assert torch.equal(x_static, x_ref)
    # single-system solvers
    rp, c, v = I.diffusion2d_random(70, 42)
    n = len(rp) - 1
    A = csr(rp, c)
    vt = to_dev(v)
    bs = to_dev(I.rhs_uniform(n, 5))
    xs = torch.empty_like(bs)
    g2 = _capture(lambda: sla.cg(A, vt, bs, rtol=1e-10, out=xs))
    rpc, cc, vc = I.convdiff3d(14, 6.0)
    Ac = csr(rpc, cc)
    vct = to_dev(vc)
    bc = to_dev(I.rhs_uniform(14 ** 3, 6))
    xc = torch.empty_like(bc)
    g3 = _capture(lambda: sla.bicgstab(Ac, vct, bc, rtol=1e-10, out=xc))
    bs.copy_(to_dev(I.rhs_uniform(n, 8)))
    bc.copy_(to_dev(I.rhs_uniform(14 ** 3, 9)))
    g2.replay()
    g3.replay()
    torch.cuda.synchronize()
    x2, i2 = sla.cg(A, vt, bs, rtol=1e-10)
    x3, i3 = sla.bicgstab(Ac, vct, bc, rtol=1e-10)
    torch.cuda.synchronize()
    assert i2.status == 0 and i3.status == 0
    assert torch.equal(xs, x2) and torch.equal(xc, x3)


def test_batched_adjoint_matches_single_solves():
    B, N = 5, 16
    rp, c, vals = I.batched_shared_2d(N, B, seed0=21, sigma=0.5)
    A = csr(rp, c)
    v = to_dev(vals).requires_grad_(True)
    b = to_dev(I.rhs_uniform(N * N, 3, batch=B)).requires_grad_(True)
    x = sla.solve_batched(A, v, b, rtol=1e-12)
    (x * x).sum().backward()
    for s in range(B):
        xo, _ = oracle.pcg(rp, c, vals[s], b[s].detach().cpu().numpy(), rtol=1e-13)
        gb, gv, _ = oracle.adjoint_backward(rp, c, vals[s], xo, 2 * xo, rtol=1e-13)
        assert rel(b.grad[s].cpu().numpy(), gb) <= 1e-6
        assert elementwise_rel(b.grad[s].cpu().numpy(), gb) <= 1e-6
        assert rel(v.grad[s].cpu().numpy(), gv) <= 1e-6
        assert elementwise_rel(v.grad[s].cpu().numpy(), gv) <= 1e-6


@pytest.mark.slow
def test_full_size_shared_1024_systems_64():
    """The shared-pattern batch at full size: 1024 systems on the 64 x 64
    five-point pattern, faces exp(N(0, 0.5^2)) from seeds 1000 + s, rtol 1e-8:
    sampled systems against the oracle, every system's residual by the
    oracle's SpMV."""
    B, N = 1024, 64
    rp, c, vals = I.batched_shared_2d(N, B, seed0=1000, sigma=0.5)
    b = I.rhs_uniform(N * N, 7, batch=B)
    x, info = sla.cg_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-8)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    assert (np.atleast_1d(info.status) == 0).all()
    for s in range(B):
        r = b[s] - oracle.spmv(rp, c, vals[s], xh[s])
        assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b[s])
    _per_system_check([rp] * B, [c] * B, vals, b, xh, info, 1e-8, idx=[0, 1, 511, 1023])
    # the same launch at rtol 1e-10 against the oracle's x* on 16 systems
    x10, i10 = sla.cg_batched(csr(rp, c), to_dev(vals), to_dev(b), rtol=1e-10)
    torch.cuda.synchronize()
    assert (np.atleast_1d(i10.status) == 0).all()
    idx = sorted(set(np.random.default_rng(8).choice(B, 14, replace=False).tolist()) | {0, B - 1})
    _vs_oracle_xstar([rp] * B, [c] * B, vals, b, x10.cpu().numpy(), idx)


@pytest.mark.slow
@pytest.mark.parametrize("config", [0, 64])
def test_full_size_fem_list_512(config):
    """512 jittered, holed P1 FEM Laplacians with n log-uniform in [1e3, 5e4]
    (+1e-3 I), rtol 1e-8, in one launch; also with the team systems on the
    pipelined PCG (config bit 64)."""
    mats = I.fem_list(512, seed0=2000)
    P = sla.CSRList([(rp, c) for rp, c, _ in mats])
    vals = np.concatenate([v for _, _, v in mats])
    bs = [I.rhs_uniform(len(rp) - 1, 3000 + s) for s, (rp, _, _) in enumerate(mats)]
    x, info = sla.cg_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-8, config=config)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    assert (np.atleast_1d(info.status) == 0).all()
    xs = [xh[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
    for s, (rp, c, v) in enumerate(mats):
        r = bs[s] - oracle.spmv(rp, c, v, xs[s])
        assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(bs[s])
    big = int(np.argmax([len(m[0]) for m in mats]))
    if config == 0:
        _per_system_check([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, xs, info,
                          1e-8, iters_tol=5, idx=[0, 1, big])
        # the same launch at rtol 1e-10 against the oracle's x* on 16 systems,
        # the four largest (block teams) among them
        x10, i10 = sla.cg_batched_list(P, to_dev(vals), to_dev(np.concatenate(bs)), rtol=1e-10)
        torch.cuda.synchronize()
        assert (np.atleast_1d(i10.status) == 0).all()
        xh10 = x10.cpu().numpy()
        x10s = [xh10[P.n_off_h[s]:P.n_off_h[s + 1]] for s in range(len(mats))]
        sizes = np.array([len(m[0]) for m in mats])
        idx = set(np.argsort(sizes)[-4:].tolist()) | set(np.random.default_rng(9).choice(len(mats), 12, replace=False).tolist())
        _vs_oracle_xstar([m[0] for m in mats], [m[1] for m in mats], [m[2] for m in mats], bs, x10s, sorted(idx))
        return
    # the team systems ran the pipelined PCG: against the oracle's pipelined PCG
    its = np.atleast_1d(info.iters)
    rp, c, v = mats[big]
    assert int(rp[-1]) >= 32768
    xo, io = oracle.pcg_pipelined(rp, c, v, bs[big], rtol=1e-8)
    assert io["status"] == 0 and rel(xs[big], xo) <= 1e-7 and abs(int(its[big]) - io["iters"]) <= 5
