"""Learned factored preconditioner: kernels against the FP64 oracle
(oracle/mpnn.py), and what training gains over Jacobi-PCG."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import mpnn as OM
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import learned as LP
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, elementwise_rel, rel, to_dev

pytestmark = pytest.mark.gpu


def oracle_params(model):
    """The exact values the kernels read: BF16 weight matrices, FP32 vectors."""
    pb = model.params_numpy(bf16=True)
    pf = model.params_numpy(bf16=False)
    return {k: (pb[k] if pb[k].ndim == 2 else pf[k]) for k in pf}


def test_zero_head_gives_the_jacobi_factor_exactly():
    rp, c, v = I.diffusion2d_random(24, 3)
    model = LP.LearnedPreconditioner(seed=0)
    G, gv = model.factor(csr(rp, c), to_dev(v), normalize=False)
    grp, gcol, og = OM.forward(oracle_params(model), rp, c, v)
    g, o = gv.cpu().numpy(), og.numpy()
    assert np.array_equal(G.rowptr.cpu().numpy(), grp) and np.array_equal(G.col.cpu().numpy(), gcol)
    # G = D^{-1/2} (off-diagonal zero) to rounding: within 2 ulps of the oracle
    relerr = np.abs(g - o) / np.where(o != 0, np.abs(o), 1.0)
    assert relerr.max() <= 4.5e-16, relerr.max()
    rows = np.repeat(np.arange(len(grp) - 1), np.diff(grp))
    assert not g[rows != gcol].any()


@pytest.mark.parametrize("mat", ["var2d", "var3d", "fem"])
def test_column_normalisation_matches_oracle(mat):
    """sla_ggt_normalize on the network's factor (untrained, non-zero head)
    against the oracle's loop form, and the normalised factor's property
    diag(G^T A G) = I by an independent SpMV; Jacobi stays Jacobi."""
    rp, c, v = {"var2d": lambda: I.diffusion2d_random(30, 4, 1.5), "var3d": lambda: I.diffusion3d_random(9, 5),
                "fem": lambda: I.fem_p1_laplacian(20, 6)}[mat]()
    n = len(rp) - 1
    model = LP.LearnedPreconditioner(seed=2)
    model.view("v").fill_(0.05)
    model._sync_bf16()
    A = csr(rp, c)
    G, raw = model.factor(A, to_dev(v), normalize=False)
    G2, gv = model.factor(A, to_dev(v))
    grp, gcol = G.rowptr.cpu().numpy(), G.col.cpu().numpy()
    ref = OM.column_normalize(grp, gcol, raw.cpu().numpy(), rp, c, v)
    assert rel(gv.cpu().numpy(), ref) <= 1e-14
    # (G^T A G)_jj = ||A^{1/2} G e_j||^2 = (G e_j)^T A (G e_j) for a few columns
    import scipy.sparse as sp
    Gs = sp.csr_matrix((gv.cpu().numpy(), gcol, grp), shape=(n, n))
    As = sp.csr_matrix((v, c, rp), shape=(n, n))
    for j in (0, n // 3, n - 1):
        gj = Gs[:, j].toarray().ravel()
        assert abs(gj @ (As @ gj) - 1.0) <= 1e-13
    # the zero head (Jacobi) is a fixed point to rounding
    mz = LP.LearnedPreconditioner(seed=0)
    Gz, gz = mz.factor(A, to_dev(v))
    gz = gz.cpu().numpy()
    zrows = np.repeat(np.arange(n), np.diff(Gz.rowptr.cpu().numpy()))
    zdiag = zrows == Gz.col.cpu().numpy()
    d = v[c == np.repeat(np.arange(n), np.diff(rp))]
    assert rel(gz[zdiag], 1.0 / np.sqrt(d)) <= 1e-15 and not gz[~zdiag].any()


@pytest.mark.parametrize("mat", ["var2d", "var3d", "fem"])
def test_forward_and_gradients_match_oracle(mat):
    if mat == "var2d":
        rp, c, v = I.diffusion2d_random(20, 4, 1.5)
    elif mat == "var3d":
        rp, c, v = I.diffusion3d_random(7, 5)
    else:
        rp, c, v = I.fem_p1_laplacian(16, 7)
    n = len(rp) - 1
    model = LP.LearnedPreconditioner(seed=1)
    # a non-zero head so that every parameter matters
    model.view("v").copy_(torch.linspace(-0.3, 0.3, 32, device="cuda"))
    model.view("vd").copy_(torch.linspace(0.2, -0.2, 32, device="cuda"))
    model._sync_bf16()
    A = csr(rp, c)
    vt = to_dev(v)
    gr = model.graph(A, vt)
    gv = model.forward(gr).cpu().numpy()
    P = oracle_params(model)
    _, _, og = OM.forward(P, rp, c, v)
    assert rel(gv, og.numpy()) <= 1e-5
    b = np.random.default_rng(0).standard_normal(n)
    xs, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    Lg = float(model.loss_grad(gr, to_dev(b), to_dev(xs)))
    model.backward(gr)
    Lo, grads, _ = OM.loss_and_grads(P, rp, c, v, b, xs)
    assert abs(Lg - Lo) <= 1e-4 * abs(Lo)
    for k, go in grads.items():
        gk = model.view(k, "g").double().cpu().numpy()
        assert rel(gk, go) <= 2e-3, (k, rel(gk, go))


@pytest.mark.parametrize("mat", ["var2d", "var3d", "fem", "dense"])
def test_fsai_factor_matches_oracle(mat):
    """sla_fsai_factor (the classical factor the learned one is measured
    against) equals the oracle's column-by-column definition; with every
    entry stored (dense A) it is the exact factor, G G^T = A^{-1}, and PCG
    with it converges in one iteration."""
    if mat == "var2d":
        rp, c, v = I.diffusion2d_random(11, 5, 1.5)
    elif mat == "var3d":
        rp, c, v = I.diffusion3d_random(6, 7)
    elif mat == "fem":
        rp, c, v = I.fem_p1_laplacian(9, 4)
    else:
        rng = np.random.default_rng(2)
        n = 10
        X = rng.standard_normal((n, n))
        M = X @ X.T + n * np.eye(n)
        rp = np.arange(0, n * n + 1, n, dtype=np.int32)
        c = np.tile(np.arange(n, dtype=np.int32), n)
        v = M.reshape(-1).copy()
    n = len(rp) - 1
    A = csr(rp, c)
    G, gv, fb = LP.fsai_factor(A, to_dev(v))
    assert fb == 0
    Go = OM.fsai_factor(rp, c, v)
    grp, gcol, g = G.rowptr.cpu().numpy(), G.col.cpu().numpy(), gv.cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(grp))
    assert np.allclose(g, Go[rows, gcol], rtol=1e-12, atol=1e-14)
    assert np.count_nonzero(Go) == len(g)
    # the solve applies G's values stored in FP32 (G32 G32^T), as does the oracle here
    b = I.rhs_uniform(n, 3)
    x, info = sla.cg_ggt(A, to_dev(v), G, gv, to_dev(b), rtol=1e-12)
    g32 = g.astype(np.float32).astype(np.float64)
    xo, io = oracle.pcg(rp, c, v, b, rtol=1e-12, precond="ggt", G=(grp, gcol, g32))
    assert info.status == 0 and io["status"] == 0
    assert rel(x.cpu().numpy(), xo) <= 1e-8 and abs(info.iters - io["iters"]) <= 2
    if mat == "dense":
        # G G^T = A^{-1} up to the FP32 storage of G: a handful of iterations
        assert info.iters <= 4


@pytest.mark.parametrize("scale_free", [False, True])
def test_loss_gradient_wrt_g_matches_oracle(scale_free):
    """sla_ggt_loss_grad (mode 0, and mode 1: the error of the best multiple
    of G G^T b, its gradient taken at the minimising scale) against the
    oracle's loss and autograd's gradient (through the scale in mode 1)."""
    import torch as T
    rp, c, v = I.diffusion2d_random(12, 6)
    n = len(rp) - 1
    model = LP.LearnedPreconditioner(seed=2)
    model.view("v").fill_(0.1)
    model._sync_bf16()
    gr = model.graph(csr(rp, c), to_dev(v))
    gv = model.forward(gr).cpu().numpy()
    b = np.random.default_rng(1).standard_normal(n)
    xs, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    Lg = float(model.loss_grad(gr, to_dev(b), to_dev(xs), scale_free))
    dG = gr.dG[:gr.nnz_g].cpu().numpy()
    g = T.tensor(gv, requires_grad=True)
    L = OM.loss(gr.G.rowptr.cpu().numpy(), gr.G.col.cpu().numpy(), g, rp, c, v, b, xs, scale_free=scale_free)
    L.backward()
    Lo = float(L.detach())
    assert abs(Lg - Lo) <= 1e-12 * abs(Lo)
    tol = 1e-10 if scale_free else 1e-12
    assert rel(dG, g.grad.numpy()) <= tol
    assert elementwise_rel(dG, g.grad.numpy()) <= tol
    if scale_free:
        # the loss and its gradient do not see a scale of G
        gr.g_val[:gr.nnz_g].mul_(2.5)
        assert abs(float(model.loss_grad(gr, to_dev(b), to_dev(xs), True)) - Lg) <= 1e-12 * Lg


def test_training_beats_jacobi_on_unseen_system():
    torch.manual_seed(0)
    model = LP.LearnedPreconditioner(seed=3)
    hist = LP.train(model, systems=16, steps=300, lr=3e-3, n_lo=32, n_hi=64, log_every=50)
    assert hist[-1] < hist[0]
    rp, c, v = I.diffusion2d_random(96, 990001, 1.5)   # unseen size and seed
    A = csr(rp, c)
    vt = to_dev(v)
    b = to_dev(I.rhs_uniform(len(rp) - 1, 5))
    x, info, fb = model.solve(A, vt, b, rtol=1e-8)
    xj, ij = sla.cg(A, vt, b, rtol=1e-8)
    torch.cuda.synchronize()
    assert info.status == 0 and not fb
    assert info.true_rel_res <= 2e-8
    assert info.iters < ij.iters
    assert rel(x.cpu().numpy(), xj.cpu().numpy()) <= 1e-6


@pytest.mark.slow
def test_trained_factor_on_unseen_1024_system():
    """Config 5 evaluation size: after the bench's short training recipe the
    learned G G^T PCG reaches rtol 1e-8 on the unseen 2D 1024^2 system with
    the FP64 true residual inside 2 rtol, in fewer iterations than
    Jacobi-PCG, and the solution agrees with Jacobi-PCG's."""
    model = LP.LearnedPreconditioner(seed=0)
    LP.train(model, systems=48, steps=800, lr=3e-3, n_lo=64, n_hi=128, log_every=400)
    rp, c, v = I.diffusion2d_random(1024, 900001, 1.0)
    A = csr(rp, c)
    vt = to_dev(v)
    bt = to_dev(I.rhs_uniform(len(rp) - 1, 77))
    xj, ij = sla.cg(A, vt, bt, rtol=1e-8)
    G, gv = model.factor(A, vt)
    xg, ig = sla.cg_ggt(A, vt, G, gv, bt, rtol=1e-8)
    torch.cuda.synchronize()
    assert ig.status == 0 and ij.status == 0
    assert ig.true_rel_res <= 2e-8
    assert ig.iters * 1.5 < ij.iters
    r = bt - sla.spmv(A, vt, xg)
    assert float(r.norm() / bt.norm()) <= 2e-8
    assert rel(xg.cpu().numpy(), xj.cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("n,K1,K2,M,relu,res,pre", [
    (300, 32, 32, 32, 1, 1, 1),     # a message-passing layer: [H | Agg] W^T, relu, residual (3 tiles, ragged)
    (129, 32, 0, 96, 0, 0, 0),      # the head's [P | Q | R] = H Uh^T + bh (a 1-row tail tile)
    (70000, 32, 32, 32, 1, 1, 0),   # many tiles per CTA
    (77, 4, 0, 16, 1, 0, 1),        # K padded to 16, M = 16, one partial tile
])
def test_dense_layer_tensor_cores_match_definition(n, K1, K2, M, relu, res, pre):
    """The dense layer on the tcgen05 tensor cores (FP32 activations split
    into three BF16 pieces, BF16 weights, FP32 accumulation in TMEM) against
    its definition Y = relu([X1 | X2] W^T + b) + R in FP64 and against the
    CUDA-core kernel, element by element."""
    import ctypes
    lib = LP._bind()
    g = np.random.default_rng(n + M)
    X1 = g.standard_normal((n, K1)).astype(np.float32)
    X2 = g.standard_normal((n, K2)).astype(np.float32) if K2 else None
    W = torch.from_numpy(0.2 * g.standard_normal((M, K1 + K2))).to(torch.bfloat16)
    b = g.standard_normal(M).astype(np.float32)
    R = g.standard_normal((n, M)).astype(np.float32) if res else None
    Xc = np.concatenate([X1, X2], 1) if K2 else X1
    ypre = Xc.astype(np.float64) @ W.double().numpy().T + b
    y = (np.maximum(ypre, 0.0) if relu else ypre) + (R if res else 0.0)
    out = {}
    dev = {k: (torch.from_numpy(a).cuda() if a is not None else None) for k, a in
           (("X1", X1), ("X2", X2), ("b", b), ("R", R))}
    Wd = W.cuda()
    for kern in (LP.L.SLA_MP_DENSE_SIMT, LP.L.SLA_MP_DENSE_TC):
        Y = torch.full((n, M), float("nan"), device="cuda")
        Yp = torch.full((n, M), float("nan"), device="cuda") if pre else None
        ptr = lambda t: t.data_ptr() if t is not None else None
        rc = lib.sla_mp_dense_fwd_ex(n, K1, ptr(dev["X1"]), K2, ptr(dev["X2"]), M, Wd.data_ptr(), ptr(dev["b"]),
                                     ptr(dev["R"]), relu, ptr(Yp), Y.data_ptr(), kern, None)
        torch.cuda.synchronize()
        assert rc == 0, (kern, rc)
        out[kern] = (Y.cpu().double().numpy(), Yp.cpu().double().numpy() if pre else None)
    flag = ctypes.c_int32(-1)
    assert lib.sla_mp_tc_errors(ctypes.byref(flag)) == 0 and flag.value == 0
    scale = np.abs(y).max()
    for kern, (Y, Yp) in out.items():
        assert np.abs(Y - y).max() <= 1e-6 * scale, (kern, np.abs(Y - y).max() / scale)
        if pre:
            assert np.abs(Yp - ypre).max() <= 1e-6 * np.abs(ypre).max()
    ts, tt = out[LP.L.SLA_MP_DENSE_SIMT][0], out[LP.L.SLA_MP_DENSE_TC][0]
    assert np.abs(ts - tt).max() <= 1e-6 * scale


def test_dense_layer_tensor_core_shape_rules():
    """The tensor-core form takes K1, K2 multiples of 4 and M a multiple of
    16 (up to 96); other shapes are refused for it and run on the CUDA cores
    under automatic selection (the 3-feature input layer)."""
    lib = LP._bind()
    n = 40
    X = torch.randn(n, 3, device="cuda")
    W = torch.randn(32, 3, device="cuda").to(torch.bfloat16)
    Y = torch.empty(n, 32, device="cuda")
    assert lib.sla_mp_dense_fwd_ex(n, 3, X.data_ptr(), 0, None, 32, W.data_ptr(), None, None, 1, None,
                                   Y.data_ptr(), LP.L.SLA_MP_DENSE_TC, None) == LP.L.SLA_ERR_INVALID
    assert lib.sla_mp_dense_fwd_ex(n, 3, X.data_ptr(), 0, None, 32, W.data_ptr(), None, None, 1, None,
                                   Y.data_ptr(), LP.L.SLA_MP_DENSE_AUTO, None) == 0
    torch.cuda.synchronize()
    ref = torch.relu(X.double() @ W.double().t())
    assert float((Y.double() - ref).abs().max()) <= 1e-6 * float(ref.abs().max())
    assert lib.sla_mp_dense_fwd_ex(n, 3, X.data_ptr(), 0, None, 32, W.data_ptr(), None, None, 1, None,
                                   Y.data_ptr(), 7, None) == LP.L.SLA_ERR_INVALID


@pytest.mark.parametrize("scale_free", [False, True])
def test_training_through_the_normalisation_matches_oracle(scale_free):
    """sla_ggt_normalize_bwd against autograd through the oracle's
    differentiable normalisation, and the loss of the normalised factor with
    its gradient w.r.t. the network's values (normalise, loss, backward of
    the normalisation) against the oracle's autograd of the same chain."""
    import torch as T
    rp, c, v = I.diffusion2d_random(14, 8, 1.2)
    n = len(rp) - 1
    model = LP.LearnedPreconditioner(seed=4)
    model.view("v").copy_(T.linspace(-0.2, 0.2, 32, device="cuda"))
    model.view("vd").fill_(0.05)
    model._sync_bf16()
    gr = model.graph(csr(rp, c), to_dev(v))
    gv = model.forward(gr).clone()
    grp, gcol = gr.G.rowptr.cpu().numpy(), gr.G.col.cpu().numpy()
    # the backward alone, on a random dL/dGn
    dgn = np.random.default_rng(5).standard_normal(gr.nnz_g)
    dG = T.empty_like(gv)
    lib = LP._bind()
    rc = lib.sla_ggt_normalize_bwd(ctypes.byref(gr.A.c), gr.val.data_ptr(), ctypes.byref(gr.G.c),
                                   ctypes.byref(gr.G._transpose_c), gv.data_ptr(), to_dev(dgn).data_ptr(),
                                   dG.data_ptr(), sla._stream_ptr(gv.device))
    assert rc == 0
    g = T.tensor(gv.cpu().numpy(), requires_grad=True)
    (OM.column_normalize_t(grp, gcol, g, rp, c, v) * T.tensor(dgn)).sum().backward()
    assert rel(dG.cpu().numpy(), g.grad.numpy()) <= 1e-12
    # the whole chain
    b = np.random.default_rng(6).standard_normal(n)
    xs, _ = oracle.pcg(rp, c, v, b, rtol=1e-13)
    L = float(model.loss_grad_normalised(gr, to_dev(b), to_dev(xs), scale_free))
    got = gr.dG[:gr.nnz_g].cpu().numpy()
    g2 = T.tensor(gv.cpu().numpy(), requires_grad=True)
    Lo = OM.loss(grp, gcol, OM.column_normalize_t(grp, gcol, g2, rp, c, v), rp, c, v, b, xs, scale_free=scale_free)
    Lo.backward()
    assert abs(L - float(Lo.detach())) <= 1e-12 * abs(float(Lo.detach()))
    assert rel(got, g2.grad.numpy()) <= 1e-10 and elementwise_rel(got, g2.grad.numpy()) <= 1e-10
