"""The eigenvalue path (Sec. 3.2 "Eigenvalue problems", Eq. 4; Tab. 5
"Eigenvalue (k = 6)") through the C ABI: LOBPCG eigenpairs against the
oracle's definition (dense symmetric eigensolve), the Hellmann-Feynman
gradient against the oracle's loop and against central differences of the
library's own eigenvalues."""
import numpy as np
import pytest
import torch

from oracle import eigen as OE
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, to_dev

pytestmark = pytest.mark.gpu


def laplacian_1d(n):
    rp, c, v = [0], [], []
    for i in range(n):
        for j, a in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                c.append(j)
                v.append(a)
        rp.append(len(c))
    return np.array(rp, np.int32), np.array(c, np.int32), np.array(v)


def check_pairs(lam, V, lo, Vo, tol):
    assert np.abs(lam - lo).max() <= 1e-10 * np.abs(lo).max()
    for i in range(len(lo)):
        gap = min([abs(lo[i] - lo[j]) for j in range(len(lo)) if j != i] + [np.inf])
        cosv = abs(float(V[:, i] @ Vo[:, i])) / np.linalg.norm(V[:, i])
        assert 1.0 - cosv <= max(1e-10, 10 * (tol * lo[i] / gap) ** 2), (i, 1.0 - cosv)


@pytest.mark.parametrize("name,gen,k", [
    ("lap1d_200", lambda: laplacian_1d(200), 6),
    ("diff2d_37", lambda: I.diffusion2d_random(37, 5), 6),
    ("diff3d_12", lambda: I.diffusion3d_random(12, 2), 4),
    ("fem_20", lambda: I.fem_p1_laplacian(20, 3), 8),
    ("lap1d_k1", lambda: laplacian_1d(64), 1),
])
def test_eigsh_matches_oracle(name, gen, k):
    rp, c, v = gen()
    A = csr(rp, c)
    lam, V, info = sla.eigsh(A, to_dev(v), k, tol=1e-9)
    lo, Vo = OE.smallest_eigenpairs(rp, c, v, k)
    assert info.status == 0 and info.true_rel_res <= 2e-9
    check_pairs(lam.cpu().numpy(), V.cpu().numpy(), lo, Vo, 1e-9)
    # unit columns
    assert np.abs(np.linalg.norm(V.cpu().numpy(), axis=0) - 1.0).max() <= 1e-12


def test_hellmann_feynman_gradient_matches_oracle_and_fd():
    rp, c, v = I.diffusion2d_random(24, 7)
    k = 6
    A = csr(rp, c)
    val = to_dev(v).requires_grad_(True)
    w = torch.tensor([1.0, -0.5, 2.0, 0.25, 1.5, -1.0], dtype=torch.float64, device="cuda")
    lam, V, info = sla.eigsh(A, val, k, tol=1e-10)
    (lam * w).sum().backward()
    lo, Vo = OE.smallest_eigenpairs(rp, c, v, k)
    go = OE.eigenvalue_grad_values(rp, c, Vo, w.cpu().numpy())
    g = val.grad.cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-7 * np.linalg.norm(go)
    # the direct kernel call gives the same
    g2 = sla.eig_grad_values(A, V, w).cpu().numpy()
    assert np.array_equal(g, g2)
    # central differences of the library's eigenvalues along symmetric
    # perturbations of the stored entries (eps = 1e-5; Tab. 5: 2.1e-6)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    rng = np.random.default_rng(3)
    eps = 1e-5
    for _ in range(2):
        D = np.zeros((len(rp) - 1,) * 2)
        D[rows, c] = rng.standard_normal(len(v))
        D = 0.5 * (D + D.T)
        dv = D[rows, c]
        lp, _, _ = sla.eigsh(A, to_dev(v + eps * dv), k, tol=1e-10, v0=V.detach().reshape(-1))
        lm, _, _ = sla.eigsh(A, to_dev(v - eps * dv), k, tol=1e-10, v0=V.detach().reshape(-1))
        fd = float(((lp - lm) * w).sum()) / (2 * eps)
        assert abs(fd - float(g @ dv)) <= 2.1e-6 * abs(fd)


def test_eigsh_edge_cases_and_determinism():
    rp, c, v = I.diffusion2d_random(30, 4)
    A = csr(rp, c)
    vt = to_dev(v)
    l1, V1, i1 = sla.eigsh(A, vt, 6)
    l2, V2, i2 = sla.eigsh(A, vt, 6)
    assert torch.equal(l1, l2) and torch.equal(V1, V2) and i1.iters == i2.iters
    # start at the eigenvectors: converged at once
    l3, _, i3 = sla.eigsh(A, vt, 6, v0=V1.reshape(-1).contiguous())
    assert i3.status == 0 and i3.iters <= 1
    assert torch.allclose(l3, l1, rtol=1e-12, atol=0)
    # iteration cap
    _, _, i4 = sla.eigsh(A, vt, 6, tol=1e-14, max_iter=5, strict=False)
    assert i4.status_name == "NOT_CONVERGED" and i4.iters == 5
    # non-positive diagonal with Jacobi
    v2 = v.copy()
    v2[rp[3]:rp[4]][c[rp[3]:rp[4]] == 3] = 0.0
    _, _, i5 = sla.eigsh(A, to_dev(v2), 4, strict=False)
    assert i5.status_name == "NOT_SPD"
    # no preconditioner converges to the same pairs
    l6, _, i6 = sla.eigsh(A, vt, 6, precond="none", max_iter=20000)
    assert i6.status == 0 and torch.allclose(l6, l1, rtol=1e-10, atol=0)
    with pytest.raises(ValueError):
        sla.eigsh(A, vt, 9)
    # V carries a gradient; a V-only loss leaves the eigenvalue part zero
    val = vt.clone().requires_grad_(True)
    lam, V, _ = sla.eigsh(A, val, 2)
    assert V.requires_grad
    V[:, 0].sum().backward()
    assert torch.isfinite(val.grad).all() and bool(val.grad.abs().max() > 0)
    # through the COO front end
    n = len(rp) - 1
    row = torch.from_numpy(np.repeat(np.arange(n), np.diff(rp)).astype(np.int64)).cuda()
    col = torch.from_numpy(c.astype(np.int64)).cuda()
    T = sla.SparseTensor(vt.clone(), row, col, (n, n))
    l7, _, _ = T.eigsh(6)
    assert torch.allclose(l7, l1, rtol=1e-10, atol=0)


@pytest.mark.slow
def test_eigsh_at_128():
    """The bench workload (2D 128^2, sigma = 1, k = 6, tol 1e-8): converged,
    true residuals within 2 tol, and eigenvalues against ARPACK shift-invert
    (a library eigensolver, independent of the LOBPCG path)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    rp, c, v = I.diffusion2d_random(128, 11, 1.0)
    n = len(rp) - 1
    A = csr(rp, c)
    lam, V, info = sla.eigsh(A, to_dev(v), 6, tol=1e-8)
    assert info.status == 0 and info.true_rel_res <= 2e-8
    ref = np.sort(spla.eigsh(sp.csr_matrix((v, c, rp), shape=(n, n)), k=6, sigma=0, which="LM")[0])
    assert np.abs(lam.cpu().numpy() - ref).max() <= 1e-10 * ref.max()


@pytest.mark.parametrize("n,k", [(4, 4), (6, 4), (10, 8), (3, 1)])
def test_eigsh_tiny_systems(n, k):
    """n <= k + 2: the block spans (nearly) the whole space, the Gram matrix
    is rank-deficient by construction (its Cholesky factor fails and the
    eigendecomposition route drops the dependent directions); every wanted
    pair still matches the dense eigensolve."""
    rng = np.random.default_rng(n * 10 + k)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = Q @ np.diag(np.linspace(1.0, 3.0, n)) @ Q.T
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    c = np.tile(np.arange(n, dtype=np.int32), n)
    v = M.reshape(-1)
    A = csr(rp, c)
    lam, V, info = sla.eigsh(A, to_dev(v), k, tol=1e-10)
    lo, Vo = OE.smallest_eigenpairs(rp, c, v, k)
    assert info.status == 0
    assert np.abs(lam.cpu().numpy() - lo).max() <= 1e-12 * lo.max()
    Vn = V.cpu().numpy()
    for i in range(k):
        assert abs(abs(float(Vn[:, i] @ Vo[:, i])) - 1.0) <= 1e-10


# ---------------------------------------------------------------------------
# Eigenvector gradients (Sec. 3.2: one deflated solve per pair)
# ---------------------------------------------------------------------------

def _vector_adjoint(rp, c, v, lam, V, gV, **kw):
    A = csr(rp, c)
    mu, info = sla.eig_vector_adjoint(A, to_dev(v), to_dev(np.asarray(lam)), to_dev(np.ascontiguousarray(V)),
                                      to_dev(np.ascontiguousarray(gV)), **kw)
    torch.cuda.synchronize()
    return mu.cpu().numpy(), info


@pytest.mark.parametrize("precond", ["jacobi", "none"])
@pytest.mark.parametrize("name,gen,k", [("diff2d_12", lambda: I.diffusion2d_random(12, 5), 4),
                                        ("diff3d_6", lambda: I.diffusion3d_random(6, 6), 6),
                                        ("lap1d_40", lambda: laplacian_1d(40), 8)])
def test_eigenvector_adjoint_matches_oracle(name, gen, k, precond):
    """mu against the oracle's bordered solve on the oracle's own pairs;
    every pair converged, v_j^T mu_j = 0, and bit-identical on a repeat."""
    rp, c, v = gen()
    lam, V = OE.smallest_eigenpairs(rp, c, v, k)
    gV = np.random.default_rng(11).standard_normal((len(rp) - 1, k))
    mu_o = OE.eigenvector_adjoint(rp, c, v, lam, V, gV)
    mu, info = _vector_adjoint(rp, c, v, lam, V, gV, rtol=1e-12, precond=precond)
    assert (np.atleast_1d(info.status) == 0).all(), info.status_name
    assert (np.atleast_1d(info.true_rel_res) <= 1e-11).all()
    for j in range(k):
        assert np.linalg.norm(mu[:, j] - mu_o[:, j]) <= 1e-9 * np.linalg.norm(mu_o[:, j]), (j, precond)
        assert abs(V[:, j] @ mu[:, j]) <= 1e-10 * np.linalg.norm(mu_o[:, j])
    mu2, _ = _vector_adjoint(rp, c, v, lam, V, gV, rtol=1e-12, precond=precond)
    assert np.array_equal(mu, mu2)


def test_eigenvector_adjoint_edge_cases():
    """k = n (span(V)^perp is empty: the closed form alone, no iteration);
    gV = 0 (mu = 0); gV along V only (b = 0, mu from the closed form);
    a repeated eigenvalue (BREAKDOWN for the pairs involved, OK for the
    rest); max_iter = 0 (NOT_CONVERGED)."""
    rp, c, v = laplacian_1d(5)
    lam, V = OE.smallest_eigenpairs(rp, c, v, 5)
    gV = np.random.default_rng(1).standard_normal((5, 5))
    mu, info = _vector_adjoint(rp, c, v, lam, V, gV)
    assert (np.atleast_1d(info.status) == 0).all() and (np.atleast_1d(info.iters) == 0).all()
    assert np.abs(mu - OE.eigenvector_adjoint(rp, c, v, lam, V, gV)).max() <= 1e-12 * np.abs(mu).max()
    rp, c, v = I.diffusion2d_random(10, 2)
    lam, V = OE.smallest_eigenpairs(rp, c, v, 3)
    mu, info = _vector_adjoint(rp, c, v, lam, V, np.zeros((100, 3)))
    assert not mu.any() and (np.atleast_1d(info.iters) == 0).all() and (np.atleast_1d(info.status) == 0).all()
    gV = V @ np.random.default_rng(2).standard_normal((3, 3))
    mu, info = _vector_adjoint(rp, c, v, lam, V, gV)
    assert (np.atleast_1d(info.status) == 0).all()
    mu_o = OE.eigenvector_adjoint(rp, c, v, lam, V, gV)
    assert np.abs(mu - mu_o).max() <= 1e-10 * np.abs(mu_o).max()
    d = np.array([1.0, 2.0, 2.0, 3.0, 4.0, 5.0])
    rpd, cd = np.arange(7, dtype=np.int32), np.arange(6, dtype=np.int32)
    Vd = np.eye(6)[:, :3]
    _, info = _vector_adjoint(rpd, cd, d, d[:3], Vd, np.random.default_rng(3).standard_normal((6, 3)))
    assert list(np.atleast_1d(info.status)) == [0, 2, 2]
    _, info = _vector_adjoint(rp, c, v, lam, V, np.random.default_rng(4).standard_normal((100, 3)), max_iter=0)
    assert (np.atleast_1d(info.status) == 1).all()


def test_eigsh_eigenvector_gradient_matches_oracle_and_fd():
    """Through eigsh's autograd: L = sum glam_j lambda_j + sum gV_j^T v_j
    on the library's own pairs (sign rule: largest-magnitude entry
    positive, as the oracle's); d L / d val against the oracle's full
    gradient, and against central differences of the library's own L
    (eps = 1e-5; Tab. 5 reports 2.1e-6 for k = 6)."""
    rp, c, v = I.diffusion2d_random(16, 21)
    n, k = len(rp) - 1, 6
    A = csr(rp, c)
    rng = np.random.default_rng(22)
    glam = to_dev(rng.uniform(0.5, 1.5, k))
    gV = to_dev(rng.standard_normal((n, k)))

    def loss(vals):
        lam, V, _ = sla.eigsh(A, vals, k, tol=1e-12, max_iter=20000)
        return (glam * lam).sum() + (gV * V).sum(), V

    val = to_dev(v).requires_grad_(True)
    Lv, V = loss(val)
    Lv.backward()
    g = val.grad.cpu().numpy()
    lo, Vo = OE.smallest_eigenpairs(rp, c, v, k)
    assert np.abs(V.detach().cpu().numpy() - Vo).max() <= 1e-8
    go = OE.eigen_loss_grad(rp, c, v, k, glam.cpu().numpy(), gV.cpu().numpy())
    assert np.linalg.norm(g - go) <= 1e-7 * np.linalg.norm(go)
    eps = 1e-5
    rows = np.repeat(np.arange(n), np.diff(rp))
    errs = []
    for s in range(3):
        dd = np.random.default_rng(30 + s).standard_normal(len(v))
        D = np.zeros((n, n))
        D[rows, c] = dd
        D = 0.5 * (D + D.T)
        dv = to_dev(D[rows, c])
        with torch.no_grad():
            lp = float(loss(to_dev(v) + eps * dv)[0])
            lm = float(loss(to_dev(v) - eps * dv)[0])
        fd = (lp - lm) / (2 * eps)
        errs.append(abs(fd - float(g @ D[rows, c])) / abs(fd))
    assert max(errs) <= 1e-5, errs


def test_coo_eigsh_eigenvector_gradient_with_duplicates():
    """SparseTensor.eigsh from COO with some entries split into two
    duplicates (summed on ingest): d L / d val of each duplicate equals the
    oracle's gradient at the summed CSR entry, for L = sum gV_j^T v_j +
    sum lambda_j."""
    rp, c, v = I.diffusion2d_random(10, 41)
    n, k = len(rp) - 1, 3
    rows = np.repeat(np.arange(n), np.diff(rp))
    rng = np.random.default_rng(42)
    dup = rng.choice(len(v), 40, replace=False)
    r2 = np.concatenate([rows, rows[dup]])
    c2 = np.concatenate([c, c[dup]])
    v2 = np.concatenate([v, np.zeros(len(dup))])
    v2[dup] *= 0.5
    v2[len(v):] = v[dup] * 0.5
    src = np.concatenate([np.arange(len(v)), dup])  # CSR entry of each COO entry
    o = rng.permutation(len(v2))
    r2, c2, v2, src = r2[o], c2[o], v2[o], src[o]
    val = torch.from_numpy(v2).cuda().requires_grad_(True)
    T = sla.SparseTensor(val, torch.from_numpy(r2.astype(np.int64)).cuda(),
                         torch.from_numpy(c2.astype(np.int64)).cuda(), (n, n))
    gV = rng.standard_normal((n, k))
    # tol 1e-10 converges (70 iterations); 1e-12 is out of reach for this
    # n = 100 solve (it ends NOT_CONVERGED near 1e-8), so it is not asked for
    lam, V, _ = T.eigsh(k, tol=1e-10, max_iter=20000, strict=True)
    ((to_dev(gV) * V).sum() + lam.sum()).backward()
    go = OE.eigen_loss_grad(rp, c, v, k, np.ones(k), gV)
    assert np.abs(val.grad.cpu().numpy() - go[src]).max() <= 1e-7 * np.abs(go).max()


@pytest.mark.slow
def test_eigenvector_adjoint_at_128():
    """The bench workload (2D 128^2, sigma = 1, k = 6 pairs from eigsh at
    tol 1e-10, random dL/dV, rtol 1e-10), where the oracle's dense bordered
    solve is too large: the defining equations checked on the CPU for every
    pair -- ||(A - lambda_j I) mu_j - (I - v_j v_j^T) gV_j|| small against
    the eigen residual's share, v_j^T mu_j = 0 -- and the closed-form part
    against v_l^T gV_j / (lambda_l - lambda_j)."""
    import scipy.sparse as sp
    rp, c, v = I.diffusion2d_random(128, 11, 1.0)
    n, k = len(rp) - 1, 6
    A = csr(rp, c)
    lam, V, info = sla.eigsh(A, to_dev(v), k, tol=1e-10, max_iter=20000)
    gV = np.random.default_rng(5).standard_normal((n, k))
    mu, mi = sla.eig_vector_adjoint(A, to_dev(v), lam, V, to_dev(gV), rtol=1e-10)
    torch.cuda.synchronize()
    assert (np.atleast_1d(mi.status) == 0).all() and (np.atleast_1d(mi.true_rel_res) <= 2e-10).all()
    lam, V, mu = lam.cpu().numpy(), V.cpu().numpy(), mu.cpu().numpy()
    M = sp.csr_matrix((v, c, rp), shape=(n, n))
    for j in range(k):
        vj, gj = V[:, j], gV[:, j]
        rhs = gj - vj * (vj @ gj)
        res = M @ mu[:, j] - lam[j] * mu[:, j] - rhs
        # V is accurate to the eigensolver's 1e-10 only: its residual enters through the
        # closed-form part, so the bound is relative to ||mu_j|| ||A V - V Lambda||
        ev = np.linalg.norm(M @ V - V * lam, axis=0).max()
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(rhs) + 4 * ev * np.linalg.norm(mu[:, j]), j
        assert abs(vj @ mu[:, j]) <= 1e-9 * np.linalg.norm(mu[:, j])
        for l in range(k):
            if l != j:
                ref = (V[:, l] @ gj) / (lam[l] - lam[j])
                assert abs(V[:, l] @ mu[:, j] - ref) <= 1e-6 * max(abs(ref), np.linalg.norm(mu[:, j]) * 1e-3)
