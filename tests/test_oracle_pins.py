"""Pins for the CPU oracle: each test ties an oracle routine to something other
than itself -- dense LU, the closed-form Poisson eigenpairs, brute force on
tiny inputs, central finite differences, an independent library, or the
paper's own naive-vs-adjoint agreement (Sec. 4.2, App. D)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2601_13994_b300 import inputs as I


def dense(rp, c, v, n=None):
    n = len(rp) - 1 if n is None else n
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, c[k]] += v[k]
    return A


def rand_csr(n, seed, density=0.3, empty_rows=(), intvals=False):
    rng = np.random.default_rng(seed)
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        if i in empty_rows:
            rp.append(rp[-1])
            continue
        m = rng.random(n) < density
        c = np.nonzero(m)[0]
        v = rng.integers(-5, 6, size=c.size).astype(float) if intvals else rng.uniform(-1, 1, c.size)
        cols.append(c)
        vals.append(v)
        rp.append(rp[-1] + c.size)
    return (np.array(rp, np.int32), np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32),
            np.concatenate(vals) if vals else np.zeros(0))


# ---------------------------------------------------------------- SpMV

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_spmv_brute_force(seed):
    rp, c, v = rand_csr(37, seed, empty_rows={0, 5, 36})
    x = np.random.default_rng(seed + 10).uniform(-1, 1, 37)
    y = oracle.spmv(rp, c, v, x)
    yd = dense(rp, c, v) @ x
    assert np.allclose(y, yd, rtol=1e-14, atol=1e-14)
    assert y[0] == 0.0 and y[5] == 0.0 and y[36] == 0.0


def test_spmv_integer_exact():
    rp, c, v = rand_csr(50, 7, intvals=True)
    x = np.random.default_rng(3).integers(-9, 10, 50).astype(float)
    y = oracle.spmv(rp, c, v, x)
    assert np.array_equal(y, dense(rp, c, v) @ x)


def test_diag_matches_dense():
    rp, c, v = rand_csr(20, 4, density=0.5)
    assert np.array_equal(oracle.diag(rp, c, v), np.diag(dense(rp, c, v)))


# ---------------------------------------------------------------- generators vs closed forms

def test_poisson2d_eigenvalues_closed_form():
    N = 8
    A = dense(*I.poisson2d(N))
    ev = np.sort(np.linalg.eigvalsh(A))
    j = np.arange(1, N + 1)
    mu1 = 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2
    cf = np.sort((mu1[:, None] + mu1[None, :]).ravel())
    assert np.allclose(ev, cf, rtol=0, atol=1e-12)


def test_generators_symmetric_positive_definite():
    for rp, c, v in [I.diffusion2d_random(9, 3), I.diffusion3d_random(5, 4), I.fem_p1_laplacian(12, 6)]:
        A = dense(rp, c, v)
        assert np.array_equal(A, A.T)
        np.linalg.cholesky(A)
        # column indices ascending and distinct within rows
        for i in range(len(rp) - 1):
            assert np.all(np.diff(c[rp[i]:rp[i + 1]]) > 0)


def test_nnz_formulas():
    for N in (3, 8, 17):
        assert I.poisson2d(N)[0][-1] == I.nnz_2d(N)
        assert I.diffusion3d_random(N, 0)[0][-1] == I.nnz_3d(N)
        assert I.convdiff3d(N)[0][-1] == I.nnz_3d(N)


# ---------------------------------------------------------------- PCG

def test_pcg_vs_dense_lu_poisson64():
    rp, c, v = I.poisson2d(64)
    b = I.rhs_uniform(4096, 0)
    x, info = oracle.pcg(rp, c, v, b, rtol=1e-10)
    xs = sp.linalg.spsolve(sp.csr_matrix((v, c, rp)).tocsc(), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    assert info["true_rel_res"] <= 2e-10


@pytest.mark.parametrize("jk", [(1, 1), (3, 5), (8, 2)])
def test_pcg_poisson_eigenvector_closed_form(jk):
    N = 24
    j, k = jk
    rp, c, v = I.poisson2d(N)
    p = np.arange(1, N + 1)
    vec = np.outer(np.sin(k * np.pi * p / (N + 1)), np.sin(j * np.pi * p / (N + 1))).ravel()
    mu = 4 * math.sin(j * math.pi / (2 * (N + 1))) ** 2 + 4 * math.sin(k * math.pi / (2 * (N + 1))) ** 2
    x, info = oracle.pcg(rp, c, v, vec, rtol=1e-13)
    assert info["status"] == 0
    assert np.allclose(x, vec / mu, rtol=0, atol=1e-12 * np.abs(vec / mu).max())
    # an eigenvector is solved by (P)CG in exactly one step
    assert info["iters"] == 1


def test_jacobi_pcg_equals_cg_for_constant_diagonal():
    rp, c, v = I.poisson2d(20)
    b = I.rhs_uniform(400, 1)
    x1, i1 = oracle.pcg(rp, c, v, b, rtol=1e-10, precond="jacobi")
    x0, i0 = oracle.pcg(rp, c, v, b, rtol=1e-10, precond="none")
    assert abs(i1["iters"] - i0["iters"]) <= 1
    assert np.allclose(x1, x0, rtol=0, atol=1e-9 * np.abs(x0).max())


def test_pcg_3d_variable_coefficient_vs_lu():
    rp, c, v = I.diffusion3d_random(10, 1)
    b = I.rhs_uniform(1000, 2)
    x, info = oracle.pcg(rp, c, v, b, rtol=1e-12)
    xs = np.linalg.solve(dense(rp, c, v), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9


def test_pcg_edge_cases():
    rp, c, v = I.poisson2d(6)
    n = 36
    x, info = oracle.pcg(rp, c, v, np.zeros(n))
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    # negative diagonal -> NOT_SPD before iterating
    v2 = v.copy()
    v2[rp[3]:rp[4]][c[rp[3]:rp[4]] == 3] = -1.0
    _, info = oracle.pcg(rp, c, v2, np.ones(n))
    assert info["status_name"] == "NOT_SPD"
    # indefinite with positive diagonal -> p^T A p <= 0
    rpi = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    vi = np.array([1.0, 2.0, 2.0, 1.0])
    _, info = oracle.pcg(rpi, ci, vi, np.array([1.0, -1.0]))
    assert info["status_name"] == "NOT_SPD"
    # iteration cap
    b = I.rhs_uniform(n, 0)
    _, info = oracle.pcg(rp, c, v, b, rtol=1e-14, max_iter=2)
    assert info["status_name"] == "NOT_CONVERGED" and info["iters"] == 2
    # NaN in b
    bn = b.copy()
    bn[4] = np.nan
    _, info = oracle.pcg(rp, c, v, bn)
    assert info["status_name"] == "BREAKDOWN"
    # warm start from the exact solution converges immediately
    xs = np.linalg.solve(dense(rp, c, v), b)
    _, info = oracle.pcg(rp, c, v, b, x0=xs, rtol=1e-10)
    assert info["status"] == 0 and info["iters"] <= 1


def test_pcg_ggt_special_cases():
    rp, c, v = I.diffusion2d_random(5, 9)
    n = 25
    A = dense(rp, c, v)
    b = I.rhs_uniform(n, 5)
    # G = D^{-1/2} reproduces Jacobi-PCG
    d = np.diag(A)
    G1 = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), 1 / np.sqrt(d))
    xg, ig = oracle.pcg(rp, c, v, b, rtol=1e-12, precond="ggt", G=G1)
    xj, ij = oracle.pcg(rp, c, v, b, rtol=1e-12, precond="jacobi")
    assert ig["iters"] == ij["iters"]
    assert np.allclose(xg, xj, rtol=0, atol=1e-12 * np.abs(xj).max())
    # lower-triangular G with G G^T = A^{-1} (full tril pattern): one iteration
    Linv = np.linalg.inv(np.linalg.cholesky(A))   # A = L L^T -> A^{-1} = L^{-T} L^{-1}
    Gd = np.linalg.cholesky(np.linalg.inv(A))     # lower, Gd Gd^T = A^{-1}
    Gs = sp.csr_matrix(np.tril(Gd))
    assert Linv is not None
    xg, ig = oracle.pcg(rp, c, v, b, rtol=1e-10, precond="ggt",
                        G=(Gs.indptr.astype(np.int32), Gs.indices.astype(np.int32), Gs.data))
    assert ig["status"] == 0 and ig["iters"] == 1


# ---------------------------------------------------------------- pipelined PCG

def _krylov_minimiser(A, b, dinv, k):
    """Independent statement of what the k-th PCG iterate is (x0 = 0): the
    minimiser of the A-norm error over the preconditioned Krylov space
    span{M^-1 b, (M^-1 A) M^-1 b, ...} of dimension k, from an orthonormal
    basis of that space and the k x k Galerkin system."""
    v = dinv * b
    cols = []
    for _ in range(k):
        cols.append(v / np.linalg.norm(v))
        v = dinv * (A @ cols[-1])
    V, _ = np.linalg.qr(np.stack(cols, axis=1))
    y = np.linalg.solve(V.T @ A @ V, V.T @ b)
    return V @ y


@pytest.mark.parametrize("fn", ["pcg", "pcg_pipelined"])
@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_pcg_iterates_are_krylov_minimisers(fn, precond):
    rp, c, v = I.diffusion2d_random(6, 3)
    n = 36
    A = dense(rp, c, v)
    b = I.rhs_uniform(n, 11)
    dinv = 1.0 / np.diag(A) if precond == "jacobi" else np.ones(n)
    for k in range(1, 8):
        x, info = getattr(oracle, fn)(rp, c, v, b, rtol=0.0, max_iter=k, precond=precond)
        assert info["iters"] == k and info["status_name"] == "NOT_CONVERGED"
        xk = _krylov_minimiser(A, b, dinv, k)
        assert np.linalg.norm(x - xk) <= 1e-9 * np.linalg.norm(xk), (fn, k)


def test_pipelined_finite_termination_and_eigenvector():
    rng = np.random.default_rng(5)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 9.0, n)) @ Q.T
    As = sp.csr_matrix(A)
    rp, c, v = As.indptr.astype(np.int32), As.indices.astype(np.int32), As.data
    b = rng.uniform(-1, 1, n)
    x, info = oracle.pcg_pipelined(rp, c, v, b, rtol=0.0, max_iter=n, precond="none")
    xs = np.linalg.solve(A, b)
    assert info["iters"] == n
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    # a Poisson eigenvector (constant diagonal 4, so also one of D^-1 A) takes one step
    N = 16
    rp, c, v = I.poisson2d(N)
    p = np.arange(1, N + 1)
    vec = np.outer(np.sin(3 * np.pi * p / (N + 1)), np.sin(2 * np.pi * p / (N + 1))).ravel()
    mu = 4 * math.sin(2 * math.pi / (2 * (N + 1))) ** 2 + 4 * math.sin(3 * math.pi / (2 * (N + 1))) ** 2
    x, info = oracle.pcg_pipelined(rp, c, v, vec, rtol=1e-13)
    assert info["status"] == 0 and info["iters"] == 1
    assert np.allclose(x, vec / mu, rtol=0, atol=1e-12 * np.abs(vec / mu).max())


def test_pipelined_vs_sparse_lu_poisson64():
    rp, c, v = I.poisson2d(64)
    b = I.rhs_uniform(4096, 0)
    x, info = oracle.pcg_pipelined(rp, c, v, b, rtol=1e-10)
    xs = sp.linalg.spsolve(sp.csr_matrix((v, c, rp)).tocsc(), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    assert info["true_rel_res"] <= 2e-10
    _, ref = oracle.pcg(rp, c, v, b, rtol=1e-10)
    assert abs(info["iters"] - ref["iters"]) <= 2


def test_pipelined_edge_cases():
    rp, c, v = I.poisson2d(6)
    n = 36
    x, info = oracle.pcg_pipelined(rp, c, v, np.zeros(n))
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    v2 = v.copy()
    v2[rp[3]:rp[4]][c[rp[3]:rp[4]] == 3] = -1.0
    _, info = oracle.pcg_pipelined(rp, c, v2, np.ones(n))
    assert info["status_name"] == "NOT_SPD" and info["iters"] == 0
    # [[1,2],[2,1]], b = (1,-1): u = b, w = A u = (-1,1), p^T A p = (w,u) = -2
    rpi = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    vi = np.array([1.0, 2.0, 2.0, 1.0])
    _, info = oracle.pcg_pipelined(rpi, ci, vi, np.array([1.0, -1.0]))
    assert info["status_name"] == "NOT_SPD" and info["iters"] == 0
    b = I.rhs_uniform(n, 0)
    _, info = oracle.pcg_pipelined(rp, c, v, b, rtol=1e-14, max_iter=2)
    assert info["status_name"] == "NOT_CONVERGED" and info["iters"] == 2
    _, info = oracle.pcg_pipelined(rp, c, v, b, max_iter=0)
    assert info["status_name"] == "NOT_CONVERGED" and info["iters"] == 0
    bn = b.copy()
    bn[4] = np.nan
    _, info = oracle.pcg_pipelined(rp, c, v, bn)
    assert info["status_name"] == "BREAKDOWN"
    xs = np.linalg.solve(dense(rp, c, v), b)
    _, info = oracle.pcg_pipelined(rp, c, v, b, x0=xs, rtol=1e-10)
    assert info["status"] == 0 and info["iters"] <= 1
    with pytest.raises(ValueError):
        oracle.pcg_pipelined(rp, c, v, b, precond="ggt")
    # below the recurrences' attainable accuracy: the late p^T A p <= 0 is
    # rounding (A is SPD), so the true-residual check and restarts take over
    rp, c, v = I.poisson2d(30)
    b = I.rhs_uniform(900, 4)
    _, info = oracle.pcg_pipelined(rp, c, v, b, rtol=1e-15, max_restarts=0)
    assert info["status_name"] == "NOT_CONVERGED" and info["true_rel_res"] <= 1e-10
    _, info = oracle.pcg_pipelined(rp, c, v, b, rtol=1e-15, max_restarts=3)
    assert info["status_name"] == "OK" and info["true_rel_res"] <= 2e-15


def test_cg_fixed_matches_naive_torch_loop():
    torch = pytest.importorskip("torch")
    rp, c, v = I.poisson2d(10)
    b = I.rhs_uniform(100, 2)
    k = 17
    x = oracle.cg_fixed(rp, c, v, b, k)
    A = torch.tensor(dense(rp, c, v))
    bt = torch.tensor(b)
    xt = torch.zeros(100, dtype=torch.float64)
    r = bt.clone(); p = r.clone(); rho = r @ r
    for _ in range(k):
        q = A @ p
        a = rho / (p @ q)
        xt = xt + a * p
        r = r - a * q
        rn = r @ r
        p = r + (rn / rho) * p
        rho = rn
    assert np.allclose(x, xt.numpy(), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- BiCGStab

@pytest.mark.parametrize("N,pe", [(8, 10.0), (12, 1.0), (6, 0.0)])
def test_bicgstab_vs_dense_lu(N, pe):
    rp, c, v = I.convdiff3d(N, pe)
    n = N ** 3
    b = I.rhs_uniform(n, N)
    x, info = oracle.bicgstab(rp, c, v, b, rtol=1e-12)
    xs = np.linalg.solve(dense(rp, c, v), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    assert info["true_rel_res"] <= 2e-12


def test_bicgstab_edge_cases():
    rp, c, v = I.convdiff3d(4)
    n = 64
    x, info = oracle.bicgstab(rp, c, v, np.zeros(n))
    assert info["status"] == 0 and info["iters"] == 0 and not x.any()
    v0 = v.copy()
    v0[(c == 0) & (np.arange(len(c)) < rp[1])] = 0.0  # A_00 = 0 with Jacobi
    _, info = oracle.bicgstab(rp, c, v0, np.ones(n))
    assert info["status_name"] == "INVALID"
    b = I.rhs_uniform(n, 1)
    _, info = oracle.bicgstab(rp, c, v, b, rtol=1e-15, max_iter=1)
    assert info["status_name"] == "NOT_CONVERGED"
    bn = b.copy(); bn[0] = np.inf
    _, info = oracle.bicgstab(rp, c, v, bn)
    assert info["status_name"] == "BREAKDOWN"


def test_bicgstab_symmetric_agrees_with_pcg():
    rp, c, v = I.diffusion2d_random(12, 3)
    b = I.rhs_uniform(144, 4)
    x1, _ = oracle.bicgstab(rp, c, v, b, rtol=1e-12)
    x2, _ = oracle.pcg(rp, c, v, b, rtol=1e-12)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-9


# ---------------------------------------------------------------- pattern utilities

@pytest.mark.parametrize("seed", [0, 1])
def test_transpose_vs_dense_and_scipy(seed):
    rp, c, v = rand_csr(31, seed, density=0.2, empty_rows={3, 4})
    rpT, cT, pT = oracle.transpose(rp, c)
    vT = v[pT]
    assert np.array_equal(dense(rpT, cT, vT), dense(rp, c, v).T)
    S = sp.csr_matrix((v, c, rp), shape=(31, 31)).T.tocsr()
    S.sort_indices()
    assert np.array_equal(rpT, S.indptr) and np.array_equal(cT, S.indices) and np.array_equal(vT, S.data)
    # stable: inside a row of A^T the source slots increase
    for j in range(31):
        assert np.all(np.diff(pT[rpT[j]:rpT[j + 1]]) > 0)


def test_coo_to_csr_duplicates_and_perm():
    rng = np.random.default_rng(11)
    n, m = 23, 300
    row = rng.integers(0, n, m)
    col = rng.integers(0, n, m)
    val = rng.uniform(-1, 1, m)
    rp, c, v, perm = oracle.coo_to_csr(n, row, col, val)
    D = np.zeros((n, n))
    np.add.at(D, (row, col), val)
    assert np.allclose(dense(rp, c, v, n), D, rtol=0, atol=1e-14)
    # every COO entry maps to the CSR slot holding its (row, col)
    rows_csr = np.repeat(np.arange(n), np.diff(rp))
    assert np.array_equal(rows_csr[perm], row) and np.array_equal(c[perm], col)
    for i in range(n):
        assert np.all(np.diff(c[rp[i]:rp[i + 1]]) > 0)
    assert len(c) == len(set(zip(row.tolist(), col.tolist())))


# ---------------------------------------------------------------- adjoint (Eq. 3)

def test_adjoint_closed_form_poisson_eigenvector():
    N = 16
    j, k = 2, 3
    rp, c, v = I.poisson2d(N)
    p = np.arange(1, N + 1)
    vec = np.outer(np.sin(k * np.pi * p / (N + 1)), np.sin(j * np.pi * p / (N + 1))).ravel()
    mu = 4 * math.sin(j * math.pi / (2 * (N + 1))) ** 2 + 4 * math.sin(k * math.pi / (2 * (N + 1))) ** 2
    x, _ = oracle.pcg(rp, c, v, vec, rtol=1e-14)
    g = 2 * x                                   # L = sum x^2
    gb, gv, info = oracle.adjoint_backward(rp, c, v, x, g, rtol=1e-14)
    assert info["status"] == 0
    assert np.allclose(gb, 2 * vec / mu ** 2, rtol=0, atol=1e-12 * np.abs(vec).max() / mu ** 2)
    rows = np.repeat(np.arange(N * N), np.diff(rp))
    ref = -2 * vec[rows] * vec[c] / mu ** 3
    assert np.allclose(gv, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("kind", ["spd", "nonsym"])
def test_adjoint_vs_dense_formula(kind):
    if kind == "spd":
        rp, c, v = I.diffusion2d_random(7, 2)
        method = "cg"
    else:
        rp, c, v = I.convdiff3d(4, 3.0)
        method = "bicgstab"
    n = len(rp) - 1
    A = dense(rp, c, v)
    b = I.rhs_uniform(n, 9)
    g = I.rhs_uniform(n, 10)
    x = np.linalg.solve(A, b)
    gb, gv, info = oracle.adjoint_backward(rp, c, v, x, g, method=method, rtol=1e-14)
    lam = np.linalg.solve(A.T, g)                # A^T lambda = g
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.allclose(gb, lam, rtol=0, atol=1e-11 * np.abs(lam).max())
    assert np.allclose(gv, -lam[rows] * x[c], rtol=0, atol=1e-11 * np.abs(lam).max() * np.abs(x).max())
    if kind == "nonsym":
        # the transposed operand matters: A lambda = g gives a different answer
        lam_wrong = np.linalg.solve(A, g)
        assert np.abs(lam_wrong - lam).max() > 1e-3 * np.abs(lam).max()


@pytest.mark.parametrize("kind", ["spd", "nonsym"])
def test_adjoint_central_finite_differences(kind):
    """Central FD with eps = 1e-5 on random entries of A and b (Sec. 4.3),
    with the perturbed solves done by dense LU so that solver error does not
    enter the difference quotient."""
    if kind == "spd":
        rp, c, v = I.diffusion2d_random(6, 5)
        method = "cg"
    else:
        rp, c, v = I.convdiff3d(3, 2.0)
        method = "bicgstab"
    n = len(rp) - 1
    b = I.rhs_uniform(n, 21)
    w = I.rhs_uniform(n, 22)

    def loss(vv, bb):
        x = np.linalg.solve(dense(rp, c, vv), bb)
        return float(np.sum(w * x * x)), x

    L0, x = loss(v, b)
    g = 2 * w * x
    gb, gv, _ = oracle.adjoint_backward(rp, c, v, x, g, method=method, rtol=1e-14)
    eps = 1e-5
    rng = np.random.default_rng(0)
    for k in rng.choice(len(v), 12, replace=False):
        vp = v.copy(); vp[k] += eps
        vm = v.copy(); vm[k] -= eps
        fd = (loss(vp, b)[0] - loss(vm, b)[0]) / (2 * eps)
        assert abs(fd - gv[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gv[k])
    for i in rng.choice(n, 8, replace=False):
        bp = b.copy(); bp[i] += eps
        bm = b.copy(); bm[i] -= eps
        fd = (loss(v, bp)[0] - loss(v, bm)[0]) / (2 * eps)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(fd))


def _load_paper_e4():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_adjoint_vs_naive.txt")
    out = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, val = line.split("=")
            out[k.strip()] = float(val)
    return out


def test_adjoint_agrees_with_naive_autograd_through_cg():
    """Sec. 4.2 / App. D: naive autograd through k CG iterations (scatter
    SpMV, val * x[col] then index_add) vs the adjoint gradient after full
    convergence.  The paper reports loss agreement 1.96e-16 and dL/db
    agreement 2.6e-14 at N = 4096; here a 16 x 16 grid is used."""
    torch = pytest.importorskip("torch")
    paper = _load_paper_e4()
    N = 16
    n = N * N
    rp, c, v = I.poisson2d(N)
    b = I.rhs_uniform(n, 3)
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(rp)))
    cols = torch.tensor(c.astype(np.int64))
    vt = torch.tensor(v, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)

    def mv(x):
        return torch.zeros(n, dtype=torch.float64).index_add(0, rows, vt * x[cols])

    x = torch.zeros(n, dtype=torch.float64)
    r = bt.clone(); p = r.clone(); rho = r @ r
    for _ in range(400):
        if float(rho.detach().sqrt()) <= 1e-13 * float(bt.detach().norm()):
            break
        q = mv(p)
        a = rho / (p @ q)
        x = x + a * p
        r = r - a * q
        rn = r @ r
        p = r + (rn / rho) * p
        rho = rn
    Ln = (x * x).sum()
    Ln.backward()
    xo, _ = oracle.pcg(rp, c, v, b, rtol=1e-14)
    Lo = float((xo * xo).sum())
    gb, gv, _ = oracle.adjoint_backward(rp, c, v, xo, 2 * xo, rtol=1e-14)
    assert abs(Lo - float(Ln)) / abs(Lo) <= 100 * paper["loss_rel_err"]
    assert np.linalg.norm(gb - bt.grad.numpy()) / np.linalg.norm(gb) <= 100 * paper["grad_b_rel_err"]
    # the matrix-gradient gap is round-off of the naive recurrence (App. D
    # explains the paper's 6.8e-4 the same way); it bounds the naive path, so
    # only its order of magnitude is checked here
    assert np.linalg.norm(gv - vt.grad.numpy()) / np.linalg.norm(gv) <= 10 * paper["grad_A_rel_err"]


# ---------------------------------------------------------------- learned factor (MPNN) oracle

def test_mpnn_zero_head_is_jacobi_factor():
    from oracle import mpnn
    rp, c, v = I.diffusion2d_random(9, 1)
    P = mpnn.init_params(0, zero_head=True)
    grp, gcol, gv = mpnn.forward(P, rp, c, v)
    n = len(rp) - 1
    d = np.diag(dense(rp, c, v))
    G = dense(grp, gcol, gv.numpy(), n)
    assert np.allclose(G, np.diag(1 / np.sqrt(d)), rtol=0, atol=1e-15)
    # and the factor has exactly the pattern of tril(A)
    A = dense(rp, c, v)
    assert np.array_equal(dense(grp, gcol, np.ones(len(gcol)), n) != 0, np.tril(A) != 0)


def test_mpnn_loss_zero_for_exact_factor_and_gradcheck():
    import torch
    from oracle import mpnn
    rp, c, v = I.diffusion2d_random(4, 2)
    n = len(rp) - 1
    A = dense(rp, c, v)
    b = np.random.default_rng(0).standard_normal(n)
    xs = np.linalg.solve(A, b)
    # full lower factor with G G^T = A^{-1}: loss 0
    Gd = np.linalg.cholesky(np.linalg.inv(A))
    rpf = np.array([0] + list(np.cumsum(np.arange(1, n + 1))), np.int32)
    cf = np.concatenate([np.arange(i + 1) for i in range(n)]).astype(np.int32)
    gvf = torch.tensor(np.concatenate([Gd[i, :i + 1] for i in range(n)]))
    assert float(mpnn.loss(rpf, cf, gvf, rp, c, v, b, xs)) < 1e-24
    # autograd of the oracle's forward + loss against central differences
    P = mpnn.init_params(3, zero_head=False)

    def f(*flat):
        d = dict(zip(P.keys(), flat))
        grp, gcol, gv = mpnn.forward(d, rp, c, v)
        return mpnn.loss(grp, gcol, gv, rp, c, v, b, xs)

    ts = tuple(torch.tensor(P[k] * 0.5, requires_grad=True) for k in P)
    assert torch.autograd.gradcheck(f, ts, eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)


def test_mpnn_scale_free_loss_is_the_minimum_over_scales():
    """The scale-free training loss is min over k of the A-norm error of
    x* - k G G^T b: pinned by the plain loss, which is a quadratic in k
    (three evaluations with G scaled by sqrt(k) give its exact minimum), by
    invariance under G -> a G, by a loss of 0 for an exact factor times any
    scale, by 1 for G = 0, and by autograd's gradient (through k) against
    central differences."""
    import torch
    from oracle import mpnn
    rp, c, v = I.diffusion2d_random(5, 4, 1.2)
    n = len(rp) - 1
    A = dense(rp, c, v)
    b = np.random.default_rng(3).standard_normal(n)
    xs = np.linalg.solve(A, b)
    P = mpnn.init_params(5, zero_head=False)
    grp, gcol, gv = mpnn.forward({k: torch.tensor(t * 0.5) for k, t in P.items()}, rp, c, v)
    gv = gv.detach()
    L = lambda g, sf=False: float(mpnn.loss(grp, gcol, g, rp, c, v, b, xs, scale_free=sf))
    # plain loss at scales k = 0, 1, 4 of G G^T: q(k) = a k^2 + b1 k + q0
    q0, q1, q4 = L(gv * 0.0), L(gv), L(gv * 2.0)
    a = (q4 - 4 * q1 + 3 * q0) / 12.0
    b1 = q1 - q0 - a
    kmin = -b1 / (2 * a)
    lmin = q0 - b1 * b1 / (4 * a)
    Lsf = L(gv, True)
    assert a > 0 and abs(q0 - 1.0) <= 1e-14
    assert abs(Lsf - lmin) <= 1e-12 and Lsf <= q1 + 1e-15
    assert abs(L(gv * math.sqrt(kmin)) - lmin) <= 1e-12
    for s_ in (0.37, 3.0, -1.5):
        assert abs(L(gv * s_, True) - Lsf) <= 1e-12
    assert L(gv * 0.0, True) == 1.0
    # an exact factor (G G^T = A^-1) times any scale: loss 0
    Gd = np.linalg.cholesky(np.linalg.inv(A))
    rpf = np.array([0] + list(np.cumsum(np.arange(1, n + 1))), np.int32)
    cf = np.concatenate([np.arange(i + 1) for i in range(n)]).astype(np.int32)
    gvf = torch.tensor(np.concatenate([Gd[i, :i + 1] for i in range(n)]) * 1.7)
    assert float(mpnn.loss(rpf, cf, gvf, rp, c, v, b, xs, scale_free=True)) < 1e-24
    assert float(mpnn.loss(rpf, cf, gvf, rp, c, v, b, xs)) > 1.0
    # gradient w.r.t. G's values through k, against central differences
    g0 = gv.clone().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda g: mpnn.loss(grp, gcol, g, rp, c, v, b, xs, scale_free=True), (g0,),
                                     eps=1e-6, atol=1e-7, rtol=1e-5)


def test_column_normalize_torch_form_matches_loops_and_gradcheck():
    """The differentiable normalisation (for the gradient of training through
    it) equals the loop form value for value, gives diag(G^T A G) = I, and
    its autograd gradient matches central differences."""
    import torch
    from oracle import mpnn
    rp, c, v = I.diffusion2d_random(5, 9, 1.3)
    n = len(rp) - 1
    P = mpnn.init_params(6, zero_head=False)
    grp, gcol, gv = mpnn.forward({k: torch.tensor(t * 0.5) for k, t in P.items()}, rp, c, v)
    gv = gv.detach()
    ref = mpnn.column_normalize(grp, gcol, gv.numpy(), rp, c, v)
    got = mpnn.column_normalize_t(grp, gcol, gv, rp, c, v).numpy()
    assert np.allclose(got, ref, rtol=1e-14, atol=0)
    Gn = dense(grp, gcol, got, n)
    A = dense(rp, c, v)
    assert np.allclose(np.diag(Gn.T @ A @ Gn), 1.0, rtol=1e-13)
    g0 = gv.clone().requires_grad_(True)
    w = torch.tensor(np.random.default_rng(2).standard_normal(len(gcol)))
    assert torch.autograd.gradcheck(lambda g: (mpnn.column_normalize_t(grp, gcol, g, rp, c, v) * w).sum(), (g0,),
                                     eps=1e-6, atol=1e-7, rtol=1e-5)


def _mpnn_path3_case():
    """A 3-node path graph and hand-chosen weights for which every step of the
    network can be followed on paper (the design: scaled entries, three node
    features, an input layer, three residual message-passing layers, the head
    on tril(A), G = D^{-1/2} Gt)."""
    # A = [[4, -2, 0], [-2, 4, -1], [0, -1, 4]]: d = 4 everywhere, so
    # e_01 = e_10 = -2/4 = -0.5 and e_12 = e_21 = -1/4 = -0.25
    rp = np.array([0, 2, 5, 7], np.int32)
    c = np.array([0, 1, 0, 1, 2, 1, 2], np.int32)
    v = np.array([4.0, -2.0, -2.0, 4.0, -1.0, -1.0, 4.0])
    from oracle import mpnn
    P = {k: np.zeros(s) for k, s in mpnn.param_shapes().items()}
    W = mpnn.WIDTH
    # input layer: h0 = relu(sum|e|), h1 = relu(sum e + 1), h2 = relu(deg/8)
    P["W0"][0, 0] = 1.0
    P["W0"][1, 1] = 1.0
    P["b0"][1] = 1.0
    P["W0"][2, 2] = 1.0
    # layer 0: h3 += relu(-agg(h0)); layer 1: h4 += relu(-agg(h3));
    # layer 2: h5 += relu(h1 + agg(h4) - 0.3)   (agg_i = sum_{j != i} e_ij h_j)
    P["W_0"][3, W + 0] = -1.0
    P["W_1"][4, W + 3] = -1.0
    P["W_2"][5, 1] = 1.0
    P["W_2"][5, W + 4] = 1.0
    P["c_2"][5] = -0.3
    # head: P0 = h5, Q0 = h3, ue0 = -1, v0 = 1; Q1 = h0 + 0.1, v1 = -2;
    # R0 = h4 - 0.1, vd0 = 1
    P["Uh"][0, 5] = 1.0
    P["Uh"][W + 0, 3] = 1.0
    P["ue"][0] = -1.0
    P["v"][0] = 1.0
    P["Uh"][W + 1, 0] = 1.0
    P["bh"][W + 1] = 0.1
    P["v"][1] = -2.0
    P["Uh"][2 * W + 0, 4] = 1.0
    P["bh"][2 * W + 0] = -0.1
    P["vd"][0] = 1.0
    return rp, c, v, P


def test_mpnn_forward_hand_worked_path3():
    """The oracle's forward against values worked out by hand.

    Features (sum|e|, sum e, deg/8): node 0 (0.5, -0.5, 1/8), node 1
    (0.75, -0.75, 2/8), node 2 (0.25, -0.25, 1/8), so
    h0 = (0.5, 0.75, 0.25), h1 = (0.5, 0.25, 0.75).
    Layer 0, agg(h0) with messages from the neighbour j:
      node 0: e_01 h0_1 = -0.5 * 0.75 = -0.375
      node 1: e_10 h0_0 + e_12 h0_2 = -0.25 - 0.0625 = -0.3125
      node 2: e_21 h0_1 = -0.25 * 0.75 = -0.1875      -> h3 = (0.375, 0.3125, 0.1875)
    Layer 1, agg(h3): -0.15625, -0.1875 - 0.046875, -0.078125
                                                     -> h4 = (0.15625, 0.234375, 0.078125)
    Layer 2, agg(h4): -0.1171875, -0.078125 - 0.01953125, -0.05859375
      h5 = relu(h1 + agg - 0.3) = (0.0828125, 0, 0.39140625)
    Head, entry (1, 0): relu(h5_1 + h3_0 + 0.5) = 0.875, relu(h0_0 + 0.1) = 0.6,
      theta = 0.875 - 2 * 0.6 = -0.325
    entry (2, 1): relu(h5_2 + h3_1 + 0.25) = 0.95390625, relu(h0_1 + 0.1) = 0.85,
      theta = 0.95390625 - 1.7 = -0.74609375
    diagonal: theta_ii = relu(h4_i - 0.1) = (0.05625, 0.134375, 0)
    G = D^{-1/2} Gt with D^{-1/2} = 1/2, CSR order (0,0) (1,0) (1,1) (2,1) (2,2).

    A message taken from the row's own node instead of the neighbour, the
    two sums of the features swapped, or the e_ij term of the head dropped
    each changes at least one of these values by more than 0.01."""
    from oracle import mpnn
    rp, c, v, P = _mpnn_path3_case()
    grp, gcol, gv = mpnn.forward(P, rp, c, v)
    assert grp.tolist() == [0, 1, 3, 5]
    assert gcol.tolist() == [0, 0, 1, 1, 2]
    want = np.array([0.5 * math.exp(0.05625), 0.5 * -0.325, 0.5 * math.exp(0.134375),
                     0.5 * -0.74609375, 0.5 * math.exp(0.0)])
    assert np.allclose(gv.numpy(), want, rtol=1e-14, atol=1e-15)


def test_mpnn_permutation_equivariance():
    from oracle import mpnn
    rp, c, v = I.diffusion2d_random(5, 3)
    n = len(rp) - 1
    A = dense(rp, c, v)
    P = mpnn.init_params(4, zero_head=False)
    grp, gcol, gv = mpnn.forward(P, rp, c, v)
    G = dense(grp, gcol, gv.numpy(), n)
    # reverse the order of the unknowns: tril <-> triu, so compare the symmetric part of the
    # message-passing embedding through the diagonal of G, which is order independent
    perm = np.random.default_rng(1).permutation(n)
    Ap = A[np.ix_(perm, perm)]
    S = sp.csr_matrix(Ap)
    S.sort_indices()
    grp2, gcol2, gv2 = mpnn.forward(P, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data)
    G2 = dense(grp2, gcol2, gv2.numpy(), n)
    assert np.allclose(np.diag(G2), np.diag(G)[perm], rtol=1e-12, atol=0)


def _fsai_factor(rp, c, v):
    from oracle import mpnn
    return mpnn.fsai_factor(rp, c, v)


def test_fsai_factor_is_exact_on_a_full_pattern():
    """With every entry of A stored, the pattern of tril(A) is the full
    lower triangle, and the FSAI factor is exact: G G^T = A^{-1}; on a
    sparse pattern it has unit columns in the A-norm, diag(G^T A G) = I."""
    rng = np.random.default_rng(3)
    n = 9
    X = rng.standard_normal((n, n))
    A = X @ X.T + n * np.eye(n)
    S = sp.csr_matrix(A)
    S.sort_indices()
    G = _fsai_factor(S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data)
    assert np.allclose(np.tril(G), G, atol=0)
    assert np.allclose(G @ G.T @ A, np.eye(n), rtol=0, atol=1e-12)
    rp, c, v = I.diffusion2d_random(6, 4)
    Gs = _fsai_factor(rp, c, v)
    Ad = dense(rp, c, v)
    assert np.allclose(np.diag(Gs.T @ Ad @ Gs), 1.0, rtol=0, atol=1e-13)
    assert np.array_equal(Gs != 0, np.tril(Ad) != 0)


def _csr_of(G):
    S = sp.csr_matrix(G)
    S.sort_indices()
    return S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.copy()


def _kaporin(M):
    n = M.shape[0]
    sign, logdet = np.linalg.slogdet(M)
    assert sign > 0
    return n * np.log(np.trace(M) / n) - logdet


@pytest.mark.parametrize("mat", ["var2d", "var3d", "fem"])
def test_column_normalize_invariants(mat):
    """The normalised factor has diag(G^T A G) = I (checked with dense
    products); positive column scalings of G do not change it; FSAI factors
    (already normalised by construction) and the Jacobi factor D^{-1/2} are
    fixed points; and Kaporin's condition number does not increase."""
    from oracle import mpnn
    rp, c, v = {"var2d": lambda: I.diffusion2d_random(7, 4, 1.5), "var3d": lambda: I.diffusion3d_random(4, 5),
                "fem": lambda: I.fem_p1_laplacian(6, 6)}[mat]()
    n = len(rp) - 1
    A = dense(rp, c, v)
    rng = np.random.default_rng(7)
    # a random factor on the pattern of tril(A), positive diagonal
    L = np.tril(A != 0) * rng.uniform(-0.4, 0.4, (n, n))
    L[np.diag_indices(n)] = rng.uniform(0.2, 2.0, n)
    grp, gcol, gv = _csr_of(L)
    g1 = mpnn.column_normalize(grp, gcol, gv, rp, c, v)
    G1 = dense(grp, gcol, g1, n)
    assert np.allclose(np.diag(G1.T @ A @ G1), 1.0, rtol=1e-13, atol=0)
    # invariant under positive column scalings
    s = rng.uniform(0.1, 10.0, n)
    g2 = mpnn.column_normalize(grp, gcol, gv * s[gcol], rp, c, v)
    assert np.allclose(g2, g1, rtol=1e-13, atol=0)
    # Kaporin's number of G^T A G does not increase
    assert _kaporin(G1.T @ A @ G1) <= _kaporin(L.T @ A @ L) + 1e-12
    # FSAI and Jacobi are fixed points
    F = _fsai_factor(rp, c, v)
    frp, fcol, fv = _csr_of(F)
    assert np.allclose(mpnn.column_normalize(frp, fcol, fv, rp, c, v), fv, rtol=1e-13, atol=0)
    d = np.diag(A)
    jv = 1.0 / np.sqrt(d)
    jrp = np.arange(n + 1, dtype=np.int32)
    assert np.allclose(mpnn.column_normalize(jrp, np.arange(n, dtype=np.int32), jv, rp, c, v), jv, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- inverse problem (Sec. 4.6)

def test_inverse_assembly_theta_zero_is_poisson_and_spd():
    """kappa = 1 puts coefficient 1 on every face, boundary faces included:
    the unscaled 2D Poisson matrix exactly; any theta gives a symmetric
    positive definite A (Cholesky succeeds, values equal their transpose)."""
    import oracle.inverse as OI
    for N in (1, 2, 7):
        rp, c, v = OI.assemble(np.zeros((N, N)))
        r2, c2, v2 = I.poisson2d(N)
        assert np.array_equal(rp, r2) and np.array_equal(c, c2) and np.array_equal(v, v2)
    th = I.gaussian_random_field(9, 5, sigma_cells=2.0)
    rp, c, v = OI.assemble(th)
    rpt, ct, pt = oracle.transpose(rp, c)
    assert np.array_equal(rp, rpt) and np.array_equal(c, ct) and np.array_equal(v, v[pt])
    np.linalg.cholesky(dense(rp, c, v))


def test_inverse_single_cell_closed_form():
    """One cell: four boundary faces, A = [4 kappa], x = b / (4 e^theta),
    L = (x - x_t)^2, dL/dtheta = -2 (x - x_t) x."""
    import oracle.inverse as OI
    th = np.array([[0.3]])
    b = np.array([[0.7], [-0.2]])
    xt = np.array([[0.1], [0.05]])
    L, g, _ = OI.loss_and_grad(th, b, xt)
    x = b[:, 0] / (4.0 * math.exp(0.3))
    assert abs(L - np.mean((x - xt[:, 0]) ** 2)) <= 1e-15
    gref = np.mean(-2.0 * (x - xt[:, 0]) * x)
    assert abs(g[0, 0] - gref) <= 1e-14 * abs(gref)


def test_inverse_oracle_gradient_central_differences():
    """dL/dtheta of the oracle (adjoint per right-hand side + chain rule)
    against central differences (eps = 1e-5, Sec. 4.3) of the loss from
    dense LU solves: random directions and single cells."""
    import oracle.inverse as OI
    N, k = 8, 3
    th = I.gaussian_random_field(N, 3, sigma_cells=2.0)
    B = I.rhs_uniform(N * N, 5, batch=k)
    Xt = OI.solve_dense(I.gaussian_random_field(N, 4, sigma_cells=2.0), B)
    L, g, gB = OI.loss_and_grad(th, B, Xt)
    assert abs(L - OI.loss_dense(th, B, Xt)) <= 1e-12 * L
    rng = np.random.default_rng(0)
    eps = 1e-5
    dirs = [rng.standard_normal(th.shape) for _ in range(3)]
    for (q, p) in ((0, 0), (3, 5), (7, 7), (0, 6)):
        e = np.zeros(th.shape)
        e[q, p] = 1.0
        dirs.append(e)
    for d in dirs:
        fd = (OI.loss_dense(th + eps * d, B, Xt) - OI.loss_dense(th - eps * d, B, Xt)) / (2 * eps)
        an = float((g * d).sum())
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


def test_gaussian_random_field_recipe():
    """Zero mean, the requested standard deviation, deterministic per seed,
    and smooth: neighbouring cells of a sigma = 8 field are highly correlated
    while white noise is not."""
    f = I.gaussian_random_field(64, 11)
    assert abs(f.mean()) <= 1e-12 and abs(f.std() - 0.5) <= 1e-12
    assert np.array_equal(f, I.gaussian_random_field(64, 11))
    corr = np.corrcoef(f[:, 1:].ravel(), f[:, :-1].ravel())[0, 1]
    assert corr > 0.95
    w = I.gaussian_random_field(64, 11, sigma_cells=1e-3)
    assert abs(np.corrcoef(w[:, 1:].ravel(), w[:, :-1].ravel())[0, 1]) < 0.1


def test_inverse_torch_assembly_matches_oracle_on_cpu():
    """The product's differentiable assembly (torch, here on CPU tensors)
    against the oracle's loops: values to rounding, and its autograd chain
    rule against the oracle's face-by-face one."""
    import torch

    import oracle.inverse as OI
    from paper_2601_13994_b300.inverse import _selection, assemble_values
    N = 6
    th = I.gaussian_random_field(N, 8, sigma_cells=1.5)
    rp, c, v = OI.assemble(th)
    t = torch.tensor(th, requires_grad=True)
    vt = assemble_values(t, _selection(N, "cpu"))
    assert np.max(np.abs(vt.detach().numpy() - v)) <= 4e-16 * np.max(np.abs(v))
    gv = np.random.default_rng(1).standard_normal(len(v))
    vt.backward(torch.tensor(gv))
    ref = OI.chain_theta(th, rp, c, gv)
    assert np.max(np.abs(t.grad.numpy() - ref)) <= 1e-14 * np.max(np.abs(ref))


# ---------------------------------------------------------------- nonlinear adjoint (Sec. 3.2)

def _nl_case(N, seed):
    rng = np.random.default_rng(seed)
    theta = 0.5 * rng.standard_normal((N, N))
    f = 1.0 + 0.5 * rng.uniform(-1, 1, N * N)
    return theta, f


def test_nonlinear_newton_manufactured_solution():
    """f built from a chosen u_e with the dense A(theta): Newton from 0 must
    return u_e, with quadratic convergence at the end."""
    from oracle import inverse as OI
    from oracle import nonlinear as ON
    N, gamma = 7, 10.0
    theta, _ = _nl_case(N, 1)
    rng = np.random.default_rng(2)
    ue = rng.uniform(0.0, 2.0, N * N)
    A = OI.dense(*OI.assemble(theta))
    h2 = 1.0 / (N + 1) ** 2
    f = (A @ ue) / h2 + gamma * ue ** 3
    u, hist = ON.newton(theta, f, gamma, tol=1e-14)
    assert np.linalg.norm(u - ue) <= 1e-12 * np.linalg.norm(ue)
    assert len(hist) <= 12
    # quadratic: ||F_{k+1}|| <= C ||F_k||^2 once in the basin
    k = max(i for i in range(1, len(hist) - 1) if hist[i] > 1e-10 * hist[0]) if len(hist) > 3 else 1
    assert hist[k + 1] <= 10.0 * hist[k] ** 2 / hist[0] + 1e-13 * hist[0]


def test_nonlinear_single_cell_closed_form():
    """N = 1: A = [4 kappa] (four boundary faces), h^2 = 1/4:
    4 kappa u + (gamma u^3 - f)/4 = 0 and, by implicit differentiation,
    du/dtheta = -4 kappa u / (4 kappa + 3 gamma u^2 / 4)."""
    from oracle import nonlinear as ON
    for th, gamma, f, ut in ((0.3, 2.0, 5.0, 0.1), (-0.7, 10.0, 3.0, -0.2), (0.0, 0.0, 4.0, 0.0)):
        theta = np.array([[th]])
        kap = math.exp(th)
        roots = np.roots([gamma / 4.0, 0.0, 4.0 * kap, -f / 4.0]) if gamma > 0 else np.array([f / (16 * kap)])
        u_exact = float(np.real(roots[np.abs(np.imag(roots)) < 1e-12][0]))
        L, g, u = ON.loss_and_grad(theta, np.array([f]), gamma, np.array([ut]))
        assert abs(u[0] - u_exact) <= 1e-13 * max(1.0, abs(u_exact))
        dudt = -4 * kap * u_exact / (4 * kap + 3 * gamma * u_exact ** 2 / 4)
        assert abs(L - (u_exact - ut) ** 2) <= 1e-14
        assert abs(g[0, 0] - 2 * (u_exact - ut) * dudt) <= 1e-12 * max(1.0, abs(dudt))


def test_nonlinear_adjoint_central_differences():
    """dL/dtheta from one adjoint solve at u* against central differences
    of the Newton loss (eps = 1e-5, the paper's FD check, Tab. 5)."""
    from oracle import nonlinear as ON
    N, gamma = 6, 10.0
    theta, f = _nl_case(N, 3)
    theta_t, _ = _nl_case(N, 4)
    ut, _ = ON.newton(theta_t, f, gamma, tol=1e-14)
    L, g, _ = ON.loss_and_grad(theta, f, gamma, ut)
    rng = np.random.default_rng(5)
    eps = 1e-5
    for _ in range(3):
        d = rng.standard_normal(theta.shape)
        fd = (ON.loss(theta + eps * d, f, gamma, ut) - ON.loss(theta - eps * d, f, gamma, ut)) / (2 * eps)
        assert abs(fd - float((g * d).sum())) <= 1e-6 * abs(fd)
    for (q, p) in ((0, 0), (2, 3), (5, 1)):
        e = np.zeros_like(theta)
        e[q, p] = 1.0
        fd = (ON.loss(theta + eps * e, f, gamma, ut) - ON.loss(theta - eps * e, f, gamma, ut)) / (2 * eps)
        assert abs(fd - g[q, p]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max())


# ---------------------------------------------------------------- eigenvalue path (Sec. 3.2, Eq. 4)

def _laplacian_1d(n):
    rp, c, v = [0], [], []
    for i in range(n):
        for j, a in ((i - 1, -1.0), (i, 2.0), (i + 1, -1.0)):
            if 0 <= j < n:
                c.append(j)
                v.append(a)
        rp.append(len(c))
    return np.array(rp, np.int32), np.array(c, np.int32), np.array(v)


def test_eigen_oracle_closed_forms():
    """1D Laplacian: lambda_j = 4 sin^2(j pi / 2(n+1)), v_j(i) ~ sin(j pi i/(n+1));
    2D Poisson: the six smallest of 4 sin^2(a pi/2(N+1)) + 4 sin^2(b pi/2(N+1))."""
    from oracle import eigen as OE
    n, k = 40, 6
    rp, c, v = _laplacian_1d(n)
    lam, V = OE.smallest_eigenpairs(rp, c, v, k)
    j = np.arange(1, k + 1)
    assert np.abs(lam - 4 * np.sin(j * np.pi / (2 * (n + 1))) ** 2).max() <= 1e-13
    i = np.arange(1, n + 1)
    for q in range(k):
        ref = np.sin((q + 1) * np.pi * i / (n + 1))
        ref /= np.linalg.norm(ref)
        assert abs(abs(ref @ V[:, q]) - 1.0) <= 1e-12
        assert V[np.argmax(np.abs(V[:, q])), q] > 0
    N = 12
    rp, c, v = I.poisson2d(N)
    lam, _ = OE.smallest_eigenpairs(rp, c, v, k)
    a = np.arange(1, N + 1)
    allv = np.sort((4 * np.sin(a[:, None] * np.pi / (2 * (N + 1))) ** 2
                    + 4 * np.sin(a[None, :] * np.pi / (2 * (N + 1))) ** 2).ravel())
    assert np.abs(lam - allv[:k]).max() <= 1e-12


def test_hellmann_feynman_closed_form_and_central_differences():
    """Eq. 4: on the 1D Laplacian d lambda_j / d A_ii = v_j(i)^2 =
    2/(n+1) sin^2(j pi i/(n+1)); on a variable-coefficient system the
    gradient of L = sum_j w_j lambda_j matches central differences along
    symmetric perturbations of the stored entries (eps = 1e-5; Tab. 5
    reports 2.1e-6)."""
    from oracle import eigen as OE
    n, k = 30, 4
    rp, c, v = _laplacian_1d(n)
    lam, V = OE.smallest_eigenpairs(rp, c, v, k)
    for q in range(k):
        g = np.zeros(k)
        g[q] = 1.0
        gv = OE.eigenvalue_grad_values(rp, c, V, g)
        for i in range(n):
            e = [e for e in range(rp[i], rp[i + 1]) if c[e] == i][0]
            ref = 2.0 / (n + 1) * np.sin((q + 1) * np.pi * (i + 1) / (n + 1)) ** 2
            assert abs(gv[e] - ref) <= 1e-13
    rp, c, v = I.diffusion2d_random(7, 3)
    k = 6
    lam, V = OE.smallest_eigenpairs(rp, c, v, k)
    assert np.diff(lam).min() > 1e-3  # simple eigenvalues
    w = np.random.default_rng(1).uniform(0.5, 1.5, k)
    gv = OE.eigenvalue_grad_values(rp, c, V, w)
    A = OE.dense(rp, c, v)
    rng = np.random.default_rng(2)
    eps = 1e-5
    for _ in range(4):
        D = np.zeros_like(A)
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        d = rng.standard_normal(len(v))
        D[rows, c] = d
        D = 0.5 * (D + D.T)
        dv = D[rows, c]
        lp = np.linalg.eigvalsh(A + eps * D)[:k]
        lm = np.linalg.eigvalsh(A - eps * D)[:k]
        fd = float(w @ (lp - lm)) / (2 * eps)
        assert abs(fd - float(gv @ dv)) <= 1e-6 * abs(fd)


def _eig_loss(A, k, glam, gV):
    """L = sum_j glam_j lambda_j + sum_j gV_j^T v_j for the k smallest pairs
    of a dense matrix (symmetric: eigh; else eig, real parts), each v_j of
    unit norm with its largest-magnitude entry positive."""
    if np.array_equal(A, A.T):
        lam, V = np.linalg.eigh(A)
    else:
        lam, V = np.linalg.eig(A)
        o = np.argsort(lam.real)
        lam, V = lam.real[o], V.real[:, o]
    lam, V = lam[:k], V[:, :k] / np.linalg.norm(V[:, :k], axis=0)
    for j in range(k):
        if V[np.argmax(np.abs(V[:, j])), j] < 0:
            V[:, j] = -V[:, j]
    return float(glam @ lam) + float(np.sum(gV * V))


def test_eigenvector_adjoint_diagonal_closed_form():
    """A = diag(d), d distinct: v_j = e_j and the deflated solve is diagonal,
    mu_j[m] = gV_j[m] / (d_m - d_j) for m != j, mu_j[j] = 0."""
    from oracle import eigen as OE
    rng = np.random.default_rng(5)
    n, k = 9, 4
    d = np.sort(rng.uniform(1.0, 5.0, n))
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    lam, V = OE.smallest_eigenpairs(rp, c, d, k)
    assert np.array_equal(V, np.eye(n)[:, :k])
    gV = rng.standard_normal((n, k))
    mu = OE.eigenvector_adjoint(rp, c, d, lam, V, gV)
    for j in range(k):
        ref = np.array([0.0 if m == j else gV[m, j] / (d[m] - d[j]) for m in range(n)])
        assert np.abs(mu[:, j] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_eigenvector_gradient_central_differences():
    """The full gradient (Hellmann-Feynman plus the deflated-solve
    eigenvector part) of L = sum glam_j lambda_j + sum gV_j^T v_j against
    central differences (eps = 1e-5, as Tab. 5): along symmetric
    perturbations of the stored entries, and along single off-diagonal
    entries (a non-symmetric perturbation: the right eigenvectors), which
    tells -mu_a v_b from its transpose -mu_b v_a."""
    from oracle import eigen as OE
    rp, c, v = I.diffusion2d_random(6, 8)
    n, k = len(rp) - 1, 4
    lam, _ = OE.smallest_eigenpairs(rp, c, v, k + 1)
    assert np.diff(lam).min() > 1e-2
    rng = np.random.default_rng(9)
    glam = rng.uniform(0.5, 1.5, k)
    gV = rng.standard_normal((n, k))
    g = OE.eigen_loss_grad(rp, c, v, k, glam, gV)
    A = OE.dense(rp, c, v)
    rows = np.repeat(np.arange(n), np.diff(rp))
    eps = 1e-5
    for _ in range(3):
        D = np.zeros_like(A)
        D[rows, c] = rng.standard_normal(len(v))
        D = 0.5 * (D + D.T)
        fd = (_eig_loss(A + eps * D, k, glam, gV) - _eig_loss(A - eps * D, k, glam, gV)) / (2 * eps)
        assert abs(fd - float(g @ D[rows, c])) <= 1e-6 * abs(fd)
    off = [e for e in range(len(v)) if rows[e] != c[e]]
    for e in rng.choice(off, 4, replace=False):
        D = np.zeros_like(A)
        D[rows[e], c[e]] = 1.0
        fd = (_eig_loss(A + eps * D, k, glam, gV) - _eig_loss(A - eps * D, k, glam, gV)) / (2 * eps)
        et = [t for t in range(len(v)) if rows[t] == c[e] and c[t] == rows[e]][0]
        assert abs(fd - g[e]) <= 1e-6 * max(abs(fd), 1e-3), (e, fd, g[e])
        assert abs(g[e] - g[et]) > 1e-3 * abs(fd)  # the transpose differs: the check can tell them apart


# ---------------------------------------------------------------- all-core (OpenMP) oracle PCG

@pytest.mark.parametrize("threads", [1, 4])
def test_pcg_omp_matches_lu_and_single_thread_oracle(threads):
    """The OpenMP build of the oracle's Jacobi-PCG: same steps as pcg, so the
    solution matches dense LU and the single-threaded oracle's to rounding,
    and the iteration count to within a few (only the inner products'
    summation order differs)."""
    rp, c, v = I.diffusion3d_random(14, 5)
    n = len(rp) - 1
    b = I.rhs_uniform(n, 6)
    xs = np.linalg.solve(dense(rp, c, v), b)
    for pc in ("jacobi", "none"):
        x, io = oracle.pcg_omp(rp, c, v, b, rtol=1e-12, precond=pc, threads=threads)
        assert io["threads"] == threads
        xo, ioo = oracle.pcg(rp, c, v, b, rtol=1e-12, precond=pc)
        assert io["status"] == 0 and ioo["status"] == 0
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
        assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)
        assert abs(io["iters"] - ioo["iters"]) <= 2
        assert io["true_rel_res"] <= 2e-12


def test_pcg_omp_edge_cases_match_oracle():
    rp, c, v = I.poisson2d(6)
    n = 36
    # b = 0: x = 0 after 0 iterations, OK
    x, io = oracle.pcg_omp(rp, c, v, np.zeros(n), threads=2)
    assert io["status"] == 0 and io["iters"] == 0 and not x.any()
    # non-positive diagonal: NOT_SPD before iterating, as the oracle
    v2 = v.copy()
    v2[(np.repeat(np.arange(n), np.diff(rp)) == 3) & (c == 3)] = -1.0
    _, io = oracle.pcg_omp(rp, c, v2, np.ones(n), threads=2)
    _, ioo = oracle.pcg(rp, c, v2, np.ones(n))
    assert io["status"] == ioo["status"] == 3 and io["iters"] == 0
    # iteration cap
    b = I.rhs_uniform(n, 2)
    _, io = oracle.pcg_omp(rp, c, v, b, rtol=1e-15, max_iter=3, max_restarts=0, threads=2)
    _, ioo = oracle.pcg(rp, c, v, b, rtol=1e-15, max_iter=3, max_restarts=0)
    assert io["status"] == ioo["status"] == 1 and io["iters"] == ioo["iters"] == 3
    # indefinite: p^T A p <= 0 -> NOT_SPD
    rpi = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    vi = np.array([1.0, 3.0, 3.0, 1.0])
    _, io = oracle.pcg_omp(rpi, ci, vi, np.array([1.0, -1.0]), precond="none", threads=2)
    _, ioo = oracle.pcg(rpi, ci, vi, np.array([1.0, -1.0]), precond="none")
    assert io["status"] == ioo["status"] == 3


# ---------------------------------------------------------------- nonsymmetric batch generators

def test_convdiff2d_generator_is_diffusion_plus_upwind():
    """With zero velocity the rectangle generator is the diffusion operator
    (square case: the same CSR as diffusion2d); with velocity w the
    difference is the first-order upwind matrix: +|w_x| + |w_y| on the
    diagonal, -|w_x| on the upstream x-neighbour, -|w_y| on the upstream
    y-neighbour, nothing downstream."""
    rng = np.random.default_rng(0)
    N = 5
    cx = np.exp(rng.standard_normal((N, N + 1)))
    cy = np.exp(rng.standard_normal((N + 1, N)))
    d0 = I.diffusion2d(cx, cy)
    c0 = I.convdiff2d_rect(cx, cy, 0.0, 0.0)
    for a, b in zip(d0, c0):
        assert np.array_equal(a, b)
    Ny, Nx = 3, 4
    cx = np.exp(rng.standard_normal((Ny, Nx + 1)))
    cy = np.exp(rng.standard_normal((Ny + 1, Nx)))
    for wx, wy in ((2.5, -1.5), (-3.0, 0.7)):
        D = dense(*I.convdiff2d_rect(cx, cy, 0.0, 0.0))
        C = dense(*I.convdiff2d_rect(cx, cy, wx, wy))
        U = np.zeros_like(D)
        for q in range(Ny):
            for p in range(Nx):
                i = p + Nx * q
                U[i, i] = abs(wx) + abs(wy)
                up_x = p - 1 if wx > 0 else p + 1
                up_y = q - 1 if wy > 0 else q + 1
                if 0 <= up_x < Nx:
                    U[i, up_x + Nx * q] = -abs(wx)
                if 0 <= up_y < Ny:
                    U[i, p + Nx * up_y] = -abs(wy)
        assert np.allclose(C - D, U, rtol=0, atol=1e-14)
        assert not np.allclose(C, C.T)
        # weak diagonal dominance everywhere, strict on the boundary rows
        off = np.abs(C).sum(axis=1) - np.abs(np.diag(C))
        assert (np.diag(C) - off >= -1e-12).all() and (np.diag(C) - off > 1e-12).any()


def test_bicgstab_warm_start_at_the_solution_is_converged():
    """A start that already meets the stopping test ||r|| <= max(rtol ||b||,
    atol) is converged after 0 iterations, for BiCGStab as for PCG."""
    rp, c, v = I.convdiff3d(6, 10.0)
    b = I.rhs_uniform(len(rp) - 1, 3)
    xs = np.linalg.solve(dense(rp, c, v), b)
    x, io = oracle.bicgstab(rp, c, v, b, rtol=1e-8, x0=xs)
    assert io["status"] == 0 and io["iters"] == 0 and np.array_equal(x, xs)
    rp2, c2, v2 = I.poisson2d(6)
    b2 = I.rhs_uniform(36, 3)
    xs2 = np.linalg.solve(dense(rp2, c2, v2), b2)
    _, io2 = oracle.pcg(rp2, c2, v2, b2, rtol=1e-8, x0=xs2)
    assert io2["status"] == 0 and io2["iters"] == 0
    # a start that does not meet it still iterates
    x, io = oracle.bicgstab(rp, c, v, b, rtol=1e-8, x0=0.5 * xs)
    assert io["status"] == 0 and io["iters"] > 0
