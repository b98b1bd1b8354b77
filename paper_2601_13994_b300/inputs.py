"""Seeded synthetic input generators (CSR matrices and right-hand sides).

This module only *builds inputs*: stencil/FEM matrix assembly and random
draws.  It contains none of the solver arithmetic (no SpMV, no Krylov step,
no adjoint) and imports neither the CUDA library nor the CPU oracle, so that
both sides can be fed identical data.

All matrices are returned as ``(rowptr int32[n+1], col int32[nnz],
val float64[nnz])`` with column indices ascending inside each row.

Workload shapes follow the paper's 2D Poisson experiments (Tab. 3, Sec. 4.2)
and the variable-coefficient diffusion of the inverse problem (Sec. 4.4),
extended to 3D, to an upwind convection-diffusion operator (nonsymmetric,
the BiCGStab case of Sec. 3.1), to batches with shared patterns and to
P1 finite-element Laplacians on irregular meshes (the SparseTensorList case
of Sec. 3.1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "poisson2d", "diffusion2d", "diffusion2d_random", "diffusion3d",
    "diffusion3d_random", "convdiff3d", "rhs_uniform", "powerlaw_matrix",
    "batched_shared_2d", "fem_p1_laplacian", "fem_list", "nnz_2d", "nnz_3d",
    "gaussian_random_field",
]


def nnz_2d(N: int) -> int:
    """Stored entries of the N x N interior 5-point stencil."""
    return 5 * N * N - 4 * N


def nnz_3d(N: int) -> int:
    """Stored entries of the N^3 interior 7-point stencil."""
    return 7 * N ** 3 - 6 * N * N


def _compress(cols: np.ndarray, vals: np.ndarray, mask: np.ndarray):
    """(n, w) candidate columns/values + validity mask -> CSR (row-major)."""
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(cols.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = cols[mask].astype(np.int32, copy=False)
    val = vals[mask]
    return rowptr.astype(np.int32), np.ascontiguousarray(col), np.ascontiguousarray(val)


def diffusion2d(cx: np.ndarray, cy: np.ndarray):
    """Five-point operator of -div(c grad u) on an N x N interior grid.

    ``cx`` has shape (N, N+1): cx[q, p] is the coefficient on the x-face
    between cells p-1 and p of row q (p = 0 and p = N are the Dirichlet
    boundary faces).  ``cy`` has shape (N+1, N): cy[q, p] sits between rows
    q-1 and q.  Unknown index i = p + N q.  A_ii = sum of the 4 face
    coefficients, A_ij = -c_face for interior neighbours (unscaled, i.e.
    h^2 times the discrete operator)."""
    N = cx.shape[0]
    assert cx.shape == (N, N + 1) and cy.shape == (N + 1, N)
    n = N * N
    q, p = np.divmod(np.arange(n, dtype=np.int64), N)
    w = cx[q, p]
    e = cx[q, p + 1]
    s = cy[q, p]
    nn = cy[q + 1, p]
    i = np.arange(n, dtype=np.int64)
    cols = np.stack([i - N, i - 1, i, i + 1, i + N], axis=1)
    vals = np.stack([-s, -w, w + e + s + nn, -e, -nn], axis=1)
    mask = np.stack([q > 0, p > 0, np.ones(n, bool), p < N - 1, q < N - 1], axis=1)
    return _compress(cols, vals, mask)


def poisson2d(N: int):
    """Constant-coefficient 2D Poisson (diag 4, off-diagonal -1), N^2 unknowns.

    Its eigenpairs are v_jk(p, q) = sin(j pi (p+1)/(N+1)) sin(k pi (q+1)/(N+1))
    with mu_jk = 4 sin^2(j pi / 2(N+1)) + 4 sin^2(k pi / 2(N+1))."""
    return diffusion2d(np.ones((N, N + 1)), np.ones((N + 1, N)))


def diffusion2d_random(N: int, seed: int, sigma: float = 1.0):
    """2D five-point diffusion with face coefficients exp(N(0, sigma^2)).

    One ``default_rng(seed)`` stream draws the x-faces (row-major (N, N+1))
    then the y-faces ((N+1, N))."""
    rng = np.random.default_rng(seed)
    cx = np.exp(sigma * rng.standard_normal((N, N + 1)))
    cy = np.exp(sigma * rng.standard_normal((N + 1, N)))
    return diffusion2d(cx, cy)


def diffusion3d(cx: np.ndarray, cy: np.ndarray, cz: np.ndarray):
    """Seven-point operator of -div(c grad u) on an N^3 interior grid.

    Index i = p + N q + N^2 s.  ``cx`` (N, N, N+1) holds the x-faces,
    ``cy`` (N, N+1, N) the y-faces, ``cz`` (N+1, N, N) the z-faces, each
    including the boundary faces to the Dirichlet ghosts; arrays are indexed
    [s, q, p]."""
    N = cx.shape[0]
    n = N ** 3
    rowptr = np.zeros(n + 1, dtype=np.int64)
    # build row by row in slabs to bound the temporary memory
    cols_out = []
    vals_out = []
    counts = np.empty(n, dtype=np.int64)
    slab = max(1, min(N, (1 << 22) // (N * N)))
    for s0 in range(0, N, slab):
        s1 = min(N, s0 + slab)
        ss, qq, pp = np.meshgrid(np.arange(s0, s1), np.arange(N), np.arange(N), indexing="ij")
        ss = ss.ravel(); qq = qq.ravel(); pp = pp.ravel()
        i = pp + N * qq + N * N * ss
        w = cx[ss, qq, pp]; e = cx[ss, qq, pp + 1]
        so = cy[ss, qq, pp]; no = cy[ss, qq + 1, pp]
        b = cz[ss, qq, pp]; t = cz[ss + 1, qq, pp]
        cols = np.stack([i - N * N, i - N, i - 1, i, i + 1, i + N, i + N * N], axis=1)
        vals = np.stack([-b, -so, -w, w + e + so + no + b + t, -e, -no, -t], axis=1)
        ones = np.ones(i.shape[0], bool)
        mask = np.stack([ss > 0, qq > 0, pp > 0, ones, pp < N - 1, qq < N - 1, ss < N - 1], axis=1)
        counts[i[0]:i[-1] + 1] = mask.sum(axis=1)
        cols_out.append(cols[mask].astype(np.int32))
        vals_out.append(vals[mask])
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), np.concatenate(cols_out), np.concatenate(vals_out)


def diffusion3d_random(N: int, seed: int, sigma: float = 1.0):
    """3D seven-point diffusion with face coefficients exp(N(0, sigma^2)).

    One ``default_rng(seed)`` stream draws x-faces, then y-faces, then
    z-faces, each in lexicographic [s, q, p] order."""
    rng = np.random.default_rng(seed)
    cx = np.exp(sigma * rng.standard_normal((N, N, N + 1)))
    cy = np.exp(sigma * rng.standard_normal((N, N + 1, N)))
    cz = np.exp(sigma * rng.standard_normal((N + 1, N, N)))
    return diffusion3d(cx, cy, cz)


def convdiff3d(N: int, peclet: float = 10.0):
    """3D convection-diffusion, unit diffusion plus first-order upwind
    convection along +(1,1,1) at cell Peclet number ``peclet`` per axis.

    A_ii = 6 + 3 Pe, upstream neighbours (i-1, i-N, i-N^2) get -1 - Pe,
    downstream neighbours -1.  Nonsymmetric, diagonally dominant M-matrix."""
    n = N ** 3
    i = np.arange(n, dtype=np.int64)
    s, rem = np.divmod(i, N * N)
    q, p = np.divmod(rem, N)
    up = -1.0 - peclet
    dn = -1.0
    cols = np.stack([i - N * N, i - N, i - 1, i, i + 1, i + N, i + N * N], axis=1)
    vals = np.empty((n, 7))
    vals[:, 0] = up; vals[:, 1] = up; vals[:, 2] = up
    vals[:, 3] = 6.0 + 3.0 * peclet
    vals[:, 4] = dn; vals[:, 5] = dn; vals[:, 6] = dn
    ones = np.ones(n, bool)
    mask = np.stack([s > 0, q > 0, p > 0, ones, p < N - 1, q < N - 1, s < N - 1], axis=1)
    return _compress(cols, vals, mask)


def rhs_uniform(n: int, seed: int, batch: int | None = None) -> np.ndarray:
    """b ~ U[-1, 1] from ``default_rng(seed)``; shape (n,) or (batch, n)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if batch is None else (batch, n)
    return rng.uniform(-1.0, 1.0, size=shape)


def powerlaw_matrix(n: int, seed: int, mean_len: float = 8.0, alpha: float = 1.6,
                    max_len: int | None = None, empty_frac: float = 0.05,
                    diag_dominant: bool = True):
    """Irregular CSR for SpMV edge cases: row lengths drawn from a Pareto-like
    law (a few very long rows), a fraction of empty rows, random sorted
    distinct columns and U[-1,1] values.  With ``diag_dominant`` every
    non-empty row also stores its diagonal, set to 1 + sum |off-diagonal|."""
    rng = np.random.default_rng(seed)
    max_len = n if max_len is None else min(max_len, n)
    raw = (rng.pareto(alpha, size=n) + 1.0) * mean_len * (alpha - 1.0) / alpha
    lens = np.clip(raw.astype(np.int64), 1, max_len)
    lens[rng.random(n) < empty_frac] = 0
    rowptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    vals = []
    for i in range(n):
        L = int(lens[i])
        if L == 0:
            continue
        c = rng.choice(n, size=L, replace=False) if L < n else np.arange(n)
        if diag_dominant and i not in c:
            c[0] = i
        c = np.unique(c)
        v = rng.uniform(-1.0, 1.0, size=c.shape[0])
        if diag_dominant:
            d = c == i
            v[d] = 1.0 + np.abs(v[~d]).sum()
        cols.append(c)
        vals.append(v)
        lens[i] = c.shape[0]
    np.cumsum(lens, out=rowptr[1:])
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return rowptr.astype(np.int32), col, val


def batched_shared_2d(N: int, batch: int, seed0: int, sigma: float = 0.5):
    """``batch`` 2D five-point diffusion systems on one shared N x N pattern.

    System k uses face coefficients exp(N(0, sigma^2)) from
    ``default_rng(seed0 + k)``.  Returns (rowptr, col, val[batch, nnz])."""
    vals = None
    rowptr = col = None
    for k in range(batch):
        rp, c, v = diffusion2d_random(N, seed0 + k, sigma)
        if vals is None:
            rowptr, col = rp, c
            vals = np.empty((batch, v.shape[0]))
        vals[k] = v
    return rowptr, col, vals


# ---------------------------------------------------------------------------
# 2D convection-diffusion batches (nonsymmetric: the BiCGStab batches)
# ---------------------------------------------------------------------------

def convdiff2d_rect(cx: np.ndarray, cy: np.ndarray, wx: float, wy: float):
    """Five-point operator of -div(c grad u) + w . grad u on an Ny x Nx
    interior grid (unit spacing, Dirichlet boundary), convection by first
    order upwinding.  ``cx`` (Ny, Nx+1) and ``cy`` (Ny+1, Nx) are the face
    coefficients as in ``diffusion2d``; (wx, wy) the cell Peclet numbers per
    axis, of either sign.  Unknown i = p + Nx q.  The neighbour upstream
    along x (west for wx > 0, east for wx < 0) gets -|wx| on top of its
    diffusion coefficient and the diagonal gets +|wx| (likewise along y), so
    A is a diagonally dominant, nonsymmetric M-matrix; the five-point pattern
    does not depend on (wx, wy)."""
    Ny, Nx = cx.shape[0], cx.shape[1] - 1
    assert cy.shape == (Ny + 1, Nx)
    n = Nx * Ny
    q, p = np.divmod(np.arange(n, dtype=np.int64), Nx)
    w = cx[q, p]
    e = cx[q, p + 1]
    s = cy[q, p]
    nn = cy[q + 1, p]
    i = np.arange(n, dtype=np.int64)
    ax, ay = abs(wx), abs(wy)
    cols = np.stack([i - Nx, i - 1, i, i + 1, i + Nx], axis=1)
    vals = np.stack([-s - max(wy, 0.0), -w - max(wx, 0.0), w + e + s + nn + ax + ay,
                     -e - max(-wx, 0.0), -nn - max(-wy, 0.0)], axis=1)
    mask = np.stack([q > 0, p > 0, np.ones(n, bool), p < Nx - 1, q < Ny - 1], axis=1)
    return _compress(cols, vals, mask)


def convdiff2d_random(Nx: int, Ny: int, seed: int, sigma: float = 0.5, pe_max: float = 10.0):
    """One seeded system of ``convdiff2d_rect``: from ``default_rng(seed)``
    the x-faces, then the y-faces (exp(N(0, sigma^2))), then the velocity
    direction theta ~ U[0, 2 pi) and cell Peclet magnitude ~ U[0, pe_max]."""
    rng = np.random.default_rng(seed)
    cx = np.exp(sigma * rng.standard_normal((Ny, Nx + 1)))
    cy = np.exp(sigma * rng.standard_normal((Ny + 1, Nx)))
    theta = rng.uniform(0.0, 2.0 * math.pi)
    pe = rng.uniform(0.0, pe_max)
    return convdiff2d_rect(cx, cy, pe * math.cos(theta), pe * math.sin(theta))


def batched_convdiff_2d(N: int, batch: int, seed0: int, sigma: float = 0.5, pe_max: float = 10.0):
    """``batch`` nonsymmetric convection-diffusion systems on one shared
    N x N five-point pattern, system k from seed ``seed0 + k``.  Returns
    (rowptr, col, val[batch, nnz])."""
    vals = None
    rowptr = col = None
    for k in range(batch):
        rp, c, v = convdiff2d_random(N, N, seed0 + k, sigma, pe_max)
        if vals is None:
            rowptr, col = rp, c
            vals = np.empty((batch, v.shape[0]))
        vals[k] = v
    return rowptr, col, vals


def convdiff_list(count: int, seed0: int, n_lo: float = 1e3, n_hi: float = 5e4,
                  sigma: float = 0.5, pe_max: float = 10.0):
    """``count`` nonsymmetric systems with distinct patterns: system k draws,
    from ``default_rng(seed0 + k)``, a size log-uniform in [n_lo, n_hi] and
    an aspect ratio log-uniform in [1/2, 2], giving an Nx x Ny rectangle,
    then is ``convdiff2d_random(Nx, Ny, seed0 + k)``."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        aspect = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        Nx = max(2, int(round(math.sqrt(target * aspect))))
        Ny = max(2, int(round(target / Nx)))
        out.append(convdiff2d_random(Nx, Ny, seed0 + k, sigma, pe_max))
    return out


# ---------------------------------------------------------------------------
# P1 finite elements on jittered, holed triangulations (distinct patterns)
# ---------------------------------------------------------------------------

def fem_p1_laplacian(m: int, seed: int, hole_frac: float = 0.10, jitter: float = 0.2,
                     shift: float = 1e-3):
    """P1 stiffness matrix of -Laplace on a jittered m x m vertex grid of the
    unit square.  Each quad is split along a random diagonal, ``hole_frac``
    of the quads are removed, interior vertices are jittered by
    U[-jitter h, jitter h] per axis.  Vertices on the outer boundary are
    Dirichlet (eliminated); hole edges carry natural conditions.  Unknowns
    are the remaining vertices that touch a kept cell.  ``shift * I`` is
    added so that isolated pieces stay SPD."""
    rng = np.random.default_rng(seed)
    h = 1.0 / (m - 1)
    gy, gx = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    X = gx.astype(np.float64) * h
    Y = gy.astype(np.float64) * h
    interior = (gx > 0) & (gx < m - 1) & (gy > 0) & (gy < m - 1)
    jx = rng.uniform(-jitter * h, jitter * h, size=(m, m))
    jy = rng.uniform(-jitter * h, jitter * h, size=(m, m))
    X = np.where(interior, X + jx, X).ravel()
    Y = np.where(interior, Y + jy, Y).ravel()
    nq = (m - 1) * (m - 1)
    keep = rng.random(nq) >= hole_frac
    diag = rng.random(nq) < 0.5
    qy, qx = np.divmod(np.arange(nq), m - 1)
    v00 = qx + m * qy
    v10 = v00 + 1
    v01 = v00 + m
    v11 = v01 + 1
    t1 = np.where(diag[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(diag[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    tris = np.concatenate([t1[keep], t2[keep]], axis=0)
    # element stiffness: K_ab = (grad phi_a . grad phi_b) * area
    x = X[tris]; y = Y[tris]
    b = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], 1)
    c = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], 1)
    area2 = np.abs(b[:, 0] * c[:, 1] - b[:, 1] * c[:, 0])
    Ke = (b[:, :, None] * b[:, None, :] + c[:, :, None] * c[:, None, :]) / (2.0 * area2[:, None, None])
    on_bnd = ~interior.ravel()
    used = np.zeros(m * m, bool)
    used[tris.ravel()] = True
    unk = used & ~on_bnd
    num = -np.ones(m * m, dtype=np.int64)
    num[unk] = np.arange(int(unk.sum()))
    n = int(unk.sum())
    ra = np.repeat(tris, 3, axis=1).ravel()
    cb = np.tile(tris, (1, 3)).ravel()
    vv = Ke.reshape(-1)
    ok = unk[ra] & unk[cb]
    r = num[ra[ok]]
    cc = num[cb[ok]]
    v = vv[ok]
    key = r * n + cc
    order = np.argsort(key, kind="stable")
    key = key[order]; v = v[order]
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(v, start) if v.shape[0] else v
    rows = uniq // n
    cols = (uniq % n).astype(np.int32)
    sums = sums + np.where(rows == cols, shift, 0.0)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    return rowptr.astype(np.int32), cols, sums


def fem_list(count: int, seed0: int, n_lo: float = 1e3, n_hi: float = 5e4):
    """``count`` FEM systems with target sizes log-uniform in [n_lo, n_hi].

    System k draws its target from ``default_rng(seed0 + k)`` and uses the
    same seed for its mesh; the vertex grid side m is chosen so that the
    unknown count is close to the target (about 0.9 m^2 after holes and the
    boundary are removed)."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        m = max(4, int(round(math.sqrt(target / 0.9))) + 2)
        out.append(fem_p1_laplacian(m, seed0 + k))
    return out


def gaussian_random_field(N: int, seed: int, sigma_cells: float = 8.0, std: float = 0.5) -> np.ndarray:
    """Smooth random field on N x N cells: white noise N(0, 1) from
    ``default_rng(seed)`` convolved with a Gaussian of standard deviation
    ``sigma_cells`` cells (product with the Gaussian's transform under the
    FFT, on the field extended by mirror reflection by ceil(4 sigma) cells per
    side so that the borders do not wrap around), cropped back to N x N, then
    shifted to zero mean and scaled to standard deviation ``std``.  The
    log-coefficient of the inverse problem (Sec. 4.6, scaled to 512 x 512)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((N, N))
    pad = int(math.ceil(4.0 * sigma_cells))
    wp = np.pad(w, pad, mode="symmetric")
    f0 = np.fft.fftfreq(wp.shape[0])
    f1 = np.fft.fftfreq(wp.shape[1])
    g = np.exp(-2.0 * (math.pi * sigma_cells) ** 2 * (f0[:, None] ** 2 + f1[None, :] ** 2))
    sm = np.real(np.fft.ifft2(np.fft.fft2(wp) * g))[pad:pad + N, pad:pad + N]
    sm = sm - sm.mean()
    sd = sm.std()
    return std * sm / sd if sd > 0 else sm
