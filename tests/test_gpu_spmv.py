"""SpMV parity: the CUDA kernel against the oracle's plain CSR product on the
same seeded inputs, element by element.  Integer-valued inputs are exact in
FP64 whatever the summation order, so they must agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, to_dev

pytestmark = pytest.mark.gpu


def run(rp, c, v, x):
    A = csr(rp, c)
    y = sla.spmv(A, to_dev(v), to_dev(x))
    torch.cuda.synchronize()
    return y.cpu().numpy()


def cases():
    yield "poisson2d_64", I.poisson2d(64)
    yield "poisson2d_ragged_37", I.poisson2d(37)
    yield "diffusion3d_33", I.diffusion3d_random(33, 1)
    yield "convdiff3d_20", I.convdiff3d(20)
    yield "fem_p1", I.fem_p1_laplacian(50, 3)
    # long rows: several rows above the 2048-entry staging capacity, many empty rows
    yield "powerlaw_long", I.powerlaw_matrix(6000, 5, mean_len=12, alpha=1.2, max_len=6000, empty_frac=0.1)
    yield "powerlaw_short", I.powerlaw_matrix(3001, 6, mean_len=4, alpha=2.5, empty_frac=0.2)


@pytest.mark.parametrize("name,mat", list(cases()), ids=[c[0] for c in cases()])
def test_spmv_matches_oracle(name, mat):
    rp, c, v = mat
    n = len(rp) - 1
    x = np.random.default_rng(n).uniform(-1, 1, n)
    y = run(rp, c, v, x)
    ref = oracle.spmv(rp, c, v, x)
    # per-row bound: |error| <= nnz_row * eps * sum |a_ij x_j|
    absrow = oracle.spmv(rp, c, np.abs(v), np.abs(x))
    lens = np.diff(rp)
    tol = (lens + 2) * 2.3e-16 * absrow + 1e-300
    assert np.all(np.abs(y - ref) <= tol), name
    if name == "powerlaw_long":
        assert lens.max() > 2048


@pytest.mark.parametrize("mat", [I.poisson2d(41), I.powerlaw_matrix(5000, 7, mean_len=20, alpha=1.3,
                                                                    max_len=5000)])
def test_spmv_integer_values_bit_exact(mat):
    rp, c, v = mat
    n = len(rp) - 1
    rng = np.random.default_rng(1)
    vi = rng.integers(-8, 9, size=len(v)).astype(np.float64)
    x = rng.integers(-8, 9, size=n).astype(np.float64)
    assert np.array_equal(run(rp, c, vi, x), oracle.spmv(rp, c, vi, x))


def test_spmv_degenerate_sizes():
    # one row, an all-empty matrix, and n = 0
    assert np.array_equal(run(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]),
                              np.array([2.0])), np.array([6.0]))
    n = 300
    y = run(np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0), np.ones(n))
    assert not y.any()
    A = csr(np.zeros(1, np.int32), np.zeros(0, np.int32))
    y = sla.spmv(A, torch.zeros(0, dtype=torch.float64, device="cuda"),
                 torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert y.numel() == 0


def test_csr_check_rejects_bad_patterns():
    with pytest.raises(ValueError):
        csr(np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32))       # rowptr decreasing
    with pytest.raises(ValueError):
        csr(np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32))       # column out of range
    with pytest.raises(ValueError):
        csr(np.array([0, 2, 2], np.int32), np.array([1, 0], np.int32))       # unsorted row


def test_spmv_deterministic_and_stream_ordered():
    rp, c, v = I.diffusion3d_random(40, 2)
    n = len(rp) - 1
    A = csr(rp, c)
    vt = to_dev(v)
    x = to_dev(np.random.default_rng(0).uniform(-1, 1, n))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        y1 = sla.spmv(A, vt, x)
        y2 = sla.spmv(A, vt, x)
    s.synchronize()
    assert torch.equal(y1, y2)


def _arrow(n, seed):
    """Dense first row and first column plus a diagonal (SPD-like): one row of
    n entries among rows of 2."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        if i == 0:
            cs = np.arange(n)
        else:
            cs = np.array([0, i])
        rows.append(np.full(len(cs), i)); cols.append(cs)
    r = np.concatenate(rows); c = np.concatenate(cols)
    rp = np.zeros(n + 1, np.int64); np.add.at(rp, r + 1, 1); rp = np.cumsum(rp)
    v = rng.uniform(-1, 1, len(c))
    return rp.astype(np.int32), c.astype(np.int32), v


def merge_cases():
    yield "arrow_20000", _arrow(20000, 1)
    yield "arrow_300001", _arrow(300001, 2)
    yield "powerlaw_long", I.powerlaw_matrix(6000, 5, mean_len=12, alpha=1.2, max_len=6000, empty_frac=0.1)
    yield "powerlaw_big", I.powerlaw_matrix(40000, 9, mean_len=6, alpha=1.1, max_len=40000, empty_frac=0.3)
    yield "poisson2d_37", I.poisson2d(37)
    yield "fem_p1", I.fem_p1_laplacian(40, 3)


@pytest.mark.parametrize("name,mat", list(merge_cases()), ids=[c[0] for c in merge_cases()])
def test_merge_path_and_row_kernels_match_oracle(name, mat):
    """sla_spmv_merge (rows crossing up to tens of thousands of 8-item
    chunks, empty rows) and the row kernels, both forced, against the oracle
    within the per-row rounding bound; the merge path is deterministic."""
    rp, c, v = mat
    n = len(rp) - 1
    A = csr(rp, c)
    x = np.random.default_rng(n + 1).uniform(-1, 1, n)
    vt, xt = to_dev(v), to_dev(x)
    ym = sla.spmv(A, vt, xt, scheme="merge")
    ym2 = sla.spmv(A, vt, xt, scheme="merge")
    yr = sla.spmv(A, vt, xt, scheme="rows")
    torch.cuda.synchronize()
    assert torch.equal(ym, ym2)
    ref = oracle.spmv(rp, c, v, x)
    absrow = oracle.spmv(rp, c, np.abs(v), np.abs(x))
    tol = (np.diff(rp) + 2) * 2.3e-16 * absrow + 1e-300
    for y in (ym, yr):
        assert np.all(np.abs(y.cpu().numpy() - ref) <= tol), name


def test_spmv_scheme_from_row_statistics():
    """The automatic choice: the merge path for patterns with a dominant long
    row, the row kernels for stencils; the statistics are the longest row and
    the count of rows above 1024 entries; integer data agree bit for bit."""
    rp, c, v = _arrow(50000, 3)
    A = csr(rp, c)
    assert A.row_stats() == (50000, 1)
    assert A.spmv_scheme == 1
    B = csr(*I.poisson2d(64)[:2])
    assert B.row_stats() == (5, 0) and B.spmv_scheme == 0
    rng = np.random.default_rng(4)
    vi = rng.integers(-8, 9, size=len(v)).astype(np.float64)
    xi = rng.integers(-8, 9, size=len(rp) - 1).astype(np.float64)
    y = sla.spmv(A, to_dev(vi), to_dev(xi))
    assert np.array_equal(y.cpu().numpy(), oracle.spmv(rp, c, vi, xi))


def test_merge_path_degenerate_sizes():
    one = sla.spmv(csr(np.array([0, 1], np.int32), np.array([0], np.int32)), to_dev(np.array([3.0])),
                   to_dev(np.array([2.0])), scheme="merge")
    assert one.cpu().numpy().tolist() == [6.0]
    n = 300
    y = sla.spmv(csr(np.zeros(n + 1, np.int32), np.zeros(0, np.int32)), torch.zeros(0, dtype=torch.float64,
                 device="cuda"), to_dev(np.ones(n)), scheme="merge")
    assert not y.cpu().numpy().any()
