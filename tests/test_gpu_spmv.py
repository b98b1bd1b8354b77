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
