"""Pattern utilities vs the oracle: CSR transpose and COO ingest must match
bit for bit (integer work; duplicate sums in the same COO order)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla
from tests.gpu_util import csr, to_dev

pytestmark = pytest.mark.gpu


def patterns():
    yield "poisson2d_37", I.poisson2d(37)
    yield "diffusion3d_20", I.diffusion3d_random(20, 1)
    yield "convdiff3d_11", I.convdiff3d(11)
    yield "fem", I.fem_p1_laplacian(30, 4)
    yield "powerlaw", I.powerlaw_matrix(3000, 2, mean_len=10, alpha=1.3, max_len=3000, empty_frac=0.1)


@pytest.mark.parametrize("name,mat", list(patterns()), ids=[p[0] for p in patterns()])
def test_transpose_bit_exact(name, mat):
    rp, c, v = mat
    A = csr(rp, c)
    rpT, cT, pT = sla.csr_transpose(A)
    torch.cuda.synchronize()
    orp, oc, op = oracle.transpose(rp, c)
    assert np.array_equal(rpT.cpu().numpy(), orp)
    assert np.array_equal(cT.cpu().numpy(), oc)
    assert np.array_equal(pT.cpu().numpy(), op)
    vT = sla.gather_values(pT, to_dev(v)).cpu().numpy()
    assert np.array_equal(vT, v[op])


def test_transpose_degenerate():
    # empty matrix, one entry, all entries in one column
    rp, c, _ = np.zeros(6, np.int32), np.zeros(0, np.int32), None
    rpT, cT, pT = sla.csr_transpose(csr(rp, c))
    assert not rpT.cpu().numpy().any() and cT.numel() == 0
    n = 500
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.full(n, 7, np.int32)
    rpT, cT, pT = sla.csr_transpose(csr(rp, c))
    orp, oc, op = oracle.transpose(rp, c)
    assert np.array_equal(rpT.cpu().numpy(), orp) and np.array_equal(cT.cpu().numpy(), oc)
    assert np.array_equal(pT.cpu().numpy(), op)


@pytest.mark.parametrize("seed,n,m", [(0, 50, 400), (1, 3000, 20000), (2, 70000, 300000), (3, 1, 5)])
def test_coo_ingest_bit_exact(seed, n, m):
    rng = np.random.default_rng(seed)
    row = rng.integers(0, n, m)
    col = rng.integers(0, n, m)
    val = rng.uniform(-1, 1, m)
    A, vcsr, perm, order, segptr = sla.coo_to_csr(n, to_dev(row), to_dev(col), to_dev(val))
    torch.cuda.synchronize()
    orp, oc, ov, operm = oracle.coo_to_csr(n, row, col, val)
    assert np.array_equal(A.rowptr.cpu().numpy(), orp)
    assert np.array_equal(A.col.cpu().numpy(), oc)
    assert np.array_equal(vcsr.cpu().numpy(), ov)
    assert np.array_equal(perm.cpu().numpy(), operm)
    # new values on the same pattern, and the gradient map back to COO order
    val2 = rng.uniform(-1, 1, m)
    v2 = sla.segment_sum(segptr, order, to_dev(val2)).cpu().numpy()
    _, _, ov2, _ = oracle.coo_to_csr(n, row, col, val2)
    assert np.array_equal(v2, ov2)


def test_coo_ingest_of_a_generated_matrix_and_bad_index():
    rp, c, v = I.diffusion3d_random(12, 3)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    p = np.random.default_rng(0).permutation(len(c))
    A, vcsr, perm, _, _ = sla.coo_to_csr(n, to_dev(rows[p]), to_dev(c[p].astype(np.int64)), to_dev(v[p]))
    assert np.array_equal(A.rowptr.cpu().numpy(), rp) and np.array_equal(A.col.cpu().numpy(), c)
    assert np.array_equal(vcsr.cpu().numpy(), v)
    with pytest.raises(ValueError):
        sla.coo_to_csr(4, to_dev(np.array([0, 4])), to_dev(np.array([0, 1])), to_dev(np.array([1.0, 2.0])))
