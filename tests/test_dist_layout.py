"""Host-side metadata of the distributed layer (Sec. 3.3): the row-block
partition, the halo sets, the extended local columns and the transposed
exchange lists, checked against brute force; and the adjoint identity
<H x, g> = <x, H^T g> (Eq. 5-6) with the exchange written out in numpy."""
import numpy as np
import pytest

from paper_2601_13994_b300 import distributed as D
from paper_2601_13994_b300 import inputs as I


def _cases():
    yield "poisson12", I.poisson2d(12)
    yield "var3d6", I.diffusion3d_random(6, 2)
    yield "fem", I.fem_p1_laplacian(9, 5)


@pytest.mark.parametrize("P", [1, 3, 5])
@pytest.mark.parametrize("balance", ["rows", "nnz"])
def test_layout_against_brute_force(P, balance):
    for name, (rp, c, v) in _cases():
        n = len(rp) - 1
        off = D.partition_rows(n, P, rp, balance)
        assert off[0] == 0 and off[-1] == n and (np.diff(off) >= 1).all()
        lay = D.build_layout(rp, c, off)
        src, cext, own = lay["src"], lay["col_ext"], lay["own_pos"]
        for p in range(P):
            o0, o1 = off[p], off[p + 1]
            cols = c[rp[o0]:rp[o1]]
            halo = sorted(set(int(j) for j in cols if j < o0 or j >= o1))
            a, e = lay["ext_off"][p], lay["ext_off"][p + 1]
            assert e - a == (o1 - o0) + len(halo) == lay["n_own"][p] + lay["n_halo"][p]
            assert src[a:a + o1 - o0].tolist() == list(range(o0, o1))
            assert src[a + o1 - o0:e].tolist() == halo
            # every local column points into this partition's segment and holds the right index
            ce = cext[rp[o0]:rp[o1]]
            assert ((ce >= a) & (ce < e)).all()
            assert np.array_equal(src[ce], cols)
            assert np.array_equal(own[o0:o1], np.arange(a, a + o1 - o0))
        # transposed exchange lists: for each i, exactly the halo copies of i, ascending
        hptr, hlist = lay["hptr"], lay["hlist"]
        is_own = np.zeros(lay["total_ext"], bool)
        is_own[own] = True
        for i in range(n):
            want = [e for e in range(lay["total_ext"]) if src[e] == i and not is_own[e]]
            assert hlist[hptr[i]:hptr[i + 1]].tolist() == want, (name, i)


def test_halo_exchange_adjoint_identity_and_local_spmv():
    rng = np.random.default_rng(0)
    rp, c, v = I.diffusion3d_random(7, 3)
    n = len(rp) - 1
    lay = D.build_layout(rp, c, D.partition_rows(n, 4))
    src, own, hptr, hlist = lay["src"], lay["own_pos"], lay["hptr"], lay["hlist"]

    def H(x):
        return x[src]

    def HT(g):
        out = g[own].copy()
        for i in range(n):
            for t in range(hptr[i], hptr[i + 1]):
                out[i] += g[hlist[t]]
        return out

    x = rng.standard_normal(n)
    g = rng.standard_normal(lay["total_ext"])
    lhs, rhs = H(x) @ g, x @ HT(g)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the local SpMVs on the extended vectors are the global product
    xe = H(x)
    rows = np.repeat(np.arange(n), np.diff(rp))
    y_loc = np.zeros(n)
    np.add.at(y_loc, rows, v * xe[lay["col_ext"]])
    y = np.zeros(n)
    np.add.at(y, rows, v * x[c])
    assert np.allclose(y_loc, y, rtol=0, atol=1e-13)
    # halos shrink with fewer partitions; one partition has none
    assert D.build_layout(rp, c, D.partition_rows(n, 1))["total_ext"] == n
