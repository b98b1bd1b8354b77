"""GPU test of sla_cg_noalloc, the allocation-free CG entry point.

It serves callers that cannot allocate device memory when they solve (code
inside an allocator hook, hosts that reserve all memory at start-up,
plug-ins without an allocator): its scratch is a fixed array inside the
library instead of a caller workspace.  Its output must match sla_cg's (the
workspace entry point) within the solution tolerance used by the other
parity tests, on two calls in a row that share the array.

Kept in a file that pytest collects last, so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2601_13994_b300 import _lib as L
from paper_2601_13994_b300 import inputs as I
from paper_2601_13994_b300 import sla

pytestmark = pytest.mark.gpu

REL_TOL = 1e-8  # relative solution tolerance of the CG parity tests


def _info_host(raw):
    h = raw.cpu().numpy().reshape(-1)
    return int(h[:4].view(np.int32)[0]), int(h[4:8].view(np.int32)[0]), float(h[8:16].view(np.float64)[0])


def _solve_noalloc(A, val, b, rtol, flags=0):
    x = torch.empty_like(b)
    info = torch.empty(L.INFO_BYTES, dtype=torch.uint8, device=b.device)
    o = L.SlaOpts(rtol, 0.0, sla.default_max_iter(A.n), 2, L.SLA_PRECOND_JACOBI, 0, flags)
    rc = L.lib().sla_cg_noalloc(ctypes.byref(A.c), val.data_ptr(), b.data_ptr(), x.data_ptr(),
                                ctypes.byref(o), info.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == L.SLA_OK, rc
    torch.cuda.synchronize()
    return x, _info_host(info)


def _solve_workspace(A, val, b, rtol):
    x = torch.empty_like(b)
    info = torch.empty(L.INFO_BYTES, dtype=torch.uint8, device=b.device)
    o = L.SlaOpts(rtol, 0.0, sla.default_max_iter(A.n), 2, L.SLA_PRECOND_JACOBI, 0, 0)
    nbytes = L.workspace_size(L.SLA_WS_CG, A.n, A.nnz)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=b.device)
    rc = L.lib().sla_cg(ctypes.byref(A.c), val.data_ptr(), b.data_ptr(), x.data_ptr(), ctypes.byref(o),
                        info.data_ptr(), ws.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    assert rc == L.SLA_OK, rc
    torch.cuda.synchronize()
    return x, _info_host(info)


def test_noalloc_matches_workspace_entry_point_two_calls():
    rp, c, v = I.diffusion3d_random(28, 4)
    n = 28 ** 3
    A = sla.CSRMatrix.from_numpy(rp, c, device="cuda")
    val = torch.from_numpy(v).cuda()
    for seed in (5, 6):  # two calls in a row on the shared array
        bh = I.rhs_uniform(n, seed)
        b = torch.from_numpy(bh).cuda()
        x_ref, (it_ref, st_ref, _) = _solve_workspace(A, val, b, 1e-10)
        # and the oracle's solution, converged well below the solve's tolerance
        x_or, io = oracle.pcg(rp, c, v, bh, rtol=1e-13)
        assert io["status"] == 0
        x_na, (it_na, st_na, _) = _solve_noalloc(A, val, b, 1e-10)
        assert st_ref == st_na == L.SLA_OK
        assert it_na == it_ref
        err = float(torch.linalg.norm(x_na - x_ref) / torch.linalg.norm(x_ref))
        assert err <= REL_TOL, err
        xo = torch.from_numpy(x_or).cuda()
        assert float(torch.linalg.norm(x_na - xo) / torch.linalg.norm(xo)) <= REL_TOL
        # the host-driven per-phase kernels (what sizes beyond the cooperative
        # launch take) on the same array
        x_h, (it_h, st_h, _) = _solve_noalloc(A, val, b, 1e-10, flags=L.SLA_FLAG_NO_COOP)
        assert st_h == L.SLA_OK and abs(it_h - it_ref) <= 2
        err = float(torch.linalg.norm(x_h - x_ref) / torch.linalg.norm(x_ref))
        assert err <= REL_TOL, err
        assert float(torch.linalg.norm(x_h - xo) / torch.linalg.norm(xo)) <= REL_TOL


def test_noalloc_rejects_sizes_beyond_the_array():
    fake = ctypes.c_void_p(0x1000)
    A = L.SlaCsr(L.SLA_NOALLOC_MAX_N + 1, 7, fake, fake)
    o = L.SlaOpts(1e-8, 0.0, 100, 2, L.SLA_PRECOND_JACOBI, 0, 0)
    rc = L.lib().sla_cg_noalloc(ctypes.byref(A), fake, fake, ctypes.c_void_p(0x2000), ctypes.byref(o),
                                fake, None)
    assert rc == L.SLA_ERR_WORKSPACE
