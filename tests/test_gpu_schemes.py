"""Every SpMV scheme against the oracle: the solvers pick the row-per-thread
kernels at n <= 4 Mi rows and the TMA tile pipeline above; SLA_SPMV_KERNEL
forces one scheme for a whole process, so each scheme runs here in a child
process on small systems (SpMV, CG, BiCGStab, G G^T PCG; the solves with
cooperative=False, since at these sizes they would otherwise run as one
cooperative launch that does not use the SpMV kernels)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle
from paper_2601_13994_b300 import inputs as I, sla
out = {}
def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
rp, c, v = I.powerlaw_matrix(3000, 5)
x = I.rhs_uniform(3000, 6)
A = sla.CSRMatrix.from_numpy(rp, c)
y = sla.spmv(A, torch.from_numpy(v).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
out["spmv"] = rel(y, oracle.spmv(rp, c, v, x))
# misaligned arrays (views offset by one element): the TMA pipeline's bulk
# copies need 16-byte alignment, so every tile takes the warp-per-row path
cpad = torch.zeros(len(c) + 1, dtype=torch.int32, device="cuda"); cpad[1:] = torch.from_numpy(c).cuda()
vpad = torch.zeros(len(v) + 1, dtype=torch.float64, device="cuda"); vpad[1:] = torch.from_numpy(v).cuda()
rpad = torch.zeros(len(rp) + 1, dtype=torch.int32, device="cuda"); rpad[1:] = torch.from_numpy(rp).cuda()
Am = sla.CSRMatrix(rpad[1:], cpad[1:])
ym = sla.spmv(Am, vpad[1:], torch.from_numpy(x).cuda()).cpu().numpy()
out["spmv_misaligned"] = rel(ym, oracle.spmv(rp, c, v, x))
rp, c, v = I.diffusion3d_random(20, 3)
b = I.rhs_uniform(len(rp) - 1, 4)
A = sla.CSRMatrix.from_numpy(rp, c)
xg, info = sla.cg(A, torch.from_numpy(v).cuda(), torch.from_numpy(b).cuda(), rtol=1e-10, cooperative=False)
xo, io = oracle.pcg(rp, c, v, b, rtol=1e-13)
out["cg"] = [rel(xg.cpu().numpy(), xo), int(info.status)]
rp, c, v = I.convdiff3d(16, 10.0)
b = I.rhs_uniform(len(rp) - 1, 5)
A = sla.CSRMatrix.from_numpy(rp, c)
xg, info = sla.bicgstab(A, torch.from_numpy(v).cuda(), torch.from_numpy(b).cuda(), rtol=1e-10, cooperative=False)
xo, io = oracle.bicgstab(rp, c, v, b, rtol=1e-13)
out["bicgstab"] = [rel(xg.cpu().numpy(), xo), int(info.status)]
rp, c, v = I.diffusion2d_random(40, 5)
n = len(rp) - 1
d = v[c == np.repeat(np.arange(n), np.diff(rp))]
rows = np.repeat(np.arange(n), np.diff(rp))
keep = c <= rows
grp = np.zeros(n + 1, np.int32); np.add.at(grp, rows[keep] + 1, 1); grp = np.cumsum(grp).astype(np.int32)
gcol = c[keep].astype(np.int32)
gval = np.where(gcol == rows[keep], 1.0 / np.sqrt(d[rows[keep]]), -0.05 / np.sqrt(d[rows[keep]]))
b = I.rhs_uniform(n, 6)
G = sla.CSRMatrix.from_numpy(grp, gcol)
xg, info = sla.cg_ggt(A := sla.CSRMatrix.from_numpy(rp, c), torch.from_numpy(v).cuda(), G,
                      torch.from_numpy(gval).cuda(), torch.from_numpy(b).cuda(), rtol=1e-10, cooperative=False)
xo, io = oracle.pcg(rp, c, v, b, rtol=1e-13)
out["ggt"] = [rel(xg.cpu().numpy(), xo), int(info.status)]
print(json.dumps(out))
'''


@pytest.mark.parametrize("scheme", ["rows", "tma", "tile"])
def test_every_spmv_scheme_matches_oracle(scheme):
    env = dict(os.environ, SLA_SPMV_KERNEL=scheme)
    code = "ROOT = %r\n" % ROOT + CHILD
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    assert out["spmv"] <= 1e-14 and out["spmv_misaligned"] <= 1e-14
    for k in ("cg", "bicgstab", "ggt"):
        assert out[k][1] == 0, (k, out[k])
        assert out[k][0] <= 1e-8, (k, out[k])
