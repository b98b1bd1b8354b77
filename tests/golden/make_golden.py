"""Writes the stored expected values used by the full-size parity tests and
by the CPU baseline.  Calls only the oracle and the seeded input generators.

  python tests/golden/make_golden.py diffusion3d 256
  python tests/golden/make_golden.py convdiff3d 128

``diffusion3d N`` writes tests/golden/oracle_diffusion3d_<N>.json with, for
the seeded 3D 7-point variable-coefficient system (faces exp(N(0,1)) from
seed 1, b ~ U[-1,1] from seed 11):
  - the oracle's Jacobi-PCG iteration count and residuals at rtol 1e-8,
  - the oracle's solution at rtol 1e-12 on 256 sampled indices,
  - the wall time of the oracle's rtol 1e-8 solve (single thread).

``convdiff3d N`` writes tests/golden/oracle_convdiff3d_<N>.json with, for
the 3D upwind convection-diffusion system at cell Peclet 10 (b ~ U[-1,1]
from seed 5), the oracle's right-preconditioned BiCGStab iteration count and
residuals at rtol 1e-8 and its solution at rtol 1e-12 (a warm continuation)
on 256 sampled indices.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2601_13994_b300 import inputs as I  # noqa: E402


def diffusion3d(N: int):
    rp, c, v = I.diffusion3d_random(N, 1)
    n = N ** 3
    b = I.rhs_uniform(n, 11)
    t0 = time.time()
    x8, info8 = oracle.pcg(rp, c, v, b, rtol=1e-8)
    t8 = time.time() - t0
    x12, info12 = oracle.pcg(rp, c, v, b, rtol=1e-12, x0=x8)
    idx = np.sort(np.random.default_rng(123).choice(n, 256, replace=False))
    out = {
        "workload": "diffusion3d_%d" % N,
        "recipe": "inputs.diffusion3d_random(N, seed=1), b = inputs.rhs_uniform(N^3, seed=11)",
        "n": n, "nnz": int(rp[-1]),
        "pcg_rtol_1e-8": {k: info8[k] for k in ("iters", "status", "rel_res", "true_rel_res")},
        "pcg_rtol_1e-8_seconds_single_thread": t8,
        "pcg_rtol_1e-12_warm": {k: info12[k] for k in ("iters", "status", "rel_res", "true_rel_res")},
        "sample_idx": idx.tolist(),
        "x_star_sample": x12[idx].tolist(),
        "x_star_norm2": float(np.linalg.norm(x12)),
    }
    path = os.path.join(HERE, "oracle_diffusion3d_%d.json" % N)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["pcg_rtol_1e-8"], t8)


def convdiff3d(N: int, peclet: float = 10.0):
    rp, c, v = I.convdiff3d(N, peclet)
    n = N ** 3
    b = I.rhs_uniform(n, 5)
    t0 = time.time()
    x8, info8 = oracle.bicgstab(rp, c, v, b, rtol=1e-8)
    t8 = time.time() - t0
    x12, info12 = oracle.bicgstab(rp, c, v, b, rtol=1e-12, x0=x8)
    idx = np.sort(np.random.default_rng(123).choice(n, 256, replace=False))
    out = {
        "workload": "convdiff3d_%d_pe%g" % (N, peclet),
        "recipe": "inputs.convdiff3d(N, peclet=%g), b = inputs.rhs_uniform(N^3, seed=5)" % peclet,
        "n": n, "nnz": int(rp[-1]),
        "bicgstab_rtol_1e-8": {k: info8[k] for k in ("iters", "status", "rel_res", "true_rel_res")},
        "bicgstab_rtol_1e-8_seconds_single_thread": t8,
        "bicgstab_rtol_1e-12_warm": {k: info12[k] for k in ("iters", "status", "rel_res", "true_rel_res")},
        "sample_idx": idx.tolist(),
        "x_star_sample": x12[idx].tolist(),
        "x_star_norm2": float(np.linalg.norm(x12)),
    }
    path = os.path.join(HERE, "oracle_convdiff3d_%d.json" % N)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["bicgstab_rtol_1e-8"], t8)


if __name__ == "__main__":
    kind, N = sys.argv[1], int(sys.argv[2])
    if kind == "diffusion3d":
        diffusion3d(N)
    elif kind == "convdiff3d":
        convdiff3d(N)
    else:
        raise SystemExit("unknown kind " + kind)
