#!/usr/bin/env python
"""Benchmark of the Jacobi-PCG hot path on one B300 per rank.

Workload (one step = one full solve, inputs resident in HBM): the 3D 7-point
variable-coefficient diffusion operator on an N^3 interior grid (default
N = 464, the largest configuration: n = 99,897,344 unknowns, nnz =
697,989,632), face coefficients exp(N(0,1)) from seed 1, b ~ U[-1,1] from
seed 11, Jacobi-preconditioned CG from x0 = 0 to relative residual 1e-8
(recursive residual, then the true residual is recomputed).  The working set
(~20 GB) is far larger than L2, so no flush is needed between steps.

Ranks (torchrun) are independent replicas: each solves its own copy, no
collective touches the data path (the solve does not shard on one box).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (its OpenMP build on every host core), on bounded samples of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time to rel-res 1e-8 & SpMV GB/s vs 8 TB/s; learned vs Jacobi-PCG speedup"
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6400.0
# DRAM bytes (read + write) of one PCG iteration of the three per-phase kernels
# (K1 TMA SpMV, K2, K3 of CG on D^-1/2 A D^-1/2), captured by ncu at 176^3 (a
# small case under the capture size rule) and scaled by rows to the bench's
# N (traffic grows in proportion to the rows; profiles/pcg_iteration_diffusion3d_256.md);
# valid only for these kernels.
TRAFFIC_PER_ITER_176 = 918527488  # K1 561.3 MB + K2 268.0 MB + K3 89.2 MB, the kernels as they are
# FP64 peak: the driver measures none, so the run measures it itself
# (sla_fp64_probe: independent FMA chains on every SM at full occupancy, best
# of 5 after a warm-up, outside the timed region) and reports the derived
# figure beside it: 2 DFMA per clock per SM (ncu's peak_sustained for the
# FP64 pipe) x 148 SMs x 2 flop x 2.032 GHz.  The derived value stands until
# the probe has run (and where it cannot).
FP64_DERIVED_TFLOPS = 1.203
FP64_PEAK_TFLOPS = FP64_DERIVED_TFLOPS
FP64_PEAK_KIND = "derived: 2 DFMA/clk/SM (ncu FP64 pipe peak) x 148 SMs x 2 flop x 2.032 GHz"


def measure_fp64_peak(dev) -> None:
    """Sets FP64_PEAK_TFLOPS from the library's FP64 FMA probe."""
    global FP64_PEAK_TFLOPS, FP64_PEAK_KIND
    from paper_2601_13994_b300 import sla
    FP64_PEAK_TFLOPS = sla.fp64_peak_tflops(dev)
    FP64_PEAK_KIND = ("measured in this run: sla_fp64_probe (8 independent FMA chains a thread, 8 blocks of "
                      "256 a SM, best of 5); derived %.3f TFLOP/s" % FP64_DERIVED_TFLOPS)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=464, help="grid side N of the N^3 system")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--cpu-iters", type=int, default=0,
                    help="oracle iterations per CPU sample (0: pick from a time budget of ~10 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="end-to-end steps timed (at most --steps; each copies the inputs in)")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the solver kernels from a host loop instead of one graph (profiling)")
    ap.add_argument("--max-iter", type=int, default=None,
                    help="iteration cap (bounded profiling runs; the timed numbers are then not a solve)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other rows' measurements (BiCGStab, adjoint, batched)")
    ap.add_argument("--profile-row", choices=sorted(PROFILE_ROWS), default=None,
                    help="run one bounded solve of another row's workload from a host loop "
                         "(for ncu captures; default 20 iterations) and exit")
    return ap.parse_args()


def _profile_ggt(dev, max_iter, precond):
    """2D 1024^2 sigma = 1 (the learned preconditioner's unseen 2D system):
    G-PCG with an untrained but non-trivial head (the kernels' cost does not
    depend on the weights), or Jacobi-PCG; per-phase kernels from a host
    loop, or (coop, ggt_coop) the single cooperative launch."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import learned as LP
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion2d_random(1024, 900001, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(len(rp) - 1, 77)).to(dev)
    if precond == "jacobi":
        x, info = sla.cg(A, vt, bt, rtol=1e-8, max_iter=max_iter, graph=False)
    elif precond == "coop":
        # Jacobi-PCG as one cooperative launch (init, iterations, final residual)
        x, info = sla.cg(A, vt, bt, rtol=1e-8, max_iter=max_iter, max_restarts=0)
    else:
        m = LP.LearnedPreconditioner(device=dev, seed=0)
        m.view("v").fill_(0.05)
        m._sync_bf16()
        G, gv = m.factor(A, vt)
        if precond == "ggt_coop":
            x, info = sla.cg_ggt(A, vt, G, gv, bt, rtol=1e-8, max_iter=max_iter, max_restarts=0)
        else:
            x, info = sla.cg_ggt(A, vt, G, gv, bt, rtol=1e-8, max_iter=max_iter, graph=False)
    return {"iters": info.iters, "status": info.status}


def _profile_multi(dev, max_iter):
    """512^2 inverse-problem matrix at theta_true, 16 right-hand sides."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    from paper_2601_13994_b300.inverse import _selection, assemble_values
    N, k = 512, 16
    rp, c, _ = I.poisson2d(N)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    th = torch.from_numpy(I.gaussian_random_field(N, 4000)).to(dev)
    vals = assemble_values(th, _selection(N, dev)).contiguous()
    B = torch.from_numpy(I.rhs_uniform(N * N, 4001, batch=k)).to(dev)
    X, info = sla.cg_multi(A, vals, B, rtol=1e-8, max_iter=max_iter, graph=False)
    return {"iters": [int(i) for i in info.iters]}


def _profile_bicgstab(dev, max_iter):
    """3D convection-diffusion 128^3, cell Peclet 10 (the BiCGStab row)."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.convdiff3d(128, 10.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(len(rp) - 1, 5)).to(dev)
    x, info = sla.bicgstab(A, vt, bt, rtol=1e-8, max_iter=max_iter, graph=False)
    return {"iters": info.iters, "status": info.status}


def _profile_factor(dev, max_iter):
    """Learned-factor inference on the unseen 3D 128^3 system (features,
    three message-passing layers, head, column normalisation), twice; the
    network's weights do not change the kernels' cost."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import learned as LP
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion3d_random(128, 900002, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    m = LP.LearnedPreconditioner(device=dev, seed=0)
    m.view("v").fill_(0.05)
    m._sync_bf16()
    for _ in range(2):
        G, gv = m.factor(A, vt)
    torch.cuda.synchronize()
    return {"nnz_g": int(G.nnz)}


def _profile_fem_list(dev, max_iter):
    """512 P1 FEM systems, n log-uniform in [1e3, 5e4] (the distinct-pattern
    batch): block teams for the systems with at least 32768 entries, then the
    single-CTA kernel; max_iter bounds every system."""
    import numpy as np
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    mats = I.fem_list(512, seed0=2000)
    P = sla.CSRList([(m[0], m[1]) for m in mats], device=dev)
    vt = torch.from_numpy(np.concatenate([m[2] for m in mats])).to(dev)
    bt = torch.from_numpy(np.concatenate([I.rhs_uniform(len(m[0]) - 1, 3000 + s)
                                          for s, m in enumerate(mats)])).to(dev)
    x, info = sla.cg_batched_list(P, vt, bt, rtol=1e-8, max_iter=max_iter)
    return {"iters_max": int(np.atleast_1d(info.iters).max())}


def _profile_2d_512(dev, max_iter, pipelined):
    """2D 512^2 sigma = 1 (262,144 rows, in L2): Jacobi-PCG as one
    cooperative launch, standard (three grid barriers per iteration) or
    pipelined (one)."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion2d_random(512, 11, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(len(rp) - 1, 12)).to(dev)
    x, info = sla.cg(A, vt, bt, rtol=1e-8, max_iter=max_iter, max_restarts=0, pipelined=pipelined)
    return {"iters": info.iters, "status": info.status}


def _profile_eigsh(dev, max_iter):
    """LOBPCG for the 6 smallest eigenpairs of the 2D 128^2 variable-
    coefficient system (sigma = 1), max_iter iterations."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion2d_random(128, 11, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    lam, V, info = sla.eigsh(A, torch.from_numpy(v).to(dev), 6, tol=1e-8, max_iter=max_iter, strict=None)
    return {"iters": info.iters, "status": info.status}


def _profile_eigvec(dev, max_iter):
    """The eigenvector adjoint of the 6 smallest pairs of the 2D 128^2
    variable-coefficient system (sigma = 1): LOBPCG to 1e-8 (20000
    iterations at most), then one cooperative launch of the six deflated
    solves, at most max_iter iterations, for a random dL/dV (seed 5)."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion2d_random(128, 11, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    lam, V, _ = sla.eigsh(A, vt, 6, tol=1e-8, max_iter=20000, strict=None)
    gV = torch.from_numpy(np.random.default_rng(5).standard_normal((len(rp) - 1, 6))).to(dev)
    mu, info = sla.eig_vector_adjoint(A, vt, lam, V, gV, rtol=1e-10, max_iter=max_iter)
    torch.cuda.synchronize()
    return {"iters": [int(x) for x in np.atleast_1d(info.iters)], "status": [int(x) for x in np.atleast_1d(info.status)]}


PROFILE_ROWS = {
    "eigsh_2d_128": _profile_eigsh,
    "eigvec_adjoint_2d_128": _profile_eigvec,
    "coop_2d_512": lambda dev, mi: _profile_2d_512(dev, mi, False),
    "pipe_2d_512": lambda dev, mi: _profile_2d_512(dev, mi, True),
    "bicgstab_convdiff3d_128": _profile_bicgstab,
    "fem_list_512": _profile_fem_list,
    "factor_3d_128": _profile_factor,
    "ggt_2d_1024": lambda dev, mi: _profile_ggt(dev, mi, "ggt"),
    "jacobi_2d_1024": lambda dev, mi: _profile_ggt(dev, mi, "jacobi"),
    "coop_2d_1024": lambda dev, mi: _profile_ggt(dev, mi, "coop"),
    "ggt_coop_2d_1024": lambda dev, mi: _profile_ggt(dev, mi, "ggt_coop"),
    "multi_512x16": _profile_multi,
}


def workload(N: int):
    from paper_2601_13994_b300 import inputs as I
    rp, c, v = I.diffusion3d_random(N, 1)
    b = I.rhs_uniform(N ** 3, 11)
    return rp, c, v, b


def bytes_per_iter(n: int, nnz: int) -> int:
    """Algorithmic bytes of one Jacobi-PCG iteration as the per-phase kernels
    run it (int32 CSR, FP64; CG on D^-1/2 A D^-1/2): 12 nnz + 4 (n+1) for the
    matrix, 12 n-vector streams of 8 bytes (K1: p, q; K2: x rw, r rw, p, q,
    diag; K3: r, p rw)."""
    return 12 * nnz + 4 * (n + 1) + 96 * n


def flops_per_iter(n: int, nnz: int) -> int:
    """FP64 flops of one iteration: 2 per stored entry (SpMV) + 14 per row
    (p.q, two axpys, D^-1 r, r.z, r.r, p update; FMA = 2)."""
    return 2 * nnz + 14 * n


def spmv_bytes(n: int, nnz: int) -> int:
    return 12 * nnz + 4 * (n + 1) + 16 * n


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def golden(N: int):
    p = os.path.join(ROOT, "tests", "golden", "oracle_diffusion3d_%d.json" % N)
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.rows = []
        self.proc = None
        self.bus_id = bus_id

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(self.rows),
                "reasons": sorted(reasons)}


def bench_config(N: int, n: int, nnz: int, rtol: float) -> dict:
    """The workload description both arms print (same keys, same values)."""
    return {"workload": "diffusion3d_%d_jacobi_pcg_rtol%.0e" % (N, rtol), "n": n, "nnz": nnz,
            "precond": "jacobi", "x0": "zero",
            "l2": "inputs larger than L2 (%.1f GB working set)" % ((12 * nnz + 4 * n + 7 * 8 * n) / 1e9),
            "parallelism": "replicas"}


def host_cores() -> int:
    """Cores this process may run on (the all-core CPU baseline's threads)."""
    return len(os.sched_getaffinity(0))


def cpu_run(rp, c, v, b, iters: int, threads: int) -> float:
    """Seconds of one oracle run of `iters` Jacobi-PCG iterations on the full
    system (set-up, the iterations and the final residual), as it stands:
    threads == 1 the single-threaded oracle, else its OpenMP build."""
    import oracle
    t0 = time.perf_counter()
    if threads == 1:
        _, info = oracle.pcg(rp, c, v, b, rtol=0.0, atol=0.0, max_iter=iters, max_restarts=0)
    else:
        _, info = oracle.pcg_omp(rp, c, v, b, rtol=0.0, atol=0.0, max_iter=iters, max_restarts=0,
                                 threads=threads)
    assert info["iters"] == iters, info
    return time.perf_counter() - t0


class CpuLeg:
    """Time to solution of the oracle on a bounded sample of the workload: a
    1-iteration run and k-iteration runs give the cost of one iteration
    (difference quotient) and the fixed cost of a solve (set-up, initial and
    final residual); time to solution = fixed + per-iteration x the solve's
    iteration count (the oracle's own from tests/golden when stored)."""

    def __init__(self, rp, c, v, b, threads: int, budget_s: float):
        self.args = (rp, c, v, b)
        self.threads = threads
        t1 = cpu_run(rp, c, v, b, 1, threads)
        # a 1-iteration run costs about 3 iterations' worth (set-up + final residual)
        self.k = int(max(2, min(400, budget_s / max(t1 / 3.0, 1e-6))))
        self.t1 = t1
        self.per_iter = []

    def sample(self, k: int | None = None) -> float:
        k = k or self.k
        tk = cpu_run(*self.args, k, self.threads)
        s = max(tk - self.t1, 0.0) / (k - 1) if k > 1 else tk / 3.0
        self.per_iter.append(s)
        return s

    def summary(self, iters: int, iters_src: str, N: int) -> dict:
        s = statistics.median(self.per_iter)
        fixed = max(self.t1 - s, 0.0)
        return {"value": fixed + s * iters, "unit": "s", "cores": self.threads, "kind": "oracle",
                "seconds_per_iteration": s, "fixed_seconds": fixed,
                "sample": "%s oracle (%s) on the full %d^3 system: a 1-iteration run and %d run(s) of %d "
                          "iterations give %.3f s/iteration and %.2f s of fixed cost; time to solution = "
                          "fixed + s/iteration x %d iterations (%s)"
                          % ("single-threaded" if self.threads == 1 else "OpenMP (%d threads)" % self.threads,
                             "oracle/sla_oracle.c" if self.threads == 1 else "oracle/sla_oracle_omp.c",
                             N, len(self.per_iter), self.k, s, fixed, iters, iters_src)}


def _time(fn, reps=3, warm=1):
    """Median milliseconds of fn() over `reps` runs, CUDA events on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), out


def extra_rows(dev, args, peak):
    """Measurements of the other rows of the path on their own workloads
    (each after one warm-up run, median of 3, CUDA events)."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    out = {}
    # BiCGStab: 3D convection-diffusion 128^3, cell Peclet 10, rtol 1e-8
    rp, c, v = I.convdiff3d(128, 10.0)
    n, nnz = len(rp) - 1, int(rp[-1])
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(n, 5)).to(dev)
    ms, (x, info) = _time(lambda: sla.bicgstab(A, vt, bt, rtol=1e-8))
    # two SpMVs with A D^{-1} + 20 vector streams a row (p: r, p, v, p; v = A p: p,
    # r^, v; s: r, v, s; t = A s: s, s, t; x: x^, p, s, t, r^, x^, r)
    bpi = 2 * (12 * nnz + 4 * (n + 1)) + 160 * n
    gbs = bpi * info.iters / (ms / 1e3) / 1e9
    # the algorithmic model of a BiCGStab iteration the scope table gives:
    # two SpMVs and about 23 streams of n doubles
    bpi_model = 2 * (12 * nnz + 4 * n) + 23 * 8 * n
    gbs_model = bpi_model * info.iters / (ms / 1e3) / 1e9
    out["bicgstab_convdiff3d_128_pe10"] = {"s": ms / 1e3, "iters": info.iters, "status": info.status,
                                           "gbs": gbs, "frac_of_measured_hbm": gbs / peak,
                                           "bytes_per_iter": bpi,
                                           "bytes_per_iter_scope_model": bpi_model,
                                           "frac_of_measured_hbm_scope_model": gbs_model / peak}
    del A, vt, bt, x
    # 3D 256^3 (the previous headline size): the PCG solve with its roofline,
    # then the adjoint backward A^T lambda = 2x (L = sum x^2) + gradient pass
    N2 = 256
    rp, c, v, b = workload(N2)
    n, nnz = len(rp) - 1, int(rp[-1])
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(b).to(dev)
    ms, (x, info) = _time(lambda: sla.cg(A, vt, bt, rtol=args.rtol))
    gbs = bytes_per_iter(n, nnz) * info.iters / (ms / 1e3) / 1e9
    out["pcg_diffusion3d_%d" % N2] = {"s": ms / 1e3, "iters": info.iters, "status": info.status,
                                      "true_rel_res": info.true_rel_res, "gbs": gbs,
                                      "frac_of_measured_hbm": gbs / peak,
                                      "frac_of_8tbs": gbs / NOMINAL_HBM_GBS}
    g = 2 * x
    ms, (gb, gv, info) = _time(lambda: sla.adjoint_backward(A, vt, x, g, rtol=args.rtol))
    out["adjoint_backward_diffusion3d_%d" % N2] = {"s": ms / 1e3, "iters": info.iters,
                                                   "status": info.status}
    del A, vt, bt, x, g, gb, gv
    # batched, shared pattern: 1024 systems on the 64^2 five-point pattern
    B, N = 1024, 64
    rp, c, vals = I.batched_shared_2d(N, B, seed0=1000, sigma=0.5)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(vals).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(N * N, 7, batch=B)).to(dev)
    sla.cg_batched(A, vt, bt, rtol=1e-8, config="tune")
    ms, (x, info) = _time(lambda: sla.cg_batched(A, vt, bt, rtol=1e-8))
    its = np.atleast_1d(info.iters)
    fl = float((2 * int(rp[-1]) + 14 * N * N) * its.sum())
    tuned = sla.tuned_configs().get(("shared", N * N, int(rp[-1]), B))
    g2 = 2 * x  # dL/dx of L = sum x^2
    adj = batched_adjoint_row(lambda: sla.adjoint_backward_batched(A, vt, x, g2, rtol=1e-8),
                              (2 * int(rp[-1]) + 14 * N * N), 2 * B * int(rp[-1]))
    out["batched_shared_1024x64x64"] = {"s": ms / 1e3, "iters_mean": float(its.mean()), "adjoint": adj,
                                        "iters_max": int(its.max()),
                                        "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
                                        "fp64_tflops": fl / (ms / 1e3) / 1e12,
                                        "fp64_frac": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                                        "tuned_config": tuned,
                                        "tuned_shape": sla.config_shape(tuned) if tuned is not None else None,
                                        "candidates": len(sla.BATCH_CONFIGS)}
    del A, vt, bt, x
    # batched, distinct patterns: 512 P1 FEM systems, n log-uniform in [1e3, 5e4]
    mats = I.fem_list(512, seed0=2000)
    P = sla.CSRList([(m[0], m[1]) for m in mats], device=dev)
    vt = torch.from_numpy(np.concatenate([m[2] for m in mats])).to(dev)
    bt = torch.from_numpy(np.concatenate([I.rhs_uniform(len(m[0]) - 1, 3000 + s)
                                          for s, m in enumerate(mats)])).to(dev)
    sla.cg_batched_list(P, vt, bt, rtol=1e-8, config="tune")
    ms, (x, info) = _time(lambda: sla.cg_batched_list(P, vt, bt, rtol=1e-8))
    its = np.atleast_1d(info.iters)
    fl = 0.0
    for s, m in enumerate(mats):
        fl += (2 * int(m[0][-1]) + 14 * (len(m[0]) - 1)) * int(its[s])
    # the team launch with the standard and with the pipelined PCG (config bit 64)
    ms_std, _ = _time(lambda: sla.cg_batched_list(P, vt, bt, rtol=1e-8, config=0))
    ms_pipe, _ = _time(lambda: sla.cg_batched_list(P, vt, bt, rtol=1e-8, config=64))
    tuned = sla.tuned_configs().get(("list", P.n_max, P.total_rows, P.total_nnz, P.batch))
    g2 = 2 * x  # dL/dx of L = sum x^2
    adj = batched_adjoint_row(lambda: sla.adjoint_backward_batched_list(P, vt, x, g2, rtol=1e-8),
                              [(2 * int(m[0][-1]) + 14 * (len(m[0]) - 1)) for m in mats], 2 * P.total_nnz)
    out["batched_list_512_fem"] = {"s": ms / 1e3, "total_rows": P.total_rows, "iters_mean": float(its.mean()),
                                   "adjoint": adj,
                                   "tuned_config": tuned,
                                   "tuned_shape": sla.config_shape(tuned) if tuned is not None else None,
                                   "candidates": len(sla.LIST_CONFIGS),
                                   "teams_standard_s": ms_std / 1e3, "teams_pipelined_s": ms_pipe / 1e3,
                                   "iters_max": int(its.max()),
                                   "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
                                   "fp64_tflops": fl / (ms / 1e3) / 1e12,
                                   "fp64_frac": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    del P, vt, bt, x
    out.update(batched_bicgstab_rows(dev))
    out["distributed_emulated_diffusion3d_64_p8"] = distributed_row(dev)
    out["pipelined_vs_standard"] = pipelined_rows(dev)
    out["nonlinear_newton_512"] = nonlinear_row(dev)
    out["eigsh_2d_128_k6"] = eigen_row(dev)
    out["learned_vs_jacobi"] = learned_vs_jacobi(dev)
    out["inverse_512_16rhs"] = inverse_rows(dev, peak)
    return out


def batched_bicgstab_rows(dev):
    """Nonsymmetric batches by BiCGStab in one persistent launch (rtol 1e-8,
    tuned block size / vector placement): 1024 2D upwind convection-diffusion
    systems on one 64 x 64 five-point pattern (faces exp(N(0, 0.5^2)), cell
    Peclet up to 10 in a random direction, seeds 1000 + s), and 512 such
    systems on rectangles with n log-uniform in [1e3, 5e4] (seeds 5000 + s).
    FP64 operations per iteration and row: 2 SpMVs (2 nnz/n) + 15."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    out = {}
    B, N = 1024, 64
    rp, c, vals = I.batched_convdiff_2d(N, B, seed0=1000)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(vals).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(N * N, 7, batch=B)).to(dev)
    sla.bicgstab_batched(A, vt, bt, rtol=1e-8, config="tune")
    ms, (x, info) = _time(lambda: sla.bicgstab_batched(A, vt, bt, rtol=1e-8))
    its = np.atleast_1d(info.iters)
    fl = float((2 * 2 * int(rp[-1]) + 2 * 15 * N * N) * its.sum())
    g2 = 2 * x  # dL/dx of L = sum x^2
    adj = batched_adjoint_row(
        lambda: sla.adjoint_backward_batched(A, vt, x, g2, method="bicgstab", rtol=1e-8),
        (2 * 2 * int(rp[-1]) + 2 * 15 * N * N), 2 * B * int(rp[-1]))
    out["bicgstab_batched_shared_1024x64x64"] = {"adjoint": adj,
        "s": ms / 1e3, "iters_mean": float(its.mean()), "iters_max": int(its.max()),
        "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
        "fp64_tflops": fl / (ms / 1e3) / 1e12, "fp64_frac": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
        "tuned_config": sla.tuned_configs().get(("bicg_shared", N * N, int(rp[-1]), B))}
    del A, vt, bt, x
    mats = I.convdiff_list(512, seed0=5000)
    P = sla.CSRList([(m[0], m[1]) for m in mats], device=dev)
    vt = torch.from_numpy(np.concatenate([m[2] for m in mats])).to(dev)
    bt = torch.from_numpy(np.concatenate([I.rhs_uniform(len(m[0]) - 1, 6000 + s)
                                          for s, m in enumerate(mats)])).to(dev)
    sla.bicgstab_batched_list(P, vt, bt, rtol=1e-8, config="tune")
    ms, (x, info) = _time(lambda: sla.bicgstab_batched_list(P, vt, bt, rtol=1e-8))
    its = np.atleast_1d(info.iters)
    fl = 0.0
    for s, m in enumerate(mats):
        fl += (2 * 2 * int(m[0][-1]) + 2 * 15 * (len(m[0]) - 1)) * int(its[s])
    # one CTA per system (1024 threads, vectors in the workspace) against the
    # default block teams (3 blocks from 32768 entries)
    g2 = 2 * x  # dL/dx of L = sum x^2
    adj = batched_adjoint_row(
        lambda: sla.adjoint_backward_batched_list(P, vt, x, g2, method="bicgstab", rtol=1e-8),
        [(2 * 2 * int(m[0][-1]) + 2 * 15 * (len(m[0]) - 1)) for m in mats], 2 * P.total_nnz)
    ms_cta, _ = _time(lambda: sla.bicgstab_batched_list(P, vt, bt, rtol=1e-8, config=3 | 16 | 32))
    ms_team, _ = _time(lambda: sla.bicgstab_batched_list(P, vt, bt, rtol=1e-8, config=0))
    tuned = sla.tuned_configs().get(("bicg_list", P.n_max, P.total_rows, P.total_nnz, P.batch))
    out["bicgstab_batched_list_512_convdiff"] = {
        "s": ms / 1e3, "total_rows": P.total_rows, "iters_mean": float(its.mean()), "iters_max": int(its.max()),
        "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
        "fp64_tflops": fl / (ms / 1e3) / 1e12, "fp64_frac": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
        "tuned_config": tuned, "tuned_shape": sla.bicg_list_shape(tuned) if tuned is not None else None,
        "candidates": len(sla.BICG_LIST_CONFIGS), "one_cta_s": ms_cta / 1e3, "teams_default_s": ms_team / 1e3,
        "adjoint": adj}
    return out


def batched_adjoint_row(run, flops_per_iter, grad_flops):
    """The batch's backward pass for L = sum x^2 (one call of
    sla_adjoint_backward_batched_*: every system's adjoint solve in one
    launch, then the gradient pass), timed with CUDA events.  flops_per_iter:
    FP64 operations of one iteration, for every system alike (a number) or
    per system (a list); grad_flops: those of the gradient pass."""
    ms, (gb, gv, info) = _time(run)
    its = np.atleast_1d(info.iters)
    per = np.asarray(flops_per_iter, dtype=np.float64)
    fl = float((per * its).sum()) + grad_flops
    return {"s": ms / 1e3, "iters_mean": float(its.mean()), "iters_max": int(its.max()),
            "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
            "fp64_tflops": fl / (ms / 1e3) / 1e12, "fp64_frac": fl / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS}


def distributed_row(dev, N=64, P=8):
    """Sec. 3.3's distributed CG (Algorithm 1) with 8 row-block partitions
    emulated on one GPU, on the 3D 64^3 variable-coefficient system at rtol
    1e-8, against the single-system solve: iterations, time (the emulation
    reads its two all-reduced scalars on the host every iteration, as the
    algorithm's ranks receive them) and the halo sizes."""
    import torch

    from paper_2601_13994_b300 import distributed as D
    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion3d_random(N, 1)
    n = len(rp) - 1
    vt = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(I.rhs_uniform(n, 11)).to(dev)
    DA = D.DistributedMatrix(rp, c, P, device=dev)
    ms_d, (xd, inf) = _time(lambda: D.dist_cg(DA, vt, bt, rtol=1e-8))
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    ms_s, (xs, ins) = _time(lambda: sla.cg(A, vt, bt, rtol=1e-8))
    return {"n": n, "partitions": P, "halo_sizes": inf["halo_sizes"], "halo_fraction": sum(inf["halo_sizes"]) / n,
            "dist_s": ms_d / 1e3, "dist_iters": inf["iters"], "dist_status": inf["status"],
            "dist_true_rel_res": inf["true_rel_res"], "single_s": ms_s / 1e3, "single_iters": ins.iters,
            "max_abs_diff": float((xd - xs).abs().max())}


def eigen_row(dev, N=128, k=6):
    """Sec. 3.2 / Tab. 5 eigenvalue path: the 6 smallest eigenpairs of the
    2D 128^2 variable-coefficient system (sigma = 1) by LOBPCG with the
    Jacobi preconditioner to relative residual 1e-8, then the Hellmann-
    Feynman gradient of sum(lambda) on the pattern, and the eigenvector
    adjoint for a random dL/dV (the six deflated solves to 1e-10 in one
    cooperative launch, then -mu v^T on the pattern).  Median of 3 after one
    warm-up (the eigsh call synchronises its stream)."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    rp, c, v = I.diffusion2d_random(N, 11, 1.0)
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    vt = torch.from_numpy(v).to(dev)
    ms, (lam, V, info) = _time(lambda: sla.eigsh(A, vt, k, tol=1e-8))
    g = torch.ones(k, dtype=torch.float64, device=dev)
    gms, _ = _time(lambda: sla.eig_grad_values(A, V, g), reps=5)
    gV = torch.from_numpy(np.random.default_rng(5).standard_normal((len(rp) - 1, k))).to(dev)

    def vec_backward():
        mu, inf = sla.eig_vector_adjoint(A, vt, lam, V, gV, rtol=1e-10)
        return sla.eig_vector_grad_values(A, mu, V), inf
    vms, (_, vinfo) = _time(vec_backward)
    return {"n": len(rp) - 1, "k": k, "s": ms / 1e3, "iters": info.iters, "status": info.status,
            "us_per_iter": 1e3 * ms / max(info.iters, 1), "true_rel_res": info.true_rel_res,
            "lambda": [float(x) for x in lam.cpu()], "grad_ms": gms,
            "eigvec_adjoint_ms": vms, "eigvec_adjoint_iters": [int(x) for x in np.atleast_1d(vinfo.iters)],
            "eigvec_adjoint_status": [int(x) for x in np.atleast_1d(vinfo.status)],
            "eigvec_adjoint_us_per_iter": 1e3 * vms / max(int(np.max(vinfo.iters)), 1)}


def nonlinear_row(dev, N=512):
    """Sec. 3.2 / Tab. 5 nonlinear path on 512^2 cells: Newton from u = 0 on
    F = A(theta) u + h^2 (gamma u^3 - f) (gamma = 10, theta a smooth random
    field), every step's Jacobian from coloured Jacobian-vector products and
    its solve by Jacobi-PCG (rtol 1e-10), to ||F|| <= 1e-10 ||F(0)||; then the
    backward pass, one adjoint solve plus one vector-Jacobian product.
    Median of 3 after one warm-up, CUDA events around forward and backward."""
    import torch

    from paper_2601_13994_b300 import nonlinear as NL
    P = NL.SemilinearDiffusion(N=N, device=dev)
    opts = dict(tol=1e-10, lin_rtol=1e-10)
    ut = P.target(**opts)
    fw, bw = [], []
    for rep in range(4):
        th = P.theta0.clone().requires_grad_(True)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        L = P.loss(th, ut, **opts)
        e1.record()
        L.backward()
        e2.record()
        e2.synchronize()
        if rep:
            fw.append(e0.elapsed_time(e1))
            bw.append(e1.elapsed_time(e2))
    info = P.jac.last_info
    return {"n": P.n, "gamma": P.gamma, "colours": P.jac.ncolours, "newton_iters": info.newton_iters,
            "krylov_iters": info.krylov_iters, "residual_drop": info.residual_norms[-1] / info.residual_norms[0],
            "forward_ms": statistics.median(fw), "backward_ms": statistics.median(bw), "loss": float(L.detach()),
            "backward_over_forward": statistics.median(bw) / statistics.median(fw)}


def pipelined_rows(dev):
    """Jacobi-PCG in one cooperative launch: the standard form (three grid
    barriers per iteration) against the pipelined form (one merged reduction
    and one barrier per iteration), on the 2D Poisson 64^2 system (rtol
    1e-10) and on variable-coefficient systems of 2D 512^2 and 3D 64^3
    (sigma = 1, rtol 1e-8).  Median of 3 solves after one warm-up each."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import sla
    cases = [("poisson2d_64", lambda: I.poisson2d(64), 1e-10),
             ("diffusion2d_512", lambda: I.diffusion2d_random(512, 11, 1.0), 1e-8),
             ("diffusion3d_64", lambda: I.diffusion3d_random(64, 1), 1e-8)]
    res = {}
    for name, gen, rtol in cases:
        rp, c, v = gen()
        n, nnz = len(rp) - 1, int(rp[-1])
        A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
        vt = torch.from_numpy(v).to(dev)
        bt = torch.from_numpy(I.rhs_uniform(n, 12)).to(dev)
        row = {}
        for tag, kw in (("standard", {}), ("pipelined", {"pipelined": True})):
            ms, (x, info) = _time(lambda: sla.cg(A, vt, bt, rtol=rtol, **kw))
            row[tag] = {"ms": ms, "iters": info.iters, "status": info.status,
                        "us_per_iter": 1e3 * ms / max(info.iters, 1), "true_rel_res": info.true_rel_res}
        row["speedup"] = row["standard"]["ms"] / row["pipelined"]["ms"]
        row["n"], row["nnz"], row["rtol"] = n, nnz, rtol
        res[name] = row
    return res


def inverse_rows(dev, peak, N=512, k=16):
    """Config 4: 2D inverse coefficient problem on 512^2 cells with 16
    right-hand sides.  Times (a) the 16-column PCG to rtol 1e-8 at the true
    field against 16 single-column solves of the same systems and (b) one
    loss + gradient step (multi-RHS forward, multi-RHS adjoint, autograd
    through the assembly) at theta = 0."""
    import torch

    from paper_2601_13994_b300 import sla
    from paper_2601_13994_b300.inverse import InverseProblem
    P = InverseProblem(N, k, device=dev)
    vals = P.values(P.theta_true)
    ms_m, (X, info) = _time(lambda: sla.cg_multi(P.A, vals, P.B, rtol=1e-8))
    its = np.atleast_1d(info.iters)

    def singles():
        return [sla.cg(P.A, vals, P.B[j].contiguous(), rtol=1e-8) for j in range(k)]

    ms_s, outs = _time(singles)
    n, nnz = P.n, P.A.nnz
    bpi = 12 * nnz + 4 * (n + 1) + 104 * n * k
    gbs = bpi * int(its.max()) / (ms_m / 1e3) / 1e9
    # FP64 flops: every column's SpMV (2 nnz) and vector work (14 n) for the
    # iterations that column ran
    fl = float(sum((2 * nnz + 14 * n) * int(i) for i in its))
    fp64_tf = fl / (ms_m / 1e3) / 1e12
    th0 = torch.zeros((N, N), dtype=torch.float64, device=dev)

    def step():
        t = th0.clone().requires_grad_(True)
        L = P.loss(t)
        L.backward()
        return L.detach()

    ms_step, L = _time(step)
    return {"n": n, "k": k, "multi_s": ms_m / 1e3, "iters_max": int(its.max()), "iters_mean": float(its.mean()),
            "all_ok": bool((np.atleast_1d(info.status) == 0).all()),
            "us_per_iter": ms_m * 1e3 / int(its.max()), "gbs_model": gbs, "frac_of_measured_hbm": gbs / peak,
            "fp64_tflops": fp64_tf, "fp64_frac": fp64_tf / FP64_PEAK_TFLOPS,
            "bytes_per_iter": bpi, "singles_s": ms_s / 1e3,
            "singles_iters": [int(o[1].iters) for o in outs], "speedup_vs_singles": ms_s / ms_m,
            "step_s": ms_step / 1e3, "loss_theta0": float(L)}


def learned_vs_jacobi(dev, systems=48, steps=800, lr=3e-3, n_lo=64, n_hi=128, evals=None, scale_free=False,
                      normalised=False):
    """Config 5: train the learned G G^T preconditioner (seeded, on systems the
    library's CG solves), then time PCG to rtol 1e-8 with it and with Jacobi on
    unseen systems; the FP64 true residual is checked by the solver."""
    import torch

    from paper_2601_13994_b300 import inputs as I
    from paper_2601_13994_b300 import learned as LP
    from paper_2601_13994_b300 import sla
    model = LP.LearnedPreconditioner(device=dev, seed=0)
    zero = LP.LearnedPreconditioner(device=dev, seed=0)  # untrained: zero head
    t0 = time.perf_counter()
    hist = LP.train(model, systems=systems, steps=steps, lr=lr, n_lo=n_lo, n_hi=n_hi, log_every=max(1, steps // 8),
                    scale_free=scale_free, normalised=normalised)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # the scale-free loss (A-norm error of the best multiple of G G^T b) of
    # the normalised factors PCG uses on the training systems: trained,
    # untrained (zero head: Jacobi) and FSAI; and of the trained network's
    # factor before its columns are normalised
    ev = {"trained": LP.evaluate(model, systems, n_lo, n_hi),
          "trained_unnormalised": LP.evaluate(model, systems, n_lo, n_hi, normalize=False),
          "zero_head": LP.evaluate(zero, systems, n_lo, n_hi),
          "fsai": LP.evaluate(zero, systems, n_lo, n_hi, fsai=True)}
    out = {"train": {"systems": systems, "steps": steps, "grid": [n_lo, n_hi], "seconds": t_train,
                     "loss": ("scale-free" if scale_free else "plain")
                     + (", of the normalised factor" if normalised else ""),
                     "loss_first": hist[0], "loss_last": hist[-1], "scale_free_loss_normalised": ev}}
    evals = evals or [("2d_1024_sigma1", lambda: I.diffusion2d_random(1024, 900001, 1.0)),
                      ("3d_128_sigma1", lambda: I.diffusion3d_random(128, 900002, 1.0))]
    for name, gen in evals:
        rp, c, v = gen()
        A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
        vt = torch.from_numpy(v).to(dev)
        bt = torch.from_numpy(I.rhs_uniform(len(rp) - 1, 77)).to(dev)
        ms_j, (xj, ij) = _time(lambda: sla.cg(A, vt, bt, rtol=1e-8))
        ms_f, fac = _time(lambda: model.factor(A, vt))
        ms_g, (xg, ig) = _time(lambda: sla.cg_ggt(A, vt, fac[0], fac[1], bt, rtol=1e-8))
        # the same G-PCG with the factor of an untrained network (zero head:
        # G = D^{-1/2}, normalisation keeps it, i.e. Jacobi through the G
        # kernels) and with the classical FSAI factor on the same pattern
        ms_z, zfac = _time(lambda: zero.factor(A, vt))
        ms_gz, (_, iz) = _time(lambda: sla.cg_ggt(A, vt, zfac[0], zfac[1], bt, rtol=1e-8))
        ms_ff, ffac = _time(lambda: LP.fsai_factor(A, vt))
        ms_gf, (_, iff) = _time(lambda: sla.cg_ggt(A, vt, ffac[0], ffac[1], bt, rtol=1e-8))
        out[name] = {"jacobi_s": ms_j / 1e3, "jacobi_iters": ij.iters, "learned_s": ms_g / 1e3,
                     "learned_iters": ig.iters, "learned_status": ig.status,
                     "learned_true_rel_res": ig.true_rel_res, "factor_s": ms_f / 1e3,
                     "iters_ratio": ij.iters / max(1, ig.iters), "speedup_solve": ms_j / ms_g,
                     "speedup_with_factor": ms_j / (ms_g + ms_f),
                     "zero_head": {"s": ms_gz / 1e3, "iters": iz.iters, "status": iz.status,
                                   "factor_s": ms_z / 1e3},
                     "fsai": {"s": ms_gf / 1e3, "iters": iff.iters, "status": iff.status,
                              "factor_s": ms_ff / 1e3, "jacobi_fallback_columns": ffac[2],
                              "speedup_with_factor": ms_j / (ms_gf + ms_ff)},
                     "learned_vs_fsai_with_factor": (ms_gf + ms_ff) / (ms_g + ms_f)}
    return out


def run_reference(args):
    """The reference arm: the oracle as it stands, timed on the host's cores
    (its OpenMP build on every core this process may use; the line's value),
    each step a bounded sample of the workload, plus one bounded sample of
    the single-threaded oracle.  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    N = args.size
    rp, c, v, b = workload(N)
    n, nnz = len(rp) - 1, int(rp[-1])
    g = golden(N)
    iters_solve = g["pcg_rtol_1e-8"]["iters"] if g else None
    iters_src = "the oracle's own at rtol 1e-8, tests/golden" if g else "unknown: no stored oracle count"
    cores = host_cores()
    # the timed steps share ~90 s of CPU work
    leg = CpuLeg(rp, c, v, b, cores, budget_s=90.0 / max(1, args.steps))
    if args.cpu_iters:
        leg.k = max(2, args.cpu_iters)
    for _ in range(args.warmup):
        cpu_run(rp, c, v, b, 2, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        leg.sample()
    wall = time.perf_counter() - t0
    base = leg.summary(iters_solve or 0, iters_src, N)
    single = None
    if not args.no_cpu_baseline:
        one = CpuLeg(rp, c, v, b, 1, budget_s=12.0)
        one.sample()
        single = one.summary(iters_solve or 0, iters_src, N)
    value = base["value"] if iters_solve else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(N, n, nnz, args.rtol),
        "seconds_per_iteration": base["seconds_per_iteration"],
        "cpu_baseline": base,
        "cpu_baseline_single_thread": single,
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The job's time for a per-rank time: the slowest rank's (an all-reduce
    MAX over the process group; the value itself with one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2601_13994_b300 import sla

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    N = args.size
    rp, c, v, b = workload(N)
    n, nnz = len(rp) - 1, int(rp[-1])
    A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
    val = torch.from_numpy(v).to(dev)
    bt = torch.from_numpy(b).to(dev)
    stream = torch.cuda.current_stream(dev)

    # ---- warm-up and timed solves (device-resident inputs)
    solve_kw = {"rtol": args.rtol, "graph": not args.host_loop, "max_iter": args.max_iter}
    for _ in range(args.warmup):
        x, info = sla.cg(A, val, bt, **solve_kw)
    torch.cuda.synchronize(dev)
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        pass
    sampler = ClockSampler(bus) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        x, info = sla.cg(A, val, bt, **solve_kw)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = sampler.stop() if sampler else None
    ms_max = max_over_ranks(ms, world, dev)
    iters_all = [i.iters for i in infos]
    status_all = [i.status for i in infos]
    true_rel = infos[-1].true_rel_res

    # ---- standalone SpMV (same row-tile code as the solver's K1), events on its stream
    xs = torch.from_numpy(np.random.default_rng(0).uniform(-1, 1, n)).to(dev)
    ys = torch.empty_like(xs)
    for _ in range(3):
        sla.spmv(A, val, xs, out=ys)
    reps = 20
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(reps):
        sla.spmv(A, val, xs, out=ys)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    spmv_ms = s0.elapsed_time(s1) / reps

    # ---- end to end through the public call with host buffers
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(rp).pin_memory()
        h_c = torch.from_numpy(c).pin_memory()
        h_v = torch.from_numpy(v).pin_memory()
        h_b = torch.from_numpy(b).pin_memory()
        h_x = torch.empty(n, dtype=torch.float64).pin_memory()
        d_rp = torch.empty_like(h_rp, device=dev)
        d_c = torch.empty_like(h_c, device=dev)
        d_v = torch.empty_like(h_v, device=dev)
        d_b = torch.empty_like(h_b, device=dev)

        def e2e_step():
            d_rp.copy_(h_rp, non_blocking=True)
            d_c.copy_(h_c, non_blocking=True)
            d_v.copy_(h_v, non_blocking=True)
            d_b.copy_(h_b, non_blocking=True)
            Ad = sla.CSRMatrix(d_rp, d_c, check=False)
            xd, inf = sla.cg(Ad, d_v, d_b, **solve_kw)
            h_x.copy_(xd, non_blocking=True)
            return inf

        e2e_step()
        torch.cuda.synchronize(dev)
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(e2e_steps):
            inf = e2e_step()
        k1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        e2e_ms = max_over_ranks(k0.elapsed_time(k1) / e2e_steps, world, dev)
        h2d = rp.nbytes + c.nbytes + v.nbytes + b.nbytes
        d2h = 8 * n + 24  # x and the info record
        # the host-to-device copies alone (the link is shared with the other
        # GPUs of the host, so their rate varies between machines and runs)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for d_t, h_t in ((d_rp, h_rp), (d_c, h_c), (d_v, h_v), (d_b, h_b)):
            d_t.copy_(h_t, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        h2d_ms = c0.elapsed_time(c1)
        e2e = {"value": e2e_ms / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "iters": inf.iters, "steps": e2e_steps,
               "h2d_ms": h2d_ms, "h2d_gbs": h2d / (h2d_ms / 1e3) / 1e9}

    peak, peak_kind = measured_peaks()
    measure_fp64_peak(dev)
    it = statistics.median(iters_all)
    bpi = bytes_per_iter(n, nnz)
    achieved = bpi * it / (ms_max / 1e3) / 1e9
    fpi = flops_per_iter(n, nnz)
    fp64_tf = fpi * it / (ms_max / 1e3) / 1e12
    spmv_gbs = spmv_bytes(n, nnz) / (spmv_ms / 1e3) / 1e9
    # per solve: descriptor write, init, scale (D^-1/2 A D^-1/2), unscale, final, and
    # three kernels per loop body (the iterations and the true-residual check)
    launches = args.steps * (1 + 4 + 3 * (it + 1))

    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g = golden(N)
        oracle_iters = g["pcg_rtol_1e-8"]["iters"] if g else None
        used = oracle_iters if oracle_iters else int(it)
        src = "the oracle's own at rtol 1e-8, tests/golden" if oracle_iters else "the GPU solve's"
        # all host cores (OpenMP build), then one core (the plain oracle); ~10-15 s each
        legs = []
        for threads, budget in ((host_cores(), 10.0), (1, 12.0)):
            leg = CpuLeg(rp, c, v, b, threads, budget_s=budget)
            if args.cpu_iters:
                leg.k = max(2, args.cpu_iters)
            leg.sample()
            legs.append(leg.summary(used, src, N))
        cpu, cpu1 = legs
    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = extra_rows(dev, args, peak)
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": ms_max / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(N, n, nnz, args.rtol),
        "iters": it, "status": sorted(set(status_all)), "true_rel_res": true_rel,
        "pcg_gbs": achieved, "pcg_frac_of_8tbs": achieved / NOMINAL_HBM_GBS,
        "spmv_gbs": spmv_gbs, "spmv_frac_of_8tbs": spmv_gbs / NOMINAL_HBM_GBS,
        "spmv_ms": spmv_ms,
        "fp64": {"achieved_tflops": fp64_tf, "peak_tflops": FP64_PEAK_TFLOPS, "peak_kind": FP64_PEAK_KIND,
                 "frac": fp64_tf / FP64_PEAK_TFLOPS, "derived_peak_tflops": FP64_DERIVED_TFLOPS,
                 "flops_per_iter": fpi},
        "roofline": {"kernel": "Jacobi-PCG iteration (cg_spmv_pq + cg_update + cg_pupdate)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_launch": bpi,
                     "traffic": TRAFFIC_PER_ITER_176 * (N / 176.0) ** 3 if N >= 176 else None,
                     "traffic_unit": "bytes per iteration (3 kernels), ncu at 176^3 scaled by rows"},
        "roofline_spmv": {"kernel": "spmv_tma_kernel", "bound": "hbm", "achieved": spmv_gbs, "peak": peak,
                          "unit": "GB/s", "frac": spmv_gbs / peak, "bytes_per_launch": spmv_bytes(n, nnz)},
        "cpu_baseline": cpu,
        "cpu_baseline_single_thread": cpu1,
        "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "extra": extra,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.profile_row is not None:
        import torch
        dev = torch.device("cuda", 0)
        out = PROFILE_ROWS[args.profile_row](dev, args.max_iter or 20)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_row": args.profile_row, **out}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
