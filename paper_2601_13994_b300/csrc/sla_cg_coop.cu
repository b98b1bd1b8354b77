// sla_cg_coop.cu -- PCG in one cooperative launch per solve: Jacobi PCG
// (as sla_cg) and G G^T PCG (as sla_cg_ggt).
//
// The methods, state machines and exits are those of the graph loops in
// sla_cg.cu and sla_cg_ggt.cu (Algorithm 1; the Jacobi preconditioner of
// Sec. 4.1, or z = G (G^T r); initial check, iterations, true-residual check
// with restart, final residual).  This form is for systems of up to a few
// million rows, where a kernel boundary inside the graph (launch, ramp-up,
// drain) is a large share of an iteration.  Every block stays resident for
// the whole solve -- a cooperative launch guarantees it -- and each kernel
// boundary becomes a grid barrier (grid_sync).
//
// Ownership: thread g of the T threads of the grid owns rows g, g + T, ... in
// every phase, so the streaming updates touch only the thread's own rows,
// and the only data that crosses threads are the SpMV gathers (p, r, t; x in
// the residual checks) and the per-block partial sums, each read after a
// barrier and never through the read-only (non-coherent) path.
//
// Reductions: each block writes its partial sums, a barrier follows, then
// every block adds all partials in the same fixed order, so every block
// holds the same bits of alpha, beta and of each convergence test and takes
// the same branch with no further synchronisation.  Partials alternate
// between two buffers, so a block that starts the next reduction never
// overwrites values a slower block is still reading.
//
// Jacobi iteration: q = A p and p.q | reduce | x += alpha p, r -= alpha q,
// z = D^{-1} r, r.z, r.r | reduce | p = z + beta p | barrier.
// G G^T iteration: q = A p and p.q | reduce | x += alpha p, r -= alpha q,
// r.r | barrier | t = G^T r, t.t | reduce (t.t, r.r) | p = G t + beta p |
// barrier (the graph form reduces r.r in a kernel of its own).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "sla_cg_pipe.cuh"
#include "sla_coop.cuh"

namespace sla {

struct CoopArgs {
  KrylovDesc d;
  KrylovState* st;
  double* part;
  double* r;
  double* z;
  double* p;
  double* q;
  double* dinv;
};

// Block-uniform solver scalars, kept in shared memory (written by thread 0
// after each grid reduction, read by all threads after a block barrier):
// registers are the limit on resident threads here.
struct CoopState {
  double bnorm, thresh, rho, rr, alpha, beta, ttt;
  long long body;
  int iters, restarts, status, phase, zero_rhs, bad;
};

// Decisions after the initial sums (||b||^2, ||r||^2, r.z, bad diagonal).
__device__ __forceinline__ void coop_after_init(CoopState& s, const double* t, const KrylovDesc& d) {
  s.bnorm = sqrt(t[0]);
  s.thresh = fmax(d.rtol * s.bnorm, d.atol);
  s.rho = t[2];
  s.rr = t[1];
  s.alpha = s.beta = s.ttt = 0.0;
  s.body = 0;
  s.iters = s.restarts = s.zero_rhs = s.bad = 0;
  s.status = SLA_NOT_CONVERGED;
  s.phase = kPhaseRun;
  if (t[3] > 0.0) {
    s.bad = 1;
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else if (s.bnorm == 0.0) {
    s.zero_rhs = 1;
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(t[2]) || !isfinite(t[1])) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(t[1]) <= s.thresh) {
    s.phase = kPhaseCheck;
  } else if (d.max_iter <= 0) {
    s.phase = kPhaseDone;
  }
}

// After p.q: alpha, or the end of the solve on a breakdown.
__device__ __forceinline__ void coop_after_pq(CoopState& s, double tpq) {
  if (!isfinite(tpq)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (!(tpq > 0.0)) {
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else {
    s.alpha = s.rho / tpq;
  }
}

// After r.z and r.r: convergence of the recursive residual, beta.
__device__ __forceinline__ void coop_after_update(CoopState& s, double trz, double trr, const KrylovDesc& d) {
  s.iters += 1;
  s.rr = trr;
  if (!isfinite(trz) || !isfinite(trr)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(trr) <= s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseCheck;
  } else if (!(trz > 0.0)) {
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else {
    s.beta = trz / s.rho;
    s.rho = trz;
    if (s.iters >= d.max_iter) {
      s.status = SLA_NOT_CONVERGED;
      s.phase = kPhaseDone;
    }
  }
}

// End of a loop body: hard cap on bodies (each one advances iters or
// consumes a restart, so this only fires if the state machine is broken).
__device__ __forceinline__ void coop_end_body(CoopState& s, const KrylovDesc& d) {
  s.body += 1;
  const long long cap = (long long)d.max_iter + 2LL * d.max_restarts + 8;
  if (s.phase != kPhaseDone && s.body > cap) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  }
}

// After the true-residual check (t.t, t.z): done, or restart from t.
__device__ __forceinline__ void coop_after_check(CoopState& s, double ttt, double trz, const KrylovDesc& d) {
  if (sqrt(ttt) <= 2.0 * s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(ttt) || !isfinite(trz)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (s.restarts >= d.max_restarts || s.iters >= d.max_iter) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  } else {
    s.restarts += 1;
    s.rho = trz;
    s.rr = ttt;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseRun;
  }
}

// One Jacobi-PCG solve by a team; d (shared memory) describes the system,
// r, z, p, q, dinv are its n-vectors.  Rank 0 writes *d.info.  Returns
// false if a barrier ran out (the caller must then leave the kernel).
// check_err: also report a timeout flagged by any block of the launch.
__device__ __forceinline__ bool jacobi_team_solve(const KrylovDesc& d, double* r, double* z, double* p, double* q,
                                                  double* dinv, Team& tm, bool check_err, CoopSmem& sm,
                                                  CoopState& s) {
  const int n = d.n;
  const int T = tm.size * kCoopThreads;
  const int g0 = tm.rank * kCoopThreads + threadIdx.x;
  const bool t0 = threadIdx.x == 0;
  int buf = 0;
  bool ok = true;
  auto col_at = [&](int k) { return __ldg(d.col + k); };
  auto val_at = [&](int k) { return __ldg(d.val + k); };

  // ---- init: dinv, r = b - A x0, z = D^{-1} r, p = z; ||b||^2, ||r||^2, r.z, bad diagonal
  {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = g0; i < n; i += T) {
      const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
      double diag = 0.0, ax = 0.0;
      for (int j = a; j < e; ++j) {
        const int c = __ldg(d.col + j);
        const double v = __ldg(d.val + j);
        if (c == i) diag += v;
        if (d.use_x0) ax = fma(v, d.x[c], ax);
      }
      const double bi = __ldg(d.b + i);
      const double ri = bi - ax;
      double di = 1.0;
      if (d.precond == SLA_PRECOND_JACOBI) {
        if (!(diag > 0.0)) acc[3] = 1.0;
        di = 1.0 / diag;
      }
      const double zi = di * ri;
      dinv[i] = di;
      r[i] = ri;
      z[i] = zi;
      p[i] = zi;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
      acc[2] = fma(ri, zi, acc[2]);
    }
    if (!d.use_x0)
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    ok = coop_sums(acc, tm, buf, sm);
    if (ok && t0) coop_after_init(s, acc, d);
    __syncthreads();
  }

  // ---- iterations
  while (ok && s.phase != kPhaseDone) {
    if (s.phase == kPhaseRun) {
      // q = A p, p.q
      {
        double v[1] = {0.0};
        coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
          const double y = row_sum_batched(a, e, col_at, val_at, Coherent{p});
          q[i] = y;
          v[0] = fma(p[i], y, v[0]);
        });
        if (!(ok = coop_sums(v, tm, buf, sm))) break;
        if (t0) coop_after_pq(s, v[0]);
        __syncthreads();
        if (s.phase == kPhaseDone) break;
      }
      // x += alpha p, r -= alpha q, z = D^{-1} r; r.z, r.r
      {
        const double alpha = s.alpha;
        double v[2] = {0.0, 0.0};
        for (int i0 = g0; i0 < n; i0 += kCoopUnroll * T) {
          double pi[kCoopUnroll], qi[kCoopUnroll], di[kCoopUnroll], xi[kCoopUnroll], ri[kCoopUnroll];
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) {
              pi[u] = p[i];
              qi[u] = q[i];
              di[u] = dinv[i];
              xi[u] = d.x[i];
              ri[u] = r[i];
            }
          }
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) {
              const double xn = fma(alpha, pi[u], xi[u]);
              const double rn = fma(-alpha, qi[u], ri[u]);
              const double zn = di[u] * rn;
              d.x[i] = xn;
              r[i] = rn;
              z[i] = zn;
              v[0] = fma(rn, zn, v[0]);
              v[1] = fma(rn, rn, v[1]);
            }
          }
        }
        if (!(ok = coop_sums(v, tm, buf, sm))) break;
        if (t0) {
          coop_after_update(s, v[0], v[1], d);
          coop_end_body(s, d);
        }
        __syncthreads();
      }
      if (s.phase == kPhaseRun) {
        // p = z + beta p, then a barrier before the next SpMV gathers p
        const double beta = s.beta;
        for (int i0 = g0; i0 < n; i0 += kCoopUnroll * T) {
          double zi[kCoopUnroll], pi[kCoopUnroll];
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) {
              zi[u] = z[i];
              pi[u] = p[i];
            }
          }
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) p[i] = fma(beta, pi[u], zi[u]);
          }
        }
        if (!(ok = team_sync(tm, sm))) break;
      }
    } else {
      // true residual t = b - A x; restart from it (r = t, z = D^{-1} t, p = z)
      double v[2] = {0.0, 0.0};  // t.t, t.z
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, col_at, val_at, Coherent{d.x});
        const double zi = dinv[i] * ti;
        r[i] = ti;
        z[i] = zi;
        p[i] = zi;
        v[0] = fma(ti, ti, v[0]);
        v[1] = fma(ti, zi, v[1]);
      });
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) {
        coop_after_check(s, v[0], v[1], d);
        coop_end_body(s, d);
      }
      __syncthreads();
    }
  }

  // ---- final: residual of the returned x (x = 0 for a zero right-hand side)
  if (ok && !s.bad) {
    if (s.zero_rhs) {
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    } else {
      double v[1] = {0.0};
      for (int i = g0; i < n; i += T) {
        const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, col_at, val_at, Coherent{d.x});
        v[0] = fma(ti, ti, v[0]);
      }
      ok = coop_sums(v, tm, buf, sm);
      if (t0) s.ttt = v[0];
    }
  }
  if (tm.rank == 0 && t0) {
    sla_info inf;
    inf.iters = s.iters;
    if (!ok || (check_err && __ldcg(tm.err) != 0)) {
      inf.status = SLA_ERR_TIMEOUT;
      inf.rel_res = NAN;
      inf.true_rel_res = NAN;
    } else {
      inf.status = s.status;
      if (s.zero_rhs) {
        inf.rel_res = 0.0;
        inf.true_rel_res = 0.0;
      } else if (s.bad) {
        inf.rel_res = NAN;
        inf.true_rel_res = NAN;
      } else {
        inf.rel_res = sqrt(s.rr) / s.bnorm;
        inf.true_rel_res = sqrt(s.ttt) / s.bnorm;
      }
    }
    *d.info = inf;
  }
  return ok;
}

__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) cg_coop_kernel(CoopArgs A) {
  __shared__ CoopSmem sm;
  __shared__ CoopState s;
  __shared__ KrylovDesc sd;
  if (threadIdx.x == 0) sd = A.d;
  __syncthreads();
  Team tm{GridSync{&A.st->cnt[5], 0u}, (int)gridDim.x, (int)blockIdx.x, A.part, &A.st->err};
  jacobi_team_solve(sd, A.r, A.z, A.p, A.q, A.dinv, tm, true, sm, s);
}

// ------------------------------------------------------------------ G G^T

struct GgtCoopArgs {
  KrylovDesc d;
  KrylovState* st;
  double* part;
  double* r;
  double* p;
  double* q;
  double* t;
  const float* gv;   // FP32 values of G and of G^T, written before the launch
  const float* gtv;
};

// Phase of the start and of a restart: apply the preconditioner only.
constexpr int kPhasePrecondG = 4;

// After the SpMV of a RUN body (p.q): alpha, or the end on a breakdown.
// After a CHECK body (t.t of the true residual t): done, or a restart
// through the preconditioner phase.
__device__ __forceinline__ void ggt_after_k1(CoopState& s, int ph, double v, const KrylovDesc& d) {
  if (ph == kPhaseRun) {
    coop_after_pq(s, v);
    return;
  }
  s.ttt = v;
  if (sqrt(v) <= 2.0 * s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(v)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (s.restarts >= d.max_restarts || s.iters >= d.max_iter) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  } else {
    s.restarts += 1;
    s.rr = v;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhasePrecondG;
  }
}

// After t = G^T r: r.z = t.t; RUN: convergence and beta; PRECOND: rho and a
// fresh p.  `fresh` (block-uniform) tells the next p update not to read p.
__device__ __forceinline__ void ggt_after_gt(CoopState& s, int ph, double trz, const KrylovDesc& d) {
  const double rnorm = sqrt(s.rr);
  if (ph == kPhasePrecondG) {
    s.rho = trz;
    s.bad = 1;  // fresh p
    s.status = SLA_NOT_CONVERGED;
    if (!isfinite(trz) || !isfinite(rnorm)) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else if (rnorm <= s.thresh) {
      s.phase = kPhaseCheck;
    } else if (s.iters >= d.max_iter) {
      s.phase = kPhaseDone;
    } else {
      s.phase = kPhaseRun;
    }
  } else {
    if (!isfinite(trz) || !isfinite(rnorm)) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else if (rnorm <= s.thresh) {
      s.status = SLA_OK;
      s.phase = kPhaseCheck;
    } else if (!(trz > 0.0)) {
      s.status = SLA_NOT_SPD;
      s.phase = kPhaseDone;
    } else {
      s.beta = trz / s.rho;
      s.rho = trz;
      s.bad = 0;
      if (s.iters >= d.max_iter) {
        s.status = SLA_NOT_CONVERGED;
        s.phase = kPhaseDone;
      }
    }
  }
  // hard cap on loop bodies (each advances the iteration count or a restart)
  s.body += 1;
  if (s.phase != kPhaseDone && s.body > (long long)d.max_iter + 3LL * d.max_restarts + 8) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  }
}

// CoopState.bad is reused here as the fresh-p flag (the G G^T solve has no
// diagonal test).
__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) ggt_coop_kernel(GgtCoopArgs A) {
  __shared__ CoopSmem sm;
  __shared__ CoopState s;
  const KrylovDesc& d = A.d;
  const int n = d.n;
  const int T = gridDim.x * kCoopThreads;
  const int g0 = blockIdx.x * kCoopThreads + threadIdx.x;
  const bool t0 = threadIdx.x == 0;
  Team tm{GridSync{&A.st->cnt[5], 0u}, (int)gridDim.x, (int)blockIdx.x, A.part, &A.st->err};
  int buf = 0;
  bool ok = true;
  auto a_col = [&](int k) { return __ldg(d.col + k); };
  auto a_val = [&](int k) { return __ldg(d.val + k); };
  auto gt_col = [&](int k) { return __ldg(d.col_t + k); };
  auto gt_val = [&](int k) { return to_f64(__ldg(A.gtv + k)); };
  auto g_col = [&](int k) { return __ldg(d.g_col + k); };
  auto g_val = [&](int k) { return to_f64(__ldg(A.gv + k)); };

  // ---- init: r = b - A x0 (x = 0 unless use_x0); ||b||^2, ||r||^2
  {
    double acc[2] = {0.0, 0.0};
    for (int i = g0; i < n; i += T) {
      double ax = 0.0;
      if (d.use_x0) {
        const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
        ax = row_sum_batched(a, e, a_col, a_val, Coherent{d.x});
      }
      const double bi = __ldg(d.b + i);
      const double ri = bi - ax;
      A.r[i] = ri;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
    }
    if (!d.use_x0)
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    ok = coop_sums(acc, tm, buf, sm);
    if (ok && t0) {
      s.bnorm = sqrt(acc[0]);
      s.thresh = fmax(d.rtol * s.bnorm, d.atol);
      s.rr = acc[1];
      s.rho = s.alpha = s.beta = s.ttt = 0.0;
      s.body = 0;
      s.iters = s.restarts = s.zero_rhs = s.bad = 0;
      s.status = SLA_NOT_CONVERGED;
      if (s.bnorm == 0.0) {
        s.zero_rhs = 1;
        s.status = SLA_OK;
        s.phase = kPhaseDone;
      } else {
        s.phase = kPhasePrecondG;
      }
    }
    __syncthreads();
  }

  while (ok && s.phase != kPhaseDone) {
    const int ph = s.phase;
    double rr_part = 0.0;
    if (ph == kPhaseRun || ph == kPhaseCheck) {
      // RUN: q = A p, p.q.  CHECK: r = b - A x (the true residual), r.r
      double v[1] = {0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        if (ph == kPhaseRun) {
          const double y = row_sum_batched(a, e, a_col, a_val, Coherent{A.p});
          A.q[i] = y;
          v[0] = fma(A.p[i], y, v[0]);
        } else {
          const double ti = __ldg(d.b + i) - row_sum_batched(a, e, a_col, a_val, Coherent{d.x});
          A.r[i] = ti;
          v[0] = fma(ti, ti, v[0]);
        }
      });
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) ggt_after_k1(s, ph, v[0], d);
      __syncthreads();
      if (s.phase == kPhaseDone) break;
      if (ph == kPhaseRun) {
        // x += alpha p, r -= alpha q; r.r joins the next reduction
        const double alpha = s.alpha;
        for (int i0 = g0; i0 < n; i0 += kCoopUnroll * T) {
          double pi[kCoopUnroll], qi[kCoopUnroll], xi[kCoopUnroll], ri[kCoopUnroll];
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) {
              pi[u] = A.p[i];
              qi[u] = A.q[i];
              xi[u] = d.x[i];
              ri[u] = A.r[i];
            }
          }
#pragma unroll
          for (int u = 0; u < kCoopUnroll; ++u) {
            const int i = i0 + u * T;
            if (i < n) {
              d.x[i] = fma(alpha, pi[u], xi[u]);
              const double rn = fma(-alpha, qi[u], ri[u]);
              A.r[i] = rn;
              rr_part = fma(rn, rn, rr_part);
            }
          }
        }
        // G^T gathers r
        if (!(ok = team_sync(tm, sm))) break;
      }
    }
    // RUN or PRECOND (possibly entered by a restart in this body)
    const int ph2 = s.phase;
    {
      // t = G^T r, t.t (= r.z)
      double v[2] = {0.0, rr_part};
      coop_rows(n, g0, T, d.rowptr_t, [&](int i, int a, int e) {
        const double y = row_sum_batched(a, e, gt_col, gt_val, Coherent{A.r});
        A.t[i] = y;
        v[0] = fma(y, y, v[0]);
      });
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) {
        if (ph2 == kPhaseRun) {
          s.rr = v[1];
          s.iters += 1;
        }
        ggt_after_gt(s, ph2, v[0], d);
      }
      __syncthreads();
    }
    if (s.phase == kPhaseRun) {
      // p = G t + beta p (p = G t right after a (re)start: p is not read)
      const bool fresh = s.bad != 0;
      const double beta = fresh ? 0.0 : s.beta;
      coop_rows(n, g0, T, d.g_rowptr, [&](int i, int a, int e) {
        const double y = row_sum_batched(a, e, g_col, g_val, Coherent{A.t});
        A.p[i] = fresh ? y : fma(beta, A.p[i], y);
      });
      // the next SpMV gathers p
      if (!(ok = team_sync(tm, sm))) break;
    }
  }

  // ---- final: residual of the returned x (x = 0 for a zero right-hand side)
  if (ok) {
    if (s.zero_rhs) {
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    } else {
      double v[1] = {0.0};
      for (int i = g0; i < n; i += T) {
        const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, a_col, a_val, Coherent{d.x});
        v[0] = fma(ti, ti, v[0]);
      }
      ok = coop_sums(v, tm, buf, sm);
      if (t0) s.ttt = v[0];
    }
  }
  if (blockIdx.x == 0 && t0) {
    sla_info inf;
    inf.iters = s.iters;
    if (!ok || __ldcg(tm.err) != 0) {
      inf.status = SLA_ERR_TIMEOUT;
      inf.rel_res = NAN;
      inf.true_rel_res = NAN;
    } else {
      inf.status = s.status;
      if (s.zero_rhs) {
        inf.rel_res = inf.true_rel_res = 0.0;
      } else {
        inf.rel_res = sqrt(s.rr) / s.bnorm;
        inf.true_rel_res = sqrt(s.ttt) / s.bnorm;
      }
    }
    *d.info = inf;
  }
}

// ------------------------------------------------------------------ batched teams
//
// The large systems of a distinct-pattern batch (sla_cg_batched_list): a
// single-CTA solve of such a system runs at one SM's FP64 rate and sets the
// whole batch's time (the tail).  Here teams of kTeamBlocks consecutive
// blocks of one cooperative launch each take a system from a queue and
// solve it with the Jacobi-PCG above (team barriers on a counter of the
// team's own); when a team meets a system with fewer than min_nnz entries
// it splits into single blocks that take the rest of the queue one system
// each, so the small systems fill the time the last large ones take.

// Team size and (in sla_batched.cu) the entry threshold, swept on the 512
// FEM systems (B300, ms for the whole batch, single-CTA systems in a second
// launch): teams of 3 from 32768 entries 156.5; of 4 from 8192-65536 entries
// 160-167; of 2 188-203; of 6 175; of 8 186-215; without teams 219.  With the
// small systems in the same launch: 3 / 32768 150.3, 3 / 16384 151.1,
// 3 / 65536 152.2, 4 / 65536 163.3, 3 / 131072 168.0, 2 / 65536 183.3.  Large teams pay their barriers with few rows
// per thread; without teams the largest system runs at one SM's rate.
constexpr int kTeamBlocks = 3;

struct TeamBatchArgs {
  int batch, min_nnz;
  const int* rowptr;
  const int* col;
  const int* n_off;
  const int* nnz_off;
  const int* order;   // optional
  const double* val;
  const double* b;
  double* x;
  sla_info* info;
  double* gvec;       // per row of the batch: 5 doubles at 5 n_off[s], or 8 at 8 n_off[s] (pipelined)
  unsigned* counters; // [teams] barrier counters, zero at launch
  int* slots;         // [teams] queue position handed to each team
  unsigned* next;     // queue counter, zero at launch
  double* parts;      // [teams][2 * 4 * kTeamBlocks]
  int* err;
  double rtol, atol;
  int max_iter, max_restarts, precond, use_x0;
};

// Fills sd (shared) for system `sys` of the batch; returns its first row.
__device__ __forceinline__ long long team_system_desc(const TeamBatchArgs& B, int sys, KrylovDesc& sd) {
  const int e0 = B.nnz_off[sys], n0 = B.n_off[sys];
  KrylovDesc t = {};
  t.n = B.n_off[sys + 1] - n0;
  t.nnz = B.nnz_off[sys + 1] - e0;
  t.rowptr = B.rowptr + n0 + sys;
  t.col = B.col + e0;
  t.val = B.val + e0;
  t.b = B.b + n0;
  t.x = B.x + n0;
  t.info = B.info + sys;
  t.rtol = B.rtol;
  t.atol = B.atol;
  t.max_iter = B.max_iter;
  t.max_restarts = B.max_restarts;
  t.precond = B.precond;
  t.use_x0 = B.use_x0;
  sd = t;
  return n0;
}

// Teams take systems from the queue while they are large; the first small
// system a team meets turns it into single blocks, which take the rest of
// the queue one system per block (the queue is largest first, so from then
// on every system is small), so no block waits while others finish.
// PIPE: the systems solved by teams take the pipelined PCG (one merged
// reduction and one team barrier per iteration, sla_cg_pipe.cuh); single
// blocks keep the standard form, whose barriers are block barriers and
// whose FP64 work per row is smaller.  The vectors of a system start at
// 8 row0 with PIPE (so that the 8-double records of a team system and the
// 5 vectors of a single-block system never overlap), else at 5 row0.
template <bool PIPE>
__device__ __forceinline__ bool batch_solve(const KrylovDesc& sd, double* gvec, long long row0, Team& tm,
                                            CoopSmem& sm, CoopState& s, PipeState& ps) {
  const size_t n = (size_t)sd.n;
  double* vec = gvec + (PIPE ? 8 : 5) * (size_t)row0;
  if (PIPE && tm.size > 1) return pipe_team_solve(sd, vec, vec + 6 * n, vec + 7 * n, tm, false, sm, ps);
  return jacobi_team_solve(sd, vec, vec + n, vec + 2 * n, vec + 3 * n, vec + 4 * n, tm, false, sm, s);
}

template <bool PIPE>
__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) batched_team_kernel(TeamBatchArgs B) {
  __shared__ CoopSmem sm;
  __shared__ CoopState s;
  __shared__ PipeState ps;
  __shared__ KrylovDesc sd;
  __shared__ long long s_row0;
  __shared__ int s_k;
  const int q = blockIdx.x / kTeamBlocks, rank = blockIdx.x % kTeamBlocks;
  Team tm{GridSync{B.counters + q, 0u}, kTeamBlocks, rank, B.parts + (size_t)q * 8 * kTeamBlocks, B.err};
  int first = -1;  // queue position a block takes first in single mode
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) B.slots[q] = (int)atomicAdd(B.next, 1u);
    if (!team_sync(tm, sm)) return;
    if (threadIdx.x == 0) {
      const int k = __ldcg(B.slots + q);
      s_k = k;
      s_row0 = -2;  // queue exhausted
      if (k < B.batch) {
        const int sys = B.order ? B.order[k] : k;
        s_row0 = -1;  // a small system: single mode from here
        if (B.nnz_off[sys + 1] - B.nnz_off[sys] >= B.min_nnz) s_row0 = team_system_desc(B, sys, sd);
      }
    }
    __syncthreads();
    const long long row0 = s_row0;
    if (row0 == -2) return;
    if (row0 == -1) {
      if (rank == 0) first = s_k;
      break;
    }
    if (!batch_solve<PIPE>(sd, B.gvec, row0, tm, sm, s, ps)) return;
  }
  // single mode: every block solves whole systems on its own
  Team solo{GridSync{nullptr, 0u}, 1, 0, nullptr, B.err};
  for (;;) {
    if (threadIdx.x == 0) {
      const int k = first >= 0 ? first : (int)atomicAdd(B.next, 1u);
      s_row0 = -2;
      if (k < B.batch) s_row0 = team_system_desc(B, B.order ? B.order[k] : k, sd);
    }
    first = -1;
    __syncthreads();
    const long long row0 = s_row0;
    if (row0 < 0) return;
    if (!batch_solve<PIPE>(sd, B.gvec, row0, solo, sm, s, ps)) return;
    __syncthreads();  // sd and s_row0 are rewritten for the next system
  }
}

// ------------------------------------------------------------------ host

// Zeroes the barrier counter and the error flag of the state before a launch.
__global__ void coop_arm_kernel(KrylovState* st) {
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
}

// Largest n solved by the cooperative kernels, from the measured crossover
// with the graph of per-phase kernels (B300, us per iteration, cooperative
// vs graph): Jacobi 2D 1024^2 48.1 vs 54.3, 3D 128^3 (2.1 M) 91.3 vs 96.0,
// 3D 160^3 (4.1 M) 172 vs 159; G G^T 1024^2 78.6 vs 82.5, 128^3 164 vs 157.
// SLA_CG_COOP=0 disables them, =1 uses them at every size.
constexpr long long kCoopMaxNJacobi = 5LL << 19;  // 2.5 Mi rows
constexpr long long kCoopMaxNGgt = 3LL << 19;     // 1.5 Mi rows

bool use_coop(long long n, long long limit) {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("SLA_CG_COOP");
    forced = -1;
    if (e != nullptr) {
      if (strcmp(e, "0") == 0) forced = 0;
      else if (strcmp(e, "1") == 0) forced = 1;
    }
  }
  if (forced == 0) return false;
  if (forced == 1) return true;
  return n <= limit;
}

bool use_cg_coop(long long n, bool ggt) { return use_coop(n, ggt ? kCoopMaxNGgt : kCoopMaxNJacobi); }

namespace {
std::mutex g_coop_mu;
// resident blocks per SM of each kernel per device (0: not yet queried,
// -1: the device has no cooperative launch)
int g_occ_cg[64] = {}, g_occ_ggt[64] = {}, g_occ_team[64] = {}, g_occ_team_pipe[64] = {};
}  // namespace

int coop_occupancy_of(int dev, int* cache, const void* fn) {
  std::lock_guard<std::mutex> lk(g_coop_mu);
  if (cache[dev] == 0) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cache[dev] = coop ? occupancy(fn, kCoopThreads) : -1;
    cudaGetLastError();
  }
  return cache[dev];
}

// Launches the cooperative Jacobi-PCG solve; *launched is false (and nothing
// was enqueued) when the device cannot run it, so that the caller takes the
// graph path instead.
int launch_cg_coop(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const int occ = coop_occupancy_of(dev, g_occ_cg, (const void*)cg_coop_kernel);
  if (occ <= 0) return SLA_OK;
  const CgLayout L = cg_layout(desc.n);
  char* base = (char*)ws;
  CoopArgs A;
  A.d = desc;
  A.st = (KrylovState*)(base + L.state);
  A.part = (double*)(base + L.part);
  A.r = (double*)(base + L.r);
  A.z = (double*)(base + L.z);
  A.p = (double*)(base + L.p);
  A.q = (double*)(base + L.q);
  A.dinv = (double*)(base + L.dinv);
  coop_arm_kernel<<<1, 1, 0, s>>>(A.st);
  SLA_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cg_coop_kernel, dim3(coop_grid(dev, desc.n, occ)),
                                           dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

// The same for G G^T PCG; gv / gtv hold the FP32 values of G and G^T
// (written by an earlier launch on the same stream).
int launch_ggt_coop(const KrylovDesc& desc, KrylovState* st, double* part, double* r, double* p, double* q,
                    double* t, const float* gv, const float* gtv, cudaStream_t s, bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const int occ = coop_occupancy_of(dev, g_occ_ggt, (const void*)ggt_coop_kernel);
  if (occ <= 0) return SLA_OK;
  GgtCoopArgs A;
  A.d = desc;
  A.st = st;
  A.part = part;
  A.r = r;
  A.p = p;
  A.q = q;
  A.t = t;
  A.gv = gv;
  A.gtv = gtv;
  coop_arm_kernel<<<1, 1, 0, s>>>(st);
  SLA_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)ggt_coop_kernel, dim3(coop_grid(dev, desc.n, occ)),
                                           dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

// Marks every system as timed out before the launch, so that a system no
// block reached (blocks that left after a barrier ran out) does not keep a
// stale record; each solve overwrites its own.
__global__ void team_info_prefill_kernel(int batch, sla_info* info) {
  for (int sys = blockIdx.x * blockDim.x + threadIdx.x; sys < batch; sys += gridDim.x * blockDim.x)
    info[sys] = sla_info{0, SLA_ERR_TIMEOUT, NAN, NAN};
}

size_t team_scratch_bytes() {
  return al256(sizeof(unsigned) * kCoopMaxGrid) + al256(sizeof(int) * kCoopMaxGrid) + 256 +
         al256(sizeof(double) * 8 * kCoopMaxGrid);
}

TeamScratch team_scratch(void* scratch) {
  char* base = (char*)scratch;
  TeamScratch t;
  t.counters = (unsigned*)base;
  base += al256(sizeof(unsigned) * kCoopMaxGrid);
  t.slots = (int*)base;
  base += al256(sizeof(int) * kCoopMaxGrid);
  t.next = (unsigned*)base;
  t.err = (int*)(base + 128);
  base += 256;
  t.parts = (double*)base;
  return t;
}

int team_scratch_arm(void* scratch, int batch, sla_info* info, cudaStream_t s) {
  const TeamScratch t = team_scratch(scratch);
  SLA_CUDA_TRY(cudaMemsetAsync(scratch, 0, (char*)t.parts - (char*)scratch, s));
  team_info_prefill_kernel<<<(batch + 255) / 256, 256, 0, s>>>(batch, info);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// Solves the systems of a concatenated batch with at least min_nnz entries
// by teams of blocks (one cooperative launch); *launched is false (nothing
// enqueued) when the device cannot run it.
int launch_batched_teams(int batch, int min_nnz, const int* rowptr, const int* col, const int* n_off,
                         const int* nnz_off, const int* order, const double* val, const double* b, double* x,
                         sla_info* info, double* gvec, void* scratch, double rtol, double atol, int max_iter,
                         int max_restarts, int precond, int use_x0, bool pipelined, cudaStream_t s,
                         bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const void* fn = pipelined ? (const void*)batched_team_kernel<true> : (const void*)batched_team_kernel<false>;
  const int occ = coop_occupancy_of(dev, pipelined ? g_occ_team_pipe : g_occ_team, fn);
  if (occ <= 0) return SLA_OK;
  int grid = num_sms(dev) * occ;
  if (grid > kCoopMaxGrid) grid = kCoopMaxGrid;
  grid -= grid % kTeamBlocks;
  if (grid < kTeamBlocks) return SLA_OK;
  const TeamScratch ts = team_scratch(scratch);
  TeamBatchArgs B;
  B.batch = batch;
  B.min_nnz = min_nnz;
  B.rowptr = rowptr;
  B.col = col;
  B.n_off = n_off;
  B.nnz_off = nnz_off;
  B.order = order;
  B.val = val;
  B.b = b;
  B.x = x;
  B.info = info;
  B.gvec = gvec;
  B.counters = ts.counters;
  B.slots = ts.slots;
  B.next = ts.next;
  B.err = ts.err;
  B.parts = ts.parts;
  B.rtol = rtol;
  B.atol = atol;
  B.max_iter = max_iter;
  B.max_restarts = max_restarts;
  B.precond = precond;
  B.use_x0 = use_x0;
  // counters, queue and error flag start at zero
  const int rc = team_scratch_arm(scratch, batch, info, s);
  if (rc != SLA_OK) return rc;
  void* args[] = {&B};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

// ------------------------------------------------------------------ self-test

// `rounds` grid barriers with a given wait budget; block `absent` (if any)
// never arrives, so the others' waits run out.  word[0]: blocks whose wait
// ran out, word[1]: blocks that passed every barrier, word[2]: the barrier
// counter, word[3]: the error flag.
__global__ void grid_barrier_selftest_kernel(int* word, int absent, long long budget, int rounds) {
  __shared__ int flag;
  if ((int)blockIdx.x == absent) return;
  GridSync gs{(unsigned*)(word + 2), 0u};
  for (int k = 0; k < rounds; ++k) {
    if (!grid_sync(gs, gridDim.x, word + 3, &flag, budget)) {
      if (threadIdx.x == 0) atomicAdd(word, 1);
      return;
    }
  }
  if (threadIdx.x == 0) atomicAdd(word + 1, 1);
}

int occupancy_selftest() {
  static int occ = 0;
  if (occ == 0) occ = occupancy((const void*)grid_barrier_selftest_kernel, kCoopThreads);
  return occ;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_selftest_grid_barrier(int32_t blocks, int32_t absent, int64_t budget_cycles,
                                             int32_t rounds, int32_t* word, void* stream) {
  if (word == nullptr || blocks < 1 || rounds < 0 || budget_cycles < 1 || absent >= blocks) return SLA_ERR_INVALID;
  const int dev = current_device();
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || blocks > num_sms(dev) * occupancy_selftest()) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  SLA_CUDA_TRY(cudaMemsetAsync(word, 0, 4 * sizeof(int32_t), s));
  int a = absent < 0 ? -1 : absent;
  long long budget = budget_cycles;
  int r = rounds;
  void* args[] = {&word, &a, &budget, &r};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)grid_barrier_selftest_kernel, dim3(blocks),
                                           dim3(kCoopThreads), args, 0, s));
  return SLA_OK;
}
