// sla_cg_pipe.cuh -- the pipelined Jacobi-PCG solve (Ghysels-Vanroose; one
// merged reduction and one barrier per iteration) as a device function of a
// Team, shared by the single-system cooperative kernel (sla_cg_pipe.cu) and
// the distinct-pattern batch (sla_cg_coop.cu).  The method, its readings and
// its exits are described in sla_cg_pipe.cu.
#pragma once

#include <cmath>

#include "sla_coop.cuh"

namespace sla {

// The vectors only a row's owner touches -- r, w, z, s, p and D^{-1} -- sit in
// one 48-byte record per row, read and written as three 16-byte pairs
// (r, w), (z, s), (p, dinv): one base pointer instead of six keeps the kernel
// within 64 registers (two blocks of 512 threads per SM) without spills.
enum : int { kRecR = 0, kRecW = 1, kRecZ = 2, kRecS = 3, kRecP = 4, kRecD = 5, kRec = 6 };

// Block-uniform solver scalars (shared memory; thread 0 writes them after a
// reduction, every thread reads them after a block barrier).
struct PipeState {
  double bnorm, thresh, rr, ttt, alpha, beta, gamma_prev, alpha_prev;
  long long body;
  int iters, restarts, status, phase, zero_rhs, bad, fresh;
};

// Start of the recurrence (at the first start and after a restart):
// w = A u, m = D^{-1} w and the first sums.
constexpr int kPhasePrime = 3;

// After the initial sums (||b||^2, ||r||^2, bad diagonal).
__device__ __forceinline__ void pipe_after_init(PipeState& s, const double* t, const KrylovDesc& d) {
  s.bnorm = sqrt(t[0]);
  s.thresh = fmax(d.rtol * s.bnorm, d.atol);
  s.rr = t[1];
  s.ttt = s.alpha = s.beta = s.gamma_prev = s.alpha_prev = 0.0;
  s.body = 0;
  s.iters = s.restarts = s.zero_rhs = s.bad = 0;
  s.fresh = 1;
  s.status = SLA_NOT_CONVERGED;
  s.phase = kPhasePrime;
  if (t[2] > 0.0) {
    s.bad = 1;
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else if (s.bnorm == 0.0) {
    s.zero_rhs = 1;
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(t[1])) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(t[1]) <= s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseCheck;
  }
}

// After the sums of a prime or an iteration: gamma = r.u, delta = w.u,
// rr = r.r.  Convergence, the iteration cap, then alpha and beta.
__device__ __forceinline__ void pipe_decide(PipeState& s, double gamma, double delta, double rr,
                                            const KrylovDesc& d) {
  s.rr = rr;
  if (!isfinite(gamma) || !isfinite(delta) || !isfinite(rr)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(rr) <= s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseCheck;
  } else if (s.iters >= d.max_iter) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  } else if (!(gamma > 0.0)) {
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else {
    double beta, denom;
    if (s.fresh) {
      beta = 0.0;
      denom = delta;
    } else {
      beta = gamma / s.gamma_prev;
      denom = delta - beta * gamma / s.alpha_prev;
    }
    if (!isfinite(denom)) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else if (!(denom > 0.0)) {
      if (s.fresh) {
        s.status = SLA_NOT_SPD;
        s.phase = kPhaseDone;
      } else {
        // the recurrences are exhausted: to the true-residual check
        s.status = SLA_OK;
        s.phase = kPhaseCheck;
      }
    } else {
      s.alpha = gamma / denom;
      s.beta = beta;
      s.gamma_prev = gamma;
      s.alpha_prev = s.alpha;
      s.status = SLA_NOT_CONVERGED;
      s.phase = kPhaseRun;
    }
  }
}

// After the true-residual check (t.t): done, or a restart from x.
__device__ __forceinline__ void pipe_after_check(PipeState& s, double tt, const KrylovDesc& d) {
  s.ttt = tt;
  if (sqrt(tt) <= 2.0 * s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(tt)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (s.restarts >= d.max_restarts || s.iters >= d.max_iter) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  } else {
    s.restarts += 1;
    s.rr = tt;
    s.fresh = 1;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhasePrime;
  }
}

// Hard cap on phases (each iteration, check and prime is one; the state
// machine stops long before this unless it is broken).
__device__ __forceinline__ void pipe_end_body(PipeState& s, const KrylovDesc& d) {
  s.body += 1;
  const long long cap = (long long)d.max_iter + 3LL * d.max_restarts + 8;
  if (s.phase != kPhaseDone && s.body > cap) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  }
}

// One pipelined Jacobi-PCG solve by a team (the whole grid of a cooperative
// launch, a group of its blocks, or one block); d (shared memory) describes
// the system; rec [n][kRec], m0 [n], m1 [n] are its work vectors.  Rank 0
// writes *d.info.  Returns false if a barrier ran out (the caller must then
// leave the kernel).  check_err: also report a timeout flagged by any block
// of the launch.
__device__ __forceinline__ bool pipe_team_solve(const KrylovDesc& d, double* rec_, double* m0, double* m1,
                                                Team& tm, bool check_err, CoopSmem& sm, PipeState& s) {
  const int n = d.n;
  const int T = tm.size * kCoopThreads;
  const int g0 = tm.rank * kCoopThreads + threadIdx.x;
  const bool t0 = threadIdx.x == 0;
  double* __restrict__ rec = rec_;
  auto pair = [&](int i, int k) { return reinterpret_cast<double2*>(rec + (size_t)i * kRec + k); };
  // m of the next iteration is in buffer `cur` (0: m0, 1: m1)
  auto mbuf = [&](int k) { return k ? m1 : m0; };
  int cur = 0;
  int buf = 0;
  bool ok = true;
  auto col_at = [&](int k) { return __ldg(d.col + k); };
  auto val_at = [&](int k) { return __ldg(d.val + k); };

  // ---- init: dinv, r = b - A x0, u = D^{-1} r into buffer 1; ||b||^2, ||r||^2, bad diagonal
  {
    double acc[3] = {0.0, 0.0, 0.0};
    double* u = mbuf(cur ^ 1);
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
        if (!(diag > 0.0)) acc[2] = 1.0;
        di = 1.0 / diag;
      }
      rec[(size_t)i * kRec + kRecR] = ri;
      rec[(size_t)i * kRec + kRecD] = di;
      u[i] = di * ri;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
    }
    if (!d.use_x0)
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    ok = coop_sums(acc, tm, buf, sm);
    if (ok && t0) pipe_after_init(s, acc, d);
    __syncthreads();
  }

  while (ok && s.phase != kPhaseDone) {
    if (s.phase == kPhaseRun) {
      // one iteration: nv = A m, the recurrences, the next m and the sums
      const double alpha = s.alpha, beta = s.beta;
      const bool fresh = s.fresh != 0;
      const double* __restrict__ m = mbuf(cur);
      double* __restrict__ mn = mbuf(cur ^ 1);
      double v[3] = {0.0, 0.0, 0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double nv = row_sum_batched(a, e, col_at, val_at, Coherent{m});
        const double2 rw = *pair(i, kRecR);
        const double2 pd = *pair(i, kRecP);
        const double di = pd.y, ri = rw.x, wi = rw.y;
        const double ui = di * ri;
        double zi, si, pi;
        if (fresh) {
          zi = nv;
          si = wi;
          pi = ui;
        } else {
          const double2 zs = *pair(i, kRecZ);
          zi = fma(beta, zs.x, nv);
          si = fma(beta, zs.y, wi);
          pi = fma(beta, pd.x, ui);
        }
        const double xn = fma(alpha, pi, d.x[i]);
        const double rn = fma(-alpha, si, ri);
        const double wn = fma(-alpha, zi, wi);
        const double un = di * rn;
        *pair(i, kRecR) = make_double2(rn, wn);
        *pair(i, kRecZ) = make_double2(zi, si);
        rec[(size_t)i * kRec + kRecP] = pi;
        d.x[i] = xn;
        mn[i] = di * wn;
        v[0] = fma(rn, un, v[0]);
        v[1] = fma(wn, un, v[1]);
        v[2] = fma(rn, rn, v[2]);
      });
      cur ^= 1;
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) {
        s.iters += 1;
        s.fresh = 0;
        pipe_decide(s, v[0], v[1], v[2], d);
        pipe_end_body(s, d);
      }
      __syncthreads();
    } else if (s.phase == kPhasePrime) {
      // w = A u (u = D^{-1} r in buffer cur ^ 1), m = D^{-1} w into buffer cur
      const double* __restrict__ u = mbuf(cur ^ 1);
      double* __restrict__ m = mbuf(cur);
      double v[3] = {0.0, 0.0, 0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double wi = row_sum_batched(a, e, col_at, val_at, Coherent{u});
        const double di = rec[(size_t)i * kRec + kRecD], ri = rec[(size_t)i * kRec + kRecR];
        const double ui = di * ri;
        rec[(size_t)i * kRec + kRecW] = wi;
        m[i] = di * wi;
        v[0] = fma(ri, ui, v[0]);
        v[1] = fma(wi, ui, v[1]);
        v[2] = fma(ri, ri, v[2]);
      });
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) {
        s.fresh = 1;
        pipe_decide(s, v[0], v[1], v[2], d);
        pipe_end_body(s, d);
      }
      __syncthreads();
    } else {
      // true residual t = b - A x; on a restart r = t and u = D^{-1} t
      double* u = mbuf(cur ^ 1);
      double v[1] = {0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, col_at, val_at, Coherent{d.x});
        rec[(size_t)i * kRec + kRecR] = ti;
        u[i] = rec[(size_t)i * kRec + kRecD] * ti;
        v[0] = fma(ti, ti, v[0]);
      });
      if (!(ok = coop_sums(v, tm, buf, sm))) break;
      if (t0) {
        pipe_after_check(s, v[0], d);
        pipe_end_body(s, d);
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

}  // namespace sla
