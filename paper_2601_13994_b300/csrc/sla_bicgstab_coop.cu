// sla_bicgstab_coop.cu -- right-preconditioned BiCGStab in one cooperative
// launch per solve.
//
// The method, state machine and exits are those of the graph loop in
// sla_bicgstab.cu (van der Vorst's BiCGStab with shadow residual r^ = r0 and
// M = diag(A); the half-step exit when |s| meets the target; the
// true-residual check and restart; the final residual), for systems where a
// kernel boundary is a large share of an iteration.  Every block stays
// resident for the whole solve and each of the graph's kernel boundaries
// becomes a grid barrier; the reductions are summed in the same order by
// every block, which therefore takes the same decisions (sla_coop.cuh).
//
// One iteration: p = r + beta (p - omega v), p^ = M^-1 p | barrier |
// v = A p^, r^.v | reduce | s = r - alpha v, s^ = M^-1 s, s.s | reduce |
// t = A s^, t.t, t.s | reduce | x += alpha p^ + omega s^, r = s - omega t,
// r.r, r^.r | reduce.
#include <cmath>

#include "sla_coop.cuh"

namespace sla {
namespace {

constexpr int kPhaseHalf = 3;  // as in sla_bicgstab.cu

struct BiCoopArgs {
  KrylovDesc d;
  KrylovState* st;
  double* part;
  double *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;
};

// Block-uniform solver scalars in shared memory (thread 0 writes them after a
// reduction; all threads read them after a block barrier).
struct BiState {
  double bnorm, thresh, rr, rho, rho_prev, alpha, omega, beta;
  long long body;
  int iters, restarts, status, phase, zero_rhs, bad;
};

__device__ __forceinline__ void bi_after_init(BiState& s, const double* t, const KrylovDesc& d) {
  s.bnorm = sqrt(t[0]);
  s.thresh = fmax(d.rtol * s.bnorm, d.atol);
  s.rr = t[1];
  s.rho = t[1];  // r^ = r0
  s.rho_prev = s.alpha = s.omega = 1.0;
  s.beta = 0.0;
  s.body = 0;
  s.iters = s.restarts = s.zero_rhs = s.bad = 0;
  s.status = SLA_NOT_CONVERGED;
  s.phase = kPhaseRun;
  if (t[2] > 0.0) {
    s.bad = 1;
    s.status = SLA_ERR_INVALID;
    s.phase = kPhaseDone;
  } else if (s.bnorm == 0.0) {
    s.zero_rhs = 1;
    s.status = SLA_OK;
    s.phase = kPhaseDone;
  } else if (!isfinite(t[1])) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(t[1]) <= s.thresh) {
    s.phase = kPhaseCheck;
  } else if (d.max_iter <= 0) {
    s.phase = kPhaseDone;
  } else if (fabs(s.rho) < 1e-300) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else {
    s.beta = (s.rho / s.rho_prev) * (s.alpha / s.omega);
  }
}

// End of a loop body: hard cap on bodies (each advances the iteration count
// or consumes a restart, so this only fires if the state machine is broken).
__device__ __forceinline__ void bi_end_body(BiState& s, const KrylovDesc& d) {
  s.body += 1;
  const long long cap = 2LL * d.max_iter + 3LL * d.max_restarts + 8;
  if (s.phase != kPhaseDone && s.body > cap) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  }
}

// After r^.v: alpha, or a breakdown.
__device__ __forceinline__ void bi_after_rv(BiState& s, double rv) {
  if (!isfinite(rv) || rv == 0.0) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else {
    s.alpha = s.rho / rv;
  }
}

// After s.s: the iteration count, and the half-step exit when |s| meets the
// target (x += alpha p^ then closes the solve).
__device__ __forceinline__ void bi_after_ss(BiState& s, double ss) {
  s.iters += 1;
  if (sqrt(ss) <= s.thresh) {
    s.rr = ss;
    s.status = SLA_OK;
    s.phase = kPhaseHalf;
  }
}

// After t.t and t.s: omega, or a breakdown.
__device__ __forceinline__ void bi_after_tt(BiState& s, double tt, double ts) {
  if (!isfinite(tt) || !isfinite(ts) || tt == 0.0) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else {
    s.omega = ts / tt;
  }
}

// After r.r and r^.r: convergence of the recursive residual, the next beta.
__device__ __forceinline__ void bi_after_x(BiState& s, double rr, double rho_new, const KrylovDesc& d) {
  s.rr = rr;
  if (!isfinite(rr)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (sqrt(rr) <= s.thresh) {
    s.status = SLA_OK;
    s.phase = kPhaseCheck;
  } else if (s.omega == 0.0) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (s.iters >= d.max_iter) {
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseDone;
  } else {
    s.rho_prev = s.rho;
    s.rho = rho_new;
    if (!isfinite(rho_new) || fabs(rho_new) < 1e-300) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else {
      s.beta = (s.rho / s.rho_prev) * (s.alpha / s.omega);
    }
  }
}

// After the true-residual check (t.t): done, or a restart from t (r = r^ =
// t, p = v = 0; the first p update then gives p = r).
__device__ __forceinline__ void bi_after_check(BiState& s, double tt, const KrylovDesc& d) {
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
    s.rho = tt;
    s.rho_prev = s.alpha = s.omega = 1.0;
    s.status = SLA_NOT_CONVERGED;
    if (fabs(tt) < 1e-300) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else {
      s.beta = tt;
      s.phase = kPhaseRun;
    }
  }
}

__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) bicg_coop_kernel(BiCoopArgs A) {
  __shared__ CoopSmem sm;
  __shared__ BiState s;
  __shared__ KrylovDesc sd;
  const bool t0 = threadIdx.x == 0;
  if (t0) sd = A.d;
  __syncthreads();
  const KrylovDesc& d = sd;
  const int n = d.n;
  const int T = gridDim.x * kCoopThreads;
  const int g0 = blockIdx.x * kCoopThreads + threadIdx.x;
  Team tm{GridSync{&A.st->cnt[5], 0u}, (int)gridDim.x, (int)blockIdx.x, A.part, &A.st->err};
  int buf = 0;
  bool ok = true;
  auto col_at = [&](int k) { return __ldg(d.col + k); };
  auto val_at = [&](int k) { return __ldg(d.val + k); };

  // ---- init: dinv, r = r^ = b - A x0, p = v = 0; ||b||^2, ||r||^2, bad diagonal
  {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int i = g0; i < n; i += T) {
      const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
      double diag = 0.0, ax = 0.0;
      for (int k = a; k < e; ++k) {
        const int c = __ldg(d.col + k);
        const double v = __ldg(d.val + k);
        if (c == i) diag += v;
        if (d.use_x0) ax = fma(v, d.x[c], ax);
      }
      double di = 1.0;
      if (d.precond == SLA_PRECOND_JACOBI) {
        di = 1.0 / diag;
        if (diag == 0.0 || !isfinite(di)) acc[2] = 1.0;
      }
      const double bi = __ldg(d.b + i);
      const double ri = bi - ax;
      A.dinv[i] = di;
      A.r[i] = ri;
      A.rh[i] = ri;
      A.p[i] = 0.0;
      A.v[i] = 0.0;
      acc[0] = fma(bi, bi, acc[0]);
      acc[1] = fma(ri, ri, acc[1]);
    }
    if (!d.use_x0)
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    ok = coop_sums(acc, tm, buf, sm);
    if (ok && t0) bi_after_init(s, acc, d);
    __syncthreads();
  }

  while (ok && s.phase != kPhaseDone) {
    if (s.phase == kPhaseRun) {
      // p = r + beta (p - omega v), p^ = M^-1 p; the SpMV below gathers p^
      {
        const double beta = s.beta, omega = s.omega;
        for (int i = g0; i < n; i += T) {
          const double pn = fma(beta, fma(-omega, A.v[i], A.p[i]), A.r[i]);
          A.p[i] = pn;
          A.ph[i] = A.dinv[i] * pn;
        }
        if (!(ok = team_sync(tm, sm))) break;
      }
      // v = A p^, r^.v -> alpha
      {
        double w[1] = {0.0};
        coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
          const double y = row_sum_batched(a, e, col_at, val_at, Coherent{A.ph});
          A.v[i] = y;
          w[0] = fma(A.rh[i], y, w[0]);
        });
        if (!(ok = coop_sums(w, tm, buf, sm))) break;
        if (t0) {
          bi_after_rv(s, w[0]);
          if (s.phase == kPhaseDone) bi_end_body(s, d);
        }
        __syncthreads();
        if (s.phase == kPhaseDone) break;
      }
      // s = r - alpha v, s^ = M^-1 s, s.s -> iteration count, half-step exit
      {
        const double alpha = s.alpha;
        double w[1] = {0.0};
        for (int i = g0; i < n; i += T) {
          const double sn = fma(-alpha, A.v[i], A.r[i]);
          A.s[i] = sn;
          A.sh[i] = A.dinv[i] * sn;
          w[0] = fma(sn, sn, w[0]);
        }
        if (!(ok = coop_sums(w, tm, buf, sm))) break;
        if (t0) bi_after_ss(s, w[0]);
        __syncthreads();
      }
      if (s.phase == kPhaseRun) {
        // t = A s^, t.t, t.s -> omega
        {
          double w[2] = {0.0, 0.0};
          coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
            const double y = row_sum_batched(a, e, col_at, val_at, Coherent{A.sh});
            A.t[i] = y;
            w[0] = fma(y, y, w[0]);
            w[1] = fma(y, A.s[i], w[1]);
          });
          if (!(ok = coop_sums(w, tm, buf, sm))) break;
          if (t0) {
            bi_after_tt(s, w[0], w[1]);
            if (s.phase == kPhaseDone) bi_end_body(s, d);
          }
          __syncthreads();
          if (s.phase == kPhaseDone) break;
        }
        // x += alpha p^ + omega s^, r = s - omega t; r.r, r^.r
        {
          const double alpha = s.alpha, omega = s.omega;
          double w[2] = {0.0, 0.0};
          for (int i = g0; i < n; i += T) {
            d.x[i] = fma(omega, A.sh[i], fma(alpha, A.ph[i], d.x[i]));
            const double rn = fma(-omega, A.t[i], A.s[i]);
            A.r[i] = rn;
            w[0] = fma(rn, rn, w[0]);
            w[1] = fma(A.rh[i], rn, w[1]);
          }
          if (!(ok = coop_sums(w, tm, buf, sm))) break;
          if (t0) {
            bi_after_x(s, w[0], w[1], d);
            bi_end_body(s, d);
          }
          __syncthreads();
        }
      } else {
        // half step: x += alpha p^; the check that follows gathers x
        const double alpha = s.alpha;
        for (int i = g0; i < n; i += T) d.x[i] = fma(alpha, A.ph[i], d.x[i]);
        if (!(ok = team_sync(tm, sm))) break;
        if (t0) {
          s.phase = kPhaseCheck;
          bi_end_body(s, d);
        }
        __syncthreads();
      }
    } else {
      // true residual t = b - A x; restart from it (r = r^ = t, p = v = 0)
      double w[1] = {0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, col_at, val_at, Coherent{d.x});
        A.r[i] = ti;
        A.rh[i] = ti;
        A.p[i] = 0.0;
        A.v[i] = 0.0;
        w[0] = fma(ti, ti, w[0]);
      });
      if (!(ok = coop_sums(w, tm, buf, sm))) break;
      if (t0) {
        bi_after_check(s, w[0], d);
        bi_end_body(s, d);
      }
      __syncthreads();
    }
  }

  // ---- final: residual of the returned x (x = 0 for a zero right-hand side)
  double ttt = 0.0;
  if (ok && !s.bad) {
    if (s.zero_rhs) {
      for (int i = g0; i < n; i += T) d.x[i] = 0.0;
    } else {
      double w[1] = {0.0};
      coop_rows(n, g0, T, d.rowptr, [&](int i, int a, int e) {
        const double ti = __ldg(d.b + i) - row_sum_batched(a, e, col_at, val_at, Coherent{d.x});
        w[0] = fma(ti, ti, w[0]);
      });
      ok = coop_sums(w, tm, buf, sm);
      ttt = w[0];
    }
  }
  if (blockIdx.x == 0 && t0) {
    sla_info inf;
    inf.iters = s.iters;
    if (!ok || __ldcg(tm.err) != 0) {
      inf.status = SLA_ERR_TIMEOUT;
      inf.rel_res = inf.true_rel_res = NAN;
    } else {
      inf.status = s.phase == kPhaseDone ? s.status : SLA_NOT_CONVERGED;
      if (s.zero_rhs) {
        inf.rel_res = inf.true_rel_res = 0.0;
      } else if (s.bad) {
        inf.rel_res = inf.true_rel_res = NAN;
      } else {
        inf.rel_res = sqrt(s.rr) / s.bnorm;
        inf.true_rel_res = sqrt(ttt) / s.bnorm;
      }
    }
    *d.info = inf;
  }
}

__global__ void bicg_coop_arm_kernel(KrylovState* st) {
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
}

int g_occ_bicg[64] = {};

}  // namespace

// Largest n solved by the cooperative BiCGStab, from the measured crossover
// with the graph of per-phase kernels (B300, 3D convection-diffusion Pe 10,
// us per iteration cooperative vs graph, the graph on A D^{-1} with the
// preconditioner folded in): 32^3 27.1 vs 37.0, 48^3 32.0 vs 44.1, 64^3 41.4
// vs 52.4, 80^3 56.1 vs 66.1, 96^3 94.1 vs 92.4, 128^3 186.6 vs 159.4 -- two
// SpMV phases per iteration at 1024 threads per SM lose to the graph's
// kernels from somewhat under 1 M rows.
constexpr long long kCoopMaxNBicg = 3LL << 18;  // 768 Ki rows

bool use_bicg_coop(long long n) { return use_coop(n, kCoopMaxNBicg); }

// Launches the cooperative BiCGStab solve; *launched is false (nothing
// enqueued) when the device cannot run it.
int launch_bicgstab_coop(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const int occ = coop_occupancy_of(dev, g_occ_bicg, (const void*)bicg_coop_kernel);
  if (occ <= 0) return SLA_OK;
  const BiLayout L = bicg_layout(desc.n);
  char* base = (char*)ws;
  BiCoopArgs A;
  A.d = desc;
  A.st = (KrylovState*)(base + L.state);
  A.part = (double*)(base + L.part);
  double* vecs[9];
  for (int j = 0; j < 9; ++j) vecs[j] = (double*)(base + L.vec + (size_t)j * L.vec_stride);
  A.r = vecs[0];
  A.rh = vecs[1];
  A.p = vecs[2];
  A.ph = vecs[3];
  A.v = vecs[4];
  A.s = vecs[5];
  A.sh = vecs[6];
  A.t = vecs[7];
  A.dinv = vecs[8];
  bicg_coop_arm_kernel<<<1, 1, 0, s>>>(A.st);
  SLA_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bicg_coop_kernel, dim3(coop_grid(dev, desc.n, occ)),
                                           dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

}  // namespace sla
