// sla_bicgstab.cu -- right-preconditioned BiCGStab for nonsymmetric A.
//
// The paper's GPU-native backend offers BiCGStab (van der Vorst 1992) for
// nonsymmetric systems (Sec. 1, Sec. 3.1); it gives no variant, so this is the
// textbook right-preconditioned form with shadow residual r^ = r0 and the
// Jacobi preconditioner M = diag(A):
//
//   rho = r^.r ; beta = (rho / rho_prev)(alpha / omega)
//   KA  p = r + beta (p - omega v) ;  p^ = M^-1 p
//   KB  v = A p^ ,  partial r^.v              -> alpha = rho / r^.v
//   KC  s = r - alpha v ; s^ = M^-1 s ; |s|^2 -> half-step exit test
//   KD  t = A s^ ,  partial t.t, t.s          -> omega = t.s / t.t
//   KE  x += alpha p^ + omega s^ ; r = s - omega t ; |r|^2, r^.r
//                                             -> convergence, next beta
//
// The same device state machine, graph WHILE loop / host loop, descriptor,
// true-residual check and restart rule as the CG solver.  KB and KD are the
// TMA-pipelined SpMV with dot-product epilogues.
//
// Algorithmic bytes per iteration: 2 (12 nnz + 4 (n+1)) + 200 n.
#include <cmath>
#include <mutex>
#include <vector>

#include "sla_internal.cuh"
#include "sla_tma.cuh"
#include "sla_workspace.h"

namespace sla {

namespace {

constexpr int kVT = 256;  // vector-kernel block size
constexpr int kU = 4;     // streaming unroll
constexpr int kPhaseHalf = 3;

struct BiPtrs {
  KrylovDesc* d;
  KrylovState* st;
  double* part;
  double *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;
  double* valh;  // A D^{-1}: the values with each column scaled by D^{-1}
};

// The matrix the iteration multiplies: A D^{-1} with the Jacobi
// preconditioner (x in the iteration is then x^ = D x), A itself without.
__device__ __forceinline__ const double* bicg_vals(const BiPtrs& P, const KrylovDesc& d) {
  return d.precond == SLA_PRECOND_JACOBI ? P.valh : d.val;
}

struct VSmem {
  double red[4 * kVT + 4];
  bool last;
};

__global__ void bicg_write_desc_kernel(KrylovDesc* dst, KrylovDesc src, KrylovState* st) {
  *dst = src;
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
}

// -------------------------------------------------------------- init
__global__ void __launch_bounds__(kVT) bicg_init_kernel(BiPtrs P) {
  __shared__ VSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  double acc[3] = {0.0, 0.0, 0.0};  // bb, rr, bad
  const int stride = gridDim.x * kVT;
  for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) {
    const int a = d.rowptr[i], e = d.rowptr[i + 1];
    double diag = 0.0, ax = 0.0;
    for (int k = a; k < e; ++k) {
      const int c = d.col[k];
      const double v = d.val[k];
      if (c == i) diag += v;
      if (d.use_x0) ax = fma(v, d.x[c], ax);
    }
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      di = 1.0 / diag;
      if (diag == 0.0 || !isfinite(di)) acc[2] = 1.0;
    }
    const double bi = d.b[i];
    const double ri = bi - ax;
    P.dinv[i] = di;
    P.r[i] = ri;
    P.rh[i] = ri;
    P.p[i] = 0.0;
    P.v[i] = 0.0;
    acc[0] = fma(bi, bi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
  }
  if (!d.use_x0)
    for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) d.x[i] = 0.0;
  block_sums<kVT, 3>(acc, sm.red);
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) P.part[j * kMaxBlocks + blockIdx.x] = acc[j];
  if (!last_block_arrive(&P.st->cnt[0], &sm.last)) return;
  double t[3];
  reduce_partials<kVT, 3>(P.part, kMaxBlocks, gridDim.x, t, sm.red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    const double tbb = t[0], trr = t[1], tbad = t[2];
    s.bnorm = sqrt(tbb);
    s.thresh = fmax(d.rtol * s.bnorm, d.atol);
    s.rr = trr;
    s.rho = trr;  // r^ = r0
    s.rho_prev = s.alpha = s.omega = 1.0;
    s.beta = 0.0;
    s.iters = s.restarts = s.body = 0;
    s.zero_rhs = s.bad_diag = 0;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseRun;
    if (tbad > 0.0) {
      s.bad_diag = 1;
      s.status = SLA_ERR_INVALID;
      s.phase = kPhaseDone;
    } else if (s.bnorm == 0.0) {
      s.zero_rhs = 1;
      s.status = SLA_OK;
      s.phase = kPhaseDone;
    } else if (!isfinite(trr)) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else if (sqrt(trr) <= s.thresh) {
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
}

// Right preconditioning folded into the matrix: A^ = A D^{-1} (each column j
// scaled by dinv_j) and x^ = D x, so that the iteration needs neither p^ =
// D^{-1} p nor s^ = D^{-1} s -- two vectors and two products a row fewer
// (BiCGStab on A^ with x = D^{-1} x^ is right-preconditioned BiCGStab).
// After bicg_init_kernel (which needs every dinv and the caller's x).
__global__ void __launch_bounds__(kVT) bicg_scale_kernel(BiPtrs P) {
  const KrylovDesc d = *P.d;
  if (d.precond != SLA_PRECOND_JACOBI || __ldcg(&P.st->bad_diag)) return;
  const int n = d.n;
  for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += gridDim.x * kVT) {
    for (int k = __ldg(d.rowptr + i); k < __ldg(d.rowptr + i + 1); ++k)
      P.valh[k] = __ldg(d.val + k) * __ldg(P.dinv + __ldg(d.col + k));
    d.x[i] = d.x[i] / P.dinv[i];
  }
}

// x = D^{-1} x^ at exit (after the final residual, which gathers x^).
__global__ void __launch_bounds__(kVT) bicg_unscale_kernel(BiPtrs P) {
  const KrylovDesc d = *P.d;
  if (d.precond != SLA_PRECOND_JACOBI || __ldcg(&P.st->bad_diag) || __ldcg(&P.st->zero_rhs)) return;
  for (int i = blockIdx.x * kVT + threadIdx.x; i < d.n; i += gridDim.x * kVT) d.x[i] *= P.dinv[i];
}

// -------------------------------------------------------------- KA
__global__ void __launch_bounds__(kVT) bicg_p_kernel(BiPtrs P) {
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const int n = P.d->n;
  const double beta = __ldcg(&P.st->beta), omega = __ldcg(&P.st->omega);
  const int stride = gridDim.x * kVT;
  for (int i0 = blockIdx.x * kVT + threadIdx.x; i0 < n; i0 += kU * stride) {
    double ri[kU], pi[kU], vi[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        ri[u] = __ldg(P.r + i);
        pi[u] = P.p[i];
        vi[u] = __ldg(P.v + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) P.p[i] = fma(beta, fma(-omega, vi[u], pi[u]), ri[u]);
    }
  }
}

// -------------------------------------------------------------- KB / KD
// which == 0: v = A^ p, partial r^.v ;  which == 1: t = A^ s, partials t.t, t.s
// (A^ = A D^{-1}; r^ here is the shadow residual r0, not a preconditioned vector)
// run(x, aux, epi) performs y = A x through one of the SpMV schemes.
template <int which, int NT, int M, class Run>
__device__ __forceinline__ void bicg_spmv_body(const BiPtrs& P, double (&red)[M], bool* s_last, Run&& run) {
  double a0 = 0.0, a1 = 0.0;
  if (which == 0) {
    double* __restrict__ v = P.v;
    run(P.p, P.rh, [&](int row, double y, double rhr) {
      v[row] = y;
      a0 = fma(rhr, y, a0);
    });
  } else {
    double* __restrict__ t = P.t;
    run(P.s, P.s, [&](int row, double y, double sr) {
      t[row] = y;
      a0 = fma(y, y, a0);
      a1 = fma(y, sr, a1);
    });
  }
  double acc[2] = {a0, a1};
  block_sums<NT, 2>(acc, red);
  if (threadIdx.x == 0) {
    P.part[blockIdx.x] = acc[0];
    P.part[kMaxBlocks + blockIdx.x] = acc[1];
  }
  if (!last_block_arrive(&P.st->cnt[which == 0 ? 1 : 3], s_last)) return;
  reduce_partials<NT, 2>(P.part, kMaxBlocks, gridDim.x, acc, red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    if (__ldcg(&s.err) != 0) {
      s.status = SLA_ERR_TIMEOUT;
      s.phase = kPhaseDone;
    } else if (which == 0) {
      const double rv = acc[0];
      if (!isfinite(rv) || rv == 0.0) {
        s.status = SLA_BREAKDOWN;
        s.phase = kPhaseDone;
      } else {
        s.alpha = s.rho / rv;
      }
    } else {
      const double tt = acc[0], ts = acc[1];
      s.tt = tt;
      s.ts = ts;
      if (!isfinite(tt) || !isfinite(ts) || tt == 0.0) {
        s.status = SLA_BREAKDOWN;
        s.phase = kPhaseDone;
      } else {
        s.omega = ts / tt;
      }
    }
  }
}

template <int which>
__global__ void __launch_bounds__(tma::kThreads, 3) bicg_spmv_tma_kernel(BiPtrs P) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::Smem& sm = *reinterpret_cast<tma::Smem*>(dsm);
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  bicg_spmv_body<which, tma::kThreads>(P, sm.red, &sm.last, [&](const double* x, const double* aux, auto&& epi) {
    tma::spmv_pipeline(d.n, d.nnz, d.rowptr, d.col, bicg_vals(P, d), x, aux, sm, &P.st->err, epi);
  });
}

template <int which>
__global__ void __launch_bounds__(kRowThreads) bicg_spmv_rows_kernel(BiPtrs P) {
  __shared__ double red[2 * kRowThreads + 2];
  __shared__ bool s_last;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  bicg_spmv_body<which, kRowThreads>(P, red, &s_last, [&](const double* x, const double* aux, auto&& epi) {
    csr_rows(d.n, d.rowptr, d.col, bicg_vals(P, d), x, aux, epi);
  });
}

// -------------------------------------------------------------- KC
__global__ void __launch_bounds__(kVT) bicg_s_kernel(BiPtrs P) {
  __shared__ VSmem sm;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const int n = P.d->n;
  const double alpha = __ldcg(&P.st->alpha);
  const int stride = gridDim.x * kVT;
  double ss0 = 0.0, ss1 = 0.0;
  for (int i0 = blockIdx.x * kVT + threadIdx.x; i0 < n; i0 += kU * stride) {
    double ri[kU], vi[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        ri[u] = __ldg(P.r + i);
        vi[u] = __ldg(P.v + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        const double sn = fma(-alpha, vi[u], ri[u]);
        P.s[i] = sn;
        if (u & 1) ss1 = fma(sn, sn, ss1);
        else ss0 = fma(sn, sn, ss0);
      }
    }
  }
  double acc[1] = {ss0 + ss1};
  block_sums<kVT, 1>(acc, sm.red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = acc[0];
  if (!last_block_arrive(&P.st->cnt[2], &sm.last)) return;
  reduce_partials<kVT, 1>(P.part, kMaxBlocks, gridDim.x, acc, sm.red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    s.iters += 1;
    s.ss = acc[0];
    if (sqrt(acc[0]) <= s.thresh) {  // half-step exit: x^ += alpha p in KE
      s.rr = acc[0];
      s.status = SLA_OK;
      s.phase = kPhaseHalf;
    }
  }
}

// -------------------------------------------------------------- KE
__global__ void __launch_bounds__(kVT)
bicg_x_kernel(BiPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ VSmem sm;
  const int phase = __ldcg(&P.st->phase);
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int stride = gridDim.x * kVT;
  double acc[2] = {0.0, 0.0};
  if (phase == kPhaseRun) {
    const double alpha = __ldcg(&P.st->alpha), omega = __ldcg(&P.st->omega);
    double rr1 = 0.0, rh1 = 0.0;
    for (int i0 = blockIdx.x * kVT + threadIdx.x; i0 < n; i0 += kU * stride) {
      double xi[kU], phi[kU], si[kU], ti[kU], rhi[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * stride;
        if (i < n) {
          xi[u] = d.x[i];
          phi[u] = __ldg(P.p + i);
          si[u] = __ldg(P.s + i);
          ti[u] = __ldg(P.t + i);
          rhi[u] = __ldg(P.rh + i);
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * stride;
        if (i < n) {
          d.x[i] = fma(omega, si[u], fma(alpha, phi[u], xi[u]));
          const double rn = fma(-omega, ti[u], si[u]);
          P.r[i] = rn;
          if (u & 1) {
            rr1 = fma(rn, rn, rr1);
            rh1 = fma(rhi[u], rn, rh1);
          } else {
            acc[0] = fma(rn, rn, acc[0]);
            acc[1] = fma(rhi[u], rn, acc[1]);
          }
        }
      }
    }
    acc[0] += rr1;
    acc[1] += rh1;
  } else if (phase == kPhaseHalf) {
    const double alpha = __ldcg(&P.st->alpha);
    for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride)
      d.x[i] = fma(alpha, __ldg(P.p + i), d.x[i]);
  } else if (phase == kPhaseCheck) {
    for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) {
      const double ti = d.b[i] - row_dot(d.rowptr, d.col, bicg_vals(P, d), d.x, i);
      P.r[i] = ti;
      P.rh[i] = ti;
      P.p[i] = 0.0;
      P.v[i] = 0.0;
      acc[0] = fma(ti, ti, acc[0]);
    }
  }
  if (phase == kPhaseRun || phase == kPhaseCheck) {
    block_sums<kVT, 2>(acc, sm.red);
    if (threadIdx.x == 0) {
      P.part[blockIdx.x] = acc[0];
      P.part[kMaxBlocks + blockIdx.x] = acc[1];
    }
  }
  if (!last_block_arrive(&P.st->cnt[4], &sm.last)) return;
  if (phase == kPhaseRun || phase == kPhaseCheck)
    reduce_partials<kVT, 2>(P.part, kMaxBlocks, gridDim.x, acc, sm.red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    if (phase == kPhaseRun) {
      const double rr = acc[0], rho_new = acc[1];
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
    } else if (phase == kPhaseHalf) {
      s.phase = kPhaseCheck;
    } else if (phase == kPhaseCheck) {
      const double tt = acc[0];
      s.tt = tt;
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
    s.body += 1;
    const int cap = 2 * d.max_iter + 3 * d.max_restarts + 8;
    if (s.phase != kPhaseDone && s.body > cap) {
      s.status = SLA_NOT_CONVERGED;
      s.phase = kPhaseDone;
    }
    if (use_cond) cudaGraphSetConditional(cond, s.phase != kPhaseDone ? 1u : 0u);
  }
}

// -------------------------------------------------------------- final
__global__ void __launch_bounds__(kVT) bicg_final_kernel(BiPtrs P) {
  __shared__ VSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int zero_rhs = __ldcg(&P.st->zero_rhs), bad = __ldcg(&P.st->bad_diag);
  const int stride = gridDim.x * kVT;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) {
    if (zero_rhs) {
      d.x[i] = 0.0;
    } else if (!bad) {
      const double ti = d.b[i] - row_dot(d.rowptr, d.col, bicg_vals(P, d), d.x, i);
      acc[0] = fma(ti, ti, acc[0]);
    }
  }
  block_sums<kVT, 1>(acc, sm.red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = acc[0];
  if (!last_block_arrive(&P.st->cnt[5], &sm.last)) return;
  reduce_partials<kVT, 1>(P.part, kMaxBlocks, gridDim.x, acc, sm.red);
  if (threadIdx.x == 0) {
    const KrylovState& s = *P.st;
    sla_info inf;
    inf.iters = s.iters;
    inf.status = s.phase == kPhaseDone ? s.status : SLA_NOT_CONVERGED;
    if (s.zero_rhs) {
      inf.rel_res = inf.true_rel_res = 0.0;
    } else if (s.bad_diag) {
      inf.rel_res = inf.true_rel_res = NAN;
    } else {
      inf.rel_res = sqrt(s.rr) / s.bnorm;
      inf.true_rel_res = sqrt(acc[0]) / s.bnorm;
    }
    *d.info = inf;
  }
}

// -------------------------------------------------------------- host side
struct BiGraphKey {
  int dev;
  const void* ws;
  int n, nnz, gs, gv, kind;
  bool operator==(const BiGraphKey& o) const {
    return dev == o.dev && ws == o.ws && n == o.n && nnz == o.nnz && gs == o.gs && gv == o.gv && kind == o.kind;
  }
};

std::mutex g_mu;
std::vector<std::pair<BiGraphKey, cudaGraphExec_t>> g_cache;

// The two SpMV kernels of the body: row-per-thread for n <= kRowsKernelMaxN,
// else the TMA pipeline.
struct SpmvKernels {
  const void* kb;
  const void* kd;
  int threads;
  unsigned smem;
  int kind;
};

SpmvKernels spmv_kernels(int n) {
  if (spmv_kind(n) == kSpmvRows)
    return SpmvKernels{(const void*)bicg_spmv_rows_kernel<0>, (const void*)bicg_spmv_rows_kernel<1>, kRowThreads, 0u,
                       kSpmvRows};
  return SpmvKernels{(const void*)bicg_spmv_tma_kernel<0>, (const void*)bicg_spmv_tma_kernel<1>, tma::kThreads,
                     (unsigned)tma::kSmemBytes, kSpmvTma};
}

void grids(int dev, int n, const SpmvKernels& k, int* gs, int* gv) {
  static int occ_s = 0, occ_r = 0, occ_v = 0;
  if (occ_s == 0) {
    cudaFuncSetAttribute(bicg_spmv_tma_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma::kSmemBytes);
    cudaFuncSetAttribute(bicg_spmv_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma::kSmemBytes);
    occ_s = occupancy((const void*)bicg_spmv_tma_kernel<0>, tma::kThreads, tma::kSmemBytes);
    occ_r = occupancy((const void*)bicg_spmv_rows_kernel<1>, kRowThreads);
  }
  if (occ_v == 0) occ_v = occupancy((const void*)bicg_x_kernel, kVT);
  if (k.kind == kSpmvRows)
    *gs = persistent_grid(dev, ((long long)n + kRowThreads - 1) / kRowThreads, occ_r < 8 ? occ_r : 8, kMaxBlocks);
  else
    *gs = persistent_grid(dev, (n + tma::kRows - 1) / tma::kRows, occ_s, kMaxBlocks);
  *gv = persistent_grid(dev, ((long long)n + kVT - 1) / kVT, occ_v, kMaxBlocks);
}

int build_graph(BiPtrs P, const SpmvKernels& k, int gs, int gv, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  SLA_CUDA_TRY(cudaGraphCreate(&g, 0));
  int rc = SLA_ERR_CUDA;
  do {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNode_t n_init, n_scale, n_while, na, nb, nc, nd, ne, n_final, n_unscale;
    void* a[] = {&P};
    int use_cond = 1;
    void* ae[] = {&P, &h, &use_cond};
    if (add_kernel(g, nullptr, 0, &n_init, (const void*)bicg_init_kernel, gv, kVT, a) != cudaSuccess) break;
    if (add_kernel(g, &n_init, 1, &n_scale, (const void*)bicg_scale_kernel, gv, kVT, a) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&n_while, g, &n_scale, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (add_kernel(body, nullptr, 0, &na, (const void*)bicg_p_kernel, gv, kVT, a) != cudaSuccess) break;
    if (add_kernel(body, &na, 1, &nb, k.kb, gs, k.threads, a, k.smem) != cudaSuccess) break;
    if (add_kernel(body, &nb, 1, &nc, (const void*)bicg_s_kernel, gv, kVT, a) != cudaSuccess) break;
    if (add_kernel(body, &nc, 1, &nd, k.kd, gs, k.threads, a, k.smem) != cudaSuccess) break;
    if (add_kernel(body, &nd, 1, &ne, (const void*)bicg_x_kernel, gv, kVT, ae) != cudaSuccess) break;
    if (add_kernel(g, &n_while, 1, &n_final, (const void*)bicg_final_kernel, gv, kVT, a) != cudaSuccess) break;
    if (add_kernel(g, &n_final, 1, &n_unscale, (const void*)bicg_unscale_kernel, gv, kVT, a) != cudaSuccess)
      break;
    if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) break;
    rc = SLA_OK;
  } while (0);
  cudaGraphDestroy(g);
  return rc;
}

int run_host_loop(BiPtrs P, const KrylovDesc& desc, const SpmvKernels& k, int gs, int gv, cudaStream_t s) {
  void* a[] = {&P};
  bicg_write_desc_kernel<<<1, 1, 0, s>>>(P.d, desc, P.st);
  bicg_init_kernel<<<gv, kVT, 0, s>>>(P);
  bicg_scale_kernel<<<gv, kVT, 0, s>>>(P);
  const long long cap = 2LL * desc.max_iter + 3LL * desc.max_restarts + 8;
  for (long long body = 0; body < cap; ++body) {
    bicg_p_kernel<<<gv, kVT, 0, s>>>(P);
    SLA_CUDA_TRY(cudaLaunchKernel(k.kb, dim3(gs), dim3(k.threads), a, k.smem, s));
    bicg_s_kernel<<<gv, kVT, 0, s>>>(P);
    SLA_CUDA_TRY(cudaLaunchKernel(k.kd, dim3(gs), dim3(k.threads), a, k.smem, s));
    bicg_x_kernel<<<gv, kVT, 0, s>>>(P, cudaGraphConditionalHandle(0), 0);
    if ((body + 1) % 16 == 0) {
      int phase = 0;
      SLA_CUDA_TRY(cudaMemcpyAsync(&phase, &P.st->phase, sizeof(int), cudaMemcpyDeviceToHost, s));
      SLA_CUDA_TRY(cudaStreamSynchronize(s));
      if (phase == kPhaseDone) break;
    }
  }
  bicg_final_kernel<<<gv, kVT, 0, s>>>(P);
  bicg_unscale_kernel<<<gv, kVT, 0, s>>>(P);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaStreamSynchronize(s));
  return SLA_OK;
}

}  // namespace

bool use_bicg_coop(long long n);
int launch_bicgstab_coop(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched);

int launch_bicgstab(const KrylovDesc& desc, void* ws, cudaStream_t s, int flags) {
  if (!(flags & (SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP)) && use_bicg_coop(desc.n)) {
    // one cooperative launch per solve (sla_bicgstab_coop.cu) where the device runs it
    bool launched = false;
    const int rc = launch_bicgstab_coop(desc, ws, s, &launched);
    if (rc != SLA_OK || launched) return rc;
  }
  const BiLayout L = bicg_layout(desc.n);
  char* base = (char*)ws;
  BiPtrs P;
  P.d = (KrylovDesc*)(base + L.desc);
  P.st = (KrylovState*)(base + L.state);
  P.part = (double*)(base + L.part);
  double* vecs[9];
  for (int j = 0; j < 9; ++j) vecs[j] = (double*)(base + L.vec + (size_t)j * L.vec_stride);
  P.r = vecs[0]; P.rh = vecs[1]; P.p = vecs[2]; P.ph = vecs[3]; P.v = vecs[4];
  P.s = vecs[5]; P.sh = vecs[6]; P.t = vecs[7]; P.dinv = vecs[8];
  P.valh = (double*)(base + al256(L.total));
  const int dev = current_device();
  int gs, gv;
  const SpmvKernels sk = spmv_kernels(desc.n);
  grids(dev, desc.n, sk, &gs, &gv);
  if (flags & SLA_FLAG_HOST_LOOP) return run_host_loop(P, desc, sk, gs, gv, s);
  BiGraphKey key{dev, ws, desc.n, desc.nnz, gs, gv, sk.kind};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& e : g_cache)
      if (e.first == key) exec = e.second;
    if (exec == nullptr) {
      const int rc = build_graph(P, sk, gs, gv, &exec);
      if (rc != SLA_OK) return rc;
      if (g_cache.size() >= 64) {
        SLA_CUDA_TRY(cudaDeviceSynchronize());
        for (auto& e : g_cache) cudaGraphExecDestroy(e.second);
        g_cache.clear();
      }
      g_cache.push_back({key, exec});
    }
  }
  bicg_write_desc_kernel<<<1, 1, 0, s>>>(P.d, desc, P.st);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaGraphLaunch(exec, s));
  return SLA_OK;
}

KrylovDesc make_desc(const sla_csr* A, const double* val, const double* b, double* x,
                     const sla_opts* o, sla_info* info) {
  KrylovDesc d = {};
  d.n = A->n;
  d.nnz = A->nnz;
  d.rowptr = A->rowptr;
  d.col = A->col;
  d.val = val;
  d.b = b;
  d.x = x;
  d.info = info;
  d.rtol = o->rtol;
  d.atol = o->atol;
  d.max_iter = o->max_iter;
  d.max_restarts = o->max_restarts;
  d.precond = o->precond;
  d.use_x0 = o->use_x0;
  d.sym_scale = o->precond == SLA_PRECOND_JACOBI ? 1 : 0;  // read by the CG kernels only
  return d;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_bicgstab(const sla_csr* A, const double* val, const double* b, double* x,
                                const sla_opts* opts, sla_info* info, void* ws, size_t ws_bytes,
                                void* stream) {
  if (A == nullptr) return SLA_ERR_INVALID;
  const size_t need = bicg_ws_bytes(A->n > 0 ? A->n : 0, A->nnz > 0 ? A->nnz : 0);
  int rc = validate_solve_args(A, val, b, x, opts, info, ws, ws_bytes, need);
  if (rc != SLA_OK) return rc;
  if (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n == 0) return write_info(info, sla_info{0, SLA_OK, 0.0, 0.0}, s);
  return launch_bicgstab(make_desc(A, val, b, x, opts, info), ws, s, opts->flags);
}
