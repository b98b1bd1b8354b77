// sla_cg_ggt.cu -- PCG with a factored approximate inverse M^{-1} = G G^T.
//
// Algorithm 1 (P = 1) with z = G (G^T r).  G is lower triangular (for the
// learned preconditioner it lives on the pattern of tril(A)); applying it
// as two SpMVs keeps M SPD for any nonsingular G.  One iteration is four
// kernels in the graph's WHILE body:
//
//   K1  q = A p, partial p.q                    -> alpha
//       (phase CHECK: r = b - A x, the true residual, and the restart rule)
//   K2  x += alpha p, r -= alpha q, partial r.r -> iteration count
//   GT  t = G^T r, partial t.t                  -> convergence, beta
//   GZ  p = G t + beta p   (p = G t right after a (re)start)
//
// r.z = r^T G G^T r = ||G^T r||^2, so the preconditioned inner product comes
// from GT's epilogue, and since beta is known before GZ starts, z = G t is
// folded into the p update and never stored.  The loop condition is set
// once per body: by GT's last block, or by K1's when it ends the solve.  The factor's values are
// held in FP32 (converted once per solve; the network produces FP32 values
// anyway) and widened exactly inside the SpMVs: the preconditioner is the
// fixed SPD operator G32 G32^T, while the recurrence and the residual check
// stay FP64.  Phase PRECOND (start and after a restart) runs only GT and GZ.
// Algorithmic bytes per iteration: 12 nnz + 4(n+1) + 2 (8 nnz_g + 4(n+1))
// + 96 n.
#include <cmath>
#include <mutex>
#include <vector>

#include "sla_internal.cuh"
#include "sla_tma.cuh"
#include "sla_workspace.h"

namespace sla {
namespace {

constexpr int kVT = 256;
constexpr int kU = 4;
constexpr int kPhasePrecond = 4;

struct GPtrs {
  KrylovDesc* d;
  KrylovState* st;
  double* part;
  double *r, *z, *p, *q, *t;
  float *gv, *gtv;
};

// FP32 copy of a factor value, subnormals flushed (the widening in the
// SpMVs maps them to zero, so both operators see the same value).
__device__ __forceinline__ float f32_of(double v) {
  float f = __double2float_rn(v);
  if (fabsf(f) < 1.17549435e-38f) f = 0.0f;
  return f;
}

struct VSmem {
  double red[4 * kVT + 4];
  bool last;
};

// FP32 values of G and of G^T (gathered through perm_t), for the
// cooperative solve, which takes them ready-made.
__global__ void __launch_bounds__(kVT) ggt_values_kernel(const double* __restrict__ g_val,
                                                         const int* __restrict__ perm_t, int nnz_g,
                                                         float* __restrict__ gv, float* __restrict__ gtv) {
  const int stride = gridDim.x * kVT;
  for (int k = blockIdx.x * kVT + threadIdx.x; k < nnz_g; k += stride) {
    gv[k] = f32_of(__ldg(g_val + k));
    gtv[k] = f32_of(__ldg(g_val + __ldg(perm_t + k)));
  }
}

__global__ void ggt_write_desc_kernel(KrylovDesc* dst, KrylovDesc src, KrylovState* st) {
  *dst = src;
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
  st->fresh_p = 0;
}

// r = b - A x0 (x = 0 unless use_x0), partial ||b||^2, ||r||^2; gathers the
// values of G^T.
__global__ void __launch_bounds__(kVT) ggt_init_kernel(GPtrs P) {
  __shared__ VSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int stride = gridDim.x * kVT;
  for (long long k = blockIdx.x * (long long)kVT + threadIdx.x; k < d.nnz_g; k += stride) {
    P.gv[k] = f32_of(__ldg(d.g_val + k));
    P.gtv[k] = f32_of(__ldg(d.g_val + __ldg(d.perm_t + k)));
  }
  double acc[2] = {0.0, 0.0};
  for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) {
    const double ax = d.use_x0 ? row_dot(d.rowptr, d.col, d.val, d.x, i) : 0.0;
    const double bi = d.b[i];
    const double ri = bi - ax;
    P.r[i] = ri;
    acc[0] = fma(bi, bi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
  }
  if (!d.use_x0)
    for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) d.x[i] = 0.0;
  block_sums<kVT, 2>(acc, sm.red);
  if (threadIdx.x == 0) {
    P.part[blockIdx.x] = acc[0];
    P.part[kMaxBlocks + blockIdx.x] = acc[1];
  }
  if (!last_block_arrive(&P.st->cnt[0], &sm.last)) return;
  reduce_partials<kVT, 2>(P.part, kMaxBlocks, gridDim.x, acc, sm.red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    s.bnorm = sqrt(acc[0]);
    s.thresh = fmax(d.rtol * s.bnorm, d.atol);
    s.rr = acc[1];
    s.rho = s.alpha = s.beta = 0.0;
    s.iters = s.restarts = s.body = 0;
    s.zero_rhs = s.bad_diag = 0;
    s.fresh_p = 0;
    s.status = SLA_NOT_CONVERGED;
    if (s.bnorm == 0.0) {
      s.zero_rhs = 1;
      s.status = SLA_OK;
      s.phase = kPhaseDone;
    } else {
      s.phase = kPhasePrecond;
    }
  }
}

// Ends the loop: marks the solve done and clears the WHILE condition.
__device__ __forceinline__ void finish(KrylovState& s, int status, cudaGraphConditionalHandle cond,
                                       int use_cond) {
  s.status = status;
  s.phase = kPhaseDone;
  if (use_cond) cudaGraphSetConditional(cond, 0u);
}

// K1: RUN: q = A p, p.q -> alpha.  CHECK: r = b - A x (true residual) ->
// done, or a restart through phase PRECOND.  DONE at entry: clear the loop
// condition (nothing else runs in this body).  run(x, aux, epi) performs the
// SpMV y = A x through one of the schemes.
template <int NT, int M, class Run>
__device__ __forceinline__ void ggt_k1_body(GPtrs P, int ph, cudaGraphConditionalHandle cond, int use_cond,
                                            double (&red)[M], bool* s_last, Run&& run) {
  const KrylovDesc d = *P.d;
  double acc = 0.0;
  if (ph == kPhaseRun) {
    double* __restrict__ q = P.q;
    run(P.p, P.p, [&](int row, double y, double prow) {
      q[row] = y;
      acc = fma(prow, y, acc);
    });
  } else {
    double* __restrict__ r = P.r;
    run(d.x, d.b, [&](int row, double y, double brow) {
      const double ti = brow - y;
      r[row] = ti;
      acc = fma(ti, ti, acc);
    });
  }
  double v[1] = {acc};
  block_sums<NT, 1>(v, red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[1], s_last)) return;
  reduce_partials<NT, 1>(P.part, kMaxBlocks, gridDim.x, v, red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    if (__ldcg(&s.err) != 0) {
      finish(s, SLA_ERR_TIMEOUT, cond, use_cond);
    } else if (ph == kPhaseRun) {
      if (!isfinite(v[0])) finish(s, SLA_BREAKDOWN, cond, use_cond);
      else if (!(v[0] > 0.0)) finish(s, SLA_NOT_SPD, cond, use_cond);
      else s.alpha = s.rho / v[0];
    } else {
      const double tt = v[0];
      s.tt = tt;
      if (sqrt(tt) <= 2.0 * s.thresh) finish(s, SLA_OK, cond, use_cond);
      else if (!isfinite(tt)) finish(s, SLA_BREAKDOWN, cond, use_cond);
      else if (s.restarts >= d.max_restarts || s.iters >= d.max_iter)
        finish(s, SLA_NOT_CONVERGED, cond, use_cond);
      else {
        s.restarts += 1;
        s.rr = tt;
        s.status = SLA_NOT_CONVERGED;
        s.phase = kPhasePrecond;
      }
    }
  }
}

// Phase gate of K1: DONE clears the loop condition; only RUN and CHECK work.
__device__ __forceinline__ int ggt_k1_phase(const GPtrs& P, cudaGraphConditionalHandle cond, int use_cond) {
  const int ph = __ldcg(&P.st->phase);
  if (ph == kPhaseDone && blockIdx.x == 0 && threadIdx.x == 0 && use_cond) cudaGraphSetConditional(cond, 0u);
  return ph;
}

__global__ void __launch_bounds__(tma::kThreads, 3)
ggt_spmv_pq_kernel(GPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::Smem& sm = *reinterpret_cast<tma::Smem*>(dsm);
  const int ph = ggt_k1_phase(P, cond, use_cond);
  if (ph != kPhaseRun && ph != kPhaseCheck) return;
  const KrylovDesc d = *P.d;
  ggt_k1_body<tma::kThreads>(P, ph, cond, use_cond, sm.red, &sm.last, [&](const double* x, const double* aux, auto&& epi) {
    tma::spmv_pipeline(d.n, d.nnz, d.rowptr, d.col, d.val, x, aux, sm, &P.st->err, epi);
  });
}

__global__ void __launch_bounds__(kRowThreads)
ggt_spmv_pq_rows_kernel(GPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double red[kRowThreads + 2];
  __shared__ bool s_last;
  const int ph = ggt_k1_phase(P, cond, use_cond);
  if (ph != kPhaseRun && ph != kPhaseCheck) return;
  const KrylovDesc d = *P.d;
  ggt_k1_body<kRowThreads>(P, ph, cond, use_cond, red, &s_last, [&](const double* x, const double* aux, auto&& epi) {
    csr_rows(d.n, d.rowptr, d.col, d.val, x, aux, epi);
  });
}

// K2: x += alpha p, r -= alpha q, ||r||^2 (RUN only)
__global__ void __launch_bounds__(kVT) ggt_update_kernel(GPtrs P) {
  __shared__ VSmem sm;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const double alpha = __ldcg(&P.st->alpha);
  const int stride = gridDim.x * kVT;
  double rr0 = 0.0, rr1 = 0.0;
  for (int i0 = blockIdx.x * kVT + threadIdx.x; i0 < n; i0 += kU * stride) {
    double pi[kU], qi[kU], xi[kU], ri[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        pi[u] = __ldg(P.p + i);
        qi[u] = __ldg(P.q + i);
        xi[u] = d.x[i];
        ri[u] = P.r[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        d.x[i] = fma(alpha, pi[u], xi[u]);
        const double rn = fma(-alpha, qi[u], ri[u]);
        P.r[i] = rn;
        if (u & 1) rr1 = fma(rn, rn, rr1);
        else rr0 = fma(rn, rn, rr0);
      }
    }
  }
  double v[1] = {rr0 + rr1};
  block_sums<kVT, 1>(v, sm.red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[2], &sm.last)) return;
  reduce_partials<kVT, 1>(P.part, kMaxBlocks, gridDim.x, v, sm.red);
  if (threadIdx.x == 0) {
    P.st->rr = v[0];
    P.st->iters += 1;
  }
}

// GT: t = G^T r and ||t||^2 = r.z; decisions (RUN: convergence and beta;
// PRECOND: rho and a fresh p).  run(epi) performs t = G^T r.
template <int NT, int M, class Run>
__device__ __forceinline__ void ggt_gt_body(GPtrs P, int ph, cudaGraphConditionalHandle cond, int use_cond,
                                            double (&red)[M], bool* s_last, Run&& run) {
  const KrylovDesc d = *P.d;
  double* __restrict__ t = P.t;
  double tt = 0.0;
  run([&](int row, double y, double) {
    t[row] = y;
    tt = fma(y, y, tt);
  });
  double v[1] = {tt};
  block_sums<NT, 1>(v, red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[3], s_last)) return;
  reduce_partials<NT, 1>(P.part, kMaxBlocks, gridDim.x, v, red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    const double trz = v[0], rnorm = sqrt(s.rr);
    if (__ldcg(&s.err) != 0) {
      s.status = SLA_ERR_TIMEOUT;
      s.phase = kPhaseDone;
    } else if (ph == kPhasePrecond) {
      s.rho = trz;
      s.fresh_p = 1;
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
        s.fresh_p = 0;
        if (s.iters >= d.max_iter) {
          s.status = SLA_NOT_CONVERGED;
          s.phase = kPhaseDone;
        }
      }
    }
    // hard cap on loop bodies (each advances the iteration count or a
    // restart); only fires if the state machine is broken
    s.body += 1;
    if (s.phase != kPhaseDone && s.body > d.max_iter + 3 * d.max_restarts + 8) {
      s.status = SLA_NOT_CONVERGED;
      s.phase = kPhaseDone;
    }
    if (use_cond) cudaGraphSetConditional(cond, s.phase != kPhaseDone ? 1u : 0u);
  }
}

// Two rows per thread need more registers: three blocks per SM for RPT = 2.
template <int RPT>
__global__ void __launch_bounds__(tma::kThreads, RPT == 2 ? 3 : tma::kMinBlocks)
ggt_gt_kernel(GPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::SmemT<float, RPT>& sm = *reinterpret_cast<tma::SmemT<float, RPT>*>(dsm);
  const int ph = __ldcg(&P.st->phase);
  if (ph != kPhaseRun && ph != kPhasePrecond) return;
  const KrylovDesc d = *P.d;
  ggt_gt_body<tma::kThreads>(P, ph, cond, use_cond, sm.red, &sm.last, [&](auto&& epi) {
    tma::spmv_pipeline<RPT>(d.n, d.nnz_g, d.rowptr_t, d.col_t, (const float*)P.gtv, P.r, (const double*)nullptr,
                            sm, &P.st->err, epi);
  });
}

__global__ void __launch_bounds__(kRowThreads) ggt_gt_rows_kernel(GPtrs P, cudaGraphConditionalHandle cond,
                                                                  int use_cond) {
  __shared__ double red[kRowThreads + 2];
  __shared__ bool s_last;
  const int ph = __ldcg(&P.st->phase);
  if (ph != kPhaseRun && ph != kPhasePrecond) return;
  const KrylovDesc d = *P.d;
  ggt_gt_body<kRowThreads>(P, ph, cond, use_cond, red, &s_last, [&](auto&& epi) {
    csr_rows(d.n, d.rowptr_t, d.col_t, (const float*)P.gtv, P.r, (const double*)nullptr, epi);
  });
}

// GZ: p = G t + beta p (p = G t right after a (re)start); RUN only, after GT
template <int RPT>
__global__ void __launch_bounds__(tma::kThreads, RPT == 2 ? 3 : tma::kMinBlocks) ggt_gz_kernel(GPtrs P) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::SmemT<float, RPT>& sm = *reinterpret_cast<tma::SmemT<float, RPT>*>(dsm);
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  // after a (re)start p holds stale memory (possibly NaN): do not read it
  const bool fresh = __ldcg(&P.st->fresh_p) != 0;
  const double beta = fresh ? 0.0 : __ldcg(&P.st->beta);
  const KrylovDesc d = *P.d;
  double* __restrict__ p = P.p;
  tma::spmv_pipeline<RPT>(d.n, d.nnz_g, d.g_rowptr, d.g_col, (const float*)P.gv, P.t, fresh ? nullptr : p, sm,
                     &P.st->err, [&](int row, double y, double prow) { p[row] = fma(beta, prow, y); });
}

__global__ void __launch_bounds__(kRowThreads) ggt_gz_rows_kernel(GPtrs P) {
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const bool fresh = __ldcg(&P.st->fresh_p) != 0;
  const double beta = fresh ? 0.0 : __ldcg(&P.st->beta);
  const KrylovDesc d = *P.d;
  double* __restrict__ p = P.p;
  csr_rows(d.n, d.g_rowptr, d.g_col, (const float*)P.gv, P.t, fresh ? nullptr : p,
           [&](int row, double y, double prow) { p[row] = fma(beta, prow, y); });
}

__global__ void __launch_bounds__(kVT) ggt_final_kernel(GPtrs P) {
  __shared__ VSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int zero_rhs = __ldcg(&P.st->zero_rhs);
  const int stride = gridDim.x * kVT;
  double v[1] = {0.0};
  for (int i = blockIdx.x * kVT + threadIdx.x; i < n; i += stride) {
    if (zero_rhs) {
      d.x[i] = 0.0;
    } else {
      const double ti = d.b[i] - row_dot(d.rowptr, d.col, d.val, d.x, i);
      v[0] = fma(ti, ti, v[0]);
    }
  }
  block_sums<kVT, 1>(v, sm.red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[5], &sm.last)) return;
  reduce_partials<kVT, 1>(P.part, kMaxBlocks, gridDim.x, v, sm.red);
  if (threadIdx.x == 0) {
    const KrylovState& s = *P.st;
    sla_info inf;
    inf.iters = s.iters;
    inf.status = s.phase == kPhaseDone ? s.status : SLA_NOT_CONVERGED;
    if (s.zero_rhs) {
      inf.rel_res = inf.true_rel_res = 0.0;
    } else {
      inf.rel_res = sqrt(s.rr) / s.bnorm;
      inf.true_rel_res = sqrt(v[0]) / s.bnorm;
    }
    *d.info = inf;
  }
}

// One loop kernel of the body: function, grid, block, dynamic shared memory.
struct LoopKernel {
  const void* fn;
  int grid, threads;
  unsigned smem;
};

// The body's SpMV kernels: K1 (A), GT (G^T), GZ (G).  Row-per-thread kernels
// for n <= kRowsKernelMaxN, else the TMA pipeline, whose factor SpMVs take two
// rows per consumer thread (512-row tiles) when G averages at most 4 entries
// per row, so that a tile still fits a stage.
struct BodyKernels {
  LoopKernel k1, gt, gz;
  int gv, kind, rpt;
};

int factor_rpt(int n, int nnz_g) { return (long long)nnz_g <= 4LL * n ? 2 : 1; }

BodyKernels body_kernels(int dev, int n, int nnz_g) {
  static std::once_flag once;
  static int occ_s = 0, occ_v = 0, occ_g[3] = {0, 0, 0}, occ_r[3] = {0, 0, 0};
  std::call_once(once, [] {
    cudaFuncSetAttribute(ggt_spmv_pq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::kSmemBytes);
    cudaFuncSetAttribute(ggt_gt_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::kSmemBytesF32);
    cudaFuncSetAttribute(ggt_gz_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::kSmemBytesF32);
    cudaFuncSetAttribute(ggt_gt_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::kSmemBytesF32x2);
    cudaFuncSetAttribute(ggt_gz_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma::kSmemBytesF32x2);
    occ_s = occupancy((const void*)ggt_spmv_pq_kernel, tma::kThreads, tma::kSmemBytes);
    occ_g[1] = occupancy((const void*)ggt_gt_kernel<1>, tma::kThreads, tma::kSmemBytesF32);
    occ_g[2] = occupancy((const void*)ggt_gt_kernel<2>, tma::kThreads, tma::kSmemBytesF32x2);
    occ_r[0] = occupancy((const void*)ggt_spmv_pq_rows_kernel, kRowThreads);
    occ_r[1] = occupancy((const void*)ggt_gt_rows_kernel, kRowThreads);
    occ_r[2] = occupancy((const void*)ggt_gz_rows_kernel, kRowThreads);
    occ_v = occupancy((const void*)ggt_update_kernel, kVT);
  });
  BodyKernels k;
  k.kind = spmv_kind(n) == kSpmvRows ? kSpmvRows : kSpmvTma;
  k.rpt = factor_rpt(n, nnz_g);
  k.gv = persistent_grid(dev, ((long long)n + kVT - 1) / kVT, occ_v, kMaxBlocks);
  if (k.kind == kSpmvRows) {
    const long long blocks = ((long long)n + kRowThreads - 1) / kRowThreads;
    auto g = [&](int occ) { return persistent_grid(dev, blocks, occ < 8 ? occ : 8, kMaxBlocks); };
    k.k1 = LoopKernel{(const void*)ggt_spmv_pq_rows_kernel, g(occ_r[0]), kRowThreads, 0u};
    k.gt = LoopKernel{(const void*)ggt_gt_rows_kernel, g(occ_r[1]), kRowThreads, 0u};
    k.gz = LoopKernel{(const void*)ggt_gz_rows_kernel, g(occ_r[2]), kRowThreads, 0u};
  } else {
    const int tr = tma::kRows * k.rpt;
    const int gs = persistent_grid(dev, (n + tma::kRows - 1) / tma::kRows, occ_s, kMaxBlocks);
    const int gg = persistent_grid(dev, (n + tr - 1) / tr, occ_g[k.rpt], kMaxBlocks);
    k.k1 = LoopKernel{(const void*)ggt_spmv_pq_kernel, gs, tma::kThreads, (unsigned)tma::kSmemBytes};
    if (k.rpt == 2) {
      k.gt = LoopKernel{(const void*)ggt_gt_kernel<2>, gg, tma::kThreads, (unsigned)tma::kSmemBytesF32x2};
      k.gz = LoopKernel{(const void*)ggt_gz_kernel<2>, gg, tma::kThreads, (unsigned)tma::kSmemBytesF32x2};
    } else {
      k.gt = LoopKernel{(const void*)ggt_gt_kernel<1>, gg, tma::kThreads, (unsigned)tma::kSmemBytesF32};
      k.gz = LoopKernel{(const void*)ggt_gz_kernel<1>, gg, tma::kThreads, (unsigned)tma::kSmemBytesF32};
    }
  }
  return k;
}

struct Key {
  int dev;
  const void* ws;
  int n, nnz, nnz_g, g1, gg, gv, kind, rpt;
  bool operator==(const Key& o) const {
    return dev == o.dev && ws == o.ws && n == o.n && nnz == o.nnz && nnz_g == o.nnz_g && g1 == o.g1 &&
           gg == o.gg && gv == o.gv && kind == o.kind && rpt == o.rpt;
  }
};

std::mutex g_mu;
std::vector<std::pair<Key, cudaGraphExec_t>> g_cache;

cudaError_t add_loop_kernel(cudaGraph_t g, cudaGraphNode_t* dep, cudaGraphNode_t* out, const LoopKernel& k,
                            void** args) {
  return add_kernel(g, dep, dep ? 1 : 0, out, k.fn, k.grid, k.threads, args, k.smem);
}

int build_graph(GPtrs P, const BodyKernels& k, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  SLA_CUDA_TRY(cudaGraphCreate(&g, 0));
  int rc = SLA_ERR_CUDA;
  do {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNode_t n_init, n_while, n1, n2, n3, n4, n_final;
    void* a[] = {&P};
    int use_cond = 1;
    void* ac[] = {&P, &h, &use_cond};
    if (add_kernel(g, nullptr, 0, &n_init, (const void*)ggt_init_kernel, k.gv, kVT, a) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (add_loop_kernel(body, nullptr, &n1, k.k1, ac) != cudaSuccess) break;
    if (add_kernel(body, &n1, 1, &n2, (const void*)ggt_update_kernel, k.gv, kVT, a) != cudaSuccess) break;
    if (add_loop_kernel(body, &n2, &n3, k.gt, ac) != cudaSuccess) break;
    if (add_loop_kernel(body, &n3, &n4, k.gz, a) != cudaSuccess) break;
    if (add_kernel(g, &n_while, 1, &n_final, (const void*)ggt_final_kernel, k.gv, kVT, a) != cudaSuccess) break;
    if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) break;
    rc = SLA_OK;
  } while (0);
  cudaGraphDestroy(g);
  return rc;
}

int run_host_loop(GPtrs P, const KrylovDesc& desc, const BodyKernels& k, cudaStream_t s) {
  ggt_write_desc_kernel<<<1, 1, 0, s>>>(P.d, desc, P.st);
  ggt_init_kernel<<<k.gv, kVT, 0, s>>>(P);
  cudaGraphConditionalHandle h0 = 0;
  int uc = 0;
  void* ac[] = {&P, &h0, &uc};
  void* a[] = {&P};
  auto launch = [&](const LoopKernel& lk, void** args) {
    return cudaLaunchKernel(lk.fn, dim3(lk.grid), dim3(lk.threads), args, lk.smem, s);
  };
  const long long cap = (long long)desc.max_iter + 3LL * desc.max_restarts + 8;
  for (long long body = 0; body < cap; ++body) {
    SLA_CUDA_TRY(launch(k.k1, ac));
    ggt_update_kernel<<<k.gv, kVT, 0, s>>>(P);
    SLA_CUDA_TRY(launch(k.gt, ac));
    SLA_CUDA_TRY(launch(k.gz, a));
    if ((body + 1) % 16 == 0) {
      int phase = 0;
      SLA_CUDA_TRY(cudaMemcpyAsync(&phase, &P.st->phase, sizeof(int), cudaMemcpyDeviceToHost, s));
      SLA_CUDA_TRY(cudaStreamSynchronize(s));
      if (phase == kPhaseDone) break;
    }
  }
  ggt_final_kernel<<<k.gv, kVT, 0, s>>>(P);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaStreamSynchronize(s));
  return SLA_OK;
}

}  // namespace

KrylovDesc make_desc(const sla_csr* A, const double* val, const double* b, double* x,
                     const sla_opts* o, sla_info* info);
bool use_cg_coop(long long n, bool ggt);
int launch_ggt_coop(const KrylovDesc& desc, KrylovState* st, double* part, double* r, double* p, double* q,
                    double* t, const float* gv, const float* gtv, cudaStream_t s, bool* launched);

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_cg_ggt(const sla_csr* A, const double* val, const sla_csr* G,
                              const double* g_val, const sla_csr_t* GT, const double* b, double* x,
                              const sla_opts* opts, sla_info* info, void* ws, size_t ws_bytes,
                              void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr) return SLA_ERR_INVALID;
  const int n = A->n;
  if (G->n != n || G->nnz < 0) return SLA_ERR_INVALID;
  if (n > 0 && (G->rowptr == nullptr || GT->rowptr_t == nullptr)) return SLA_ERR_INVALID;
  if (G->nnz > 0 && (G->col == nullptr || g_val == nullptr || GT->col_t == nullptr ||
                     GT->perm_t == nullptr))
    return SLA_ERR_INVALID;
  const GgtLayout L = ggt_layout(n > 0 ? n : 0, G->nnz);
  int rc = validate_solve_args(A, val, b, x, opts, info, ws, ws_bytes, L.total);
  if (rc != SLA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) return write_info(info, sla_info{0, SLA_OK, 0.0, 0.0}, s);
  KrylovDesc d = make_desc(A, val, b, x, opts, info);
  d.precond = SLA_PRECOND_GGT;
  d.g_rowptr = G->rowptr;
  d.g_col = G->col;
  d.g_val = g_val;
  d.nnz_g = G->nnz;
  d.rowptr_t = GT->rowptr_t;
  d.col_t = GT->col_t;
  d.perm_t = GT->perm_t;
  char* base = (char*)ws;
  GPtrs P;
  P.d = (KrylovDesc*)(base + L.desc);
  P.st = (KrylovState*)(base + L.state);
  P.part = (double*)(base + L.part);
  P.r = (double*)(base + L.r);
  P.z = (double*)(base + L.z);
  P.p = (double*)(base + L.p);
  P.q = (double*)(base + L.q);
  P.t = (double*)(base + L.t);
  P.gv = (float*)(base + L.gv);
  P.gtv = (float*)(base + L.gtv);
  const int dev = current_device();
  if (!(opts->flags & (SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP)) && use_cg_coop(n, true)) {
    // one cooperative launch per solve (sla_cg_coop.cu) where the device runs it
    if (G->nnz > 0) {
      const int grid = persistent_grid(dev, ((long long)G->nnz + kVT - 1) / kVT, 8, kMaxBlocks);
      ggt_values_kernel<<<grid, kVT, 0, s>>>(g_val, GT->perm_t, G->nnz, P.gv, P.gtv);
      SLA_CUDA_TRY(cudaGetLastError());
    }
    bool launched = false;
    rc = launch_ggt_coop(d, P.st, P.part, P.r, P.p, P.q, P.t, P.gv, P.gtv, s, &launched);
    if (rc != SLA_OK || launched) return rc;
  }
  const BodyKernels bk = body_kernels(dev, n, G->nnz);
  if (opts->flags & SLA_FLAG_HOST_LOOP) return run_host_loop(P, d, bk, s);
  Key key{dev, ws, n, A->nnz, G->nnz, bk.k1.grid, bk.gt.grid, bk.gv, bk.kind, bk.rpt};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& e : g_cache)
      if (e.first == key) exec = e.second;
    if (exec == nullptr) {
      rc = build_graph(P, bk, &exec);
      if (rc != SLA_OK) return rc;
      if (g_cache.size() >= 64) {
        SLA_CUDA_TRY(cudaDeviceSynchronize());
        for (auto& e : g_cache) cudaGraphExecDestroy(e.second);
        g_cache.clear();
      }
      g_cache.push_back({key, exec});
    }
  }
  ggt_write_desc_kernel<<<1, 1, 0, s>>>(P.d, d, P.st);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaGraphLaunch(exec, s));
  return SLA_OK;
}
