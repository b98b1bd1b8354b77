// sla_cg.cu -- preconditioned conjugate gradient for SPD A.
//
// Algorithm 1 (App. C) with a single process: every all_reduce becomes an
// in-kernel grid reduction, and the halo exchange disappears.  The Jacobi
// preconditioner z = D^{-1} r is the one the paper's CG backend uses
// (Sec. 4.1).  One iteration is three kernels:
//
//   K1  q = A p, partial p.q            -> last block: alpha = rho / p.q
//   K2  x += alpha p, r -= alpha q, z = D^{-1} r, partial r.z, r.r
//                                       -> last block: convergence, beta
//   K3  p = z + beta p   (or, once the recursive residual has converged,
//       the true-residual check b - A x with an optional restart)
//                                       -> last block: loop condition
//
// The loop runs inside one CUDA graph as a conditional WHILE node whose
// condition K3's last block sets, so a whole solve is one graph launch and
// no host synchronisation.  Per-call arguments live in a descriptor in the
// workspace, so the instantiated graph depends only on the workspace address
// and the sizes and is cached.
//
// With the Jacobi preconditioner the kernels run CG on the symmetrically
// scaled system A^ = D^{-1/2} A D^{-1/2}, x^ = D^{1/2} x, b^ = D^{-1/2} b (its
// values written once per solve): the iterates are those of Jacobi PCG (r^ =
// D^{-1/2} r, p^ = D^{1/2} p, r^.r^ = r.z), but z = D^{-1} r is never formed,
// and the stopping test keeps ||r||^2 = sum_i d_i r^_i^2.
//
// Algorithmic bytes per iteration (int32 CSR, FP64): 12 nnz + 4 (n+1)
// + 96 n  (K1: p, q; K2: x rw, r rw, p, q, diag; K3: r, p rw); without the
// scaling (no preconditioner, or the allocation-free entry) + 104 n (K2 reads
// dinv and writes z, K3 reads z).
#include <cmath>
#include <mutex>
#include <vector>

#include "sla_internal.cuh"
#include "sla_tma.cuh"
#include "sla_workspace.h"

namespace sla {

constexpr int kVecThreads = 256;

struct CgPtrs {
  KrylovDesc* d;
  KrylovState* st;
  double* part;
  double* r;
  double* z;
  double* p;
  double* q;
  double* dinv;  // D^{-1}; with sym_scale the diagonal d itself
  double* ahat;  // values of D^{-1/2} A D^{-1/2} (sym_scale)
};

// sym_scale: z holds s = d^{-1/2}.
__device__ __forceinline__ const double* cg_vals(const CgPtrs& P, const KrylovDesc& d) {
  return d.sym_scale ? P.ahat : d.val;
}

// Writes the per-call descriptor and zeroes the ticket counters, so that a
// workspace whose memory held anything before still starts every solve with
// every grid reduction armed (the loop condition depends on them).
__global__ void cg_write_desc_kernel(KrylovDesc* dst, KrylovDesc src, KrylovState* st) {
  *dst = src;
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
}

// Shared scratch of the vector kernels: up to 4 reduced values per block.
constexpr int kRedSlots = 4;
struct VecSmem {
  double red[kRedSlots * kVecThreads + kRedSlots];
  bool last;
};

// Unroll factor of the streaming loops: U independent elements per thread
// per pass keep 5 U loads in flight.
constexpr int kUnroll = 4;

// ---------------------------------------------------------------- init
// dinv = 1 / diag(A) (or 1 without preconditioner), r = b - A x0,
// z = dinv r, p = z; sums ||b||^2, ||r||^2, r.z and a bad-diagonal flag.
__global__ void __launch_bounds__(kVecThreads) cg_init_kernel(CgPtrs P) {
  __shared__ VecSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // bb, rr, rz, bad
  const int stride = gridDim.x * kVecThreads;
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += stride) {
    const int a = d.rowptr[i], e = d.rowptr[i + 1];
    double diag = 0.0, ax = 0.0;
    for (int k = a; k < e; ++k) {
      const int c = d.col[k];
      const double v = d.val[k];
      if (c == i) diag += v;
      if (d.use_x0) ax = fma(v, d.x[c], ax);
    }
    const double bi = d.b[i];
    const double ri = bi - ax;
    acc[0] = fma(bi, bi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
    if (d.sym_scale) {
      // r^ = s r with s = d^{-1/2}; p^ = r^; r.z = r^.r^
      if (!(diag > 0.0)) acc[3] = 1.0;
      const double si = rsqrt(diag);
      const double rh = si * ri;
      P.dinv[i] = diag;
      P.z[i] = si;
      P.r[i] = rh;
      P.p[i] = rh;
      acc[2] = fma(rh, rh, acc[2]);
      continue;
    }
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      if (!(diag > 0.0)) acc[3] = 1.0;
      di = 1.0 / diag;
    }
    const double zi = di * ri;
    P.dinv[i] = di;
    P.r[i] = ri;
    P.z[i] = zi;
    P.p[i] = zi;
    acc[2] = fma(ri, zi, acc[2]);
  }
  if (!d.use_x0) {
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += stride) d.x[i] = 0.0;
  }
  block_sums<kVecThreads, 4>(acc, sm.red);
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) P.part[j * kMaxBlocks + blockIdx.x] = acc[j];
  if (!last_block_arrive(&P.st->cnt[0], &sm.last)) return;
  double t[4];
  reduce_partials<kVecThreads, 4>(P.part, kMaxBlocks, gridDim.x, t, sm.red);
  if (threadIdx.x == 0) {
    const double tbb = t[0], trr = t[1], trz = t[2], tbad = t[3];
    KrylovState& s = *P.st;
    s.bnorm = sqrt(tbb);
    s.thresh = fmax(d.rtol * s.bnorm, d.atol);
    s.rho = trz;
    s.rr = trr;
    s.tt = 0.0;
    s.alpha = s.beta = 0.0;
    s.iters = 0;
    s.restarts = 0;
    s.body = 0;
    s.zero_rhs = 0;
    s.bad_diag = 0;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseRun;
    if (tbad > 0.0) {
      s.bad_diag = 1;
      s.status = SLA_NOT_SPD;
      s.phase = kPhaseDone;
    } else if (s.bnorm == 0.0) {
      s.zero_rhs = 1;
      s.status = SLA_OK;
      s.phase = kPhaseDone;
    } else if (!isfinite(trz) || !isfinite(trr)) {
      s.status = SLA_BREAKDOWN;
      s.phase = kPhaseDone;
    } else if (sqrt(trr) <= s.thresh) {
      s.phase = kPhaseCheck;
    } else if (d.max_iter <= 0) {
      s.phase = kPhaseDone;
    }
  }
}

// sym_scale: A^ = D^{-1/2} A D^{-1/2} (a_ij s_i s_j) and x^ = D^{1/2} x =
// x d s.  After cg_init_kernel (which needs every s and the caller's x).
__global__ void __launch_bounds__(kVecThreads) cg_scale_kernel(CgPtrs P) {
  const KrylovDesc d = *P.d;
  if (!d.sym_scale || __ldcg(&P.st->bad_diag)) return;
  const double* __restrict__ sv = P.z;
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < d.n; i += gridDim.x * kVecThreads) {
    const double si = sv[i];
    for (int k = __ldg(d.rowptr + i); k < __ldg(d.rowptr + i + 1); ++k)
      P.ahat[k] = __ldg(d.val + k) * si * sv[__ldg(d.col + k)];
    d.x[i] = d.x[i] * (P.dinv[i] * si);
  }
}

// sym_scale: x = D^{-1/2} x^ at exit, before the final residual.
__global__ void __launch_bounds__(kVecThreads) cg_unscale_kernel(CgPtrs P) {
  const KrylovDesc d = *P.d;
  if (!d.sym_scale || __ldcg(&P.st->bad_diag) || __ldcg(&P.st->zero_rhs)) return;
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < d.n; i += gridDim.x * kVecThreads)
    d.x[i] *= P.z[i];
}

// ---------------------------------------------------------------- K1
// Last block of K1: alpha = rho / p.q, or the solve's end on a breakdown.
__device__ __forceinline__ void k1_finish(const CgPtrs& P, double tpq) {
  KrylovState& s = *P.st;
  s.pq = tpq;
  if (__ldcg(&s.err) != 0) {
    s.status = SLA_ERR_TIMEOUT;
    s.phase = kPhaseDone;
  } else if (!isfinite(tpq)) {
    s.status = SLA_BREAKDOWN;
    s.phase = kPhaseDone;
  } else if (!(tpq > 0.0)) {
    s.status = SLA_NOT_SPD;
    s.phase = kPhaseDone;
  } else {
    s.alpha = s.rho / tpq;
  }
}

// K1 body for a block of NT threads: run(epi) performs q = A p through one
// of the SpMV schemes, calling epi(row, (A p)_row, p_row).
template <int NT, int M, class Run>
__device__ __forceinline__ void k1_body(const CgPtrs& P, double (&red)[M], bool* s_last, Run&& run) {
  double* __restrict__ q = P.q;
  double pq = 0.0;
  run([&](int row, double s, double prow) {
    q[row] = s;
    pq = fma(prow, s, pq);
  });
  double v[1] = {pq};
  block_sums<NT, 1>(v, red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[1], s_last)) return;
  reduce_partials<NT, 1>(P.part, kMaxBlocks, gridDim.x, v, red);
  if (threadIdx.x == 0) k1_finish(P, v[0]);
}

// K1 on register-staged tiles.
__global__ void __launch_bounds__(kTileThreads) cg_spmv_pq_kernel(CgPtrs P) {
  __shared__ TileSmem sm;
  __shared__ bool s_last;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  const double* __restrict__ p = P.p;
  k1_body<kTileThreads>(P, sm.val, &s_last, [&](auto&& epi) {
    const int ntiles = (d.n + kTileRows - 1) / kTileRows;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
      spmv_tile(t, d.n, d.rowptr, d.col, cg_vals(P, d), p, sm,
                [&](int row, double s) { epi(row, s, __ldg(p + row)); });
  });
}

// K1 on the TMA-pipelined tiles (see sla_tma.cuh), four blocks per SM.  The
// matrix comes from the device descriptor through a shared-memory record
// (tma::MatShared): with the descriptor's fields in registers, the p.q
// epilogue and the state update needed 68 registers (three blocks per SM;
// forced to 56 they spilled).
__global__ void __launch_bounds__(tma::kThreads, 4) cg_spmv_pq_tma_kernel(CgPtrs P) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::Smem& sm = *reinterpret_cast<tma::Smem*>(dsm);
  __shared__ tma::MatRecord mat;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  if (threadIdx.x == 0) {
    const KrylovDesc* d = P.d;
    mat.n = d->n;
    mat.nnz = d->nnz;
    mat.rowptr = d->rowptr;
    mat.col = d->col;
    mat.val = d->sym_scale ? (const void*)P.ahat : (const void*)d->val;
  }
  __syncthreads();
  k1_body<tma::kThreads>(P, sm.red, &sm.last, [&](auto&& epi) {
    tma::spmv_pipeline_m<1, double>(tma::MatShared<double>{&mat}, P.p, P.p, sm, &P.st->err, epi);
  });
}

// K1 with one thread per row (csr_rows): the scheme for n <= kRowsKernelMaxN.
__global__ void __launch_bounds__(kRowThreads) cg_spmv_pq_rows_kernel(CgPtrs P) {
  __shared__ double red[kRowThreads + 2];
  __shared__ bool s_last;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  k1_body<kRowThreads>(P, red, &s_last,
                       [&](auto&& epi) { csr_rows(d.n, d.rowptr, d.col, cg_vals(P, d), P.p, P.p, epi); });
}

// ---------------------------------------------------------------- K2
__global__ void __launch_bounds__(kVecThreads) cg_update_kernel(CgPtrs P) {
  __shared__ VecSmem sm;
  if (__ldcg(&P.st->phase) != kPhaseRun) return;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const double alpha = __ldcg(&P.st->alpha);
  double* __restrict__ x = d.x;
  double* __restrict__ r = P.r;
  double* __restrict__ z = P.z;
  const double* __restrict__ p = P.p;
  const double* __restrict__ q = P.q;
  const double* __restrict__ dinv = P.dinv;
  double rz0 = 0.0, rz1 = 0.0, rr0 = 0.0, rr1 = 0.0;
  const int stride = gridDim.x * kVecThreads;
  if (d.sym_scale) {
    // x^ += alpha p^, r^ -= alpha q^; r.z = r^.r^, ||r||^2 = sum d r^^2
    const double* __restrict__ dg = P.dinv;
    for (int i0 = blockIdx.x * kVecThreads + threadIdx.x; i0 < n; i0 += kUnroll * stride) {
      double pi[kUnroll], qi[kUnroll], di[kUnroll], xi[kUnroll], ri[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * stride;
        if (i < n) {
          pi[u] = __ldg(p + i);
          qi[u] = __ldg(q + i);
          di[u] = __ldg(dg + i);
          xi[u] = x[i];
          ri[u] = r[i];
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * stride;
        if (i < n) {
          const double rn = fma(-alpha, qi[u], ri[u]);
          x[i] = fma(alpha, pi[u], xi[u]);
          r[i] = rn;
          const double rn2 = rn * rn;
          if (u & 1) {
            rz1 += rn2;
            rr1 = fma(di[u], rn2, rr1);
          } else {
            rz0 += rn2;
            rr0 = fma(di[u], rn2, rr0);
          }
        }
      }
    }
  } else
  for (int i0 = blockIdx.x * kVecThreads + threadIdx.x; i0 < n; i0 += kUnroll * stride) {
    double pi[kUnroll], qi[kUnroll], di[kUnroll], xi[kUnroll], ri[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        pi[u] = __ldg(p + i);
        qi[u] = __ldg(q + i);
        di[u] = __ldg(dinv + i);
        xi[u] = x[i];
        ri[u] = r[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * stride;
      if (i < n) {
        const double xn = fma(alpha, pi[u], xi[u]);
        const double rn = fma(-alpha, qi[u], ri[u]);
        const double zn = di[u] * rn;
        x[i] = xn;
        r[i] = rn;
        z[i] = zn;
        if (u & 1) {
          rz1 = fma(rn, zn, rz1);
          rr1 = fma(rn, rn, rr1);
        } else {
          rz0 = fma(rn, zn, rz0);
          rr0 = fma(rn, rn, rr0);
        }
      }
    }
  }
  double v[2] = {rz0 + rz1, rr0 + rr1};
  block_sums<kVecThreads, 2>(v, sm.red);
  if (threadIdx.x == 0) {
    P.part[0 * kMaxBlocks + blockIdx.x] = v[0];
    P.part[1 * kMaxBlocks + blockIdx.x] = v[1];
  }
  if (!last_block_arrive(&P.st->cnt[2], &sm.last)) return;
  reduce_partials<kVecThreads, 2>(P.part, kMaxBlocks, gridDim.x, v, sm.red);
  if (threadIdx.x == 0) {
    const double trz = v[0], trr = v[1];
    KrylovState& s = *P.st;
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
}

// ---------------------------------------------------------------- K3
__global__ void __launch_bounds__(kVecThreads)
cg_pupdate_kernel(CgPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ VecSmem sm;
  const int phase = __ldcg(&P.st->phase);
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int stride = gridDim.x * kVecThreads;
  double v[2] = {0.0, 0.0};  // tt, rz of the check pass
  if (phase == kPhaseRun) {
    const double beta = __ldcg(&P.st->beta);
    const double* __restrict__ z = d.sym_scale ? P.r : P.z;  // p^ = r^ + beta p^ when scaled
    double* __restrict__ p = P.p;
    for (int i0 = blockIdx.x * kVecThreads + threadIdx.x; i0 < n; i0 += kUnroll * stride) {
      double zi[kUnroll], pi[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * stride;
        if (i < n) {
          zi[u] = __ldg(z + i);
          pi[u] = p[i];
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * stride;
        if (i < n) p[i] = fma(beta, pi[u], zi[u]);
      }
    }
  } else if (phase == kPhaseCheck && d.sym_scale) {
    // t^ = b^ - A^ x^ = s (b - A x); ||t||^2 = sum d t^^2, t.z = t^.t^
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += stride) {
      const double si = P.z[i];
      const double th = d.b[i] * si - row_dot(d.rowptr, d.col, P.ahat, d.x, i);
      P.r[i] = th;
      P.p[i] = th;
      const double th2 = th * th;
      v[0] = fma(P.dinv[i], th2, v[0]);
      v[1] += th2;
    }
    block_sums<kVecThreads, 2>(v, sm.red);
    if (threadIdx.x == 0) {
      P.part[0 * kMaxBlocks + blockIdx.x] = v[0];
      P.part[1 * kMaxBlocks + blockIdx.x] = v[1];
    }
  } else if (phase == kPhaseCheck) {
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += stride) {
      const double ti = d.b[i] - row_dot(d.rowptr, d.col, d.val, d.x, i);
      const double zi = P.dinv[i] * ti;
      P.r[i] = ti;
      P.z[i] = zi;
      P.p[i] = zi;
      v[0] = fma(ti, ti, v[0]);
      v[1] = fma(ti, zi, v[1]);
    }
    block_sums<kVecThreads, 2>(v, sm.red);
    if (threadIdx.x == 0) {
      P.part[0 * kMaxBlocks + blockIdx.x] = v[0];
      P.part[1 * kMaxBlocks + blockIdx.x] = v[1];
    }
  }
  if (!last_block_arrive(&P.st->cnt[3], &sm.last)) return;
  if (phase == kPhaseCheck) reduce_partials<kVecThreads, 2>(P.part, kMaxBlocks, gridDim.x, v, sm.red);
  if (threadIdx.x == 0) {
    KrylovState& s = *P.st;
    if (phase == kPhaseCheck) {
      const double ttt = v[0], trz = v[1];
      const double tn = sqrt(ttt);
      s.tt = ttt;
      if (tn <= 2.0 * s.thresh) {
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
    // hard cap on loop bodies: each one either advances iters or consumes a
    // restart, so this only fires if the state machine is broken
    s.body += 1;
    const int cap = d.max_iter + 2 * d.max_restarts + 8;
    if (s.phase != kPhaseDone && s.body > cap) {
      s.status = SLA_NOT_CONVERGED;
      s.phase = kPhaseDone;
    }
    if (use_cond) cudaGraphSetConditional(cond, s.phase != kPhaseDone ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- final
__global__ void __launch_bounds__(kVecThreads) cg_final_kernel(CgPtrs P) {
  __shared__ VecSmem sm;
  const KrylovDesc d = *P.d;
  const int n = d.n;
  const int zero_rhs = __ldcg(&P.st->zero_rhs);
  const int bad = __ldcg(&P.st->bad_diag);
  const int stride = gridDim.x * kVecThreads;
  double v[1] = {0.0};
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += stride) {
    if (zero_rhs || bad) {
      if (zero_rhs) d.x[i] = 0.0;
    } else {
      const double ti = d.b[i] - row_dot(d.rowptr, d.col, d.val, d.x, i);
      v[0] = fma(ti, ti, v[0]);
    }
  }
  block_sums<kVecThreads, 1>(v, sm.red);
  if (threadIdx.x == 0) P.part[blockIdx.x] = v[0];
  if (!last_block_arrive(&P.st->cnt[4], &sm.last)) return;
  reduce_partials<kVecThreads, 1>(P.part, kMaxBlocks, gridDim.x, v, sm.red);
  if (threadIdx.x == 0) {
    const double ttt = v[0];
    const KrylovState& s = *P.st;
    sla_info inf;
    inf.iters = s.iters;
    inf.status = s.phase == kPhaseDone ? s.status : SLA_NOT_CONVERGED;
    if (s.zero_rhs) {
      inf.rel_res = 0.0;
      inf.true_rel_res = 0.0;
    } else if (s.bad_diag) {
      inf.rel_res = NAN;
      inf.true_rel_res = NAN;
    } else {
      inf.rel_res = sqrt(s.rr) / s.bnorm;
      inf.true_rel_res = sqrt(ttt) / s.bnorm;
    }
    *d.info = inf;
  }
}

__global__ void write_info_kernel(sla_info* info, sla_info v) { *info = v; }

int occupancy(const void* fn, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b <= 0)
    b = 1;
  return b;
}

cudaError_t add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                       cudaGraphNode_t* out, const void* fn, int grid, int block, void** args,
                       unsigned smem) {
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = smem;
  kp.kernelParams = args;
  kp.extra = nullptr;
  return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}


int write_info(sla_info* info, sla_info v, cudaStream_t s) {
  write_info_kernel<<<1, 1, 0, s>>>(info, v);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// ---------------------------------------------------------------- graph
namespace {

struct CgGraphKey {
  int dev;
  const void* ws;
  int n, nnz, g1, gv, tma;
  bool operator==(const CgGraphKey& o) const {
    return dev == o.dev && ws == o.ws && n == o.n && nnz == o.nnz && g1 == o.g1 && gv == o.gv &&
           tma == o.tma;
  }
};

struct CgGraphEntry {
  CgGraphKey key;
  cudaGraphExec_t exec;
};

std::mutex g_mu;
std::vector<CgGraphEntry> g_cache;
constexpr size_t kCacheMax = 64;

// The K1 variant in use: kernel, block size and dynamic shared memory.
struct K1Launch {
  const void* fn;
  int threads;
  unsigned smem;
};

K1Launch k1_launch(int kind) {
  if (kind == kSpmvTma) return K1Launch{(const void*)cg_spmv_pq_tma_kernel, tma::kThreads, (unsigned)tma::kSmemBytes};
  if (kind == kSpmvRows) return K1Launch{(const void*)cg_spmv_pq_rows_kernel, kRowThreads, 0u};
  return K1Launch{(const void*)cg_spmv_pq_kernel, kTileThreads, 0u};
}

int build_graph(CgPtrs P, K1Launch k1, int g1, int gv, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  SLA_CUDA_TRY(cudaGraphCreate(&g, 0));
  int rc = SLA_ERR_CUDA;
  do {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNode_t n_init, n_scale, n_while, n1, n2, n3, n_unscale, n_final;
    void* a_init[] = {&P};
    if (add_kernel(g, nullptr, 0, &n_init, (const void*)cg_init_kernel, gv, kVecThreads, a_init) != cudaSuccess) break;
    if (add_kernel(g, &n_init, 1, &n_scale, (const void*)cg_scale_kernel, gv, kVecThreads, a_init) != cudaSuccess)
      break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&n_while, g, &n_scale, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    int use_cond = 1;
    void* a1[] = {&P};
    void* a3[] = {&P, &h, &use_cond};
    if (add_kernel(body, nullptr, 0, &n1, k1.fn, g1, k1.threads, a1, k1.smem) != cudaSuccess) break;
    if (add_kernel(body, &n1, 1, &n2, (const void*)cg_update_kernel, gv, kVecThreads, a1) != cudaSuccess) break;
    if (add_kernel(body, &n2, 1, &n3, (const void*)cg_pupdate_kernel, gv, kVecThreads, a3) != cudaSuccess) break;
    if (add_kernel(g, &n_while, 1, &n_unscale, (const void*)cg_unscale_kernel, gv, kVecThreads, a_init) !=
        cudaSuccess)
      break;
    if (add_kernel(g, &n_unscale, 1, &n_final, (const void*)cg_final_kernel, gv, kVecThreads, a_init) != cudaSuccess)
      break;
    if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) break;
    rc = SLA_OK;
  } while (0);
  cudaGraphDestroy(g);
  return rc;
}

}  // namespace

int cg_grids(int dev, int n, int kind, int* g1, int* gv) {
  static int occ1 = 0, occ1t = 0, occ1r = 0, occv = 0;
  if (occ1 == 0) occ1 = occupancy((const void*)cg_spmv_pq_kernel, kTileThreads);
  if (occ1t == 0) {
    cudaFuncSetAttribute(cg_spmv_pq_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma::kSmemBytes);
    occ1t = occupancy((const void*)cg_spmv_pq_tma_kernel, tma::kThreads, tma::kSmemBytes);
  }
  if (occ1r == 0) occ1r = occupancy((const void*)cg_spmv_pq_rows_kernel, kRowThreads);
  if (occv == 0) occv = occupancy((const void*)cg_update_kernel, kVecThreads);
  if (kind == kSpmvRows)
    *g1 = persistent_grid(dev, ((long long)n + kRowThreads - 1) / kRowThreads, occ1r < 8 ? occ1r : 8, kMaxBlocks);
  else
    *g1 = persistent_grid(dev, (n + kTileRows - 1) / kTileRows, kind == kSpmvTma ? occ1t : occ1, kMaxBlocks);
  *gv = persistent_grid(dev, ((long long)n + kVecThreads - 1) / kVecThreads, occv, kMaxBlocks);
  return SLA_OK;
}

// Host-driven loop: the same kernels as the graph, launched one by one.  The
// device state is polled every kPollEvery loop bodies; kernels of a finished
// solve return immediately, so overshooting the poll is harmless.
constexpr int kPollEvery = 16;

int run_host_loop(const CgPtrs& P, const KrylovDesc& desc, K1Launch k1, int g1, int gv,
                  cudaStream_t s) {
  cg_write_desc_kernel<<<1, 1, 0, s>>>(P.d, desc, P.st);
  cg_init_kernel<<<gv, kVecThreads, 0, s>>>(P);
  cg_scale_kernel<<<gv, kVecThreads, 0, s>>>(P);
  const long long cap = (long long)desc.max_iter + 2LL * desc.max_restarts + 8;
  for (long long body = 0; body < cap; ++body) {
    void* a1[] = {const_cast<CgPtrs*>(&P)};
    SLA_CUDA_TRY(cudaLaunchKernel(k1.fn, dim3(g1), dim3(k1.threads), a1, k1.smem, s));
    cg_update_kernel<<<gv, kVecThreads, 0, s>>>(P);
    cg_pupdate_kernel<<<gv, kVecThreads, 0, s>>>(P, cudaGraphConditionalHandle(0), 0);
    if ((body + 1) % kPollEvery == 0) {
      int phase = 0;
      SLA_CUDA_TRY(cudaMemcpyAsync(&phase, &P.st->phase, sizeof(int), cudaMemcpyDeviceToHost, s));
      SLA_CUDA_TRY(cudaStreamSynchronize(s));
      if (phase == kPhaseDone) break;
    }
  }
  cg_unscale_kernel<<<gv, kVecThreads, 0, s>>>(P);
  cg_final_kernel<<<gv, kVecThreads, 0, s>>>(P);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaStreamSynchronize(s));
  return SLA_OK;
}

bool use_cg_coop(long long n, bool ggt);
int launch_cg_coop(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched);
int launch_cg_pipe(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched);

// allow_graph = false: where the cooperative launch is not taken, drive the
// loop from the host (no graph objects), as the allocation-free entry needs.
int launch_cg(const KrylovDesc& desc, void* ws, cudaStream_t s, int flags, bool allow_graph = true) {
  const int n = desc.n;
  if (flags & SLA_FLAG_CG_PIPELINED) {
    // pipelined PCG (sla_cg_pipe.cu): cooperative only, at every size
    bool launched = false;
    const int rc = launch_cg_pipe(desc, ws, s, &launched);
    if (rc != SLA_OK) return rc;
    return launched ? SLA_OK : SLA_ERR_CUDA;
  }
  if (!(flags & (SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP)) && use_cg_coop(n, false)) {
    // one cooperative launch per solve (sla_cg_coop.cu) where the device runs it
    bool launched = false;
    const int rc = launch_cg_coop(desc, ws, s, &launched);
    if (rc != SLA_OK || launched) return rc;
  }
  if (!allow_graph) {
    // the host-driven loop polls and synchronises the stream, which a
    // stream capture does not allow: refuse before enqueueing anything
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SLA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SLA_ERR_INVALID;
    flags |= SLA_FLAG_HOST_LOOP;
  }
  const CgLayout L = cg_layout(n);
  char* base = (char*)ws;
  CgPtrs P;
  P.d = (KrylovDesc*)(base + L.desc);
  P.st = (KrylovState*)(base + L.state);
  P.part = (double*)(base + L.part);
  P.r = (double*)(base + L.r);
  P.z = (double*)(base + L.z);
  P.p = (double*)(base + L.p);
  P.q = (double*)(base + L.q);
  P.dinv = (double*)(base + L.dinv);
  P.ahat = (double*)(base + al256(L.total));
  const int dev = current_device();
  const int kind = spmv_kind(n);
  const K1Launch k1 = k1_launch(kind);
  int g1, gv;
  cg_grids(dev, n, kind, &g1, &gv);
  if (flags & SLA_FLAG_HOST_LOOP) return run_host_loop(P, desc, k1, g1, gv, s);
  CgGraphKey key{dev, ws, n, desc.nnz, g1, gv, kind};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& e : g_cache)
      if (e.key == key) exec = e.exec;
    if (exec == nullptr) {
      const int rc = build_graph(P, k1, g1, gv, &exec);
      if (rc != SLA_OK) return rc;
      if (g_cache.size() >= kCacheMax) {
        SLA_CUDA_TRY(cudaDeviceSynchronize());
        for (auto& e : g_cache) cudaGraphExecDestroy(e.exec);
        g_cache.clear();
      }
      g_cache.push_back(CgGraphEntry{key, exec});
    }
  }
  cg_write_desc_kernel<<<1, 1, 0, s>>>(P.d, desc, P.st);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaGraphLaunch(exec, s));
  return SLA_OK;
}

int validate_solve_args(const sla_csr* A, const double* val, const double* b, const double* x,
                        const sla_opts* o, const sla_info* info, const void* ws, size_t ws_bytes,
                        size_t need, int allowed_flags) {
  if (A == nullptr || o == nullptr || info == nullptr) return SLA_ERR_INVALID;
  if (A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n > 0 && (A->rowptr == nullptr || b == nullptr || x == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if (A->n > 0 && (const void*)b == (const void*)x) return SLA_ERR_INVALID;
  if (!(o->rtol >= 0.0) || !(o->atol >= 0.0) || o->max_iter < 0 || o->max_restarts < 0 ||
      o->max_restarts > 16 || (o->use_x0 != 0 && o->use_x0 != 1) ||
      (o->flags & ~allowed_flags) != 0)
    return SLA_ERR_INVALID;
  if ((o->flags & SLA_FLAG_CG_PIPELINED) && (o->flags & (SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP)))
    return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) != 0 || ws_bytes < need) return SLA_ERR_WORKSPACE;
  return SLA_OK;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_cg(const sla_csr* A, const double* val, const double* b, double* x,
                          const sla_opts* opts, sla_info* info, void* ws, size_t ws_bytes,
                          void* stream) {
  if (A == nullptr || opts == nullptr) return SLA_ERR_INVALID;
  const int nn = A->n > 0 ? A->n : 0;
  const size_t need = (opts->flags & SLA_FLAG_CG_PIPELINED) ? cg_pipe_layout(nn).total
                                                            : cg_ws_bytes(nn, A->nnz > 0 ? A->nnz : 0);
  int rc = validate_solve_args(A, val, b, x, opts, info, ws, ws_bytes, need,
                               SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP | SLA_FLAG_CG_PIPELINED);
  if (rc != SLA_OK) return rc;
  if (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n == 0) {
    sla_info v{0, SLA_OK, 0.0, 0.0};
    write_info_kernel<<<1, 1, 0, s>>>(info, v);
    SLA_CUDA_TRY(cudaGetLastError());
    return SLA_OK;
  }
  KrylovDesc d = {};
  d.n = A->n;
  d.nnz = A->nnz;
  d.rowptr = A->rowptr;
  d.col = A->col;
  d.val = val;
  d.b = b;
  d.x = x;
  d.info = info;
  d.rtol = opts->rtol;
  d.atol = opts->atol;
  d.max_iter = opts->max_iter;
  d.max_restarts = opts->max_restarts;
  d.precond = opts->precond;
  d.use_x0 = opts->use_x0;
  d.sym_scale = opts->precond == SLA_PRECOND_JACOBI ? 1 : 0;
  return launch_cg(d, ws, s, opts->flags);
}

// ---------------------------------------------------------------------------
// Allocation-free CG.  The paper has no counterpart: this exists for callers
// that cannot allocate device memory when they solve -- code running inside a
// framework's allocator or memory hook (a cudaMalloc there would re-enter the
// allocator), serving or real-time hosts that reserve all device memory once
// at start-up and forbid allocations afterwards, and plug-ins that receive a
// stream but no allocator.  Such callers still pass inputs and outputs; the
// scratch space (descriptor, state, partial sums, five n-vectors) lives in
// the fixed-size array below, which every device that loads this library
// holds until the process exits.
// ---------------------------------------------------------------------------
static constexpr size_t kNoallocScratchBytes = sla::cg_layout(SLA_NOALLOC_MAX_N).total;
static __device__ __align__(256) unsigned char sla_noalloc_scratch[kNoallocScratchBytes];

namespace {
// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, never a device address, so
// it is resolved with cudaGetSymbolAddress -- on every call (it allocates
// nothing), so that an address never outlives the context it came from.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, sla_noalloc_scratch) != cudaSuccess || p == nullptr)
    return SLA_ERR_CUDA;
  *out = p;
  return SLA_OK;
}
}  // namespace

extern "C" int32_t sla_cg_noalloc(const sla_csr* A, const double* val, const double* b, double* x,
                                  const sla_opts* opts, sla_info* info, void* stream) {
  if (A == nullptr || opts == nullptr) return SLA_ERR_INVALID;
  if (A->n > SLA_NOALLOC_MAX_N) return SLA_ERR_WORKSPACE;
  void* ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc != SLA_OK) return rc;
  const size_t need = cg_layout(A->n > 0 ? A->n : 0).total;
  rc = validate_solve_args(A, val, b, x, opts, info, ws, kNoallocScratchBytes, need,
                           SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP);
  if (rc != SLA_OK) return rc;
  if (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n == 0) {
    sla_info v{0, SLA_OK, 0.0, 0.0};
    write_info_kernel<<<1, 1, 0, s>>>(info, v);
    SLA_CUDA_TRY(cudaGetLastError());
    return SLA_OK;
  }
  KrylovDesc d = {};
  d.n = A->n;
  d.nnz = A->nnz;
  d.rowptr = A->rowptr;
  d.col = A->col;
  d.val = val;
  d.b = b;
  d.x = x;
  d.info = info;
  d.rtol = opts->rtol;
  d.atol = opts->atol;
  d.max_iter = opts->max_iter;
  d.max_restarts = opts->max_restarts;
  d.precond = opts->precond;
  d.use_x0 = opts->use_x0;
  d.sym_scale = 0;  // the fixed scratch has no room for the scaled values
  // one cooperative launch, else plain launches from a host loop: no graph
  // objects are created either way
  return launch_cg(d, ws, s, opts->flags, /*allow_graph=*/false);
}
