// sla_multi.cu -- CG for one SPD matrix and k right-hand sides at once.
//
// A X = B for k <= 32 right-hand sides sharing A: k independent Jacobi-PCG
// iterations (Algorithm 1, Jacobi per Sec. 4.1), each with its own alpha,
// beta, convergence test, true-residual check and restarts, advanced in
// lock step by the same kernels.  This is the shape of the paper's inverse
// problem (Sec. 4.6) once it carries a batch of right-hand sides: every
// iteration then reads A once for all k columns instead of once per column,
// and one graph launch replaces k.
//
// Layout.  The caller's B and X are [k, n] (column j at b + j n).  Inside the
// workspace every vector is interleaved, element (i, j) at i W + j, with
// W = k rounded up to a power of two (the W - k padding columns hold zeros
// and are DONE from the start), so the W values of a row are one contiguous
// W x 8-byte segment: a gather x[col] of the SpMM and every stream of the
// vector updates moves whole sectors.  A thread owns one column j = tid % W
// for the whole solve (grid x 256 is a multiple of W), so per-column sums
// are a shuffle butterfly over the lanes of equal j plus one pass over the
// block's warps, in fixed order.
//
// One loop body is three kernels, as for one right-hand side:
//   K1  Q = A P and p_j . q_j            -> last block: alpha_j
//   K2  X += alpha P, R -= alpha Q, Z = D^{-1} R, r_j . z_j, r_j . r_j
//                                        -> last block: convergence, beta_j
//   K3  P = Z + beta P for running columns; true residual B - A X for
//       columns whose recursive residual converged (with restart)
//                                        -> last block: loop condition
// inside one conditional-WHILE CUDA graph node.
//
// Algorithmic bytes per iteration: 12 nnz + 4 (n+1) + 104 n W (the single
// right-hand-side schedule with every n-vector W columns wide).
#include <cmath>
#include <mutex>
#include <vector>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

namespace {

constexpr int kMT = 256;              // threads of every multi kernel
constexpr int kMW = kMT / kWarp;      // warps per block
constexpr int kMaxK = SLA_MULTI_MAX_RHS;

struct MultiDesc {
  int n, nnz, k, w;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* b;
  double* x;
  sla_info* info;
  double rtol, atol;
  int max_iter, max_restarts, precond, use_x0;
};

struct MCol {
  double bnorm, thresh, rho, rr, alpha, beta, tt, pq;
  int iters, restarts, status, phase, zero_rhs, pad;
};

struct MultiState {
  MCol c[kMaxK];
  unsigned cnt[8];
  int err, bad_diag, body, pad;
};

// Per-block partial sums: value m of column j of block b at
// part[(m kMaxK + j) kMaxBlocks + b].
constexpr int kMParts = 3;

struct MultiPtrs {
  MultiDesc* d;
  MultiState* st;
  double* part;
  double* bi;    // B interleaved
  double* xi;    // X interleaved
  double* r;
  double* z;
  double* p;
  double* q;
  double* dinv;  // n
};

// Column-wise block sums.  Every thread holds NV values of its column
// j = tid % w; on return part[...] holds the block's sums for columns < w.
template <int NV>
__device__ __forceinline__ void col_block_sums(double (&v)[NV], int w, double* part,
                                               double (&sh)[kMParts * kMW * kMaxK]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int m = 0; m < NV; ++m) {
    double s = v[m];
    for (int o = 16; o >= w; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[m] = s;
  }
  __syncthreads();
  if (lane < w) {
#pragma unroll
    for (int m = 0; m < NV; ++m) sh[(m * kMW + warp) * kMaxK + lane] = v[m];
  }
  __syncthreads();
  if (tid < NV * w) {
    const int m = tid / w, j = tid % w;
    double s = sh[(m * kMW + 0) * kMaxK + j];
    for (int q = 1; q < kMW; ++q) s += sh[(m * kMW + q) * kMaxK + j];
    part[(m * kMaxK + j) * kMaxBlocks + blockIdx.x] = s;
  }
}

// Last block: column sums over the grid's partials; result in
// out[m * kMaxK + j] (shared memory).  Each (value, column) pair gets G
// threads (G a power of two, G * NV * w <= kMT); thread g adds blocks g,
// g + G, ... with eight independent loads in flight, then the G partial sums
// are added in thread order -- a fixed order for a given grid.
template <int NV>
__device__ __forceinline__ void col_grid_sums(const double* part, int w, int nblocks, double* out,
                                              double* scratch /* kMT doubles */) {
  const int nvw = NV * w;
  int G = 1;
  while (G * 2 * nvw <= kMT) G *= 2;
  const int tid = threadIdx.x;
  const int mj = tid / G, g = tid % G;
  double s = 0.0;
  if (mj < nvw) {
    const int m = mj / w, j = mj % w;
    const double* src = part + (m * kMaxK + j) * kMaxBlocks;
    int b = g;
    // 16 loads in flight per round (one L2 round trip each), added in order
    for (; b + 15 * G < nblocks; b += 16 * G) {
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = __ldcg(src + b + u * G);
#pragma unroll
      for (int u = 0; u < 16; ++u) s += v[u];
    }
    for (; b < nblocks; b += G) s += __ldcg(src + b);
  }
  scratch[tid] = s;
  __syncthreads();
  if (tid < nvw) {
    double t = scratch[tid * G];
    for (int q = 1; q < G; ++q) t += scratch[tid * G + q];
    out[(tid / w) * kMaxK + (tid % w)] = t;
  }
  __syncthreads();
}

struct MSmem {
  double sh[kMParts * kMW * kMaxK];
  double scratch[kMT];
  double tot[kMParts * kMaxK];
  int phase[kMaxK];
  double alpha[kMaxK];
  bool last;
  int any;
};

// Row i of A times column j of an interleaved vector (width w).
__device__ __forceinline__ double row_dot_col(const int* __restrict__ rowptr, const int* __restrict__ col,
                                              const double* __restrict__ val, const double* v, int w,
                                              int i, int j) {
  const int a = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
  double s = 0.0;
  int k = a;
  for (; k + 4 <= e; k += 4) {
    const int c0 = __ldg(col + k), c1 = __ldg(col + k + 1), c2 = __ldg(col + k + 2), c3 = __ldg(col + k + 3);
    const double v0 = __ldg(val + k), v1 = __ldg(val + k + 1), v2 = __ldg(val + k + 2), v3 = __ldg(val + k + 3);
    const double x0 = v[(size_t)c0 * w + j], x1 = v[(size_t)c1 * w + j], x2 = v[(size_t)c2 * w + j],
                 x3 = v[(size_t)c3 * w + j];
    s = fma(v0, x0, s);
    s = fma(v1, x1, s);
    s = fma(v2, x2, s);
    s = fma(v3, x3, s);
  }
  for (; k < e; ++k) s = fma(__ldg(val + k), v[(size_t)__ldg(col + k) * w + j], s);
  return s;
}

// Loads the phases of the w columns into shared memory; returns whether any
// column is in `want` (the same answer in every block of the grid).
__device__ __forceinline__ bool load_phases(const MultiState* st, int w, MSmem& sm, int want0, int want1) {
  if (threadIdx.x == 0) sm.any = 0;
  __syncthreads();
  if (threadIdx.x < w) {
    const int ph = __ldcg(&st->c[threadIdx.x].phase);
    sm.phase[threadIdx.x] = ph;
    if (ph == want0 || ph == want1) atomicOr(&sm.any, 1);
  }
  __syncthreads();
  return sm.any != 0;
}

__global__ void multi_write_desc_kernel(MultiDesc* dst, MultiDesc src, MultiState* st) {
  *dst = src;
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
  st->bad_diag = 0;
  st->body = 0;
}

// [k, n] -> interleaved [n, w] (zero padding columns), 32 rows per tile.
__global__ void __launch_bounds__(kMT) multi_interleave_kernel(int n, int k, int w, const double* __restrict__ src,
                                                               double* __restrict__ dst, int zero) {
  __shared__ double tile[32][kMaxK + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = (n + 31) / 32;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = t * 32;
    for (int j = warp; j < w; j += kMW) {
      const int i = i0 + lane;
      tile[lane][j] = (!zero && j < k && i < n) ? src[(size_t)j * n + i] : 0.0;
    }
    __syncthreads();
    const int rows = min(32, n - i0);
    for (int e = threadIdx.x; e < rows * w; e += kMT) dst[(size_t)i0 * w + e] = tile[e / w][e % w];
    __syncthreads();
  }
}

// interleaved [n, w] -> [k, n].
__global__ void __launch_bounds__(kMT) multi_deinterleave_kernel(int n, int k, int w, const double* __restrict__ src,
                                                                 double* __restrict__ dst) {
  __shared__ double tile[32][kMaxK + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = (n + 31) / 32;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int i0 = t * 32;
    const int rows = min(32, n - i0);
    for (int e = threadIdx.x; e < rows * w; e += kMT) tile[e / w][e % w] = src[(size_t)i0 * w + e];
    __syncthreads();
    for (int j = warp; j < k; j += kMW) {
      const int i = i0 + lane;
      if (i < n) dst[(size_t)j * n + i] = tile[lane][j];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- init
// dinv, R = B - A X0, Z = dinv R, P = Z; per column ||b||^2, ||r||^2, r.z;
// a bad Jacobi diagonal stops every column.
__global__ void __launch_bounds__(kMT) multi_init_kernel(MultiPtrs P) {
  __shared__ MSmem sm;
  const MultiDesc d = *P.d;
  const int n = d.n, w = d.w;
  const int j = threadIdx.x % w;
  const size_t e0 = (size_t)blockIdx.x * kMT + threadIdx.x;
  const int i0 = (int)(e0 / w);
  const int rs = gridDim.x * kMT / w;
  double acc[3] = {0.0, 0.0, 0.0};
  int bad = 0;
  for (int i = i0; i < n; i += rs) {
    const int a = d.rowptr[i], e = d.rowptr[i + 1];
    double diag = 0.0;
    for (int kk = a; kk < e; ++kk)
      if (d.col[kk] == i) diag += d.val[kk];
    const size_t el = (size_t)i * w + j;
    const double bi = P.bi[el];
    const double ax = d.use_x0 ? row_dot_col(d.rowptr, d.col, d.val, P.xi, w, i, j) : 0.0;
    const double ri = bi - ax;
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      if (!(diag > 0.0)) bad = 1;
      di = 1.0 / diag;
    }
    const double zi = di * ri;
    if (j == 0) P.dinv[i] = di;
    P.r[el] = ri;
    P.z[el] = zi;
    P.p[el] = zi;
    acc[0] = fma(bi, bi, acc[0]);
    acc[1] = fma(ri, ri, acc[1]);
    acc[2] = fma(ri, zi, acc[2]);
  }
  if (bad) atomicOr(&P.st->bad_diag, 1);
  col_block_sums<3>(acc, w, P.part, sm.sh);
  if (!last_block_arrive(&P.st->cnt[0], &sm.last)) return;
  col_grid_sums<3>(P.part, w, gridDim.x, sm.tot, sm.scratch);
  if (threadIdx.x < w) {
    const int c = threadIdx.x;
    const double tbb = sm.tot[0 * kMaxK + c], trr = sm.tot[1 * kMaxK + c], trz = sm.tot[2 * kMaxK + c];
    MCol& s = P.st->c[c];
    s.bnorm = sqrt(tbb);
    s.thresh = fmax(d.rtol * s.bnorm, d.atol);
    s.rho = trz;
    s.rr = trr;
    s.tt = 0.0;
    s.alpha = s.beta = s.pq = 0.0;
    s.iters = 0;
    s.restarts = 0;
    s.zero_rhs = 0;
    s.status = SLA_NOT_CONVERGED;
    s.phase = kPhaseRun;
    if (__ldcg(&P.st->bad_diag)) {
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

// ---------------------------------------------------------------- K1
// Each thread sums kRU rows of its column at once; the first kEB entries of
// every row have their column indices, values and gathers all issued before
// the first FMA (rows longer than kEB finish one entry at a time).  The FMA
// loop exits at the row's end, so no padding FMA reaches the FP64 pipe.
// (Measured at 512^2 x 16: one row per thread at four blocks per SM beats
// two rows per thread, whose 98 registers allow only two blocks.)
constexpr int kRU = 1;
constexpr int kEB = 8;

__global__ void __launch_bounds__(kMT) multi_spmm_kernel(MultiPtrs P) {
  __shared__ MSmem sm;
  const MultiDesc d = *P.d;
  const int w = d.w;
  if (!load_phases(P.st, w, sm, kPhaseRun, kPhaseRun)) return;
  const int n = d.n;
  const int j = threadIdx.x % w;
  const bool run = sm.phase[j] == kPhaseRun;
  const int i0 = (int)(((size_t)blockIdx.x * kMT + threadIdx.x) / w);
  const int rs = gridDim.x * kMT / w;
  const int* __restrict__ rowptr = d.rowptr;
  const int* __restrict__ col = d.col;
  const double* __restrict__ val = d.val;
  const double* __restrict__ p = P.p;
  double* __restrict__ q = P.q;
  double pq[1] = {0.0};
  if (run) {
    for (int ib = i0; ib < n; ib += kRU * rs) {
      int a[kRU], len[kRU];
      double pi[kRU];
#pragma unroll
      for (int u = 0; u < kRU; ++u) {
        const int i = ib + u * rs;
        a[u] = 0;
        len[u] = 0;
        pi[u] = 0.0;
        if (i < n) {
          a[u] = __ldg(rowptr + i);
          len[u] = __ldg(rowptr + i + 1) - a[u];
          pi[u] = __ldg(p + (size_t)i * w + j);
        }
      }
      int cc[kRU][kEB];
      double vv[kRU][kEB], xx[kRU][kEB];
#pragma unroll
      for (int u = 0; u < kRU; ++u)
#pragma unroll
        for (int t = 0; t < kEB; ++t) {
          const bool ok = t < len[u];
          cc[u][t] = ok ? __ldg(col + a[u] + t) : 0;
          vv[u][t] = ok ? __ldg(val + a[u] + t) : 0.0;
        }
#pragma unroll
      for (int u = 0; u < kRU; ++u)
#pragma unroll
        for (int t = 0; t < kEB; ++t) xx[u][t] = t < len[u] ? __ldg(p + (size_t)cc[u][t] * w + j) : 0.0;
      double acc[kRU];
#pragma unroll
      for (int u = 0; u < kRU; ++u) {
        acc[u] = 0.0;
#pragma unroll
        for (int t = 0; t < kEB; ++t) {
          if (t >= len[u]) break;
          acc[u] = fma(vv[u][t], xx[u][t], acc[u]);
        }
        for (int kk = a[u] + kEB; kk < a[u] + len[u]; ++kk)
          acc[u] = fma(__ldg(val + kk), __ldg(p + (size_t)__ldg(col + kk) * w + j), acc[u]);
      }
#pragma unroll
      for (int u = 0; u < kRU; ++u) {
        const int i = ib + u * rs;
        if (i < n) {
          q[(size_t)i * w + j] = acc[u];
          pq[0] = fma(pi[u], acc[u], pq[0]);
        }
      }
    }
  }
  col_block_sums<1>(pq, w, P.part, sm.sh);
  if (!last_block_arrive(&P.st->cnt[1], &sm.last)) return;
  col_grid_sums<1>(P.part, w, gridDim.x, sm.tot, sm.scratch);
  if (threadIdx.x < w && sm.phase[threadIdx.x] == kPhaseRun) {
    MCol& s = P.st->c[threadIdx.x];
    const double tpq = sm.tot[threadIdx.x];
    s.pq = tpq;
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
}

// ---------------------------------------------------------------- K2
__global__ void __launch_bounds__(kMT) multi_update_kernel(MultiPtrs P) {
  __shared__ MSmem sm;
  const MultiDesc d = *P.d;
  const int w = d.w;
  if (!load_phases(P.st, w, sm, kPhaseRun, kPhaseRun)) return;
  const int n = d.n;
  const int j = threadIdx.x % w;
  // K1's last block may have stopped a column: re-read this thread's phase
  const bool run = __ldcg(&P.st->c[j].phase) == kPhaseRun;
  const double alpha = __ldcg(&P.st->c[j].alpha);
  const int i0 = (int)(((size_t)blockIdx.x * kMT + threadIdx.x) / w);
  const int rs = gridDim.x * kMT / w;
  double v[2] = {0.0, 0.0};  // rz, rr
  if (run) {
    constexpr int U = 4;
    for (int ib = i0; ib < n; ib += U * rs) {
      double pi[U], qi[U], di[U], xi[U], ri[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + u * rs;
        if (i < n) {
          const size_t el = (size_t)i * w + j;
          pi[u] = __ldg(P.p + el);
          qi[u] = __ldg(P.q + el);
          di[u] = __ldg(P.dinv + i);
          xi[u] = P.xi[el];
          ri[u] = P.r[el];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + u * rs;
        if (i < n) {
          const size_t el = (size_t)i * w + j;
          const double xn = fma(alpha, pi[u], xi[u]);
          const double rn = fma(-alpha, qi[u], ri[u]);
          const double zn = di[u] * rn;
          P.xi[el] = xn;
          P.r[el] = rn;
          P.z[el] = zn;
          v[0] = fma(rn, zn, v[0]);
          v[1] = fma(rn, rn, v[1]);
        }
      }
    }
  }
  col_block_sums<2>(v, w, P.part, sm.sh);
  if (!last_block_arrive(&P.st->cnt[2], &sm.last)) return;
  col_grid_sums<2>(P.part, w, gridDim.x, sm.tot, sm.scratch);
  if (threadIdx.x < w && __ldcg(&P.st->c[threadIdx.x].phase) == kPhaseRun) {
    MCol& s = P.st->c[threadIdx.x];
    const double trz = sm.tot[0 * kMaxK + threadIdx.x], trr = sm.tot[1 * kMaxK + threadIdx.x];
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
// The end of a loop body (one thread): count it, stop every live column once
// the hard cap on bodies is passed (each body advances some column's iters or
// consumes a restart, so the cap only fires if the state machine is broken),
// and set the loop's condition.
__device__ void close_body(MultiState& st, const MultiDesc& d, int w, cudaGraphConditionalHandle cond,
                           int use_cond) {
  st.body += 1;
  const int cap = d.max_iter + 2 * d.max_restarts + 8;
  int live = 0;
  for (int c = 0; c < w; ++c)
    if (st.c[c].phase != kPhaseDone) live = 1;
  if (live && st.body > cap) {
    for (int c = 0; c < w; ++c)
      if (st.c[c].phase != kPhaseDone) {
        st.c[c].status = SLA_NOT_CONVERGED;
        st.c[c].phase = kPhaseDone;
      }
    live = 0;
  }
  if (use_cond) cudaGraphSetConditional(cond, live ? 1u : 0u);
}

// P = Z + beta P for the running columns.  Only a column in its
// true-residual pass (phase Check) has sums to make: without one, no block
// writes partials and block 0 closes the body at the start (the p update
// changes no phase, so the condition is already known); with one, the last
// block adds the sums, takes the column's decision and closes the body.
__global__ void __launch_bounds__(kMT)
multi_pupdate_kernel(MultiPtrs P, cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ MSmem sm;
  const MultiDesc d = *P.d;
  const int w = d.w, n = d.n;
  load_phases(P.st, w, sm, kPhaseRun, kPhaseCheck);
  bool checking = false;
  for (int c = 0; c < w; ++c) checking |= sm.phase[c] == kPhaseCheck;
  if (!checking && blockIdx.x == 0 && threadIdx.x == 0) close_body(*P.st, d, w, cond, use_cond);
  const int j = threadIdx.x % w;
  const int ph = sm.phase[j];
  const int i0 = (int)(((size_t)blockIdx.x * kMT + threadIdx.x) / w);
  const int rs = gridDim.x * kMT / w;
  double v[2] = {0.0, 0.0};  // tt, rz of the check pass
  if (ph == kPhaseRun) {
    const double beta = __ldcg(&P.st->c[j].beta);
    constexpr int U = 4;
    for (int ib = i0; ib < n; ib += U * rs) {
      double zi[U], pi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + u * rs;
        if (i < n) {
          const size_t el = (size_t)i * w + j;
          zi[u] = __ldg(P.z + el);
          pi[u] = P.p[el];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = ib + u * rs;
        if (i < n) P.p[(size_t)i * w + j] = fma(beta, pi[u], zi[u]);
      }
    }
  } else if (ph == kPhaseCheck) {
    for (int i = i0; i < n; i += rs) {
      const size_t el = (size_t)i * w + j;
      const double ti = P.bi[el] - row_dot_col(d.rowptr, d.col, d.val, P.xi, w, i, j);
      const double zi = P.dinv[i] * ti;
      P.r[el] = ti;
      P.z[el] = zi;
      P.p[el] = zi;
      v[0] = fma(ti, ti, v[0]);
      v[1] = fma(ti, zi, v[1]);
    }
  }
  if (!checking) return;
  col_block_sums<2>(v, w, P.part, sm.sh);
  if (!last_block_arrive(&P.st->cnt[3], &sm.last)) return;
  col_grid_sums<2>(P.part, w, gridDim.x, sm.tot, sm.scratch);
  if (threadIdx.x < w && sm.phase[threadIdx.x] == kPhaseCheck) {
    MCol& s = P.st->c[threadIdx.x];
    const double ttt = sm.tot[0 * kMaxK + threadIdx.x], trz = sm.tot[1 * kMaxK + threadIdx.x];
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
  __syncthreads();
  if (threadIdx.x == 0) close_body(*P.st, d, w, cond, use_cond);
}

// ---------------------------------------------------------------- final
// True residual of every column, the info records, and X back to [k, n].
__global__ void __launch_bounds__(kMT) multi_final_kernel(MultiPtrs P) {
  __shared__ MSmem sm;
  const MultiDesc d = *P.d;
  const int w = d.w, n = d.n;
  const int j = threadIdx.x % w;
  const int i0 = (int)(((size_t)blockIdx.x * kMT + threadIdx.x) / w);
  const int rs = gridDim.x * kMT / w;
  const int bad = __ldcg(&P.st->bad_diag);
  const int zero = __ldcg(&P.st->c[j].zero_rhs);
  double v[1] = {0.0};
  for (int i = i0; i < n; i += rs) {
    const size_t el = (size_t)i * w + j;
    if (zero) {
      P.xi[el] = 0.0;
    } else if (!bad) {
      const double ti = P.bi[el] - row_dot_col(d.rowptr, d.col, d.val, P.xi, w, i, j);
      v[0] = fma(ti, ti, v[0]);
    }
  }
  col_block_sums<1>(v, w, P.part, sm.sh);
  if (!last_block_arrive(&P.st->cnt[4], &sm.last)) return;
  col_grid_sums<1>(P.part, w, gridDim.x, sm.tot, sm.scratch);
  if (threadIdx.x < d.k) {
    const MCol& s = P.st->c[threadIdx.x];
    sla_info inf;
    inf.iters = s.iters;
    inf.status = s.phase == kPhaseDone ? s.status : SLA_NOT_CONVERGED;
    if (s.zero_rhs) {
      inf.rel_res = 0.0;
      inf.true_rel_res = 0.0;
    } else if (bad) {
      inf.rel_res = NAN;
      inf.true_rel_res = NAN;
    } else {
      inf.rel_res = sqrt(s.rr) / s.bnorm;
      inf.true_rel_res = sqrt(sm.tot[threadIdx.x]) / s.bnorm;
    }
    d.info[threadIdx.x] = inf;
  }
}

// grad_val[e] = -sum_j lambda_j[row e] x_j[col e] over the k columns, with
// lambda and x interleaved (width w, zero padding).  The w lanes of a row
// add their products with a fixed butterfly.
__global__ void __launch_bounds__(kMT) multi_grad_kernel(int n, int w, const int* __restrict__ rowptr,
                                                         const int* __restrict__ col,
                                                         const double* __restrict__ lam,
                                                         const double* __restrict__ x,
                                                         double* __restrict__ grad_val) {
  const int lane = threadIdx.x & 31;
  const int j = lane % w;
  const int rows_per_warp = kWarp / w;
  const int warp_global = (blockIdx.x * kMT + threadIdx.x) >> 5;
  const int nwarps = gridDim.x * kMW;
  for (int ib = warp_global * rows_per_warp; ib < n; ib += nwarps * rows_per_warp) {
    const int i = ib + lane / w;
    const bool ok = i < n;
    const int a = ok ? __ldg(rowptr + i) : 0, e = ok ? __ldg(rowptr + i + 1) : 0;
    const double li = ok ? __ldg(lam + (size_t)i * w + j) : 0.0;
    int cnt = e - a;
    for (int o = 16; o >= 1; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
    for (int m = 0; m < cnt; ++m) {
      const bool has = a + m < e;
      double s = has ? li * __ldg(x + (size_t)__ldg(col + a + m) * w + j) : 0.0;
      for (int o = w >> 1; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (has && j == 0) grad_val[a + m] = -s;
    }
  }
}

// ---------------------------------------------------------------- host
struct MultiLayout {
  size_t desc, state, part, bi, xi, r, z, p, q, dinv, total;
};

MultiLayout multi_layout(int n, int w) {
  MultiLayout L{};
  size_t o = 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t vec = al256(sizeof(double) * nn * (size_t)w);
  L.desc = o;  o += al256(sizeof(MultiDesc));
  L.state = o; o += al256(sizeof(MultiState));
  L.part = o;  o += al256(sizeof(double) * kMParts * kMaxK * kMaxBlocks);
  L.bi = o;    o += vec;
  L.xi = o;    o += vec;
  L.r = o;     o += vec;
  L.z = o;     o += vec;
  L.p = o;     o += vec;
  L.q = o;     o += vec;
  L.dinv = o;  o += al256(sizeof(double) * nn);
  L.total = o;
  return L;
}

int width_of(int k) {
  int w = 1;
  while (w < k) w <<= 1;
  return w;
}

MultiPtrs carve(void* ws, int n, int w) {
  const MultiLayout L = multi_layout(n, w);
  char* base = (char*)ws;
  MultiPtrs P;
  P.d = (MultiDesc*)(base + L.desc);
  P.st = (MultiState*)(base + L.state);
  P.part = (double*)(base + L.part);
  P.bi = (double*)(base + L.bi);
  P.xi = (double*)(base + L.xi);
  P.r = (double*)(base + L.r);
  P.z = (double*)(base + L.z);
  P.p = (double*)(base + L.p);
  P.q = (double*)(base + L.q);
  P.dinv = (double*)(base + L.dinv);
  return P;
}

// Grids of the loop kernels: persistent, at most kBlocksPerSm blocks per SM
// (any grid works: 256 threads per block keep every thread on one column).
// Few blocks keep the last block's pass over the per-block partials short;
// the unrolled loops keep enough loads in flight.
constexpr int kBlocksPerSm = 4;
struct MultiGrids {
  int g1, g2, g3, gv;
};

MultiGrids multi_grids(int dev, int n, int w) {
  static int o1 = 0, o2 = 0, o3 = 0, ov = 0;
  if (o1 == 0) {
    o1 = occupancy((const void*)multi_spmm_kernel, kMT);
    o2 = occupancy((const void*)multi_update_kernel, kMT);
    o3 = occupancy((const void*)multi_pupdate_kernel, kMT);
    ov = occupancy((const void*)multi_init_kernel, kMT);
  }
  const long long blocks = ((long long)n * w + kMT - 1) / kMT;
  return MultiGrids{persistent_grid(dev, blocks, min(o1, kBlocksPerSm), kMaxBlocks),
                    persistent_grid(dev, blocks, min(o2, kBlocksPerSm), kMaxBlocks),
                    persistent_grid(dev, blocks, min(o3, kBlocksPerSm), kMaxBlocks),
                    persistent_grid(dev, blocks, min(ov, kBlocksPerSm), kMaxBlocks)};
}

struct MultiKey {
  int dev;
  const void* ws;
  int n, nnz, w, g1, g2, g3, gv;
  bool operator==(const MultiKey& o) const {
    return dev == o.dev && ws == o.ws && n == o.n && nnz == o.nnz && w == o.w && g1 == o.g1 && g2 == o.g2 &&
           g3 == o.g3 && gv == o.gv;
  }
};
struct MultiEntry {
  MultiKey key;
  cudaGraphExec_t exec;
};
std::mutex g_mmu;
std::vector<MultiEntry> g_mcache;
constexpr size_t kMCacheMax = 64;

int build_multi_graph(MultiPtrs P, MultiGrids g, cudaGraphExec_t* exec) {
  cudaGraph_t gr = nullptr;
  SLA_CUDA_TRY(cudaGraphCreate(&gr, 0));
  int rc = SLA_ERR_CUDA;
  do {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    cudaGraphNode_t n_init, n_while, n1, n2, n3, n_final;
    void* a[] = {&P};
    if (add_kernel(gr, nullptr, 0, &n_init, (const void*)multi_init_kernel, g.gv, kMT, a) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&n_while, gr, &n_init, nullptr, 1, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    int use_cond = 1;
    void* a3[] = {&P, &h, &use_cond};
    if (add_kernel(body, nullptr, 0, &n1, (const void*)multi_spmm_kernel, g.g1, kMT, a) != cudaSuccess) break;
    if (add_kernel(body, &n1, 1, &n2, (const void*)multi_update_kernel, g.g2, kMT, a) != cudaSuccess) break;
    if (add_kernel(body, &n2, 1, &n3, (const void*)multi_pupdate_kernel, g.g3, kMT, a3) != cudaSuccess) break;
    if (add_kernel(gr, &n_while, 1, &n_final, (const void*)multi_final_kernel, g.gv, kMT, a) != cudaSuccess) break;
    if (cudaGraphInstantiate(exec, gr, 0) != cudaSuccess) break;
    rc = SLA_OK;
  } while (0);
  cudaGraphDestroy(gr);
  return rc;
}

constexpr int kMPollEvery = 16;

// Runs the solve of d (already validated) in workspace ws: interleave,
// graph (or host loop), de-interleave of X into d.x.
int launch_multi(const MultiDesc& d, void* ws, cudaStream_t s, int flags) {
  const MultiPtrs P = carve(ws, d.n, d.w);
  const int dev = current_device();
  const MultiGrids g = multi_grids(dev, d.n, d.w);
  const int gt = persistent_grid(dev, (d.n + 31) / 32, 8, kMaxBlocks);
  multi_write_desc_kernel<<<1, 1, 0, s>>>(P.d, d, P.st);
  multi_interleave_kernel<<<gt, kMT, 0, s>>>(d.n, d.k, d.w, d.b, P.bi, 0);
  multi_interleave_kernel<<<gt, kMT, 0, s>>>(d.n, d.k, d.w, d.x, P.xi, d.use_x0 ? 0 : 1);
  SLA_CUDA_TRY(cudaGetLastError());
  if (flags & SLA_FLAG_HOST_LOOP) {
    multi_init_kernel<<<g.gv, kMT, 0, s>>>(P);
    const long long cap = (long long)d.max_iter + 2LL * d.max_restarts + 8;
    for (long long body = 0; body < cap; ++body) {
      multi_spmm_kernel<<<g.g1, kMT, 0, s>>>(P);
      multi_update_kernel<<<g.g2, kMT, 0, s>>>(P);
      multi_pupdate_kernel<<<g.g3, kMT, 0, s>>>(P, cudaGraphConditionalHandle(0), 0);
      if ((body + 1) % kMPollEvery == 0) {
        MultiState hs;
        SLA_CUDA_TRY(cudaMemcpyAsync(&hs, P.st, sizeof(MultiState), cudaMemcpyDeviceToHost, s));
        SLA_CUDA_TRY(cudaStreamSynchronize(s));
        bool live = false;
        for (int c = 0; c < d.w; ++c) live = live || hs.c[c].phase != kPhaseDone;
        if (!live) break;
      }
    }
    multi_final_kernel<<<g.gv, kMT, 0, s>>>(P);
  } else {
    MultiKey key{dev, ws, d.n, d.nnz, d.w, g.g1, g.g2, g.g3, g.gv};
    cudaGraphExec_t exec = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_mmu);
      for (auto& e : g_mcache)
        if (e.key == key) exec = e.exec;
      if (exec == nullptr) {
        const int rc = build_multi_graph(P, g, &exec);
        if (rc != SLA_OK) return rc;
        if (g_mcache.size() >= kMCacheMax) {
          SLA_CUDA_TRY(cudaDeviceSynchronize());
          for (auto& e : g_mcache) cudaGraphExecDestroy(e.exec);
          g_mcache.clear();
        }
        g_mcache.push_back(MultiEntry{key, exec});
      }
    }
    SLA_CUDA_TRY(cudaGraphLaunch(exec, s));
  }
  multi_deinterleave_kernel<<<gt, kMT, 0, s>>>(d.n, d.k, d.w, P.xi, d.x);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

int make_multi_desc(const sla_csr* A, const double* val, int k, const double* b, double* x,
                    const sla_opts* o, sla_info* info, void* ws, size_t ws_bytes, MultiDesc* d) {
  if (A == nullptr || o == nullptr || info == nullptr) return SLA_ERR_INVALID;
  if (k < 1 || k > kMaxK) return SLA_ERR_INVALID;
  if (A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if ((long long)A->n * width_of(k) > (long long)INT32_MAX) return SLA_ERR_INVALID;
  if (A->n > 0 && (A->rowptr == nullptr || b == nullptr || x == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if (A->n > 0 && (const void*)b == (const void*)x) return SLA_ERR_INVALID;
  if (!(o->rtol >= 0.0) || !(o->atol >= 0.0) || o->max_iter < 0 || o->max_restarts < 0 ||
      o->max_restarts > 16 || (o->use_x0 != 0 && o->use_x0 != 1) || (o->flags & ~1) != 0)
    return SLA_ERR_INVALID;
  if (o->precond != SLA_PRECOND_NONE && o->precond != SLA_PRECOND_JACOBI) return SLA_ERR_INVALID;
  const int w = width_of(k);
  if (ws == nullptr || ((uintptr_t)ws & 255u) != 0 || ws_bytes < multi_layout(A->n, w).total)
    return SLA_ERR_WORKSPACE;
  *d = MultiDesc{};
  d->n = A->n;
  d->nnz = A->nnz;
  d->k = k;
  d->w = w;
  d->rowptr = A->rowptr;
  d->col = A->col;
  d->val = val;
  d->b = b;
  d->x = x;
  d->info = info;
  d->rtol = o->rtol;
  d->atol = o->atol;
  d->max_iter = o->max_iter;
  d->max_restarts = o->max_restarts;
  d->precond = o->precond;
  d->use_x0 = o->use_x0;
  return SLA_OK;
}

__global__ void multi_zero_info_kernel(sla_info* info, int k) {
  const int i = threadIdx.x;
  if (i < k) info[i] = sla_info{0, SLA_OK, 0.0, 0.0};
}

}  // namespace

size_t multi_ws_bytes(int n, int k) {
  if (k < 1) k = 1;
  if (k > kMaxK) k = kMaxK;
  return multi_layout(n, width_of(k)).total;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_cg_multi(const sla_csr* A, const double* val, int32_t k, const double* b, double* x,
                                const sla_opts* opts, sla_info* info, void* ws, size_t ws_bytes,
                                void* stream) {
  MultiDesc d;
  const int rc = make_multi_desc(A, val, k, b, x, opts, info, ws, ws_bytes, &d);
  if (rc != SLA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (d.n == 0) {
    multi_zero_info_kernel<<<1, kMaxK, 0, s>>>(info, k);
    SLA_CUDA_TRY(cudaGetLastError());
    return SLA_OK;
  }
  return launch_multi(d, ws, s, opts->flags);
}

extern "C" int32_t sla_adjoint_backward_multi(const sla_csr* A, const double* val, int32_t k,
                                              const double* x, const double* grad_x, double* grad_b,
                                              double* grad_val, const sla_opts* opts, sla_info* info,
                                              void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr) return SLA_ERR_INVALID;
  if (A->n > 0 && (x == nullptr || grad_b == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && grad_val == nullptr) return SLA_ERR_INVALID;
  if (A->n > 0 && ((const void*)x == (const void*)grad_b || (const void*)grad_x == (const void*)grad_b))
    return SLA_ERR_INVALID;
  if (A->n > 0 && A->nnz > 0 && k > 0 &&
      (ranges_overlap(grad_val, 8 * (size_t)A->nnz, x, 8 * (size_t)A->n * k) ||
       ranges_overlap(grad_val, 8 * (size_t)A->nnz, grad_b, 8 * (size_t)A->n * k)))
    return SLA_ERR_INVALID;
  MultiDesc d;
  int rc = make_multi_desc(A, val, k, grad_x, grad_b, opts, info, ws, ws_bytes, &d);
  if (rc != SLA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (d.n == 0) {
    multi_zero_info_kernel<<<1, kMaxK, 0, s>>>(info, k);
    SLA_CUDA_TRY(cudaGetLastError());
    return SLA_OK;
  }
  // lambda_j: A^T lambda_j = grad_x_j with A^T = A (Eq. 3, SPD); the
  // interleaved lambda stays in the workspace's X slot
  rc = launch_multi(d, ws, s, opts->flags);
  if (rc != SLA_OK) return rc;
  if (d.nnz == 0) return SLA_OK;
  // x interleaved into the B slot (free once the solve has finished)
  const MultiPtrs P = carve(ws, d.n, d.w);
  const int dev = current_device();
  const int gt = persistent_grid(dev, (d.n + 31) / 32, 8, kMaxBlocks);
  multi_interleave_kernel<<<gt, kMT, 0, s>>>(d.n, d.k, d.w, x, P.bi, 0);
  const int rows_per_block = kMW * (kWarp / d.w);
  const int gg = persistent_grid(dev, (d.n + rows_per_block - 1) / rows_per_block, 8, 1 << 20);
  multi_grad_kernel<<<gg, kMT, 0, s>>>(d.n, d.w, d.rowptr, d.col, P.xi, P.bi, grad_val);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
