// sla_eig_adjoint.cu -- eigenvector gradients (Sec. 3.2, "Eigenvalue
// problems": one additional deflated linear solve per eigenpair).
//
// For a simple pair (lambda_j, v_j) of symmetric A, the adjoint of the
// constrained residual F(v, lambda; A) = (A v - lambda v, (v^T v - 1)/2)
// (Eq. 4's setting) reduces to the deflated system
//     (A - lambda_j I) mu_j = (I - v_j v_j^T) gV_j,   v_j^T mu_j = 0,
// and the eigenvector part of dL/dA is -mu_j[a] v_j[b] on the pattern.
// With the k computed pairs V, mu_j splits into the part along the other
// pairs, sum_{l != j} (v_l^T gV_j) / (lambda_l - lambda_j) v_l (closed
// form), and y_j in span(V)^perp, where A - lambda_j I restricted to
// span(V)^perp has the eigenvalues lambda_m - lambda_j > 0 (m > k): SPD, so
// y_j is found by CG on P (A - lambda_j I) P with P = I - V V^T and the
// preconditioner P D^{-1} P (D = diag A, or I).
//
// One cooperative launch solves all k systems together: a group of lanes
// per row (lane j = pair j; 1, 2, 4 or 8 lanes, the kernel is instantiated
// per k), three grid barriers per iteration (the SpMV gathers p
// at other blocks' rows; two reductions of k projections onto V plus two
// inner products per pair).  Every block adds the partial sums in the same
// order, so every block takes the same per-pair decisions.
#include <algorithm>
#include <cmath>

#include "sla.h"
#include "sla_coop.cuh"
#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {
namespace {

constexpr int kEvK = SLA_EIG_MAX_K;
constexpr int kEvThreads = 512;
constexpr int kEvLanes = 8;                      // stride of a slot in the partials
constexpr int kEvNv = kEvK + 2;                  // per lane: k projections, two sums
constexpr int kEvS0 = kEvK, kEvS1 = kEvK + 1;    // slots of the two sums
constexpr int kEvPart = kEvNv * kEvLanes;        // doubles of one block partial
constexpr int kEvChunks = 16;                    // most block ranges in the totals

// Lanes per row for k pairs (a power of two, so that a warp holds whole rows).
__host__ __device__ constexpr int ev_lanes(int k) { return k <= 1 ? 1 : k <= 2 ? 2 : k <= 4 ? 4 : 8; }
constexpr int kEvMaxGrid = 512;
// |lambda_l - lambda_j| <= this * max(|lambda_l|, |lambda_j|): a repeated
// eigenvalue, where the eigenvector gradient is not defined.
constexpr double kEvDegenerate = 1e-12;
// ||b_j|| <= this * ||gV_j||: b_j = (I - V V^T) gV_j is rounding noise (gV_j
// in span(V), or k = n), taken as zero.
constexpr double kEvNoise = 64.0 * 2.220446049250313e-16;

struct EvArgs {
  int n, k, max_iter, precond;
  double rtol, atol;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* lambda;
  const double* V;
  const double* gV;
  double* mu;
  sla_info* info;
  unsigned* count;
  int* err;
  double* dinv;
  double* r;
  double* p;
  double* q;
  double* part1;
  double* part2;
};

struct EvSmem {
  double red[kEvThreads / 32][kEvPart];
  double chunk[kEvChunks][kEvPart];
  double tot[kEvPart];  // totals of the last reduction: [slot * 8 + pair]
  double C[kEvK][kEvLanes];  // C[l][j] = v_l^T gV_j
  double rho[kEvLanes], alpha[kEvLanes], beta[kEvLanes], bnorm[kEvLanes], rr[kEvLanes], gnorm[kEvLanes];
  int active[kEvLanes], status[kEvLanes], iters[kEvLanes];
  int flag;
};

// The live values of a reduction for k pairs: slots 0..k-1 (projections)
// and the two sums, lanes 0..k-1; live index t -> partial index.
template <int K>
__device__ __forceinline__ int ev_live(int t) {
  const int v = t / K, l = t % K;
  return (v < K ? v : kEvK + (v - K)) * kEvLanes + l;
}

// Block sums of acc[slot] per pair lane: out[slot * 8 + pair] for the live
// values, fixed order (the rows of a warp by butterflies, then the warps in
// order).
template <int K>
__device__ __forceinline__ void ev_block_sums(double (&acc)[kEvNv], EvSmem& sm, double* out) {
  constexpr int L = ev_lanes(K);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < kEvNv; ++v) {
    if (v >= K && v < kEvK) continue;  // projection slots beyond k
    double a = acc[v];
#pragma unroll
    for (int o = L; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane < K) sm.red[warp][v * kEvLanes + lane] = a;
  }
  __syncthreads();
  if (threadIdx.x < (K + 2) * K) {
    const int idx = ev_live<K>(threadIdx.x);
    double s = 0.0;
    for (int w = 0; w < kEvThreads / 32; ++w) s += sm.red[w][idx];
    out[idx] = s;
  }
}

// sm.tot = the sum over the G block partials of the live values, in the
// same order in every block (contiguous ranges of blocks, then the ranges
// in order).
template <int K>
__device__ __forceinline__ void ev_totals(const double* part, int G, EvSmem& sm) {
  constexpr int NL = (K + 2) * K;
  constexpr int CH = kEvThreads / NL < kEvChunks ? kEvThreads / NL : kEvChunks;
  const int t = threadIdx.x;
  if (t < CH * NL) {
    const int idx = ev_live<K>(t % NL), c = t / NL;
    const int b0 = (int)((long long)G * c / CH), b1 = (int)((long long)G * (c + 1) / CH);
    double s = 0.0;
    for (int b = b0; b < b1; ++b) s += __ldcg(part + (size_t)b * kEvPart + idx);
    sm.chunk[c][idx] = s;
  }
  __syncthreads();
  if (t < NL) {
    const int idx = ev_live<K>(t);
    double s = 0.0;
    for (int c = 0; c < CH; ++c) s += sm.chunk[c][idx];
    sm.tot[idx] = s;
  }
  __syncthreads();
}

__global__ void ev_arm_kernel(unsigned* count, int* err) {
  *count = 0u;
  *err = 0;
}

template <int K>
__global__ void __launch_bounds__(kEvThreads, 1) eigvec_adjoint_kernel(EvArgs a) {
  __shared__ EvSmem sm;
  GridSync gs{a.count, 0u};
  constexpr int k = K, L = ev_lanes(K), kEvRows = kEvThreads / L;
  const int G = gridDim.x, n = a.n;
  const int j = threadIdx.x & (L - 1), slot = threadIdx.x / L;
  const bool on = j < k;
  const double lam_j = on ? __ldg(a.lambda + j) : 0.0;
  const size_t ks = (size_t)k;
  const int i0 = blockIdx.x * kEvRows + slot, di = G * kEvRows;
  double acc[kEvNv];
  auto zero = [&]() {
#pragma unroll
    for (int v = 0; v < kEvNv; ++v) acc[v] = 0.0;
  };
  auto sync = [&]() { return grid_sync(gs, (unsigned)G, a.err, &sm.flag); };

  // Jacobi diagonal, C = V^T gV and ||gV_j||^2 (slot S0); slot S1 of lane 0
  // counts the rows whose diagonal is not positive
  zero();
  for (int i = i0; i < n; i += di) {
    const double* vi = a.V + (size_t)i * ks;
    if (j == 0) {
      double dg = 0.0;
      for (int e = __ldg(a.rowptr + i); e < __ldg(a.rowptr + i + 1); ++e)
        if (__ldg(a.col + e) == i) dg += __ldg(a.val + e);
      if (a.precond == SLA_PRECOND_JACOBI) {
        if (!(dg > 0.0)) acc[kEvS1] += 1.0;
        a.dinv[i] = dg > 0.0 ? 1.0 / dg : 0.0;
      } else {
        a.dinv[i] = 1.0;
      }
    }
    if (on) {
      const double g = __ldg(a.gV + (size_t)i * ks + j);
#pragma unroll
      for (int l = 0; l < kEvK; ++l)
        if (l < k) acc[l] = fma(__ldg(vi + l), g, acc[l]);
      acc[kEvS0] = fma(g, g, acc[kEvS0]);
    }
  }
  ev_block_sums<K>(acc, sm, a.part1 + (size_t)blockIdx.x * kEvPart);
  if (!sync()) return;
  ev_totals<K>(a.part1, G, sm);
  if (threadIdx.x < K) {
    const int jj = threadIdx.x;
    for (int l = 0; l < kEvK; ++l) sm.C[l][jj] = sm.tot[l * kEvLanes + jj];
    const bool bad = sm.tot[kEvS1 * kEvLanes] > 0.0;
    sm.status[jj] = bad ? SLA_NOT_SPD : SLA_OK;
    sm.active[jj] = jj < k && !bad;
    sm.iters[jj] = 0;
    sm.rho[jj] = 0.0;
    sm.gnorm[jj] = sqrt(sm.tot[kEvS0 * kEvLanes + jj]);
  }
  __syncthreads();

  // b = P gV (P = I - V V^T), r = b, y = 0 (y lives in mu), u = D^{-1} r;
  // sums V^T u, r.u, r.r
  zero();
  for (int i = i0; i < n; i += di) {
    if (!on) continue;
    const size_t o = (size_t)i * ks + j;
    const double* vi = a.V + (size_t)i * ks;
    double b = __ldg(a.gV + o);
    for (int l = 0; l < k; ++l) b -= __ldg(vi + l) * sm.C[l][j];
    a.r[o] = b;
    a.mu[o] = 0.0;
    const double u = a.dinv[i] * b;
#pragma unroll
    for (int l = 0; l < kEvK; ++l)
      if (l < k) acc[l] = fma(__ldg(vi + l), u, acc[l]);
    acc[kEvS0] = fma(b, u, acc[kEvS0]);
    acc[kEvS1] = fma(b, b, acc[kEvS1]);
  }
  ev_block_sums<K>(acc, sm, a.part2 + (size_t)blockIdx.x * kEvPart);
  if (!sync()) return;

  for (int it = 0;; ++it) {
    // decisions from (V^T u, r.u, r.r); z = u - V (V^T u), p = z + beta p
    ev_totals<K>(a.part2, G, sm);
    if (threadIdx.x < K) {
      const int jj = threadIdx.x;
      const double ru = sm.tot[kEvS0 * kEvLanes + jj], rr = sm.tot[kEvS1 * kEvLanes + jj];
      sm.rr[jj] = rr;
      if (it == 0) {
        sm.bnorm[jj] = sqrt(rr);
        if (sm.bnorm[jj] <= kEvNoise * sm.gnorm[jj]) {
          sm.bnorm[jj] = 0.0;  // y_j = 0; rel_res and true_rel_res reported as 0
          sm.active[jj] = 0;
        }
      }
      double beta = 0.0;
      if (sm.active[jj]) {
        const double target = fmax(a.rtol * sm.bnorm[jj], a.atol);
        if (sqrt(rr) <= target) {
          sm.active[jj] = 0;
        } else if (sm.iters[jj] >= a.max_iter) {
          sm.active[jj] = 0;
          sm.status[jj] = SLA_NOT_CONVERGED;
        } else if (!(ru > 0.0) || !isfinite(ru)) {
          sm.active[jj] = 0;
          sm.status[jj] = SLA_BREAKDOWN;
        } else {
          beta = it == 0 ? 0.0 : ru / sm.rho[jj];
          sm.rho[jj] = ru;
        }
      }
      sm.beta[jj] = beta;
    }
    __syncthreads();
    int any = 0;
    for (int l = 0; l < k; ++l) any |= sm.active[l];
    if (!any) break;
    for (int i = i0; i < n; i += di) {
      if (!on || !sm.active[j]) continue;
      const size_t o = (size_t)i * ks + j;
      const double* vi = a.V + (size_t)i * ks;
      double z = a.dinv[i] * a.r[o];
      for (int l = 0; l < k; ++l) z -= __ldg(vi + l) * sm.tot[l * kEvLanes + j];
      a.p[o] = it == 0 ? z : fma(sm.beta[j], a.p[o], z);
    }
    if (!sync()) return;

    // q = (A - lambda_j I) p; sums V^T q, p.q
    zero();
    for (int i = i0; i < n; i += di) {
      if (!on || !sm.active[j]) continue;
      double s = 0.0;
      for (int e = __ldg(a.rowptr + i); e < __ldg(a.rowptr + i + 1); ++e)
        s = fma(__ldg(a.val + e), a.p[(size_t)__ldg(a.col + e) * ks + j], s);
      const size_t o = (size_t)i * ks + j;
      const double* vi = a.V + (size_t)i * ks;
      const double pi = a.p[o];
      const double qv = fma(-lam_j, pi, s);
      a.q[o] = qv;
#pragma unroll
      for (int l = 0; l < kEvK; ++l)
        if (l < k) acc[l] = fma(__ldg(vi + l), qv, acc[l]);
      acc[kEvS0] = fma(pi, qv, acc[kEvS0]);
    }
    ev_block_sums<K>(acc, sm, a.part1 + (size_t)blockIdx.x * kEvPart);
    if (!sync()) return;

    // alpha = rho / p.q; y += alpha p, r -= alpha P q; sums for the next step
    ev_totals<K>(a.part1, G, sm);
    if (threadIdx.x < K) {
      const int jj = threadIdx.x;
      double al = 0.0;
      if (sm.active[jj]) {
        const double pq = sm.tot[kEvS0 * kEvLanes + jj];
        if (!(pq > 0.0) || !isfinite(pq)) {
          sm.active[jj] = 0;
          sm.status[jj] = SLA_NOT_SPD;
        } else {
          al = sm.rho[jj] / pq;
          sm.iters[jj] += 1;
        }
      }
      sm.alpha[jj] = al;
    }
    __syncthreads();
    zero();
    for (int i = i0; i < n; i += di) {
      if (!on) continue;
      const size_t o = (size_t)i * ks + j;
      const double* vi = a.V + (size_t)i * ks;
      double rv = a.r[o];
      if (sm.active[j]) {
        double pq = a.q[o];
        for (int l = 0; l < k; ++l) pq -= __ldg(vi + l) * sm.tot[l * kEvLanes + j];
        a.mu[o] = fma(sm.alpha[j], a.p[o], a.mu[o]);
        rv = fma(-sm.alpha[j], pq, rv);
        a.r[o] = rv;
      }
      const double u = a.dinv[i] * rv;
#pragma unroll
      for (int l = 0; l < kEvK; ++l)
        if (l < k) acc[l] = fma(__ldg(vi + l), u, acc[l]);
      acc[kEvS0] = fma(rv, u, acc[kEvS0]);
      acc[kEvS1] = fma(rv, rv, acc[kEvS1]);
    }
    ev_block_sums<K>(acc, sm, a.part2 + (size_t)blockIdx.x * kEvPart);
    if (!sync()) return;
  }

  // true residual of the deflated system: t = P gV - (A - lambda_j I) y
  zero();
  for (int i = i0; i < n; i += di) {
    if (!on) continue;
    const size_t o = (size_t)i * ks + j;
    const double* vi = a.V + (size_t)i * ks;
    double b = __ldg(a.gV + o);
    for (int l = 0; l < k; ++l) b -= __ldg(vi + l) * sm.C[l][j];
    double s = 0.0;
    for (int e = __ldg(a.rowptr + i); e < __ldg(a.rowptr + i + 1); ++e)
      s = fma(__ldg(a.val + e), a.mu[(size_t)__ldg(a.col + e) * ks + j], s);
    const double t = b - fma(-lam_j, a.mu[o], s);
    acc[kEvS1] = fma(t, t, acc[kEvS1]);
  }
  ev_block_sums<K>(acc, sm, a.part1 + (size_t)blockIdx.x * kEvPart);
  if (!sync()) return;
  ev_totals<K>(a.part1, G, sm);

  // mu = y + sum_{l != j} C[l][j] / (lambda_l - lambda_j) v_l
  double coef[kEvK];
  bool degenerate = false;
#pragma unroll
  for (int l = 0; l < kEvK; ++l) {
    coef[l] = 0.0;
    if (on && l < k && l != j) {
      const double ll = __ldg(a.lambda + l), dl = ll - lam_j;
      if (fabs(dl) <= kEvDegenerate * fmax(fabs(ll), fabs(lam_j)))
        degenerate = true;
      else
        coef[l] = sm.C[l][j] / dl;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < k) {
    sla_info inf;
    inf.iters = sm.iters[j];
    inf.status = (degenerate && sm.status[j] == SLA_OK) ? SLA_BREAKDOWN : sm.status[j];
    const double bn = sm.bnorm[j];
    inf.rel_res = bn > 0.0 ? sqrt(sm.rr[j]) / bn : 0.0;
    inf.true_rel_res = bn > 0.0 ? sqrt(sm.tot[kEvS1 * kEvLanes + j]) / bn : 0.0;
    a.info[j] = inf;
  }
  for (int i = i0; i < n; i += di) {
    if (!on) continue;
    const size_t o = (size_t)i * ks + j;
    const double* vi = a.V + (size_t)i * ks;
    double m = a.mu[o];
#pragma unroll
    for (int l = 0; l < kEvK; ++l)
      if (l < k) m = fma(coef[l], __ldg(vi + l), m);
    a.mu[o] = m;
  }
}

// A barrier that ran out: every pair's record says so.
__global__ void ev_finish_kernel(const int* err, sla_info* info, int k) {
  if (*err == 0 || threadIdx.x >= (unsigned)k) return;
  sla_info inf;
  inf.iters = 0;
  inf.status = SLA_ERR_TIMEOUT;
  inf.rel_res = NAN;
  inf.true_rel_res = NAN;
  info[threadIdx.x] = inf;
}

// Eigenvector part of the gradient on the pattern: out[e] (+)= -sum_j
// mu[row_e][j] V[col_e][j], one row per thread.
__global__ void eigvec_grad_kernel(int n, int k, const int* __restrict__ rowptr, const int* __restrict__ col,
                                   const double* __restrict__ mu, const double* __restrict__ V,
                                   double* __restrict__ out, int accumulate) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double w[kEvK];
#pragma unroll
    for (int j = 0; j < kEvK; ++j) w[j] = j < k ? __ldg(mu + (size_t)i * k + j) : 0.0;
    for (int e = __ldg(rowptr + i); e < __ldg(rowptr + i + 1); ++e) {
      const double* vc = V + (size_t)__ldg(col + e) * k;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < kEvK; ++j)
        if (j < k) s = fma(w[j], __ldg(vc + j), s);
      out[e] = accumulate ? out[e] - s : -s;
    }
  }
}

int g_occ_ev[kEvK + 1][64] = {};

const void* ev_kernel(int k) {
  switch (k) {
    case 1: return (const void*)eigvec_adjoint_kernel<1>;
    case 2: return (const void*)eigvec_adjoint_kernel<2>;
    case 3: return (const void*)eigvec_adjoint_kernel<3>;
    case 4: return (const void*)eigvec_adjoint_kernel<4>;
    case 5: return (const void*)eigvec_adjoint_kernel<5>;
    case 6: return (const void*)eigvec_adjoint_kernel<6>;
    case 7: return (const void*)eigvec_adjoint_kernel<7>;
    default: return (const void*)eigvec_adjoint_kernel<8>;
  }
}

struct EvLayout {
  size_t ctl, dinv, r, p, q, part1, part2, total;
};

EvLayout ev_layout(int n, int k) {
  const size_t nn = (size_t)(n > 0 ? n : 1), nk = nn * (size_t)k;
  EvLayout L;
  size_t o = 0;
  L.ctl = o;   o += 256;
  L.dinv = o;  o += al256(sizeof(double) * nn);
  L.r = o;     o += al256(sizeof(double) * nk);
  L.p = o;     o += al256(sizeof(double) * nk);
  L.q = o;     o += al256(sizeof(double) * nk);
  L.part1 = o; o += al256(sizeof(double) * kEvMaxGrid * kEvPart);
  L.part2 = o; o += al256(sizeof(double) * kEvMaxGrid * kEvPart);
  L.total = o;
  return L;
}

}  // namespace

size_t eigvec_ws_bytes(int n, int k) { return ev_layout(n, k).total; }

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_eig_vector_adjoint(const sla_csr* A, const double* val, int32_t k, const double* lambda,
                                          const double* V, const double* gV, double* mu, const sla_opts* opts,
                                          sla_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || opts == nullptr || info == nullptr) return SLA_ERR_INVALID;
  const int n = A->n;
  if (n < 1 || k < 1 || k > kEvK || k > n) return SLA_ERR_INVALID;
  if (A->nnz < 0 || A->rowptr == nullptr || (A->nnz > 0 && (A->col == nullptr || val == nullptr)))
    return SLA_ERR_INVALID;
  if (lambda == nullptr || V == nullptr || gV == nullptr || mu == nullptr) return SLA_ERR_INVALID;
  if (!(opts->rtol >= 0.0) || !(opts->atol >= 0.0) || opts->max_iter < 0 || opts->use_x0 != 0 ||
      (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) || opts->flags != 0)
    return SLA_ERR_INVALID;
  const EvLayout Lw = ev_layout(n, k);
  if (ws == nullptr || ((uintptr_t)ws & 255u) != 0 || ws_bytes < Lw.total) return SLA_ERR_WORKSPACE;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_ERR_CUDA;
  const void* fn = ev_kernel(k);
  const int occ = coop_occupancy_of(dev, g_occ_ev[k], fn);
  if (occ < 1) return SLA_ERR_CUDA;  // no cooperative launch on this device
  const int rows = kEvThreads / ev_lanes(k);
  const long long want = ((long long)n + rows - 1) / rows;
  const int grid = (int)std::max(1LL, std::min<long long>({want, (long long)num_sms(dev) * std::min(occ, 2),
                                                           (long long)kEvMaxGrid}));
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)ws;
  EvArgs a;
  a.n = n;
  a.k = k;
  a.max_iter = opts->max_iter;
  a.precond = opts->precond;
  a.rtol = opts->rtol;
  a.atol = opts->atol;
  a.rowptr = A->rowptr;
  a.col = A->col;
  a.val = val;
  a.lambda = lambda;
  a.V = V;
  a.gV = gV;
  a.mu = mu;
  a.info = info;
  a.count = (unsigned*)(w + Lw.ctl);
  a.err = (int*)(w + Lw.ctl + 64);
  a.dinv = (double*)(w + Lw.dinv);
  a.r = (double*)(w + Lw.r);
  a.p = (double*)(w + Lw.p);
  a.q = (double*)(w + Lw.q);
  a.part1 = (double*)(w + Lw.part1);
  a.part2 = (double*)(w + Lw.part2);
  ev_arm_kernel<<<1, 1, 0, s>>>(a.count, a.err);
  void* args[] = {&a};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kEvThreads), args,
                                           0, s));
  ev_finish_kernel<<<1, 32, 0, s>>>(a.err, info, k);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_eig_vector_grad_values(const sla_csr* A, int32_t k, const double* mu, const double* V,
                                              double* grad_val, int32_t accumulate, void* stream) {
  if (A == nullptr || k < 1 || k > kEvK || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (accumulate != 0 && accumulate != 1) return SLA_ERR_INVALID;
  if (A->n == 0 || A->nnz == 0) return SLA_OK;
  if (A->rowptr == nullptr || A->col == nullptr || mu == nullptr || V == nullptr || grad_val == nullptr)
    return SLA_ERR_INVALID;
  const long long b = ((long long)A->n + 255) / 256;
  const int grid = (int)std::max(1LL, std::min(b, 4096LL));
  eigvec_grad_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(A->n, k, A->rowptr, A->col, mu, V, grad_val,
                                                             accumulate);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
