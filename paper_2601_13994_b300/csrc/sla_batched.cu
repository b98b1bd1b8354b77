// sla_batched.cu -- many Jacobi-PCG solves in one persistent launch.
//
// The paper's SparseTensor holds a batch on one shared pattern and
// SparseTensorList a batch of distinct patterns (Sec. 3.1); both dispatch
// solves per element.  Here a whole batch is one kernel launch: persistent
// CTAs take systems from an atomic counter (largest first when an order is
// given) and each CTA runs the complete PCG recurrence of its system --
// Algorithm 1 with P = 1 and the Jacobi preconditioner, the same stopping
// rule, true-residual restart and statuses as the single-system solver --
// with block-level reductions only.  A system's convergence ends only its
// own CTA's loop, which is the per-system convergence mask.  No block ever
// waits for another, so the launch always terminates.
//
// On this part a batched small system is FP64-bound, not memory-bound: with
// the Krylov vectors in shared memory (when 5 n doubles fit; otherwise in a
// per-CTA global slot) an iteration reads only the values and the pattern.
#include <cmath>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {
namespace {

struct BatchDesc {
  int batch, shared_pattern;
  int n, nnz;                 // shared pattern sizes
  const int* rowptr;          // shared: [n+1]; list: per-system rowptrs concatenated
  const int* col;             // shared: [nnz]; list: local columns concatenated
  const int* n_off;           // list: [batch+1] row offsets (device)
  const int* nnz_off;         // list: [batch+1] entry offsets (device)
  const double* val;          // shared: [batch, nnz]; list: concatenated
  const double* b;
  double* x;
  sla_info* info;             // [batch]
  const int* order;           // optional processing order
  unsigned* next;             // scheduling counter (zeroed before launch)
  double* gvec;               // per-system vector storage: 5 n doubles at 5 * (row offset)
  int n_max, smem_rows;       // rows whose vectors fit the dynamic shared memory
  double rtol, atol;
  int max_iter, max_restarts, precond, use_x0;
  int skip_nnz;               // list: systems with at least this many entries are
                              // solved by block teams (0: none)
};

// The threads that solve one system: the whole CTA (SPC = 1), or one of SPC
// equal slices of it (systems per CTA), which synchronise on a named barrier
// of their own -- slices finish their systems at different times, so no
// CTA-wide barrier may be used once SPC > 1.
template <int GT, int SPC>
struct Grp {
  int id;  // slice 0 .. SPC-1
  int t;   // thread index in the slice
  __device__ __forceinline__ void sync() const {
    if constexpr (SPC == 1) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(GT) : "memory");
    }
  }
};

// block_sums over the GT threads of a group (same parking scheme and the
// same fixed order, so SPC = 1 gives block_sums' bits).
template <int GT, int SPC, int NV, int M>
__device__ __forceinline__ void group_sums(const Grp<GT, SPC>& g, double (&v)[NV], double (&sh)[M]) {
  static_assert(GT % kWarp == 0 && GT <= 1024 && NV <= GT / kWarp, "group size");
  static_assert(M >= NV * GT + NV, "reduction scratch too small");
  const int lane = g.t & 31, w = g.t >> 5;
  g.sync();
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j * GT + g.t] = v[j];
  g.sync();
  if (w < NV) {
    const double* col = sh + w * GT + lane;
    double s = col[0];
#pragma unroll
    for (int k = 1; k < GT / kWarp; ++k) s += col[kWarp * k];
    s = warp_sum(s);
    if (lane == 0) sh[NV * GT + w] = s;
  }
  g.sync();
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = sh[NV * GT + j];
}

template <int GT>
struct BRed {
  double red[2 * GT + 2];
};

// Sum of row i of (rp, cl, v) times w, entries in order.  w may live in
// shared memory or be written earlier in this same launch (x, p), so it is
// read with plain generic loads, never through the read-only path; the
// pattern and values are read-only.  With the vectors on chip the gathers
// are short-latency, so no batching (which would cost registers here).
__device__ __forceinline__ double brow(const int* __restrict__ rp, const int* __restrict__ cl,
                                       const double* __restrict__ v, const double* w, int i) {
  const int a = __ldg(rp + i), e = __ldg(rp + i + 1);
  double acc = 0.0;
  for (int k = a; k < e; ++k) acc = fma(__ldg(v + k), w[__ldg(cl + k)], acc);
  return acc;
}

// f(i, (A w)_i) for every row i of the system.  TPR = 1: a row per thread
// (the sum in entry order).  TPR > 1 (threads per row): TPR adjacent threads
// of a warp share a row, thread j taking entries a + j, a + j + TPR, ...,
// then a fixed xor butterfly; f runs in the slice's first thread.  The pass
// count is the same for every thread of the group, so the shuffles always
// see full warps.  Long rows are where more threads per row pay; the
// autotuner measures it per batch.
template <int GT, int TPR, class F>
__device__ __forceinline__ void rows_apply(int gt, int n, const int* __restrict__ rp, const int* __restrict__ cl,
                                           const double* __restrict__ v, const double* w, F&& f) {
  if constexpr (TPR == 1) {
    for (int i = gt; i < n; i += GT) f(i, brow(rp, cl, v, w, i));
  } else {
    static_assert(TPR == 2 || TPR == 4 || TPR == 8, "threads per row");
    constexpr int RPP = GT / TPR;  // rows per pass
    const int sub = gt & (TPR - 1);
    const int passes = (n + RPP - 1) / RPP;
    for (int k = 0; k < passes; ++k) {
      const int i = gt / TPR + k * RPP;
      double acc = 0.0;
      if (i < n) {
        const int a = __ldg(rp + i), e = __ldg(rp + i + 1);
        for (int kk = a + sub; kk < e; kk += TPR) acc = fma(__ldg(v + kk), w[__ldg(cl + kk)], acc);
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (i < n && sub == 0) f(i, acc);
    }
  }
}

template <int GT, int SPC, int TPR>
__device__ void solve_system(const BatchDesc& d, const Grp<GT, SPC>& g, int n, const int* __restrict__ rp,
                             const int* __restrict__ cl, const double* __restrict__ v,
                             const double* __restrict__ b, double* __restrict__ x, double* vec,
                             BRed<GT>& sm, sla_info* info) {
  double* r = vec;
  double* z = vec + n;
  double* p = vec + 2 * (size_t)n;
  double* q = vec + 3 * (size_t)n;
  double* dinv = vec + 4 * (size_t)n;
  const int t = g.t;
  // ---- init: dinv, r = b - A x0, bnorm, bad diagonal
  double acc[2] = {0.0, 0.0};  // bb, bad
  for (int i = t; i < n; i += GT) {
    double diag = 0.0;
    for (int k = __ldg(rp + i); k < __ldg(rp + i + 1); ++k)
      if (__ldg(cl + k) == i) diag += __ldg(v + k);
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      if (!(diag > 0.0)) acc[1] = 1.0;
      di = 1.0 / diag;
    }
    dinv[i] = di;
    if (!d.use_x0) x[i] = 0.0;
    acc[0] = fma(b[i], b[i], acc[0]);
  }
  group_sums(g, acc, sm.red);
  const double bnorm = sqrt(acc[0]);
  const double thresh = fmax(d.rtol * bnorm, d.atol);
  sla_info inf{0, SLA_NOT_CONVERGED, 0.0, 0.0};
  if (acc[1] > 0.0) {
    if (t == 0) *info = sla_info{0, SLA_NOT_SPD, NAN, NAN};
    return;
  }
  if (bnorm == 0.0) {
    for (int i = t; i < n; i += GT) x[i] = 0.0;
    if (t == 0) *info = sla_info{0, SLA_OK, 0.0, 0.0};
    return;
  }
  int it = 0, status = SLA_NOT_CONVERGED;
  double rnorm = 0.0;
  for (int restart = 0; restart <= d.max_restarts; ++restart) {
    // r = b - A x ; z = dinv r ; p = z ; rho = r.z
    double s2[2] = {0.0, 0.0};  // rz, rr
    rows_apply<GT, TPR>(t, n, rp, cl, v, x, [&](int i, double ax) {
      const double ri = b[i] - ax;
      const double zi = dinv[i] * ri;
      r[i] = ri;
      z[i] = zi;
      p[i] = zi;
      s2[0] = fma(ri, zi, s2[0]);
      s2[1] = fma(ri, ri, s2[1]);
    });
    group_sums(g, s2, sm.red);  // also orders the p writes before the SpMV
    double rho = s2[0];
    rnorm = sqrt(s2[1]);
    status = SLA_NOT_CONVERGED;
    if (!isfinite(rho) || !isfinite(rnorm)) {
      status = SLA_BREAKDOWN;
      break;
    }
    while (!(rnorm <= thresh) && it < d.max_iter) {
      double pq[1] = {0.0};
      rows_apply<GT, TPR>(t, n, rp, cl, v, p, [&](int i, double qi) {
        q[i] = qi;
        pq[0] = fma(p[i], qi, pq[0]);
      });
      group_sums(g, pq, sm.red);
      if (!isfinite(pq[0])) { status = SLA_BREAKDOWN; break; }
      if (!(pq[0] > 0.0)) { status = SLA_NOT_SPD; break; }
      const double alpha = rho / pq[0];
      double u[2] = {0.0, 0.0};  // rz, rr
      for (int i = t; i < n; i += GT) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        const double zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        u[0] = fma(ri, zi, u[0]);
        u[1] = fma(ri, ri, u[1]);
      }
      group_sums(g, u, sm.red);
      const double rho_new = u[0];
      rnorm = sqrt(u[1]);
      ++it;
      if (!isfinite(rho_new) || !isfinite(rnorm)) { status = SLA_BREAKDOWN; break; }
      if (rnorm <= thresh) { status = SLA_OK; break; }
      if (!(rho_new > 0.0)) { status = SLA_NOT_SPD; break; }
      const double beta = rho_new / rho;
      for (int i = t; i < n; i += GT) p[i] = fma(beta, p[i], z[i]);
      g.sync();
      rho = rho_new;
    }
    if (rnorm <= thresh) status = SLA_OK;
    if (status != SLA_OK) break;
    // true residual
    double tt[1] = {0.0};
    rows_apply<GT, TPR>(t, n, rp, cl, v, x, [&](int i, double ax) {
      const double ti = b[i] - ax;
      tt[0] = fma(ti, ti, tt[0]);
    });
    group_sums(g, tt, sm.red);
    if (sqrt(tt[0]) <= 2.0 * thresh) break;
    if (restart == d.max_restarts) {
      status = SLA_NOT_CONVERGED;
      break;
    }
  }
  double tt[1] = {0.0};
  rows_apply<GT, TPR>(t, n, rp, cl, v, x, [&](int i, double ax) {
    const double ti = b[i] - ax;
    tt[0] = fma(ti, ti, tt[0]);
  });
  group_sums(g, tt, sm.red);
  inf.iters = it;
  inf.status = status;
  inf.rel_res = rnorm / bnorm;
  inf.true_rel_res = sqrt(tt[0]) / bnorm;
  if (t == 0) *info = inf;
}

// NT threads per CTA, SPC systems per CTA at a time (NT / SPC threads each),
// TPR threads per row in the SpMVs.
template <int NT, int SPC, int TPR>
__global__ void __launch_bounds__(NT, 1024 / NT) batched_pcg_kernel(BatchDesc d) {
  constexpr int GT = NT / SPC;
  extern __shared__ __align__(16) double dyn[];
  __shared__ BRed<GT> red[SPC];
  __shared__ int sys[SPC];
  const Grp<GT, SPC> g{(int)threadIdx.x / GT, (int)threadIdx.x % GT};
  for (;;) {
    g.sync();
    if (g.t == 0) sys[g.id] = (int)atomicAdd(d.next, 1u);
    g.sync();
    const int k = sys[g.id];
    if (k >= d.batch) break;
    const int s = d.order ? d.order[k] : k;
    int n;
    size_t row0;
    const int *rp, *cl;
    const double *v, *b;
    double* x;
    if (d.shared_pattern) {
      n = d.n;
      row0 = (size_t)s * n;
      rp = d.rowptr;
      cl = d.col;
      v = d.val + (size_t)s * d.nnz;
      b = d.b + (size_t)s * n;
      x = d.x + (size_t)s * n;
    } else {
      const int n0 = d.n_off[s];
      n = d.n_off[s + 1] - n0;
      row0 = (size_t)n0;
      const int e0 = d.nnz_off[s];
      if (d.skip_nnz > 0 && d.nnz_off[s + 1] - e0 >= d.skip_nnz) continue;  // a team's system
      rp = d.rowptr + n0 + s;
      cl = d.col + e0;
      v = d.val + e0;
      b = d.b + n0;
      x = d.x + n0;
    }
    double* vec = n <= d.smem_rows ? dyn + (size_t)g.id * 5 * d.smem_rows : d.gvec + 5 * row0;
    solve_system<GT, SPC, TPR>(d, g, n, rp, cl, v, b, x, vec, red[g.id], d.info + s);
  }
}

template <int NT, int SPC, int TPR>
int launch_batched(const BatchDesc& d0, bool use_smem, cudaStream_t s) {
  BatchDesc d = d0;
  static int smem_limit = 0;
  if (smem_limit == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, current_device());
    smem_limit = v > 0 ? v : 48 * 1024;
  }
  const int static_bytes = (int)(SPC * (sizeof(BRed<NT / SPC>) + sizeof(int))) + 1024;
  int rows = use_smem ? (smem_limit - static_bytes) / (5 * SPC * (int)sizeof(double)) : 0;
  if (rows > d.n_max) rows = d.n_max;
  if (rows < 0) rows = 0;
  d.smem_rows = rows;
  const size_t dyn = (size_t)rows * 5 * SPC * sizeof(double);
  SLA_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<NT, SPC, TPR>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_pcg_kernel<NT, SPC, TPR>, NT, dyn) !=
          cudaSuccess || per_sm <= 0)
    per_sm = 1;
  const int grid = persistent_grid(current_device(), (d.batch + SPC - 1) / SPC, per_sm, kMaxBlocks);
  SLA_CUDA_TRY(cudaMemsetAsync(d.next, 0, sizeof(unsigned), s));
  batched_pcg_kernel<NT, SPC, TPR><<<grid, NT, dyn, s>>>(d);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// config: low 4 bits = block size code (1: 256, 2: 512, 3: 1024; 0: auto),
// bit 4 = keep the vectors in global memory even when they fit on chip,
// bit 5 = no block teams for the large systems of a list, bit 6 = the block
// teams solve their systems by the pipelined PCG (sla_cg_pipe.cuh),
// bits 8-9 = log2 of the threads per row (1, 2, 4, 8), bits 10-11 = log2 of
// the systems per CTA (1, 2, 4; with one thread per row).
constexpr int kConfigNoTeams = 32;
constexpr int kConfigPipelined = 64;
constexpr int kConfigKnown = 15 | 16 | kConfigNoTeams | kConfigPipelined | (3 << 8) | (3 << 10);
// Systems of a list with at least kTeamMinNnz entries are solved by teams of
// blocks; the team launch is made when some system can have that many
// (n_max >= kTeamMinRows).
constexpr int kTeamMinNnz = 32768;
constexpr int kTeamMinRows = 2048;

template <int NT>
int dispatch_shape(const BatchDesc& d, bool use_smem, int tpr_log2, int spc_log2, cudaStream_t s) {
  if (spc_log2 != 0 && tpr_log2 != 0) return SLA_ERR_INVALID;  // systems per CTA with one thread per row
  switch (spc_log2 == 0 ? tpr_log2 : 4 + spc_log2) {
    case 0: return launch_batched<NT, 1, 1>(d, use_smem, s);
    case 1: return launch_batched<NT, 1, 2>(d, use_smem, s);
    case 2: return launch_batched<NT, 1, 4>(d, use_smem, s);
    case 3: return launch_batched<NT, 1, 8>(d, use_smem, s);
    case 5: return launch_batched<NT, 2, 1>(d, use_smem, s);
    case 6: return launch_batched<NT, 4, 1>(d, use_smem, s);
    default: return SLA_ERR_INVALID;
  }
}

int dispatch(const BatchDesc& d, int config, cudaStream_t s) {
  if (config & ~kConfigKnown) return SLA_ERR_INVALID;
  int code = config & 15;
  const bool use_smem = ((config >> 4) & 1) == 0;
  const int tpr_log2 = (config >> 8) & 3, spc_log2 = (config >> 10) & 3;
  if (code == 0) code = d.n_max >= 2048 ? 2 : 1;
  switch (code) {
    case 1: return dispatch_shape<256>(d, use_smem, tpr_log2, spc_log2, s);
    case 2: return dispatch_shape<512>(d, use_smem, tpr_log2, spc_log2, s);
    case 3: return dispatch_shape<1024>(d, use_smem, tpr_log2, spc_log2, s);
    default: return SLA_ERR_INVALID;
  }
}

int check_opts(const sla_opts* o) {
  if (o == nullptr || !(o->rtol >= 0.0) || !(o->atol >= 0.0) || o->max_iter < 0 ||
      o->max_restarts < 0 || o->max_restarts > 16 || (o->use_x0 != 0 && o->use_x0 != 1) ||
      (o->precond != SLA_PRECOND_NONE && o->precond != SLA_PRECOND_JACOBI))
    return SLA_ERR_INVALID;
  return SLA_OK;
}

void fill_opts(BatchDesc& d, const sla_opts* o) {
  d.rtol = o->rtol;
  d.atol = o->atol;
  d.max_iter = o->max_iter;
  d.max_restarts = o->max_restarts;
  d.precond = o->precond;
  d.use_x0 = o->use_x0;
}

// batched gradient: grad_val[s, k] = -lambda[s, row k] x[s, col k]
__global__ void batched_grad_kernel(int batch, int shared_pattern, int n, int nnz,
                                    const int* __restrict__ rowptr, const int* __restrict__ col,
                                    const int* __restrict__ n_off, const int* __restrict__ nnz_off,
                                    const double* __restrict__ lambda, const double* __restrict__ x,
                                    double* __restrict__ g) {
  for (int s = blockIdx.y; s < batch; s += gridDim.y) {
    int ns, e0, n0;
    const int* rp;
    if (shared_pattern) {
      ns = n;
      rp = rowptr;
      e0 = s * nnz;
      n0 = s * n;
    } else {
      n0 = n_off[s];
      ns = n_off[s + 1] - n0;
      rp = rowptr + n0 + s;
      e0 = nnz_off[s];
    }
    const int* cl = shared_pattern ? col : col + e0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
      const double li = -lambda[n0 + i];
      for (int k = rp[i]; k < rp[i + 1]; ++k) g[(size_t)e0 + k] = li * x[n0 + cl[k]];
    }
  }
}

}  // namespace

size_t team_scratch_bytes();
int launch_batched_teams(int batch, int min_nnz, const int* rowptr, const int* col, const int* n_off,
                         const int* nnz_off, const int* order, const double* val, const double* b, double* x,
                         sla_info* info, double* gvec, void* scratch, double rtol, double atol, int max_iter,
                         int max_restarts, int precond, int use_x0, bool pipelined, cudaStream_t s,
                         bool* launched);

// Workspace: scheduling counter | block-team scratch | 8 doubles per row of
// the batch (used by the systems whose vectors do not fit in shared memory,
// and by the systems the teams solve).
size_t batched_ws_bytes(long long total_rows) {
  return 256 + team_scratch_bytes() + al256((size_t)8 * sizeof(double) * (size_t)(total_rows > 0 ? total_rows : 1));
}

double* batched_gvec(void* ws) { return (double*)((char*)ws + 256 + team_scratch_bytes()); }

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_cg_batched_shared(const sla_csr* A, int32_t batch, const double* val,
                                         const double* b, double* x, const sla_opts* opts,
                                         sla_info* info, int32_t config, void* ws, size_t ws_bytes,
                                         void* stream) {
  if (A == nullptr || batch < 0 || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (check_opts(opts) != SLA_OK) return SLA_ERR_INVALID;
  if (batch == 0 || A->n == 0) return batch == 0 ? SLA_OK : SLA_ERR_INVALID;
  if (A->rowptr == nullptr || b == nullptr || x == nullptr || info == nullptr) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) ||
      ws_bytes < batched_ws_bytes((long long)batch * A->n))
    return SLA_ERR_WORKSPACE;
  BatchDesc d = {};
  d.batch = batch;
  d.shared_pattern = 1;
  d.n = A->n;
  d.nnz = A->nnz;
  d.rowptr = A->rowptr;
  d.col = A->col;
  d.val = val;
  d.b = b;
  d.x = x;
  d.info = info;
  d.next = (unsigned*)ws;
  d.gvec = batched_gvec(ws);
  d.n_max = A->n;
  fill_opts(d, opts);
  return dispatch(d, config, (cudaStream_t)stream);
}

extern "C" int32_t sla_cg_batched_list(int32_t batch, int32_t n_max, int32_t total_rows,
                                       const int32_t* n_off,
                                       const int32_t* nnz_off, const int32_t* rowptr,
                                       const int32_t* col, const double* val, const double* b,
                                       double* x, const int32_t* order, const sla_opts* opts,
                                       sla_info* info, int32_t config, void* ws, size_t ws_bytes,
                                       void* stream) {
  if (batch < 0 || n_max < 0 || total_rows < 0 || check_opts(opts) != SLA_OK) return SLA_ERR_INVALID;
  if (config & ~kConfigKnown) return SLA_ERR_INVALID;
  if (batch == 0) return SLA_OK;
  if (n_off == nullptr || nnz_off == nullptr || rowptr == nullptr || col == nullptr ||
      val == nullptr || b == nullptr || x == nullptr || info == nullptr)
    return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < batched_ws_bytes(total_rows))
    return SLA_ERR_WORKSPACE;
  BatchDesc d = {};
  d.batch = batch;
  d.shared_pattern = 0;
  d.rowptr = rowptr;
  d.col = col;
  d.n_off = n_off;
  d.nnz_off = nnz_off;
  d.val = val;
  d.b = b;
  d.x = x;
  d.info = info;
  d.order = order;
  d.next = (unsigned*)ws;
  d.gvec = batched_gvec(ws);
  d.n_max = n_max;
  fill_opts(d, opts);
  cudaStream_t s = (cudaStream_t)stream;
  if (!(config & kConfigNoTeams) && n_max >= kTeamMinRows) {
    // the large systems first, by teams of blocks (sla_cg_coop.cu)
    bool launched = false;
    const int rc = launch_batched_teams(batch, kTeamMinNnz, rowptr, col, n_off, nnz_off, order, val, b, x, info,
                                        d.gvec, (char*)ws + 256, opts->rtol, opts->atol, opts->max_iter,
                                        opts->max_restarts, opts->precond, opts->use_x0,
                                        (config & kConfigPipelined) != 0, s, &launched);
    if (rc != SLA_OK) return rc;
    if (launched) return SLA_OK;  // the team launch also solved the small systems
  }
  return dispatch(d, config, s);
}

extern "C" int32_t sla_grad_values_batched(int32_t batch, int32_t shared_pattern, int32_t n,
                                           int32_t nnz, const int32_t* rowptr, const int32_t* col,
                                           const int32_t* n_off, const int32_t* nnz_off,
                                           const double* lambda, const double* x,
                                           double* grad_val, void* stream) {
  if (batch < 0 || n < 0 || nnz < 0) return SLA_ERR_INVALID;
  if (batch == 0) return SLA_OK;
  if (rowptr == nullptr || col == nullptr || lambda == nullptr || x == nullptr || grad_val == nullptr)
    return SLA_ERR_INVALID;
  if (!shared_pattern && (n_off == nullptr || nnz_off == nullptr || n <= 0)) return SLA_ERR_INVALID;
  const int gx = (n + 255) / 256;
  dim3 grid((unsigned)(gx > 64 ? 64 : (gx > 0 ? gx : 1)), (unsigned)(batch < 65535 ? batch : 65535));
  batched_grad_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(batch, shared_pattern, n, nnz, rowptr, col,
                                                              n_off, nnz_off, lambda, x, grad_val);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
