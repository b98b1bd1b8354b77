// sla_bicgstab_batched.cu -- many right-preconditioned BiCGStab solves in one
// persistent launch (the nonsymmetric twin of sla_batched.cu).
//
// The paper's batched SparseTensor (one shared pattern) and SparseTensorList
// (distinct patterns) route every solver through one batch API (Sec. 3.1,
// App. B), BiCGStab for nonsymmetric systems among them.  Here persistent
// CTAs take systems from an atomic counter (largest first when an order is
// given) and each CTA runs the complete BiCGStab recurrence of its system:
// van der Vorst's method with r^ = r0 and the right Jacobi preconditioner,
// the half-step exit on ||s||, the same breakdown tests, true-residual check,
// restarts and statuses as the single-system solver and the oracle.  A
// system's convergence ends only its own CTA's loop (the per-system
// convergence mask); no block ever waits for another, so the launch always
// terminates.
//
// Per system the CTA keeps seven n-vectors: r (which also holds s), r^,
// p^ = D^-1 p, v = A p^, s^ = D^-1 s, t = A s^ and D^-1.  The search
// direction is carried preconditioned,
//   p^ <- D^-1 r + beta (p^ - omega D^-1 v),
// the oracle's p = r + beta (p - omega v) followed by p^ = D^-1 p written on
// p^ (equal in exact arithmetic), so no unpreconditioned p is stored.  Each
// iteration is four passes over the rows, each ending in one block
// reduction:
//   1. v = A p^ and r^.v                      -> alpha
//   2. s = r - alpha v (in place of r), s^ = D^-1 s, ||s||^2  -> half-step exit
//   3. t = A s^, t.t and t.s                   -> omega
//   4. x += alpha p^ + omega s^, r = s - omega t, p^ -= omega D^-1 v,
//      ||r||^2 and the next rho = r^.r          -> convergence, beta
// and the next iteration starts with p^ = D^-1 r + beta p^ inside pass 1.
// As many of the seven vectors as fit live in shared memory (the gathered
// p^ and s^ first); the others in the system's slot of the workspace (eight
// doubles per row of the batch, shared with the CG batch's layout).  On this
// part a batched small system is FP64-bound, so the passes are fused to
// keep the FP64 operations per row minimal.
#include <cmath>

#include "sla_coop.cuh"
#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

// from sla_batched.cu: workspace layout of the batched solvers
size_t batched_ws_bytes(long long total_rows);
double* batched_gvec(void* ws);

namespace {

constexpr int kVecs = 7;  // p^, s^, r(s), v, t, D^-1, r^ (in this order of priority for shared memory)

struct BicgBatchDesc {
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
  double* gvec;               // per-system slots: 8 doubles per row at 8 * (row offset)
  int smem_doubles;           // dynamic shared memory, in doubles
  double rtol, atol;
  int max_iter, max_restarts, precond, use_x0;
};

template <int NT>
struct BBSmem {
  double red[2 * NT + 2];
  int sys;
};

// The threads that solve one system and how they meet.  CtaGroup: one CTA
// (rows strided by its NT threads, block barriers, block sums).  TeamGroup:
// a team of blocks of one cooperative launch (rows strided by the team's
// threads, team barriers with a bounded wait, sums added in the same order
// by every block, so every block holds the same bits of every scalar and
// takes the same branches); its sync() and sums() are false when a barrier
// ran out, and the solve then returns false at once.
template <int NT>
struct CtaGroup {
  BBSmem<NT>& sm;
  __device__ __forceinline__ int first() const { return threadIdx.x; }
  __device__ __forceinline__ int stride() const { return NT; }
  __device__ __forceinline__ bool lead() const { return threadIdx.x == 0; }
  __device__ __forceinline__ bool sync() {
    __syncthreads();
    return true;
  }
  template <int NV>
  __device__ __forceinline__ bool sums(double (&v)[NV]) {
    block_sums<NT, NV>(v, sm.red);
    return true;
  }
};

struct TeamGroup {
  Team& tm;
  CoopSmem& sm;
  int buf;
  __device__ __forceinline__ int first() const { return tm.rank * kCoopThreads + (int)threadIdx.x; }
  __device__ __forceinline__ int stride() const { return tm.size * kCoopThreads; }
  __device__ __forceinline__ bool lead() const { return tm.rank == 0 && threadIdx.x == 0; }
  __device__ __forceinline__ bool sync() { return team_sync(tm, sm); }
  template <int NV>
  __device__ __forceinline__ bool sums(double (&v)[NV]) {
    return coop_sums(v, tm, buf, sm);
  }
};

// Row i of (rp, cl, v) times w, entries in order; w may be in shared memory
// or written earlier in this launch, so it is read with plain loads.
__device__ __forceinline__ double bb_row(const int* __restrict__ rp, const int* __restrict__ cl,
                                         const double* __restrict__ v, const double* w, int i) {
  const int a = __ldg(rp + i), e = __ldg(rp + i + 1);
  double acc = 0.0;
  for (int k = a; k < e; ++k) acc = fma(__ldg(v + k), w[__ldg(cl + k)], acc);
  return acc;
}

// One system's BiCGStab solve by the group g; false if a team barrier ran
// out (the caller then leaves the kernel).
template <class Grp>
__device__ bool bicg_system(const BicgBatchDesc& d, int n, const int* __restrict__ rp,
                            const int* __restrict__ cl, const double* __restrict__ v,
                            const double* __restrict__ b, double* __restrict__ x,
                            double* const (&vec)[kVecs], Grp& g, sla_info* info) {
  double* ph = vec[0];   // p^ = D^-1 p
  double* sh = vec[1];   // s^ = D^-1 s
  double* r = vec[2];    // r, and s in place of r within an iteration
  double* vv = vec[3];   // v = A p^
  double* t = vec[4];    // t = A s^
  double* dinv = vec[5];
  double* rh = vec[6];   // shadow residual r^ = r0
  const int first = g.first(), T = g.stride();

  // ---- init: D^-1 (A_ii = 0 or a non-finite inverse: invalid), x0, ||b||
  double acc[2] = {0.0, 0.0};  // bb, bad
  for (int i = first; i < n; i += T) {
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      double diag = 0.0;
      for (int k = __ldg(rp + i); k < __ldg(rp + i + 1); ++k)
        if (__ldg(cl + k) == i) diag += __ldg(v + k);
      di = 1.0 / diag;
      if (diag == 0.0 || !isfinite(di)) acc[1] = 1.0;
    }
    dinv[i] = di;
    if (!d.use_x0) x[i] = 0.0;
    acc[0] = fma(b[i], b[i], acc[0]);
  }
  if (!g.sums(acc)) return false;
  const double bnorm = sqrt(acc[0]);
  const double thresh = fmax(d.rtol * bnorm, d.atol);
  if (acc[1] > 0.0) {
    if (g.lead()) *info = sla_info{0, SLA_ERR_INVALID, NAN, NAN};
    return true;
  }
  if (bnorm == 0.0) {
    for (int i = first; i < n; i += T) x[i] = 0.0;
    if (g.lead()) *info = sla_info{0, SLA_OK, 0.0, 0.0};
    return true;
  }

  int it = 0, status = SLA_NOT_CONVERGED;
  double rnorm = 0.0;
  for (int restart = 0; restart <= d.max_restarts; ++restart) {
    // r = b - A x ; r^ = r ; p^ = v = 0 ; rho = r^.r = r.r
    double s0[1] = {0.0};
    for (int i = first; i < n; i += T) {
      const double ri = b[i] - bb_row(rp, cl, v, x, i);
      r[i] = ri;
      rh[i] = ri;
      ph[i] = 0.0;
      vv[i] = 0.0;
      s0[0] = fma(ri, ri, s0[0]);
    }
    if (!g.sums(s0)) return false;
    double rho = s0[0];
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    rnorm = sqrt(s0[0]);
    status = SLA_NOT_CONVERGED;
    if (!isfinite(rnorm)) {
      status = SLA_BREAKDOWN;
      break;
    }
    while (!(rnorm <= thresh) && it < d.max_iter) {
      if (!isfinite(rho) || fabs(rho) < 1e-300) {
        status = SLA_BREAKDOWN;
        break;
      }
      const double beta = (rho / rho_prev) * (alpha / omega);
      // pass 1a: p^ = D^-1 r + beta p^  (p^ already holds p^ - omega D^-1 v)
      for (int i = first; i < n; i += T) ph[i] = fma(beta, ph[i], dinv[i] * r[i]);
      if (!g.sync()) return false;
      // pass 1b: v = A p^, r^.v
      double a1[1] = {0.0};
      for (int i = first; i < n; i += T) {
        const double vi = bb_row(rp, cl, v, ph, i);
        vv[i] = vi;
        a1[0] = fma(rh[i], vi, a1[0]);
      }
      if (!g.sums(a1)) return false;
      const double rv = a1[0];
      if (!isfinite(rv) || rv == 0.0) {
        status = SLA_BREAKDOWN;
        break;
      }
      alpha = rho / rv;
      // pass 2: s = r - alpha v (in place), s^ = D^-1 s, ||s||^2
      double a2[1] = {0.0};
      for (int i = first; i < n; i += T) {
        const double si = fma(-alpha, vv[i], r[i]);
        r[i] = si;
        sh[i] = dinv[i] * si;
        a2[0] = fma(si, si, a2[0]);
      }
      if (!g.sums(a2)) return false;
      ++it;
      const double snorm = sqrt(a2[0]);
      if (snorm <= thresh) {  // half-step exit: x += alpha p^
        for (int i = first; i < n; i += T) x[i] = fma(alpha, ph[i], x[i]);
        if (!g.sync()) return false;  // the true residual next gathers other threads' x
        rnorm = snorm;
        status = SLA_OK;
        break;
      }
      // pass 3: t = A s^, t.t, t.s
      double a3[2] = {0.0, 0.0};
      for (int i = first; i < n; i += T) {
        const double ti = bb_row(rp, cl, v, sh, i);
        t[i] = ti;
        a3[0] = fma(ti, ti, a3[0]);
        a3[1] = fma(ti, r[i], a3[1]);
      }
      if (!g.sums(a3)) return false;
      if (!isfinite(a3[0]) || !isfinite(a3[1]) || a3[0] == 0.0) {
        status = SLA_BREAKDOWN;
        break;
      }
      omega = a3[1] / a3[0];
      // pass 4: x += alpha p^ + omega s^, r = s - omega t, p^ -= omega D^-1 v,
      // ||r||^2 and the next rho = r^.r
      double a4[2] = {0.0, 0.0};
      for (int i = first; i < n; i += T) {
        const double pi = ph[i];
        x[i] = x[i] + (alpha * pi + omega * sh[i]);
        const double ri = fma(-omega, t[i], r[i]);
        r[i] = ri;
        ph[i] = fma(-omega, dinv[i] * vv[i], pi);
        a4[0] = fma(ri, ri, a4[0]);
        a4[1] = fma(rh[i], ri, a4[1]);
      }
      if (!g.sums(a4)) return false;
      rnorm = sqrt(a4[0]);
      if (!isfinite(rnorm)) {
        status = SLA_BREAKDOWN;
        break;
      }
      if (rnorm <= thresh) {
        status = SLA_OK;
        break;
      }
      if (omega == 0.0) {
        status = SLA_BREAKDOWN;
        break;
      }
      rho_prev = rho;
      rho = a4[1];
    }
    // a start that already meets the stopping test is converged
    if (status == SLA_NOT_CONVERGED && rnorm <= thresh) status = SLA_OK;
    if (status != SLA_OK) break;
    // true residual
    double tt[1] = {0.0};
    for (int i = first; i < n; i += T) {
      const double ti = b[i] - bb_row(rp, cl, v, x, i);
      tt[0] = fma(ti, ti, tt[0]);
    }
    if (!g.sums(tt)) return false;
    if (sqrt(tt[0]) <= 2.0 * thresh) break;
    if (restart == d.max_restarts) {
      status = SLA_NOT_CONVERGED;
      break;
    }
  }
  double tt[1] = {0.0};
  for (int i = first; i < n; i += T) {
    const double ti = b[i] - bb_row(rp, cl, v, x, i);
    tt[0] = fma(ti, ti, tt[0]);
  }
  if (!g.sums(tt)) return false;
  if (g.lead()) *info = sla_info{it, status, rnorm / bnorm, sqrt(tt[0]) / bnorm};
  return true;
}

template <int NT>
__global__ void __launch_bounds__(NT) batched_bicgstab_kernel(BicgBatchDesc d) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ BBSmem<NT> sm;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm.sys = (int)atomicAdd(d.next, 1u);
    __syncthreads();
    const int k = sm.sys;
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
      rp = d.rowptr + n0 + s;
      cl = d.col + e0;
      v = d.val + e0;
      b = d.b + n0;
      x = d.x + n0;
    }
    // the first vectors that fit go to shared memory, the others to the
    // system's slot of the workspace
    const int on_chip = n > 0 ? min(kVecs, d.smem_doubles / n) : kVecs;
    double* slot = d.gvec + 8 * row0;
    double* vec[kVecs];
#pragma unroll
    for (int j = 0; j < kVecs; ++j)
      vec[j] = j < on_chip ? dyn + (size_t)j * n : slot + (size_t)j * n;
    CtaGroup<NT> g{sm};
    bicg_system(d, n, rp, cl, v, b, x, vec, g, d.info + s);
  }
}

// ------------------------------------------------------------------ block teams
//
// A distinct-pattern batch whose largest systems, each on one CTA, would run
// at one SM's FP64 rate and set the batch's time: teams of `team`
// consecutive blocks of one cooperative launch take systems from the queue
// (largest first) while they have at least min_nnz entries and solve each
// together (TeamGroup); the first smaller system a team meets splits it into
// single blocks, which take the rest of the queue one system each, so the
// small systems fill the time the last large ones take.  Every vector of a
// system lives in its workspace slot (other blocks of the team gather it).

struct BicgTeamArgs {
  BicgBatchDesc d;  // the list (shared_pattern = 0)
  int team, min_nnz;
  TeamScratch ts;
};

struct SysRef {
  long long row0;
  const int* rp;
  const int* cl;
  const double* v;
  const double* b;
  double* x;
  int n, sys;
};

__device__ __forceinline__ void list_system(const BicgBatchDesc& d, int sys, SysRef& r) {
  const int n0 = d.n_off[sys], e0 = d.nnz_off[sys];
  r.row0 = n0;
  r.n = d.n_off[sys + 1] - n0;
  r.rp = d.rowptr + n0 + sys;
  r.cl = d.col + e0;
  r.v = d.val + e0;
  r.b = d.b + n0;
  r.x = d.x + n0;
  r.sys = sys;
}

template <class Grp>
__device__ __forceinline__ bool solve_ref(const BicgBatchDesc& d, const SysRef& r, Grp& g) {
  const size_t n = (size_t)r.n;
  double* slot = d.gvec + 8 * (size_t)r.row0;
  double* const vec[kVecs] = {slot, slot + n, slot + 2 * n, slot + 3 * n, slot + 4 * n, slot + 5 * n, slot + 6 * n};
  return bicg_system(d, r.n, r.rp, r.cl, r.v, r.b, r.x, vec, g, d.info + r.sys);
}

__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) bicg_team_kernel(BicgTeamArgs A) {
  __shared__ CoopSmem sm;
  __shared__ SysRef sr;
  __shared__ int s_k, s_mode;
  const BicgBatchDesc& d = A.d;
  const int q = blockIdx.x / A.team, rank = blockIdx.x % A.team;
  Team tm{GridSync{A.ts.counters + q, 0u}, A.team, rank, A.ts.parts + (size_t)q * 8 * A.team, A.ts.err};
  int first = -1;  // queue position this block takes first in single mode
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) A.ts.slots[q] = (int)atomicAdd(A.ts.next, 1u);
    if (!team_sync(tm, sm)) return;
    if (threadIdx.x == 0) {
      const int k = __ldcg(A.ts.slots + q);
      s_k = k;
      s_mode = 2;  // queue exhausted
      if (k < d.batch) {
        const int sys = d.order ? d.order[k] : k;
        s_mode = 1;  // a small system: single mode from here
        if (d.nnz_off[sys + 1] - d.nnz_off[sys] >= A.min_nnz) {
          list_system(d, sys, sr);
          s_mode = 0;
        }
      }
    }
    __syncthreads();
    const int mode = s_mode;
    if (mode == 2) return;
    if (mode == 1) {
      if (rank == 0) first = s_k;
      break;
    }
    TeamGroup g{tm, sm, 0};
    if (!solve_ref(d, sr, g)) return;
  }
  // single mode: every block solves whole systems on its own
  Team solo{GridSync{nullptr, 0u}, 1, 0, nullptr, A.ts.err};
  for (;;) {
    __syncthreads();  // sr and s_mode are rewritten for the next system
    if (threadIdx.x == 0) {
      const int k = first >= 0 ? first : (int)atomicAdd(A.ts.next, 1u);
      s_mode = 2;
      if (k < d.batch) {
        list_system(d, d.order ? d.order[k] : k, sr);
        s_mode = 0;
      }
    }
    first = -1;
    __syncthreads();
    if (s_mode != 0) return;
    TeamGroup g{solo, sm, 0};
    if (!solve_ref(d, sr, g)) return;
  }
}

int g_occ_bicg_team[64] = {};

// The team launch of a list; *launched is false (nothing enqueued) when the
// device has no cooperative launch.
int launch_teams(const BicgBatchDesc& d, int team, int min_nnz, void* scratch, cudaStream_t s, bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const int occ = coop_occupancy_of(dev, g_occ_bicg_team, (const void*)bicg_team_kernel);
  if (occ <= 0) return SLA_OK;
  int grid = num_sms(dev) * occ;
  if (grid > kCoopMaxGrid) grid = kCoopMaxGrid;
  grid -= grid % team;
  if (grid < team) return SLA_OK;
  BicgTeamArgs A;
  A.d = d;
  A.team = team;
  A.min_nnz = min_nnz;
  A.ts = team_scratch(scratch);
  const int rc = team_scratch_arm(scratch, d.batch, d.info, s);
  if (rc != SLA_OK) return rc;
  void* args[] = {&A};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bicg_team_kernel, dim3(grid), dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

template <int NT>
int launch(const BicgBatchDesc& d0, int n_max, bool use_smem, cudaStream_t s) {
  BicgBatchDesc d = d0;
  static int smem_limit = 0;
  if (smem_limit == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, current_device());
    smem_limit = v > 0 ? v : 48 * 1024;
  }
  const int static_bytes = (int)sizeof(BBSmem<NT>) + 1024;
  long long doubles = use_smem ? (smem_limit - static_bytes) / (int)sizeof(double) : 0;
  // no more than the largest system can use
  if (doubles > (long long)kVecs * n_max) doubles = (long long)kVecs * n_max;
  // whole vectors of the largest system only (smaller systems fit more)
  if (n_max > 0 && doubles >= n_max) doubles = (doubles / n_max) * n_max;
  if (doubles < 0) doubles = 0;
  d.smem_doubles = (int)doubles;
  const size_t dyn = (size_t)doubles * sizeof(double);
  SLA_CUDA_TRY(cudaFuncSetAttribute(batched_bicgstab_kernel<NT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_bicgstab_kernel<NT>, NT, dyn) !=
          cudaSuccess || per_sm <= 0)
    per_sm = 1;
  const int grid = persistent_grid(current_device(), d.batch, per_sm, kMaxBlocks);
  SLA_CUDA_TRY(cudaMemsetAsync(d.next, 0, sizeof(unsigned), s));
  batched_bicgstab_kernel<NT><<<grid, NT, dyn, s>>>(d);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// config: low 4 bits = block size code (1: 256, 2: 512, 3: 1024; 0: auto),
// bit 4 = every vector in the workspace slot (none in shared memory); for a
// list also bit 5 = no block teams, bits 8-9 = team size code (0: 3 blocks,
// 1: 2, 2: 4, 3: 6), bits 10-11 = the entries from which a system goes to a
// team (0: 32768, 1: 16384, 2: 65536, 3: 131072).  The team shapes were swept
// on 512 convection-diffusion rectangles; the autotuner searches them.
constexpr int kConfigNoTeams = 32;
constexpr int kConfigShared = 15 | 16;
constexpr int kConfigList = kConfigShared | kConfigNoTeams | (3 << 8) | (3 << 10);
constexpr int kTeamSizes[4] = {3, 2, 4, 6};
constexpr int kTeamMinNnz[4] = {32768, 16384, 65536, 131072};
// the team launch is made when some system can have that many entries
constexpr int kTeamMinRows = 2048;

int dispatch(const BicgBatchDesc& d, int n_max, int config, cudaStream_t s) {
  config &= kConfigShared;
  int code = config & 15;
  const bool use_smem = ((config >> 4) & 1) == 0;
  if (code == 0) code = n_max >= 2048 ? 2 : 1;
  switch (code) {
    case 1: return launch<256>(d, n_max, use_smem, s);
    case 2: return launch<512>(d, n_max, use_smem, s);
    case 3: return launch<1024>(d, n_max, use_smem, s);
    default: return SLA_ERR_INVALID;
  }
}

int check_opts(const sla_opts* o) {
  if (o == nullptr || !(o->rtol >= 0.0) || !(o->atol >= 0.0) || o->max_iter < 0 ||
      o->max_restarts < 0 || o->max_restarts > 16 || (o->use_x0 != 0 && o->use_x0 != 1) ||
      (o->precond != SLA_PRECOND_NONE && o->precond != SLA_PRECOND_JACOBI) || o->flags != 0)
    return SLA_ERR_INVALID;
  return SLA_OK;
}

void fill_opts(BicgBatchDesc& d, const sla_opts* o) {
  d.rtol = o->rtol;
  d.atol = o->atol;
  d.max_iter = o->max_iter;
  d.max_restarts = o->max_restarts;
  d.precond = o->precond;
  d.use_x0 = o->use_x0;
}

// out[s, m] = val[s, perm[m]] for every system s of a shared pattern
__global__ void gather_batched_kernel(int batch, long long nnz, const int* __restrict__ perm,
                                      const double* __restrict__ val, double* __restrict__ out) {
  for (int s = blockIdx.y; s < batch; s += gridDim.y) {
    const double* vs = val + (size_t)s * nnz;
    double* os = out + (size_t)s * nnz;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < nnz;
         m += (long long)gridDim.x * blockDim.x)
      os[m] = __ldg(vs + __ldg(perm + m));
  }
}

}  // namespace

// The argument checks of sla_bicgstab_batched_* that need no pointer: its
// options and the config word of the layout (shared pattern or list).
// The batched adjoint runs them before it enqueues the values gather.
int bicg_batched_precheck(const sla_opts* opts, int config, bool list) {
  if (check_opts(opts) != SLA_OK) return SLA_ERR_INVALID;
  if (config & ~(list ? kConfigList : kConfigShared)) return SLA_ERR_INVALID;
  return (config & 15) <= 3 ? SLA_OK : SLA_ERR_INVALID;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_bicgstab_batched_shared(const sla_csr* A, int32_t batch, const double* val,
                                               const double* b, double* x, const sla_opts* opts,
                                               sla_info* info, int32_t config, void* ws,
                                               size_t ws_bytes, void* stream) {
  if (A == nullptr || batch < 0 || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (check_opts(opts) != SLA_OK) return SLA_ERR_INVALID;
  if (batch == 0 || A->n == 0) return batch == 0 ? SLA_OK : SLA_ERR_INVALID;
  if (A->rowptr == nullptr || b == nullptr || x == nullptr || info == nullptr) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if ((const void*)b == (const void*)x) return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) ||
      ws_bytes < batched_ws_bytes((long long)batch * A->n))
    return SLA_ERR_WORKSPACE;
  if (config & ~kConfigShared) return SLA_ERR_INVALID;
  BicgBatchDesc d = {};
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
  fill_opts(d, opts);
  return dispatch(d, A->n, config, (cudaStream_t)stream);
}

extern "C" int32_t sla_bicgstab_batched_list(int32_t batch, int32_t n_max, int32_t total_rows,
                                             const int32_t* n_off, const int32_t* nnz_off,
                                             const int32_t* rowptr, const int32_t* col,
                                             const double* val, const double* b, double* x,
                                             const int32_t* order, const sla_opts* opts,
                                             sla_info* info, int32_t config, void* ws,
                                             size_t ws_bytes, void* stream) {
  if (batch < 0 || n_max < 0 || total_rows < 0 || check_opts(opts) != SLA_OK) return SLA_ERR_INVALID;
  if (config & ~kConfigList) return SLA_ERR_INVALID;
  if (batch == 0) return SLA_OK;
  if (n_off == nullptr || nnz_off == nullptr || rowptr == nullptr || col == nullptr ||
      val == nullptr || b == nullptr || x == nullptr || info == nullptr)
    return SLA_ERR_INVALID;
  if ((const void*)b == (const void*)x) return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < batched_ws_bytes(total_rows))
    return SLA_ERR_WORKSPACE;
  BicgBatchDesc d = {};
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
  fill_opts(d, opts);
  cudaStream_t s = (cudaStream_t)stream;
  if (!(config & kConfigNoTeams) && n_max >= kTeamMinRows) {
    // the large systems by teams of blocks, the small ones by single blocks,
    // in one cooperative launch
    bool launched = false;
    const int rc = launch_teams(d, kTeamSizes[(config >> 8) & 3], kTeamMinNnz[(config >> 10) & 3],
                                (char*)ws + 256, s, &launched);
    if (rc != SLA_OK || launched) return rc;
  }
  return dispatch(d, n_max, config, s);
}

extern "C" int32_t sla_gather_values_batched(int32_t batch, int64_t nnz, const int32_t* perm,
                                             const double* val, double* out, void* stream) {
  if (batch < 0 || nnz < 0) return SLA_ERR_INVALID;
  if (batch == 0 || nnz == 0) return SLA_OK;
  if (perm == nullptr || val == nullptr || out == nullptr) return SLA_ERR_INVALID;
  if (ranges_overlap(val, 8 * (size_t)nnz * batch, out, 8 * (size_t)nnz * batch)) return SLA_ERR_INVALID;
  const long long gx = (nnz + 255) / 256;
  dim3 grid((unsigned)(gx > 256 ? 256 : gx), (unsigned)(batch < 65535 ? batch : 65535));
  gather_batched_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(batch, nnz, perm, val, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
