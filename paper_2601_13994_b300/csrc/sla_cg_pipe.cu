// sla_cg_pipe.cu -- pipelined Jacobi PCG in one cooperative launch.
//
// The method is the pipelined PCG of Ghysels and Vanroose ("Hiding global
// synchronization latency in the preconditioned Conjugate Gradient
// algorithm", Parallel Computing 2014): one of the CG variants that merge the
// inner products of an iteration into one reduction, which App. C names as
// the way past the reduction latency of Algorithm 1.  In exact arithmetic its
// iterates are those of Algorithm 1.  It carries w = A u, s = A p and
// z = A D^{-1} s as recurrences, so that the three inner products of an
// iteration are one reduction and the iteration's SpMV (of m = D^{-1} w)
// does not wait for that reduction.  Here each iteration is ONE phase between
// two grid barriers:
//
//   (r.u, w.u, r.r) of the previous phase -> convergence test, alpha, beta
//       (every block adds the same partials in the same order, so all take
//       the same decision);
//   nv = A m                        (m written by the previous phase)
//   z = nv + beta z,  s = w + beta s,  p = u + beta p
//   x += alpha p,  r -= alpha s,  w -= alpha z,  u = D^{-1} r
//   m' = D^{-1} w and the partial sums of r.u, w.u, r.r,
//
// against three barriers per iteration (two reductions and the p update) in
// the standard form (sla_cg_coop.cu).  The price is vector traffic: z, s, w
// and m are read or written each iteration, 120 bytes per row against 104.
// m is double-buffered: a phase gathers m from one buffer while every block
// writes the next m into the other, and the barrier at the end of the phase
// orders the two.
//
// Reading for the Jacobi (or identity) preconditioner: u = D^{-1} r is
// recomputed from r rather than carried by the general method's recurrence
// u -= alpha q, q = m + beta q (equal in exact arithmetic), so q is not
// stored.  Exits and restarts are those of the standard solve: the
// recursive-residual test, the true residual b - A x with at most
// max_restarts restarts from x, NOT_SPD when r.u <= 0 or when the
// denominator (= p^T A p) is <= 0 on the first step of a start (where it is
// u^T A u from a fresh product), BREAKDOWN on a non-finite scalar.  A
// denominator <= 0 on a later step comes from rounding in the recurrences
// of w, s, z near the attainable accuracy -- the pipelined method's known
// weakness -- not from an indefinite A: it sends the solve to the
// true-residual check, which accepts within twice the target or restarts
// from x (fresh recurrences) while restarts remain.
//
// Ownership: thread g of the T threads of the grid owns rows g, g + T, ...;
// only m (and x in the residual checks) is gathered across threads, always
// after a barrier and through plain (coherent) loads.
#include "sla_cg_pipe.cuh"

namespace sla {

struct PipeArgs {
  KrylovDesc d;
  KrylovState* st;
  double* part;
  double* rec;  // [n][kRec]
  double* m0;   // [n] m = D^{-1} w, two buffers
  double* m1;
};

__global__ void __launch_bounds__(kCoopThreads, kCoopMinBlocks) cg_pipe_kernel(PipeArgs A) {
  __shared__ CoopSmem sm;
  __shared__ PipeState s;
  __shared__ KrylovDesc d;
  if (threadIdx.x == 0) d = A.d;
  __syncthreads();
  Team tm{GridSync{&A.st->cnt[5], 0u}, (int)gridDim.x, (int)blockIdx.x, A.part, &A.st->err};
  pipe_team_solve(d, A.rec, A.m0, A.m1, tm, true, sm, s);
}

// Zeroes the barrier counters and the error flag before a launch.
__global__ void pipe_arm_kernel(KrylovState* st) {
  for (int i = 0; i < 8; ++i) st->cnt[i] = 0u;
  st->err = 0;
}

namespace {
int g_occ_pipe[64] = {};
}  // namespace

// Launches the pipelined solve; *launched is false (nothing enqueued) when
// the device has no cooperative launch.
int launch_cg_pipe(const KrylovDesc& desc, void* ws, cudaStream_t s, bool* launched) {
  *launched = false;
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return SLA_OK;
  const int occ = coop_occupancy_of(dev, g_occ_pipe, (const void*)cg_pipe_kernel);
  if (occ <= 0) return SLA_OK;
  const CgPipeLayout L = cg_pipe_layout(desc.n);
  char* base = (char*)ws;
  PipeArgs A;
  A.d = desc;
  A.st = (KrylovState*)(base + L.state);
  A.part = (double*)(base + L.part);
  A.rec = (double*)(base + L.rec);
  A.m0 = (double*)(base + L.m0);
  A.m1 = (double*)(base + L.m1);
  pipe_arm_kernel<<<1, 1, 0, s>>>(A.st);
  SLA_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  SLA_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cg_pipe_kernel, dim3(coop_grid(dev, desc.n, occ)),
                                           dim3(kCoopThreads), args, 0, s));
  *launched = true;
  return SLA_OK;
}

}  // namespace sla
