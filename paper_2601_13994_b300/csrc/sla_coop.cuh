// sla_coop.cuh -- pieces shared by the cooperative (one launch per solve)
// kernels: block shape, the shared scratch of a block, teams of blocks with
// their bounded barrier, and team-wide deterministic sums.  A team is the
// whole grid of a cooperative launch or a group of its blocks; every block of
// a team adds the team's partial sums in the same order, so every block
// holds the same bits of each reduced scalar.
#pragma once

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

constexpr int kCoopThreads = 512;
constexpr int kCoopMinBlocks = 2;
// two buffers of four partial arrays of gridDim.x doubles in the partials area
constexpr int kCoopMaxGrid = kMaxBlocks * kPartSlots / 8;
constexpr int kCoopUnroll = 2;

struct CoopSmem {
  double red[4 * kCoopThreads + 4];
  int flag;
};

// Gathered operand written earlier in this launch: plain (coherent) loads.
struct Coherent {
  const double* a;
  __device__ __forceinline__ double operator()(int i) const { return a[i]; }
};

// Calls f(i, a, e) for this thread's rows i = g0, g0 + T, ... < n, with
// [a, e) the row's entries.  (Loading the next row's bounds one row ahead
// was measured: no change.)
template <class F>
__device__ __forceinline__ void coop_rows(int n, int g0, int T, const int* __restrict__ rowptr, F&& f) {
  for (int i = g0; i < n; i += T) f(i, __ldg(rowptr + i), __ldg(rowptr + i + 1));
}

// The blocks that solve one system together: the whole grid, or a team of
// `size` consecutive blocks of a cooperative launch with its own barrier
// counter and partial-sum buffers (2 x 4 x size doubles).
struct Team {
  GridSync gs;
  int size, rank;
  double* part;
  int* err;
};

// A team of one block needs only the block barrier.
__device__ __forceinline__ bool team_sync(Team& tm, CoopSmem& sm) {
  if (tm.size == 1) {
    __syncthreads();
    return true;
  }
  return grid_sync(tm.gs, (unsigned)tm.size, tm.err, &sm.flag);
}

// Team totals of NV values: block sums -> partials -> barrier -> every block
// adds all partials in the same order.  False if the barrier ran out.
template <int NV>
__device__ __forceinline__ bool coop_sums(double (&v)[NV], Team& tm, int& buf, CoopSmem& sm) {
  block_sums<kCoopThreads, NV>(v, sm.red);
  if (tm.size == 1) return true;  // the block total is the team total
  const int G = tm.size;
  double* pb = tm.part + (size_t)buf * 4 * G;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) pb[j * G + tm.rank] = v[j];
  }
  buf ^= 1;
  if (!team_sync(tm, sm)) return false;
  reduce_partials<kCoopThreads, NV>(pb, G, G, v, sm.red);
  return true;
}

// Block-team scratch at the head of the batched workspace: a barrier counter
// and a queue slot per team (at most kCoopMaxGrid teams), the queue counter,
// the error flag, and 2 x 4 partial sums per block of the launch (a team of
// G blocks with index q uses parts[8 G q, 8 G (q + 1))).
struct TeamScratch {
  unsigned* counters;
  int* slots;
  unsigned* next;
  int* err;
  double* parts;
};
size_t team_scratch_bytes();
TeamScratch team_scratch(void* scratch);
// Zeroes the counters, slots, queue counter and error flag of the scratch and
// marks systems [0, batch) as timed out (a system no block reached keeps that
// record; each solve overwrites its own), on stream s.
int team_scratch_arm(void* scratch, int batch, sla_info* info, cudaStream_t s);

// Grid size of a cooperative solve over n rows at `occ` resident blocks per
// SM (one row per thread in every phase).
inline int coop_grid(int dev, int n, int occ) {
  return persistent_grid(dev, ((long long)n + kCoopThreads - 1) / kCoopThreads, occ, kCoopMaxGrid);
}

// Resident blocks per SM of a cooperative kernel on a device, or -1 when the
// device has no cooperative launch (cached by the caller).
int coop_occupancy_of(int dev, int* cache, const void* fn);

// true when a solve of n rows takes the cooperative form (SLA_CG_COOP=0 / 1
// forces it off / on); `limit` is the solver's measured crossover.
bool use_coop(long long n, long long limit);

}  // namespace sla
