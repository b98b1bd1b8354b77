// sla_internal.cuh -- helpers shared by the CUDA translation units of the
// library: error handling, deterministic block reductions, the
// "last block done" grid reduction, and the shared-memory-staged CSR row tile
// used by every SpMV in the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "sla.h"

namespace sla {

#define SLA_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t err__ = (expr);                              \
    if (err__ != cudaSuccess) return SLA_ERR_CUDA;           \
  } while (0)

constexpr int kWarp = 32;

// Round up to a multiple of 256 bytes (workspace carving granularity).
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device properties cached per device ordinal.
int num_sms(int device);
int current_device();

// ------------------------------------------------------------------------
// Deterministic reductions.  The xor butterfly gives every lane the same
// value (a + b == b + a exactly), and the block tree has a fixed shape, so a
// fixed launch configuration always reproduces the same bits.
// ------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; result valid in every thread.  `sh` needs NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  static_assert(NT % kWarp == 0 && NT <= 1024, "block size");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (lane < NT / kWarp) ? sh[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// Each block publishes `nv` partial sums (thread 0's values) to
// part[j * stride + blockIdx.x]; returns true in every thread of the last
// block to arrive, after which that block may read all partials.  The ticket
// counter is reset by the last block so the next launch starts from zero.
// No thread ever waits on another block.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, bool* s_last) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    *s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  bool last = *s_last;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Fixed-order sum of part[0..m) by one block (strided per thread, then tree).
template <int NT>
__device__ __forceinline__ double reduce_partials(const double* part, int m, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += NT) s += __ldcg(part + i);
  return block_sum<NT>(s, sh);
}

// ------------------------------------------------------------------------
// CSR row tile, staged through shared memory.
//
// A tile is kTileRows consecutive rows.  Its column indices and values are
// copied into shared memory with coalesced loads, then each thread
// sums one row sequentially from shared memory (one FP64 FMA per entry and
// no shuffle reduction, which matters on a part whose FP64 pipe is the
// scarce unit).  A tile whose entries exceed kTileCap is cut into chunks of
// whole rows that fit; a single row longer than kTileCap is summed by the
// whole block (strided partials + fixed tree).  The x gathers go through the
// read-only path so that L1/L2 serve the stencil neighbours.
// ------------------------------------------------------------------------
constexpr int kTileRows = 256;                // == block size of tile kernels
constexpr int kTileCap = 2048;                // staged entries per chunk
constexpr int kTileThreads = kTileRows;

struct TileSmem {
  int rp[kTileRows + 1];
  int col[kTileCap];
  double val[kTileCap];
  double red[kTileThreads / kWarp];
  int cnt;
};

// Calls epi(row, y_row) once for every row of the tile, from exactly one
// thread.  Must be called by all threads of the block.
template <class Epi>
__device__ __forceinline__ void spmv_tile(int tile, int n, const int* __restrict__ rowptr,
                                          const int* __restrict__ col,
                                          const double* __restrict__ val,
                                          const double* __restrict__ x, TileSmem& sm,
                                          Epi&& epi) {
  const int tid = threadIdx.x;
  const int r0 = tile * kTileRows;
  const int nr = min(kTileRows, n - r0);
  for (int i = tid; i <= nr; i += kTileThreads) sm.rp[i] = __ldg(rowptr + r0 + i);
  __syncthreads();
  int a = 0;
  while (a < nr) {
    const int base = sm.rp[a];
    const int r = a + 1 + tid;
    const int fits = (r <= nr) && (sm.rp[r] - base <= kTileCap);
    const int b = a + __syncthreads_count(fits);
    if (b == a) {
      // one row longer than the chunk capacity: whole block sums it
      const int e = sm.rp[a + 1];
      double s = 0.0;
      for (int k = base + tid; k < e; k += kTileThreads)
        s = fma(__ldg(val + k), __ldg(x + __ldg(col + k)), s);
      s = block_sum<kTileThreads>(s, sm.red);
      if (tid == 0) epi(r0 + a, s);
      __syncthreads();
      a += 1;
      continue;
    }
    const int kn = sm.rp[b] - base;
    // stage entries [base, base + kn): up to kTileCap / kTileThreads per thread
    constexpr int kPer = kTileCap / kTileThreads;
    int cv[kPer];
    double vv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kTileThreads;
      if (i < kn) {
        cv[j] = __ldg(col + base + i);
        vv[j] = __ldg(val + base + i);
      }
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kTileThreads;
      if (i < kn) {
        sm.col[i] = cv[j];
        sm.val[i] = vv[j];
      }
    }
    __syncthreads();
    const int row = a + tid;
    if (row < b) {
      const int s0 = sm.rp[row] - base, s1 = sm.rp[row + 1] - base;
      double s = 0.0;
      for (int k = s0; k < s1; ++k) s = fma(sm.val[k], __ldg(x + sm.col[k]), s);
      epi(r0 + row, s);
    }
    __syncthreads();
    a = b;
  }
}

// Grid size for a kernel that loops over `units` work items, `per_sm`
// resident blocks per SM, capped at `cap`.
inline int persistent_grid(int device, long long units, int per_sm, int cap) {
  long long g = (long long)num_sms(device) * per_sm;
  if (g > units) g = units;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace sla
