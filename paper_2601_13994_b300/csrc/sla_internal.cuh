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

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
inline bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na > 0 && nb > 0 && x < y + nb && y < x + na;
}

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

// Sums NV values over the block; on return v[j] holds block total j in every
// thread.  Each thread parks its values in shared memory and warp j adds
// value j: lane l takes entries l, l+32, l+64, ... in that order
// (bank-conflict free), then a 5-level butterfly.  That is NT/32 + 4 FP64
// adds per lane of one warp per value, instead of a butterfly in every warp
// -- FP64 adds are the scarce unit on this part.  Needs NV <= NT/32; the
// scratch array must hold NV*NT + NV doubles (checked at compile time).
template <int NT, int NV, int M>
__device__ __forceinline__ void block_sums(double (&v)[NV], double (&sh)[M]) {
  static_assert(NT % kWarp == 0 && NT <= 1024 && NV <= NT / kWarp, "block size");
  static_assert(M >= NV * NT + NV, "reduction scratch too small");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j * NT + tid] = v[j];
  __syncthreads();
  if (w < NV) {
    const double* col = sh + w * NT + lane;
    double s = col[0];
#pragma unroll
    for (int k = 1; k < NT / kWarp; ++k) s += col[kWarp * k];
    s = warp_sum(s);
    if (lane == 0) sh[NV * NT + w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = sh[NV * NT + j];
}

// Single-value form of block_sums.
template <int NT, int M>
__device__ __forceinline__ double block_sum(double v, double (&sh)[M]) {
  double a[1] = {v};
  block_sums<NT, 1>(a, sh);
  return a[0];
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

// ------------------------------------------------------------------------
// Grid-wide barrier of a cooperative launch (every block resident).  One
// counter that only grows: thread 0 of each block adds 1 with release
// semantics (making the block's writes, ordered before it by the block
// barrier, visible), and barrier k of the launch is complete once the
// counter reaches (k + 1) * members (compared modulo 2^32), which thread 0
// polls with acquire loads.  `epoch` counts the barriers this block has
// passed (the same in every block); the counter is zero at launch.  Measured
// 0.8 us (8 blocks) to 1.6 us (296 blocks) per barrier, against 1.2-2.1 us
// for a ticket counter re-armed by the last arrival plus a generation word.
// The poll is bounded by a clock64 budget (about 2 s at the highest clock):
// a wait that runs out sets *err and returns false in every thread of the
// block, which must then leave the kernel -- the other blocks run out at
// their next barrier, so the launch always ends.
// ------------------------------------------------------------------------
constexpr long long kGridWaitBudgetCycles = 4000000000LL;

struct GridSync {
  unsigned* count;
  unsigned epoch;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// `members`: the number of blocks that take part (the whole grid, or a team
// of blocks of a cooperative launch with a counter of its own).
__device__ __forceinline__ bool grid_sync(GridSync& g, unsigned members, int* err, int* s_flag,
                                          long long budget = kGridWaitBudgetCycles) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned goal = (g.epoch + 1u) * members;
    int ok = 1;
    red_add_release_gpu(g.count, 1u);
    if ((int)(ld_acquire_gpu(g.count) - goal) < 0) {
      const long long t0 = clock64();
      while ((int)(ld_acquire_gpu(g.count) - goal) < 0) {
        if (clock64() - t0 > budget) {
          atomicOr(err, 1);
          ok = 0;
          break;
        }
      }
    }
    *s_flag = ok;
  }
  __syncthreads();
  g.epoch += 1u;
  return *s_flag != 0;
}

// Fixed-order sums of NV partial arrays part[j*stride + 0..m) by one block
// (strided per thread, then block_sums).  The loads of four strides of every
// array are issued before their adds (this runs in the last block of a
// kernel, on the critical path between kernels: one L2 round trip per four
// strides instead of one per value); the adds keep the strided order.
template <int NT, int NV, int M>
__device__ __forceinline__ void reduce_partials(const double* part, int stride, int m,
                                                double (&out)[NV], double (&sh)[M]) {
  constexpr int kU = 4;
#pragma unroll
  for (int j = 0; j < NV; ++j) out[j] = 0.0;
  for (int i0 = threadIdx.x; i0 < m; i0 += kU * NT) {
    double v[NV][kU];
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int i = i0 + u * NT;
        v[j][u] = i < m ? __ldcg(part + j * stride + i) : 0.0;
      }
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
      for (int u = 0; u < kU; ++u)
        if (i0 + u * NT < m) out[j] += v[j][u];
  }
  block_sums<NT, NV>(out, sh);
}

// ------------------------------------------------------------------------
// One row's sum  sum_k val[k] x[col[k]]  over k in [a, e), with the gathers
// batched: the column indices of up to kGatherBatch entries are read first,
// then their x loads are issued back to back, then the FMAs run in entry
// order (the same sequential sum as one entry at a time, so the bits do not
// change).  A row therefore waits for one gather latency per batch instead
// of one per entry.  col_at(k) / val_at(k) read entry k (shared or global memory); x is
// an array or a functor of the column (gather_at); its element type is the
// type of val_at's result and of the sum.
// ------------------------------------------------------------------------
constexpr int kGatherBatch = 4;  // 4 (vs 8) keeps the TMA consumers at four blocks per SM

// ------------------------------------------------------------------------
// Element types of the SpMVs.  Matrix values are FP64, or FP32 for factors
// whose values carry no more (the learned G); FP32 values are widened to
// FP64 exactly with integer bit operations (to_f64), since a hardware
// conversion would occupy the FP64 pipe, the scarce unit on this part.
// ------------------------------------------------------------------------
__device__ __forceinline__ double to_f64(double v) { return v; }

// Exact float -> double for normal numbers, signed zero for zero/subnormal
// inputs (callers store no subnormal values), inf/nan kept.
__device__ __forceinline__ double to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (ex == 0) return __longlong_as_double((long long)sign);
  const unsigned long long e64 = ex == 0xffu ? 2047ull : (unsigned long long)(ex + 896u);
  const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | (e64 << 52) | man));
}

// A stored value in the arithmetic type X of the sum: FP64 values as they
// are, FP32 values widened exactly for an FP64 sum or kept for an FP32 sum.
template <class X>
__device__ __forceinline__ X as_x(double v) { return v; }
template <class X>
__device__ __forceinline__ X as_x(float v);
template <>
__device__ __forceinline__ double as_x<double>(float v) { return to_f64(v); }
template <>
__device__ __forceinline__ float as_x<float>(float v) { return v; }

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_any(double v) { return warp_sum(v); }
__device__ __forceinline__ float warp_sum_any(float v) { return warp_sum_f(v); }

// The epilogue operand of a row: aux[row] for an array (0 when null), or
// aux(row) for a functor.
template <class A>
__device__ __forceinline__ A aux_at(const A* __restrict__ aux, int row) {
  return aux ? __ldg(aux + row) : A(0);
}
template <class F>
__device__ __forceinline__ auto aux_at(F& f, int row) -> decltype(f(row)) {
  return f(row);
}

// x[c] for a gathered operand given as an array (read through the read-only
// path) or as a functor of the column (an operand formed on the fly).
template <class T>
__device__ __forceinline__ T gather_at(const T* __restrict__ x, int c) {
  return __ldg(x + c);
}
template <class F>
__device__ __forceinline__ auto gather_at(F& f, int c) -> decltype(f(c)) {
  return f(c);
}

// acc = fma(v, x, acc) in the threads where `on` holds, as a predicated
// instruction: threads without the predicate issue no FP64 operation.  (A
// guarded fma in C++ -- `if (j < rem) acc = fma(...)` in an unrolled loop --
// was measured to execute in every thread, 8.93 DFMA per row in the PCG
// SpMV where 7.97 were needed: the compiler evaluates it unconditionally and
// keeps the old value where the guard fails.)
__device__ __forceinline__ double fma_if(bool on, double v, double x, double acc) {
  asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t@p fma.rn.f64 %0, %1, %2, %0;\n\t}"
      : "+d"(acc)
      : "d"(v), "d"(x), "r"((unsigned)on));
  return acc;
}
__device__ __forceinline__ float fma_if(bool on, float v, float x, float acc) {
  asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t@p fma.rn.f32 %0, %1, %2, %0;\n\t}"
      : "+f"(acc)
      : "f"(v), "f"(x), "r"((unsigned)on));
  return acc;
}

// FullWarp: every lane of the warp calls this together, once per row (the
// TMA pipeline's consumers); the remainder then issues only as many FMAs as
// the warp's longest remainder needs, behind warp-uniform guards, so a warp
// of rows with 7 entries (4 + 3) issues 7 FMAs per row, not 8.
template <int B = kGatherBatch, bool FullWarp = false, class ColAt, class ValAt, class XAt>
__device__ __forceinline__ auto row_sum_batched(int a, int e, ColAt&& col_at, ValAt&& val_at, XAt&& x)
    -> decltype(gather_at(x, 0)) {
  using T = decltype(gather_at(x, 0));
  T acc = T(0);
  int k0 = a;
  for (; k0 + B <= e; k0 += B) {
    int c[B];
    T v[B], xv[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      c[j] = col_at(k0 + j);
      v[j] = val_at(k0 + j);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) xv[j] = gather_at(x, c[j]);
#pragma unroll
    for (int j = 0; j < B; ++j) acc = fma(v[j], xv[j], acc);
  }
  const int rem = e - k0;  // 0 .. B-1
  // every lane reaches this once (after its own main loop)
  const int rmax = FullWarp ? __reduce_max_sync(0xffffffffu, rem) : B - 1;
  if (rem > 0) {
    int c[B];
    T v[B], xv[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      v[j] = T(0);
      xv[j] = T(0);
      if (j < rem) {
        c[j] = col_at(k0 + j);
        v[j] = val_at(k0 + j);
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (j < rem) xv[j] = gather_at(x, c[j]);
    // predicated, and (FullWarp) no further than the warp's longest
    // remainder: the FP64 pipe must not see the padding entries
#pragma unroll
    for (int j = 0; j < B - 1; ++j) {
      if (j >= rmax) break;
      acc = fma_if(j < rem, v[j], xv[j], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------------
// Rows of a CSR matrix, one thread per row (grid-stride), each row's gathers
// batched (row_sum_batched); calls epi(row, y_row, aux_row).  No staging and
// no pipeline: with 256-thread blocks at up to 8 per SM, the many rows in
// flight hide the gather latency, which makes this the faster SpMV below a
// few million rows (a tile pipeline pays one gather latency per tile per
// block, and at 1-2 M rows a block owns only a handful of tiles), and as
// fast at 16.7 M rows (3D 7-point: 298 vs 299 us).
// ------------------------------------------------------------------------
template <int B = kGatherBatch, class V, class XAt, class AuxAt, class Epi>
__device__ __forceinline__ void csr_rows(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                         const V* __restrict__ val, XAt x, AuxAt aux, Epi&& epi) {
  using X = decltype(gather_at(x, 0));
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const auto av = aux_at(aux, i);
    const int a = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
    const X s = row_sum_batched<B>(
        a, e, [&](int k) { return __ldg(col + k); }, [&](int k) { return as_x<X>(__ldg(val + k)); }, x);
    epi(i, s, av);
  }
}

// Threads per block of the row-per-thread SpMV kernels, and the size at or
// below which the solvers use them instead of the TMA tile pipeline.
constexpr int kRowThreads = 256;
constexpr long long kRowsKernelMaxN = 4LL << 20;

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
  double val[kTileCap];   // doubles as reduction scratch between tiles
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
      s = block_sum<kTileThreads>(s, sm.val);
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
      const double s = row_sum_batched(
          s0, s1, [&](int k) { return sm.col[k]; }, [&](int k) { return sm.val[k]; }, x);
      epi(r0 + row, s);
    }
    __syncthreads();
    a = b;
  }
}

// Row i of A times v, summed sequentially from global memory.
__device__ __forceinline__ double row_dot(const int* __restrict__ rowptr,
                                          const int* __restrict__ col,
                                          const double* __restrict__ val,
                                          const double* __restrict__ v, int i) {
  const int a = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
  double s = 0.0;
  for (int k = a; k < e; ++k) s = fma(__ldg(val + k), __ldg(v + __ldg(col + k)), s);
  return s;
}

// Host helpers shared by the solvers (defined in sla_cg.cu).
int occupancy(const void* fn, int threads, size_t smem = 0);
cudaError_t add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                       cudaGraphNode_t* out, const void* fn, int grid, int block, void** args,
                       unsigned smem = 0);
int write_info(sla_info* info, sla_info v, cudaStream_t s);
// allowed_flags: the SLA_FLAG_* bits the entry point accepts.
int validate_solve_args(const sla_csr* A, const double* val, const double* b, const double* x,
                        const sla_opts* o, const sla_info* info, const void* ws, size_t ws_bytes,
                        size_t need, int allowed_flags = SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP);

// Device-wide exclusive scan of int32 (sla_pattern.cu): tmp needs
// scan_tmp_ints(n) ints; *total (device, may be null) receives the sum.
long long scan_tmp_ints(long long n);
int device_exclusive_scan(const int* in, long long n, int* out, int* tmp, int* total, cudaStream_t s);

// SpMV kernel family chosen once per process: the TMA-pipelined tiles
// (default) or the register-staged tiles (environment SLA_SPMV_KERNEL=tile).
// SpMV scheme of a solve with n rows: kSpmvRows (one thread per row) for
// n <= kRowsKernelMaxN, else kSpmvTma; SLA_SPMV_KERNEL=tile|tma|rows forces one.
enum : int { kSpmvTile = 0, kSpmvTma = 1, kSpmvRows = 2 };
int spmv_kind(long long n);

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
