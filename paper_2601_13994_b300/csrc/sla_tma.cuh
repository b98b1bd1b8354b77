// sla_tma.cuh -- TMA-pipelined CSR row tiles (sm_100+ bulk copies).
//
// A persistent block owns tiles blockIdx.x, blockIdx.x + G, ...  One producer
// warp streams each 256-row tile's row pointers, column indices and values
// from HBM into a ring of kStages shared-memory stages with cp.async.bulk
// (the 1-D TMA path), completing on an mbarrier with a byte count.  Eight
// consumer warps then sum one row per thread from shared memory (one FP64
// FMA per entry, no shuffles) and release the stage on a second mbarrier.
// The producer runs up to kStages tiles ahead without registers or extra
// threads; its 32 lanes load the row bounds of 32 tiles at once, so a tile
// costs it no global round trip.
//
// (A warp-specialised variant -- separate gather warps storing x[col[k]]
// into shared memory for the FMA warps -- was measured 1.3x slower at
// 16.7 M rows: each stage then waits for two latencies in sequence, and the
// extra 16 KB per stage leaves one block per SM.)
//
// Bulk copies need 16-byte aligned addresses and sizes: the copied entry
// range is widened down/up to multiples of 4 (int32) / 16 bytes (values) but
// never past the end of the arrays; entries outside the copied window (the
// array tail) and tiles that do not fit a stage (too many entries, the last
// partial tile, or misaligned base pointers) are read from global memory
// directly, one warp per row.
//
// Every mbarrier wait is bounded by a clock64 budget (about 2 s at the
// highest clock); a wait that runs out sets *err and the warp leaves its
// loop, and the producer waits (bounded) for its copies still in flight
// before it leaves, so the kernel always terminates with no copy pending.
#pragma once

#include "sla_internal.cuh"

namespace sla {
namespace tma {

constexpr int kRows = 256;                  // rows per tile == consumer threads
constexpr int kCap = 2048;                  // entries per stage
// Two stages and four blocks per SM: measured (3D 7-point, 16.7 M rows) 299
// against 362 us per SpMV for four stages and two blocks per SM -- the
// extra resident consumer warps hide the gather latency better than deeper
// prefetch does; the copy ring still holds ~200 KB per SM.
constexpr int kStages = 2;
constexpr int kConsumerWarps = kRows / kWarp;
constexpr int kThreads = kRows + kWarp;     // + one producer warp
constexpr int kMinBlocks = 4;
constexpr int kPairBatch = 8;               // entries per gather batch of a row pair
constexpr long long kWaitBudgetCycles = 4000000000LL;

// Matrix values are FP64, or FP32 for factors whose values carry no more
// (the learned G); FP32 values are widened to FP64 exactly with integer bit
// operations (to_f64), since a hardware conversion would occupy the FP64
// pipe, the scarce unit on this part.
template <class V, int RPT = 1>
struct StageT {
  int rp[kRows * RPT];       // rowptr[r0 .. r0 + 256 RPT)
  int col[kCap + 8];         // entries [ka_c, kb_c)
  V val[kCap + 8];           // entries [ka_v, kb_v)
  int hdr[8];                // mode, k1, ka_c, kb_c, ka_v, kb_v, r0, nr
};

template <class V, int RPT = 1>
struct SmemT {
  StageT<V, RPT> st[kStages];
  unsigned long long full[kStages];
  unsigned long long empty[kStages];
  double red[2 * kThreads + 2];  // block_sums of up to two values
  bool last;
};

using Stage = StageT<double>;
using Smem = SmemT<double>;
constexpr size_t kSmemBytes = sizeof(Smem);
constexpr size_t kSmemBytesF32 = sizeof(SmemT<float>);
constexpr size_t kSmemBytesF32x2 = sizeof(SmemT<float, 2>);
static_assert(kMinBlocks * kSmemBytes <= 232448, "TMA pipeline stages exceed the shared memory of an SM");

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and *err set) if
// the budget ran out.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitBudgetCycles) {
      atomicOr(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Row `row` of the matrix from global memory by one warp (lane-strided
// entries, fixed butterfly); result valid in every lane.
template <class V, class XAt>
__device__ __forceinline__ auto warp_row(const int* __restrict__ rowptr, const int* __restrict__ col,
                                         const V* __restrict__ val, XAt&& x, int row, int lane)
    -> decltype(gather_at(x, 0)) {
  using X = decltype(gather_at(x, 0));
  const int a = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
  X s = X(0);
  for (int k = a + lane; k < e; k += kWarp) s = fma(as_x<X>(__ldg(val + k)), gather_at(x, __ldg(col + k)), s);
  return warp_sum_any(s);
}

// Sums of two adjacent rows whose entries are [a, m) and [m, e): the column
// indices and values of up to kPairBatch entries of the pair are read first, their x
// gathers issued back to back, then each row's FMAs run in entry order as
// predicated instructions (no padding FMA reaches the FP64 pipe); pairs
// with more entries continue one entry at a time.
template <class X, class ColAt, class ValAt, class XAt>
__device__ __forceinline__ void two_row_sum(int a, int m, int e, ColAt&& col_at, ValAt&& val_at, XAt&& x,
                                            X& acc0, X& acc1) {
  constexpr int B = kPairBatch;
  acc0 = X(0);
  acc1 = X(0);
  const int cnt = e - a;
  int c[B];
  X v[B], xv[B];
#pragma unroll
  for (int j = 0; j < B; ++j) {
    v[j] = X(0);
    xv[j] = X(0);
    if (j < cnt) {
      c[j] = col_at(a + j);
      v[j] = val_at(a + j);
    }
  }
#pragma unroll
  for (int j = 0; j < B; ++j)
    if (j < cnt) xv[j] = gather_at(x, c[j]);
  const int n0 = m - a;  // entries of the first row
  // predicated (fma_if): no padding FMA reaches the FP64 pipe
#pragma unroll
  for (int jj = 0; jj < B; ++jj) acc0 = fma_if(jj < n0 && jj < cnt, v[jj], xv[jj], acc0);
  for (int k = a + B; k < m; ++k) acc0 = fma(val_at(k), gather_at(x, col_at(k)), acc0);
#pragma unroll
  for (int jj = 0; jj < B; ++jj) acc1 = fma_if(jj >= n0 && jj < cnt, v[jj], xv[jj], acc1);
  for (int k = max(m, a + B); k < e; ++k) acc1 = fma(val_at(k), gather_at(x, col_at(k)), acc1);
}

// Runs the pipelined tile loop over all rows (tiles of 256 RPT rows, RPT
// adjacent rows per consumer thread); x is an array or a functor of the
// column (gather_at), aux an array or a functor of the row (aux_at); calls
// epi(row, y_row, aux_row)
// once per row from exactly one consumer thread, where aux_row = aux[row]
// (prefetched before the row's gathers; 0 when aux is null; any element
// type).  The sum y_row
// is formed in the type X of x: FP64, or FP32 (values V = float) for a
// preconditioner applied in single precision.  Must be called
// by all kThreads threads of the block, with `sm` in dynamic shared memory.
// The producer warp returns from this function as soon as its copies have
// landed; nothing after the call may rely on its values.
template <int RPT = 1, class V, class Mat, class XAt, class AuxAt, class Epi>
__device__ __forceinline__ void spmv_pipeline_m(const Mat& mat, XAt x, AuxAt aux, SmemT<V, RPT>& sm, int* err,
                                                Epi&& epi) {
  using X = decltype(gather_at(x, 0));
  const int n = mat.n(), nnz = mat.nnz();
  static_assert(RPT == 1 || RPT == 2, "one or two rows per consumer thread");
  constexpr int kVE = 16 / (int)sizeof(V);  // values per 16 bytes
  constexpr int kTR = kRows * RPT;          // rows per tile
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int ntiles = (n + kTR - 1) / kTR;
  const bool aligned = ((reinterpret_cast<uintptr_t>(mat.rowptr()) | reinterpret_cast<uintptr_t>(mat.col()) |
                         reinterpret_cast<uintptr_t>(mat.val())) & 15u) == 0;
  if (warp == kConsumerWarps) {
    // ---------------- producer warp
    // The row-pointer bounds of the next 32 tiles are loaded by the 32 lanes
    // at once; lane 0 then waits for free stages and issues the bulk copies.
    const int nnz_c = nnz & ~3, nnz_v = nnz & ~(kVE - 1);
    int k = 0;
    bool ok = true;
    for (int tb = blockIdx.x; tb < ntiles && ok; tb += 32 * gridDim.x) {
      const int tl = tb + lane * gridDim.x;
      int k0l = 0, k1l = 0;
      if (tl < ntiles) {
        const int r0 = tl * kTR;
        k0l = __ldg(mat.rowptr() + r0);
        k1l = __ldg(mat.rowptr() + r0 + min(kTR, n - r0));
      }
      for (int j = 0; j < 32; ++j) {
        const int t = tb + j * gridDim.x;
        if (t >= ntiles) break;
        const int k0 = __shfl_sync(0xffffffffu, k0l, j);
        const int k1 = __shfl_sync(0xffffffffu, k1l, j);
        int good = 1;
        if (lane == 0) {
          const int s = k % kStages;
          const unsigned round = (unsigned)(k / kStages);
          if (!mbar_wait(&sm.empty[s], (round & 1u) ^ 1u, err)) {
            good = 0;
          } else {
            StageT<V, RPT>& S = sm.st[s];
            const int r0 = t * kTR;
            const int nr = min(kTR, n - r0);
            int mode = 1;
            int ka_c = 0, kb_c = 0, ka_v = 0, kb_v = 0;
            if (aligned && nr == kTR && k1 - k0 <= kCap) {
              mode = 0;
              ka_c = k0 & ~3;
              kb_c = min((k1 + 3) & ~3, nnz_c);
              if (kb_c < ka_c) kb_c = ka_c;
              ka_v = k0 & ~(kVE - 1);
              kb_v = min((k1 + kVE - 1) & ~(kVE - 1), nnz_v);
              if (kb_v < ka_v) kb_v = ka_v;
            }
            S.hdr[0] = mode;
            S.hdr[1] = k1;
            S.hdr[2] = ka_c;
            S.hdr[3] = kb_c;
            S.hdr[4] = ka_v;
            S.hdr[5] = kb_v;
            S.hdr[6] = r0;
            S.hdr[7] = nr;
            if (mode == 0) {
              const unsigned bc = (unsigned)(kb_c - ka_c) * 4u;
              const unsigned bv = (unsigned)(kb_v - ka_v) * (unsigned)sizeof(V);
              mbar_arrive_expect_tx(&sm.full[s], (unsigned)(kTR * 4) + bc + bv);
              bulk_g2s(S.rp, mat.rowptr() + r0, kTR * 4, &sm.full[s]);
              if (bc) bulk_g2s(S.col, mat.col() + ka_c, bc, &sm.full[s]);
              if (bv) bulk_g2s(S.val, mat.val() + ka_v, bv, &sm.full[s]);
            } else {
              mbar_arrive(&sm.full[s]);
            }
          }
        }
        if (!__shfl_sync(0xffffffffu, good, 0)) {
          ok = false;
          break;
        }
        ++k;
      }
    }
    // Drain: the last (up to kStages) stages filled may still have copies in
    // flight if the consumers gave up; wait for them before leaving.
    if (lane == 0) {
      for (int kk = max(0, k - kStages); kk < k; ++kk)
        if (!mbar_wait(&sm.full[kk % kStages], (unsigned)(kk / kStages) & 1u, err)) break;
    }
    __syncwarp();
    return;
  }
  // ---------------- consumer warps
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int s = k % kStages;
    const unsigned round = (unsigned)(k / kStages);
    if (!mbar_wait(&sm.full[s], round & 1u, err)) break;
    const StageT<V, RPT>& S = sm.st[s];
    const int mode = S.hdr[0];
    const int r0 = S.hdr[6], nr = S.hdr[7];
    if (mode == 0) {
      const int k1 = S.hdr[1], ka_c = S.hdr[2], kb_c = S.hdr[3], ka_v = S.hdr[4], kb_v = S.hdr[5];
      auto col_at = [&](int kk) { return kk < kb_c ? S.col[kk - ka_c] : __ldg(mat.col() + kk); };
      auto val_at = [&](int kk) { return as_x<X>(kk < kb_v ? S.val[kk - ka_v] : __ldg(mat.val() + kk)); };
      if constexpr (RPT == 1) {
        const auto av = aux_at(aux, r0 + tid);
        const int a = S.rp[tid];
        const int e = (tid + 1 < kRows) ? S.rp[tid + 1] : k1;
        // every consumer lane sums one row of the tile: whole warps
        const X acc = row_sum_batched<kGatherBatch, true>(a, e, col_at, val_at, x);
        epi(r0 + tid, acc, av);
      } else {
        const int i0 = 2 * tid;
        const auto av0 = aux_at(aux, r0 + i0);
        const auto av1 = aux_at(aux, r0 + i0 + 1);
        const int a = S.rp[i0], m = S.rp[i0 + 1];
        const int e = (i0 + 2 < kTR) ? S.rp[i0 + 2] : k1;
        X acc0, acc1;
        two_row_sum(a, m, e, col_at, val_at, x, acc0, acc1);
        epi(r0 + i0, acc0, av0);
        epi(r0 + i0 + 1, acc1, av1);
      }
    } else {
      for (int rr = warp; rr < nr; rr += kConsumerWarps) {
        const X acc = warp_row(mat.rowptr(), mat.col(), mat.val(), x, r0 + rr, lane);
        if (lane == 0) epi(r0 + rr, acc, aux_at(aux, r0 + rr));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[s]);
  }
}


// The matrix of a pipeline by value: for kernels that receive it as launch
// parameters (the standalone SpMV), where the fields cost no registers.
template <class V>
struct MatByValue {
  int n_, nnz_;
  const int* rp_;
  const int* c_;
  const V* v_;
  __device__ __forceinline__ int n() const { return n_; }
  __device__ __forceinline__ int nnz() const { return nnz_; }
  __device__ __forceinline__ const int* rowptr() const { return rp_; }
  __device__ __forceinline__ const int* col() const { return c_; }
  __device__ __forceinline__ const V* val() const { return v_; }
};

// The matrix of a pipeline read from a small shared-memory record at every
// use, for kernels that find it in a device-side descriptor (one captured
// graph serves every call): loaded from device memory, the pointers would
// stay live in registers through the whole tile loop although only the
// producer and the rare fallback paths use them; the volatile shared loads
// keep them out of the loop's registers.  With this record the PCG kernel
// K1 (SpMV + p.q) fits the 56 registers of four blocks per SM without
// spilling.
struct MatRecord {
  int n, nnz;
  const int* rowptr;
  const int* col;
  const void* val;
};

template <class V>
struct MatShared {
  const volatile MatRecord* r;
  __device__ __forceinline__ int n() const { return r->n; }
  __device__ __forceinline__ int nnz() const { return r->nnz; }
  __device__ __forceinline__ const int* rowptr() const { return r->rowptr; }
  __device__ __forceinline__ const int* col() const { return r->col; }
  __device__ __forceinline__ const V* val() const { return (const V*)r->val; }
};

template <int RPT = 1, class V, class XAt, class AuxAt, class Epi>
__device__ __forceinline__ void spmv_pipeline(int n, int nnz, const int* __restrict__ rowptr,
                                              const int* __restrict__ col,
                                              const V* __restrict__ val, XAt x, AuxAt aux,
                                              SmemT<V, RPT>& sm, int* err, Epi&& epi) {
  spmv_pipeline_m<RPT, V>(MatByValue<V>{n, nnz, rowptr, col, val}, x, aux, sm, err, epi);
}

}  // namespace tma
}  // namespace sla
