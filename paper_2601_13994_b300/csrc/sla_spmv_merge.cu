// sla_spmv_merge.cu -- load-balanced CSR SpMV along the merge path, and the
// row-length statistics that choose between it and the row kernels.
//
// y = A x (Algorithm 1 step 3a) for matrices whose row lengths are very
// uneven (a power-law degree distribution, a dense row): the row-per-thread
// and tile kernels give a row to one thread or one warp, so one long row can
// take as long as the rest of the matrix.  Here the work is the merge of the
// n row ends with the nnz nonzeros (n + nnz items); thread c takes items
// [c IPT, (c + 1) IPT) whatever rows they belong to, so every thread does the
// same work.  A thread finds its start (row, nonzero) by binary search on its
// diagonal of the merge grid, then walks: a nonzero adds val * x[col] to the
// running sum, a row end closes the row.  A row that starts and ends inside
// one thread is written directly.  A row that crosses chunk boundaries leaves
// partial sums: `carry_out` from every chunk in which it is still open at the
// chunk's end, and `carry_end` from the chunk in which it ends; the fix-up
// kernels add them (the run of chunks starts at the chunk holding the row's
// first item, r + rowptr[r]) in a fixed order: one thread per run, one block
// per run longer than 64 chunks.  Results are deterministic;
// rows that cross chunks are summed in a different order than the sequential
// row sum (a partial sum per chunk, then the fixed-order sum of the parts).
#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

constexpr int kMergeIPT = 8;      // merge items per thread
constexpr int kMergeThreads = 256;

// Row index of the merge-path point on diagonal d (the nonzero index is
// d - row): the first row whose end has not been passed by the d items,
// searched in rows [lo, hi].
__device__ __forceinline__ int merge_search(long long d, long long lo, long long hi, int nnz,
                                            const int* __restrict__ rowptr) {
  if (lo < d - nnz) lo = d - nnz;
  if (hi > d) hi = d;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if ((long long)__ldg(rowptr + mid + 1) <= d - mid - 1) lo = mid + 1;
    else hi = mid;
  }
  return (int)lo;
}

// A chunk's nonzeros are consecutive (at most kMergeIPT of them from its
// first nonzero j0), so their columns, values and x entries are loaded
// before the walk, which takes them in order from a shift register; rows
// are closed at their row-end items as before.
__global__ void __launch_bounds__(kMergeThreads)
merge_spmv_kernel(int n, int nnz, long long nchunks, const int* __restrict__ rowptr, const int* __restrict__ col,
                  const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                  double* __restrict__ carry_out, int* __restrict__ carry_out_row, double* __restrict__ carry_end,
                  int* __restrict__ carry_end_row) {
  __shared__ int s_rows[2];
  const long long items = (long long)n + nnz;
  // the block's rows: one search of its first and of its last diagonal
  const long long b0 = (long long)blockIdx.x * kMergeThreads * kMergeIPT;
  if (threadIdx.x < 2) {
    long long db = b0 + (long long)threadIdx.x * kMergeThreads * kMergeIPT;
    if (db > items) db = items;
    s_rows[threadIdx.x] = merge_search(db, 0, n, nnz, rowptr);
  }
  __syncthreads();
  const long long c = (long long)blockIdx.x * kMergeThreads + threadIdx.x;
  if (c >= nchunks) return;
  const long long d0 = c * kMergeIPT;
  const long long d1 = d0 + kMergeIPT < items ? d0 + kMergeIPT : items;
  int i = merge_search(d0, s_rows[0], s_rows[1], nnz, rowptr);
  int j = (int)(d0 - i);
  const int i0 = i;
  const bool first_here = i0 >= n || j == __ldg(rowptr + i0);
  double vv[kMergeIPT], xv[kMergeIPT];
  {
    int cc[kMergeIPT];
#pragma unroll
    for (int u = 0; u < kMergeIPT; ++u) {
      const bool in = j + u < nnz;
      cc[u] = in ? __ldg(col + j + u) : 0;
      vv[u] = in ? __ldg(val + j + u) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kMergeIPT; ++u) xv[u] = j + u < nnz ? __ldg(x + cc[u]) : 0.0;
  }
  int end = i < n ? __ldg(rowptr + i + 1) : nnz;
  double acc = 0.0;
  int cer = -1;
  double ce = 0.0;
  const int steps = (int)(d1 - d0);
#pragma unroll
  for (int t = 0; t < kMergeIPT; ++t) {
    if (t < steps && i < n) {
      if (j < end) {
        acc = fma(vv[0], xv[0], acc);
#pragma unroll
        for (int u = 0; u + 1 < kMergeIPT; ++u) {
          vv[u] = vv[u + 1];
          xv[u] = xv[u + 1];
        }
        ++j;
      } else {
        if (i > i0 || first_here) {
          y[i] = acc;
        } else {
          cer = i;
          ce = acc;
        }
        acc = 0.0;
        ++i;
        end = i < n ? __ldg(rowptr + i + 1) : nnz;
      }
    }
  }
  carry_end_row[c] = cer;
  carry_end[c] = ce;
  // the chunk ends inside row i after consuming some of its entries
  const bool open = i < n && (j > __ldg(rowptr + i));
  carry_out_row[c] = open ? i : -1;
  carry_out[c] = open ? acc : 0.0;
}

// One thread per chunk that ends a row begun in an earlier chunk: the row's
// parts from chunks a .. c-1 (carry_out) and c (carry_end), added left to
// right.  Runs longer than kMergeLongRun chunks are listed for
// merge_fixup_long_kernel instead.
constexpr int kMergeLongRun = 64;

__global__ void __launch_bounds__(kMergeThreads)
merge_fixup_kernel(long long nchunks, const int* __restrict__ rowptr, const double* __restrict__ carry_out,
                   const double* __restrict__ carry_end, const int* __restrict__ carry_end_row,
                   double* __restrict__ y, long long* __restrict__ longs, int* __restrict__ nlong, int cap) {
  const long long c = (long long)blockIdx.x * kMergeThreads + threadIdx.x;
  if (c >= nchunks) return;
  const int r = carry_end_row[c];
  if (r < 0) return;
  const long long a = ((long long)r + __ldg(rowptr + r)) / kMergeIPT;
  if (c - a > kMergeLongRun) {
    const int slot = atomicAdd(nlong, 1);
    if (slot < cap) longs[slot] = c;
    return;
  }
  double s = 0.0;
  for (long long t = a; t < c; ++t) s += carry_out[t];
  y[r] = s + carry_end[c];
}

// One block per long run: the parts summed by the block's threads in a fixed
// stride pattern, then block_sums (same bits whichever block takes the run).
__global__ void __launch_bounds__(kMergeThreads)
merge_fixup_long_kernel(const int* __restrict__ rowptr, const double* __restrict__ carry_out,
                        const double* __restrict__ carry_end, const int* __restrict__ carry_end_row,
                        double* __restrict__ y, const long long* __restrict__ longs, const int* __restrict__ nlong,
                        int cap) {
  __shared__ double red[kMergeThreads + 2];
  const int m = min(*nlong, cap);
  for (int q = blockIdx.x; q < m; q += gridDim.x) {
    const long long c = longs[q];
    const int r = carry_end_row[c];
    const long long a = ((long long)r + __ldg(rowptr + r)) / kMergeIPT;
    double s = 0.0;
    for (long long t = a + threadIdx.x; t < c; t += kMergeThreads) s += carry_out[t];
    s = block_sum<kMergeThreads>(s, red);
    if (threadIdx.x == 0) y[r] = s + carry_end[c];
    __syncthreads();
  }
}

// Longest row and number of rows longer than 1024 entries.
__global__ void row_stats_kernel(int n, const int* __restrict__ rowptr, int* out) {
  int mx = 0, longrows = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int len = __ldg(rowptr + i + 1) - __ldg(rowptr + i);
    mx = max(mx, len);
    longrows += len > 1024;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    longrows += __shfl_xor_sync(0xffffffffu, longrows, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, mx);
    atomicAdd(out + 1, longrows);
  }
}

// Rows whose run is longer than kMergeLongRun chunks fill at least
// kMergeLongRun - 1 whole chunks with their nonzeros: at most
// nnz / ((kMergeLongRun - 1) IPT) of them.
long long merge_long_cap(long long nnz) { return nnz / ((long long)(kMergeLongRun - 1) * kMergeIPT) + 1; }

size_t spmv_merge_ws_bytes(int n, long long nnz) {
  const long long items = (long long)(n > 0 ? n : 0) + (nnz > 0 ? nnz : 0);
  const long long chunks = (items + kMergeIPT - 1) / kMergeIPT;
  const size_t c = (size_t)(chunks > 0 ? chunks : 1);
  return 2 * al256(sizeof(double) * c) + 2 * al256(sizeof(int) * c) + 256 +
         al256(sizeof(long long) * (size_t)merge_long_cap(nnz > 0 ? nnz : 0));
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_spmv_merge(const sla_csr* A, const double* val, const double* x, double* y, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (A == nullptr || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n > 0 && (A->rowptr == nullptr || x == nullptr || y == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if (A->n > 0 && x == y) return SLA_ERR_INVALID;
  if (ws == nullptr || ((uintptr_t)ws & 255u) != 0 || ws_bytes < spmv_merge_ws_bytes(A->n, A->nnz))
    return SLA_ERR_WORKSPACE;
  if (A->n == 0) return SLA_OK;
  const long long items = (long long)A->n + A->nnz;
  const long long chunks = (items + kMergeIPT - 1) / kMergeIPT;
  const size_t cd = al256(sizeof(double) * (size_t)chunks), ci = al256(sizeof(int) * (size_t)chunks);
  char* base = (char*)ws;
  double* carry_out = (double*)base;
  double* carry_end = (double*)(base + cd);
  int* carry_out_row = (int*)(base + 2 * cd);
  int* carry_end_row = (int*)(base + 2 * cd + ci);
  int* nlong = (int*)(base + 2 * cd + 2 * ci);
  long long* longs = (long long*)(base + 2 * cd + 2 * ci + 256);
  const int cap = (int)merge_long_cap(A->nnz);
  cudaStream_t s = (cudaStream_t)stream;
  SLA_CUDA_TRY(cudaMemsetAsync(nlong, 0, sizeof(int), s));
  const long long blocks = (chunks + kMergeThreads - 1) / kMergeThreads;
  merge_spmv_kernel<<<(unsigned)blocks, kMergeThreads, 0, s>>>(A->n, A->nnz, chunks, A->rowptr, A->col, val, x, y,
                                                               carry_out, carry_out_row, carry_end, carry_end_row);
  SLA_CUDA_TRY(cudaGetLastError());
  merge_fixup_kernel<<<(unsigned)blocks, kMergeThreads, 0, s>>>(chunks, A->rowptr, carry_out, carry_end,
                                                                carry_end_row, y, longs, nlong, cap);
  SLA_CUDA_TRY(cudaGetLastError());
  merge_fixup_long_kernel<<<cap < 1024 ? cap : 1024, kMergeThreads, 0, s>>>(A->rowptr, carry_out, carry_end,
                                                                             carry_end_row, y, longs, nlong, cap);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_spmv_scheme(int32_t n, int64_t nnz, int32_t max_row) {
  // sla_spmv gives a row to one thread (n <= 4 Mi rows) or, in an over-full
  // tile, to one warp; its time grows with the longest row at about 0.13 us
  // (thread) or 4 ns (warp) per entry, while the merge path costs about
  // 0.01 ns per item of n + nnz (B300: a 300001-entry row 28.1 ms against
  // 40 us; power-law rows up to 4824 entries 717 against 39 us; 5- and
  // 7-point stencils 15.5 and 42 us against 75 and 175 us).
  const long long items = (long long)(n > 0 ? n : 0) + (nnz > 0 ? nnz : 0);
  const long long per = (long long)n <= kRowsKernelMaxN ? 8192 : 256;
  const long long limit = items / per > 256 ? items / per : 256;
  return (long long)max_row > limit ? SLA_SPMV_MERGE : SLA_SPMV_ROWS;
}

extern "C" int32_t sla_csr_row_stats(const sla_csr* A, int32_t* out, void* stream) {
  if (A == nullptr || A->n < 0 || out == nullptr) return SLA_ERR_INVALID;
  if (A->n > 0 && A->rowptr == nullptr) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  SLA_CUDA_TRY(cudaMemsetAsync(out, 0, 2 * sizeof(int32_t), s));
  if (A->n == 0) return SLA_OK;
  const int grid = persistent_grid(current_device(), ((long long)A->n + 255) / 256, 8, 1 << 16);
  row_stats_kernel<<<grid, 256, 0, s>>>(A->n, A->rowptr, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
