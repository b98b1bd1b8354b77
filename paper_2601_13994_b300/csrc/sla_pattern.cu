// sla_pattern.cu -- sparsity-pattern utilities.
//
//  * sla_csr_transpose: CSR of A^T with a permutation into A's values, so
//    that valT = val[permT] (the adjoint A^T lambda = dL/dx of Eq. 3 needs
//    A^T for nonsymmetric A).  Stable: inside a row of A^T the entries keep
//    increasing source row.
//  * sla_coo_to_csr: the COO input of SparseTensor(val, row, col, shape)
//    (App. B) sorted by (row, col), duplicates summed in increasing COO
//    index, plus perm[e] = CSR slot of COO entry e (to return gradients in
//    the caller's order).
//
// Both are built on a stable LSD radix sort of (uint32 key, uint32 value)
// pairs and a device-wide exclusive scan, written here; every result is
// deterministic (integer work, or sums in a fixed order).
#include <vector>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {
namespace {

// ------------------------------------------------------------------ scan
constexpr int kScanT = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanT * kScanItems;

__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total) {
  // sh: kScanT ints.  Hillis-Steele over the block (integers: exact).
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < kScanT; o <<= 1) {
    const int a = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  const int incl = sh[t];
  *total = sh[kScanT - 1];
  __syncthreads();
  return incl - v;
}

// per-tile sums of in[0..n)
__global__ void __launch_bounds__(kScanT) scan_reduce_kernel(const int* __restrict__ in, long long n,
                                                             int* __restrict__ tile_sum) {
  __shared__ int sh[kScanT];
  const long long base = (long long)blockIdx.x * kScanTile;
  int s = 0;
  for (int j = 0; j < kScanItems; ++j) {
    const long long i = base + (long long)j * kScanT + threadIdx.x;
    if (i < n) s += in[i];
  }
  int total;
  block_excl_scan(s, sh, &total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// exclusive scan of tile_sum[0..m) in place by one block; *grand = total
__global__ void __launch_bounds__(kScanT) scan_tiles_kernel(int* tile_sum, int m, int* grand) {
  __shared__ int sh[kScanT];
  int carry = 0;
  for (int c0 = 0; c0 < m; c0 += kScanT) {
    const int i = c0 + threadIdx.x;
    const int v = i < m ? tile_sum[i] : 0;
    int total;
    const int ex = block_excl_scan(v, sh, &total);
    if (i < m) tile_sum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0 && grand) *grand = carry;
}

// out[i] = exclusive prefix of in (out may alias in)
__global__ void __launch_bounds__(kScanT) scan_final_kernel(const int* in, long long n,
                                                            const int* __restrict__ tile_off,
                                                            int* out) {
  __shared__ int sh[kScanT];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
  for (int j = 0; j < kScanItems; ++j) {
    const long long i = base + j;
    v[j] = i < n ? in[i] : 0;
    s += v[j];
  }
  int total;
  int run = block_excl_scan(s, sh, &total) + tile_off[blockIdx.x];
  for (int j = 0; j < kScanItems; ++j) {
    const long long i = base + j;
    if (i < n) out[i] = run;
    run += v[j];
  }
}

long long scan_tiles(long long n) { return (n + kScanTile - 1) / kScanTile; }

// Exclusive scan of in[0..n) into out (may alias); *grand (device, may be
// null) receives the total.  tmp needs scan_tiles(n) ints.
int exclusive_scan(const int* in, long long n, int* out, int* tmp, int* grand, cudaStream_t s) {
  const long long tiles = scan_tiles(n);
  if (tiles == 0) {
    if (grand) SLA_CUDA_TRY(cudaMemsetAsync(grand, 0, sizeof(int), s));
    return SLA_OK;
  }
  scan_reduce_kernel<<<(unsigned)tiles, kScanT, 0, s>>>(in, n, tmp);
  scan_tiles_kernel<<<1, kScanT, 0, s>>>(tmp, (int)tiles, grand);
  scan_final_kernel<<<(unsigned)tiles, kScanT, 0, s>>>(in, n, tmp, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsT = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsT * kRsItems;
constexpr int kRsWarps = kRsT / kWarp;

// hist[d * tiles + tile] = count of digit d in the tile
__global__ void __launch_bounds__(kRsT) rs_hist_kernel(const unsigned* __restrict__ keys, long long n,
                                                       int shift, int tiles, int* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kRsTile;
  for (int r = 0; r < kRsItems; ++r) {
    const long long i = base + (long long)r * kRsT + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter.  Items of a tile are taken in rounds (round r holds items
// r*256 + t), so tile order = (round, thread); inside a round, equal digits
// are ranked by lane (match_any) and by warp (per-warp counts).
__global__ void __launch_bounds__(kRsT) rs_scatter_kernel(const unsigned* __restrict__ kin,
                                                          const unsigned* __restrict__ vin,
                                                          long long n, int shift, int tiles,
                                                          const int* __restrict__ off,
                                                          unsigned* __restrict__ kout,
                                                          unsigned* __restrict__ vout) {
  __shared__ int run[256];
  __shared__ int wcnt[kRsWarps][256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  run[t] = 0;
  for (int j = 0; j < kRsWarps; ++j) wcnt[j][t] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kRsTile;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kRsItems; ++r) {
    const long long i = base + (long long)r * kRsT + t;
    const bool valid = i < n;
    unsigned key = 0, val = 0;
    int d = 256;  // invalid items form their own group
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (int)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int lrank = __popc(peers & lt_mask);
    if (valid && lrank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pre = 0;
      for (int j = 0; j < w; ++j) pre += wcnt[j][d];
      const int pos = off[(long long)d * tiles + blockIdx.x] + run[d] + pre + lrank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    int add = 0;
    for (int j = 0; j < kRsWarps; ++j) {
      add += wcnt[j][t];
      wcnt[j][t] = 0;
    }
    run[t] += add;
    __syncthreads();
  }
}

int key_bits(long long max_key) {
  int b = 0;
  while (b < 32 && (max_key >> b) > 0) ++b;
  return b;
}

struct SortBufs {
  unsigned *k0, *v0, *k1, *v1;
  int *hist, *scan_tmp;
};

// Sorts (k0, v0)[0..n) by the low `bits` bits of the keys, stably; returns
// in *kres/*vres the buffers that hold the result (k0/v0 or k1/v1).
int radix_sort(SortBufs& B, long long n, int bits, unsigned** kres, unsigned** vres,
               cudaStream_t s) {
  unsigned *ka = B.k0, *va = B.v0, *kb = B.k1, *vb = B.v1;
  const int tiles = (int)((n + kRsTile - 1) / kRsTile);
  for (int shift = 0; shift < bits && n > 0; shift += 8) {
    rs_hist_kernel<<<tiles, kRsT, 0, s>>>(ka, n, shift, tiles, B.hist);
    int rc = exclusive_scan(B.hist, 256LL * tiles, B.hist, B.scan_tmp, nullptr, s);
    if (rc != SLA_OK) return rc;
    rs_scatter_kernel<<<tiles, kRsT, 0, s>>>(ka, va, n, shift, tiles, B.hist, kb, vb);
    SLA_CUDA_TRY(cudaGetLastError());
    unsigned* t;
    t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  *kres = ka;
  *vres = va;
  return SLA_OK;
}

// ------------------------------------------------------------------ helpers
__global__ void iota_copy_kernel(long long n, const int* __restrict__ key_src, unsigned* keys,
                                 unsigned* vals) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    keys[i] = (unsigned)key_src[i];
    vals[i] = (unsigned)i;
  }
}

// row index of every CSR entry (tile of rows in shared memory, binary search)
__global__ void __launch_bounds__(256) entry_rows_kernel(int n, const int* __restrict__ rowptr,
                                                         unsigned* __restrict__ rows) {
  __shared__ int rp[257];
  const int ntiles = (n + 255) / 256;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * 256, nr = min(256, n - r0);
    for (int i = threadIdx.x; i <= nr; i += 256) rp[i] = rowptr[r0 + i];
    __syncthreads();
    for (int k = rp[0] + threadIdx.x; k < rp[nr]; k += 256) {
      int lo = 0, hi = nr;  // rp[lo] <= k < rp[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rp[mid] <= k) lo = mid;
        else hi = mid;
      }
      rows[k] = (unsigned)(r0 + lo);
    }
    __syncthreads();
  }
}

// ptr[j] = first position p with key[p] >= j, for j in [0, n]; keys sorted
__global__ void boundaries_kernel(long long m, int n, const unsigned* __restrict__ keys, int* ptr) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p <= m; p += stride) {
    const long long lo = p == 0 ? 0 : (long long)keys[p - 1] + 1;
    const long long hi = p == m ? n : (long long)keys[p];
    for (long long j = lo; j <= hi; ++j) ptr[j] = (int)p;
  }
}

__global__ void transpose_finish_kernel(long long nnz, const unsigned* __restrict__ sorted_keys,
                                        const unsigned* __restrict__ sorted_vals,
                                        const unsigned* __restrict__ rows, int* colT, int* permT) {
  (void)sorted_keys;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const unsigned k = sorted_vals[p];
    permT[p] = (int)k;
    colT[p] = (int)rows[k];
  }
}

// COO: keys = column, values = entry index; flags out-of-range entries
__global__ void coo_keys_kernel(long long m, int n, const int64_t* __restrict__ row,
                                const int64_t* __restrict__ col, unsigned* keys, unsigned* vals,
                                int* bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += stride) {
    const long long r = row[e], c = col[e];
    if (r < 0 || r >= n || c < 0 || c >= n) atomicOr(bad, 1);
    keys[e] = (unsigned)min(max((long long)c, 0LL), (long long)n - 1);
    vals[e] = (unsigned)e;
  }
}

// second pass keys: row of the entry now at position p
__global__ void coo_rowkeys_kernel(long long m, int n, const int64_t* __restrict__ row,
                                   const unsigned* __restrict__ order, unsigned* keys) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += stride)
    keys[p] = (unsigned)min(max((long long)row[order[p]], 0LL), (long long)n - 1);
}

// head flags of (row, col) runs in sorted order
__global__ void coo_heads_kernel(long long m, int n, const int64_t* __restrict__ row,
                                 const int64_t* __restrict__ col, const unsigned* __restrict__ order,
                                 int* flag) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += stride) {
    const unsigned e = order[p];
    int f = 1;
    if (p > 0) {
      const unsigned q = order[p - 1];
      f = (row[e] != row[q] || col[e] != col[q]) ? 1 : 0;
    }
    flag[p] = f;
  }
}

// slots[p] = exclusive scan of heads; every run head writes its CSR entry
// (value = sequential sum of the run in sorted order = increasing COO index)
__global__ void coo_emit_kernel(long long m, int n, const int64_t* __restrict__ row,
                                const int64_t* __restrict__ col, const double* __restrict__ val,
                                const unsigned* __restrict__ order, const int* __restrict__ flag,
                                const int* __restrict__ slot_excl, int* col_out, double* val_out,
                                int* perm, int* rowcnt, int* order_out, int* segptr) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m; p += stride) {
    const unsigned e = order[p];
    const int slot = slot_excl[p] + flag[p] - 1;  // inclusive count - 1
    perm[e] = slot;
    if (order_out) order_out[p] = (int)e;
    if (flag[p]) {
      if (segptr) segptr[slot] = (int)p;
      double s = val[e];
      for (long long q = p + 1; q < m && !flag[q]; ++q) s += val[order[q]];
      col_out[slot] = (int)min(max((long long)col[e], 0LL), (long long)n - 1);
      val_out[slot] = s;
      atomicAdd(&rowcnt[min(max((long long)row[e], 0LL), (long long)n - 1)], 1);
    }
  }
}

__global__ void coo_status_kernel(const int* bad, const int* nnz_total, int* nnz_out, int* segptr,
                                  long long m) {
  *nnz_out = *bad ? -1 : *nnz_total;
  if (segptr && !*bad) segptr[*nnz_total] = (int)m;
}

// out[s] = sum of val[idx[q]] for q in [seg[s], seg[s+1]), in increasing q
__global__ void segment_sum_kernel(int nseg, const int* __restrict__ seg, const int* __restrict__ idx,
                                   const double* __restrict__ val, double* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int sg = blockIdx.x * blockDim.x + threadIdx.x; sg < nseg; sg += stride) {
    const int a = seg[sg], e = seg[sg + 1];
    double acc = 0.0;
    for (int q = a; q < e; ++q) acc += __ldg(val + __ldg(idx + q));
    out[sg] = acc;
  }
}

// ---------------------------------------------- transpose of a pattern list
// The list (per-system row pointers back to back, local columns, offsets
// n_off / nnz_off) is the block-diagonal matrix whose global column of a
// local entry (s, i, c) is n_off[s] + c.  Sorting all entries by that key
// (stably) gives each system's transposed entries, in order, exactly in the
// system's own entry range [nnz_off[s], nnz_off[s+1]): every key of system s
// lies in [n_off[s], n_off[s+1]).

// system of global position p, given offsets off[0..batch] (off[batch] > p)
__device__ __forceinline__ int list_system(const int* __restrict__ off, int batch, long long p) {
  int lo = 0, hi = batch;  // off[lo] <= p < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= p) lo = mid;
    else hi = mid;
  }
  return lo;
}

// keys = global column, vals = global entry index, rows = global row
__global__ void list_keys_kernel(int batch, int total_rows, const int* __restrict__ n_off,
                                 const int* __restrict__ nnz_off, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, unsigned* keys, unsigned* vals,
                                 unsigned* rows) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total_rows; g += stride) {
    const int s = list_system(n_off, batch, g);
    const int n0 = n_off[s], e0 = nnz_off[s];
    const int* rp = rowptr + n0 + s;
    const int i = (int)(g - n0);
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      keys[e0 + k] = (unsigned)(n0 + col[e0 + k]);
      vals[e0 + k] = (unsigned)(e0 + k);
      rows[e0 + k] = (unsigned)g;
    }
  }
}

// list-layout row pointers of the transposes from the global boundaries
// ptr[0..total_rows]: row j of system s starts at ptr[n_off[s] + j] - nnz_off[s]
__global__ void list_rowptr_kernel(int batch, int total_rows, const int* __restrict__ n_off,
                                   const int* __restrict__ nnz_off, const int* __restrict__ ptr,
                                   int* rowptrT) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total_rows; g += stride) {
    const int s = list_system(n_off, batch, g);
    rowptrT[g + s] = ptr[g] - nnz_off[s];
  }
  // each system's closing entry (its entry count; the only entry of an empty system)
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < batch; s += stride)
    rowptrT[n_off[s + 1] + s] = nnz_off[s + 1] - nnz_off[s];
}

__global__ void list_finish_kernel(int batch, long long nnz, const int* __restrict__ n_off,
                                   const int* __restrict__ nnz_off, const unsigned* __restrict__ sorted_vals,
                                   const unsigned* __restrict__ rows, int* colT, int* permT) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int s = list_system(nnz_off, batch, p);
    const unsigned k = sorted_vals[p];
    permT[p] = (int)k;
    colT[p] = (int)rows[k] - n_off[s];
  }
}

int grid_for(long long n) {
  return persistent_grid(current_device(), (n + 255) / 256, 8, 1 << 20);
}

// ------------------------------------------------------------------ layouts
struct PatternLayout {
  size_t k0, v0, k1, v1, hist, scan_tmp, extra, misc, total;
};

PatternLayout pattern_layout(long long m, int n) {
  PatternLayout L{};
  const size_t e4 = al256(4 * (size_t)(m > 0 ? m : 1));
  const long long tiles = (m + kRsTile - 1) / kRsTile;
  const long long hist_n = 256 * (tiles > 0 ? tiles : 1);
  const long long big = hist_n > (long long)m ? hist_n : (long long)m + 1;
  const long long cap = big > (long long)n + 1 ? big : (long long)n + 1;
  size_t o = 0;
  L.k0 = o; o += e4;
  L.v0 = o; o += e4;
  L.k1 = o; o += e4;
  L.v1 = o; o += e4;
  L.hist = o; o += al256(4 * (size_t)hist_n);
  L.scan_tmp = o; o += al256(4 * (size_t)(scan_tiles(cap) + 1));
  L.extra = o; o += al256(4 * (size_t)(((long long)n + 1) > m ? (long long)n + 1 : m));
  L.misc = o; o += 256;
  L.total = o;
  return L;
}

}  // namespace

size_t transpose_ws_bytes(int n, int nnz) { return pattern_layout(nnz, n).total; }

// list transpose: the transpose layout over all entries + the global boundaries
size_t list_transpose_ws_bytes(int total_rows, int total_nnz) {
  return pattern_layout(total_nnz, total_rows).total + al256(4 * ((size_t)(total_rows > 0 ? total_rows : 0) + 1));
}

long long scan_tmp_ints(long long n) { return scan_tiles(n) + 1; }

int device_exclusive_scan(const int* in, long long n, int* out, int* tmp, int* total, cudaStream_t s) {
  return exclusive_scan(in, n, out, tmp, total, s);
}
size_t coo_ws_bytes(int n, long long m) { return pattern_layout(m, n).total; }

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_csr_transpose(const sla_csr* A, int32_t* rowptrT, int32_t* colT,
                                     int32_t* permT, void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  const int n = A->n, nnz = A->nnz;
  if (n > 0 && (A->rowptr == nullptr || rowptrT == nullptr)) return SLA_ERR_INVALID;
  if (nnz > 0 && (A->col == nullptr || colT == nullptr || permT == nullptr)) return SLA_ERR_INVALID;
  const PatternLayout L = pattern_layout(nnz, n);
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < L.total) return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  if (nnz == 0) {
    if (n >= 0 && rowptrT) SLA_CUDA_TRY(cudaMemsetAsync(rowptrT, 0, sizeof(int) * ((size_t)n + 1), s));
    return SLA_OK;
  }
  SortBufs B{(unsigned*)(base + L.k0), (unsigned*)(base + L.v0), (unsigned*)(base + L.k1),
             (unsigned*)(base + L.v1), (int*)(base + L.hist), (int*)(base + L.scan_tmp)};
  iota_copy_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, A->col, B.k0, B.v0);
  unsigned *ks, *vs;
  int rc = radix_sort(B, nnz, key_bits(n > 0 ? n - 1 : 0), &ks, &vs, s);
  if (rc != SLA_OK) return rc;
  boundaries_kernel<<<grid_for(nnz + 1), 256, 0, s>>>(nnz, n, ks, rowptrT);
  unsigned* rows = (unsigned*)(base + L.extra);
  entry_rows_kernel<<<grid_for(n), 256, 0, s>>>(n, A->rowptr, rows);
  transpose_finish_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, ks, vs, rows, colT, permT);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_csr_list_transpose(int32_t batch, int32_t total_rows, int32_t total_nnz,
                                          const int32_t* n_off, const int32_t* nnz_off,
                                          const int32_t* rowptr, const int32_t* col,
                                          int32_t* rowptrT, int32_t* colT, int32_t* permT,
                                          void* ws, size_t ws_bytes, void* stream) {
  if (batch < 0 || total_rows < 0 || total_nnz < 0) return SLA_ERR_INVALID;
  if (batch == 0) return total_rows == 0 && total_nnz == 0 ? SLA_OK : SLA_ERR_INVALID;
  if (n_off == nullptr || nnz_off == nullptr || rowptr == nullptr || rowptrT == nullptr)
    return SLA_ERR_INVALID;
  if (total_nnz > 0 && (col == nullptr || colT == nullptr || permT == nullptr)) return SLA_ERR_INVALID;
  if ((const void*)rowptr == (const void*)rowptrT || (total_nnz > 0 && (const void*)col == (const void*)colT))
    return SLA_ERR_INVALID;
  const PatternLayout L = pattern_layout(total_nnz, total_rows);
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < list_transpose_ws_bytes(total_rows, total_nnz))
    return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  int* ptr = (int*)(base + L.total);
  SortBufs B{(unsigned*)(base + L.k0), (unsigned*)(base + L.v0), (unsigned*)(base + L.k1),
             (unsigned*)(base + L.v1), (int*)(base + L.hist), (int*)(base + L.scan_tmp)};
  unsigned* rows = (unsigned*)(base + L.extra);
  const unsigned* vs = B.v0;
  if (total_nnz > 0) {
    list_keys_kernel<<<grid_for(total_rows), 256, 0, s>>>(batch, total_rows, n_off, nnz_off, rowptr, col,
                                                           B.k0, B.v0, rows);
    unsigned* ks = nullptr;
    unsigned* vres = nullptr;
    int rc = radix_sort(B, total_nnz, key_bits(total_rows > 0 ? total_rows - 1 : 0), &ks, &vres, s);
    if (rc != SLA_OK) return rc;
    boundaries_kernel<<<grid_for((long long)total_nnz + 1), 256, 0, s>>>(total_nnz, total_rows, ks, ptr);
    vs = vres;
  } else {
    SLA_CUDA_TRY(cudaMemsetAsync(ptr, 0, sizeof(int) * ((size_t)total_rows + 1), s));
  }
  list_rowptr_kernel<<<grid_for((long long)total_rows + batch), 256, 0, s>>>(batch, total_rows, n_off,
                                                                              nnz_off, ptr, rowptrT);
  if (total_nnz > 0)
    list_finish_kernel<<<grid_for(total_nnz), 256, 0, s>>>(batch, total_nnz, n_off, nnz_off, vs, rows,
                                                            colT, permT);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_segment_sum(int32_t nseg, const int32_t* segptr, const int32_t* idx,
                                   const double* val, double* out, void* stream) {
  if (nseg < 0) return SLA_ERR_INVALID;
  if (nseg > 0 && (segptr == nullptr || idx == nullptr || val == nullptr || out == nullptr))
    return SLA_ERR_INVALID;
  if (nseg == 0) return SLA_OK;
  segment_sum_kernel<<<grid_for(nseg), 256, 0, (cudaStream_t)stream>>>(nseg, segptr, idx, val, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_coo_to_csr(int32_t n, int64_t m, const int64_t* row, const int64_t* col,
                                  const double* val, int32_t* rowptr, int32_t* col_out,
                                  double* val_out, int32_t* perm, int32_t* order, int32_t* segptr,
                                  int32_t* nnz_out, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || m < 0 || m > 0x7fffffffLL || nnz_out == nullptr || rowptr == nullptr)
    return SLA_ERR_INVALID;
  if (m > 0 && (row == nullptr || col == nullptr || val == nullptr || col_out == nullptr ||
                val_out == nullptr || perm == nullptr))
    return SLA_ERR_INVALID;
  if (m > 0 && n == 0) return SLA_ERR_INVALID;
  const PatternLayout L = pattern_layout(m, n);
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < L.total) return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  int* bad = (int*)(base + L.misc);
  int* total = bad + 1;
  SLA_CUDA_TRY(cudaMemsetAsync(bad, 0, 2 * sizeof(int), s));
  int* rowcnt = (int*)(base + L.extra);  // n + 1 counters, scanned into rowptr
  SLA_CUDA_TRY(cudaMemsetAsync(rowcnt, 0, sizeof(int) * ((size_t)n + 1), s));
  if (m > 0) {
    SortBufs B{(unsigned*)(base + L.k0), (unsigned*)(base + L.v0), (unsigned*)(base + L.k1),
               (unsigned*)(base + L.v1), (int*)(base + L.hist), (int*)(base + L.scan_tmp)};
    const int bits = key_bits(n - 1);
    coo_keys_kernel<<<grid_for(m), 256, 0, s>>>(m, n, row, col, B.k0, B.v0, bad);
    unsigned *ks, *vs;
    int rc = radix_sort(B, m, bits, &ks, &vs, s);  // by column
    if (rc != SLA_OK) return rc;
    // second sort by row, stable: keys into the free pair, values = order
    SortBufs B2 = B;
    if (ks == B.k0) {
      B2.k0 = B.k1; B2.v0 = vs; B2.k1 = B.k0; B2.v1 = B.v1;
    } else {
      B2.k0 = B.k0; B2.v0 = vs; B2.k1 = B.k1; B2.v1 = B.v0;
    }
    coo_rowkeys_kernel<<<grid_for(m), 256, 0, s>>>(m, n, row, vs, B2.k0);
    unsigned *ks2, *sorted;
    rc = radix_sort(B2, m, bits, &ks2, &sorted, s);
    const unsigned* order_sorted = sorted;
    if (rc != SLA_OK) return rc;
    // heads and slots: flag in the free key buffer, its scan in the other
    int* flag = (int*)(ks2 == B2.k0 ? B2.k1 : B2.k0);
    int* slot = (int*)ks2;  // keys no longer needed
    if (segptr) SLA_CUDA_TRY(cudaMemsetAsync(segptr, 0, sizeof(int), s));
    coo_heads_kernel<<<grid_for(m), 256, 0, s>>>(m, n, row, col, order_sorted, flag);
    rc = exclusive_scan(flag, m, slot, (int*)(base + L.scan_tmp), total, s);
    if (rc != SLA_OK) return rc;
    coo_emit_kernel<<<grid_for(m), 256, 0, s>>>(m, n, row, col, val, order_sorted, flag, slot,
                                                col_out, val_out, perm, rowcnt, order, segptr);
  }
  int rc = exclusive_scan(rowcnt, (long long)n + 1, rowptr, (int*)(base + L.scan_tmp), nullptr, s);
  if (rc != SLA_OK) return rc;
  coo_status_kernel<<<1, 1, 0, s>>>(bad, total, nnz_out, segptr, m);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

// ---------------------------------------------------------------------------
// Distance-2 column colouring (host).  Two columns that share a row get
// different colours, so that one Jacobian-vector product per colour -- with
// the tangent equal to 1 on the colour's columns -- recovers every entry of
// a sparse Jacobian with this pattern (Curtis, Powell and Reid, 1974): entry
// (i, j) is component i of the product for colour(j).  Greedy in increasing
// column order, each column taking the smallest colour that no column
// sharing a row with it has yet.  O(sum over rows of length^2) work.
// ---------------------------------------------------------------------------
extern "C" int32_t sla_colour_columns(int32_t n, const int32_t* rowptr, const int32_t* col,
                                      int32_t* colour, int32_t* ncolours) {
  if (n < 0 || ncolours == nullptr) return SLA_ERR_INVALID;
  *ncolours = 0;
  if (n == 0) return SLA_OK;
  if (rowptr == nullptr || colour == nullptr || rowptr[0] != 0) return SLA_ERR_INVALID;
  for (int32_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return SLA_ERR_INVALID;
  const int32_t nnz = rowptr[n];
  if (nnz > 0 && col == nullptr) return SLA_ERR_INVALID;
  for (int32_t k = 0; k < nnz; ++k)
    if (col[k] < 0 || col[k] >= n) return SLA_ERR_INVALID;
  // rows of each column (the pattern of A^T), by counting sort
  std::vector<int32_t> cptr((size_t)n + 1, 0), crow((size_t)(nnz > 0 ? nnz : 1));
  for (int32_t k = 0; k < nnz; ++k) ++cptr[(size_t)col[k] + 1];
  for (int32_t j = 0; j < n; ++j) cptr[(size_t)j + 1] += cptr[j];
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int32_t i = 0; i < n; ++i)
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) crow[(size_t)fill[col[k]]++] = i;
  }
  // mark[c] == j + 1: colour c is taken by a column sharing a row with j
  std::vector<int32_t> mark;
  int32_t used = 0;
  for (int32_t j = 0; j < n; ++j) colour[j] = -1;
  for (int32_t j = 0; j < n; ++j) {
    for (int32_t q = cptr[j]; q < cptr[(size_t)j + 1]; ++q) {
      const int32_t i = crow[q];
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int32_t c = colour[col[k]];
        if (c >= 0) mark[c] = j + 1;
      }
    }
    int32_t c = 0;
    while (c < used && mark[c] == j + 1) ++c;
    if (c == used) {
      ++used;
      mark.push_back(0);
    }
    colour[j] = c;
  }
  *ncolours = used;
  return SLA_OK;
}
