// sla_spmv.cu -- CSR SpMV y = A x (the inner product of every Krylov step;
// Algorithm 1 step 3a).
//
// Bandwidth-bound: per call it moves 12 bytes per stored entry (int32 column
// + float64 value), 4 bytes per row pointer, and 8 + 8 bytes per row for x
// (read once if the gathers hit in cache) and y.  One FP64 FMA per entry.
#include "sla_internal.cuh"
#include "sla_tma.cuh"

namespace sla {

// Persistent grid over row tiles: block b takes tiles b, b + G, b + 2G, ...
// so that at any moment the active tiles form one contiguous window of rows
// and the x entries they gather stay hot in L2.
__global__ void __launch_bounds__(kTileThreads)
spmv_tiles_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                  const double* __restrict__ val, const double* __restrict__ x,
                  double* __restrict__ y) {
  __shared__ TileSmem sm;
  const int ntiles = (n + kTileRows - 1) / kTileRows;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
    spmv_tile(t, n, rowptr, col, val, x, sm, [&](int row, double s) { y[row] = s; });
}

// Wait-budget flag of the TMA kernel (set only if a bounded wait ran out).
__device__ int g_spmv_err = 0;

__global__ void __launch_bounds__(tma::kThreads, tma::kMinBlocks)
spmv_tma_kernel(int n, int nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                const double* __restrict__ val, const double* __restrict__ x,
                double* __restrict__ y) {
  extern __shared__ __align__(128) unsigned char dsm[];
  tma::Smem& sm = *reinterpret_cast<tma::Smem*>(dsm);
  tma::spmv_pipeline(n, nnz, rowptr, col, val, x, (const double*)nullptr, sm, &g_spmv_err,
                     [&](int row, double s, double) { y[row] = s; });
}

// One thread per row (csr_rows): the scheme for n <= kRowsKernelMaxN.
__global__ void __launch_bounds__(kRowThreads)
spmv_rows_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                 const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
  csr_rows(n, rowptr, col, val, x, (const double*)nullptr, [&](int row, double s, double) { y[row] = s; });
}

int spmv_tma_blocks_per_sm() {
  static int v = 0;
  if (v == 0) {
    cudaFuncSetAttribute(spmv_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma::kSmemBytes);
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, spmv_tma_kernel, tma::kThreads,
                                                      tma::kSmemBytes) != cudaSuccess || b <= 0)
      b = 1;
    v = b;
  }
  return v;
}

int spmv_blocks_per_sm() {
  static int v = 0;
  if (v == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, spmv_tiles_kernel, kTileThreads, 0) !=
            cudaSuccess || b <= 0)
      b = 4;
    v = b;
  }
  return v;
}

int launch_spmv(int n, int nnz, const int* rowptr, const int* col, const double* val, const double* x,
                double* y, cudaStream_t s) {
  if (n == 0) return SLA_OK;
  const int dev = current_device();
  const int ntiles = (n + kTileRows - 1) / kTileRows;
  const int kind = spmv_kind(n);
  if (kind == kSpmvRows) {
    static int occ = 0;
    if (occ == 0) occ = occupancy((const void*)spmv_rows_kernel, kRowThreads);
    const int grid = persistent_grid(dev, ((long long)n + kRowThreads - 1) / kRowThreads, occ < 8 ? occ : 8, 1 << 20);
    spmv_rows_kernel<<<grid, kRowThreads, 0, s>>>(n, rowptr, col, val, x, y);
  } else if (kind == kSpmvTma) {
    const int grid = persistent_grid(dev, ntiles, spmv_tma_blocks_per_sm(), 1 << 20);
    spmv_tma_kernel<<<grid, tma::kThreads, tma::kSmemBytes, s>>>(n, nnz, rowptr, col, val, x, y);
  } else {
    const int grid = persistent_grid(dev, ntiles, spmv_blocks_per_sm(), 1 << 20);
    spmv_tiles_kernel<<<grid, kTileThreads, 0, s>>>(n, rowptr, col, val, x, y);
  }
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

}  // namespace sla

extern "C" int32_t sla_spmv(const sla_csr* A, const double* val, const double* x, double* y,
                            void* stream) {
  if (A == nullptr || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n > 0 && (A->rowptr == nullptr || x == nullptr || y == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || val == nullptr)) return SLA_ERR_INVALID;
  if (A->n > 0 && x == y) return SLA_ERR_INVALID;
  return sla::launch_spmv(A->n, A->nnz, A->rowptr, A->col, val, x, y, (cudaStream_t)stream);
}
