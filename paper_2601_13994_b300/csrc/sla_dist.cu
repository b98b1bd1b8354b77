// sla_dist.cu -- the distributed layer of Sec. 3.3 (row-block partition,
// halo exchange H and its transpose, all-reduced inner products; Algorithm 1
// of App. C), with its P partitions emulated on one GPU.
//
// Partition p owns the rows [row_off[p], row_off[p+1]) and stores A[O_p, :]
// with its columns renumbered into an extended local space: first its own
// |O_p| entries, then its halo H_p (the sorted global columns outside O_p
// that its rows reference).  All partitions' extended vectors are laid out
// back to back (partition p's at ext_off[p]); src[e] is the global index
// that extended entry e holds.  With every partition in one device memory:
//   H   (forward halo exchange, Eq. 5): x_ext[e] = x[src[e]] -- owned
//       entries copy, halo entries receive the owners' values;
//   H^T (transposed exchange, Eq. 6): g_x[i] = g_ext[own(i)] + the halo
//       gradients of every partition that holds i, summed in a fixed order
//       (partition, then halo position) -- summation at the receive site;
//   the local SpMVs of all partitions are one SpMV of the concatenated
//   local matrices (n rows, columns in the extended space);
//   an all-reduce is a fixed-order sum over partitions of per-partition
//   partial sums (each itself a fixed-shape reduction).
// One kernel runs each step over all partitions' data; no partition ever
// waits for another inside a kernel.
#include <cmath>

#include "sla_internal.cuh"

namespace sla {
namespace {

constexpr int kDT = 256;        // threads per block
constexpr int kDotBlocks = 8;   // blocks per partition in the partial dots
constexpr int kDotMaxK = 3;     // pairs per call

__global__ void halo_gather_kernel(long long total_ext, const int* __restrict__ src,
                                   const double* __restrict__ x, double* __restrict__ x_ext) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total_ext; e += stride)
    x_ext[e] = x[__ldg(src + e)];
}

__global__ void halo_scatter_kernel(int n, const int* __restrict__ own_pos, const int* __restrict__ hptr,
                                    const int* __restrict__ hlist, const double* __restrict__ g_ext,
                                    double* __restrict__ g_x) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double s = g_ext[__ldg(own_pos + i)];
    for (int t = __ldg(hptr + i); t < __ldg(hptr + i + 1); ++t) s += g_ext[__ldg(hlist + t)];
    g_x[i] = s;
  }
}

struct DotArgs {
  const double* a[kDotMaxK];
  const double* b[kDotMaxK];
};

// Block (g, p) sums a_j . b_j over rows row_off[p] + g*kDT + t, stride
// kDotBlocks*kDT, of partition p; partial[(p * kDotBlocks + g) * K + j].
template <int K>
__global__ void __launch_bounds__(kDT) dist_dots_kernel(const int* __restrict__ row_off, DotArgs args,
                                                        double* __restrict__ partial) {
  __shared__ double red[K * kDT + K];
  const int p = blockIdx.y, g = blockIdx.x;
  const int o0 = row_off[p], o1 = row_off[p + 1];
  double acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0;
  for (int i = o0 + g * kDT + threadIdx.x; i < o1; i += kDotBlocks * kDT) {
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fma(args.a[j][i], args.b[j][i], acc[j]);
  }
  block_sums<kDT, K>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) partial[(p * kDotBlocks + g) * K + j] = acc[j];
  }
}

// The all-reduce: per partition the kDotBlocks partials in block order (the
// rank's local sum), then the ranks in order 0..P-1.  out[j] = total j,
// rank_part[j * P + p] = rank p's local sum j.
template <int K>
__global__ void dist_allreduce_kernel(int P, const double* __restrict__ partial, double* __restrict__ out,
                                      double* __restrict__ rank_part) {
  if (threadIdx.x >= K) return;
  const int j = threadIdx.x;
  double tot = 0.0;
  for (int p = 0; p < P; ++p) {
    double s = 0.0;
    for (int g = 0; g < kDotBlocks; ++g) s += partial[(p * kDotBlocks + g) * K + j];
    if (rank_part) rank_part[j * P + p] = s;
    tot += s;
  }
  out[j] = tot;
}

// D^{-1} from the owned diagonal entries (extended column own(i) in row i);
// *bad = 1 if some A_ii <= 0.
__global__ void dist_diag_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col_ext,
                                 const double* __restrict__ val, const int* __restrict__ own_pos,
                                 double* __restrict__ dinv, int* bad) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int own = __ldg(own_pos + i);
    double d = 0.0;
    for (int k = __ldg(rowptr + i); k < __ldg(rowptr + i + 1); ++k)
      if (__ldg(col_ext + k) == own) d += __ldg(val + k);
    if (!(d > 0.0)) atomicOr(bad, 1);
    dinv[i] = 1.0 / d;
  }
}

// Algorithm 1 step 3c-d with the Jacobi preconditioner: x += alpha p,
// r -= alpha q, z = D^{-1} r.
__global__ void dist_cg_update_kernel(int n, double alpha, const double* __restrict__ p,
                                      const double* __restrict__ q, const double* __restrict__ dinv,
                                      double* __restrict__ x, double* __restrict__ r, double* __restrict__ z) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    z[i] = dinv[i] * ri;
  }
}

// Algorithm 1 step 3f: p = z + beta p.
__global__ void dist_cg_direction_kernel(int n, double beta, const double* __restrict__ z, double* __restrict__ p) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = fma(beta, p[i], z[i]);
}

// r = b - y, z = D^{-1} r, p = z (a start or restart; y = A x).
__global__ void dist_cg_start_kernel(int n, const double* __restrict__ b, const double* __restrict__ y,
                                     const double* __restrict__ dinv, double* __restrict__ r,
                                     double* __restrict__ z, double* __restrict__ p) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double ri = b[i] - y[i];
    const double zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = zi;
  }
}

// out[k] = g_y[i] * x_ext[col_ext[k]] for the entries k of row i: the value
// gradient of y = A_local x_ext (no communication).
__global__ void dist_outer_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col_ext,
                                  const double* __restrict__ gy, const double* __restrict__ x_ext,
                                  double* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double g = gy[i];
    for (int k = __ldg(rowptr + i); k < __ldg(rowptr + i + 1); ++k) out[k] = g * x_ext[__ldg(col_ext + k)];
  }
}

int grid_for_rows(long long n) {
  return persistent_grid(current_device(), (n + kDT - 1) / kDT, 8, 1 << 20);
}

}  // namespace
}  // namespace sla

using namespace sla;

extern "C" int32_t sla_dist_halo_gather(int64_t total_ext, const int32_t* src, const double* x, double* x_ext,
                                        void* stream) {
  if (total_ext < 0) return SLA_ERR_INVALID;
  if (total_ext == 0) return SLA_OK;
  if (src == nullptr || x == nullptr || x_ext == nullptr || (const void*)x == (const void*)x_ext)
    return SLA_ERR_INVALID;
  halo_gather_kernel<<<grid_for_rows(total_ext), kDT, 0, (cudaStream_t)stream>>>(total_ext, src, x, x_ext);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_halo_scatter(int32_t n, const int32_t* own_pos, const int32_t* hptr,
                                         const int32_t* hlist, const double* g_ext, double* g_x, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (own_pos == nullptr || hptr == nullptr || g_ext == nullptr || g_x == nullptr ||
      (const void*)g_ext == (const void*)g_x)
    return SLA_ERR_INVALID;
  halo_scatter_kernel<<<grid_for_rows(n), kDT, 0, (cudaStream_t)stream>>>(n, own_pos, hptr, hlist, g_ext, g_x);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_dots(int32_t P, const int32_t* row_off, int32_t k, const double* const* a,
                                 const double* const* b, double* partial, double* out, double* rank_part,
                                 void* stream) {
  if (P < 1 || P > 65535 || k < 1 || k > kDotMaxK || row_off == nullptr || a == nullptr || b == nullptr ||
      partial == nullptr || out == nullptr)
    return SLA_ERR_INVALID;
  DotArgs args{};
  for (int j = 0; j < k; ++j) {
    if (a[j] == nullptr || b[j] == nullptr) return SLA_ERR_INVALID;
    args.a[j] = a[j];
    args.b[j] = b[j];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid(kDotBlocks, (unsigned)P);
  switch (k) {
    case 1:
      dist_dots_kernel<1><<<grid, kDT, 0, s>>>(row_off, args, partial);
      dist_allreduce_kernel<1><<<1, 32, 0, s>>>(P, partial, out, rank_part);
      break;
    case 2:
      dist_dots_kernel<2><<<grid, kDT, 0, s>>>(row_off, args, partial);
      dist_allreduce_kernel<2><<<1, 32, 0, s>>>(P, partial, out, rank_part);
      break;
    default:
      dist_dots_kernel<3><<<grid, kDT, 0, s>>>(row_off, args, partial);
      dist_allreduce_kernel<3><<<1, 32, 0, s>>>(P, partial, out, rank_part);
      break;
  }
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_diag_inv(int32_t n, const int32_t* rowptr, const int32_t* col_ext, const double* val,
                                     const int32_t* own_pos, double* dinv, int32_t* bad, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (rowptr == nullptr || col_ext == nullptr || val == nullptr || own_pos == nullptr || dinv == nullptr ||
      bad == nullptr)
    return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  SLA_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  dist_diag_kernel<<<grid_for_rows(n), kDT, 0, s>>>(n, rowptr, col_ext, val, own_pos, dinv, bad);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_cg_start(int32_t n, const double* b, const double* y, const double* dinv, double* r,
                                     double* z, double* p, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (b == nullptr || y == nullptr || dinv == nullptr || r == nullptr || z == nullptr || p == nullptr)
    return SLA_ERR_INVALID;
  dist_cg_start_kernel<<<grid_for_rows(n), kDT, 0, (cudaStream_t)stream>>>(n, b, y, dinv, r, z, p);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_cg_update(int32_t n, double alpha, const double* p, const double* q, const double* dinv,
                                      double* x, double* r, double* z, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (p == nullptr || q == nullptr || dinv == nullptr || x == nullptr || r == nullptr || z == nullptr)
    return SLA_ERR_INVALID;
  dist_cg_update_kernel<<<grid_for_rows(n), kDT, 0, (cudaStream_t)stream>>>(n, alpha, p, q, dinv, x, r, z);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_cg_direction(int32_t n, double beta, const double* z, double* p, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (z == nullptr || p == nullptr) return SLA_ERR_INVALID;
  dist_cg_direction_kernel<<<grid_for_rows(n), kDT, 0, (cudaStream_t)stream>>>(n, beta, z, p);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

extern "C" int32_t sla_dist_outer_values(int32_t n, const int32_t* rowptr, const int32_t* col_ext,
                                         const double* gy, const double* x_ext, double* out, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (rowptr == nullptr || col_ext == nullptr || gy == nullptr || x_ext == nullptr || out == nullptr)
    return SLA_ERR_INVALID;
  dist_outer_kernel<<<grid_for_rows(n), kDT, 0, (cudaStream_t)stream>>>(n, rowptr, col_ext, gy, x_ext, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
