// sla_adjoint.cu -- the linear adjoint backward (Eq. 2-3).
//
// With residual F(x, A, b) = A x - b the Jacobian is A, so the backward pass
// of x = A^{-1} b is one adjoint solve A^T lambda = dL/dx followed by
//   dL/db = lambda,   dL/dA_ij = -lambda_i x_j  on the stored pattern.
// The solve reuses the forward solvers: CG on A itself when A is symmetric
// (A^T = A), BiCGStab on the explicit CSR of A^T otherwise (its values
// gathered once per call as valT = val[permT]).  The gradient assembly is one
// coalesced pass over the entries.
#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

int launch_cg(const KrylovDesc& desc, void* ws, cudaStream_t s, int flags, bool allow_graph = true);
int launch_bicgstab(const KrylovDesc& desc, void* ws, cudaStream_t s, int flags);
KrylovDesc make_desc(const sla_csr* A, const double* val, const double* b, double* x,
                     const sla_opts* o, sla_info* info);

namespace {

constexpr int kGT = 256;          // rows per tile == threads

// grad_val[k] = -lambda[row(k)] * x[col[k]].  A block takes 256-row tiles;
// the tile's row pointers sit in shared memory and every entry finds its row
// by binary search there, so the entry loop is coalesced in k.
__global__ void __launch_bounds__(kGT) grad_values_kernel(int n, const int* __restrict__ rowptr,
                                                          const int* __restrict__ col,
                                                          const double* __restrict__ lambda,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ grad_val) {
  __shared__ int rp[kGT + 1];
  const int ntiles = (n + kGT - 1) / kGT;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int r0 = t * kGT;
    const int nr = min(kGT, n - r0);
    for (int i = threadIdx.x; i <= nr; i += kGT) rp[i] = __ldg(rowptr + r0 + i);
    __syncthreads();
    const int k0 = rp[0], k1 = rp[nr];
    for (int k = k0 + threadIdx.x; k < k1; k += kGT) {
      // the row r with rp[r] <= k < rp[r+1] (empty rows cannot satisfy it)
      int lo = 0, hi = nr;  // invariant: rp[lo] <= k < rp[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rp[mid] <= k) lo = mid;
        else hi = mid;
      }
      grad_val[k] = -__ldg(lambda + r0 + lo) * __ldg(x + __ldg(col + k));
    }
    __syncthreads();
  }
}

__global__ void gather_values_kernel(long long nnz, const int* __restrict__ perm,
                                     const double* __restrict__ val, double* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += stride)
    out[k] = __ldg(val + __ldg(perm + k));
}

}  // namespace

int launch_grad_values(int n, const int* rowptr, const int* col, const double* lambda,
                       const double* x, double* grad_val, cudaStream_t s) {
  if (n == 0) return SLA_OK;
  const int dev = current_device();
  const int grid = persistent_grid(dev, (n + kGT - 1) / kGT, 8, 1 << 20);
  grad_values_kernel<<<grid, kGT, 0, s>>>(n, rowptr, col, lambda, x, grad_val);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

int launch_gather_values(long long nnz, const int* perm, const double* val, double* out,
                         cudaStream_t s) {
  if (nnz == 0) return SLA_OK;
  const int dev = current_device();
  const int grid = persistent_grid(dev, (nnz + 255) / 256, 8, 1 << 20);
  gather_values_kernel<<<grid, 256, 0, s>>>(nnz, perm, val, out);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_grad_values(const sla_csr* A, const double* lambda, const double* x,
                                   double* grad_val, void* stream) {
  if (A == nullptr || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n > 0 && (A->rowptr == nullptr || lambda == nullptr || x == nullptr)) return SLA_ERR_INVALID;
  if (A->nnz > 0 && (A->col == nullptr || grad_val == nullptr)) return SLA_ERR_INVALID;
  return launch_grad_values(A->n, A->rowptr, A->col, lambda, x, grad_val, (cudaStream_t)stream);
}

extern "C" int32_t sla_gather_values(int64_t nnz, const int32_t* perm, const double* val,
                                     double* out, void* stream) {
  if (nnz < 0) return SLA_ERR_INVALID;
  if (nnz > 0 && (perm == nullptr || val == nullptr || out == nullptr)) return SLA_ERR_INVALID;
  return launch_gather_values(nnz, perm, val, out, (cudaStream_t)stream);
}

extern "C" int32_t sla_adjoint_backward(const sla_csr* A, const sla_csr_t* AT, const double* val,
                                        const double* x, const double* grad_x, double* grad_b,
                                        double* grad_val, int32_t method, const sla_opts* opts,
                                        sla_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || opts == nullptr) return SLA_ERR_INVALID;
  if (method != SLA_ADJ_CG && method != SLA_ADJ_BICGSTAB) return SLA_ERR_INVALID;
  const int n = A->n, nnz = A->nnz;
  if (n > 0 && x == nullptr) return SLA_ERR_INVALID;
  if (nnz > 0 && grad_val == nullptr) return SLA_ERR_INVALID;
  // the adjoint solve writes lambda into grad_b before the gradient pass
  // reads x, so grad_b must not alias x; grad_val must overlap neither
  if (n > 0 && (const void*)grad_b == (const void*)x) return SLA_ERR_INVALID;
  if (n > 0 && nnz > 0 &&
      (ranges_overlap(grad_val, 8 * (size_t)nnz, x, 8 * (size_t)n) ||
       ranges_overlap(grad_val, 8 * (size_t)nnz, grad_b, 8 * (size_t)n)))
    return SLA_ERR_INVALID;
  if (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) return SLA_ERR_INVALID;
  size_t need = 0;
  workspace_bytes(SLA_WS_ADJOINT, n, nnz, 1, &need);
  const int allowed = SLA_FLAG_HOST_LOOP | SLA_FLAG_NO_COOP |
                      (method == SLA_ADJ_CG ? SLA_FLAG_CG_PIPELINED : 0);
  int rc = validate_solve_args(A, val, grad_x, grad_b, opts, info, ws, ws_bytes, need, allowed);
  if (rc != SLA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  sla_opts o = *opts;
  o.use_x0 = 0;
  if (n == 0) return write_info(info, sla_info{0, SLA_OK, 0.0, 0.0}, s);
  if (method == SLA_ADJ_CG) {
    // A^T = A: the forward CG solves the adjoint system as it stands
    rc = launch_cg(make_desc(A, val, grad_x, grad_b, &o, info), ws, s, o.flags);
  } else {
    if (AT == nullptr || AT->rowptr_t == nullptr || (nnz > 0 && (AT->col_t == nullptr ||
                                                                 AT->perm_t == nullptr)))
      return SLA_ERR_INVALID;
    // valT in the workspace, after the BiCGStab scratch
    const size_t off = bicg_ws_bytes(n, nnz);
    double* valT = (double*)((char*)ws + off);
    rc = launch_gather_values(nnz, AT->perm_t, val, valT, s);
    if (rc != SLA_OK) return rc;
    sla_csr At{n, nnz, AT->rowptr_t, AT->col_t};
    rc = launch_bicgstab(make_desc(&At, valT, grad_x, grad_b, &o, info), ws, s, o.flags);
  }
  if (rc != SLA_OK) return rc;
  // dL/dA_ij = -lambda_i x_j, lambda = grad_b
  return launch_grad_values(n, A->rowptr, A->col, grad_b, x, grad_val, s);
}
