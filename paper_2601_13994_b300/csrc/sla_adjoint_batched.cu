// sla_adjoint_batched.cu -- the linear adjoint backward (Eq. 2-3) for every
// system of a batch (Sec. 3.1: a SparseTensor batch on one pattern, or a
// SparseTensorList of distinct patterns).
//
// System s has its own Jacobian A_s, so its backward pass is its own adjoint
// solve A_s^T lambda_s = dL/dx_s followed by dL/db_s = lambda_s and
// dL/d(A_s)_ij = -lambda_s,i x_s,j.  All systems' adjoint solves go into ONE
// batched launch (the forward's persistent batched CG on the A_s when they
// are symmetric, else its batched BiCGStab on the transposed patterns with
// every system's values gathered once), and the gradients of all systems
// into one more kernel; nothing is synchronised on the host.
#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

int launch_gather_values(long long nnz, const int* perm, const double* val, double* out,
                         cudaStream_t s);
int bicg_batched_precheck(const sla_opts* opts, int config, bool list);

namespace {

// The checks both layouts share: method, options, and the aliasing rule of
// sla_adjoint_backward over the whole batch (rows = total rows, nnz = total
// entries).
int check_adjoint_args(int method, const sla_opts* opts, long long rows, long long nnz, const double* x,
                       const double* grad_x, const double* grad_b, const double* grad_val) {
  if (method != SLA_ADJ_CG && method != SLA_ADJ_BICGSTAB) return SLA_ERR_INVALID;
  if (opts == nullptr || opts->flags != 0) return SLA_ERR_INVALID;
  if (x == nullptr || grad_x == nullptr || grad_b == nullptr) return SLA_ERR_INVALID;
  if (nnz > 0 && grad_val == nullptr) return SLA_ERR_INVALID;
  const size_t vb = 8 * (size_t)rows, eb = 8 * (size_t)nnz;
  // lambda is written into grad_b by the solve that reads grad_x, and the
  // gradient pass then reads grad_b and x while it writes grad_val
  if (ranges_overlap(grad_b, vb, x, vb) || ranges_overlap(grad_b, vb, grad_x, vb) ||
      ranges_overlap(grad_val, eb, x, vb) || ranges_overlap(grad_val, eb, grad_b, vb))
    return SLA_ERR_INVALID;
  return SLA_OK;
}

}  // namespace
}  // namespace sla

using namespace sla;

extern "C" int32_t sla_adjoint_backward_batched_shared(const sla_csr* A, const sla_csr_t* AT, int32_t batch,
                                                       const double* val, const double* x,
                                                       const double* grad_x, double* grad_b,
                                                       double* grad_val, int32_t method,
                                                       const sla_opts* opts, sla_info* info, int32_t config,
                                                       void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || batch < 0 || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (batch == 0) return (method == SLA_ADJ_CG || method == SLA_ADJ_BICGSTAB) ? SLA_OK : SLA_ERR_INVALID;
  const long long rows = (long long)batch * A->n, nnz = (long long)batch * A->nnz;
  int rc = check_adjoint_args(method, opts, rows, nnz, x, grad_x, grad_b, grad_val);
  if (rc != SLA_OK) return rc;
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < adjoint_batched_ws_bytes(rows, nnz))
    return SLA_ERR_WORKSPACE;
  sla_opts o = *opts;
  o.use_x0 = 0;
  const size_t solve_ws = al256(batched_ws_bytes(rows));
  if (method == SLA_ADJ_CG) {
    // A_s^T = A_s: the forward batched CG solves the adjoint systems as they stand
    rc = sla_cg_batched_shared(A, batch, val, grad_x, grad_b, &o, info, config, ws, solve_ws, stream);
  } else {
    if (AT == nullptr || AT->rowptr_t == nullptr ||
        (A->nnz > 0 && (AT->col_t == nullptr || AT->perm_t == nullptr || val == nullptr)))
      return SLA_ERR_INVALID;
    if (A->n == 0 || info == nullptr || bicg_batched_precheck(&o, config, false) != SLA_OK)
      return SLA_ERR_INVALID;
    // every system's A_s^T values, after the batched solve's scratch
    double* valT = (double*)((char*)ws + solve_ws);
    rc = sla_gather_values_batched(batch, A->nnz, AT->perm_t, val, valT, stream);
    if (rc != SLA_OK) return rc;
    const sla_csr At{A->n, A->nnz, AT->rowptr_t, AT->col_t};
    rc = sla_bicgstab_batched_shared(&At, batch, valT, grad_x, grad_b, &o, info, config, ws, solve_ws,
                                     stream);
  }
  if (rc != SLA_OK) return rc;
  // dL/d(A_s)_ij = -lambda_s,i x_s,j with lambda = grad_b
  if (A->nnz == 0) return SLA_OK;
  return sla_grad_values_batched(batch, 1, A->n, A->nnz, A->rowptr, A->col, nullptr, nullptr, grad_b, x,
                                 grad_val, stream);
}

extern "C" int32_t sla_adjoint_backward_batched_list(int32_t batch, int32_t n_max, int32_t total_rows,
                                                     int32_t total_nnz, const int32_t* n_off,
                                                     const int32_t* nnz_off, const int32_t* rowptr,
                                                     const int32_t* col, const int32_t* rowptr_t,
                                                     const int32_t* col_t, const int32_t* perm_t,
                                                     const double* val, const double* x, const double* grad_x,
                                                     double* grad_b, double* grad_val, const int32_t* order,
                                                     int32_t method, const sla_opts* opts, sla_info* info,
                                                     int32_t config, void* ws, size_t ws_bytes, void* stream) {
  if (batch < 0 || n_max < 0 || total_rows < 0 || total_nnz < 0) return SLA_ERR_INVALID;
  if (batch == 0) return (method == SLA_ADJ_CG || method == SLA_ADJ_BICGSTAB) ? SLA_OK : SLA_ERR_INVALID;
  int rc = check_adjoint_args(method, opts, total_rows, total_nnz, x, grad_x, grad_b, grad_val);
  if (rc != SLA_OK) return rc;
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < adjoint_batched_ws_bytes(total_rows, total_nnz))
    return SLA_ERR_WORKSPACE;
  sla_opts o = *opts;
  o.use_x0 = 0;
  const size_t solve_ws = al256(batched_ws_bytes(total_rows));
  if (method == SLA_ADJ_CG) {
    rc = sla_cg_batched_list(batch, n_max, total_rows, n_off, nnz_off, rowptr, col, val, grad_x, grad_b, order,
                             &o, info, config, ws, solve_ws, stream);
  } else {
    if (rowptr_t == nullptr || (total_nnz > 0 && (col_t == nullptr || perm_t == nullptr || val == nullptr)))
      return SLA_ERR_INVALID;
    if (n_off == nullptr || nnz_off == nullptr || info == nullptr ||
        bicg_batched_precheck(&o, config, true) != SLA_OK)
      return SLA_ERR_INVALID;
    double* valT = (double*)((char*)ws + solve_ws);
    rc = launch_gather_values(total_nnz, perm_t, val, valT, (cudaStream_t)stream);
    if (rc != SLA_OK) return rc;
    rc = sla_bicgstab_batched_list(batch, n_max, total_rows, n_off, nnz_off, rowptr_t, col_t, valT, grad_x,
                                   grad_b, order, &o, info, config, ws, solve_ws, stream);
  }
  if (rc != SLA_OK) return rc;
  if (n_max == 0 || total_nnz == 0) return SLA_OK;
  return sla_grad_values_batched(batch, 0, n_max, 0, rowptr, col, n_off, nnz_off, grad_b, x, grad_val, stream);
}
