// sla_common.cu -- library information, device-property cache, workspace
// size query and CSR pattern validation.
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

namespace {
std::mutex g_dev_mu;
int g_sms[64] = {0};
}  // namespace

int current_device() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int spmv_kind(long long n) {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("SLA_SPMV_KERNEL");
    forced = -1;
    if (e != nullptr) {
      if (strcmp(e, "tile") == 0) forced = kSpmvTile;
      else if (strcmp(e, "tma") == 0) forced = kSpmvTma;
      else if (strcmp(e, "rows") == 0) forced = kSpmvRows;
    }
  }
  if (forced >= 0) return forced;
  return n <= kRowsKernelMaxN ? kSpmvRows : kSpmvTma;
}

int num_sms(int device) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (device < 0 || device >= 64) return 148;
  if (g_sms[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
      v = 148;
    g_sms[device] = v;
  }
  return g_sms[device];
}

// Pattern validation: one thread per row, every load bounds-checked.
__global__ void csr_check_kernel(int n, int nnz, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, int* ok) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int a = rowptr[i], b = rowptr[i + 1];
    bool good = (a >= 0) && (b >= a) && (b <= nnz);
    if (i == 0 && a != 0) good = false;
    if (i == n - 1 && b != nnz) good = false;
    if (good) {
      int prev = -1;
      for (int k = a; k < b; ++k) {
        const int c = col[k];
        if (c < 0 || c >= n || c <= prev) {
          good = false;
          break;
        }
        prev = c;
      }
    }
    if (!good) atomicAnd(ok, 0);
  }
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

}  // namespace sla

using namespace sla;

extern "C" {

const char* sla_version(void) { return "sla-b300 0.1.0 (sm_103a)"; }

const char* sla_status_string(int32_t code) {
  switch (code) {
    case SLA_OK: return "OK";
    case SLA_NOT_CONVERGED: return "NOT_CONVERGED";
    case SLA_BREAKDOWN: return "BREAKDOWN";
    case SLA_NOT_SPD: return "NOT_SPD";
    case SLA_ERR_INVALID: return "ERR_INVALID";
    case SLA_ERR_CUDA: return "ERR_CUDA";
    case SLA_ERR_WORKSPACE: return "ERR_WORKSPACE";
    case SLA_ERR_TIMEOUT: return "ERR_TIMEOUT";
    default: return "UNKNOWN";
  }
}

int32_t sla_workspace_size(int32_t kind, int32_t n, int32_t nnz, int32_t batch, size_t* bytes) {
  if (bytes == nullptr || n < 0 || nnz < 0 || batch < 0) return SLA_ERR_INVALID;
  size_t b = 0;
  if (!sla::workspace_bytes(kind, n, nnz, batch, &b)) return SLA_ERR_INVALID;
  *bytes = b;
  return SLA_OK;
}

int32_t sla_csr_check(const sla_csr* A, int32_t* ok, void* stream) {
  if (A == nullptr || ok == nullptr || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n > 0 && A->rowptr == nullptr) return SLA_ERR_INVALID;
  if (A->nnz > 0 && A->col == nullptr) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  set_int_kernel<<<1, 1, 0, s>>>(ok, 1);
  if (A->n > 0) {
    const int dev = current_device();
    const int grid = persistent_grid(dev, (A->n + 255) / 256, 8, 1 << 16);
    csr_check_kernel<<<grid, 256, 0, s>>>(A->n, A->nnz, A->rowptr, A->col, ok);
  }
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}

}  // extern "C"
