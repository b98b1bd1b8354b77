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

// FP64 FMA throughput probe: kFp64Chains independent FMA chains per thread
// (enough in flight to keep the pipe busy at full occupancy), each step
// y <- y * m + c with |m| < 1 so the values stay bounded; the chains' sum is
// written only if it equals an impossible value, so the work cannot be
// dropped.
constexpr int kFp64Chains = 8;
constexpr int kFp64Threads = 256;

__global__ void __launch_bounds__(kFp64Threads) fp64_probe_kernel(int iters, double* out) {
  double y[kFp64Chains];
  const double m = 0.999999, c = 1e-7;
#pragma unroll
  for (int k = 0; k < kFp64Chains; ++k) y[k] = 1.0 + 1e-3 * k + 1e-9 * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kFp64Chains; ++k) y[k] = fma(y[k], m, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < kFp64Chains; ++k) sum += y[k];
  if (sum == -1.0) out[0] = sum;
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

extern "C" int32_t sla_fp64_probe(int32_t iters, int32_t blocks_per_sm, double* out, int64_t* flops, void* stream) {
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || out == nullptr || flops == nullptr)
    return SLA_ERR_INVALID;
  const int grid = sla::num_sms(sla::current_device()) * blocks_per_sm;
  sla::fp64_probe_kernel<<<grid, sla::kFp64Threads, 0, (cudaStream_t)stream>>>(iters, out);
  SLA_CUDA_TRY(cudaGetLastError());
  *flops = 2LL * sla::kFp64Chains * iters * (long long)grid * sla::kFp64Threads;
  return SLA_OK;
}
