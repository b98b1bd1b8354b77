// sla_mpnn.cu -- kernels of the learned factored preconditioner M^{-1} = G G^T.
//
// The paper lists learned preconditioners as future work with no design
// (Sec. 5).  The design here: a message-passing network over the matrix
// graph, width 32, BF16 weights with FP32 accumulation and activations,
// that predicts G on the pattern of tril(A) in the scaled system
// (G = D^{-1/2} Gt, Gt_ii = exp(theta_ii), Gt_ij = theta_ij), so M stays SPD
// and a zero output layer gives exactly the Jacobi factor D^{-1/2}.
//
// The network is a handful of generic pieces, each with its backward:
//   features      d = diag(A) (FP64), e_k = A_ij / sqrt(d_i d_j), node features
//   tril          CSR of tril(A) + source entry index
//   dense         Y = [X1 | X2] W^T + b (optional relu / residual); dX = dY W;
//                 dW, db as per-block partials reduced in a fixed order
//   aggregate     Agg_i = sum_{j != i} e_ij X_j (also its own transpose for
//                 symmetric A, used by the backward)
//   head          theta per tril entry from [P | Q | R] rows; backward by rows
//                 (dP, dR) and by columns through the transposed pattern (dQ)
//   loss          FP64: (x* - G G^T b)^T A (x* - G G^T b) / (x*^T b) and
//                 dloss/dG_ij = g_i s_j + b_i h_j  (s = G^T b, g = -2 A e / c,
//                 h = G^T g) on the pattern of G
//   adam          FP32 master weights -> BF16 copies
// Every reduction is deterministic (fixed trees, no atomics on values).
#include <cuda_bf16.h>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {
namespace {

constexpr int kW = 32;     // network width
constexpr int kTN = 32;    // nodes per tile of the dense kernels
constexpr int kDT = 256;   // dense kernel block size
constexpr int kMaxK = 64;  // largest input width
constexpr int kMaxM = 96;  // largest output width

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

int grid_rows(long long n, int per_block, int cap = 1 << 16) {
  long long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------ features
__global__ void diag_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                            const double* __restrict__ v, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (c[k] == i) s += v[k];
    d[i] = s;
  }
}

__global__ void feat_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                            const double* __restrict__ v, const double* __restrict__ d,
                            float* __restrict__ e, float* __restrict__ F) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double sa = 0.0, ss = 0.0;
    int deg = 0;
    const double di = d[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = c[k];
      const double ek = v[k] / sqrt(di * d[j]);
      e[k] = (float)ek;
      if (j != i) {
        sa += fabs(ek);
        ss += ek;
        ++deg;
      }
    }
    F[3 * (size_t)i + 0] = (float)sa;
    F[3 * (size_t)i + 1] = (float)ss;
    F[3 * (size_t)i + 2] = (float)deg / 8.0f;
  }
}

// ------------------------------------------------------------ tril pattern
__global__ void tril_count_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                                  int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    int m = 0;
    if (i < n)
      for (int k = rp[i]; k < rp[i + 1]; ++k) m += c[k] <= i;
    cnt[i] = m;
  }
}

__global__ void tril_fill_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                                 const int* __restrict__ grp, int* __restrict__ gcol,
                                 int* __restrict__ gsrc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int pos = grp[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (c[k] <= i) {
        gcol[pos] = c[k];
        gsrc[pos] = k;
        ++pos;
      }
  }
}

// ------------------------------------------------------------ dense
// Y[i, m] = b[m] + sum_k [X1 | X2][i, k] W[m, k]; Ypre = that (optional);
// Y = (relu ? max(0, .) : .) + R[i, m] (optional).
__global__ void __launch_bounds__(kDT) dense_fwd_kernel(int n, int K1, const float* __restrict__ X1,
                                                        int K2, const float* __restrict__ X2, int M,
                                                        const __nv_bfloat16* __restrict__ W,
                                                        const float* __restrict__ bias,
                                                        const float* __restrict__ R, int relu,
                                                        float* __restrict__ Ypre,
                                                        float* __restrict__ Y) {
  __shared__ float WsT[kMaxK * kMaxM];  // [k][m]
  __shared__ float Xs[kTN * kMaxK];
  const int K = K1 + K2;
  for (int idx = threadIdx.x; idx < M * K; idx += kDT) {
    const int m = idx / K, k = idx % K;
    WsT[k * M + m] = __bfloat162float(W[idx]);
  }
  const int ntiles = (n + kTN - 1) / kTN;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTN * K; idx += kDT) {
      const int r = idx / K, k = idx % K;
      const int i = t * kTN + r;
      float xv = 0.0f;
      if (i < n) xv = k < K1 ? X1[(size_t)i * K1 + k] : X2[(size_t)i * K2 + (k - K1)];
      Xs[idx] = xv;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTN * M; idx += kDT) {
      const int r = idx / M, m = idx % M;
      const int i = t * kTN + r;
      if (i >= n) continue;
      float acc = bias ? bias[m] : 0.0f;
      for (int k = 0; k < K; ++k) acc = fmaf(Xs[r * K + k], WsT[k * M + m], acc);
      if (Ypre) Ypre[(size_t)i * M + m] = acc;
      float y = relu ? fmaxf(acc, 0.0f) : acc;
      if (R) y += R[(size_t)i * M + m];
      Y[(size_t)i * M + m] = y;
    }
  }
}

// dX[i, k] = (base ? base[i, k] : 0) + sum_m dY[i, m] W[m, col0 + k]
__global__ void __launch_bounds__(kDT) dense_bwdx_kernel(int n, int M, const float* __restrict__ dY,
                                                         int K, const __nv_bfloat16* __restrict__ W,
                                                         int col0, int wstride,
                                                         const float* __restrict__ base,
                                                         float* __restrict__ dX) {
  __shared__ float Ws[kMaxM * kMaxK];  // [m][k]
  __shared__ float Ds[kTN * kMaxM];
  for (int idx = threadIdx.x; idx < M * K; idx += kDT) {
    const int m = idx / K, k = idx % K;
    Ws[idx] = __bfloat162float(W[(size_t)m * wstride + col0 + k]);
  }
  const int ntiles = (n + kTN - 1) / kTN;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTN * M; idx += kDT) {
      const int r = idx / M, m = idx % M;
      const int i = t * kTN + r;
      Ds[idx] = i < n ? dY[(size_t)i * M + m] : 0.0f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTN * K; idx += kDT) {
      const int r = idx / K, k = idx % K;
      const int i = t * kTN + r;
      if (i >= n) continue;
      float acc = base ? base[(size_t)i * K + k] : 0.0f;
      for (int m = 0; m < M; ++m) acc = fmaf(Ds[r * M + m], Ws[m * K + k], acc);
      dX[(size_t)i * K + k] = acc;
    }
  }
}

// partial[block][m * (K + 1) + k] = sum over the block's nodes of dY[i, m] X[i, k]
// (k = K: dY[i, m], the bias gradient)
constexpr int kBwdW = 25;  // outputs per thread: 256 * 25 >= 96 * 65
__global__ void __launch_bounds__(kDT) dense_bwdw_kernel(int n, int M, const float* __restrict__ dY,
                                                         int K1, const float* __restrict__ X1, int K2,
                                                         const float* __restrict__ X2,
                                                         float* __restrict__ partial) {
  __shared__ float Ds[kTN * kMaxM];
  __shared__ float Xs[kTN * (kMaxK + 1)];
  const int K = K1 + K2, K1p = K + 1;
  const int nout = M * K1p;
  float acc[kBwdW];
#pragma unroll
  for (int j = 0; j < kBwdW; ++j) acc[j] = 0.0f;
  const int ntiles = (n + kTN - 1) / kTN;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTN * M; idx += kDT) {
      const int r = idx / M, m = idx % M;
      const int i = t * kTN + r;
      Ds[idx] = i < n ? dY[(size_t)i * M + m] : 0.0f;
    }
    for (int idx = threadIdx.x; idx < kTN * K1p; idx += kDT) {
      const int r = idx / K1p, k = idx % K1p;
      const int i = t * kTN + r;
      float xv = 0.0f;
      if (i < n) xv = k == K ? 1.0f : (k < K1 ? X1[(size_t)i * K1 + k] : X2[(size_t)i * K2 + (k - K1)]);
      Xs[idx] = xv;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBwdW; ++j) {
      const int o = threadIdx.x + j * kDT;
      if (o < nout) {
        const int m = o / K1p, k = o % K1p;
        float a = acc[j];
        for (int r = 0; r < kTN; ++r) a = fmaf(Ds[r * M + m], Xs[r * K1p + k], a);
        acc[j] = a;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kBwdW; ++j) {
    const int o = threadIdx.x + j * kDT;
    if (o < nout) partial[(size_t)blockIdx.x * nout + o] = acc[j];
  }
}

// out[o] = sum over blocks b (in order) of partial[b * count + o]
__global__ void reduce_blocks_kernel(int nblocks, int count, const float* __restrict__ partial,
                                     float* __restrict__ out) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < count; o += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * count + o];
    out[o] = s;
  }
}

// split [M x (K+1)] into dW [M x K] and db [M]
__global__ void split_wb_kernel(int M, int K, const float* __restrict__ wb, float* __restrict__ dW,
                                float* __restrict__ db) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < M * (K + 1); o += gridDim.x * blockDim.x) {
    const int m = o / (K + 1), k = o % (K + 1);
    if (k < K) dW[m * K + k] = wb[o];
    else if (db) db[m] = wb[o];
  }
}

// out = dY * (pre > 0)
__global__ void relu_mask_kernel(long long cnt, const float* __restrict__ dY, const float* __restrict__ pre,
                                 float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = pre[i] > 0.0f ? dY[i] : 0.0f;
}

// ------------------------------------------------------------ aggregation
// Agg[i, :] = (acc ? Agg[i, :] : 0) + sum_{k in row i, c_k != i} e_k X[c_k, :]; warp per row
__global__ void aggregate_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                                 const float* __restrict__ e, const float* __restrict__ X,
                                 float* __restrict__ Agg, int acc) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
    float s = acc ? Agg[(size_t)i * kW + lane] : 0.0f;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = c[k];
      if (j != i) s = fmaf(e[k], X[(size_t)j * kW + lane], s);
    }
    Agg[(size_t)i * kW + lane] = s;
  }
}

// ------------------------------------------------------------ head
// theta and G values per tril entry; warp per row, lane = hidden unit
__global__ void head_fwd_kernel(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                                const int* __restrict__ gsrc, const float* __restrict__ e,
                                const double* __restrict__ d, const float* __restrict__ PQR,
                                const float* __restrict__ ue, const float* __restrict__ vv,
                                const float* __restrict__ vd, float* __restrict__ theta,
                                double* __restrict__ g_val) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
    const float Pm = PQR[(size_t)i * 96 + lane];
    const float Rm = fmaxf(PQR[(size_t)i * 96 + 64 + lane], 0.0f);
    const float uem = ue[lane], vm = vv[lane], vdm = vd[lane];
    const double sdi = sqrt(d[i]);
    for (int kg = grp[i]; kg < grp[i + 1]; ++kg) {
      const int j = gcol[kg];
      float th;
      double gv;
      if (j == i) {
        th = warp_sum_f(vdm * Rm);
        gv = exp((double)th) / sdi;
      } else {
        const float pre = Pm + PQR[(size_t)j * 96 + 32 + lane] + uem * e[gsrc[kg]];
        th = warp_sum_f(vm * fmaxf(pre, 0.0f));
        gv = (double)th / sdi;
      }
      if (lane == 0) {
        theta[kg] = th;
        g_val[kg] = gv;
      }
    }
  }
}

// Backward by rows: dtheta per entry, dP and dR rows, per-block partial
// sums of dv, due, dvd (partial[block][0:32] dv, [32:64] due, [64:96] dvd).
__global__ void __launch_bounds__(256) head_bwd_rows_kernel(
    int n, const int* __restrict__ grp, const int* __restrict__ gcol, const int* __restrict__ gsrc,
    const float* __restrict__ e, const double* __restrict__ d, const float* __restrict__ PQR,
    const float* __restrict__ ue, const float* __restrict__ vv, const float* __restrict__ vd,
    const double* __restrict__ g_val, const double* __restrict__ dG, float* __restrict__ dtheta,
    float* __restrict__ dPQR, float* __restrict__ partial) {
  __shared__ float red[8][96];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float a_v = 0.0f, a_ue = 0.0f, a_vd = 0.0f;
  for (int i = blockIdx.x * 8 + w; i < n; i += gridDim.x * 8) {
    const float Pm = PQR[(size_t)i * 96 + lane];
    const float Rpre = PQR[(size_t)i * 96 + 64 + lane];
    const float uem = ue[lane], vm = vv[lane], vdm = vd[lane];
    const double sdi = sqrt(d[i]);
    float dP = 0.0f, dR = 0.0f;
    for (int kg = grp[i]; kg < grp[i + 1]; ++kg) {
      const int j = gcol[kg];
      float dth;
      if (j == i) {
        dth = (float)(dG[kg] * g_val[kg]);  // d(exp(theta)/sqrt(d))/dtheta = g
        a_vd = fmaf(fmaxf(Rpre, 0.0f), dth, a_vd);
        dR = Rpre > 0.0f ? vdm * dth : 0.0f;
      } else {
        dth = (float)(dG[kg] / sdi);
        const float ek = e[gsrc[kg]];
        const float pre = Pm + PQR[(size_t)j * 96 + 32 + lane] + uem * ek;
        const float dpre = pre > 0.0f ? vm * dth : 0.0f;
        dP += dpre;
        a_ue = fmaf(dpre, ek, a_ue);
        a_v = fmaf(fmaxf(pre, 0.0f), dth, a_v);
      }
      if (lane == 0) dtheta[kg] = dth;
    }
    dPQR[(size_t)i * 96 + lane] = dP;
    dPQR[(size_t)i * 96 + 64 + lane] = dR;
  }
  red[w][lane] = a_v;
  red[w][32 + lane] = a_ue;
  red[w][64 + lane] = a_vd;
  __syncthreads();
  if (threadIdx.x < 96) {
    float s = 0.0f;
    for (int j = 0; j < 8; ++j) s += red[j][threadIdx.x];
    partial[(size_t)blockIdx.x * 96 + threadIdx.x] = s;
  }
}

// Backward by columns (through the CSR of G^T): dQ[j] = sum over off-diagonal
// entries (i, j) of v * dtheta * (pre > 0)
__global__ void head_bwd_cols_kernel(int n, const int* __restrict__ gtrp, const int* __restrict__ gtrow,
                                     const int* __restrict__ gtperm, const int* __restrict__ gsrc,
                                     const float* __restrict__ e, const float* __restrict__ PQR,
                                     const float* __restrict__ ue, const float* __restrict__ vv,
                                     const float* __restrict__ dtheta, float* __restrict__ dPQR) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < n; j += gridDim.x * wpb) {
    const float Qm = PQR[(size_t)j * 96 + 32 + lane];
    const float uem = ue[lane], vm = vv[lane];
    float dQ = 0.0f;
    for (int t = gtrp[j]; t < gtrp[j + 1]; ++t) {
      const int i = gtrow[t];
      if (i == j) continue;
      const int kg = gtperm[t];
      const float pre = PQR[(size_t)i * 96 + lane] + Qm + uem * e[gsrc[kg]];
      if (pre > 0.0f) dQ = fmaf(vm, dtheta[kg], dQ);
    }
    dPQR[(size_t)j * 96 + 32 + lane] = dQ;
  }
}

// ------------------------------------------------------------ loss (FP64)
// y[row] = sum over entries of (vals[perm? perm[k] : k]) * x[col[k]]
__global__ void spmv_perm_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                                 const double* __restrict__ vals, const int* __restrict__ perm,
                                 const double* __restrict__ x, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) s = fma(vals[perm ? perm[k] : k], x[c[k]], s);
    y[i] = s;
  }
}

// e = xstar - y
__global__ void sub_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// one block: c = xs.u, num = e.Ae; loss = num / c; scale = -2 / c
__global__ void __launch_bounds__(1024) loss_scalars_kernel(int n, const double* __restrict__ xs,
                                                            const double* __restrict__ u,
                                                            const double* __restrict__ err,
                                                            const double* __restrict__ Ae,
                                                            double* __restrict__ out) {
  __shared__ double red[2 * 1024 + 2];
  double acc[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += 1024) {
    acc[0] = fma(xs[i], u[i], acc[0]);
    acc[1] = fma(err[i], Ae[i], acc[1]);
  }
  block_sums<1024, 2>(acc, red);
  if (threadIdx.x == 0) {
    out[0] = acc[1] / acc[0];
    out[1] = -2.0 / acc[0];
  }
}

__global__ void scale_kernel(int n, const double* __restrict__ s, const double* __restrict__ a,
                             double* __restrict__ out) {
  const double f = s[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = f * a[i];
}

// dG[k] = g[i] s[j] + u[i] h[j] on the pattern of G (thread per row)
__global__ void outer2_kernel(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                              const double* __restrict__ g, const double* __restrict__ s,
                              const double* __restrict__ u, const double* __restrict__ h,
                              double* __restrict__ dG) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double gi = g[i], ui = u[i];
    for (int k = grp[i]; k < grp[i + 1]; ++k) {
      const int j = gcol[k];
      dG[k] = fma(gi, s[j], ui * h[j]);
    }
  }
}

// ------------------------------------------------------------ adam
__global__ void adam_kernel(int np, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, float clip, __nv_bfloat16* __restrict__ pb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    if (clip > 0.0f) gi = fminf(fmaxf(gi, -clip), clip);
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(int np, const float* __restrict__ p, __nv_bfloat16* __restrict__ pb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16_rn(p[i]);
}

}  // namespace
}  // namespace sla

using namespace sla;

#define MP_LAUNCH_CHECK() SLA_CUDA_TRY(cudaGetLastError())

extern "C" int32_t sla_mp_features(const sla_csr* A, const double* val, double* d, float* e, float* F,
                                   void* stream) {
  if (A == nullptr || A->n < 0) return SLA_ERR_INVALID;
  if (A->n == 0) return SLA_OK;
  if (!A->rowptr || !A->col || !val || !d || !e || !F) return SLA_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const int g = grid_rows(A->n, 256);
  diag_kernel<<<g, 256, 0, s>>>(A->n, A->rowptr, A->col, val, d);
  feat_kernel<<<g, 256, 0, s>>>(A->n, A->rowptr, A->col, val, d, e, F);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_tril_pattern(const sla_csr* A, int32_t* g_rowptr, int32_t* g_col, int32_t* g_src,
                                    int32_t* nnz_g, void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || A->n < 0 || g_rowptr == nullptr || nnz_g == nullptr) return SLA_ERR_INVALID;
  const int n = A->n;
  const size_t need = al256(sizeof(int) * ((size_t)n + 1)) + al256(sizeof(int) * (size_t)scan_tmp_ints(n + 1));
  if (ws == nullptr || ((uintptr_t)ws & 255u) || ws_bytes < need) return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  int* cnt = (int*)ws;
  int* tmp = (int*)((char*)ws + al256(sizeof(int) * ((size_t)n + 1)));
  tril_count_kernel<<<grid_rows(n + 1, 256), 256, 0, s>>>(n, A->rowptr, A->col, cnt);
  MP_LAUNCH_CHECK();
  int rc = device_exclusive_scan(cnt, (long long)n + 1, g_rowptr, tmp, nnz_g, s);
  if (rc != SLA_OK) return rc;
  if (n > 0) tril_fill_kernel<<<grid_rows(n, 256), 256, 0, s>>>(n, A->rowptr, A->col, g_rowptr, g_col, g_src);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" size_t sla_tril_pattern_ws(int32_t n) {
  return al256(sizeof(int) * ((size_t)n + 1)) + al256(sizeof(int) * (size_t)scan_tmp_ints(n + 1));
}

extern "C" int32_t sla_mp_dense_fwd(int32_t n, int32_t K1, const float* X1, int32_t K2, const float* X2,
                                    int32_t M, const void* W_bf16, const float* bias, const float* R,
                                    int32_t relu, float* Ypre, float* Y, void* stream) {
  if (n < 0 || K1 < 0 || K2 < 0 || K1 + K2 < 1 || K1 + K2 > kMaxK || M < 1 || M > kMaxM) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (!W_bf16 || !Y || (K1 && !X1) || (K2 && !X2)) return SLA_ERR_INVALID;
  dense_fwd_kernel<<<grid_rows(n, kTN, 4096), kDT, 0, (cudaStream_t)stream>>>(
      n, K1, X1, K2, X2, M, (const __nv_bfloat16*)W_bf16, bias, R, relu, Ypre, Y);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_mp_dense_bwdx(int32_t n, int32_t M, const float* dY, int32_t K, const void* W_bf16,
                                     int32_t col0, int32_t wstride, const float* base, float* dX,
                                     void* stream) {
  if (n < 0 || M < 1 || M > kMaxM || K < 1 || K > kMaxK || col0 < 0 || col0 + K > wstride) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (!dY || !W_bf16 || !dX) return SLA_ERR_INVALID;
  dense_bwdx_kernel<<<grid_rows(n, kTN, 4096), kDT, 0, (cudaStream_t)stream>>>(
      n, M, dY, K, (const __nv_bfloat16*)W_bf16, col0, wstride, base, dX);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" size_t sla_mp_dense_bwdw_ws(int32_t M, int32_t K) {
  return al256(sizeof(float) * 148 * 4 * (size_t)M * (K + 1)) + al256(sizeof(float) * (size_t)M * (K + 1));
}

extern "C" int32_t sla_mp_dense_bwdw(int32_t n, int32_t M, const float* dY, int32_t K1, const float* X1,
                                     int32_t K2, const float* X2, float* dW, float* db, void* ws,
                                     size_t ws_bytes, void* stream) {
  const int K = K1 + K2;
  if (n < 0 || M < 1 || M > kMaxM || K < 1 || K > kMaxK || M * (K + 1) > kDT * kBwdW) return SLA_ERR_INVALID;
  if (!dW || ws == nullptr || ws_bytes < sla_mp_dense_bwdw_ws(M, K) || ((uintptr_t)ws & 255u))
    return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const int count = M * (K + 1);
  float* partial = (float*)ws;
  float* wb = (float*)((char*)ws + al256(sizeof(float) * 148 * 4 * (size_t)count));
  const int blocks = grid_rows(n > 0 ? n : 1, kTN, 148 * 4);
  dense_bwdw_kernel<<<blocks, kDT, 0, s>>>(n, M, dY, K1, X1, K2, X2, partial);
  reduce_blocks_kernel<<<grid_rows(count, 256), 256, 0, s>>>(blocks, count, partial, wb);
  split_wb_kernel<<<grid_rows(count, 256), 256, 0, s>>>(M, K, wb, dW, db);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_mp_relu_mask(int64_t count, const float* dY, const float* pre, float* out, void* stream) {
  if (count < 0) return SLA_ERR_INVALID;
  if (count == 0) return SLA_OK;
  relu_mask_kernel<<<grid_rows(count, 256), 256, 0, (cudaStream_t)stream>>>(count, dY, pre, out);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_mp_aggregate(const sla_csr* A, const float* e, const float* X, float* Agg,
                                    int32_t accumulate, void* stream) {
  if (A == nullptr || A->n < 0) return SLA_ERR_INVALID;
  if (A->n == 0) return SLA_OK;
  aggregate_kernel<<<grid_rows(A->n, 8), 256, 0, (cudaStream_t)stream>>>(A->n, A->rowptr, A->col, e, X, Agg,
                                                                        accumulate);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_mp_head_fwd(int32_t n, const int32_t* g_rowptr, const int32_t* g_col,
                                   const int32_t* g_src, const float* e, const double* d, const float* PQR,
                                   const float* ue, const float* v, const float* vd, float* theta,
                                   double* g_val, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  head_fwd_kernel<<<grid_rows(n, 8), 256, 0, (cudaStream_t)stream>>>(n, g_rowptr, g_col, g_src, e, d, PQR,
                                                                    ue, v, vd, theta, g_val);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" size_t sla_mp_head_bwd_ws(int32_t n) {
  return al256(sizeof(float) * 96 * (size_t)grid_rows(n > 0 ? n : 1, 8, 2048)) + al256(sizeof(float) * 96);
}

// grads: [dv (32) | due (32) | dvd (32)]
extern "C" int32_t sla_mp_head_bwd(int32_t n, const int32_t* g_rowptr, const int32_t* g_col,
                                   const int32_t* g_src, const int32_t* gt_rowptr, const int32_t* gt_row,
                                   const int32_t* gt_perm, const float* e, const double* d, const float* PQR,
                                   const float* ue, const float* v, const float* vd, const double* g_val,
                                   const double* dG, float* dtheta, float* dPQR, float* grads, void* ws,
                                   size_t ws_bytes, void* stream) {
  if (n < 0) return SLA_ERR_INVALID;
  if (ws == nullptr || ws_bytes < sla_mp_head_bwd_ws(n) || ((uintptr_t)ws & 255u)) return SLA_ERR_WORKSPACE;
  if (n == 0) return SLA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = grid_rows(n, 8, 2048);
  float* partial = (float*)ws;
  head_bwd_rows_kernel<<<blocks, 256, 0, s>>>(n, g_rowptr, g_col, g_src, e, d, PQR, ue, v, vd, g_val, dG, dtheta,
                                              dPQR, partial);
  head_bwd_cols_kernel<<<grid_rows(n, 8), 256, 0, s>>>(n, gt_rowptr, gt_row, gt_perm, g_src, e, PQR, ue, v,
                                                       dtheta, dPQR);
  reduce_blocks_kernel<<<1, 96, 0, s>>>(blocks, 96, partial, grads);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" size_t sla_ggt_loss_ws(int32_t n) { return 6 * al256(sizeof(double) * (size_t)(n > 0 ? n : 1)) + 256; }

// loss[0] = (x* - G G^T u)^T A (x* - G G^T u) / (x*^T u), loss[1] = -2 / (x*^T u);
// dG = dloss/dG on the pattern of G.
extern "C" int32_t sla_ggt_loss_grad(const sla_csr* A, const double* val, const sla_csr* G,
                                     const double* g_val, const sla_csr_t* GT, const double* u,
                                     const double* xstar, double* loss, double* dG, void* ws,
                                     size_t ws_bytes, void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr || A->n != G->n || A->n < 0) return SLA_ERR_INVALID;
  const int n = A->n;
  if (ws == nullptr || ws_bytes < sla_ggt_loss_ws(n) || ((uintptr_t)ws & 255u)) return SLA_ERR_WORKSPACE;
  if (n == 0) return SLA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vb = al256(sizeof(double) * (size_t)n);
  double* sv = (double*)ws;
  double* y = (double*)((char*)ws + vb);
  double* err = (double*)((char*)ws + 2 * vb);
  double* Ae = (double*)((char*)ws + 3 * vb);
  double* g = (double*)((char*)ws + 4 * vb);
  double* h = (double*)((char*)ws + 5 * vb);
  const int gr = grid_rows(n, 256);
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, GT->rowptr_t, GT->col_t, g_val, GT->perm_t, u, sv);      // s = G^T u
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, G->rowptr, G->col, g_val, nullptr, sv, y);               // y = G s
  sub_kernel<<<gr, 256, 0, s>>>(n, xstar, y, err);                                                  // e
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, A->rowptr, A->col, val, nullptr, err, Ae);                // A e
  loss_scalars_kernel<<<1, 1024, 0, s>>>(n, xstar, u, err, Ae, loss);
  scale_kernel<<<gr, 256, 0, s>>>(n, loss, Ae, g);                                                  // g
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, GT->rowptr_t, GT->col_t, g_val, GT->perm_t, g, h);       // h = G^T g
  outer2_kernel<<<gr, 256, 0, s>>>(n, G->rowptr, G->col, g, sv, u, h, dG);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_adam_step(int32_t np, float* p, const float* g, float* m, float* v, float lr, float b1,
                                 float b2, float eps, int32_t t, float clip, void* p_bf16, void* stream) {
  if (np < 0 || t < 1) return SLA_ERR_INVALID;
  if (np == 0) return SLA_OK;
  const float bc1 = 1.0f - powf(b1, (float)t), bc2 = 1.0f - powf(b2, (float)t);
  adam_kernel<<<grid_rows(np, 256), 256, 0, (cudaStream_t)stream>>>(np, p, g, m, v, lr, b1, b2, eps, bc1, bc2,
                                                                    clip, (__nv_bfloat16*)p_bf16);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_to_bf16(int32_t np, const float* p, void* p_bf16, void* stream) {
  if (np < 0) return SLA_ERR_INVALID;
  if (np == 0) return SLA_OK;
  to_bf16_kernel<<<grid_rows(np, 256), 256, 0, (cudaStream_t)stream>>>(np, p, (__nv_bfloat16*)p_bf16);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}
