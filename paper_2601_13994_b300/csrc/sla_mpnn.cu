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
    int deg = 0;
    // e_ij = (A_ij / sqrt(d_i)) / sqrt(d_j): the FP64 part is per row (one
    // thread per row, so each FP64 instruction serves 32 rows), the neighbour
    // factor is FP32 -- e is stored in FP32, so its accuracy is unchanged in
    // kind (a few FP32 ulps)
    const double rsi = 1.0 / sqrt(d[i]);
    float fa = 0.0f, fs = 0.0f;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = c[k];
      const float ek = (float)(v[k] * rsi) * rsqrtf((float)d[j]);
      e[k] = ek;
      if (j != i) {
        fa += fabsf(ek);
        fs += ek;
        ++deg;
      }
    }
    F[3 * (size_t)i + 0] = fa;
    F[3 * (size_t)i + 1] = fs;
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
template <int NM>
__global__ void __launch_bounds__(kDT) dense_fwd_kernel(int n, int K1, const float* __restrict__ X1,
                                                        int K2, const float* __restrict__ X2, int M,
                                                        const __nv_bfloat16* __restrict__ W,
                                                        const float* __restrict__ bias,
                                                        const float* __restrict__ R, int relu,
                                                        float* __restrict__ Ypre,
                                                        float* __restrict__ Y) {
  // Register-blocked: thread (rg = warp, m0 = lane) owns rows rg + 8 rr
  // (rr < 8) of a 64-row tile and columns m0 + 32 mm (mm < NM).  Inputs and
  // weights sit in shared memory with rows padded to Kp + 4 floats (Kp = K
  // rounded up to 4, zero-filled), so every step over 4 k is one 16-byte
  // load of W per column (conflict-free across the warp) and one broadcast
  // 16-byte load of X per row: 32 NM FMAs per (8 + NM) shared loads.  Each
  // output is still the sequential sum over k = 0 .. K-1 started from the
  // bias, as before.
  constexpr int kRowsT = 64, kRR = kRowsT / 8;
  // dynamic shared memory sized for this layer: W [M][S] then X [64][S]
  extern __shared__ __align__(16) float dsm_f[];
  const int K = K1 + K2;
  const int Kp = (K + 3) & ~3;
  const int S = Kp + 4;
  float* Ws = dsm_f;
  float* Xs = dsm_f + M * S;
  for (int idx = threadIdx.x; idx < M * Kp; idx += kDT) {
    const int m = idx / Kp, k = idx % Kp;
    Ws[m * S + k] = k < K ? __bfloat162float(W[m * K + k]) : 0.0f;
  }
  const int m0 = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int ntiles = (n + kRowsT - 1) / kRowsT;
  // vector loads need 16-byte aligned rows of both inputs
  const bool vec = (K1 % 4 == 0) && (K2 % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(X1) | reinterpret_cast<uintptr_t>(X2)) & 15u) == 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (vec) {
      // 16-byte chunks, all loads of the thread issued before its stores
      constexpr int kMaxC = kRowsT * kMaxK / 4 / kDT;  // chunks per thread
      const int cpr = Kp / 4, nch = kRowsT * cpr;
      float4 buf[kMaxC];
#pragma unroll
      for (int u = 0; u < kMaxC; ++u) {
        const int idx = threadIdx.x + u * kDT;
        buf[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (idx < nch) {
          const int r = idx / cpr, k = 4 * (idx % cpr);
          const int i = t * kRowsT + r;
          if (i < n)
            buf[u] = k < K1 ? *reinterpret_cast<const float4*>(X1 + (size_t)i * K1 + k)
                            : *reinterpret_cast<const float4*>(X2 + (size_t)i * K2 + (k - K1));
        }
      }
#pragma unroll
      for (int u = 0; u < kMaxC; ++u) {
        const int idx = threadIdx.x + u * kDT;
        if (idx < nch) *reinterpret_cast<float4*>(&Xs[(idx / cpr) * S + 4 * (idx % cpr)]) = buf[u];
      }
    } else {
      for (int idx = threadIdx.x; idx < kRowsT * Kp; idx += kDT) {
        const int r = idx / Kp, k = idx % Kp;
        const int i = t * kRowsT + r;
        float xv = 0.0f;
        if (i < n && k < K) xv = k < K1 ? X1[(size_t)i * K1 + k] : X2[(size_t)i * K2 + (k - K1)];
        Xs[r * S + k] = xv;
      }
    }
    __syncthreads();
    float acc[NM][kRR];
#pragma unroll
    for (int mm = 0; mm < NM; ++mm) {
      const int m = m0 + 32 * mm;
      const float b0 = (bias && m < M) ? bias[m] : 0.0f;
#pragma unroll
      for (int rr = 0; rr < kRR; ++rr) acc[mm][rr] = b0;
    }
    for (int k = 0; k < Kp; k += 4) {
      float4 w[NM];
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) {
        const int m = min(m0 + 32 * mm, M - 1);
        w[mm] = *reinterpret_cast<const float4*>(&Ws[m * S + k]);
      }
#pragma unroll
      for (int rr = 0; rr < kRR; ++rr) {
        const float4 xv = *reinterpret_cast<const float4*>(&Xs[(rg + 8 * rr) * S + k]);
#pragma unroll
        for (int mm = 0; mm < NM; ++mm) {
          float a0 = acc[mm][rr];
          a0 = fmaf(xv.x, w[mm].x, a0);
          a0 = fmaf(xv.y, w[mm].y, a0);
          a0 = fmaf(xv.z, w[mm].z, a0);
          a0 = fmaf(xv.w, w[mm].w, a0);
          acc[mm][rr] = a0;
        }
      }
    }
#pragma unroll
    for (int mm = 0; mm < NM; ++mm) {
      const int m = m0 + 32 * mm;
      if (m >= M) continue;
#pragma unroll
      for (int rr = 0; rr < kRR; ++rr) {
        const int i = t * kRowsT + rg + 8 * rr;
        if (i >= n) continue;
        const float a0 = acc[mm][rr];
        if (Ypre) Ypre[(size_t)i * M + m] = a0;
        float y = relu ? fmaxf(a0, 0.0f) : a0;
        if (R) y += R[(size_t)i * M + m];
        Y[(size_t)i * M + m] = y;
      }
    }
  }
}

// The same layer for M = 32 MS outputs with 4 x 4 register tiles: thread
// (tx, ty) of the 256-thread block owns rows ty + 32 r (r < 4) of a
// 128-row tile and, in each 32-column slab, columns 4 tx .. 4 tx + 3.  X sits
// in shared memory row-major (rows padded to Kp + 4 floats, so the four rows
// a warp reads at one time fall in different banks), W k-major (transposed
// once per block).  Per 4 steps of k a thread makes 4 16-byte loads of X
// and 4 MS of W for 64 MS FMAs: 4 + 4 MS shared-memory wavefronts per 2048
// MS FMAs of a warp, against 12 per 1024 above.  Each output is still the
// sum over k = 0 .. Kp-1 in order, started from the bias (the same bits).
template <int MS>
__global__ void __launch_bounds__(kDT) dense_fwd_tiled_kernel(int n, int K1, const float* __restrict__ X1,
                                                              int K2, const float* __restrict__ X2, int M,
                                                              const __nv_bfloat16* __restrict__ W,
                                                              const float* __restrict__ bias,
                                                              const float* __restrict__ R, int relu,
                                                              float* __restrict__ Ypre,
                                                              float* __restrict__ Y) {
  constexpr int kRowsT = 128, MW = 32 * MS, SW = MW + 4;
  extern __shared__ __align__(16) float dsm_t[];
  const int K = K1 + K2;
  const int Kp = (K + 3) & ~3;
  const int SX = Kp + 4;
  float* Ws = dsm_t;            // [Kp][SW]   k-major
  float* Xs = dsm_t + Kp * SW;  // [128][SX]  row-major
  for (int idx = threadIdx.x; idx < Kp * MW; idx += kDT) {
    const int k = idx / MW, m = idx % MW;
    Ws[k * SW + m] = (k < K && m < M) ? __bfloat162float(W[m * K + k]) : 0.0f;
  }
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int ntiles = (n + kRowsT - 1) / kRowsT;
  const bool vec = (K1 % 4 == 0) && (K2 % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(X1) | reinterpret_cast<uintptr_t>(X2)) & 15u) == 0;
  const int cpr = Kp / 4;  // 16-byte chunks per row
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (vec) {
      for (int idx = threadIdx.x; idx < kRowsT * cpr; idx += kDT) {
        const int r = idx / cpr, k = 4 * (idx % cpr);
        const int i = t * kRowsT + r;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (i < n && k < K)
          v = k < K1 ? *reinterpret_cast<const float4*>(X1 + (size_t)i * K1 + k)
                     : *reinterpret_cast<const float4*>(X2 + (size_t)i * K2 + (k - K1));
        *reinterpret_cast<float4*>(&Xs[r * SX + k]) = v;
      }
    } else {
      for (int idx = threadIdx.x; idx < kRowsT * Kp; idx += kDT) {
        const int r = idx / Kp, k = idx % Kp;
        const int i = t * kRowsT + r;
        float xv = 0.0f;
        if (i < n && k < K) xv = k < K1 ? X1[(size_t)i * K1 + k] : X2[(size_t)i * K2 + (k - K1)];
        Xs[r * SX + k] = xv;
      }
    }
    __syncthreads();
    float acc[MS][4][4];
#pragma unroll
    for (int sl = 0; sl < MS; ++sl)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = 32 * sl + 4 * tx + c;
        const float b0 = (bias && m < M) ? bias[m] : 0.0f;
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[sl][r][c] = b0;
      }
    for (int k0 = 0; k0 < Kp; k0 += 4) {
      float4 xq[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) xq[r] = *reinterpret_cast<const float4*>(&Xs[(ty + 32 * r) * SX + k0]);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int sl = 0; sl < MS; ++sl) {
          const float4 wv = *reinterpret_cast<const float4*>(&Ws[(k0 + kk) * SW + 32 * sl + 4 * tx]);
          const float wc[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float xv = kk == 0 ? xq[r].x : kk == 1 ? xq[r].y : kk == 2 ? xq[r].z : xq[r].w;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[sl][r][c] = fmaf(xv, wc[c], acc[sl][r][c]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = t * kRowsT + ty + 32 * r;
      if (i >= n) continue;
#pragma unroll
      for (int sl = 0; sl < MS; ++sl)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int m = 32 * sl + 4 * tx + c;
          if (m >= M) continue;
          const float a0 = acc[sl][r][c];
          if (Ypre) Ypre[(size_t)i * M + m] = a0;
          float y = relu ? fmaxf(a0, 0.0f) : a0;
          if (R) y += R[(size_t)i * M + m];
          Y[(size_t)i * M + m] = y;
        }
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
  // warp per row, lane = feature.  The row's first 8 column indices and
  // edge values are loaded by 8 lanes at once and broadcast, and the 8
  // neighbour rows are gathered back to back before the FMAs, which then run
  // in entry order (the same sum as one entry at a time).
  constexpr int B = 8;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
    float s = acc ? Agg[(size_t)i * kW + lane] : 0.0f;
    const int k0 = rp[i], k1 = rp[i + 1];
    const int cnt = k1 - k0;
    const int cl = lane < min(cnt, B) ? c[k0 + lane] : i;
    const float el = lane < min(cnt, B) ? e[k0 + lane] : 0.0f;
    float xs[B];
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, cl, m);
      xs[m] = j != i ? X[(size_t)j * kW + lane] : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, cl, m);
      const float em = __shfl_sync(0xffffffffu, el, m);
      if (m < cnt && j != i) s = fmaf(em, xs[m], s);
    }
    for (int k = k0 + B; k < k1; ++k) {
      const int j = c[k];
      if (j != i) s = fmaf(e[k], X[(size_t)j * kW + lane], s);
    }
    Agg[(size_t)i * kW + lane] = s;
  }
}

// The same sums with four rows per warp: 8 lanes per row, each lane owning
// 4 consecutive features (one 16-byte load per neighbour row), so a warp
// has four rows' gathers in flight instead of one.  Entries are added in
// the same order per feature as above, so the results are the same bits.
// X and Agg must be 16-byte aligned (rows of kW = 32 floats).
__global__ void aggregate4_kernel(int n, const int* __restrict__ rp, const int* __restrict__ c,
                                  const float* __restrict__ e, const float4* __restrict__ X,
                                  float4* __restrict__ Agg, int acc) {
  constexpr int B = 8;
  const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (long long i0 = 4 * w; i0 < n; i0 += 4 * warps) {
    const int i = (int)i0 + grp;
    const bool valid = i < n;
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (valid && acc) s = Agg[(size_t)i * 8 + sub];
    const int k0 = valid ? rp[i] : 0, k1 = valid ? rp[i + 1] : 0;
    const int cnt = k1 - k0;
    const int cl = sub < min(cnt, B) ? c[k0 + sub] : i;
    const float el = sub < min(cnt, B) ? e[k0 + sub] : 0.0f;
    float4 xs[B];
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, cl, m, 8);
      xs[m] = (m < cnt && j != i) ? X[(size_t)j * 8 + sub] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, cl, m, 8);
      const float em = __shfl_sync(0xffffffffu, el, m, 8);
      if (m < cnt && j != i) {
        s.x = fmaf(em, xs[m].x, s.x);
        s.y = fmaf(em, xs[m].y, s.y);
        s.z = fmaf(em, xs[m].z, s.z);
        s.w = fmaf(em, xs[m].w, s.w);
      }
    }
    for (int k = k0 + B; k < k1; ++k) {
      const int j = c[k];
      if (j != i) {
        const float ek = e[k];
        const float4 xv = X[(size_t)j * 8 + sub];
        s.x = fmaf(ek, xv.x, s.x);
        s.y = fmaf(ek, xv.y, s.y);
        s.z = fmaf(ek, xv.z, s.z);
        s.w = fmaf(ek, xv.w, s.w);
      }
    }
    if (valid) Agg[(size_t)i * 8 + sub] = s;
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
  // warp per row, lane = hidden unit; the first 8 entries of the row have
  // their columns, edge values and Q rows loaded back to back before the
  // warp sums (theta only; G values in head_gval_kernel)
  constexpr int B = 8;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  (void)d;
  (void)g_val;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += gridDim.x * wpb) {
    const float Pm = PQR[(size_t)i * 96 + lane];
    const float Rm = fmaxf(PQR[(size_t)i * 96 + 64 + lane], 0.0f);
    const float uem = ue[lane], vm = vv[lane], vdm = vd[lane];
    const int k0 = grp[i], k1 = grp[i + 1];
    const int cnt = k1 - k0;
    const int jl = lane < min(cnt, B) ? gcol[k0 + lane] : i;
    const float el = lane < min(cnt, B) ? e[gsrc[k0 + lane]] : 0.0f;
    float q[B];
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, jl, m);
      q[m] = (m < cnt && j != i) ? PQR[(size_t)j * 96 + 32 + lane] : 0.0f;
    }
#pragma unroll
    for (int m = 0; m < B; ++m) {
      if (m >= cnt) break;
      const int j = __shfl_sync(0xffffffffu, jl, m);
      const float em = __shfl_sync(0xffffffffu, el, m);
      const float th = j == i ? warp_sum_f(vdm * Rm) : warp_sum_f(vm * fmaxf(Pm + q[m] + uem * em, 0.0f));
      if (lane == 0) theta[k0 + m] = th;
    }
    for (int kg = k0 + B; kg < k1; ++kg) {
      const int j = gcol[kg];
      float th;
      if (j == i) {
        th = warp_sum_f(vdm * Rm);
      } else {
        const float pre = Pm + PQR[(size_t)j * 96 + 32 + lane] + uem * e[gsrc[kg]];
        th = warp_sum_f(vm * fmaxf(pre, 0.0f));
      }
      if (lane == 0) theta[kg] = th;
    }
  }
}

// theta with four rows per warp: 8 lanes per row, each lane owning hidden
// units 4 sub .. 4 sub + 3 (16-byte loads of P, R and the gathered Q rows),
// the per-entry sum over the 32 units reduced over the row's 8 lanes: a warp
// has four rows' gathers in flight and needs 3 instead of 5 shuffles per
// entry.  Same terms as head_fwd_kernel, summed in a fixed order (4 units
// per lane, then the 8-lane butterfly).  PQR must be 16-byte aligned.
__global__ void head4_fwd_kernel(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                                 const int* __restrict__ gsrc, const float* __restrict__ e,
                                 const float4* __restrict__ PQR4, const float* __restrict__ ue,
                                 const float* __restrict__ vv, const float* __restrict__ vd,
                                 float* __restrict__ theta) {
  constexpr int B = 8;
  const int lane = threadIdx.x & 31, sub = lane & 7, grp4 = lane >> 3;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float uem[4], vm[4], vdm[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    uem[u] = ue[4 * sub + u];
    vm[u] = vv[4 * sub + u];
    vdm[u] = vd[4 * sub + u];
  }
  auto row_sum8 = [](float x) {
    x += __shfl_xor_sync(0xffffffffu, x, 4, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 2, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 1, 8);
    return x;
  };
  for (long long i0 = 4 * w; i0 < n; i0 += 4 * warps) {
    const int i = (int)i0 + grp4;
    const bool valid = i < n;
    const int k0 = valid ? grp[i] : 0, k1 = valid ? grp[i + 1] : 0;
    const int cnt = k1 - k0;
    float4 P = make_float4(0.0f, 0.0f, 0.0f, 0.0f), Rr = P;
    if (valid) {
      P = PQR4[(size_t)i * 24 + sub];
      Rr = PQR4[(size_t)i * 24 + 16 + sub];
    }
    const float Pu[4] = {P.x, P.y, P.z, P.w};
    const float dsum = vdm[0] * fmaxf(Rr.x, 0.0f) + vdm[1] * fmaxf(Rr.y, 0.0f) + vdm[2] * fmaxf(Rr.z, 0.0f) +
                       vdm[3] * fmaxf(Rr.w, 0.0f);
    const float diag = row_sum8(dsum);
    const int jl = sub < min(cnt, B) ? gcol[k0 + sub] : i;
    const float el = sub < min(cnt, B) ? e[gsrc[k0 + sub]] : 0.0f;
    float4 q[B];
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, jl, m, 8);
      q[m] = (m < cnt && j != i) ? PQR4[(size_t)j * 24 + 8 + sub] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const int j = __shfl_sync(0xffffffffu, jl, m, 8);
      const float em = __shfl_sync(0xffffffffu, el, m, 8);
      const float qu[4] = {q[m].x, q[m].y, q[m].z, q[m].w};
      float part = 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) part += vm[u] * fmaxf(Pu[u] + qu[u] + uem[u] * em, 0.0f);
      const float off = row_sum8(part);
      if (sub == 0 && m < cnt) theta[k0 + m] = j == i ? diag : off;
    }
    // rows with more than 8 entries of tril(A) (none in the 5- and 7-point
    // stencils): the rest one entry at a time
    const int extra = cnt > B ? cnt - B : 0;
    int extra_max = extra;
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) extra_max = max(extra_max, __shfl_xor_sync(0xffffffffu, extra_max, o));
    for (int t = 0; t < extra_max; ++t) {
      const bool act = t < extra;
      const int kg = k0 + B + t;
      const int j = act ? gcol[kg] : i;
      float part = 0.0f;
      if (act && j != i) {
        const float4 qv = PQR4[(size_t)j * 24 + 8 + sub];
        const float ek = e[gsrc[kg]];
        const float qu[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) part += vm[u] * fmaxf(Pu[u] + qu[u] + uem[u] * ek, 0.0f);
      }
      const float off = row_sum8(part);
      if (act && sub == 0) theta[kg] = j == i ? diag : off;
    }
  }
}

// G values from theta, one thread per row: G_ii = exp(theta_ii) / sqrt(d_i),
// G_ij = theta_ij / sqrt(d_i).  The FP64 work is here, vectorised over rows
// (on this part an FP64 warp instruction costs its full pipe time however
// few lanes are active, so per-lane FP64 inside the warp-per-row head would
// cost 32 times as much).  exp runs in FP32 (theta is FP32).
__global__ void head_gval_kernel(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                                 const double* __restrict__ d, const float* __restrict__ theta,
                                 double* __restrict__ g_val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double rsd = 1.0 / sqrt(d[i]);
    for (int kg = grp[i]; kg < grp[i + 1]; ++kg) {
      const float th = theta[kg];
      g_val[kg] = (double)(gcol[kg] == i ? expf(th) : th) * rsd;
    }
  }
}

// dtheta per entry, one thread per row: dG * G_ii on the diagonal (the
// derivative of exp(theta)/sqrt(d)), dG / sqrt(d_i) off it.
__global__ void head_dtheta_kernel(int n, const int* __restrict__ grp, const int* __restrict__ gcol,
                                   const double* __restrict__ d, const double* __restrict__ g_val,
                                   const double* __restrict__ dG, float* __restrict__ dtheta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double rsd = 1.0 / sqrt(d[i]);
    for (int kg = grp[i]; kg < grp[i + 1]; ++kg)
      dtheta[kg] = (float)(dG[kg] * (gcol[kg] == i ? g_val[kg] : rsd));
  }
}

// Backward by rows: dP and dR rows from dtheta, per-block partial sums of
// dv, due, dvd (partial[block][0:32] dv, [32:64] due, [64:96] dvd).
__global__ void __launch_bounds__(256) head_bwd_rows_kernel(
    int n, const int* __restrict__ grp, const int* __restrict__ gcol, const int* __restrict__ gsrc,
    const float* __restrict__ e, const double* __restrict__ d, const float* __restrict__ PQR,
    const float* __restrict__ ue, const float* __restrict__ vv, const float* __restrict__ vd,
    const float* __restrict__ dtheta, float* __restrict__ dPQR, float* __restrict__ partial) {
  __shared__ float red[8][96];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float a_v = 0.0f, a_ue = 0.0f, a_vd = 0.0f;
  for (int i = blockIdx.x * 8 + w; i < n; i += gridDim.x * 8) {
    const float Pm = PQR[(size_t)i * 96 + lane];
    const float Rpre = PQR[(size_t)i * 96 + 64 + lane];
    const float uem = ue[lane], vm = vv[lane], vdm = vd[lane];
    float dP = 0.0f, dR = 0.0f;
    for (int kg = grp[i]; kg < grp[i + 1]; ++kg) {
      const int j = gcol[kg];
      const float dth = dtheta[kg];  // from head_dtheta_kernel
      if (j == i) {
        a_vd = fmaf(fmaxf(Rpre, 0.0f), dth, a_vd);
        dR = Rpre > 0.0f ? vdm * dth : 0.0f;
      } else {
        const float ek = e[gsrc[kg]];
        const float pre = Pm + PQR[(size_t)j * 96 + 32 + lane] + uem * ek;
        const float dpre = pre > 0.0f ? vm * dth : 0.0f;
        dP += dpre;
        a_ue = fmaf(dpre, ek, a_ue);
        a_v = fmaf(fmaxf(pre, 0.0f), dth, a_v);
      }
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

// one block: c = xs.u, num = e.Ae; loss = num / c; scale = -2 kappa / c
// (kappa = 1 without a scale, else *kap)
__global__ void __launch_bounds__(1024) loss_scalars_kernel(int n, const double* __restrict__ xs,
                                                            const double* __restrict__ u,
                                                            const double* __restrict__ err,
                                                            const double* __restrict__ Ae,
                                                            const double* __restrict__ kap,
                                                            double* __restrict__ out) {
  __shared__ double red[2 * 1024 + 2];
  double acc[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += 1024) {
    acc[0] = fma(xs[i], u[i], acc[0]);
    acc[1] = fma(err[i], Ae[i], acc[1]);
  }
  block_sums<1024, 2>(acc, red);
  if (threadIdx.x == 0) {
    const double k = kap != nullptr ? *kap : 1.0;
    out[0] = acc[1] / acc[0];
    out[1] = -2.0 * k / acc[0];
  }
}

// one block: the scale of y that minimises (xs - k y)^T A (xs - k y):
// k = xs.Ay / y.Ay (0 when y.Ay = 0, i.e. y = 0)
__global__ void __launch_bounds__(1024) loss_kappa_kernel(int n, const double* __restrict__ xs,
                                                          const double* __restrict__ y,
                                                          const double* __restrict__ Ay,
                                                          double* __restrict__ kap) {
  __shared__ double red[2 * 1024 + 2];
  double acc[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < n; i += 1024) {
    acc[0] = fma(xs[i], Ay[i], acc[0]);
    acc[1] = fma(y[i], Ay[i], acc[1]);
  }
  block_sums<1024, 2>(acc, red);
  if (threadIdx.x == 0) *kap = acc[1] > 0.0 ? acc[0] / acc[1] : 0.0;
}

// err = xs - k y
__global__ void sub_scaled_kernel(int n, const double* __restrict__ xs, const double* __restrict__ y,
                                  const double* __restrict__ kap, double* __restrict__ out) {
  const double k = *kap;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = fma(-k, y[i], xs[i]);
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

namespace sla {
// sla_mp_tc.cu: the tensor-core form of the dense layer
bool mp_dense_tc_applies(int K1, const float* X1, int K2, const float* X2, int M, const float* R,
                         const float* Ypre, const float* Y);
int mp_dense_fwd_tc(int n, int K1, const float* X1, int K2, const float* X2, int M, const __nv_bfloat16* W,
                    const float* bias, const float* R, int relu, float* Ypre, float* Y, cudaStream_t s);
}  // namespace sla

extern "C" int32_t sla_mp_dense_fwd(int32_t n, int32_t K1, const float* X1, int32_t K2, const float* X2,
                                    int32_t M, const void* W_bf16, const float* bias, const float* R,
                                    int32_t relu, float* Ypre, float* Y, void* stream) {
  return sla_mp_dense_fwd_ex(n, K1, X1, K2, X2, M, W_bf16, bias, R, relu, Ypre, Y, SLA_MP_DENSE_AUTO, stream);
}

extern "C" int32_t sla_mp_dense_fwd_ex(int32_t n, int32_t K1, const float* X1, int32_t K2, const float* X2,
                                       int32_t M, const void* W_bf16, const float* bias, const float* R,
                                       int32_t relu, float* Ypre, float* Y, int32_t kernel, void* stream) {
  if (n < 0 || K1 < 0 || K2 < 0 || K1 + K2 < 1 || K1 + K2 > kMaxK || M < 1 || M > kMaxM) return SLA_ERR_INVALID;
  if (kernel != SLA_MP_DENSE_AUTO && kernel != SLA_MP_DENSE_SIMT && kernel != SLA_MP_DENSE_TC)
    return SLA_ERR_INVALID;
  const bool tc_ok = mp_dense_tc_applies(K1, X1, K2, X2, M, R, Ypre, Y);
  if (kernel == SLA_MP_DENSE_TC && !tc_ok) return SLA_ERR_INVALID;
  if (n == 0) return SLA_OK;
  if (!W_bf16 || !Y || (K1 && !X1) || (K2 && !X2)) return SLA_ERR_INVALID;
  const int nm = (M + 31) / 32;
  cudaStream_t s = (cudaStream_t)stream;
  const __nv_bfloat16* Wb = (const __nv_bfloat16*)W_bf16;
  // automatic: the tensor cores wherever their form applies (2.1 M rows,
  // B300: K = 64 -> 32 outputs 458 -> 286 us, K = 32 -> 96 outputs 571 ->
  // 344 us); the CUDA cores for the rest (the 3-feature input layer)
  if (kernel == SLA_MP_DENSE_TC || (kernel == SLA_MP_DENSE_AUTO && tc_ok))
    return mp_dense_fwd_tc(n, K1, X1, K2, X2, M, Wb, bias, R, relu, Ypre, Y, s);
  if (nm == 1) {
    // register-tiled form for 32 outputs: 2.1 M rows, K = 64, 483 -> 374 us
    // (B300); for the 96-wide head it measured slower (584 vs 521 us: 116
    // registers per thread), so that layer keeps dense_fwd_kernel
    const int Kp = (K1 + K2 + 3) & ~3;
    const size_t smem_t = sizeof(float) * ((size_t)Kp * (32 * nm + 4) + (size_t)128 * (Kp + 4));
    const void* ft = (const void*)dense_fwd_tiled_kernel<1>;
    static bool attr_set = false;
    if (!attr_set) {
      const int mx = (int)(sizeof(float) * ((size_t)kMaxK * (32 + 4) + (size_t)128 * (kMaxK + 4)));
      cudaFuncSetAttribute(dense_fwd_tiled_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      attr_set = true;
    }
    int occ_t = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, ft, kDT, smem_t) != cudaSuccess || occ_t < 1) occ_t = 1;
    const int bt = grid_rows(n, 128, 148 * (occ_t < 8 ? occ_t : 8));
    dense_fwd_tiled_kernel<1><<<bt, kDT, smem_t, s>>>(n, K1, X1, K2, X2, M, Wb, bias, R, relu, Ypre, Y);
    MP_LAUNCH_CHECK();
    return SLA_OK;
  }
  const int S = ((K1 + K2 + 3) & ~3) + 4;
  const size_t smem = sizeof(float) * (size_t)(M + 64) * S;
  const void* fn = nm == 1 ? (const void*)dense_fwd_kernel<1> : nm == 2 ? (const void*)dense_fwd_kernel<2>
                                                                          : (const void*)dense_fwd_kernel<3>;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kDT, smem) != cudaSuccess || occ < 1) occ = 1;
  const int blocks = grid_rows(n, 64, 148 * (occ < 8 ? occ : 8));
  if (nm == 1) dense_fwd_kernel<1><<<blocks, kDT, smem, s>>>(n, K1, X1, K2, X2, M, Wb, bias, R, relu, Ypre, Y);
  else if (nm == 2) dense_fwd_kernel<2><<<blocks, kDT, smem, s>>>(n, K1, X1, K2, X2, M, Wb, bias, R, relu, Ypre, Y);
  else dense_fwd_kernel<3><<<blocks, kDT, smem, s>>>(n, K1, X1, K2, X2, M, Wb, bias, R, relu, Ypre, Y);
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
  static_assert(kW == 32, "aggregate4_kernel assumes rows of 32 features");
  if (((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Agg)) & 15u) == 0)
    aggregate4_kernel<<<grid_rows(A->n, 32), 256, 0, (cudaStream_t)stream>>>(
        A->n, A->rowptr, A->col, e, reinterpret_cast<const float4*>(X), reinterpret_cast<float4*>(Agg),
        accumulate);
  else
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
  if ((reinterpret_cast<uintptr_t>(PQR) & 15u) == 0)
    head4_fwd_kernel<<<grid_rows(n, 32), 256, 0, (cudaStream_t)stream>>>(
        n, g_rowptr, g_col, g_src, e, reinterpret_cast<const float4*>(PQR), ue, v, vd, theta);
  else
    head_fwd_kernel<<<grid_rows(n, 8), 256, 0, (cudaStream_t)stream>>>(n, g_rowptr, g_col, g_src, e, d, PQR,
                                                                      ue, v, vd, theta, g_val);
  head_gval_kernel<<<grid_rows(n, 256), 256, 0, (cudaStream_t)stream>>>(n, g_rowptr, g_col, d, theta, g_val);
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
  head_dtheta_kernel<<<grid_rows(n, 256), 256, 0, s>>>(n, g_rowptr, g_col, d, g_val, dG, dtheta);
  head_bwd_rows_kernel<<<blocks, 256, 0, s>>>(n, g_rowptr, g_col, g_src, e, d, PQR, ue, v, vd, dtheta, dPQR,
                                              partial);
  head_bwd_cols_kernel<<<grid_rows(n, 8), 256, 0, s>>>(n, gt_rowptr, gt_row, gt_perm, g_src, e, PQR, ue, v,
                                                       dtheta, dPQR);
  reduce_blocks_kernel<<<1, 96, 0, s>>>(blocks, 96, partial, grads);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" size_t sla_ggt_loss_ws(int32_t n) { return 6 * al256(sizeof(double) * (size_t)(n > 0 ? n : 1)) + 256; }

// loss[0] = (x* - k y)^T A (x* - k y) / (x*^T u) with y = G G^T u, k = 1
// (mode 0) or the minimising k = x*^T A y / y^T A y (mode 1);
// loss[1] = -2 k / (x*^T u); dG = dloss/dG on the pattern of G (in mode 1
// the gradient with k held at its optimum, where dloss/dk = 0).
extern "C" int32_t sla_ggt_loss_grad(const sla_csr* A, const double* val, const sla_csr* G,
                                     const double* g_val, const sla_csr_t* GT, const double* u,
                                     const double* xstar, int32_t mode, double* loss, double* dG, void* ws,
                                     size_t ws_bytes, void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr || A->n != G->n || A->n < 0) return SLA_ERR_INVALID;
  if (mode != 0 && mode != 1) return SLA_ERR_INVALID;
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
  double* kap = nullptr;
  if (mode == 1) {
    kap = (double*)((char*)ws + 6 * vb);
    spmv_perm_kernel<<<gr, 256, 0, s>>>(n, A->rowptr, A->col, val, nullptr, y, Ae);                // A y
    loss_kappa_kernel<<<1, 1024, 0, s>>>(n, xstar, y, Ae, kap);                                     // k
    sub_scaled_kernel<<<gr, 256, 0, s>>>(n, xstar, y, kap, err);                                    // e = x* - k y
  } else {
    sub_kernel<<<gr, 256, 0, s>>>(n, xstar, y, err);                                                // e = x* - y
  }
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, A->rowptr, A->col, val, nullptr, err, Ae);                // A e
  loss_scalars_kernel<<<1, 1024, 0, s>>>(n, xstar, u, err, Ae, kap, loss);
  scale_kernel<<<gr, 256, 0, s>>>(n, loss, Ae, g);                                                  // g
  spmv_perm_kernel<<<gr, 256, 0, s>>>(n, GT->rowptr_t, GT->col_t, g_val, GT->perm_t, g, h);       // h = G^T g
  outer2_kernel<<<gr, 256, 0, s>>>(n, G->rowptr, G->col, g, sv, u, h, dG);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

namespace sla {
namespace {
// A_ik from row i of A (columns ascending), 0 when not stored.
__device__ __forceinline__ double a_entry(const int* __restrict__ rowptr, const int* __restrict__ col,
                                         const double* __restrict__ val, int i, int k) {
  int lo = __ldg(rowptr + i), hi = __ldg(rowptr + i + 1);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int cm = __ldg(col + mid);
    if (cm == k) return __ldg(val + mid);
    if (cm < k) lo = mid + 1;
    else hi = mid;
  }
  return 0.0;
}

// One thread per column j of G (row j of G^T): q = sum_a G_aj (sum_b A_ab G_bj),
// then the column's entries times 1/sqrt(q).
__global__ void __launch_bounds__(256) ggt_normalize_kernel(int n, const int* __restrict__ rowptr,
                                                            const int* __restrict__ col,
                                                            const double* __restrict__ val,
                                                            const int* __restrict__ rpt, const int* __restrict__ rowt,
                                                            const int* __restrict__ perm, const double* g_val,
                                                            double* g_out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int a = __ldg(rpt + j), e = __ldg(rpt + j + 1);
    double q = 0.0;
    for (int ka = a; ka < e; ++ka) {
      const int i = __ldg(rowt + ka);
      double s = 0.0;
      for (int kb = a; kb < e; ++kb)
        s = fma(a_entry(rowptr, col, val, i, __ldg(rowt + kb)), g_val[__ldg(perm + kb)], s);
      q = fma(g_val[__ldg(perm + ka)], s, q);
    }
    const bool ok = q > 0.0 && isfinite(q);
    const double inv = ok ? 1.0 / sqrt(q) : 1.0;
    for (int ka = a; ka < e; ++ka) {
      const int p = __ldg(perm + ka);
      const double gv = g_val[p];
      g_out[p] = ok ? gv * inv : gv;
    }
  }
}
// Backward of ggt_normalize_kernel: with q_j = (G^T A G)_jj and Gn_aj =
// G_aj / sqrt(q_j), dq_j / dG_aj = 2 (A G)_aj (A symmetric), so for the
// entries of column j
//   dG_aj = dGn_aj / sqrt(q_j) - (A G)_aj w_j / q_j^{3/2},  w_j = sum_i dGn_ij G_ij;
// a column left unchanged by the forward (q not positive and finite) passes
// its gradient through.  One thread per column; the first pass forms q_j and
// w_j, the second (A G)_aj again per entry.  dG may be dGn (each column's
// entries are read before they are written, by the same thread).
__global__ void __launch_bounds__(256) ggt_normalize_bwd_kernel(
    int n, const int* __restrict__ rowptr, const int* __restrict__ col, const double* __restrict__ val,
    const int* __restrict__ rpt, const int* __restrict__ rowt, const int* __restrict__ perm,
    const double* __restrict__ g_val, const double* dGn, double* dG) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int a = __ldg(rpt + j), e = __ldg(rpt + j + 1);
    double q = 0.0, w = 0.0;
    for (int ka = a; ka < e; ++ka) {
      const int i = __ldg(rowt + ka);
      double ag = 0.0;
      for (int kb = a; kb < e; ++kb)
        ag = fma(a_entry(rowptr, col, val, i, __ldg(rowt + kb)), g_val[__ldg(perm + kb)], ag);
      const int p = __ldg(perm + ka);
      q = fma(g_val[p], ag, q);
      w = fma(dGn[p], g_val[p], w);
    }
    if (!(q > 0.0 && isfinite(q))) continue;  // unchanged by the forward: dG = dGn
    const double inv = 1.0 / sqrt(q);
    const double c3 = w * inv * inv * inv;
    for (int ka = a; ka < e; ++ka) {
      const int i = __ldg(rowt + ka);
      double ag = 0.0;
      for (int kb = a; kb < e; ++kb)
        ag = fma(a_entry(rowptr, col, val, i, __ldg(rowt + kb)), g_val[__ldg(perm + kb)], ag);
      const int p = __ldg(perm + ka);
      dG[p] = fma(-ag, c3, dGn[p] * inv);
    }
  }
}

// The factored sparse approximate inverse (Kolotilina and Yeremin) on the
// pattern of G = tril(A): one thread per column j (row j of the CSR of G^T,
// whose entries list the rows P = {i >= j : A_ij != 0} in ascending order,
// j first).  The |P| x |P| block A[P, P] is gathered by binary search in A's
// rows, factored by Cholesky (a principal block of an SPD matrix) and
// solved for y with A[P, P] y = e_1; the column is y / sqrt(y_1), so that
// (G^T A G)_jj = 1.  Columns with more than kFsaiMaxP entries, or a block
// whose factorisation fails, get the Jacobi column 1/sqrt(A_jj) and are
// counted in *fallbacks.
constexpr int kFsaiMaxP = 12;

__global__ void __launch_bounds__(128) fsai_kernel(int n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const double* __restrict__ val,
                                                   const int* __restrict__ rpt, const int* __restrict__ rowt,
                                                   const int* __restrict__ perm, double* g_out,
                                                   int* fallbacks) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int a = __ldg(rpt + j), e = __ldg(rpt + j + 1);
    const int m = e - a;
    double L[kFsaiMaxP * (kFsaiMaxP + 1) / 2];  // packed lower triangle, row-major
    double y[kFsaiMaxP];
    bool ok = m >= 1 && m <= kFsaiMaxP && __ldg(rowt + a) == j;
    if (ok) {
      // L = chol(A[P, P]), row by row
      for (int r = 0; r < m && ok; ++r) {
        const int pr = __ldg(rowt + a + r);
        for (int q = 0; q <= r; ++q) {
          double sum = a_entry(rowptr, col, val, pr, __ldg(rowt + a + q));
          for (int t = 0; t < q; ++t) sum -= L[r * (r + 1) / 2 + t] * L[q * (q + 1) / 2 + t];
          if (q < r) {
            L[r * (r + 1) / 2 + q] = sum / L[q * (q + 1) / 2 + q];
          } else {
            if (!(sum > 0.0) || !isfinite(sum)) {
              ok = false;
              break;
            }
            L[r * (r + 1) / 2 + r] = sqrt(sum);
          }
        }
      }
    }
    if (ok) {
      // L L^T y = e_1: forward (z = L^{-1} e_1), then backward
      for (int r = 0; r < m; ++r) {
        double sum = r == 0 ? 1.0 : 0.0;
        for (int t = 0; t < r; ++t) sum -= L[r * (r + 1) / 2 + t] * y[t];
        y[r] = sum / L[r * (r + 1) / 2 + r];
      }
      for (int r = m - 1; r >= 0; --r) {
        double sum = y[r];
        for (int t = r + 1; t < m; ++t) sum -= L[t * (t + 1) / 2 + r] * y[t];
        y[r] = sum / L[r * (r + 1) / 2 + r];
      }
      ok = y[0] > 0.0 && isfinite(y[0]);
    }
    if (ok) {
      const double inv = 1.0 / sqrt(y[0]);
      for (int r = 0; r < m; ++r) g_out[__ldg(perm + a + r)] = y[r] * inv;
    } else {
      const double d = a_entry(rowptr, col, val, j, j);
      for (int r = 0; r < m; ++r)
        g_out[__ldg(perm + a + r)] = (__ldg(rowt + a + r) == j && d > 0.0) ? 1.0 / sqrt(d) : 0.0;
      if (fallbacks) atomicAdd(fallbacks, 1);
    }
  }
}
}  // namespace
}  // namespace sla

extern "C" int32_t sla_fsai_factor(const sla_csr* A, const double* val, const sla_csr* G, const sla_csr_t* GT,
                                   double* g_out, int32_t* fallbacks, void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr || A->n != G->n || A->n < 0 || G->nnz < 0)
    return SLA_ERR_INVALID;
  if (A->n == 0 || G->nnz == 0) return SLA_OK;
  if (A->rowptr == nullptr || A->col == nullptr || val == nullptr || GT->rowptr_t == nullptr ||
      GT->col_t == nullptr || GT->perm_t == nullptr || g_out == nullptr)
    return SLA_ERR_INVALID;
  if (ranges_overlap(val, 8 * (size_t)A->nnz, g_out, 8 * (size_t)G->nnz)) return SLA_ERR_INVALID;
  const int n = A->n;
  cudaStream_t s = (cudaStream_t)stream;
  if (fallbacks) SLA_CUDA_TRY(cudaMemsetAsync(fallbacks, 0, sizeof(int32_t), s));
  fsai_kernel<<<grid_rows(n, 128), 128, 0, s>>>(n, A->rowptr, A->col, val, GT->rowptr_t, GT->col_t, GT->perm_t,
                                                g_out, fallbacks);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_ggt_normalize(const sla_csr* A, const double* val, const sla_csr* G, const sla_csr_t* GT,
                                     const double* g_val, double* g_out, void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr || A->n != G->n || A->n < 0 || G->nnz < 0)
    return SLA_ERR_INVALID;
  if (A->n == 0 || G->nnz == 0) return SLA_OK;
  if (A->rowptr == nullptr || A->col == nullptr || val == nullptr || GT->rowptr_t == nullptr ||
      GT->col_t == nullptr || GT->perm_t == nullptr || g_val == nullptr || g_out == nullptr)
    return SLA_ERR_INVALID;
  const int n = A->n;
  cudaStream_t s = (cudaStream_t)stream;
  ggt_normalize_kernel<<<grid_rows(n, 256), 256, 0, s>>>(n, A->rowptr, A->col, val, GT->rowptr_t, GT->col_t,
                                                          GT->perm_t, g_val, g_out);
  MP_LAUNCH_CHECK();
  return SLA_OK;
}

extern "C" int32_t sla_ggt_normalize_bwd(const sla_csr* A, const double* val, const sla_csr* G,
                                         const sla_csr_t* GT, const double* g_val, const double* dGn, double* dG,
                                         void* stream) {
  if (A == nullptr || G == nullptr || GT == nullptr || A->n != G->n || A->n < 0 || G->nnz < 0)
    return SLA_ERR_INVALID;
  if (A->n == 0 || G->nnz == 0) return SLA_OK;
  if (A->rowptr == nullptr || A->col == nullptr || val == nullptr || GT->rowptr_t == nullptr ||
      GT->col_t == nullptr || GT->perm_t == nullptr || g_val == nullptr || dGn == nullptr || dG == nullptr)
    return SLA_ERR_INVALID;
  // dG may be dGn, but neither may overlap the forward's input values
  if (ranges_overlap(dG, 8 * (size_t)G->nnz, g_val, 8 * (size_t)G->nnz)) return SLA_ERR_INVALID;
  if (dG != dGn && ranges_overlap(dG, 8 * (size_t)G->nnz, dGn, 8 * (size_t)G->nnz)) return SLA_ERR_INVALID;
  const int n = A->n;
  // a column left unchanged passes dGn through: start from a copy
  if (dG != dGn) SLA_CUDA_TRY(cudaMemcpyAsync(dG, dGn, 8 * (size_t)G->nnz, cudaMemcpyDeviceToDevice,
                                              (cudaStream_t)stream));
  ggt_normalize_bwd_kernel<<<grid_rows(n, 256), 256, 0, (cudaStream_t)stream>>>(
      n, A->rowptr, A->col, val, GT->rowptr_t, GT->col_t, GT->perm_t, g_val, dGn, dG);
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
