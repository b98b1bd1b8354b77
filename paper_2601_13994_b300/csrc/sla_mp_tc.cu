// sla_mp_tc.cu -- the dense layers of the learned preconditioner's network
// on the fifth-generation tensor cores (tcgen05.mma, accumulator in TMEM).
//
// Y = [X1 | X2] W^T (+ b, relu, residual) is a contraction of n rows with
// K <= 64 inputs and M <= 96 outputs: [n x K] x [K x M].  The weights are
// BF16 (the network's storage format); the activations are FP32.  The MMA
// takes BF16 operands, so each activation x is split exactly into three
// BF16 pieces, x = x1 + x2 + x3 (x1 = bf16(x), x2 = bf16(x - x1),
// x3 = bf16(x - x1 - x2): 3 x 8 significand bits cover FP32's 24), and
// the layer runs as one MMA chain over K' = 3 Kp with the weights repeated
// three times: sum_p sum_k x_p[k] w[k].  A product of two BF16 values is
// exact in FP32, so the result is the FP32 contraction up to the order of
// the FP32 additions (the tensor core accumulates in FP32).
//
// Per 128-row tile (the MMA's M): the CTA's 128 threads load the tile's
// activations with 16-byte loads, split them and store the pieces to shared
// memory in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices; LBO = 128 bytes between core matrices along K, SBO = K' * 16
// bytes between 8-row groups); one thread issues K'/16 tcgen05.mma (M = 128,
// N = M_out, K = 16 each) into a TMEM accumulator of M_out FP32 columns and
// commits them to an mbarrier; every warp then reads its 32 TMEM lanes (the
// tile's rows 32w .. 32w + 31) with tcgen05.ld and applies bias, relu and
// residual in registers.  Persistent CTAs walk the tiles; the weights are
// staged once per CTA.  The mbarrier wait is bounded: on timeout the kernel
// sets an error flag, stops taking tiles, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "sla_internal.cuh"
#include "sla_tma.cuh"

namespace sla {
namespace {

using tma::mbar_init;
using tma::mbar_wait;
using tma::smem_addr;

constexpr int kTcRows = 128;     // rows per tile: the MMA's M
constexpr int kTcThreads = 128;  // 4 warps: warp w owns TMEM lanes 32w .. 32w + 31
constexpr int kTcMaxK = 64;      // largest K1 + K2
constexpr int kTcMaxN = 96;      // largest M_out
constexpr int kTcParts = 3;      // BF16 pieces of an FP32 activation
// row stride (floats) of a warp's 32 x 32 output stage: 16-byte aligned rows,
// a warp's 16-byte writes of 32 rows in the 4 wavefronts they need
constexpr int kTcStage = 36;
// (8-row group, 4-chunk group) items of a tile per warp at the largest K
constexpr int kTcFill = (kTcRows / 8) * (kTcMaxK / 16) / (kTcThreads / 32);

__device__ int g_tc_err;  // nonzero once an mbarrier wait ran out (read by sla_mp_tc_errors)

// byte offset of element (r, k) in a K-major no-swizzle operand whose rows
// hold kt elements (kt a multiple of 16): 8 x 16-byte core matrices, the
// core matrices of an 8-row group side by side along K (128 bytes apart),
// the 8-row groups kt * 16 bytes apart
__device__ __forceinline__ uint32_t core_off(int r, int k, int kt) {
  return (uint32_t)((r >> 3) * (kt * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor of tcgen05 (no swizzle): start address,
// leading-dimension byte offset (along K), stride byte offset (along M/N),
// each >> 4; descriptor version 1 in bits 46-47; layout type 0 (none)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator (bits
// 4-5 = 1), BF16 A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 =
// 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (lane l: row l)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// the three BF16 pieces of x (their sum is x exactly for finite x)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  c = __float2bfloat16_rn(r2);
}

// two BF16 values in one 32-bit word, the first in the low half (memory order)
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct TcArgs {
  int n, K1, K2, M, relu;
  const float* X1;
  const float* X2;
  const __nv_bfloat16* W;  // [M][K1 + K2]
  const float* bias;       // [M] or null
  const float* R;          // [n][M] or null
  float* Ypre;             // [n][M] or null
  float* Y;                // [n][M]
};

// Bytes of the A' tile (or of the output stages, which reuse it once the
// MMA has read it, whichever is larger) for inputs padded to KP.
__host__ __device__ constexpr int tc_a_bytes(int kp) {
  return kTcRows * kTcParts * kp * 2 > kTcThreads * kTcStage * 4 ? kTcRows * kTcParts * kp * 2
                                                                   : kTcThreads * kTcStage * 4;
}

// dynamic shared memory: the A' tile [128][K'] (core layout; the four warps'
// output stages [32][kTcStage] floats alias it after the MMA), then B'
// [M][K'].  KP = K1 + K2 rounded up to 16, a template argument so that the
// tile loops and core-matrix offsets are compile-time.
template <int KP>
__global__ void __launch_bounds__(kTcThreads, 3) dense_tc_kernel(TcArgs a) {
  constexpr int Kt = kTcParts * KP;                    // K'
  constexpr int kCg = KP / 16;                         // groups of four 16-byte chunks per row
  constexpr int kFill = (kTcRows / 8) * kCg / (kTcThreads / 32);  // items per warp per tile
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  __shared__ unsigned long long bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = a.K1 + a.K2;
  const int N = a.M;
  const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
  unsigned char* As = tc_dyn;
  unsigned char* Bs = tc_dyn + tc_a_bytes(KP);
  float* stage = reinterpret_cast<float*>(tc_dyn) + warp * 32 * kTcStage;

  // weights, three times along K' (zero beyond K)
  for (int idx = tid; idx < N * Kt; idx += kTcThreads) {
    const int nn = idx / Kt, kk = idx - nn * Kt;
    const int k = kk % KP;
    const __nv_bfloat16 w = k < K ? a.W[(size_t)nn * K + k] : __float2bfloat16_rn(0.0f);
    *reinterpret_cast<__nv_bfloat16*>(Bs + core_off(nn, kk, Kt)) = w;
  }
  if (warp == 0) {
    tc_alloc(&tmem_base, ncols);
    tc_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t a_addr = smem_addr(As), b_addr = smem_addr(Bs);
  constexpr uint32_t sbo = (uint32_t)Kt * 16u;
  const uint32_t idesc = idesc_bf16(kTcRows, N);
  const int tiles = (a.n + kTcRows - 1) / kTcRows;
  // item u of warp w: 8-row group rg, chunk group cg; lane: row rg * 8 +
  // (lane & 7), chunk cg * 4 + (lane >> 3) (16 bytes at k = 16 cg + 4 (lane >> 3))
  const int kl = 4 * (lane >> 3), rl = lane & 7;
  // a tile's activations into registers: all of a thread's 16-byte loads
  // in flight together
  float4 buf[kFill];
  auto load_tile = [&](int tt) {
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int q = warp + u * (kTcThreads / 32);
      const int rg = q / kCg, cg = q % kCg;
      const int k = 16 * cg + kl, i = tt * kTcRows + rg * 8 + rl;
      buf[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (tt < tiles && i < a.n && k < K)
        buf[u] = k < a.K1 ? *reinterpret_cast<const float4*>(a.X1 + (size_t)i * a.K1 + k)
                          : *reinterpret_cast<const float4*>(a.X2 + (size_t)i * a.K2 + (k - a.K1));
    }
  };
  load_tile(blockIdx.x);
  unsigned phase = 0;
  const int cq = lane & 7;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int r0 = t * kTcRows;
    // the tile's activations (in buf, loaded one tile ahead) -> three BF16
    // pieces in A' (2 x 128 contiguous bytes of each piece per warp item)
#pragma unroll
    for (int u = 0; u < kFill; ++u) {
      const int q = warp + u * (kTcThreads / 32);
      const int rg = q / kCg, cg = q % kCg;
      const int r = rg * 8 + rl, k = 16 * cg + kl;
      __nv_bfloat16 x0, x1, x2, y0, y1, y2, z0, z1, z2, w0, w1, w2;
      split3(buf[u].x, x0, x1, x2);
      split3(buf[u].y, y0, y1, y2);
      split3(buf[u].z, z0, z1, z2);
      split3(buf[u].w, w0, w1, w2);
      *reinterpret_cast<uint2*>(As + core_off(r, k, Kt)) = make_uint2(pack2(x0, y0), pack2(z0, w0));
      *reinterpret_cast<uint2*>(As + core_off(r, KP + k, Kt)) = make_uint2(pack2(x1, y1), pack2(z1, w1));
      *reinterpret_cast<uint2*>(As + core_off(r, 2 * KP + k, Kt)) = make_uint2(pack2(x2, y2), pack2(z2, w2));
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < Kt / 16; ++kk) {
        const uint64_t ad = smem_desc(a_addr + (uint32_t)kk * 256u, 128u, sbo);
        const uint64_t bd = smem_desc(b_addr + (uint32_t)kk * 256u, 128u, sbo);
        tc_mma(tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
      }
      tc_commit(&bar);
    }
    __syncwarp();
    load_tile(t + gridDim.x);  // the next tile's loads run under this tile's MMA and epilogue
    // one thread polls the MMA's mbarrier; the others wait at the block
    // barrier, taking no issue slots from the SM's other CTAs
    bool ok = true;
    if (tid == 0) ok = mbar_wait(&bar, phase, &g_tc_err);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) break;
    tc_fence_after();
    // epilogue, 32 columns at a time: warp w reads its TMEM lanes (lane l:
    // row r0 + 32 w + l) into registers and through its shared-memory stage
    // (over A', which the MMA has consumed) writes them out row-major with
    // coalesced 16-byte accesses (8 lanes a row, 4 rows per instruction),
    // adding bias, relu and residual there
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4*>(stage + lane * kTcStage + 4 * c) =
            make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      __syncwarp();
      const int col = c0 + 4 * cq;
      if (col < N) {
        float4 bb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (a.bias) bb = make_float4(a.bias[col], a.bias[col + 1], a.bias[col + 2], a.bias[col + 3]);
        float4 rv[8];  // the residual rows, loaded before the first store
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int i = r0 + 32 * warp + 4 * it + (lane >> 3);
          rv[it] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if (a.R && i < a.n) rv[it] = *reinterpret_cast<const float4*>(a.R + (size_t)i * N + col);
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int rr = 4 * it + (lane >> 3);
          const int i = r0 + 32 * warp + rr;
          if (i < a.n) {
            float4 acc = *reinterpret_cast<const float4*>(stage + rr * kTcStage + 4 * cq);
            acc.x += bb.x;
            acc.y += bb.y;
            acc.z += bb.z;
            acc.w += bb.w;
            const size_t o = (size_t)i * N + col;
            if (a.Ypre) *reinterpret_cast<float4*>(a.Ypre + o) = acc;
            if (a.relu) {
              acc.x = fmaxf(acc.x, 0.0f);
              acc.y = fmaxf(acc.y, 0.0f);
              acc.z = fmaxf(acc.z, 0.0f);
              acc.w = fmaxf(acc.w, 0.0f);
            }
            acc.x += rv[it].x;
            acc.y += rv[it].y;
            acc.z += rv[it].z;
            acc.w += rv[it].w;
            *reinterpret_cast<float4*>(a.Y + o) = acc;
          }
        }
      }
      __syncwarp();  // the stage is rewritten for the next 32 columns
    }
    tc_fence_before();
    __syncthreads();  // TMEM read and the stages consumed before the next tile's A' and MMA
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, ncols);
  }
}

}  // namespace

// The tensor-core form of sla_mp_dense_fwd applies when both inputs are
// 16-byte aligned with K1, K2 multiples of 4, K1 + K2 <= 64, M a multiple of
// 16 up to 96 and Y (and Ypre, R) 16-byte aligned.
bool mp_dense_tc_applies(int K1, const float* X1, int K2, const float* X2, int M, const float* R,
                         const float* Ypre, const float* Y) {
  const uintptr_t al = (uintptr_t)X1 | (uintptr_t)X2 | (uintptr_t)R | (uintptr_t)Ypre | (uintptr_t)Y;
  return K1 % 4 == 0 && K2 % 4 == 0 && K1 + K2 >= 1 && K1 + K2 <= kTcMaxK && M % 16 == 0 && M >= 16 &&
         M <= kTcMaxN && (al & 15u) == 0;
}

namespace {
template <int KP>
int launch_tc(const TcArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)tc_a_bytes(KP) + (size_t)a.M * kTcParts * KP * 2;
  static bool attr_set = false;
  if (!attr_set) {
    const int mx = tc_a_bytes(KP) + kTcMaxN * kTcParts * KP * 2;
    SLA_CUDA_TRY(cudaFuncSetAttribute(dense_tc_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SLA_CUDA_TRY(cudaFuncSetAttribute(dense_tc_kernel<KP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
    attr_set = true;
  }
  // resident CTAs per SM from the kernel's registers and shared memory
  // (the occupancy query returned 1 here, where three fit); no CTA waits
  // on another, so an over-estimate would only add a second wave
  static int regs = 0, smem_sm = 0, static_smem = 0;
  if (regs == 0) {
    cudaFuncAttributes fa;
    SLA_CUDA_TRY(cudaFuncGetAttributes(&fa, dense_tc_kernel<KP>));
    regs = fa.numRegs > 0 ? fa.numRegs : 255;
    static_smem = (int)fa.sharedSizeBytes;
    SLA_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, current_device()));
  }
  const int by_regs = 65536 / (((regs + 7) & ~7) * kTcThreads);
  const int by_smem = smem_sm / ((int)smem + static_smem + 1024);
  int occ = by_regs < by_smem ? by_regs : by_smem;
  if (occ > 4) occ = 4;  // at most 4 x 128 TMEM columns on an SM
  if (occ < 1) occ = 1;
  const int tiles = (a.n + kTcRows - 1) / kTcRows;
  const int slots = num_sms(current_device()) * occ;
  dense_tc_kernel<KP><<<tiles < slots ? tiles : slots, kTcThreads, smem, s>>>(a);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
}  // namespace

int mp_dense_fwd_tc(int n, int K1, const float* X1, int K2, const float* X2, int M, const __nv_bfloat16* W,
                    const float* bias, const float* R, int relu, float* Ypre, float* Y, cudaStream_t s) {
  const TcArgs a{n, K1, K2, M, relu, X1, X2, W, bias, R, Ypre, Y};
  switch ((K1 + K2 + 15) / 16) {
    case 1: return launch_tc<16>(a, s);
    case 2: return launch_tc<32>(a, s);
    case 3: return launch_tc<48>(a, s);
    case 4: return launch_tc<64>(a, s);
    default: return SLA_ERR_INVALID;
  }
}

}  // namespace sla

using namespace sla;

// Nonzero when a tensor-core dense launch's mbarrier wait ran out since the
// last call (synchronous; resets the flag).
extern "C" int32_t sla_mp_tc_errors(int32_t* out) {
  if (out == nullptr) return SLA_ERR_INVALID;
  int v = 0;
  SLA_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_err, sizeof(int)));
  const int z = 0;
  SLA_CUDA_TRY(cudaMemcpyToSymbol(g_tc_err, &z, sizeof(int)));
  *out = v;
  return SLA_OK;
}
