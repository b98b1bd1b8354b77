// sla_workspace.h -- device workspace layouts (host + device visible).
//
// Every solver carves the caller-provided workspace into a call descriptor,
// a device-side solver state (scalars, phase, ticket counters), per-block
// partial sums and the Krylov work vectors.  All offsets are multiples of
// 256 bytes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "sla.h"

namespace sla {

constexpr int kMaxBlocks = 2048;   // cap on the grid of every reducing kernel
constexpr int kPartSlots = 4;      // partial-sum arrays of kMaxBlocks doubles

// Solver phase (CgState::phase).
enum : int { kPhaseRun = 0, kPhaseCheck = 1, kPhaseDone = 2 };

// Per-call arguments, written to device memory before the cached graph runs,
// so that one instantiated graph serves every call with the same workspace.
struct KrylovDesc {
  int n, nnz;
  const int* rowptr;
  const int* col;
  const double* val;
  const double* b;
  double* x;
  sla_info* info;
  double rtol, atol;
  int max_iter, max_restarts, precond, use_x0;
  // CSR of A^T for the BiCGStab adjoint (unused by CG); for G G^T PCG the
  // CSR of G^T (perm_t into g_val)
  const int* rowptr_t;
  const int* col_t;
  const int* perm_t;
  // lower-triangular factor G of M^{-1} = G G^T (precond SLA_PRECOND_GGT)
  const int* g_rowptr;
  const int* g_col;
  const double* g_val;
  int nnz_g;
  // CG per-phase kernels (sla_cg.cu) with the Jacobi preconditioner: 1 = run
  // CG on D^{-1/2} A D^{-1/2} (its values in the workspace), 0 = PCG on A
  int sym_scale;
};

// Device-side solver scalars.  Counters are reset by the last block of the
// kernel that uses them.
struct KrylovState {
  double rho, pq, rr, bnorm, thresh, alpha, beta, omega;
  double rho_prev, tt, ts, ss;
  int iters, status, phase, restarts, body, zero_rhs, bad_diag, err;
  int fresh_p, pad2;
  unsigned cnt[8];
};

struct CgLayout {
  size_t desc, state, part, r, z, p, q, dinv, total;
};

constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

constexpr CgLayout cg_layout(int n) {
  CgLayout L{};
  size_t o = 0;
  const size_t vec = al256(sizeof(double) * (size_t)(n > 0 ? n : 1));
  L.desc = o;  o += al256(sizeof(KrylovDesc));
  L.state = o; o += al256(sizeof(KrylovState));
  L.part = o;  o += al256(sizeof(double) * kMaxBlocks * kPartSlots);
  L.r = o;     o += vec;
  L.z = o;     o += vec;
  L.p = o;     o += vec;
  L.q = o;     o += vec;
  L.dinv = o;  o += vec;
  L.total = o;
  return L;
}

// CG scratch of the per-phase kernels: the layout above, then the values of
// D^{-1/2} A D^{-1/2} (nnz doubles).
inline size_t cg_ws_bytes(int n, int nnz) {
  return al256(cg_layout(n).total) + al256(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
}

// Pipelined Jacobi PCG (sla_cg_pipe.cu): descriptor, state, partials, the
// per-row records (r, w, z, s, p, dinv: 6 doubles a row), two m buffers.
struct CgPipeLayout {
  size_t desc, state, part, rec, m0, m1, total;
};

constexpr CgPipeLayout cg_pipe_layout(int n) {
  CgPipeLayout L{};
  size_t o = 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  L.desc = o;  o += al256(sizeof(KrylovDesc));
  L.state = o; o += al256(sizeof(KrylovState));
  L.part = o;  o += al256(sizeof(double) * kMaxBlocks * kPartSlots);
  L.rec = o;   o += al256(sizeof(double) * 6 * nn);
  L.m0 = o;    o += al256(sizeof(double) * nn);
  L.m1 = o;    o += al256(sizeof(double) * nn);
  L.total = o;
  return L;
}

// BiCGStab: descriptor, state, partials, then r, r^, p, p^, v, s, s^, t, dinv.
struct BiLayout {
  size_t desc, state, part, vec, vec_stride, total;
};

constexpr BiLayout bicg_layout(int n) {
  BiLayout L{};
  size_t o = 0;
  L.vec_stride = al256(sizeof(double) * (size_t)(n > 0 ? n : 1));
  L.desc = o;  o += al256(sizeof(KrylovDesc));
  L.state = o; o += al256(sizeof(KrylovState));
  L.part = o;  o += al256(sizeof(double) * kMaxBlocks * kPartSlots);
  L.vec = o;   o += 9 * L.vec_stride;
  L.total = o;
  return L;
}

// BiCGStab scratch: the layout above, then A D^{-1} (nnz doubles).
inline size_t bicg_ws_bytes(int n, int nnz) {
  return al256(bicg_layout(n).total) + al256(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
}

// Batched solves (sla_batched.cu); argument = total rows of the batch.
size_t batched_ws_bytes(long long total_rows);

// Batched adjoint (sla_adjoint_batched.cu): the batched solve's scratch,
// then the values of every A_s^T (total entries of the batch, doubles).
inline size_t adjoint_batched_ws_bytes(long long total_rows, long long total_nnz) {
  return al256(batched_ws_bytes(total_rows)) +
         al256(sizeof(double) * (size_t)(total_nnz > 0 ? total_nnz : 1));
}

// G G^T-preconditioned CG: descriptor, state, partials, r, z, p, q, t, then
// the FP32 values of G and of G^T (nnz_g floats each).
struct GgtLayout {
  size_t desc, state, part, r, z, p, q, t, gv, gtv, total;
};

constexpr GgtLayout ggt_layout(int n, int nnz_g) {
  GgtLayout L{};
  size_t o = 0;
  const size_t vec = al256(sizeof(double) * (size_t)(n > 0 ? n : 1));
  L.desc = o;  o += al256(sizeof(KrylovDesc));
  L.state = o; o += al256(sizeof(KrylovState));
  L.part = o;  o += al256(sizeof(double) * kMaxBlocks * kPartSlots);
  L.r = o;     o += vec;
  L.z = o;     o += vec;
  L.p = o;     o += vec;
  L.q = o;     o += vec;
  L.t = o;     o += vec;
  L.gv = o;    o += al256(sizeof(float) * (size_t)(nnz_g > 0 ? nnz_g : 1));
  L.gtv = o;   o += al256(sizeof(float) * (size_t)(nnz_g > 0 ? nnz_g : 1));
  L.total = o;
  return L;
}

// Several right-hand sides sharing one matrix (sla_multi.cu).
size_t multi_ws_bytes(int n, int k);

// LOBPCG (sla_eig.cu): k = block size; optional outputs: grid sizes.
size_t eig_ws_bytes(int n, int k, int* gram_blocks, int* upd_blocks);

// Eigenvector adjoint (sla_eig_adjoint.cu): k pairs.
size_t eigvec_ws_bytes(int n, int k);

// Merge-path SpMV carries (sla_spmv_merge.cu).
size_t spmv_merge_ws_bytes(int n, long long nnz);

// Pattern utilities (sla_pattern.cu).
size_t transpose_ws_bytes(int n, int nnz);
size_t list_transpose_ws_bytes(int total_rows, int total_nnz);
size_t coo_ws_bytes(int n, long long m);

// Adjoint: the larger of the CG scratch (either form) and BiCGStab scratch
// + valT.
inline size_t adjoint_ws_bytes(int n, int nnz) {
  const size_t a0 = cg_ws_bytes(n, nnz), a1 = cg_pipe_layout(n).total;
  const size_t a = a0 > a1 ? a0 : a1;
  const size_t b = bicg_ws_bytes(n, nnz) + al256(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  return a > b ? a : b;
}

inline bool workspace_bytes(int kind, int n, int nnz, int batch, size_t* out) {
  (void)nnz;
  (void)batch;
  switch (kind) {
    case SLA_WS_CG:
      *out = cg_ws_bytes(n, nnz);
      return true;
    case SLA_WS_CG_PIPELINED:
      *out = cg_pipe_layout(n).total;
      return true;
    case SLA_WS_EIGSH:
      if (batch < 1 || batch > SLA_EIG_MAX_K) return false;
      *out = eig_ws_bytes(n, batch, nullptr, nullptr);
      return true;
    case SLA_WS_EIG_ADJOINT:
      if (batch < 1 || batch > SLA_EIG_MAX_K) return false;
      *out = eigvec_ws_bytes(n, batch);
      return true;
    case SLA_WS_BICGSTAB:
      *out = bicg_ws_bytes(n, nnz);
      return true;
    case SLA_WS_ADJOINT:
      *out = adjoint_ws_bytes(n, nnz);
      return true;
    case SLA_WS_TRANSPOSE:
      *out = transpose_ws_bytes(n, nnz);
      return true;
    case SLA_WS_LIST_TRANSPOSE:
      *out = list_transpose_ws_bytes(n, nnz);  // n = total rows, nnz = total entries
      return true;
    case SLA_WS_COO:
      *out = coo_ws_bytes(n, nnz);
      return true;
    case SLA_WS_CG_GGT:
      *out = ggt_layout(n, nnz).total;  // nnz = entries of G
      return true;
    case SLA_WS_SPMV_MERGE:
      *out = spmv_merge_ws_bytes(n, nnz);
      return true;
    case SLA_WS_CG_MULTI:
      *out = multi_ws_bytes(n, batch);
      return true;
    case SLA_WS_BATCHED:
      *out = batched_ws_bytes((long long)n * (batch > 0 ? batch : 1));
      return true;
    case SLA_WS_ADJOINT_BATCHED:
      *out = adjoint_batched_ws_bytes((long long)n * (batch > 0 ? batch : 1),
                                      (long long)nnz * (batch > 0 ? batch : 1));
      return true;
    default:
      return false;
  }
}

}  // namespace sla
