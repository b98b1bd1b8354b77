// sla_eig.cu -- the k smallest eigenpairs of a symmetric positive definite
// CSR matrix by LOBPCG (the eigensolver Sec. 3.3 names, Knyazev 2001) with
// the Jacobi preconditioner, and the Hellmann-Feynman eigenvalue gradient
// d lambda / d A_ij = v_i v_j on the pattern (Sec. 3.2, Eq. 4).
//
// One iteration, with X the current Ritz block (n x kb, X^T X = I), W = D^{-1}
// R the preconditioned residuals and P the previous search directions:
//   S = [X W P], AS = [AX AW AP]  (AW = A W is the iteration's SpMM; AX and
//   AP are carried);
//   G = S^T S, H = S^T A S over the m active columns (kb, 2kb or 3kb);
//   Rayleigh-Ritz: the kb smallest eigenpairs (theta, C) of H c = theta G c;
//   X' = S C, AX' = AS C, P' = S[:, kb:] C[kb:, :], AP' likewise;
//   R = AX' - X' diag(theta), converged when ||r_i|| <= tol |theta_i| ||x_i||
//   for the k wanted pairs; W' = D^{-1} R.
// Soft locking: a pair whose residual has met the tolerance keeps its X
// column but its W and P columns leave the basis (their rows and columns of
// G and H are zeroed, so the scaling gives them no weight) -- otherwise the
// rounding noise of a converged pair's residual, scaled to unit norm,
// degrades the other pairs (1D Laplacian n = 200, k = 6: the largest
// residual fell to 2.7e-8 and then rose to 1e-6 without locking).
// The block carries kb = min(k + 2, n) vectors, two guard vectors beyond
// the k wanted, so that a cluster of eigenvalues split at the k-th does not
// stall the last wanted vector (3D 32^3 with lambda_5..7 = 0.0934, 0.0938,
// 0.0950 and k = 6: without guards LOBPCG took from 551 to more than 3000
// iterations depending on the start block; with two, 316-458).
// The Rayleigh-Ritz step: the columns of S are scaled to unit norm; a basis
// B with B^T G B = I comes from the Cholesky factor of the scaled G (B =
// L^{-T}), or -- when a pivot shows near dependence between X, W and P,
// which grows as the iteration converges -- from its eigendecomposition with
// the directions below 1e-12 of the largest eigenvalue dropped; the
// projected H = B^T H B is then diagonalised.  The small symmetric
// eigenproblems (m <= 30) are FP32 cyclic Jacobi sweeps with the round-robin
// ordering that makes the m/2 rotations of a step independent, then FP64
// iterative refinement (eig_eigh).  The whole step runs on one thread-block
// cluster: every CTA repeats the sequential parts on its own copy of the
// small matrices, and the FP64 products are split over the CTAs.
//
// Kernels of an iteration: SpMM (A W), Gram (block partial sums of G and H),
// Gram totals (fixed-order sums over the Gram blocks; the last cluster to
// arrive runs the Rayleigh-Ritz step), update (X', P', R, W' and the
// residual norms; the last block takes the convergence decision).  The host launches them in a
// loop and reads the device state every few iterations; once the state says
// done, further launches return at once.  S and AS are row-major [n][3k]
// and double-buffered (the update reads one pair and writes the other).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cooperative_groups.h>

#include "sla_internal.cuh"
#include "sla_workspace.h"

namespace sla {

constexpr int kEigMaxK = SLA_EIG_MAX_K;          // wanted pairs, at most 8
constexpr int kEigMaxB = kEigMaxK + 2;           // block with two guard vectors
constexpr int kEigMaxM = 3 * kEigMaxB;           // 30 columns of S
constexpr int kEigLd = kEigMaxM + 1;      // leading dimension of the small matrices
constexpr int kEigThreads = 256;
// The update kernel's block (one thread per row and output column)
constexpr int kEigUpdThreads = 256;
constexpr int kEigTile = 32;              // rows of S staged per Gram tile
constexpr int kEigPairs = kEigMaxM * (kEigMaxM + 1) / 2;
constexpr int kEigPollEvery = 8;
// The Rayleigh-Ritz step runs on one thread-block cluster of kRrCluster
// CTAs (one SM each): every CTA holds the small matrices in its own shared
// memory and repeats the sequential parts (Cholesky, the FP32 Jacobi sweeps),
// whose results are bit-identical in every CTA since they are the same
// operations on the same data; the dense m x m products -- FP64-bound on one
// SM, whose FP64 pipe retires two lane operations per clock -- are split by
// columns (CTA c owns the columns j with j mod kRrCluster = c) and the owned
// columns are written to every CTA's copy through distributed shared memory.
constexpr int kRrCluster = 8;
// blocks of the Gram totals (32 values each), a whole number of clusters
constexpr int kRrBlocks = ((2 * kEigPairs + 31) / 32 + kRrCluster - 1) / kRrCluster * kRrCluster;

struct EigDesc {
  int n, nnz, k, kb, ld, max_iter, precond, use_x0;
  double tol;
  const int* rowptr;
  const int* col;
  const double* val;
  double* lambda;
  double* V;
  sla_info* info;
};

struct EigState {
  int m;      // columns of S in the next Rayleigh-Ritz step
  int cur;    // which S / AS buffer holds the current block
  int iters, done, status, rank, bad;
  unsigned active;  // bit j: pair j not yet converged (its W, P in the basis)
  double maxres;
  unsigned ticket_gram, ticket_upd, ticket_fin;
};

struct EigPtrs {
  EigDesc* d;
  EigState* st;
  double* dinv;
  double* S[2];
  double* AS[2];
  double* gpart;   // [blocks][2 * kEigPairs]
  double* gtot;    // [2 * kEigPairs]
  double* upart;   // [blocks + 1][2 * kEigMaxB]
  double* C;       // [kEigMaxM][kEigMaxB]
  double* theta;   // [kEigMaxM]
};

size_t eig_ws_bytes(int n, int k, int* gram_blocks, int* upd_blocks);

// Counter-based start block when no initial guess is given: splitmix64 of
// the entry index, mapped to [-1, 1).
__device__ __forceinline__ double eig_start_value(unsigned long long idx) {
  unsigned long long z = idx + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

__global__ void eig_arm_kernel(EigState* st) {
  st->m = 0;
  st->cur = 0;
  st->iters = 0;
  st->done = 0;
  st->status = SLA_NOT_CONVERGED;
  st->rank = 0;
  st->bad = 0;
  st->active = 0xffffffffu;
  st->maxres = NAN;
  st->ticket_gram = st->ticket_upd = st->ticket_fin = 0u;
}

// D^{-1} (or ones) and the start block X0 into S[0][:, 0:kb]: the caller's
// k columns with use_x0, the counter-based values otherwise and for guards.
__global__ void eig_init_kernel(EigPtrs P) {
  const EigDesc& d = *P.d;
  const int n = d.n, k = d.k, kb = d.kb, ld = d.ld;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double di = 1.0;
    if (d.precond == SLA_PRECOND_JACOBI) {
      double diag = 0.0;
      for (int e = d.rowptr[i]; e < d.rowptr[i + 1]; ++e)
        if (d.col[e] == i) diag += d.val[e];
      if (!(diag > 0.0)) atomicOr(&P.st->bad, 1);
      di = 1.0 / diag;
    }
    P.dinv[i] = di;
    double* s = P.S[0] + (size_t)i * ld;
    for (int j = 0; j < kb; ++j)
      s[j] = (d.use_x0 && j < k) ? d.V[(size_t)i * k + j] : eig_start_value((unsigned long long)i * kb + j);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) P.st->m = kb;
}

// Y[:, dst_off + j] = A X[:, src_off + j], j < kb, one row per thread.
// mode 0: X of S[cur] -> AS[cur] (start); 1: W of S[cur] -> AW in AS[cur];
// 2: X of S[cur] -> AS[cur ^ 1][:, 0:kb] (the final residual check).
__global__ void __launch_bounds__(kEigThreads) eig_spmm_kernel(EigPtrs P, int mode) {
  const EigDesc& d = *P.d;
  const EigState& st = *P.st;
  if (mode != 2 && (st.done || st.bad)) return;
  const int n = d.n, kb = d.kb, ld = d.ld, cur = st.cur;
  // every 16th iteration A X is recomputed too (X and W are adjacent columns),
  // so that the carried A X (A X' = A S C) cannot drift far from the product
  const bool refresh = mode == 1 && (st.iters & 15) == 15;
  const int parts = refresh ? 2 : 1;
  for (int part = 0; part < parts; ++part) {
  const int off = (mode == 1 && !refresh) ? kb : part * kb;
  const double* X = P.S[cur] + off;
  double* Y = (mode == 2 ? P.AS[cur ^ 1] : P.AS[cur]) + off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc[kEigMaxB];
#pragma unroll
    for (int j = 0; j < kEigMaxB; ++j) acc[j] = 0.0;
    const int a = __ldg(d.rowptr + i), e = __ldg(d.rowptr + i + 1);
    for (int q = a; q < e; ++q) {
      const double v = __ldg(d.val + q);
      const double* xr = X + (size_t)__ldg(d.col + q) * ld;
#pragma unroll
      for (int j = 0; j < kEigMaxB; ++j)
        if (j < kb) acc[j] = fma(v, xr[j], acc[j]);
    }
    double* yr = Y + (size_t)i * ld;
#pragma unroll
    for (int j = 0; j < kEigMaxB; ++j)
      if (j < kb) yr[j] = acc[j];
  }
  }
}

// ---------------------------------------------------------------- Rayleigh-Ritz

// Eigen-decomposition of the symmetric m x m matrix A (shared, leading
// dimension kEigLd) by cyclic Jacobi rotations in precision T: on return the
// diagonal of A holds the eigenvalues and the columns of V the eigenvectors.
// Round-robin pairing: in step r of a sweep, position x holds index 0
// (x = 0) or 1 + (x - 1 + r) mod (m' - 1), and positions x and m' - 1 - x
// form a pair, so the m'/2 rotations of a step touch disjoint rows and
// columns.  A pair is rotated only while |a_pq| > rel sqrt|a_pp a_qq| (the
// threshold rule of cyclic Jacobi) and |a_pq| > floor_rel max_j |a_jj|; the
// first sweep that rotates nothing, or sweep max_sweeps, ends the solve.
// (In FP64 no floor is used: an absolute floor of 1e-18 or 1e-16 of the
// largest diagonal entry of the scaled Gram matrix made LOBPCG stall at a
// residual of 1.4e-7 on the 1D Laplacian, n = 200, k = 6.)
// The Jacobi rotation (c, s) that annihilates a_pq, from d = a_qq - a_pp and
// e = 2 a_pq: tan = sgn(d e) |e| / (|d| + sqrt(d^2 + e^2)) (the smaller root
// of t^2 + 2 (d/e) t - 1 = 0), cos = 1 / sqrt(1 + tan^2), sin = tan cos.
// In FP32 directly.  In FP64 the tangent is taken in FP32 (the special-
// function unit, against FP64 division and square-root sequences at two
// lanes per clock per SM -- this computation is on every step's critical
// path) and (c, s) are then scaled to unit norm by two Newton steps of
// y <- y (3 - (c^2 + s^2) y^2) / 2 in FP64, so the rotation is orthogonal to
// FP64 rounding; its angle is accurate to FP32, i.e. it leaves a_pq at
// ~1e-7 of its value, and the sweeps repeat until every a_pq passes the
// FP64 threshold (convergence is then linear with rate ~1e-7 per sweep).
__device__ __forceinline__ void rotation_of(float d, float e, float& c, float& s) {
  // special-function reciprocals and reciprocal square roots only (no IEEE
  // division or square-root sequences on the step's critical path): the
  // angle need only be accurate to a few FP32 ulps -- the sweeps repeat
  // until a_pq passes the threshold, and the FP64 refinement that follows
  // squares what error remains
  const float ad = fabsf(d), ae = fabsf(e);
  const float big = fmaxf(ad, ae), small = fminf(ad, ae);
  const float rr = __fdividef(small, big);  // in [0, 1]
  const float h2 = fmaf(rr, rr, 1.0f);      // in [1, 2]
  const float hyp = big * (h2 * rsqrtf(h2));
  float t = __fdividef(ae, ad + hyp);       // in [0, 1]
  if ((d < 0.0f) != (e < 0.0f)) t = -t;
  c = rsqrtf(fmaf(t, t, 1.0f));
  s = t * c;
}
__device__ __forceinline__ void rotation_of(double d, double e, double& c, double& s) {
  float cf, sf;
  rotation_of((float)d, (float)e, cf, sf);
  c = (double)cf;
  s = (double)sf;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double nrm = c * c + s * s;
    const double y = 0.5 * (3.0 - nrm);  // 1/sqrt(nrm) to second order, nrm = 1 + O(1e-7)
    c *= y;
    s *= y;
  }
}

template <class T>
__device__ void eig_jacobi(T* A, T* V, int m, T rel, T floor_rel, int max_sweeps, T* rot, int* s_any,
                           T* s_floor, unsigned short* items, int* stepf) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < m * kEigLd; q += nt) V[q] = T(0);
  __syncthreads();
  for (int q = tid; q < m; q += nt) V[q * kEigLd + q] = T(1);
  if (tid == 0) {
    T dmax = T(0);
    for (int j = 0; j < m; ++j) dmax = fmax(dmax, fabs(A[j * kEigLd + j]));
    *s_floor = floor_rel * dmax;
  }
  __syncthreads();
  const T floor_abs = *s_floor;
  const int mp = m + (m & 1);
  const int npair = mp / 2;
  // work items of a step: (row pair, column pair) blocks, then (row of V,
  // pair); x << 8 | y
  for (int t = tid; t < npair * npair + m * npair; t += nt) {
    int x, y;
    if (t < npair * npair) {
      x = t / npair;
      y = t - x * npair;
    } else {
      x = (t - npair * npair) / npair;
      y = (t - npair * npair) - x * npair;
    }
    items[t] = (unsigned short)((x << 8) | y);
  }
  __syncthreads();
  // The V update of a step runs in the next step's first phase, on every
  // warp but the first while warp 0 computes that step's rotations (the rotations
  // are double-buffered by step parity; V is read by no rotation), so the
  // second phase applies only A's blocks.  A step whose rotations are all
  // the identity leaves A and V as they are and skips its second phase.
  const int nblk = npair * npair, nv = m * npair;
  bool vpend = false;  // the previous step's V update is still to be applied
  int vpar = 0;        // its rotation buffer
  auto apply_v = [&](const T* rt) {
    for (int t = tid - kWarp; t < nv; t += nt - kWarp) {
      const int it = items[nblk + t];
      const int x = it >> 8, y = it & 255;
      const T sb = rt[4 * y + 3];
      if (sb == T(0)) continue;
      const int pb = (int)rt[4 * y], qb = (int)rt[4 * y + 1];
      const T cb = rt[4 * y + 2];
      const T vp = V[x * kEigLd + pb], vq = V[x * kEigLd + qb];
      V[x * kEigLd + pb] = cb * vp - sb * vq;
      V[x * kEigLd + qb] = sb * vp + cb * vq;
    }
  };
  int g = 0;  // steps so far (the rotation buffer is g & 1)
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // stepf[r]: a rotation in step r of this sweep (written only in step r's
    // rotation phase, read after its barrier, cleared here)
    if (tid == 0) *s_any = 0;
    for (int q = tid; q < mp - 1; q += nt) stepf[q] = 0;
    __syncthreads();
    for (int r = 0; r < mp - 1; ++r, ++g) {
      T* rc = rot + (g & 1) * 4 * (kEigMaxM / 2 + 1);
      if (tid < npair) {
        const int x1 = tid, x2 = mp - 1 - tid;
        // 1 + (x - 1 + r) mod (m' - 1) without a division (x - 1 + r < 2 (m' - 1))
        int p = x1 - 1 + r, q = x2 - 1 + r;
        if (p >= mp - 1) p -= mp - 1;
        if (q >= mp - 1) q -= mp - 1;
        p = x1 == 0 ? 0 : 1 + p;
        q = x2 == 0 ? 0 : 1 + q;
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        T c = T(1), s = T(0);
        if (q < m) {
          const T apq = A[p * kEigLd + q];
          const T app = A[p * kEigLd + p], aqq = A[q * kEigLd + q];
          // |a_pq| > rel sqrt|a_pp a_qq| without the square root; then, with
          // d = a_qq - a_pp and e = 2 a_pq, tan = sgn(d e) |e| / (|d| +
          // sqrt(d^2 + e^2)) (the smaller root of t^2 + 2 (d/e) t - 1 = 0),
          // cos = 1 / sqrt(1 + tan^2) -- the rotation is on every step's
          // critical path
          if (apq * apq > rel * rel * fabs(app * aqq) && fabs(apq) > floor_abs) {
            rotation_of(aqq - app, T(2) * apq, c, s);
            *s_any = 1;
            stepf[r] = 1;
          }
        }
        rc[4 * tid] = (T)p;
        rc[4 * tid + 1] = (T)q;
        rc[4 * tid + 2] = c;
        rc[4 * tid + 3] = s;
      } else if (tid >= kWarp && vpend) {
        apply_v(rot + vpar * 4 * (kEigMaxM / 2 + 1));
      }
      __syncthreads();
      vpend = false;
      if (stepf[r] == 0) continue;
      // A <- J^T A J in one pass.  The step's rotations act on disjoint
      // pairs, so every element of A lies in one 2 x 2 block (pair a's rows)
      // x (pair b's columns), which one thread rotates on both sides in
      // registers.  Items come from a table built once per solve (no integer
      // division in the step, which would run on the special-function pipe).
      for (int t = tid; t < nblk; t += nt) {
        const int it = items[t];
        const int x = it >> 8, y = it & 255;
        // block: row pair x, column pair y
        const T sa = rc[4 * x + 3], sb = rc[4 * y + 3];
        if (sa == T(0) && sb == T(0)) continue;
        const int pa = (int)rc[4 * x], qa = (int)rc[4 * x + 1];
        const int pb = (int)rc[4 * y], qb = (int)rc[4 * y + 1];
        const T ca = rc[4 * x + 2], cb = rc[4 * y + 2];
        const bool hq = qa < m, hqb = qb < m;
        const T m00 = A[pa * kEigLd + pb], m01 = hqb ? A[pa * kEigLd + qb] : T(0);
        const T m10 = hq ? A[qa * kEigLd + pb] : T(0), m11 = (hq && hqb) ? A[qa * kEigLd + qb] : T(0);
        // rows: p' = c p - s q, q' = s p + c q
        const T r00 = ca * m00 - sa * m10, r01 = ca * m01 - sa * m11;
        const T r10 = sa * m00 + ca * m10, r11 = sa * m01 + ca * m11;
        // columns likewise
        A[pa * kEigLd + pb] = cb * r00 - sb * r01;
        if (hqb) A[pa * kEigLd + qb] = sb * r00 + cb * r01;
        if (hq) A[qa * kEigLd + pb] = cb * r10 - sb * r11;
        if (hq && hqb) A[qa * kEigLd + qb] = sb * r10 + cb * r11;
      }
      vpend = true;
      vpar = g & 1;
      __syncthreads();
    }
    if (*s_any == 0) break;
    __syncthreads();
  }
  // the last step's V update
  if (vpend) {
    if (tid >= kWarp) apply_v(rot + vpar * 4 * (kEigMaxM / 2 + 1));
    __syncthreads();
  }
}

struct EigSmem {
  double G[kEigMaxM * kEigLd];
  double H[kEigMaxM * kEigLd];
  double U[kEigMaxM * kEigLd];
  double B[kEigMaxM * kEigLd];
  double T[kEigMaxM * kEigLd];
  double scale[kEigMaxM];
  double scale2[kEigMaxM];
  double rot[2 * 4 * (kEigMaxM / 2 + 1)];  // the Jacobi rotations, two steps
  union {
    struct {
      float Af[kEigMaxM * kEigLd];
      float Vf[kEigMaxM * kEigLd];
    } f;                           // the FP32 Jacobi stage
    double R[kEigMaxM * kEigLd];   // then the refinement's I - X^T X and E
  } u;
  double lam[kEigMaxM];
  double xpart[2 * kRrCluster];  // every CTA's parts of the refinement's two norms
  double nrm[2 * (kEigThreads / 32)];
  float rotf[2 * 4 * (kEigMaxM / 2 + 1)];
  int keep[kEigMaxM];
  int sel[kEigMaxM];
  unsigned short items[(kEigMaxM / 2) * (kEigMaxM / 2) + kEigMaxM * (kEigMaxM / 2)];
  int stepf[kEigMaxM];  // the Jacobi sweeps' per-step "rotated" flags
  int nkeep;
  int any;
  double floor_d;
  float floor_f;
};

// Cluster barrier of the Rayleigh-Ritz CTAs (every thread of every CTA
// calls it; it also orders their shared-memory writes, local and remote).
__device__ __forceinline__ void rr_sync() { cooperative_groups::this_cluster().sync(); }
// The same shared-memory object in CTA `rank` of the cluster.
template <class T>
__device__ __forceinline__ T* rr_peer(T* p, int rank) {
  return cooperative_groups::this_cluster().map_shared_rank(p, rank);
}
// Columns of an ncols-wide matrix owned by CTA `rank`: rank, rank + kRrCluster, ...
__device__ __forceinline__ int rr_owned(int ncols, int rank) {
  return ncols > rank ? (ncols - rank + kRrCluster - 1) / kRrCluster : 0;
}

// Y = op(X) Z + (add ? X : 0) for m x m shared matrices (op = transpose when
// tx; add only with !tx), the m^2 outputs spread over all threads of the
// block (one output, an m-long FMA chain, per thread at m <= 16; two at
// m <= 22, ...); Y must not alias X or Z.
__device__ void eig_mm(double* Y, const double* X, const double* Z, int m, bool tx, bool add = false) {
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t - i * m;
    double s = add ? X[i * kEigLd + j] : 0.0;
    if (tx) {
      for (int l = 0; l < m; ++l) s = fma(X[l * kEigLd + i], Z[l * kEigLd + j], s);
    } else {
      for (int l = 0; l < m; ++l) s = fma(X[i * kEigLd + l], Z[l * kEigLd + j], s);
    }
    Y[i * kEigLd + j] = s;
  }
  __syncthreads();
}

// Block totals of two values (every thread gets them).
__device__ __forceinline__ void eig_sum2(double& a, double& b, EigSmem& sm) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sm.nrm[2 * w] = a;
    sm.nrm[2 * w + 1] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int k = 0; k < nw; ++k) {
    a += sm.nrm[2 * k];
    b += sm.nrm[2 * k + 1];
  }
  __syncthreads();
}

// Iterative refinement of an approximate eigendecomposition of the symmetric
// m x m matrix A (Ogita and Aishima 2018, "Iterative refinement for
// symmetric eigenvalue decomposition").  With X the approximate eigenvectors
// (columns), R = I - X^T X and S = X^T A X, the exact eigenvectors are
// X (I + E) for a small E; to first order, (I + E)^T (I - R) (I + E) = I and
// (I + E)^T S (I + E) = D diagonal give
//   E_ii = r_ii / 2,  d_i = s_ii / (1 - r_ii),
//   E_ij = (s_ij + d_j r_ij) / (d_j - d_i)  (i != j),
// and X <- X + X E squares the error of X, as long as d_i and d_j are
// further apart than delta = 2 (||S - D|| + ||A|| ||R||) (Frobenius norms,
// bounds of the 2-norms); for a closer pair only the orthogonality part,
// E_ij = r_ij / 2, is applied.  A step is 3 m^3 FMAs in 3 passes, where the
// FP64 Jacobi sweeps it replaces took m - 1 dependent rotation steps per
// sweep, and two or three sweeps.
// A pair that starts within delta (delta is large at the first step, ~||A||
// times the FP32 basis's loss of orthogonality) is resolved at a later step,
// once the other pairs' corrections have shrunk delta below its gap; each
// step squares its error from there.  Only a pair that stays within delta
// (a true cluster at this precision) is left coupled.
// In: A; X in V (and Y, S, R scratch).  Out: the refined X in V and S =
// X^T A X, with the eigenvalues on its diagonal.  True when the off-diagonal
// of S and R reached rounding level; false when they did not within
// kEigRefineSteps steps (the caller then finishes with Jacobi sweeps on S).
constexpr int kEigRefineSteps = 6;

// (i, j), i <= j, of entry t of the upper triangle of an m x m matrix in row
// order (row r starts at r m - r (r - 1) / 2): the smaller root of the
// quadratic in FP32, then an exact integer correction.
__device__ __forceinline__ void eig_tri_index(int t, int m, int& i, int& j) {
  const float b = 2.0f * (float)m + 1.0f;
  int r = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)t, 0.0f))) * 0.5f);
  if (r < 0) r = 0;
  while (r > 0 && r * m - r * (r - 1) / 2 > t) --r;
  while ((r + 1) * m - (r + 1) * r / 2 <= t) ++r;
  i = r;
  j = t - (r * m - r * (r - 1) / 2) + r;
}

__device__ bool eig_refine(const double* A, double* V, double* Y, double* S, double* R, int m, EigSmem& sm,
                           int rank) {
  const int tid = threadIdx.x, nt = blockDim.x, mm = m * m;
  double a2 = 0.0, unused = 0.0;
  for (int t = tid; t < mm; t += nt) {
    const int i = t / m, j = t - i * m;
    a2 = fma(A[i * kEigLd + j], A[i * kEigLd + j], a2);
  }
  eig_sum2(a2, unused, sm);
  const double anorm = sqrt(a2);
  // rounding level of S = X^T (A X) and of I - X^T X: m-term dot products
  // over m^2 entries, with a margin
  const double tol = 64.0 * m * 1.1102230246251565e-16;
  // this CTA's columns j = rank + kRrCluster jj, jj < nown; item t of a
  // column phase is (row t / nown, column jj = t mod nown)
  const int nown = rr_owned(m, rank);
  double* X = V;  // every CTA holds all of X
  bool done = false;
  for (int step = 0;; ++step) {
    // Y = A X, the owned columns
    for (int t = tid; t < m * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      double s = 0.0;
      for (int l = 0; l < m; ++l) s = fma(A[i * kEigLd + l], X[l * kEigLd + j], s);
      Y[i * kEigLd + j] = s;
    }
    __syncthreads();
    // S = X^T Y and R = I - X^T X, the owned columns; d_i of the owned
    // diagonal entries; this CTA's parts of the two norms.  (S_ij and S_ji
    // are two roundings of x_i^T A x_j; R is symmetric bit for bit.)
    double off2 = 0.0, r2 = 0.0;
    for (int t = tid; t < m * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      double sv = 0.0, g = 0.0;
      for (int l = 0; l < m; ++l) {
        const double xi = X[l * kEigLd + i];
        sv = fma(xi, Y[l * kEigLd + j], sv);
        g = fma(xi, X[l * kEigLd + j], g);
      }
      const double rv = (i == j ? 1.0 : 0.0) - g;
      S[i * kEigLd + j] = sv;
      R[i * kEigLd + j] = rv;
      r2 = fma(rv, rv, r2);
      if (i != j) off2 = fma(sv, sv, off2);
      else sm.lam[i] = sv / g;
    }
    eig_sum2(off2, r2, sm);
    // every CTA gets the owned d_i and the two parts of every CTA
    for (int t = tid; t < kRrCluster * (nown + 1); t += nt) {
      const int dst = t / (nown + 1), q = t - dst * (nown + 1);
      if (q < nown) {
        const int j = rank + kRrCluster * q;
        rr_peer(sm.lam, dst)[j] = sm.lam[j];
      } else {
        double* xp = rr_peer(sm.xpart, dst);
        xp[2 * rank] = off2;
        xp[2 * rank + 1] = r2;
      }
    }
    rr_sync();
    off2 = 0.0;
    r2 = 0.0;
    for (int c = 0; c < kRrCluster; ++c) {  // the same order in every CTA
      off2 += sm.xpart[2 * c];
      r2 += sm.xpart[2 * c + 1];
    }
    const double off = sqrt(off2), rn = sqrt(r2);
    if (off <= tol * anorm && rn <= tol) {
      done = true;
      break;
    }
    if (step == kEigRefineSteps) break;
    const double delta = 2.0 * (off + anorm * rn);
    // E in place of R, the owned columns
    for (int t = tid; t < m * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      const double rv = R[i * kEigLd + j];
      double e = 0.5 * rv;
      if (i != j) {
        const double di = sm.lam[i], dj = sm.lam[j];
        const double den = dj - di;
        if (fabs(den) > delta) {
          // 1 / den: FP32 reciprocal and one Newton-Raphson step
          // y <- y + y (1 - den y) in FP64 (relative error ~1e-14, ample for
          // a correction of size |E|) within FP32's range, FP64 division
          // outside it
          double y;
          if (fabs(den) > 1e-30 && fabs(den) < 1e30) {
            y = (double)__frcp_rn((float)den);
            y = fma(y, fma(-den, y, 1.0), y);
          } else {
            y = 1.0 / den;
          }
          e = (S[i * kEigLd + j] + dj * rv) * y;
        }
      }
      R[i * kEigLd + j] = e;
    }
    __syncthreads();
    // X + X E, the owned columns, into every CTA's Y (no CTA reads Y again
    // in this step; every CTA still reads its X here)
    for (int t = tid; t < m * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      double s = X[i * kEigLd + j];
      for (int l = 0; l < m; ++l) s = fma(X[i * kEigLd + l], R[l * kEigLd + j], s);
      for (int dst = 0; dst < kRrCluster; ++dst) rr_peer(Y, dst)[i * kEigLd + j] = s;
    }
    rr_sync();
    double* t = X;
    X = Y;
    Y = t;
  }
  // all of S in every CTA
  for (int t = tid; t < m * nown; t += nt) {
    const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
    const double v = S[i * kEigLd + j];
    for (int dst = 0; dst < kRrCluster; ++dst)
      if (dst != rank) rr_peer(S, dst)[i * kEigLd + j] = v;
  }
  rr_sync();
  if (X != V) {
    for (int q = tid; q < m * kEigLd; q += nt) V[q] = X[q];
    __syncthreads();
  }
  return done;
}

// Mixed-precision symmetric eigensolver for the Rayleigh-Ritz step: FP32
// Jacobi sweeps (the FP32 pipe is 64 times the FP64 one) to eigenvectors
// accurate to ~1e-7 ||A|| / gap, then the FP64 iterative refinement above
// (two steps for well-separated eigenvalues, a few more for the close
// smallest Ritz values, a last pass confirming); where it does not reach
// rounding level (a cluster closer than its delta), FP64 Jacobi sweeps on
// the refined S = X^T A X, which is diagonal but for that cluster, and the
// eigenvectors X V1.  A (overwritten with its eigenvalues on
// the diagonal) and V as in eig_jacobi; S1, S2: m x m scratch.
__device__ void eig_eigh(double* A, double* V, int m, double* S1, double* S2, EigSmem& sm, int rank) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int q = tid; q < m * kEigLd; q += nt) sm.u.f.Af[q] = (float)A[q];
  __syncthreads();
  eig_jacobi<float>(sm.u.f.Af, sm.u.f.Vf, m, 1e-7f, 1e-9f, 12, sm.rotf, &sm.any, &sm.floor_f, sm.items, sm.stepf);
  for (int q = tid; q < m * kEigLd; q += nt) V[q] = (double)sm.u.f.Vf[q];
  __syncthreads();
  const bool done = eig_refine(A, V, S1, S2, sm.u.R, m, sm, rank);
  // A <- S symmetrised (S_ij and S_ji are two roundings of the same product;
  // the Jacobi sweeps read one triangle's pairs)
  for (int t = tid; t < m * m; t += nt) {
    const int i = t / m, j = t - i * m;
    A[i * kEigLd + j] = 0.5 * (S2[i * kEigLd + j] + S2[j * kEigLd + i]);
  }
  __syncthreads();
  if (done) return;
  eig_jacobi<double>(A, S2, m, 1e-15, 0.0, 30, sm.rot, &sm.any, &sm.floor_d, sm.items, sm.stepf);
  eig_mm(S1, V, S2, m, false);  // X V1
  for (int q = tid; q < m * kEigLd; q += nt) V[q] = S1[q];
  __syncthreads();
}

// Pivot j of the Cholesky factor of the scaled Gram matrix (in sm.U), by
// one thread: sets sm.any when the pivot is not above 1e-10, stores L_jj in
// the diagonal and 1 / L_jj in sm.scale2[j].
constexpr int kEigCholItems = (kEigMaxM * (kEigMaxM + 1) / 2 + kEigThreads - 1) / kEigThreads;

__device__ __forceinline__ void eig_chol_pivot(EigSmem& sm, int j) {
  const double piv = sm.U[j * kEigLd + j];
  if (!(piv > 1e-10)) sm.any = 1;
  // 1/sqrt(piv): FP32 estimate, two Newton steps in FP64 (piv in
  // (1e-10, 1] here: the scaled Gram matrix has a unit diagonal)
  const double pv = fmax(piv, 1e-300);
  double y = (double)rsqrtf((float)pv);
  y = y * (1.5 - 0.5 * pv * y * y);
  y = y * (1.5 - 0.5 * pv * y * y);
  sm.U[j * kEigLd + j] = pv * y;
  sm.scale2[j] = y;
}

// Rayleigh-Ritz in one block: G, H (full, shared) -> C [m][k] and theta [k]
// (k = the block size kb)
// in global memory; returns the number of kept directions.
__device__ int eig_rayleigh_ritz(EigSmem& sm, int m, int k, double* C, double* theta, int rank) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = tid; j < m; j += nt) {
    const double g = sm.G[j * kEigLd + j];
    sm.scale[j] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5)
    for (int j = threadIdx.x & 31; j < m; j += 32) {
    const double f = sm.scale[i] * sm.scale[j];
    sm.G[i * kEigLd + j] *= f;
    sm.H[i * kEigLd + j] *= f;
  }
  __syncthreads();
  // A basis B (m x r) with B^T G B = I.  First try the Cholesky factor of the
  // scaled G over its nonzero columns (the locked ones are zero): B = L^{-T}.
  // Where a pivot falls below 1e-10 (directions closer than ~1e-5 rad, which
  // the factor would amplify), diagonalise G instead and drop its directions
  // below 1e-12 of the largest eigenvalue.
  if (tid == 0) {
    int a = 0;
    for (int j = 0; j < m; ++j)
      if (sm.scale[j] > 0.0) sm.keep[a++] = j;
    sm.nkeep = a;
    sm.any = 0;  // Cholesky failed
  }
  __syncthreads();
  const int ma = sm.nkeep;
  for (int i = threadIdx.x >> 5; i < ma; i += blockDim.x >> 5)
    for (int j = threadIdx.x & 31; j < ma; j += 32) sm.U[i * kEigLd + j] = sm.G[sm.keep[i] * kEigLd + sm.keep[j]];
  __syncthreads();
  // Right-looking, two block barriers a column: column j of L is scaled, then
  // the trailing update runs, in which thread 0 -- the updater of entry
  // (j + 1, j + 1) -- also takes pivot j + 1 (the same operations in the
  // same order as a pivot step of its own, one barrier fewer).
  if (tid == 0 && ma > 0) eig_chol_pivot(sm, 0);
  __syncthreads();
  for (int j = 0; j < ma; ++j) {
    if (sm.any) break;
    for (int i = j + 1 + tid; i < ma; i += nt) sm.U[i * kEigLd + j] *= sm.scale2[j];
    __syncthreads();
    for (int i = j + 1 + (threadIdx.x >> 5); i < ma; i += blockDim.x >> 5)
      for (int c = j + 1 + (threadIdx.x & 31); c <= i; c += 32) {
        sm.U[i * kEigLd + c] = fma(-sm.U[i * kEigLd + j], sm.U[c * kEigLd + j], sm.U[i * kEigLd + c]);
        if (c == j + 1 && i == j + 1) eig_chol_pivot(sm, j + 1);
      }
    __syncthreads();
  }
  int r;
  if (!sm.any) {
    // T = L^{-1} by right-looking substitution: entry (i, c), i >= c, of the
    // packed lower triangle is owned by one thread (at most
    // kEigCholItems), which keeps its running value a_ic = delta_ic -
    // sum_{l < done} L_il T_lc in a register; at step l every owner with
    // i > l subtracts L_il T_lc (the same FMAs in the same order as the
    // row-by-row substitution), and the owners of row l + 1, now complete,
    // publish T_{l+1,c} = a / L_{l+1,l+1}: one block barrier a row
    // (forward substitution by one thread per column ran chains of m^2 / 2
    // dependent FMAs).
    int ei[kEigCholItems], ec[kEigCholItems];
    double ea[kEigCholItems];
#pragma unroll
    for (int h = 0; h < kEigCholItems; ++h) {
      const int e = tid + h * nt;
      ei[h] = -1;
      ec[h] = 0;
      ea[h] = 0.0;
      if (e < ma * (ma + 1) / 2) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        ei[h] = i;
        ec[h] = e - i * (i + 1) / 2;
        ea[h] = ei[h] == ec[h] ? 1.0 : 0.0;
        if (i == 0) sm.T[0] = ea[h] * sm.scale2[0];
      }
    }
    for (int q = tid; q < ma * ma; q += nt) {  // the strict upper triangle is zero
      const int i = q / ma, c = q - i * ma;
      if (c > i) sm.T[i * kEigLd + c] = 0.0;
    }
    __syncthreads();
    for (int l = 0; l + 1 < ma; ++l) {
#pragma unroll
      for (int h = 0; h < kEigCholItems; ++h) {
        if (ei[h] > l && ec[h] <= l) ea[h] = fma(-sm.U[ei[h] * kEigLd + l], sm.T[l * kEigLd + ec[h]], ea[h]);
        if (ei[h] == l + 1) sm.T[ei[h] * kEigLd + ec[h]] = ea[h] * sm.scale2[ei[h]];
      }
      __syncthreads();
    }
    // B[keep[a]][b] = (L^{-1})[b][a]; zero rows for the locked columns
    for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5)
      for (int j = threadIdx.x & 31; j < ma; j += 32) sm.B[i * kEigLd + j] = 0.0;
    __syncthreads();
    for (int a = threadIdx.x >> 5; a < ma; a += blockDim.x >> 5)
      for (int b = threadIdx.x & 31; b < ma; b += 32) sm.B[sm.keep[a] * kEigLd + b] = sm.T[b * kEigLd + a];
    __syncthreads();
    r = ma;
  } else {
    eig_eigh(sm.G, sm.U, m, sm.B, sm.T, sm, rank);  // scaled G = U diag(g) U^T
    if (tid == 0) {
      double gmax = 0.0;
      for (int j = 0; j < m; ++j) gmax = fmax(gmax, sm.G[j * kEigLd + j]);
      int rr = 0;
      for (int j = 0; j < m; ++j)
        if (sm.G[j * kEigLd + j] > 1e-12 * gmax) sm.keep[rr++] = j;
      sm.nkeep = rr;
    }
    __syncthreads();
    r = sm.nkeep;
    // B = U[:, keep] diag(g)^{-1/2}  (m x r)
    for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5)
      for (int j = threadIdx.x & 31; j < r; j += 32) {
        const int c = sm.keep[j];
        sm.B[i * kEigLd + j] = sm.U[i * kEigLd + c] / sqrt(sm.G[c * kEigLd + c]);
      }
    __syncthreads();
  }
  // T = H B (m x r), then H2 = B^T T (r x r) into G: the owned columns of
  // T, then the owned columns of H2 into every CTA's G (after a cluster
  // barrier: until then a CTA may still read its G to build B)
  {
    const int nown = rr_owned(r, rank);
    for (int t = tid; t < m * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      double s = 0.0;
      for (int l = 0; l < m; ++l) s = fma(sm.H[i * kEigLd + l], sm.B[l * kEigLd + j], s);
      sm.T[i * kEigLd + j] = s;
    }
    rr_sync();
    for (int t = tid; t < r * nown; t += nt) {
      const int i = t / nown, j = rank + kRrCluster * (t - (t / nown) * nown);
      double s = 0.0;
      for (int l = 0; l < m; ++l) s = fma(sm.B[l * kEigLd + i], sm.T[l * kEigLd + j], s);
      for (int dst = 0; dst < kRrCluster; ++dst) rr_peer(sm.G, dst)[i * kEigLd + j] = s;
    }
    rr_sync();
  }
  // symmetrise (rounding), then H2 = Y diag(theta) Y^T with Y in U
  for (int i = threadIdx.x >> 5; i < r; i += blockDim.x >> 5)
    for (int j = threadIdx.x & 31; j < r; j += 32) {
    if (i < j) {
      const double s = 0.5 * (sm.G[i * kEigLd + j] + sm.G[j * kEigLd + i]);
      sm.G[i * kEigLd + j] = s;
      sm.G[j * kEigLd + i] = s;
    }
  }
  __syncthreads();
  eig_eigh(sm.G, sm.U, r, sm.H, sm.T, sm, rank);
  // the k smallest Ritz values, ascending (selection by rank, ties by
  // index; thread i ranks value i)
  for (int i = tid; i < r; i += nt) {
    const double ti = sm.G[i * kEigLd + i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const double tj = sm.G[j * kEigLd + j];
      if (tj < ti || (tj == ti && j < i)) ++rank;
    }
    sm.sel[rank] = i;
  }
  __syncthreads();
  const int kk = r < k ? r : k;
  if (rank == 0)
    for (int j = tid; j < kk; j += nt) theta[j] = sm.G[sm.sel[j] * kEigLd + sm.sel[j]];
  // C = diag(scale) B Y[:, sel]  (m x k); CTA c writes the rows i = c mod kRrCluster
  for (int i = rank + kRrCluster * (threadIdx.x >> 5); i < m; i += kRrCluster * (blockDim.x >> 5))
    for (int j = threadIdx.x & 31; j < kk; j += 32) {
    const int c = sm.sel[j];
    double s = 0.0;
    for (int l = 0; l < r; ++l) s = fma(sm.B[i * kEigLd + l], sm.U[l * kEigLd + c], s);
    C[i * kEigMaxB + j] = sm.scale[i] * s;
  }
  __syncthreads();
  return r;
}

// G = S^T S and H = S^T (A S) over the m active columns (upper triangles),
// per block; the Gram-totals kernel adds all blocks' partials in block order.
// One pair (a, b) per thread (kEigGramThreads >= 465 pairs at m = 30): with
// 256 threads and two pairs for some, the last warps' second pairs ran alone
// at the end of every tile.
constexpr int kEigGramThreads = 512;
static_assert(kEigGramThreads >= kEigPairs, "one Gram pair per thread");

__global__ void __launch_bounds__(kEigGramThreads) eig_gram_kernel(EigPtrs P) {
  const EigDesc& d = *P.d;
  EigState* st = P.st;
  if (st->done || st->bad) return;
  __shared__ double tS[kEigTile * kEigMaxM];
  __shared__ double tA[kEigTile * kEigMaxM];
  const int n = d.n, ld = d.ld, m = st->m, cur = st->cur;
  const int npairs = m * (m + 1) / 2;
  const double* S = P.S[cur];
  const double* AS = P.AS[cur];
  const int tid = threadIdx.x;
  // this thread's pair (a <= b)
  int pa = 0, pb = 0;
  const bool has = tid < npairs;
  if (has) {
    int a = 0, rem = tid;
    while (rem >= m - a) {
      rem -= m - a;
      ++a;
    }
    pa = a;
    pb = a + rem;
  }
  double g = 0.0, hh = 0.0;
  const int tiles = (n + kEigTile - 1) / kEigTile;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int r0 = tile * kEigTile;
    const int rows = min(kEigTile, n - r0);
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < rows; i += blockDim.x >> 5)
      for (int j = threadIdx.x & 31; j < m; j += 32) {
      tS[i * kEigMaxM + j] = S[(size_t)(r0 + i) * ld + j];
      tA[i * kEigMaxM + j] = AS[(size_t)(r0 + i) * ld + j];
    }
    __syncthreads();
    if (has) {
      for (int i = 0; i < rows; ++i) {
        const double sa = tS[i * kEigMaxM + pa];
        g = fma(sa, tS[i * kEigMaxM + pb], g);
        hh = fma(sa, tA[i * kEigMaxM + pb], hh);
      }
    }
  }
  double* mine = P.gpart + (size_t)blockIdx.x * 2 * kEigPairs;
  if (has) {
    mine[tid] = g;
    mine[kEigPairs + tid] = hh;
  }
}

// Totals of the Gram partials of the gb blocks -- 2 npairs values -- then
// the Rayleigh-Ritz step in the last cluster to arrive (all of its CTAs).  Block c adds values
// 32c .. 32c + 31: a warp per 4 values, lane l summing blocks l, l + 32, ...,
// then a fixed butterfly (the same bits run to run; spread over blocks so
// that the loads are not serialised in one block).
__global__ void __cluster_dims__(kRrCluster, 1, 1) __launch_bounds__(kEigThreads, 1) eig_rr_kernel(EigPtrs P, int gb) {
  const EigDesc& d = *P.d;
  EigState* st = P.st;
  if (st->done || st->bad) return;
  __shared__ EigSmem sm;
  __shared__ bool s_last;
  const int kb = d.kb, m = st->m;
  const int npairs = m * (m + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int q = 0; q < 4; ++q) {
    const int v = blockIdx.x * 32 + w * 4 + q;  // value: G pairs, then H pairs
    if (v >= 2 * npairs) break;
    const int off = v < npairs ? v : kEigPairs + (v - npairs);
    double s = 0.0;
    for (int b = lane; b < gb; b += 32) s += __ldcg(P.gpart + (size_t)b * 2 * kEigPairs + off);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) P.gtot[v] = s;
  }
  // cluster arrival: every CTA's totals are written and fenced before the
  // barrier; CTA 0 of each cluster then takes a ticket, and the cluster
  // whose ticket is the last one runs the Rayleigh-Ritz step.  The flag is
  // written into every CTA's own shared memory, so no CTA reads another's
  // after the barrier (the other clusters leave at once).
  const int rank = (int)cooperative_groups::this_cluster().block_rank();
  __syncthreads();
  if (tid == 0) __threadfence();
  rr_sync();
  if (rank == 0 && tid == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket_gram, 1u);
    const bool last = t == gridDim.x / kRrCluster - 1;
    if (last) {
      __threadfence();
      st->ticket_gram = 0u;
    }
    for (int dst = 0; dst < kRrCluster; ++dst) *rr_peer(&s_last, dst) = last;
  }
  rr_sync();
  if (!s_last) return;
  __threadfence();
  const unsigned active = st->active;
  // the full symmetric G and H; the W and P columns of converged pairs are
  // zeroed (soft locking)
  for (int t = tid; t < npairs; t += kEigThreads) {
    int a = 0, rem = t;
    while (rem >= m - a) {
      rem -= m - a;
      ++a;
    }
    const int b = a + rem;
    double sg = __ldcg(P.gtot + t), sh = __ldcg(P.gtot + npairs + t);
    const bool la = a >= kb && !((active >> ((a - kb) % kb)) & 1u);
    const bool lb = b >= kb && !((active >> ((b - kb) % kb)) & 1u);
    if (la || lb) sg = sh = 0.0;
    sm.G[a * kEigLd + b] = sg;
    sm.G[b * kEigLd + a] = sg;
    sm.H[a * kEigLd + b] = sh;
    sm.H[b * kEigLd + a] = sh;
  }
  __syncthreads();
  const int r = eig_rayleigh_ritz(sm, m, kb, P.C, P.theta, rank);
  if (rank == 0 && tid == 0) {
    st->rank = r;
    if (r < kb) {
      st->status = SLA_BREAKDOWN;
      st->done = 1;
    }
  }
}

// X' = S C, AX' = AS C, P' = S[:, kb:m] C[kb:m], AP' likewise, R = AX' - X'
// diag(theta), W' = D^{-1} R, into the other buffer pair; per-block sums of
// ||r_i||^2 and ||x_i||^2; the last block takes the convergence decision on
// the kb pairs.  Tiles of RT = NT / kb rows: the tile's rows of S and AS
// (contiguous, RT ld doubles each) are copied to shared memory with
// coalesced loads, then thread t < RT kb computes row t / kb, output column
// t mod kb from there (the same column in every tile, so its norms are per
// column).  A thread per row reading its own row from global memory issued
// 32 addresses 8 ld bytes apart per load and waited on each (61 us a launch
// at 2D 128^2, kb = 8, against 34 us for the Gram kernel's tiles).
template <int NT>
__global__ void __launch_bounds__(NT) eig_update_kernel(EigPtrs P) {
  const EigDesc& d = *P.d;
  EigState* st = P.st;
  if (st->done || st->bad) return;
  __shared__ double sC[kEigMaxM * kEigMaxB];
  __shared__ double sT[kEigMaxB];
  // S and AS tiles, row stride ld + 1 (odd: rows fall in different banks);
  // RT (ld + 1) <= NT / kb (3 kb + 1) <= 4 NT doubles each
  __shared__ double tS[4 * NT];
  __shared__ double tA[4 * NT];
  __shared__ double red[2 * NT];
  __shared__ double tot_s[2 * kEigMaxB];
  __shared__ bool s_last;
  const int n = d.n, k = d.k, kb = d.kb, ld = d.ld, m = st->m, cur = st->cur;
  const int tid = threadIdx.x;
  for (int q = tid; q < m * kEigMaxB; q += NT) sC[q] = P.C[q];
  if (tid < kb) sT[tid] = P.theta[tid];
  const double* S = P.S[cur];
  const double* AS = P.AS[cur];
  double* Sn = P.S[cur ^ 1];
  double* ASn = P.AS[cur ^ 1];
  const int RT = NT / kb, lp = ld + 1;
  const bool active = tid < RT * kb;
  const int r = tid / kb, j = tid - r * kb;
  const int tiles = (n + RT - 1) / RT;
  double rr = 0.0, xx = 0.0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int r0 = tile * RT;
    const int rows = min(RT, n - r0);
    __syncthreads();  // the previous tile's reads are done (and sC, sT written)
    const double* s0 = S + (size_t)r0 * ld;
    const double* a0 = AS + (size_t)r0 * ld;
    for (int q = tid; q < rows * ld; q += NT) {
      const int rr_ = q / ld, cc = q - rr_ * ld;
      tS[rr_ * lp + cc] = s0[q];
      tA[rr_ * lp + cc] = a0[q];
    }
    __syncthreads();
    if (active && r < rows) {
      const double th = sT[j];
      const double* ts = tS + r * lp;
      const double* ta = tA + r * lp;
      double x = 0.0, ax = 0.0, p = 0.0, ap = 0.0;
      for (int a = 0; a < kb; ++a) {
        const double c = sC[a * kEigMaxB + j];
        x = fma(ts[a], c, x);
        ax = fma(ta[a], c, ax);
      }
      for (int a = kb; a < m; ++a) {
        const double c = sC[a * kEigMaxB + j];
        p = fma(ts[a], c, p);
        ap = fma(ta[a], c, ap);
      }
      const int i = r0 + r;
      const double xj = x + p, axj = ax + ap;
      const double rj = axj - th * xj;
      double* sn = Sn + (size_t)i * ld;
      double* asn = ASn + (size_t)i * ld;
      sn[j] = xj;
      asn[j] = axj;
      sn[kb + j] = P.dinv[i] * rj;
      sn[2 * kb + j] = p;
      asn[2 * kb + j] = ap;
      rr = fma(rj, rj, rr);
      xx = fma(xj, xj, xx);
    }
  }
  // block sums per column: the threads of column c (c, c + kb, ...), in order
  red[tid] = rr;
  red[NT + tid] = xx;
  __syncthreads();
  if (tid < 2 * kb) {
    const int c = tid >> 1, which = tid & 1;
    double sum = 0.0;
    for (int t = c; t < RT * kb; t += kb) sum += red[which * NT + t];
    P.upart[(size_t)blockIdx.x * 2 * kEigMaxB + tid] = sum;
  }
  if (!last_block_arrive(&st->ticket_upd, &s_last)) return;
  // the blocks' partials, value-major: thread t < 12 * 2 kb sums value t / 12
  // over blocks t mod 12, t mod 12 + 12, ... in order, then one thread per
  // value adds its 12 chunk sums in order.  (A warp-wide FP64 add holds the
  // SM's FP64 pipe for 16 cycles whatever its useful lanes, so a butterfly
  // over lanes for each of the 2 kb values cost more than the sums
  // themselves: 17k of the last block's 35k cycles.)
  constexpr int kChunks = 12;
  static_assert(kChunks * 2 * kEigMaxB <= NT, "one thread per (value, chunk)");
  const int nv = 2 * kb;
  if (tid < kChunks * nv) {
    const int v = tid / kChunks, c = tid - v * kChunks;
    double sum = 0.0;
    for (int b = c; b < (int)gridDim.x; b += kChunks) sum += __ldcg(P.upart + (size_t)b * 2 * kEigMaxB + v);
    red[tid] = sum;
  }
  __syncthreads();
  if (tid < nv) {
    double sum = 0.0;
    for (int c = 0; c < kChunks; ++c) sum += red[tid * kChunks + c];
    tot_s[tid] = sum;
  }
  __syncthreads();
  // each pair's relative residual by a thread of its own (FP64 square roots
  // and divisions are long sequences on the FP64 pipe), then the decision
  if (tid < kb) {
    const double r2 = tot_s[2 * tid], x2 = tot_s[2 * tid + 1];
    red[tid] = sqrt(r2) / (fabs(sT[tid]) * sqrt(x2));
  }
  __syncthreads();
  if (tid == 0) {
    double worst = 0.0;
    bool finite = true;
    unsigned act = 0u;
    for (int j = 0; j < kb; ++j) {
      const double res = red[j];
      if (!isfinite(res)) finite = false;
      if (j < k) worst = fmax(worst, res);
      if (!(res <= d.tol)) act |= 1u << j;
    }
    st->active = act;
    st->maxres = worst;
    st->cur = cur ^ 1;
    if (m > kb) st->iters += 1;
    st->m = (m == kb) ? 2 * kb : 3 * kb;
    if (!finite) {
      st->status = SLA_BREAKDOWN;
      st->done = 1;
    } else if (worst <= d.tol) {
      st->status = SLA_OK;
      st->done = 1;
    } else if (st->iters >= d.max_iter) {
      st->status = SLA_NOT_CONVERGED;
      st->done = 1;
    }
  }
}

// (|x|, index) order of the sign rule: the larger magnitude, on a tie the
// smaller index -- a total order, so any reduction order picks the same entry.
__device__ __forceinline__ bool eig_sign_better(double a, int ia, double b, int ib) {
  return a > b || (a == b && ia < ib);
}

// Final: lambda, the true residuals ||A x_i - theta_i x_i|| / (|theta_i|
// ||x_i||) of the k wanted pairs from a fresh product (AS[cur ^ 1][:, 0:kb]),
// the info record, and V = the first k columns of X with unit norm and the
// sign that makes each column's largest-magnitude entry positive (the first
// such entry on a tie), so that V is a smooth function of A near a simple
// eigenvalue.  Two launches: sums and the sign entries, then the scaled copy.
__global__ void __launch_bounds__(kEigThreads) eig_final_kernel(EigPtrs P, int phase) {
  const EigDesc& d = *P.d;
  EigState* st = P.st;
  __shared__ double red[2 * kEigMaxK * (kEigThreads / 32)];
  __shared__ double snorm[kEigMaxK];
  __shared__ bool s_last;
  const int n = d.n, k = d.k, ld = d.ld, cur = st->cur;
  const int tid = threadIdx.x;
  const double* X = P.S[cur];
  const double* AX = P.AS[cur ^ 1];
  if (phase == 1) {
    if (st->bad) return;
    if (tid < k) snorm[tid] = P.upart[(size_t)gridDim.x * 2 * kEigMaxB + tid];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + tid; i < n; i += gridDim.x * blockDim.x)
      for (int j = 0; j < k; ++j) d.V[(size_t)i * k + j] = X[(size_t)i * ld + j] * snorm[j];
    return;
  }
  double rr[kEigMaxK], xx[kEigMaxK], bx[kEigMaxK];
  int bi[kEigMaxK];
#pragma unroll
  for (int j = 0; j < kEigMaxK; ++j) {
    rr[j] = xx[j] = bx[j] = 0.0;
    bi[j] = INT_MAX;
  }
  if (!st->bad) {
    for (int i = blockIdx.x * blockDim.x + tid; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
      for (int j = 0; j < kEigMaxK; ++j) {
        if (j < k) {
          const double xj = X[(size_t)i * ld + j];
          const double rj = AX[(size_t)i * ld + j] - P.theta[j] * xj;
          rr[j] = fma(rj, rj, rr[j]);
          xx[j] = fma(xj, xj, xx[j]);
          if (eig_sign_better(fabs(xj), i, fabs(bx[j]), bi[j])) {
            bx[j] = xj;
            bi[j] = i;
          }
        }
      }
    }
  }
  const int w = tid >> 5, lane = tid & 31;
  // the sign entry of each column: warp, then block (partials after upart's)
  __shared__ double s_bx[kEigMaxK][kEigThreads / 32];
  __shared__ int s_bi[kEigMaxK][kEigThreads / 32];
  double* spart = P.upart + ((size_t)gridDim.x + 1) * 2 * kEigMaxB;
#pragma unroll
  for (int j = 0; j < kEigMaxK; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      const double ox = __shfl_xor_sync(0xffffffffu, bx[j], o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi[j], o);
      if (eig_sign_better(fabs(ox), oi, fabs(bx[j]), bi[j])) {
        bx[j] = ox;
        bi[j] = oi;
      }
    }
    if (lane == 0) {
      s_bx[j][w] = bx[j];
      s_bi[j][w] = bi[j];
    }
  }
#pragma unroll
  for (int j = 0; j < kEigMaxK; ++j) {
    for (int o = 16; o > 0; o >>= 1) {
      rr[j] += __shfl_xor_sync(0xffffffffu, rr[j], o);
      xx[j] += __shfl_xor_sync(0xffffffffu, xx[j], o);
    }
    if (lane == 0) {
      red[(2 * j) * (kEigThreads / 32) + w] = rr[j];
      red[(2 * j + 1) * (kEigThreads / 32) + w] = xx[j];
    }
  }
  __syncthreads();
  if (tid < 2 * k) {
    double sum = 0.0;
    for (int q = 0; q < kEigThreads / 32; ++q) sum += red[tid * (kEigThreads / 32) + q];
    P.upart[(size_t)blockIdx.x * 2 * kEigMaxB + tid] = sum;
  } else if (tid >= 32 && tid < 32 + k) {
    const int j = tid - 32;
    double x = s_bx[j][0];
    int ix = s_bi[j][0];
    for (int q = 1; q < kEigThreads / 32; ++q)
      if (eig_sign_better(fabs(s_bx[j][q]), s_bi[j][q], fabs(x), ix)) {
        x = s_bx[j][q];
        ix = s_bi[j][q];
      }
    spart[(size_t)blockIdx.x * 2 * kEigMaxK + 2 * j] = x;
    spart[(size_t)blockIdx.x * 2 * kEigMaxK + 2 * j + 1] = (double)ix;
  }
  if (!last_block_arrive(&st->ticket_fin, &s_last)) return;
  __shared__ double s_sign[kEigMaxK];
  if (tid < 2 * k) {
    double sum = 0.0;
#pragma unroll 8
    for (int b = 0; b < (int)gridDim.x; ++b) sum += __ldcg(P.upart + (size_t)b * 2 * kEigMaxB + tid);
    red[tid] = sum;
  } else if (tid >= 32 && tid < 32 + k) {
    const int j = tid - 32;
    double x = 0.0, ix = 2147483647.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const double bx2 = __ldcg(spart + (size_t)b * 2 * kEigMaxK + 2 * j);
      const double bi2 = __ldcg(spart + (size_t)b * 2 * kEigMaxK + 2 * j + 1);
      if (fabs(bx2) > fabs(x) || (fabs(bx2) == fabs(x) && bi2 < ix)) {
        x = bx2;
        ix = bi2;
      }
    }
    s_sign[j] = x < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    sla_info inf;
    inf.iters = st->iters;
    if (st->bad) {
      inf.status = SLA_NOT_SPD;
      inf.rel_res = NAN;
      inf.true_rel_res = NAN;
    } else {
      double worst = 0.0;
      for (int j = 0; j < k; ++j) {
        const double r2 = red[2 * j], x2 = red[2 * j + 1];
        const double nx = sqrt(x2);
        worst = fmax(worst, sqrt(r2) / (fabs(P.theta[j]) * nx));
        // sign / ||x_j|| for the copy, after the partials
        P.upart[(size_t)gridDim.x * 2 * kEigMaxB + j] = s_sign[j] / nx;
        d.lambda[j] = P.theta[j];
      }
      inf.status = st->status;
      inf.rel_res = st->maxres;
      inf.true_rel_res = worst;
    }
    *d.info = inf;
  }
}

// Hellmann-Feynman gradient (Eq. 4): out[e] = sum_i g_i V[row_e][i]
// V[col_e][i], one row per thread.
__global__ void eig_grad_kernel(int n, int k, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ V, const double* __restrict__ g,
                                double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double w[kEigMaxK];
#pragma unroll
    for (int j = 0; j < kEigMaxK; ++j) w[j] = j < k ? __ldg(g + j) * __ldg(V + (size_t)i * k + j) : 0.0;
    for (int e = __ldg(rowptr + i); e < __ldg(rowptr + i + 1); ++e) {
      const double* vc = V + (size_t)__ldg(col + e) * k;
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < kEigMaxK; ++j)
        if (j < k) s = fma(w[j], __ldg(vc + j), s);
      out[e] = s;
    }
  }
}

// ---------------------------------------------------------------- host

namespace {
int eig_grid(int n, int cap, int threads = kEigThreads) {
  const long long b = ((long long)n + threads - 1) / threads;
  return (int)std::max(1LL, std::min<long long>(b, cap));
}
}  // namespace

// Block size of a k-pair solve: two guard vectors, at most n.
int eig_block(int n, int k) { return std::min(k + 2, std::max(n, k)); }

size_t eig_ws_bytes(int n, int k, int* gram_blocks, int* upd_blocks) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int gb = std::max(1, std::min((n + kEigTile - 1) / kEigTile, 296));
  // update blocks: one tile of kEigUpdThreads / kb rows each, at most 4096
  const long long rt = std::max(1, kEigUpdThreads / eig_block(n, k));
  const int ub = (int)std::max(1LL, std::min<long long>(((long long)n + rt - 1) / rt, 4096));
  if (gram_blocks) *gram_blocks = gb;
  if (upd_blocks) *upd_blocks = ub;
  size_t o = 0;
  o += al256(sizeof(EigDesc));
  o += al256(sizeof(EigState));
  o += al256(sizeof(double) * nn);                     // dinv
  const size_t kb = (size_t)eig_block(n, k);
  o += 4 * al256(sizeof(double) * nn * 3 * kb);         // S[2], AS[2]
  o += al256(sizeof(double) * (size_t)gb * 2 * kEigPairs);
  o += al256(sizeof(double) * 2 * kEigPairs);
  // update partials + the totals, then the final kernel's sign partials
  o += al256(sizeof(double) * (((size_t)ub + 1) * 2 * kEigMaxB + (size_t)ub * 2 * kEigMaxK));
  o += al256(sizeof(double) * kEigMaxM * kEigMaxB);
  o += al256(sizeof(double) * kEigMaxM);
  return o;
}

}  // namespace sla

using namespace sla;

extern "C" int32_t sla_eigsh(const sla_csr* A, const double* val, int32_t k, double* lambda, double* V,
                             const sla_opts* opts, sla_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (A == nullptr || opts == nullptr || info == nullptr) return SLA_ERR_INVALID;
  const int n = A->n;
  if (n < 1 || k < 1 || k > kEigMaxK || k > n) return SLA_ERR_INVALID;
  if (A->nnz < 0 || A->rowptr == nullptr || (A->nnz > 0 && (A->col == nullptr || val == nullptr)))
    return SLA_ERR_INVALID;
  if (lambda == nullptr || V == nullptr) return SLA_ERR_INVALID;
  if (!(opts->rtol > 0.0) || opts->max_iter < 0 || (opts->use_x0 != 0 && opts->use_x0 != 1) ||
      (opts->precond != SLA_PRECOND_NONE && opts->precond != SLA_PRECOND_JACOBI) || opts->flags != 0)
    return SLA_ERR_INVALID;
  int gb = 0, ub = 0;
  const size_t need = eig_ws_bytes(n, k, &gb, &ub);
  if (ws == nullptr || ((uintptr_t)ws & 255u) != 0 || ws_bytes < need) return SLA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  // carve the workspace (the order of eig_ws_bytes)
  const size_t nn = (size_t)n;
  const int kb = eig_block(n, k);
  char* p = (char*)ws;
  EigPtrs P;
  P.d = (EigDesc*)p;           p += al256(sizeof(EigDesc));
  P.st = (EigState*)p;         p += al256(sizeof(EigState));
  P.dinv = (double*)p;         p += al256(sizeof(double) * nn);
  for (int b = 0; b < 2; ++b) {
    P.S[b] = (double*)p;       p += al256(sizeof(double) * nn * 3 * (size_t)kb);
    P.AS[b] = (double*)p;      p += al256(sizeof(double) * nn * 3 * (size_t)kb);
  }
  P.gpart = (double*)p;        p += al256(sizeof(double) * (size_t)gb * 2 * kEigPairs);
  P.gtot = (double*)p;         p += al256(sizeof(double) * 2 * kEigPairs);
  P.upart = (double*)p;
  p += al256(sizeof(double) * (((size_t)ub + 1) * 2 * kEigMaxB + (size_t)ub * 2 * kEigMaxK));
  P.C = (double*)p;            p += al256(sizeof(double) * kEigMaxM * kEigMaxB);
  P.theta = (double*)p;
  EigDesc d = {};
  d.n = n;
  d.nnz = A->nnz;
  d.k = k;
  d.kb = kb;
  d.ld = 3 * kb;
  d.max_iter = opts->max_iter;
  d.precond = opts->precond;
  d.use_x0 = opts->use_x0;
  d.tol = opts->rtol;
  d.rowptr = A->rowptr;
  d.col = A->col;
  d.val = val;
  d.lambda = lambda;
  d.V = V;
  d.info = info;
  SLA_CUDA_TRY(cudaMemcpyAsync(P.d, &d, sizeof(d), cudaMemcpyHostToDevice, s));
  eig_arm_kernel<<<1, 1, 0, s>>>(P.st);
  eig_init_kernel<<<eig_grid(n, 1024), kEigThreads, 0, s>>>(P);
  // start: Rayleigh-Ritz on X0 alone, then W = D^{-1} R
  eig_spmm_kernel<<<eig_grid(n, 4096), kEigThreads, 0, s>>>(P, 0);
  eig_gram_kernel<<<gb, kEigGramThreads, 0, s>>>(P);
  eig_rr_kernel<<<kRrBlocks, kEigThreads, 0, s>>>(P, gb);
  eig_update_kernel<kEigUpdThreads><<<ub, kEigUpdThreads, 0, s>>>(P);
  SLA_CUDA_TRY(cudaGetLastError());
  for (long long it = 0; it < (long long)opts->max_iter; ++it) {
    eig_spmm_kernel<<<eig_grid(n, 4096), kEigThreads, 0, s>>>(P, 1);
    eig_gram_kernel<<<gb, kEigGramThreads, 0, s>>>(P);
    eig_rr_kernel<<<kRrBlocks, kEigThreads, 0, s>>>(P, gb);
    eig_update_kernel<kEigUpdThreads><<<ub, kEigUpdThreads, 0, s>>>(P);
    if ((it + 1) % kEigPollEvery == 0) {
      int done = 0;
      SLA_CUDA_TRY(cudaMemcpyAsync(&done, &P.st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
      SLA_CUDA_TRY(cudaStreamSynchronize(s));
      if (done) break;
      int bad = 0;
      SLA_CUDA_TRY(cudaMemcpyAsync(&bad, &P.st->bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      SLA_CUDA_TRY(cudaStreamSynchronize(s));
      if (bad) break;
    }
  }
  eig_spmm_kernel<<<eig_grid(n, 4096), kEigThreads, 0, s>>>(P, 2);
  eig_final_kernel<<<ub, kEigThreads, 0, s>>>(P, 0);
  eig_final_kernel<<<ub, kEigThreads, 0, s>>>(P, 1);
  SLA_CUDA_TRY(cudaGetLastError());
  SLA_CUDA_TRY(cudaStreamSynchronize(s));
  return SLA_OK;
}

extern "C" int32_t sla_eig_grad_values(const sla_csr* A, int32_t k, const double* V, const double* g,
                                       double* grad_val, void* stream) {
  if (A == nullptr || k < 1 || k > kEigMaxK || A->n < 0 || A->nnz < 0) return SLA_ERR_INVALID;
  if (A->n == 0 || A->nnz == 0) return SLA_OK;
  if (A->rowptr == nullptr || A->col == nullptr || V == nullptr || g == nullptr || grad_val == nullptr)
    return SLA_ERR_INVALID;
  eig_grad_kernel<<<eig_grid(A->n, 4096), kEigThreads, 0, (cudaStream_t)stream>>>(A->n, k, A->rowptr, A->col,
                                                                                  V, g, grad_val);
  SLA_CUDA_TRY(cudaGetLastError());
  return SLA_OK;
}
