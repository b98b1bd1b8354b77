/*
 * sla.h -- C ABI of the B300 (sm_103a) sparse Krylov solve + adjoint library.
 *
 * The operations follow arXiv 2601.13994 ("torch-sla"): x = A.solve(b) for a
 * sparse A given on a sparsity pattern (App. B), solved by the paper's
 * GPU-native iterative backend -- Jacobi-preconditioned CG for SPD systems
 * (Sec. 3.1, Sec. 4.1, Algorithm 1 with one process) and BiCGStab for
 * nonsymmetric ones (Sec. 1, Sec. 3.1) -- and the linear adjoint backward
 * A^T lambda = dL/dx, dL/db = lambda, dL/dA_ij = -lambda_i x_j (Eq. 2-3).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Matrices are square n x n in CSR form: int32 row pointers (n+1 entries,
 *    rowptr[0] = 0, non-decreasing, rowptr[n] = nnz), int32 column indices
 *    in [0, n) (ascending and distinct inside a row), float64 values.
 *  - Every array pointer is a DEVICE pointer owned by the caller unless the
 *    argument says "host".  The library never frees caller memory and never
 *    allocates device memory: scratch space is a caller-provided workspace
 *    whose size comes from sla_workspace_size().  Workspace pointers must be
 *    256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All work is enqueued on it; no call synchronises the host
 *    except where stated.
 *  - Return value: a negative code is a synchronous argument or CUDA error
 *    and nothing was enqueued; 0 means the work was enqueued.  Numerical
 *    outcomes of a solve (converged, not converged, breakdown, not SPD) are
 *    written to the DEVICE sla_info record(s) when the enqueued work runs.
 *  - Not thread-safe for concurrent calls that share a workspace.
 */
#ifndef SLA_H_
#define SLA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes                                                         */
/* ------------------------------------------------------------------ */
#define SLA_OK 0                /* converged: ||r|| <= max(rtol*||b||, atol) */
#define SLA_NOT_CONVERGED 1     /* max_iter reached (or restarts exhausted)   */
#define SLA_BREAKDOWN 2         /* non-finite scalar, or BiCGStab rho/omega=0 */
#define SLA_NOT_SPD 3           /* CG: A_ii <= 0 with Jacobi, or p^T A p <= 0  */
#define SLA_ERR_INVALID (-1)    /* bad argument (sizes, null pointers, flags)  */
#define SLA_ERR_CUDA (-2)       /* a CUDA runtime call failed                  */
#define SLA_ERR_WORKSPACE (-3)  /* workspace too small or misaligned           */
#define SLA_ERR_TIMEOUT (-4)    /* a bounded device-side wait ran out          */

/* Preconditioners (sla_opts.precond). */
#define SLA_PRECOND_NONE 0
#define SLA_PRECOND_JACOBI 1    /* z = D^{-1} r, D = diag(A) (Sec. 4.1)       */
#define SLA_PRECOND_GGT 2       /* z = G (G^T r): a factored approximate inverse
                                   M^{-1} = G G^T (G lower triangular), e.g.
                                   the learned preconditioner the paper names
                                   as future work (Sec. 5); sla_cg_ggt only   */

/* Flags (sla_opts.flags). */
#define SLA_FLAG_HOST_LOOP 1    /* run the Krylov loop as plain stream launches
                                   driven by the host (checks the device state
                                   every 16 iterations, synchronising the
                                   stream) instead of one graph launch       */
#define SLA_FLAG_NO_COOP 2      /* sla_cg, sla_cg_ggt, sla_bicgstab,
                                   sla_cg_noalloc and sla_adjoint_backward:
                                   use the per-phase kernels (graph or host
                                   loop) even at sizes where the solve would
                                   run as one cooperative launch             */
#define SLA_FLAG_CG_PIPELINED 4 /* sla_cg and sla_adjoint_backward (method
                                   SLA_ADJ_CG), Jacobi or no preconditioner:
                                   pipelined PCG (Ghysels-Vanroose) -- the
                                   three inner products of an iteration form
                                   one reduction, one grid barrier per
                                   iteration -- in one cooperative launch at
                                   every size.  Not with SLA_FLAG_HOST_LOOP or
                                   SLA_FLAG_NO_COOP (SLA_ERR_INVALID).  Needs
                                   the SLA_WS_CG_PIPELINED workspace in sla_cg */

/* Workspace kinds for sla_workspace_size(). */
#define SLA_WS_CG 1
#define SLA_WS_BICGSTAB 2
#define SLA_WS_ADJOINT 3        /* sla_adjoint_backward                        */
#define SLA_WS_TRANSPOSE 4      /* sla_csr_transpose                           */
#define SLA_WS_LIST_TRANSPOSE 13 /* sla_csr_list_transpose: n = total rows,
                                   nnz = total entries of the list          */
#define SLA_WS_COO 5            /* sla_coo_to_csr (pass the COO entry count as nnz) */
#define SLA_WS_CG_GGT 7         /* sla_cg_ggt: pass the entry count of G as nnz */
#define SLA_WS_SPMV_MERGE 9     /* sla_spmv_merge                              */
#define SLA_WS_CG_PIPELINED 10  /* sla_cg with SLA_FLAG_CG_PIPELINED          */
#define SLA_WS_EIGSH 11         /* sla_eigsh: batch = k (1..SLA_EIG_MAX_K)     */
#define SLA_WS_EIG_ADJOINT 12   /* sla_eig_vector_adjoint: batch = k           */

#define SLA_EIG_MAX_K 8         /* largest k of sla_eigsh                      */
#define SLA_WS_CG_MULTI 8       /* sla_cg_multi / sla_adjoint_backward_multi:
                                   batch = number of right-hand sides k       */
#define SLA_WS_BATCHED 6        /* batched CG: n = rows per system (shared
                                   pattern) or total rows with batch = 1 (list) */
#define SLA_WS_ADJOINT_BATCHED 14 /* sla_adjoint_backward_batched_*: (n, nnz,
                                   batch) per system of a shared pattern, or
                                   (total rows, total entries, 1) for a list */

/* Adjoint solve methods (sla_adjoint_backward). */
#define SLA_ADJ_CG 0            /* A symmetric: A^T = A, CG on A               */
#define SLA_ADJ_BICGSTAB 1      /* general A: BiCGStab on the CSR of A^T       */

/* Pattern of a square CSR matrix (all pointers device). */
typedef struct sla_csr {
  int32_t n;              /* rows = columns, >= 0                            */
  int32_t nnz;            /* stored entries, >= 0                            */
  const int32_t* rowptr;  /* [n+1]                                           */
  const int32_t* col;     /* [nnz]                                           */
} sla_csr;

/* CSR of A^T, as produced by sla_csr_transpose (all pointers device):
 * row j of A^T lists the entries of column j of A in increasing row order;
 * perm_t[m] is the index into A's values of the m-th entry of A^T. */
typedef struct sla_csr_t {
  const int32_t* rowptr_t;  /* [n+1]                                         */
  const int32_t* col_t;     /* [nnz]                                         */
  const int32_t* perm_t;    /* [nnz]                                         */
} sla_csr_t;

/* Solver options (host struct, copied at call time). */
typedef struct sla_opts {
  double rtol;            /* relative tolerance on ||r||_2 / ||b||_2, >= 0    */
  double atol;            /* absolute floor on ||r||_2, >= 0                  */
  int32_t max_iter;       /* iteration cap, >= 0                              */
  int32_t max_restarts;   /* true-residual restarts allowed, 0..16            */
  int32_t precond;        /* SLA_PRECOND_*                                    */
  int32_t use_x0;         /* 1: x holds the initial guess; 0: start at x = 0 */
  int32_t flags;          /* SLA_FLAG_* bits, 0 by default                    */
} sla_opts;

/* Per-system solve record (DEVICE memory, written by the enqueued work). */
typedef struct sla_info {
  int32_t iters;          /* Krylov iterations performed                      */
  int32_t status;         /* SLA_OK / SLA_NOT_CONVERGED / ...                 */
  double rel_res;         /* last recursive ||r|| / ||b||                     */
  double true_rel_res;    /* ||b - A x|| / ||b|| recomputed at exit           */
} sla_info;

/* ------------------------------------------------------------------ */
/* Library information                                                  */
/* ------------------------------------------------------------------ */

/* Version string of this build (static storage). */
const char* sla_version(void);

/* Human-readable name of a status code (static storage, never NULL). */
const char* sla_status_string(int32_t code);

/* Self-test of the bounded grid barrier that the cooperative solvers use
 * between phases (no numerical work): one cooperative launch of `blocks`
 * blocks passes `rounds` barriers, each wait bounded by budget_cycles SM
 * clock cycles (the solvers use about 2 s).  Block `absent` (0 <= absent <
 * blocks) never arrives, so every other block's wait runs out and leaves
 * the kernel -- the failure the solvers report as SLA_ERR_TIMEOUT, made
 * here on purpose without any fault; absent < 0: every block arrives.
 * word: DEVICE int32[4], zeroed by the call; afterwards word[0] = blocks
 * whose wait ran out, word[1] = blocks that passed all rounds, word[2] =
 * the barrier counter, word[3] = the error flag (1 after a timeout).
 * Returns SLA_ERR_INVALID (nothing enqueued) for a null word, blocks < 1 or
 * more than can be co-resident, rounds < 0, budget_cycles < 1 or absent >=
 * blocks.  Asynchronous. */
int32_t sla_selftest_grid_barrier(int32_t blocks, int32_t absent, int64_t budget_cycles,
                                  int32_t rounds, int32_t* word, void* stream);

/* FP64 FMA throughput probe (no counterpart in the paper: the measured
 * denominator of the FP64 fractions that the solvers report, since the FP64
 * pipe is a co-limit of every Krylov kernel on this part).  Launches
 * blocks_per_sm x (SM count) blocks of 256 threads, each thread running 8
 * independent FMA chains of `iters` steps; *flops (host) receives the
 * floating-point operations enqueued (2 per FMA).  out: DEVICE double[1],
 * written only in a case that cannot occur (it keeps the work from being
 * dropped).  The caller times the launch on `stream` (CUDA events).  Returns
 * SLA_ERR_INVALID (nothing enqueued) for iters < 1, blocks_per_sm outside
 * [1, 64] or a null pointer.  Asynchronous. */
int32_t sla_fp64_probe(int32_t iters, int32_t blocks_per_sm, double* out, int64_t* flops, void* stream);

/* ------------------------------------------------------------------ */
/* Workspace size query                                                 */
/* ------------------------------------------------------------------ */

/* Bytes of device workspace needed by the entry point `kind` for a system
 * with n rows, nnz entries and `batch` systems (1 for single solves).
 * Host-only; writes *bytes.  Returns SLA_ERR_INVALID for a bad kind or
 * negative sizes. */
int32_t sla_workspace_size(int32_t kind, int32_t n, int32_t nnz,
                           int32_t batch, size_t* bytes);

/* ------------------------------------------------------------------ */
/* Pattern validation                                                   */
/* ------------------------------------------------------------------ */

/* Checks a CSR pattern on the device: rowptr[0] == 0, rowptr non-decreasing,
 * rowptr[n] == nnz, every column in [0, n), columns strictly ascending in
 * each row.  Writes 1 (valid) or 0 (invalid) to the DEVICE int32 *ok.
 * Every access is bounds-checked, so an invalid pattern cannot fault. */
int32_t sla_csr_check(const sla_csr* A, int32_t* ok, void* stream);

/* ------------------------------------------------------------------ */
/* SpMV  y = A x   (the product every Krylov step is built on:            */
/* Algorithm 1 step 3a; torch.sparse in the paper's pytorch backend)     */
/* ------------------------------------------------------------------ */

/* val [nnz], x [n] -> y [n].  x and y must not overlap.  Up to 4 Mi rows one
 * thread sums one row (gathers batched); above, persistent CTAs stream row
 * tiles into shared memory with bulk copies and sum one row per thread, rows
 * of an over-full tile one per warp.  For very uneven row lengths use
 * sla_spmv_merge (sla_spmv_scheme says which). */
/* Load-balanced SpMV along the merge path of the n row ends and the nnz
 * nonzeros: every thread takes 8 consecutive items whatever rows they
 * belong to, so a row of any length costs what its entries cost; rows that
 * cross threads are completed by a fix-up kernel from per-thread partial
 * sums added in a fixed order (deterministic; such rows are rounded in that
 * order rather than as one sequential sum).  Arguments as sla_spmv, plus a
 * workspace of sla_workspace_size(SLA_WS_SPMV_MERGE, n, nnz, 1) bytes
 * (256-byte aligned; SLA_ERR_WORKSPACE otherwise).  Asynchronous. */
int32_t sla_spmv_merge(const sla_csr* A, const double* val, const double* x,
                       double* y, void* ws, size_t ws_bytes, void* stream);

/* Row-length statistics of a pattern: out (DEVICE int32[2]) receives the
 * longest row and the number of rows longer than 1024 entries.
 * Asynchronous. */
int32_t sla_csr_row_stats(const sla_csr* A, int32_t* out, void* stream);

/* SpMV scheme for a pattern from its statistics: SLA_SPMV_ROWS (sla_spmv)
 * or SLA_SPMV_MERGE (sla_spmv_merge), the latter when the longest row is
 * long enough that the one thread (n <= 4 Mi rows) or warp (above) that
 * sla_spmv gives it would take longer than the merge path over the whole
 * matrix: max_row > max(256, (n + nnz) / 8192), resp. / 256. */
#define SLA_SPMV_ROWS 0
#define SLA_SPMV_MERGE 1
int32_t sla_spmv_scheme(int32_t n, int64_t nnz, int32_t max_row);

int32_t sla_spmv(const sla_csr* A, const double* val, const double* x,
                 double* y, void* stream);

/* ------------------------------------------------------------------ */
/* Preconditioned conjugate gradient for SPD A                           */
/* (Algorithm 1 with P = 1; Jacobi preconditioner of Sec. 4.1)           */
/* ------------------------------------------------------------------ */

/* Solves A x = b.  b [n] (read), x [n] (written; read first if use_x0).
 * Stops when ||r_k||_2 <= max(rtol ||b||_2, atol) on the recursive
 * residual, then recomputes b - A x; if that is above twice the target the
 * recurrence restarts from x (at most max_restarts times).  b = 0 gives
 * x = 0 after 0 iterations.  *info (DEVICE) receives the outcome.
 * Systems of up to 2.5 Mi rows run as ONE cooperative kernel launch (every
 * block resident, grid barriers between the phases of an iteration, the
 * convergence test taken identically in every block); larger systems, or
 * calls with SLA_FLAG_NO_COOP, run one CUDA-graph launch whose device-side
 * while-loop decides convergence.  Either way the host is not synchronised.
 * The first graph call with a given workspace address and sizes builds and
 * caches that graph.  With SLA_FLAG_HOST_LOOP the per-phase kernels are
 * launched one by one on `stream` and the call returns after the loop has
 * ended (it synchronises `stream`).  A grid barrier that waits more than
 * about 2 s ends the solve with SLA_ERR_TIMEOUT in *info.
 * With SLA_FLAG_CG_PIPELINED the solve is the pipelined PCG of Ghysels and
 * Vanroose (the merged-reduction CG variant named in App. C): the same
 * exits, restarts and info record, iterates equal to the standard ones in
 * exact arithmetic (so iteration counts agree to within rounding), one
 * cooperative launch with one grid barrier per iteration whatever n is.
 * Workspace: sla_workspace_size(SLA_WS_CG, n, nnz, 1, &bytes), or
 * SLA_WS_CG_PIPELINED with SLA_FLAG_CG_PIPELINED. */
int32_t sla_cg(const sla_csr* A, const double* val, const double* b,
               double* x, const sla_opts* opts, sla_info* info, void* ws,
               size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* CG with a factored preconditioner M^{-1} = G G^T                      */
/* ------------------------------------------------------------------ */

/* Solves A x = b (A SPD) by PCG with z = G (G^T r): two SpMVs per
 * iteration, so M stays SPD whenever G is nonsingular.  G: lower-triangular
 * CSR (device: g_rowptr [n+1], g_col, g_val [nnz_g]); GT: its transpose
 * pattern from sla_csr_transpose of G (perm into g_val; the values of G^T
 * are gathered once per call).  Same stopping rule, true-residual restart,
 * statuses (NOT_SPD on p^T A p <= 0 or r^T z <= 0), execution forms
 * (one cooperative launch up to 1.5 Mi rows unless SLA_FLAG_NO_COOP, else
 * the graph, or the host loop with SLA_FLAG_HOST_LOOP) and info record as
 * sla_cg (opts->precond is ignored).
 * Workspace: SLA_WS_CG_GGT with nnz = nnz_g. */
int32_t sla_cg_ggt(const sla_csr* A, const double* val, const sla_csr* G,
                   const double* g_val, const sla_csr_t* GT, const double* b,
                   double* x, const sla_opts* opts, sla_info* info, void* ws,
                   size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Learned factor G (message-passing network; the paper names learned    */
/* preconditioners as future work, Sec. 5, without a design)             */
/* ------------------------------------------------------------------ */
/* Network: width 32, BF16 weights (W arguments: __nv_bfloat16 bit patterns,
 * row-major [M x K]), FP32 accumulation and activations, FP32 master weights
 * for training.  All arrays are device memory; node arrays are row-major
 * [n x width].  Every reduction is deterministic. */

/* d = diag(A) (FP64 [n]); e[k] = A_ij / sqrt(d_i d_j) (FP32 [nnz]); node
 * features F [n x 3] = (sum_{j!=i} |e_ij|, sum_{j!=i} e_ij, deg_i / 8). */
int32_t sla_mp_features(const sla_csr* A, const double* val, double* d,
                        float* e, float* F, void* stream);

/* CSR of tril(A) (diagonal included): g_rowptr [n+1], g_col / g_src
 * [capacity nnz]; g_src[k] = index in A of entry k; *nnz_g (device int32)
 * receives the count.  Workspace: sla_tril_pattern_ws(n) bytes. */
int32_t sla_tril_pattern(const sla_csr* A, int32_t* g_rowptr, int32_t* g_col,
                         int32_t* g_src, int32_t* nnz_g, void* ws,
                         size_t ws_bytes, void* stream);
size_t sla_tril_pattern_ws(int32_t n);

/* Y = [X1 | X2] W^T + bias (K1 + K2 <= 64 inputs, M <= 96 outputs); Ypre
 * (optional) receives that; Y = relu(.) if relu, plus R (optional residual
 * [n x M]). */
int32_t sla_mp_dense_fwd(int32_t n, int32_t K1, const float* X1, int32_t K2,
                         const float* X2, int32_t M, const void* W_bf16,
                         const float* bias, const float* R, int32_t relu,
                         float* Ypre, float* Y, void* stream);

/* The same layer with the kernel chosen: SLA_MP_DENSE_SIMT (FP32 FMAs on
 * the CUDA cores, each output the sequential sum over k from the bias),
 * SLA_MP_DENSE_TC (tcgen05 tensor cores: each FP32 activation split
 * exactly into three BF16 pieces against the BF16 weights, FP32
 * accumulation in TMEM, bias added after; requires K1, K2 multiples of 4,
 * M a multiple of 16 up to 96 and 16-byte aligned X1, X2, R, Ypre, Y, else
 * SLA_ERR_INVALID) or SLA_MP_DENSE_AUTO (the library's choice).  The two
 * kernels agree to FP32 rounding (the order of the additions differs). */
#define SLA_MP_DENSE_AUTO 0
#define SLA_MP_DENSE_SIMT 1
#define SLA_MP_DENSE_TC 2
int32_t sla_mp_dense_fwd_ex(int32_t n, int32_t K1, const float* X1, int32_t K2,
                            const float* X2, int32_t M, const void* W_bf16,
                            const float* bias, const float* R, int32_t relu,
                            float* Ypre, float* Y, int32_t kernel, void* stream);

/* Nonzero in *out when a tensor-core dense launch's bounded mbarrier wait
 * ran out since the last call (that launch stopped early and its outputs
 * are incomplete); synchronous, resets the flag. */
int32_t sla_mp_tc_errors(int32_t* out);

/* dX = base + dY W[:, col0 : col0 + K] (W has wstride columns; base
 * optional [n x K]). */
int32_t sla_mp_dense_bwdx(int32_t n, int32_t M, const float* dY, int32_t K,
                          const void* W_bf16, int32_t col0, int32_t wstride,
                          const float* base, float* dX, void* stream);

/* dW [M x (K1+K2)] = dY^T [X1 | X2], db [M] = column sums of dY (optional):
 * per-block partials reduced in a fixed order.  Workspace:
 * sla_mp_dense_bwdw_ws(M, K1 + K2) bytes. */
int32_t sla_mp_dense_bwdw(int32_t n, int32_t M, const float* dY, int32_t K1,
                          const float* X1, int32_t K2, const float* X2,
                          float* dW, float* db, void* ws, size_t ws_bytes,
                          void* stream);
size_t sla_mp_dense_bwdw_ws(int32_t M, int32_t K);

/* out = dY * (pre > 0), elementwise over count entries. */
int32_t sla_mp_relu_mask(int64_t count, const float* dY, const float* pre,
                         float* out, void* stream);

/* Agg_i (+)= sum_{j != i} e_ij X_j over the pattern of A (X, Agg [n x 32]);
 * for symmetric A this operator is its own transpose, which the backward
 * pass uses. */
int32_t sla_mp_aggregate(const sla_csr* A, const float* e, const float* X,
                         float* Agg, int32_t accumulate, void* stream);

/* Head on the tril pattern, PQR = [P | Q | R] rows [n x 96]:
 *   off-diagonal (i,j): theta = v . relu(P_i + Q_j + ue e_ij), g = theta / sqrt(d_i)
 *   diagonal:           theta = vd . relu(R_i),                g = exp(theta) / sqrt(d_i)
 * theta [nnz_g] FP32, g_val [nnz_g] FP64. */
int32_t sla_mp_head_fwd(int32_t n, const int32_t* g_rowptr, const int32_t* g_col,
                        const int32_t* g_src, const float* e, const double* d,
                        const float* PQR, const float* ue, const float* v,
                        const float* vd, float* theta, double* g_val,
                        void* stream);

/* Backward of the head for dG = dloss/dg_val: dtheta [nnz_g], dPQR [n x 96],
 * grads [96] = (dv, due, dvd).  gt_* is the CSR of the transposed tril
 * pattern (sla_csr_transpose: gt_row = its column array, i.e. the row of
 * each entry in G).  Workspace: sla_mp_head_bwd_ws(n) bytes. */
int32_t sla_mp_head_bwd(int32_t n, const int32_t* g_rowptr, const int32_t* g_col,
                        const int32_t* g_src, const int32_t* gt_rowptr,
                        const int32_t* gt_row, const int32_t* gt_perm,
                        const float* e, const double* d, const float* PQR,
                        const float* ue, const float* v, const float* vd,
                        const double* g_val, const double* dG, float* dtheta,
                        float* dPQR, float* grads, void* ws, size_t ws_bytes,
                        void* stream);
size_t sla_mp_head_bwd_ws(int32_t n);

/* Training loss of the factor on one system (FP64), with x* = A^{-1} u and
 * y = G G^T u:
 *   loss[0] = (x* - k y)^T A (x* - k y) / (x*^T u),  loss[1] = -2 k / (x*^T u)
 * mode 0: k = 1 (the A-norm error of G G^T u itself);
 * mode 1: k = x*^T A y / y^T A y, the scale that minimises it (0 if y = 0):
 *   the error of the best multiple of G G^T, the preconditioner as PCG
 *   sees it (PCG's iterates do not change when M is scaled).
 * dG = dloss/dg_val on the pattern of G: g_i s_j + u_i h_j with s = G^T u,
 * g = -2 k A e / (x*^T u), e = x* - k y, h = G^T g (in mode 1 the total
 * derivative, since dloss/dk = 0 at the minimising k).  Other modes:
 * SLA_ERR_INVALID.  Workspace: sla_ggt_loss_ws(n) bytes. */
int32_t sla_ggt_loss_grad(const sla_csr* A, const double* val, const sla_csr* G,
                          const double* g_val, const sla_csr_t* GT,
                          const double* u, const double* xstar, int32_t mode,
                          double* loss, double* dG, void* ws, size_t ws_bytes,
                          void* stream);
size_t sla_ggt_loss_ws(int32_t n);

/* The factored sparse approximate inverse (FSAI; Kolotilina and Yeremin)
 * on the pattern G of tril(A) (sla_tril_pattern): the classical,
 * non-learned factor of M^{-1} = G G^T, against which the learned factor is
 * measured (Sec. 5 names learned preconditioners as future work).  Column j
 * of G solves A[P, P] y = e_1 on its rows P = {i >= j : A_ij != 0} and is
 * y / sqrt(y_1), so diag(G^T A G) = I.  A: SPD, columns ascending within
 * each row.  GT: sla_csr_transpose of G.  One thread per column; the block
 * A[P, P] is factored by Cholesky in local memory.  A column with more than
 * 12 entries, or whose block does not factor, gets the Jacobi column
 * 1/sqrt(A_jj) and is counted in *fallbacks (device int, optional, zeroed
 * by the call).  g_out (device, nnz_g) in G's CSR order; must not overlap
 * val.  Asynchronous. */
int32_t sla_fsai_factor(const sla_csr* A, const double* val, const sla_csr* G,
                        const sla_csr_t* GT, double* g_out, int32_t* fallbacks,
                        void* stream);

/* Column normalisation of the factor (applied when the learned factor is
 * formed for a solve): every entry G_ij of column j is divided by
 * sqrt((G^T A G)_jj), (G^T A G)_jj = sum over the entries G_ij, G_kj of
 * column j of G_ij A_ik G_kj, so that diag(G^T A G) = I.  Over positive
 * column scalings this minimises Kaporin's condition number of G^T A G; the
 * factored sparse approximate inverse (FSAI) built column by column has the
 * same normalisation.  A: SPD, columns ascending within each row (A_ik is
 * found by binary search in row i).  GT: sla_csr_transpose of G (row
 * indices of each column and perm into g_val).  A column whose form is not
 * positive and finite is copied unchanged.  g_out (device, nnz_g) may be
 * g_val itself.  One thread per column; asynchronous. */
int32_t sla_ggt_normalize(const sla_csr* A, const double* val, const sla_csr* G,
                          const sla_csr_t* GT, const double* g_val, double* g_out,
                          void* stream);

/* Backward of sla_ggt_normalize for training through the normalisation:
 * given dGn = dL/dGn on the pattern of G (Gn = the normalised factor of
 * g_val, the values BEFORE normalisation), writes dG = dL/dg_val:
 *   dG_aj = dGn_aj / sqrt(q_j) - (A G)_aj w_j / q_j^{3/2},
 *   q_j = (G^T A G)_jj, w_j = sum_i dGn_ij G_ij  (A symmetric),
 * and dG = dGn on a column whose form is not positive and finite (copied
 * unchanged by the forward).  dG may be dGn; neither may overlap g_val
 * (SLA_ERR_INVALID).  Same A, G, GT as sla_ggt_normalize.  One thread per
 * column; asynchronous. */
int32_t sla_ggt_normalize_bwd(const sla_csr* A, const double* val, const sla_csr* G,
                              const sla_csr_t* GT, const double* g_val, const double* dGn,
                              double* dG, void* stream);

/* Adam on FP32 master weights (step t >= 1; clip > 0 clips each gradient
 * entry), writing the BF16 copy the kernels read. */
int32_t sla_adam_step(int32_t np, float* p, const float* g, float* m, float* v,
                      float lr, float b1, float b2, float eps, int32_t t,
                      float clip, void* p_bf16, void* stream);
int32_t sla_to_bf16(int32_t np, const float* p, void* p_bf16, void* stream);

/* ------------------------------------------------------------------ */
/* BiCGStab for nonsymmetric A (van der Vorst 1992; the paper's GPU      */
/* iterative backend offers it for nonsymmetric systems, Sec. 1 and 3.1) */
/* ------------------------------------------------------------------ */

/* Solves A x = b with right-preconditioned BiCGStab (shadow residual
 * r^ = r0; with SLA_PRECOND_JACOBI, M = diag(A)).  Arguments, stopping rule,
 * true-residual restart, execution forms (one cooperative launch up to 896
 * Ki rows unless SLA_FLAG_NO_COOP, else the graph or the host loop) and the
 * info record are as for sla_cg.  Outcomes: OK (also at the half step, when ||s|| meets the
 * target), NOT_CONVERGED, BREAKDOWN (|rho| < 1e-300, r^.v = 0, t.t = 0,
 * omega = 0 or a non-finite scalar), and status SLA_ERR_INVALID in *info when
 * Jacobi meets a zero diagonal.  Iterations count full BiCGStab steps (two
 * SpMVs each).  Workspace: sla_workspace_size(SLA_WS_BICGSTAB, n, nnz, 1,
 * &bytes). */
int32_t sla_bicgstab(const sla_csr* A, const double* val, const double* b,
                     double* x, const sla_opts* opts, sla_info* info,
                     void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Several right-hand sides sharing one matrix                          */
/* ------------------------------------------------------------------ */

/* Largest number of right-hand sides of sla_cg_multi. */
#define SLA_MULTI_MAX_RHS 32

/* A X = B for one SPD A and k right-hand sides (1 <= k <= SLA_MULTI_MAX_RHS):
 * k independent CG / Jacobi-PCG solves (Algorithm 1; Jacobi per Sec. 4.1),
 * each with its own step sizes, stopping test ||r_j|| <= max(rtol ||b_j||,
 * atol), true-residual check and restarts exactly as sla_cg, run by the same
 * kernels so that every iteration reads A once for all k columns.  This is
 * the forward solve of the paper's inverse problem (Sec. 4.6) with a batch
 * of right-hand sides.
 *
 * b, x: [k, n] row-major (right-hand side / solution j at b + j n, x + j n),
 * device, caller-owned, not overlapping; x is the initial guess when
 * opts->use_x0 = 1 and the solution on exit.  info: device array of k
 * records.  opts->precond: SLA_PRECOND_NONE or SLA_PRECOND_JACOBI (others:
 * SLA_ERR_INVALID).  Workspace: sla_workspace_size(SLA_WS_CG_MULTI, n, nnz,
 * k, &bytes) (six n x W FP64 vectors, W = k rounded up to a power of two).
 * Asynchronous on `stream` (one cached CUDA-graph launch, or a host loop
 * with SLA_FLAG_HOST_LOOP). */
int32_t sla_cg_multi(const sla_csr* A, const double* val, int32_t k,
                     const double* b, double* x, const sla_opts* opts,
                     sla_info* info, void* ws, size_t ws_bytes, void* stream);

/* Adjoint backward of sla_cg_multi for symmetric A (Eq. 2-3 per column):
 * A lambda_j = grad_x_j, grad_b_j = lambda_j, and, since the k systems share
 * A's values, grad_val[e] = -sum_j lambda_j[row e] x_j[col e] (summed over
 * the columns in a fixed order).  x, grad_x, grad_b: [k, n] as in
 * sla_cg_multi; grad_b receives lambda and must not overlap x or grad_x.
 * grad_val: [nnz] in CSR entry order (overwritten).  info: device [k],
 * records of the adjoint solves (tolerance relative to ||grad_x_j||).
 * Workspace: SLA_WS_CG_MULTI with batch = k.  Asynchronous on `stream`. */
int32_t sla_adjoint_backward_multi(const sla_csr* A, const double* val,
                                   int32_t k, const double* x,
                                   const double* grad_x, double* grad_b,
                                   double* grad_val, const sla_opts* opts,
                                   sla_info* info, void* ws, size_t ws_bytes,
                                   void* stream);

/* ------------------------------------------------------------------ */
/* Pattern utilities                                                     */
/* ------------------------------------------------------------------ */

/* CSR of A^T (needed by the adjoint A^T lambda = dL/dx of Eq. 3 when A is
 * not symmetric).  Outputs: rowptrT [n+1], colT [nnz], permT [nnz] (device,
 * caller-owned), with valT = val[permT].  Stable: within a row of A^T the
 * entries keep increasing row of A, so the result is unique and matches a
 * sequential counting sort bit for bit.  Workspace: SLA_WS_TRANSPOSE.
 * Asynchronous on `stream`. */
int32_t sla_csr_transpose(const sla_csr* A, int32_t* rowptrT, int32_t* colT,
                          int32_t* permT, void* ws, size_t ws_bytes,
                          void* stream);

/* COO -> CSR ingest for SparseTensor(val, row, col, shape) (App. B).
 * row, col: int64 [m] in [0, n), any order, duplicates allowed; val [m].
 * Outputs (device, caller-owned, capacity m): rowptr [n+1], col_out,
 * val_out (duplicates summed in increasing COO index), perm [m] with
 * perm[e] = CSR slot of COO entry e.  Optional (may be NULL): order [m],
 * the COO entries in (row, col, index) order, and segptr [m+1], where
 * CSR slot s gathers order[segptr[s] .. segptr[s+1]) -- with
 * sla_segment_sum they rebuild CSR values from new COO values on the same
 * pattern.  *nnz_out (device int32) receives the CSR entry count, or -1 if
 * some row/col is out of range (then the other outputs are unspecified).
 * Workspace: SLA_WS_COO with nnz = m.  Asynchronous on `stream`. */
int32_t sla_coo_to_csr(int32_t n, int64_t m, const int64_t* row,
                       const int64_t* col, const double* val, int32_t* rowptr,
                       int32_t* col_out, double* val_out, int32_t* perm,
                       int32_t* order, int32_t* segptr, int32_t* nnz_out,
                       void* ws, size_t ws_bytes, void* stream);

/* out[s] = sum of val[idx[q]] for q in [segptr[s], segptr[s+1]), added in
 * increasing q, for s < nseg (duplicates of a COO input summed in COO
 * order, with idx/segptr from sla_coo_to_csr).  Device arrays. */
int32_t sla_segment_sum(int32_t nseg, const int32_t* segptr,
                        const int32_t* idx, const double* val, double* out,
                        void* stream);

/* Distance-2 colouring of the columns of a CSR pattern, for sparse
 * Jacobians from Jacobian-vector products (the Newton solves of the
 * nonlinear adjoint, Sec. 3.2; Curtis-Powell-Reid): columns that share a row
 * get different colours, so one product per colour, with a tangent of ones
 * on that colour's columns, yields every entry: J_ij is component i of the
 * product for colour[j].  Greedy in column order (smallest colour free of
 * the columns sharing a row).  HOST arrays: rowptr [n+1], col [nnz] (read),
 * colour [n] (written, values 0 .. *ncolours-1).  SLA_ERR_INVALID for a
 * malformed pattern (decreasing rowptr, column out of range).  Synchronous;
 * no device work. */
int32_t sla_colour_columns(int32_t n, const int32_t* rowptr,
                           const int32_t* col, int32_t* colour,
                           int32_t* ncolours);

/* out[k] = val[perm[k]] for k < nnz: the values of A^T in CSR-of-A^T order,
 * or gradients mapped back to the caller's COO order (perm of
 * sla_coo_to_csr).  Device arrays; asynchronous. */
int32_t sla_gather_values(int64_t nnz, const int32_t* perm, const double* val,
                          double* out, void* stream);

/* ------------------------------------------------------------------ */
/* Eigenvalues (Sec. 3.2 "Eigenvalue problems", Eq. 4; LOBPCG, Sec. 3.3) */
/* ------------------------------------------------------------------ */

/* The k smallest eigenpairs of symmetric positive definite A by LOBPCG
 * (Knyazev 2001) with the Jacobi preconditioner (opts->precond) or none.
 * k in 1..SLA_EIG_MAX_K, k <= n.  The iteration carries min(k + 2, n)
 * vectors (two guard vectors, so that a cluster split at the k-th
 * eigenvalue does not stall the last wanted pair).  opts: rtol = the
 * convergence tolerance (> 0): stop when ||A x_i - theta_i x_i|| <= rtol
 * |theta_i| ||x_i|| for the k wanted pairs;
 * max_iter = iteration cap; use_x0 = 1: V holds the start block [n][k]
 * (row-major), else a fixed pseudo-random block (splitmix64 of the entry
 * index); flags must be 0.  Outputs (device): lambda [k] ascending, V [n][k]
 * row-major with unit columns, *info: iters, status (OK, NOT_CONVERGED,
 * NOT_SPD for a non-positive diagonal with Jacobi, BREAKDOWN when the
 * search space loses rank below k), rel_res = the largest relative
 * residual of the last iteration, true_rel_res = the same from a fresh
 * product at exit.  Host-driven: three kernels per iteration (SpMM; Gram
 * sums + Rayleigh-Ritz in the last block; update), the device state read
 * every 8 iterations; the call synchronises `stream` before returning.
 * Workspace: sla_workspace_size(SLA_WS_EIGSH, n, nnz, k, &bytes). */
int32_t sla_eigsh(const sla_csr* A, const double* val, int32_t k,
                  double* lambda, double* V, const sla_opts* opts,
                  sla_info* info, void* ws, size_t ws_bytes, void* stream);

/* Hellmann-Feynman gradient of the eigenvalues on the pattern (Eq. 4):
 * grad_val[e] = sum_i g[i] V[row_e][i] V[col_e][i], with V [n][k] the unit
 * eigenvectors (row-major) and g [k] = dL/dlambda (device arrays).  Exact
 * for simple eigenvalues.  Asynchronous on `stream`. */
int32_t sla_eig_grad_values(const sla_csr* A, int32_t k, const double* V,
                            const double* g, double* grad_val, void* stream);

/* Eigenvector adjoint (Sec. 3.2: one deflated linear solve per pair).  For
 * the unit eigenvectors V [n][k] (row-major) of symmetric A with simple
 * eigenvalues lambda [k] and upstream gradients gV [n][k] = dL/dV, writes
 * mu [n][k]: column j solves (A - lambda_j I) mu_j = (I - v_j v_j^T) gV_j
 * with v_j^T mu_j = 0 -- the adjoint of the constrained residual
 * (A v - lambda v, (v^T v - 1)/2), whose multiplier on the normalisation
 * is eliminated.  The eigenvector part of dL/dA is then -mu_j[a] v_j[b]
 * (sla_eig_vector_grad_values); the eigenvalue part is Eq. 4.  mu_j is the
 * closed form sum_{l != j} (v_l^T gV_j) / (lambda_l - lambda_j) v_l over
 * the other given pairs plus the solution in span(V)^perp, found by CG on
 * (I - V V^T)(A - lambda_j I)(I - V V^T) with the preconditioner
 * (I - V V^T) D^{-1} (I - V V^T), D = diag(A) (opts->precond JACOBI) or I
 * (NONE): SPD there when lambda_j lies below every eigenvalue not in V, as
 * for the k smallest pairs of sla_eigsh.  All k solves in one cooperative
 * launch (three bounded grid barriers per iteration; asynchronous).
 * opts: rtol, atol (stop when ||r_j|| <= max(rtol ||b_j||, atol), b_j =
 * (I - V V^T) gV_j), max_iter, precond; use_x0 and flags must be 0.
 * info [k] (device): per pair iters, status (OK; NOT_CONVERGED; NOT_SPD for
 * a non-positive diagonal with Jacobi or a non-positive curvature, i.e.
 * lambda_j not below the spectrum outside V; BREAKDOWN for a non-finite
 * scalar or a repeated eigenvalue, |lambda_l - lambda_j| <= 1e-12
 * max(|lambda_l|, |lambda_j|), where the gradient is not defined and the
 * pair l is left out; SLA_ERR_TIMEOUT when a barrier ran out), rel_res =
 * the recursive ||r_j|| / ||b_j||, true_rel_res = ||b_j - (A - lambda_j I)
 * y_j|| / ||b_j|| for the span(V)^perp part y_j.  b_j with ||b_j|| <=
 * 64 eps ||gV_j|| (gV_j in span(V), or k = n) is rounding noise: y_j = 0,
 * no iteration, both residuals reported as 0.
 * Returns SLA_ERR_CUDA when the device has no cooperative launch.
 * Workspace: sla_workspace_size(SLA_WS_EIG_ADJOINT, n, nnz, k, &bytes). */
int32_t sla_eig_vector_adjoint(const sla_csr* A, const double* val, int32_t k,
                               const double* lambda, const double* V,
                               const double* gV, double* mu,
                               const sla_opts* opts, sla_info* info,
                               void* ws, size_t ws_bytes, void* stream);

/* Eigenvector part of the gradient on the pattern: grad_val[e] = -sum_j
 * mu[row_e][j] V[col_e][j] (accumulate = 1: subtracted from grad_val
 * instead of overwriting it).  mu, V [n][k] row-major device arrays.
 * Asynchronous on `stream`. */
int32_t sla_eig_vector_grad_values(const sla_csr* A, int32_t k,
                                   const double* mu, const double* V,
                                   double* grad_val, int32_t accumulate,
                                   void* stream);

/* ------------------------------------------------------------------ */
/* Linear adjoint backward (Eq. 2-3)                                     */
/* ------------------------------------------------------------------ */

/* Matrix gradient of Eq. 3 on the pattern:
 *   grad_val[k] = -lambda[i] * x[col[k]]   for every entry k of row i.
 * lambda [n], x [n] -> grad_val [nnz]; one pass over the entries. */
int32_t sla_grad_values(const sla_csr* A, const double* lambda,
                        const double* x, double* grad_val, void* stream);

/* Backward pass of x = A^{-1} b (Eq. 2 with J = A, Eq. 3): solves
 * A^T lambda = grad_x, then writes grad_b = lambda [n] and
 * grad_val[k] = -lambda[i] x[col[k]] [nnz].  x is the forward solution.
 * method SLA_ADJ_CG: A symmetric (A^T = A), CG on A; AT may be NULL.
 * method SLA_ADJ_BICGSTAB: BiCGStab on A^T given by AT (sla_csr_transpose
 * of A); its values are gathered into the workspace.
 * opts: tolerance of the adjoint solve relative to ||grad_x|| (use_x0 is
 * ignored: lambda starts at 0); *info receives the adjoint solve's record.
 * grad_b must differ from x and grad_x (lambda is written into grad_b before
 * the gradient pass reads x), and grad_val must overlap neither x nor
 * grad_b: SLA_ERR_INVALID otherwise, nothing enqueued.
 * Workspace: SLA_WS_ADJOINT.  Asynchronous (graph launch + one kernel). */
int32_t sla_adjoint_backward(const sla_csr* A, const sla_csr_t* AT,
                             const double* val, const double* x,
                             const double* grad_x, double* grad_b,
                             double* grad_val, int32_t method,
                             const sla_opts* opts, sla_info* info, void* ws,
                             size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Batched Jacobi-PCG in one persistent launch (SparseTensor batch with a  */
/* shared pattern, SparseTensorList with distinct patterns; Sec. 3.1)     */
/* ------------------------------------------------------------------ */

/* Each system is solved by one CTA running the complete PCG recurrence of
 * sla_cg (same stopping rule, restart and statuses; info[s] per system);
 * persistent CTAs take systems from a counter, so one launch serves any
 * batch and a converged system frees its CTA for the next.  The Krylov
 * vectors stay in shared memory when 5 n doubles fit, else in the
 * workspace.  config: 0 = automatic; low 4 bits 1/2/3 = 256/512/1024
 * threads per CTA, value 16 = vectors in global memory, bits 8-9 = log2 of the
 * threads per row in the SpMVs (1, 2, 4, 8: a row summed by that many adjacent
 * threads, then a fixed butterfly), bits 10-11 = log2 of the systems per CTA
 * (1, 2, 4: each solved by NT / SPC threads with a named barrier of their
 * own; only with one thread per row), value 32 (lists) = no block teams
 * for the large systems; bits 8-11 shape the single-CTA kernel (for lists
 * with the teams off); other bits SLA_ERR_INVALID (the autotuner in the
 * Python layer times these shapes per batch).  The call only enqueues kernels (no host
 * synchronisation), so it can be captured in a CUDA graph.
 * Shared pattern: val [batch, nnz], b and x [batch, n] row-major.
 * Workspace: SLA_WS_BATCHED with (n, batch). */
int32_t sla_cg_batched_shared(const sla_csr* A, int32_t batch,
                              const double* val, const double* b, double* x,
                              const sla_opts* opts, sla_info* info,
                              int32_t config, void* ws, size_t ws_bytes,
                              void* stream);

/* Distinct patterns, concatenated: n_off, nnz_off [batch+1] (device) give
 * system s rows [n_off[s], n_off[s+1]) of b and x and entries
 * [nnz_off[s], nnz_off[s+1]) of col and val; rowptr holds the per-system
 * row pointers (each starting at 0, n_s + 1 entries) back to back, so system
 * s's start at rowptr + n_off[s] + s; columns are local.  n_max = largest
 * n_s, total_rows = n_off[batch].  order (device, optional): the order in
 * which CTAs take systems (largest first balances the load).
 * With the teams on (the default) the batch is one cooperative launch:
 * systems with at least 32768 entries are solved first, each by a team of 3
 * CTAs (the same recurrence with team-wide reductions and barriers bounded
 * like sla_cg's), so that the largest systems do not run at one SM's rate
 * while the rest of the GPU idles; a team that reaches the small systems
 * splits into single CTAs, which take them one each (vectors in the
 * workspace).  config bit 32 turns the teams off (the persistent single-CTA
 * kernel above takes every system).  config bit 64 (with the teams on)
 * solves the team systems by the pipelined PCG of SLA_FLAG_CG_PIPELINED
 * instead (one merged reduction and one team barrier per iteration; results
 * agree with the standard form to rounding); single CTAs keep the standard
 * form.  Still no host synchronisation.
 * Workspace: SLA_WS_BATCHED with (total_rows, 1). */
int32_t sla_cg_batched_list(int32_t batch, int32_t n_max, int32_t total_rows,
                            const int32_t* n_off, const int32_t* nnz_off,
                            const int32_t* rowptr, const int32_t* col,
                            const double* val, const double* b, double* x,
                            const int32_t* order, const sla_opts* opts,
                            sla_info* info, int32_t config, void* ws,
                            size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* Batched BiCGStab in one persistent launch (the nonsymmetric members of  */
/* a SparseTensor batch or SparseTensorList, Sec. 3.1 and App. B)          */
/* ------------------------------------------------------------------ */

/* Each system is solved by one CTA running the complete BiCGStab of
 * sla_bicgstab (van der Vorst, r^ = r0, right Jacobi preconditioning, exit
 * at the half step when ||s|| meets the target; the same breakdown tests,
 * true-residual check, restarts and statuses; info[s] per system, a zero
 * or non-finite diagonal with Jacobi giving status SLA_ERR_INVALID with NaN
 * residuals in that system's record only).  Persistent CTAs take systems
 * from a counter (in `order` for lists, largest first by default), so a
 * converged system frees its CTA for the next.  The seven n-vectors of a
 * system (r, r^, D^-1 p, A D^-1 p, D^-1 s, A D^-1 s, D^-1) stay in shared
 * memory as far as they fit, the rest in the workspace.
 * config: 0 = automatic; low 4 bits 1/2/3 = 256/512/1024 threads per CTA;
 * config | 16 = every vector in the workspace; other bits SLA_ERR_INVALID.
 * opts->flags must be 0.  The call only enqueues kernels (no host
 * synchronisation).  b and x must differ.
 * Shared pattern: val [batch, nnz], b and x [batch, n] row-major.
 * Workspace: SLA_WS_BATCHED with (n, batch). */
int32_t sla_bicgstab_batched_shared(const sla_csr* A, int32_t batch,
                                    const double* val, const double* b,
                                    double* x, const sla_opts* opts,
                                    sla_info* info, int32_t config, void* ws,
                                    size_t ws_bytes, void* stream);

/* Distinct patterns in the concatenated layout of sla_cg_batched_list
 * (n_off, nnz_off, rowptr back to back, local columns, optional order).
 * A single CTA runs at one SM's FP64 rate, so by default (config bit 32
 * clear, n_max >= 2048, a device with cooperative launch) the systems with
 * at least a threshold of entries are solved by teams of blocks of one
 * cooperative launch (the same recurrence; team sums added in a fixed
 * order; 512 threads per block, every vector in the workspace), and the
 * rest of the queue by single blocks of that launch.  A team barrier that
 * waits longer than its bound sets status SLA_ERR_TIMEOUT in the records
 * of the systems left unsolved.
 * config: bit 32 = one CTA per system, shaped by the low 5 bits as for
 * the shared pattern; without it, bits 8-9 = team size (0: 3 blocks, 1: 2,
 * 2: 4, 3: 6), bits 10-11 = entry threshold (0: 32768, 1: 16384,
 * 2: 65536, 3: 131072); other bits SLA_ERR_INVALID.
 * Workspace: SLA_WS_BATCHED with (total_rows, 1). */
int32_t sla_bicgstab_batched_list(int32_t batch, int32_t n_max,
                                  int32_t total_rows, const int32_t* n_off,
                                  const int32_t* nnz_off,
                                  const int32_t* rowptr, const int32_t* col,
                                  const double* val, const double* b,
                                  double* x, const int32_t* order,
                                  const sla_opts* opts, sla_info* info,
                                  int32_t config, void* ws, size_t ws_bytes,
                                  void* stream);

/* CSR of A_s^T for every system of a list (Eq. 3 needs A^T lambda = dL/dx
 * per system): the same concatenated layout as the input (rowptrT: the
 * per-system row pointers of the transposes back to back, total_rows +
 * batch entries; colT: local columns; permT: for each entry of A_s^T the
 * index into the concatenated values, so valT = val[permT] is one
 * sla_gather_values call over all systems).
 * Within a row of A_s^T the entries keep increasing column order (stable),
 * bit for bit what sla_csr_transpose gives for each system alone.  Outputs
 * must not alias the inputs.  Workspace: SLA_WS_LIST_TRANSPOSE with
 * (total_rows, total_nnz).  Asynchronous. */
int32_t sla_csr_list_transpose(int32_t batch, int32_t total_rows,
                               int32_t total_nnz, const int32_t* n_off,
                               const int32_t* nnz_off, const int32_t* rowptr,
                               const int32_t* col, int32_t* rowptrT,
                               int32_t* colT, int32_t* permT, void* ws,
                               size_t ws_bytes, void* stream);

/* out[s, m] = val[s, perm[m]] for every system s of a shared pattern
 * (val, out [batch, nnz]): the values of every A_s^T in CSR-of-A^T order
 * (perm = perm_t of sla_csr_transpose).  out must not overlap val.
 * Device arrays; asynchronous. */
int32_t sla_gather_values_batched(int32_t batch, int64_t nnz,
                                  const int32_t* perm, const double* val,
                                  double* out, void* stream);

/* Batched Eq. 3 gradient: grad_val[s, k] = -lambda[s, i] x[s, col k] for the
 * entries k of row i of system s.  shared_pattern = 1: (n, nnz, rowptr,
 * col) is the pattern, lambda/x [batch, n], grad_val [batch, nnz];
 * shared_pattern = 0: the concatenated layout of sla_cg_batched_list with
 * n = n_max. */
int32_t sla_grad_values_batched(int32_t batch, int32_t shared_pattern,
                                int32_t n, int32_t nnz, const int32_t* rowptr,
                                const int32_t* col, const int32_t* n_off,
                                const int32_t* nnz_off, const double* lambda,
                                const double* x, double* grad_val,
                                void* stream);

/* Batched backward pass of x_s = A_s^{-1} b_s (Eq. 3 for every system of a
 * batch, Sec. 3.1): one batched solve of A_s^T lambda_s = grad_x[s] for all
 * systems, then grad_b = lambda and grad_val[s, k] = -lambda[s, i] x[s, col k]
 * on each system's own entries (sla_grad_values_batched).
 * method SLA_ADJ_CG: every A_s symmetric, batched CG on the A_s themselves
 * (sla_cg_batched_*); AT may be NULL.  method SLA_ADJ_BICGSTAB: batched
 * BiCGStab on the CSR of A^T (sla_bicgstab_batched_*), every system's
 * values gathered into the workspace first.
 * opts: tolerances of the adjoint solves relative to ||grad_x[s]||; use_x0
 * is ignored (lambda starts at 0); flags must be 0.  info[s] receives
 * system s's adjoint solve record.  config: the launch shape of the
 * method's batched solver (0 = automatic; the bits of sla_cg_batched_* or
 * sla_bicgstab_batched_*).  x is the forward solution.  grad_b must overlap
 * neither x nor grad_x, and grad_val neither x nor grad_b: SLA_ERR_INVALID
 * otherwise, nothing enqueued.  Device arrays; asynchronous (no host
 * synchronisation: the launches can be captured in a CUDA graph).
 *
 * Shared pattern: A (n, nnz, rowptr, col) with AT = sla_csr_transpose of A
 * for BiCGStab; val and grad_val [batch, nnz]; x, grad_x, grad_b [batch, n]
 * row-major.  Workspace: SLA_WS_ADJOINT_BATCHED with (n, nnz, batch). */
int32_t sla_adjoint_backward_batched_shared(const sla_csr* A, const sla_csr_t* AT,
                                            int32_t batch, const double* val,
                                            const double* x, const double* grad_x,
                                            double* grad_b, double* grad_val,
                                            int32_t method, const sla_opts* opts,
                                            sla_info* info, int32_t config,
                                            void* ws, size_t ws_bytes, void* stream);

/* Distinct patterns in the concatenated layout of sla_cg_batched_list
 * (n_off, nnz_off, rowptr back to back, local columns, optional order);
 * total_nnz = nnz_off[batch].  For BiCGStab, rowptr_t, col_t and perm_t are
 * the list's transposes from sla_csr_list_transpose (the same offsets
 * serve, since A_s^T has A_s's size and entry count); NULL for CG.  val,
 * grad_val [total_nnz]; x, grad_x, grad_b [total_rows].
 * Workspace: SLA_WS_ADJOINT_BATCHED with (total_rows, total_nnz, 1). */
int32_t sla_adjoint_backward_batched_list(int32_t batch, int32_t n_max,
                                          int32_t total_rows, int32_t total_nnz,
                                          const int32_t* n_off, const int32_t* nnz_off,
                                          const int32_t* rowptr, const int32_t* col,
                                          const int32_t* rowptr_t, const int32_t* col_t,
                                          const int32_t* perm_t, const double* val,
                                          const double* x, const double* grad_x,
                                          double* grad_b, double* grad_val,
                                          const int32_t* order, int32_t method,
                                          const sla_opts* opts, sla_info* info,
                                          int32_t config, void* ws, size_t ws_bytes,
                                          void* stream);

/* ------------------------------------------------------------------ */
/* Distributed layer (Sec. 3.3, Eqs. 5-6; Algorithm 1 of App. C), with    */
/* its P row-block partitions emulated on one GPU                         */
/* ------------------------------------------------------------------ */

/* Layout (built on the host by the Python layer, device arrays here):
 * partition p owns rows [row_off[p], row_off[p+1]); its extended local
 * vector holds its |O_p| owned entries, then its halo H_p (the sorted
 * global columns outside O_p that its rows reference); all partitions'
 * extended vectors lie back to back (total_ext entries), src[e] = the global
 * index extended entry e holds.  The local matrices of all partitions form
 * one CSR with n rows and columns in the extended space (col_ext). */

/* The halo exchange H (Eq. 5): x_ext[e] = x[src[e]] -- every partition's
 * owned entries and the values its halo receives from their owners.  x
 * [n], x_ext [total_ext], distinct.  Asynchronous. */
int32_t sla_dist_halo_gather(int64_t total_ext, const int32_t* src,
                             const double* x, double* x_ext, void* stream);

/* The transposed halo exchange H^T (Eq. 6): g_x[i] = g_ext[own_pos[i]] +
 * sum over t in [hptr[i], hptr[i+1]) of g_ext[hlist[t]], i.e. each owner
 * sums the halo gradients its entry received from every partition that
 * holds it (hlist ordered by partition, then halo position: a fixed
 * order).  own_pos [n], hptr [n+1], hlist [hptr[n]] device int32; g_ext
 * [total_ext] and g_x [n] distinct.  Asynchronous. */
int32_t sla_dist_halo_scatter(int32_t n, const int32_t* own_pos,
                              const int32_t* hptr, const int32_t* hlist,
                              const double* g_ext, double* g_x, void* stream);

/* All-reduced inner products (Algorithm 1's all_reduce): for j < k (1..3),
 * each partition's local sum of a[j] . b[j] over its rows (a fixed-shape
 * reduction of 8 block partials), then the sum over partitions in order
 * 0..P-1 into out[j] (device [k]); rank_part (device [k][P], optional)
 * receives the per-partition sums.  a, b: HOST arrays of k device pointers
 * to [n] vectors; row_off device [P+1]; partial: device scratch of 8 P k
 * doubles.  Asynchronous. */
int32_t sla_dist_dots(int32_t P, const int32_t* row_off, int32_t k,
                      const double* const* a, const double* const* b,
                      double* partial, double* out, double* rank_part,
                      void* stream);

/* D^{-1} of the distributed matrix: A_ii is the entry of row i whose
 * extended column is own_pos[i]; *bad (device int, zeroed by the call) = 1
 * if some A_ii <= 0.  Asynchronous. */
int32_t sla_dist_diag_inv(int32_t n, const int32_t* rowptr,
                          const int32_t* col_ext, const double* val,
                          const int32_t* own_pos, double* dinv, int32_t* bad,
                          void* stream);

/* Algorithm 1's local steps with the Jacobi preconditioner, all partitions
 * at once (alpha, beta are the all-reduced scalars, passed by value):
 * start: r = b - y (y = A x), z = D^{-1} r, p = z;
 * update: x += alpha p, r -= alpha q, z = D^{-1} r;
 * direction: p = z + beta p.  Device [n] vectors; asynchronous. */
int32_t sla_dist_cg_start(int32_t n, const double* b, const double* y,
                          const double* dinv, double* r, double* z, double* p,
                          void* stream);
int32_t sla_dist_cg_update(int32_t n, double alpha, const double* p,
                           const double* q, const double* dinv, double* x,
                           double* r, double* z, void* stream);
int32_t sla_dist_cg_direction(int32_t n, double beta, const double* z,
                              double* p, void* stream);

/* Value gradient of y = A_local x_ext on every partition's own entries (no
 * communication): out[k] = gy[i] * x_ext[col_ext[k]] for the entries k of
 * row i.  Asynchronous. */
int32_t sla_dist_outer_values(int32_t n, const int32_t* rowptr,
                              const int32_t* col_ext, const double* gy,
                              const double* x_ext, double* out, void* stream);

/* ------------------------------------------------------------------ */
/* Allocation-free CG (no counterpart in the paper)                      */
/* ------------------------------------------------------------------ */

/* Largest n accepted by sla_cg_noalloc. */
#define SLA_NOALLOC_MAX_N 393216

/* The Jacobi-PCG solve of sla_cg, for callers that cannot
 * allocate device memory at the time they solve: code that runs inside a
 * framework's allocator or memory hook (a cudaMalloc there would re-enter the
 * allocator), serving or real-time hosts that reserve all device memory at
 * start-up and forbid later allocations, and plug-ins handed a stream but no
 * allocator.  The caller passes inputs and outputs only; no workspace.
 *
 * Scratch space: a fixed array of about 16 MB (room for n <= SLA_NOALLOC_MAX_N)
 * built into the library.  Every device that loads the library holds it until
 * the process exits.  n > SLA_NOALLOC_MAX_N returns SLA_ERR_WORKSPACE and
 * enqueues nothing.  The call never calls cudaMalloc, cudaFree or any
 * allocating routine.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so an address never
 * outlives a context reset.  The first call on a device can also load the
 * library's device code there; make it before any stream capture.  All calls
 * on a device share the one array, which keeps the last
 * call's contents (everything a solve needs zeroed is cleared at its start):
 * calls that overlap on the GPU -- different streams, threads or processes
 * sharing the context -- race and must be serialised by the caller.
 *
 * Systems that sla_cg solves in one cooperative launch are solved the same
 * way here, with the same kernel and the same results (the call returns
 * without synchronising).  The others -- and every call with
 * SLA_FLAG_HOST_LOOP or SLA_FLAG_NO_COOP -- are driven from the host (no
 * graph objects are created) with the per-phase kernels in their unscaled
 * form (z = D^-1 r in the scratch array; the fixed array has no room for
 * D^-1/2 A D^-1/2), so they can differ from sla_cg's per-phase path by
 * rounding and by a few iterations; the call then returns after the solve
 * has finished on `stream`.  That host-driven form polls and synchronises
 * `stream`, so it returns SLA_ERR_INVALID, enqueueing nothing, while
 * `stream` is being captured.  Other arguments, options and the *info
 * record behave as for sla_cg. */
int32_t sla_cg_noalloc(const sla_csr* A, const double* val, const double* b,
                       double* x, const sla_opts* opts, sla_info* info,
                       void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SLA_H_ */
