/*
 * sla_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the sparse
 * Krylov solve + adjoint path of "torch-sla: Differentiable Sparse Linear
 * Algebra with Adjoint Solvers ..." (arXiv 2601.13994).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code, header or constant generator
 * with the CUDA library; the status codes below are re-declared here on
 * purpose so that the two sides stay independent.
 *
 * Every routine is the plain definition or the algorithm's steps in the
 * paper's order, with sequential (left-to-right) summation.  Compile with
 * -O2 -ffp-contract=off so that a*b+c is never fused behind the reader's back.
 *
 * Storage: CSR with int32 row pointers / column indices and float64 values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  OR_OK = 0,
  OR_NOT_CONVERGED = 1,
  OR_BREAKDOWN = 2,
  OR_NOT_SPD = 3,
  OR_ERR_INVALID = -1
};

/* ---------------------------------------------------------------------- */
/* Vector helpers (plain loops).                                           */
/* ---------------------------------------------------------------------- */
static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

/* ---------------------------------------------------------------------- */
/* SpMV y = A x (the product every Krylov step is built on; torch.sparse   */
/* in the paper's pytorch backend, Fig. 1 / Algorithm 1 step 3a).          */
/* y_i = sum_{k in row i} val_k * x_{col_k}                                */
/* ---------------------------------------------------------------------- */
void or_spmv(int32_t n, const int32_t* rowptr, const int32_t* col,
             const double* val, const double* x, double* y) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* Jacobi diagonal: d_i = A_ii (sum of stored entries on the diagonal;     */
/* Jacobi preconditioning of the CG backend, Sec. 4.1 / Tab. 3 caption).   */
void or_diag(int32_t n, const int32_t* rowptr, const int32_t* col,
             const double* val, double* d) {
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) s += val[k];
    d[i] = s;
  }
}

/* Lower-triangular factor application z = G (G^T r) on CSR G.  Used as    */
/* the learned approximate inverse M^{-1} = G G^T (paper: future work,     */
/* Sec. 5).  Written as two plain products, G^T first.                     */
static void ggt_apply(int32_t n, const int32_t* growptr, const int32_t* gcol,
                      const double* gval, const double* r, double* tmp,
                      double* z) {
  /* tmp = G^T r :  tmp_j = sum_i G_ij r_i */
  for (int32_t j = 0; j < n; ++j) tmp[j] = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = growptr[i]; k < growptr[i + 1]; ++k)
      tmp[gcol[k]] += gval[k] * r[i];
  /* z = G tmp */
  or_spmv(n, growptr, gcol, gval, tmp, z);
}

/* Preconditioner  z = M^{-1} r.  kind 0: identity, 1: Jacobi, 2: G G^T.   */
typedef struct {
  int kind;
  const double* dinv;
  int32_t n;
  const int32_t* growptr;
  const int32_t* gcol;
  const double* gval;
  double* tmp;
} precond_t;

static void apply_precond(const precond_t* M, const double* r, double* z) {
  int32_t n = M->n;
  if (M->kind == 0) {
    for (int32_t i = 0; i < n; ++i) z[i] = r[i];
  } else if (M->kind == 1) {
    for (int32_t i = 0; i < n; ++i) z[i] = M->dinv[i] * r[i];
  } else {
    ggt_apply(n, M->growptr, M->gcol, M->gval, r, M->tmp, z);
  }
}

/* ---------------------------------------------------------------------- */
/* Preconditioned conjugate gradient for SPD A.                            */
/* Algorithm 1 (App. C) with P = 1 (every all_reduce is a plain sum) and   */
/* a preconditioner z = M^{-1} r (Jacobi by default, Sec. 4.1).  Readings: */
/*  - stop when ||r_k||_2 <= max(rtol*||b||_2, atol) on the recursive r;   */
/*  - x0 = 0 unless use_x0 (Algorithm 1 step 1);                            */
/*  - b = 0 returns x = 0 after 0 iterations;                              */
/*  - A_ii <= 0 (Jacobi) or p^T A p <= 0 stops with NOT_SPD;                */
/*  - a non-finite scalar stops with BREAKDOWN;                            */
/*  - on exit the true residual ||b - A x|| / ||b|| is computed; if it is   */
/*    more than twice the target, the recurrence is restarted from the     */
/*    current x (r = b - A x), at most max_restarts times.                  */
/* out_info[0] = iterations, out_info[1] = status; out_res[0] = recursive  */
/* relative residual, out_res[1] = true relative residual.                 */
/* ---------------------------------------------------------------------- */
static int pcg_core(int32_t n, const int32_t* rowptr, const int32_t* col,
                    const double* val, const double* b, double* x,
                    double rtol, double atol, int32_t max_iter,
                    int32_t max_restarts, int32_t use_x0, const precond_t* M,
                    int32_t* out_info, double* out_res) {
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int status = OR_NOT_CONVERGED;
  int32_t it = 0;
  double bnorm = nrm2(n, b);
  double thresh = rtol * bnorm > atol ? rtol * bnorm : atol;
  double rnorm = 0.0;

  if (!use_x0)
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;

  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    out_info[0] = 0;
    out_info[1] = OR_OK;
    out_res[0] = 0.0;
    out_res[1] = 0.0;
    free(r); free(z); free(p); free(q);
    return OR_OK;
  }

  for (int32_t restart = 0; restart <= max_restarts; ++restart) {
    /* r = b - A x ; z = M^{-1} r ; p = z ; rho = r^T z */
    or_spmv(n, rowptr, col, val, x, q);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    apply_precond(M, r, z);
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot(n, r, z);
    rnorm = nrm2(n, r);
    status = OR_NOT_CONVERGED;
    if (!isfinite(rho) || !isfinite(rnorm)) { status = OR_BREAKDOWN; break; }

    while (!(rnorm <= thresh) && it < max_iter) {
      or_spmv(n, rowptr, col, val, p, q);          /* q = A p        */
      double pq = dot(n, p, q);                     /* p^T A p        */
      if (!isfinite(pq)) { status = OR_BREAKDOWN; break; }
      if (!(pq > 0.0)) { status = OR_NOT_SPD; break; }
      double alpha = rho / pq;
      for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
      apply_precond(M, r, z);
      double rho_new = dot(n, r, z);
      rnorm = nrm2(n, r);
      ++it;
      if (!isfinite(rho_new) || !isfinite(rnorm)) { status = OR_BREAKDOWN; break; }
      if (rnorm <= thresh) { status = OR_OK; break; }
      if (!(rho_new > 0.0)) { status = OR_NOT_SPD; break; }
      double beta = rho_new / rho;
      for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rho = rho_new;
    }
    if (rnorm <= thresh) status = OR_OK;
    if (status != OR_OK) break;
    /* true residual check */
    or_spmv(n, rowptr, col, val, x, q);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double tnorm = nrm2(n, r);
    if (tnorm <= 2.0 * thresh) break;
    if (restart == max_restarts) { status = OR_NOT_CONVERGED; break; }
    rnorm = tnorm; /* restart from the current x */
  }

  /* final relative residuals */
  or_spmv(n, rowptr, col, val, x, q);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  out_info[0] = it;
  out_info[1] = status;
  out_res[0] = rnorm / bnorm;
  out_res[1] = nrm2(n, r) / bnorm;
  free(r); free(z); free(p); free(q);
  return status;
}

/* precond: 0 none, 1 Jacobi, 2 G G^T (g* arrays used). */
int or_pcg(int32_t n, const int32_t* rowptr, const int32_t* col,
           const double* val, const double* b, double* x, double rtol,
           double atol, int32_t max_iter, int32_t max_restarts,
           int32_t use_x0, int32_t precond, const int32_t* growptr,
           const int32_t* gcol, const double* gval, int32_t* out_info,
           double* out_res) {
  precond_t M;
  memset(&M, 0, sizeof(M));
  M.kind = precond;
  M.n = n;
  double* d = NULL;
  if (precond == 1) {
    d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    or_diag(n, rowptr, col, val, d);
    for (int32_t i = 0; i < n; ++i) {
      if (!(d[i] > 0.0)) {
        free(d);
        out_info[0] = 0;
        out_info[1] = OR_NOT_SPD;
        out_res[0] = out_res[1] = NAN;
        return OR_NOT_SPD;
      }
      d[i] = 1.0 / d[i];
    }
    M.dinv = d;
  } else if (precond == 2) {
    M.growptr = growptr;
    M.gcol = gcol;
    M.gval = gval;
    M.tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  }
  int st = pcg_core(n, rowptr, col, val, b, x, rtol, atol, max_iter,
                    max_restarts, use_x0, &M, out_info, out_res);
  free(d);
  free(M.tmp);
  return st;
}

/* ---------------------------------------------------------------------- */
/* Pipelined PCG (Ghysels & Vanroose, "Hiding global synchronization      */
/* latency in the preconditioned Conjugate Gradient algorithm", Parallel  */
/* Computing 2014): one of the CG variants that merge the inner-product   */
/* reductions, named in App. C as the roadmap item for reduction latency. */
/* In exact arithmetic its iterates are those of pcg_core; it carries     */
/* w = A u, s = A p and z = A M^{-1} s as recurrences so that the three   */
/* inner products of an iteration form one reduction and the iteration's  */
/* SpMV (of m = M^{-1} w) does not depend on that reduction's result.     */
/* Per iteration i:                                                        */
/*   gamma = (r,u), delta = (w,u), ||r||        -- one reduction           */
/*   m = M^{-1} w ; nv = A m                                               */
/*   beta = gamma/gamma_prev, alpha = gamma/(delta - beta*gamma/alpha_prev)*/
/*   (beta = 0, alpha = gamma/delta on the first iteration of a start)     */
/*   z = nv + beta z ; s = w + beta s ; p = u + beta p                     */
/*   x += alpha p ; r -= alpha s ; w -= alpha z ; u = M^{-1} r             */
/* Reading for a pointwise (Jacobi or identity) M: u is recomputed as      */
/* M^{-1} r rather than carried by the recurrence u -= alpha q, q = m +    */
/* beta q of the general method; both equal M^{-1} r in exact arithmetic,  */
/* and q is then not needed.  Exits and restarts as in pcg_core: the       */
/* recursive-residual test, then the true residual with at most            */
/* max_restarts restarts from the current x; NOT_SPD when gamma <= 0, or   */
/* when the denominator (= p^T A p) is <= 0 on the first step of a start   */
/* (there it is u^T A u from a fresh product); BREAKDOWN on a non-finite   */
/* scalar.  Reading: a denominator <= 0 on a later step comes from the     */
/* recurrences for w, s, z, whose rounding errors grow near the attainable */
/* accuracy (the known weakness of the pipelined method, which restarts or */
/* "residual replacement" cure), not from an indefinite A, so it leads to  */
/* the true-residual check: accepted within twice the target, else a       */
/* restart from x while restarts remain, else NOT_CONVERGED.               */
/* precond: 0 none, 1 Jacobi.                                              */
/* ---------------------------------------------------------------------- */
int or_pcg_pipelined(int32_t n, const int32_t* rowptr, const int32_t* col,
                     const double* val, const double* b, double* x,
                     double rtol, double atol, int32_t max_iter,
                     int32_t max_restarts, int32_t use_x0, int32_t precond,
                     int32_t* out_info, double* out_res) {
  size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* dinv = (double*)malloc(bytes);
  double* r = (double*)malloc(bytes);
  double* u = (double*)malloc(bytes);
  double* w = (double*)malloc(bytes);
  double* m = (double*)malloc(bytes);
  double* nv = (double*)malloc(bytes);
  double* z = (double*)malloc(bytes);
  double* s = (double*)malloc(bytes);
  double* p = (double*)malloc(bytes);
  int status = OR_NOT_CONVERGED;
  int32_t it = 0;
  double bnorm = nrm2(n, b);
  double thresh = rtol * bnorm > atol ? rtol * bnorm : atol;
  double rnorm = 0.0;

  /* M^{-1} as a pointwise scale */
  if (precond == 1) {
    or_diag(n, rowptr, col, val, dinv);
    for (int32_t i = 0; i < n; ++i) {
      if (!(dinv[i] > 0.0)) {
        out_info[0] = 0;
        out_info[1] = OR_NOT_SPD;
        out_res[0] = out_res[1] = NAN;
        status = OR_NOT_SPD;
        goto out;
      }
      dinv[i] = 1.0 / dinv[i];
    }
  } else {
    for (int32_t i = 0; i < n; ++i) dinv[i] = 1.0;
  }

  if (!use_x0)
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;

  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    out_info[0] = 0;
    out_info[1] = OR_OK;
    out_res[0] = 0.0;
    out_res[1] = 0.0;
    status = OR_OK;
    goto out;
  }

  for (int32_t restart = 0; restart <= max_restarts; ++restart) {
    /* r = b - A x ; u = M^{-1} r ; w = A u ; z = s = p = 0 */
    or_spmv(n, rowptr, col, val, x, nv);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - nv[i];
    for (int32_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
    or_spmv(n, rowptr, col, val, u, w);
    for (int32_t i = 0; i < n; ++i) z[i] = s[i] = p[i] = 0.0;
    rnorm = nrm2(n, r);
    status = OR_NOT_CONVERGED;
    if (!isfinite(rnorm)) { status = OR_BREAKDOWN; break; }
    if (rnorm <= thresh) { status = OR_OK; }

    double gamma_prev = 0.0, alpha_prev = 0.0;
    int first = 1;
    while (status == OR_NOT_CONVERGED) {
      double gamma = dot(n, r, u);
      double delta = dot(n, w, u);
      rnorm = nrm2(n, r);
      if (!isfinite(gamma) || !isfinite(delta) || !isfinite(rnorm)) { status = OR_BREAKDOWN; break; }
      if (rnorm <= thresh) { status = OR_OK; break; }
      if (it >= max_iter) break;
      if (!(gamma > 0.0)) { status = OR_NOT_SPD; break; }
      double beta, denom;
      if (first) {
        beta = 0.0;
        denom = delta;
      } else {
        beta = gamma / gamma_prev;
        denom = delta - beta * gamma / alpha_prev;
      }
      if (!isfinite(denom)) { status = OR_BREAKDOWN; break; }
      if (!(denom > 0.0)) {
        if (first) { status = OR_NOT_SPD; break; }
        status = OR_OK;  /* recurrences exhausted: to the true-residual check */
        break;
      }
      double alpha = gamma / denom;
      for (int32_t i = 0; i < n; ++i) m[i] = dinv[i] * w[i];
      or_spmv(n, rowptr, col, val, m, nv);
      for (int32_t i = 0; i < n; ++i) z[i] = nv[i] + beta * z[i];
      for (int32_t i = 0; i < n; ++i) s[i] = w[i] + beta * s[i];
      for (int32_t i = 0; i < n; ++i) p[i] = u[i] + beta * p[i];
      for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
      for (int32_t i = 0; i < n; ++i) r[i] -= alpha * s[i];
      for (int32_t i = 0; i < n; ++i) w[i] -= alpha * z[i];
      for (int32_t i = 0; i < n; ++i) u[i] = dinv[i] * r[i];
      gamma_prev = gamma;
      alpha_prev = alpha;
      first = 0;
      ++it;
    }
    if (status != OR_OK) break;
    /* true residual check */
    or_spmv(n, rowptr, col, val, x, nv);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - nv[i];
    double tnorm = nrm2(n, r);
    if (tnorm <= 2.0 * thresh) { status = OR_OK; break; }
    if (!isfinite(tnorm)) { status = OR_BREAKDOWN; break; }
    if (restart == max_restarts || it >= max_iter) { status = OR_NOT_CONVERGED; break; }
  }

  /* final relative residuals */
  or_spmv(n, rowptr, col, val, x, nv);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - nv[i];
  out_info[0] = it;
  out_info[1] = status;
  out_res[0] = rnorm / bnorm;
  out_res[1] = nrm2(n, r) / bnorm;

out:
  free(dinv); free(r); free(u); free(w); free(m); free(nv); free(z); free(s); free(p);
  return status;
}

/* Fixed-k unpreconditioned CG (the setting of Sec. 4.2 / Tab. 7): exactly  */
/* k iterations of Algorithm 1 with no convergence test.                    */
void or_cg_fixed(int32_t n, const int32_t* rowptr, const int32_t* col,
                 const double* val, const double* b, double* x, int32_t k) {
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; }
  double rho = dot(n, r, r);
  for (int32_t it = 0; it < k && rho > 0.0; ++it) {
    or_spmv(n, rowptr, col, val, p, q);
    double alpha = rho / dot(n, p, q);
    for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    double rho_new = dot(n, r, r);
    for (int32_t i = 0; i < n; ++i) p[i] = r[i] + (rho_new / rho) * p[i];
    rho = rho_new;
  }
  free(r); free(p); free(q);
}

/* ---------------------------------------------------------------------- */
/* Right-preconditioned BiCGStab for nonsymmetric A (van der Vorst 1992,   */
/* cited for the nonsymmetric solver in Sec. 1 and Sec. 3.1).  Readings:    */
/* shadow residual rhat = r0; Jacobi preconditioner applied on the right    */
/* (phat = M^{-1} p, shat = M^{-1} s); early exit when ||s|| meets the      */
/* target; |rho| < 1e-300, r^T v == 0 or omega == 0 stops with BREAKDOWN;   */
/* A_ii == 0 with Jacobi is INVALID.  Same stopping rule and true-residual  */
/* restart as the CG routine.                                               */
/* ---------------------------------------------------------------------- */
int or_bicgstab(int32_t n, const int32_t* rowptr, const int32_t* col,
                const double* val, const double* b, double* x, double rtol,
                double atol, int32_t max_iter, int32_t max_restarts,
                int32_t use_x0, int32_t precond, int32_t* out_info,
                double* out_res) {
  size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *r = malloc(sz), *rh = malloc(sz), *p = malloc(sz), *v = malloc(sz);
  double *s = malloc(sz), *t = malloc(sz), *ph = malloc(sz), *sh = malloc(sz);
  double *dinv = malloc(sz);
  int status = OR_NOT_CONVERGED;
  int32_t it = 0;
  double bnorm = nrm2(n, b);
  double thresh = rtol * bnorm > atol ? rtol * bnorm : atol;
  double rnorm = 0.0;
  precond_t M;
  memset(&M, 0, sizeof(M));
  M.kind = precond == 1 ? 1 : 0;
  M.n = n;
  if (precond == 1) {
    or_diag(n, rowptr, col, val, dinv);
    for (int32_t i = 0; i < n; ++i) {
      if (dinv[i] == 0.0 || !isfinite(dinv[i])) { status = OR_ERR_INVALID; goto done_early; }
      dinv[i] = 1.0 / dinv[i];
    }
    M.dinv = dinv;
  }
  if (!use_x0)
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
  if (bnorm == 0.0) {
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
    status = OR_OK;
    goto done_early;
  }

  for (int32_t restart = 0; restart <= max_restarts; ++restart) {
    or_spmv(n, rowptr, col, val, x, t);
    for (int32_t i = 0; i < n; ++i) { r[i] = b[i] - t[i]; rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    rnorm = nrm2(n, r);
    status = OR_NOT_CONVERGED;
    if (!isfinite(rnorm)) { status = OR_BREAKDOWN; break; }
    while (!(rnorm <= thresh) && it < max_iter) {
      double rho = dot(n, rh, r);
      if (!isfinite(rho)) { status = OR_BREAKDOWN; break; }
      if (fabs(rho) < 1e-300) { status = OR_BREAKDOWN; break; }
      double beta = (rho / rho_prev) * (alpha / omega);
      for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      apply_precond(&M, p, ph);
      or_spmv(n, rowptr, col, val, ph, v);        /* v = A phat */
      double rv = dot(n, rh, v);
      if (!isfinite(rv) || rv == 0.0) { status = OR_BREAKDOWN; break; }
      alpha = rho / rv;
      for (int32_t i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
      ++it;
      double snorm = nrm2(n, s);
      if (snorm <= thresh) {                       /* half-step exit */
        for (int32_t i = 0; i < n; ++i) x[i] += alpha * ph[i];
        rnorm = snorm;
        status = OR_OK;
        break;
      }
      apply_precond(&M, s, sh);
      or_spmv(n, rowptr, col, val, sh, t);         /* t = A shat */
      double tt = dot(n, t, t);
      double ts = dot(n, t, s);
      if (!isfinite(tt) || !isfinite(ts) || tt == 0.0) { status = OR_BREAKDOWN; break; }
      omega = ts / tt;
      for (int32_t i = 0; i < n; ++i) x[i] += alpha * ph[i] + omega * sh[i];
      for (int32_t i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
      rnorm = nrm2(n, r);
      if (!isfinite(rnorm)) { status = OR_BREAKDOWN; break; }
      if (rnorm <= thresh) { status = OR_OK; break; }
      if (omega == 0.0) { status = OR_BREAKDOWN; break; }
      rho_prev = rho;
    }
    /* a start that already meets the stopping test is converged (as in
       pcg_core): the loop above then runs no iteration */
    if (status == OR_NOT_CONVERGED && rnorm <= thresh) status = OR_OK;
    if (status != OR_OK) break;
    or_spmv(n, rowptr, col, val, x, t);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    double tnorm = nrm2(n, r);
    if (tnorm <= 2.0 * thresh) break;
    if (restart == max_restarts) { status = OR_NOT_CONVERGED; break; }
    rnorm = tnorm;
  }

  or_spmv(n, rowptr, col, val, x, t);
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  out_info[0] = it;
  out_info[1] = status;
  out_res[0] = rnorm / bnorm;
  out_res[1] = nrm2(n, r) / bnorm;
  free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh); free(dinv);
  return status;

done_early:
  out_info[0] = 0;
  out_info[1] = status;
  out_res[0] = status == OR_OK ? 0.0 : NAN;
  out_res[1] = status == OR_OK ? 0.0 : NAN;
  free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh); free(dinv);
  return status;
}

/* ---------------------------------------------------------------------- */
/* CSR of A^T by a stable counting sort on the column index.  Entry        */
/* (i, j) at CSR slot k becomes row j of A^T; within a row of A^T the       */
/* entries keep increasing i.  permT[m] = k, so valT[m] = val[permT[m]].   */
/* (A^T lambda = dL/dx of Eq. 3 needs A^T for nonsymmetric A.)              */
/* ---------------------------------------------------------------------- */
void or_transpose(int32_t n, const int32_t* rowptr, const int32_t* col,
                  int32_t* rowptrT, int32_t* colT, int32_t* permT) {
  int32_t nnz = rowptr[n];
  for (int32_t j = 0; j <= n; ++j) rowptrT[j] = 0;
  for (int32_t k = 0; k < nnz; ++k) rowptrT[col[k] + 1] += 1;
  for (int32_t j = 0; j < n; ++j) rowptrT[j + 1] += rowptrT[j];
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t j = 0; j < n; ++j) next[j] = rowptrT[j];
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int32_t m = next[col[k]]++;
      colT[m] = i;
      permT[m] = k;
    }
  free(next);
}

/* ---------------------------------------------------------------------- */
/* COO -> CSR ingest: entries sorted by (row, col); duplicates summed in    */
/* increasing COO index; perm[e] = CSR slot that COO entry e landed in.     */
/* (SparseTensor(val, row, col, shape) of App. B stores COO.)               */
/* Two stable counting sorts: by col, then by row.  Returns nnz of the CSR. */
/* ---------------------------------------------------------------------- */
int32_t or_coo_to_csr(int32_t n, int64_t nnz_in, const int64_t* row,
                      const int64_t* colin, const double* val_in,
                      int32_t* rowptr, int32_t* col, double* val,
                      int32_t* perm) {
  size_t m = (size_t)(nnz_in > 0 ? nnz_in : 1);
  int64_t* ord1 = (int64_t*)malloc(sizeof(int64_t) * m);
  int64_t* ord2 = (int64_t*)malloc(sizeof(int64_t) * m);
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  /* pass 1: stable by column */
  for (int64_t e = 0; e < nnz_in; ++e) cnt[colin[e] + 1] += 1;
  for (int32_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
  for (int64_t e = 0; e < nnz_in; ++e) ord1[cnt[colin[e]]++] = e;
  /* pass 2: stable by row */
  memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t e = 0; e < nnz_in; ++e) cnt[row[e] + 1] += 1;
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  for (int64_t t = 0; t < nnz_in; ++t) {
    int64_t e = ord1[t];
    ord2[cnt[row[e]]++] = e;
  }
  /* merge duplicates, build rowptr */
  int32_t out = 0;
  for (int32_t i = 0; i <= n; ++i) rowptr[i] = 0;
  for (int64_t t = 0; t < nnz_in; ++t) {
    int64_t e = ord2[t];
    if (t > 0) {
      int64_t ep = ord2[t - 1];
      if (row[ep] == row[e] && colin[ep] == colin[e]) {
        val[out - 1] += val_in[e];
        perm[e] = out - 1;
        continue;
      }
    }
    col[out] = (int32_t)colin[e];
    val[out] = val_in[e];
    perm[e] = out;
    rowptr[row[e] + 1] += 1;
    ++out;
  }
  for (int32_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  free(ord1); free(ord2); free(cnt);
  return out;
}

/* ---------------------------------------------------------------------- */
/* Matrix gradient of the linear adjoint, Eq. 3:                            */
/*   dL/dA_ij = -lambda_i x_j, on the stored pattern only.                  */
/* ---------------------------------------------------------------------- */
void or_grad_values(int32_t n, const int32_t* rowptr, const int32_t* col,
                    const double* lambda, const double* x, double* grad_val) {
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      grad_val[k] = -lambda[i] * x[col[k]];
}

/* ---------------------------------------------------------------------- */
/* Linear adjoint backward (Eq. 2 with J = A, specialised in Eq. 3):       */
/*   solve A^T lambda = g ; grad_b = lambda ; grad_val = -lambda_i x_j.     */
/* method 0: A is symmetric, so A^T = A and the Jacobi-PCG routine is used  */
/* on A itself; method 1: BiCGStab on the explicit CSR of A^T.              */
/* The adjoint solve uses the forward tolerance relative to ||g||.          */
/* ---------------------------------------------------------------------- */
int or_adjoint_backward(int32_t n, const int32_t* rowptr, const int32_t* col,
                        const double* val, const double* x, const double* g,
                        double* grad_b, double* grad_val, int32_t method,
                        double rtol, double atol, int32_t max_iter,
                        int32_t* out_info, double* out_res) {
  int st;
  if (method == 0) {
    st = or_pcg(n, rowptr, col, val, g, grad_b, rtol, atol, max_iter, 2, 0, 1,
                NULL, NULL, NULL, out_info, out_res);
  } else {
    int32_t nnz = rowptr[n];
    size_t ni = (size_t)(nnz > 0 ? nnz : 1);
    int32_t* rpT = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t* cT = (int32_t*)malloc(sizeof(int32_t) * ni);
    int32_t* pT = (int32_t*)malloc(sizeof(int32_t) * ni);
    double* vT = (double*)malloc(sizeof(double) * ni);
    or_transpose(n, rowptr, col, rpT, cT, pT);
    for (int32_t m = 0; m < nnz; ++m) vT[m] = val[pT[m]];
    st = or_bicgstab(n, rpT, cT, vT, g, grad_b, rtol, atol, max_iter, 2, 0, 1,
                     out_info, out_res);
    free(rpT); free(cT); free(pT); free(vT);
  }
  or_grad_values(n, rowptr, col, grad_b, x, grad_val);
  return st;
}
