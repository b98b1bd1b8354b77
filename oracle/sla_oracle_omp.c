/*
 * sla_oracle_omp.c -- the oracle's Jacobi-preconditioned CG with its loops
 * spread over the host's cores by OpenMP (arXiv 2601.13994, Algorithm 1 with
 * P = 1 and the Jacobi preconditioner of Sec. 4.1).
 *
 * TEST INFRASTRUCTURE ONLY: the all-core CPU baseline that bench.py reports
 * beside the single-threaded oracle (sla_oracle.c).  Nothing in the product
 * path may call, link or load it.  It shares no code with the CUDA library
 * nor with sla_oracle.c: the steps, readings and exits below are those of
 * sla_oracle.c's pcg_core, written again with each n-length loop marked
 * "omp parallel for" and each inner product an OpenMP sum reduction.  No
 * loop is fused, blocked or reordered beyond that, so the only difference
 * from the single-threaded oracle is the summation order of the inner
 * products (partial sums per thread), i.e. rounding.
 *
 * Readings (as in sla_oracle.c): stop when ||r||_2 <= max(rtol ||b||_2,
 * atol) on the recursive residual; x0 = 0 unless use_x0; b = 0 gives x = 0
 * after 0 iterations; A_ii <= 0 or p^T A p <= 0 -> NOT_SPD; a non-finite
 * scalar -> BREAKDOWN; the true residual is recomputed at exit and a value
 * above twice the target restarts the recurrence from x (at most
 * max_restarts times).  Compile with -O2 -fopenmp -ffp-contract=off.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

enum { OMP_OK = 0, OMP_NOT_CONVERGED = 1, OMP_BREAKDOWN = 2, OMP_NOT_SPD = 3 };

int or_omp_threads(void) { return omp_get_max_threads(); }

static double dot_omp(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* y = A x, one row per iteration of the parallel loop */
void or_omp_spmv(int32_t n, const int32_t* rowptr, const int32_t* col,
                 const double* val, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* precond: 0 none, 1 Jacobi.  nthreads > 0 sets the thread count of the
 * parallel loops (0: OpenMP's default).  out_info[0] iterations, [1] status;
 * out_res[0] recursive, [1] true relative residual. */
int or_omp_pcg(int32_t n, const int32_t* rowptr, const int32_t* col,
               const double* val, const double* b, double* x, double rtol,
               double atol, int32_t max_iter, int32_t max_restarts,
               int32_t use_x0, int32_t precond, int32_t nthreads,
               int32_t* out_info, double* out_res) {
  if (nthreads > 0) omp_set_num_threads(nthreads);
  const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* dinv = (double*)malloc(bytes);
  double* r = (double*)malloc(bytes);
  double* z = (double*)malloc(bytes);
  double* p = (double*)malloc(bytes);
  double* q = (double*)malloc(bytes);
  int status = OMP_NOT_CONVERGED;
  int32_t it = 0;
  double rnorm = 0.0;
  int bad_diag = 0;

  /* Jacobi diagonal d_i = sum of the stored diagonal entries of row i */
#pragma omp parallel for schedule(static) reduction(| : bad_diag)
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) d += val[k];
    if (precond == 1) {
      if (!(d > 0.0)) bad_diag = 1;
      dinv[i] = 1.0 / d;
    } else {
      dinv[i] = 1.0;
    }
  }
  if (bad_diag) {
    out_info[0] = 0;
    out_info[1] = OMP_NOT_SPD;
    out_res[0] = out_res[1] = NAN;
    free(dinv); free(r); free(z); free(p); free(q);
    return OMP_NOT_SPD;
  }

  const double bnorm = sqrt(dot_omp(n, b, b));
  const double thresh = rtol * bnorm > atol ? rtol * bnorm : atol;
  if (!use_x0 || bnorm == 0.0) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) x[i] = 0.0;
  }
  if (bnorm == 0.0) {
    out_info[0] = 0;
    out_info[1] = OMP_OK;
    out_res[0] = out_res[1] = 0.0;
    free(dinv); free(r); free(z); free(p); free(q);
    return OMP_OK;
  }

  for (int32_t restart = 0; restart <= max_restarts; ++restart) {
    /* r = b - A x ; z = M^{-1} r ; p = z ; rho = r^T z */
    or_omp_spmv(n, rowptr, col, val, x, q);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot_omp(n, r, z);
    rnorm = sqrt(dot_omp(n, r, r));
    status = OMP_NOT_CONVERGED;
    if (!isfinite(rho) || !isfinite(rnorm)) { status = OMP_BREAKDOWN; break; }

    while (!(rnorm <= thresh) && it < max_iter) {
      or_omp_spmv(n, rowptr, col, val, p, q);            /* q = A p */
      const double pq = dot_omp(n, p, q);                 /* p^T A p */
      if (!isfinite(pq)) { status = OMP_BREAKDOWN; break; }
      if (!(pq > 0.0)) { status = OMP_NOT_SPD; break; }
      const double alpha = rho / pq;
#pragma omp parallel for schedule(static)
      for (int32_t i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for schedule(static)
      for (int32_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
#pragma omp parallel for schedule(static)
      for (int32_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
      const double rho_new = dot_omp(n, r, z);
      rnorm = sqrt(dot_omp(n, r, r));
      ++it;
      if (!isfinite(rho_new) || !isfinite(rnorm)) { status = OMP_BREAKDOWN; break; }
      if (rnorm <= thresh) { status = OMP_OK; break; }
      if (!(rho_new > 0.0)) { status = OMP_NOT_SPD; break; }
      const double beta = rho_new / rho;
#pragma omp parallel for schedule(static)
      for (int32_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rho = rho_new;
    }
    if (rnorm <= thresh) status = OMP_OK;
    if (status != OMP_OK) break;
    /* true residual check */
    or_omp_spmv(n, rowptr, col, val, x, q);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    const double tnorm = sqrt(dot_omp(n, r, r));
    if (tnorm <= 2.0 * thresh) break;
    if (restart == max_restarts) { status = OMP_NOT_CONVERGED; break; }
    rnorm = tnorm;
  }

  or_omp_spmv(n, rowptr, col, val, x, q);
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  out_info[0] = it;
  out_info[1] = status;
  out_res[0] = rnorm / bnorm;
  out_res[1] = sqrt(dot_omp(n, r, r)) / bnorm;
  free(dinv); free(r); free(z); free(p); free(q);
  return status;
}
