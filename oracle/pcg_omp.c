/*
 * pcg_omp.c -- the oracle's value update and FP64 Jacobi-PCG restated in plain
 * C with OpenMP loops, for timing the oracle on every host core.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may load or call this
 * library: only the tests, the smoke check and the CPU-baseline / reference
 * legs of the benchmark use it. It shares no code with the CUDA path. Its
 * inputs (the merged CSR pattern, the permutation src_of, the continuous
 * coefficient buffer, the right-hand side) come from the Python oracle and the
 * seeded input generator, and its results are checked against the Python
 * oracle (repart_oracle.pcg) in the tests.
 *
 * Every step is one plain loop, in the order of the textbook algorithm
 * (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.1, with a Jacobi
 * preconditioner): no fusion, no blocking. The only parallelism is OpenMP
 * over rows with static schedules; sums over rows are OpenMP reductions, so
 * the rounding of a dot product depends on the thread count (results agree
 * with the serial oracle to rounding, not bit for bit).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 7, ORC_BREAKDOWN = 8, ORC_ENOMEM = 5 };

/* Threads the library will use when asked for `want` (0: all it may use). */
int orc_threads(int want) {
#ifdef _OPENMP
  return want > 0 ? want : omp_get_max_threads();
#else
  (void)want;
  return 1;
#endif
}

#ifdef _OPENMP
#define ORC_SET_THREADS(t) omp_set_num_threads(orc_threads(t))
#else
#define ORC_SET_THREADS(t) (void)(t)
#endif

/* Value update (Sec. 3, update procedure): the continuous buffer reordered by
 * the permutation, vals[p] = buf[src_of[p]]. */
void orc_update_values(int64_t nnz, const int32_t* src_of, const double* buf, double* vals, int threads) {
  ORC_SET_THREADS(threads);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < nnz; ++p) vals[p] = buf[src_of[p]];
}

/* Jacobi preconditioner: dinv[i] = 1 / a_ii, the diagonal read at diag_pos. */
void orc_jacobi_inverse(int64_t n, const int32_t* diag_pos, const double* vals, double* dinv, int threads) {
  ORC_SET_THREADS(threads);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / vals[diag_pos[i]];
}

/* y = A x for a CSR matrix (row_ptr from 0, columns of each row in any order). */
static void spmv(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* x,
                 double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) s += vals[p] * x[col[p]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double* u, const double* v) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
  return s;
}

/* Outcome of orc_pcg, as the Python oracle's SolveResult. */
typedef struct orc_result {
  int32_t status;
  int32_t iterations;
  double rel_residual;      /* recursive residual at exit */
  double true_rel_residual; /* ||b - A x|| / ||b|| recomputed at exit */
} orc_result;

/* Jacobi-preconditioned CG from x = 0 (the merged pressure system is solved by
 * CG, Sec. 4; Jacobi preconditioner): r = b, z = D^-1 r, p = z; per iteration
 * q = A p, alpha = (r.z)/(p.q), x += alpha p, r -= alpha q; when
 * ||r|| <= tol ||b|| the true residual b - A x confirms it, else it replaces r
 * and the iteration restarts from p = z; otherwise z = D^-1 r,
 * beta = (r.z)_new/(r.z)_old, p = z + beta p. p.q <= 0 ends with
 * ORC_BREAKDOWN, max_iter iterations with ORC_NOT_CONVERGED. x receives the
 * solution (n doubles, caller-owned). */
int orc_pcg(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* vals, const double* dinv,
            const double* b, double tol, int32_t max_iter, double* x, orc_result* out, int threads) {
  ORC_SET_THREADS(threads);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!r || !z || !p || !q) {
    free(r), free(z), free(p), free(q);
    return ORC_ENOMEM;
  }
  const double bb = dot(n, b, b);
  const double thresh = tol * tol * bb;
  int32_t it = 0, status = ORC_NOT_CONVERGED, restart = 1;
  double rz = 0.0, rr;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
  }
  rr = bb;
  if (bb == 0.0) status = ORC_OK;
  while (status != ORC_OK) {
    if (restart) {
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
      }
      rz = dot(n, r, z);
      restart = 0;
      if (rr <= thresh) {
        spmv(n, row_ptr, col, vals, x, q);
        double trr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : trr)
        for (int64_t i = 0; i < n; ++i) trr += (b[i] - q[i]) * (b[i] - q[i]);
        if (trr <= thresh) {
          status = ORC_OK;
          break;
        }
      }
    }
    if (it >= max_iter) break;
    spmv(n, row_ptr, col, vals, p, q);
    const double pq = dot(n, p, q);
    if (!(pq > 0.0)) {
      status = ORC_BREAKDOWN;
      break;
    }
    const double alpha = rz / pq;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
    ++it;
    rr = dot(n, r, r);
    if (rr <= thresh) {
      /* confirm with the true residual; on failure it replaces r (restart) */
      spmv(n, row_ptr, col, vals, x, q);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
      const double trr = dot(n, q, q);
      if (trr <= thresh) {
        status = ORC_OK;
        break;
      }
      memcpy(r, q, sizeof(double) * (size_t)n);
      rr = trr;
      restart = 1;
      continue;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
    const double rz_new = dot(n, r, z);
    const double beta = rz_new / rz;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
  /* the true residual at exit */
  spmv(n, row_ptr, col, vals, x, q);
  double trr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : trr)
  for (int64_t i = 0; i < n; ++i) trr += (b[i] - q[i]) * (b[i] - q[i]);
  out->status = status;
  out->iterations = it;
  out->rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  out->true_rel_residual = bb > 0.0 ? sqrt(trr / bb) : 0.0;
  free(r), free(z), free(p), free(q);
  return 0;
}
