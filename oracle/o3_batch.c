/* O3 over a batch of columns: the heavy loops of the naive FP64 B-Lanczos.
 *
 * TEST INFRASTRUCTURE ONLY (part of the CPU oracle; the library never links
 * it). The Python driver is oracle/krylov.py, lanczos_batch(); this file holds
 * the loops that are too slow in NumPy at 10^5 - 10^6 atoms:
 *
 *   o3_spmm       Y = S X for a sparse CSR S and C column vectors;
 *   o3_cg         plain conjugate gradients for B V = U, per column;
 *   o3_seed       the Lanczos start of Sec. III-B's shared subspace:
 *                 u = e_j, v = B^-1 u, beta0 = sqrt(u.v), q1 = v/beta0,
 *                 Bq1 = u/beta0;
 *   o3_step       one Lanczos step in the B inner product (the operator
 *                 B^-1 A of the generalized shifted equations
 *                 (z B - A) x = e_j, Eq. EQ-SHIFT-EQ-J):
 *                 [v = B^-1 u, beta = sqrt(u.v), Bq_prev = Bq, Bq = u/beta,
 *                 q = v/beta], w = A q, alpha = q.w,
 *                 u = w - alpha Bq - beta_prev Bq_prev;
 *   o3_tridiag    for each shift z, (z I - T_n) y = beta0 e_1 by Gaussian
 *                 elimination with partial pivoting on the tridiagonal
 *                 matrix (the textbook banded LU with row interchanges), the
 *                 full y or only its last entry.
 *
 * Vectors are row-major [M][ld]: column c of the batch is element c of every
 * row, and only the first C (active) columns are touched. Every column's
 * arithmetic is exactly that of a one-column run; the columns share nothing
 * but the traversal of the matrix. Sums over rows are split into NBLK fixed
 * row blocks whose partial sums are added in block order, so results do not
 * depend on the number of threads. Build with -ffp-contract=off, so that no
 * multiply and add are fused on any machine.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NBLK 256

typedef double _Complex cplx;

/* Threads of the parallel loops (results do not depend on it). */
void o3_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int o3_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Y[i][c] = sum_e S.val[e] * X[S.idx[e]][c], entries of row i in CSR order. */
void o3_spmm(int64_t M, const int64_t* ptr, const int32_t* idx, const double* val, int C, int ld,
             const double* X, double* Y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i) {
    double* y = Y + i * ld;
    for (int c = 0; c < C; ++c) y[c] = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
      const double a = val[e];
      const double* x = X + (int64_t)idx[e] * ld;
      for (int c = 0; c < C; ++c) y[c] += a * x[c];
    }
  }
}

/* out[c] = sum_i X[i][c] * Y[i][c] for c < C; fixed row blocks, in order. */
static void dots(int64_t M, int C, int ld, const double* X, const double* Y, double* out, double* part) {
#pragma omp parallel for schedule(static)
  for (int b = 0; b < NBLK; ++b) {
    const int64_t i0 = M * b / NBLK, i1 = M * (b + 1) / NBLK;
    double* pb = part + (int64_t)b * C;
    for (int c = 0; c < C; ++c) pb[c] = 0.0;
    for (int64_t i = i0; i < i1; ++i)
      for (int c = 0; c < C; ++c) pb[c] += X[i * ld + c] * Y[i * ld + c];
  }
  for (int c = 0; c < C; ++c) out[c] = 0.0;
  for (int b = 0; b < NBLK; ++b)
    for (int c = 0; c < C; ++c) out[c] += part[(int64_t)b * C + c];
}

/* Plain CG for B V = U, each column on its own: V = 0, R = U, P = R; while
 * r.r > tol^2 u.u: a = r.r / p.Bp, V += a P, R -= a BP, b = r.r_new / r.r,
 * P = R + b P. R, P, BP: [M][ld] work arrays. Returns the largest iteration
 * count over the columns, or -1 if a column did not reach tol in max_iter. */
int o3_cg(int64_t M, const int64_t* ptr, const int32_t* idx, const double* val, int C, int ld,
          const double* U, double* V, double tol, int max_iter, double* R, double* P, double* BP) {
  double* part = (double*)malloc(sizeof(double) * NBLK * (C > 0 ? C : 1));
  double* rr = (double*)malloc(sizeof(double) * 5 * (C > 0 ? C : 1));
  double *target = rr + C, *pbp = rr + 2 * C, *rrn = rr + 3 * C, *coef = rr + 4 * C;
  int* active = (int*)malloc(sizeof(int) * (C > 0 ? C : 1));
  int worst = 0, it = 0, n_act = 0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int c = 0; c < C; ++c) {
      V[i * ld + c] = 0.0;
      R[i * ld + c] = U[i * ld + c];
      P[i * ld + c] = U[i * ld + c];
    }
  dots(M, C, ld, R, R, rr, part);
  dots(M, C, ld, U, U, target, part);
  for (int c = 0; c < C; ++c) {
    target[c] *= tol * tol;
    active[c] = rr[c] > target[c];
    n_act += active[c];
  }
  while (n_act > 0 && it < max_iter) {
    ++it;
    o3_spmm(M, ptr, idx, val, C, ld, P, BP);
    dots(M, C, ld, P, BP, pbp, part);
    for (int c = 0; c < C; ++c) coef[c] = active[c] ? rr[c] / pbp[c] : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i)
      for (int c = 0; c < C; ++c)
        if (active[c]) {
          V[i * ld + c] += coef[c] * P[i * ld + c];
          R[i * ld + c] -= coef[c] * BP[i * ld + c];
        }
    dots(M, C, ld, R, R, rrn, part);
    for (int c = 0; c < C; ++c) coef[c] = active[c] ? rrn[c] / rr[c] : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i)
      for (int c = 0; c < C; ++c)
        if (active[c]) P[i * ld + c] = R[i * ld + c] + coef[c] * P[i * ld + c];
    n_act = 0;
    for (int c = 0; c < C; ++c)
      if (active[c]) {
        rr[c] = rrn[c];
        active[c] = rrn[c] > target[c];
        if (!active[c] && it > worst) worst = it;
        n_act += active[c];
      }
  }
  free(part);
  free(rr);
  free(active);
  return n_act > 0 ? -1 : worst;
}

/* Seed of each column: u = e_{rows[c]}, v = B^-1 u (CG to bsolve_tol),
 * beta0 = sqrt(u.v), q = v / beta0, Bq = u / beta0, Bq_prev = 0. */
int o3_seed(int64_t M, const int64_t* bptr, const int32_t* bidx, const double* bval, int C, int ld,
            const int32_t* rows, double bsolve_tol, int max_cg, double* q, double* Bq, double* Bqp,
            double* u, double* v, double* R, double* P, double* BP, double* beta0) {
  double* part = (double*)malloc(sizeof(double) * NBLK * (C > 0 ? C : 1));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int c = 0; c < C; ++c) u[i * ld + c] = (i == rows[c]) ? 1.0 : 0.0;
  const int cg = o3_cg(M, bptr, bidx, bval, C, ld, u, v, bsolve_tol, max_cg, R, P, BP);
  dots(M, C, ld, u, v, beta0, part);
  for (int c = 0; c < C; ++c) beta0[c] = sqrt(beta0[c]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int c = 0; c < C; ++c) {
      q[i * ld + c] = v[i * ld + c] / beta0[c];
      Bq[i * ld + c] = u[i * ld + c] / beta0[c];
      Bqp[i * ld + c] = 0.0;
    }
  free(part);
  return cg;
}

/* One Lanczos step for the C active columns. When first == 0 it starts by
 * finishing the previous step: v = B^-1 u, beta = sqrt(u.v) (returned in
 * beta[c]), Bq_prev = Bq, Bq = u / beta, q = v / beta, beta_prev = beta.
 * Then w = A q, alpha = q.w, u = w - alpha Bq - beta_prev Bq_prev,
 * unorm = ||u||_2. q on the pattern rows of column c (pat_rows[pat_off[c]] ..
 * pat_rows[pat_off[c+1]-1]) is copied to qp[pat_off[c] ..]. The A-product is
 * written to v, whose old contents are no longer needed. Returns the CG
 * iteration count of the B-solve (0 when first), -1 if it did not converge. */
int o3_step(int64_t M, const int64_t* aptr, const int32_t* aidx, const double* aval, const int64_t* bptr,
            const int32_t* bidx, const double* bval, int C, int ld, int first, double bsolve_tol, int max_cg,
            double* q, double* Bq, double* Bqp, double* u, double* v, double* R, double* P, double* BP,
            double* beta_prev, double* alpha, double* beta, double* unorm, const int64_t* pat_off,
            const int32_t* pat_rows, double* qp) {
  double* part = (double*)malloc(sizeof(double) * NBLK * (C > 0 ? C : 1));
  int cg = 0;
  if (!first) {
    cg = o3_cg(M, bptr, bidx, bval, C, ld, u, v, bsolve_tol, max_cg, R, P, BP);
    dots(M, C, ld, u, v, beta, part);
    for (int c = 0; c < C; ++c) beta[c] = sqrt(beta[c]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i)
      for (int c = 0; c < C; ++c) {
        Bqp[i * ld + c] = Bq[i * ld + c];
        Bq[i * ld + c] = u[i * ld + c] / beta[c];
        q[i * ld + c] = v[i * ld + c] / beta[c];
      }
    for (int c = 0; c < C; ++c) beta_prev[c] = beta[c];
  }
  double* w = v;
  o3_spmm(M, aptr, aidx, aval, C, ld, q, w);
  dots(M, C, ld, q, w, alpha, part);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < M; ++i)
    for (int c = 0; c < C; ++c)
      u[i * ld + c] = w[i * ld + c] - alpha[c] * Bq[i * ld + c] - beta_prev[c] * Bqp[i * ld + c];
  dots(M, C, ld, u, u, unorm, part);
  for (int c = 0; c < C; ++c) {
    unorm[c] = sqrt(unorm[c]);
    for (int64_t t = pat_off[c]; t < pat_off[c + 1]; ++t) qp[t] = q[(int64_t)pat_rows[t] * ld + c];
  }
  free(part);
  return cg;
}

/* (z I - T) y = beta0 e_1 with T = tridiag(beta, alpha, beta) of order n, by
 * Gaussian elimination with partial pivoting (each step keeps the larger of
 * the pivot and the entry below it, which fills one extra superdiagonal).
 * The elimination runs over the whole matrix; back substitution gives y in
 * full when y != NULL. Returns y_n (the last entry). Work: 4 n complex. */
static cplx tridiag_solve(int n, const double* alpha, const double* beta, double beta0, cplx z, cplx* work,
                          cplx* y) {
  cplx* d = work;          /* pivot row diagonal */
  cplx* du = work + n;     /* first superdiagonal */
  cplx* du2 = work + 2 * n;/* second superdiagonal (from interchanges) */
  cplx* b = work + 3 * n;  /* right-hand side */
  for (int i = 0; i < n; ++i) {
    d[i] = z - alpha[i];
    du[i] = (i + 1 < n) ? -beta[i] : 0.0;
    du2[i] = 0.0;
    b[i] = 0.0;
  }
  b[0] = beta0;
  for (int i = 0; i + 1 < n; ++i) {
    const cplx l = -beta[i];       /* entry (i+1, i) */
    if (cabs(d[i]) >= cabs(l)) {
      const cplx m = l / d[i];
      d[i + 1] -= m * du[i];
      b[i + 1] -= m * b[i];
    } else {
      /* interchange rows i and i+1 */
      const cplx m = d[i] / l;
      const cplx di1 = d[i + 1], dui1 = (i + 2 < n) ? du[i + 1] : 0.0, bi = b[i];
      d[i] = l;
      d[i + 1] = du[i] - m * di1;
      du[i] = di1;
      du2[i] = dui1;
      if (i + 2 < n) du[i + 1] = -m * dui1;
      b[i] = b[i + 1];
      b[i + 1] = bi - m * b[i + 1];
    }
  }
  const cplx last = b[n - 1] / d[n - 1];
  if (y) {
    y[n - 1] = last;
    if (n >= 2) y[n - 2] = (b[n - 2] - du[n - 2] * y[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) y[i] = (b[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
  }
  return last;
}

/* For each shift k < S: solve (z_k I - T_n) y = beta0 e_1. z: S complex
 * (interleaved re, im). last[k] receives y_n (interleaved); when y_full !=
 * NULL it receives y column-major per shift: y_full[(k * n + i) * 2 + {0,1}]. */
void o3_tridiag(int n, const double* alpha, const double* beta, double beta0, int S, const double* z,
                double* last, double* y_full) {
#pragma omp parallel
  {
    cplx* work = (cplx*)malloc(sizeof(cplx) * 4 * (size_t)n);
#pragma omp for schedule(dynamic, 1)
    for (int k = 0; k < S; ++k) {
      const cplx zk = z[2 * k] + z[2 * k + 1] * I;
      cplx* y = y_full ? (cplx*)(y_full + (size_t)k * n * 2) : NULL;
      const cplx r = tridiag_solve(n, alpha, beta, beta0, zk, work, y);
      last[2 * k] = creal(r);
      last[2 * k + 1] = cimag(r);
    }
    free(work);
  }
}
