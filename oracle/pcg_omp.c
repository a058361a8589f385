/*
 * Textbook Jacobi-preconditioned conjugate gradients on a CSR matrix, FP64, with OpenMP over
 * rows (oracle timing baseline).
 *
 * TEST INFRASTRUCTURE ONLY: the "fair CPU" figure of the benchmark -- the oracle's iterative
 * solve of a state system K u = F (the SPD systems of Sec. 6.2 eq. compli_weak and Sec. 6.3
 * eq. heat_weak, restricted to the free DOFs) on all host cores.  It shares nothing with the
 * CUDA library.  The iteration is the classical Hestenes-Stiefel recurrence with z = D^{-1} r:
 *   r = b - K x, z = D^{-1} r, p = z;  repeat: q = K p, alpha = (r, z) / (p, q),
 *   x += alpha p, r -= alpha q, z = D^{-1} r, beta = (r, z)_new / (r, z)_old, p = z + beta p,
 * until ||r||_2 <= rtol ||b||_2 or maxit iterations.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t *ip, const int32_t *ix, const double *a, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = ip[i]; k < ip[i + 1]; ++k) s += a[k] * x[ix[k]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double *u, const double *v) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
  return s;
}

/* Returns 0 on convergence, 1 when maxit was reached, -1 on a bad argument or no memory.
 * x holds the start value on entry and the solution on exit.  *threads = OpenMP threads used. */
int oracle_pcg_csr(int64_t n, const int64_t *ip, const int32_t *ix, const double *a, const double *b, double *x,
                   double rtol, int maxit, int *iters, double *relres, int *threads) {
  if (n <= 0 || !ip || !ix || !a || !b || !x) return -1;
  double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
  double *q = malloc(sizeof(double) * n), *dinv = malloc(sizeof(double) * n);
  if (!r || !z || !p || !q || !dinv) {
    free(r), free(z), free(p), free(q), free(dinv);
    return -1;
  }
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  if (threads) *threads = nt;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t k = ip[i]; k < ip[i + 1]; ++k)
      if (ix[k] == i) d += a[k];
    dinv[i] = d != 0.0 ? 1.0 / d : 1.0;
  }
  spmv(n, ip, ix, a, x, q);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - q[i];
    z[i] = dinv[i] * r[i];
    p[i] = z[i];
  }
  const double bb = dot(n, b, b);
  double rz = dot(n, r, z), rr = dot(n, r, r);
  int it = 0;
  while (rr > rtol * rtol * bb && it < maxit) {
    spmv(n, ip, ix, a, p, q);
    const double alpha = rz / dot(n, p, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      z[i] = dinv[i] * r[i];
    }
    const double rz_new = dot(n, r, z);
    rr = dot(n, r, r);
    const double beta = rz_new / rz;
    rz = rz_new;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    ++it;
  }
  if (iters) *iters = it;
  if (relres) *relres = bb > 0 ? sqrt(rr / bb) : 0.0;
  free(r), free(z), free(p), free(q), free(dinv);
  return rr > rtol * rtol * bb ? 1 : 0;
}
