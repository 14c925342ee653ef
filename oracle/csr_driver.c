/*
 * TEST INFRASTRUCTURE ONLY (part of the FP64 CPU oracle): multi-threaded drivers of the oracle's
 * assembled Crank--Nicolson step and RK4 step, used as the CPU baselines that are timed beside the
 * GPU library.
 *
 * Each step forms b = B z + dt h and solves A z' = b (Eq. theta-method with theta = 1/2,
 * A = M + dt/2 D, B = M - dt/2 D, Eq. system-matrix-rhs) by restarted GMRES(restart) with modified
 * Gram--Schmidt Arnoldi, Givens rotations and right point-Jacobi preconditioning, stopping when
 * ||b - A z|| <= tol ||b||: the same algorithm as oracle/steppers.py gmres(), written in C with
 * OpenMP loops (sparse matrix-vector products, dot products, vector updates) over all host cores.
 * The matrices come from oracle/dg.py (scipy CSR: row pointers, column indices, values).  It
 * shares nothing with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

static void spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Returns the number of threads used (`threads` > 0 sets it, 0 keeps the OpenMP default: all host
 * cores); *iterations = GMRES iterations summed over the steps; -1 on allocation failure.  z (in/out)
 * holds the state. */
int oracle_cn_gmres_steps(int64_t n, const int64_t* arp, const int32_t* aci, const double* av, const int64_t* brp,
                          const int32_t* bci, const double* bv, const double* dth, double* z, int nsteps,
                          double tol, int restart, int maxit, int threads, int64_t* iterations) {
  const int m = restart;
  if (threads > 0) omp_set_num_threads(threads);
  double* dinv = malloc(sizeof(double) * n);
  double* b = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* w = malloc(sizeof(double) * n);
  double* V = malloc(sizeof(double) * (size_t)n * (m + 1));
  double* H = calloc((size_t)(m + 1) * m, sizeof(double));
  double* g = calloc(m + 1, sizeof(double));
  double* cs = calloc(m, sizeof(double));
  double* sn = calloc(m, sizeof(double));
  double* y = calloc(m, sizeof(double));
  if (!dinv || !b || !r || !w || !V || !H || !g || !cs || !sn || !y) {
    free(dinv); free(b); free(r); free(w); free(V); free(H); free(g); free(cs); free(sn); free(y);
    return -1;
  }
  /* diagonal of A for the point-Jacobi preconditioner */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t k = arp[i]; k < arp[i + 1]; ++k)
      if (aci[k] == i) d += av[k];
    dinv[i] = 1.0 / d;
  }
  int64_t its = 0;
  for (int step = 0; step < nsteps; ++step) {
    spmv(n, brp, bci, bv, z, b);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) b[i] += dth[i];
    const double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
      memset(z, 0, sizeof(double) * n);
      continue;
    }
    int step_its = 0;
    while (step_its < maxit) {
      spmv(n, arp, aci, av, z, r);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
      const double beta = sqrt(dot(n, r, r));
      if (beta <= tol * bnorm) break;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
      memset(g, 0, sizeof(double) * (m + 1));
      g[0] = beta;
      int jdone = 0;
      for (int j = 0; j < m; ++j) {
        double* vj = V + (size_t)j * n;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) r[i] = dinv[i] * vj[i];
        spmv(n, arp, aci, av, r, w);
        for (int i2 = 0; i2 <= j; ++i2) { /* modified Gram--Schmidt */
          const double* vi = V + (size_t)i2 * n;
          const double hij = dot(n, vi, w);
          H[(size_t)i2 * m + j] = hij;
#pragma omp parallel for schedule(static)
          for (int64_t i = 0; i < n; ++i) w[i] -= hij * vi[i];
        }
        const double hn = sqrt(dot(n, w, w));
        H[(size_t)(j + 1) * m + j] = hn;
        if (hn > 0.0) {
          double* vn = V + (size_t)(j + 1) * n;
#pragma omp parallel for schedule(static)
          for (int64_t i = 0; i < n; ++i) vn[i] = w[i] / hn;
        }
        for (int i2 = 0; i2 < j; ++i2) { /* previous Givens rotations */
          const double a0 = H[(size_t)i2 * m + j], a1 = H[(size_t)(i2 + 1) * m + j];
          H[(size_t)i2 * m + j] = cs[i2] * a0 + sn[i2] * a1;
          H[(size_t)(i2 + 1) * m + j] = -sn[i2] * a0 + cs[i2] * a1;
        }
        const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
        const double den = hypot(a0, a1);
        cs[j] = a0 / den;
        sn[j] = a1 / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++step_its;
        jdone = j + 1;
        if (fabs(g[j + 1]) <= tol * bnorm || step_its >= maxit) break;
      }
      for (int i2 = jdone - 1; i2 >= 0; --i2) { /* y = R^-1 g */
        double v = g[i2];
        for (int k2 = i2 + 1; k2 < jdone; ++k2) v -= H[(size_t)i2 * m + k2] * y[k2];
        y[i2] = v / H[(size_t)i2 * m + i2];
      }
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) { /* z += P^-1 V y (right preconditioning) */
        double s = 0.0;
        for (int k2 = 0; k2 < jdone; ++k2) s += V[(size_t)k2 * n + i] * y[k2];
        z[i] += dinv[i] * s;
      }
    }
    its += step_its;
  }
  *iterations = its;
  free(dinv); free(b); free(r); free(w); free(V); free(H); free(g); free(cs); free(sn); free(y);
  return omp_get_max_threads();
}

/* Classical RK4 (Sec. 3.4) on zeta' = M^-1 (h - D zeta), the algorithm of oracle/steppers.py rk4(),
 * with the oracle's assembled D (CSR) and the inverses of its block-diagonal mass matrix: minv holds,
 * per cell, the inverse of the nloc x nloc mass block that every one of the cell's n coefficient
 * rows shares (degree of freedom (cell n + r) nloc + a).  OpenMP loops over all host cores (or
 * `threads`).  Returns the number of threads, -1 on allocation failure; z (in/out) holds the state. */
int oracle_rk4_steps(int64_t ncell, int n, int nloc, const int64_t* rp, const int32_t* ci, const double* v,
                     const double* minv, const double* h, double* z, int nsteps, double dt, int threads) {
  if (threads > 0) omp_set_num_threads(threads);
  const int64_t N = ncell * (int64_t)n * nloc;
  double* t = malloc(sizeof(double) * N);
  double* y = malloc(sizeof(double) * N);
  double* k = malloc(sizeof(double) * N);
  double* acc = malloc(sizeof(double) * N);
  if (!t || !y || !k || !acc) {
    free(t); free(y); free(k); free(acc);
    return -1;
  }
  const double a[4] = {0.5, 0.5, 1.0, 0.0};          /* stage input Y_{s+1} = z + a_s dt k_s */
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  for (int step = 0; step < nsteps; ++step) {
    memcpy(y, z, sizeof(double) * N);
    memcpy(acc, z, sizeof(double) * N);
    for (int st = 0; st < 4; ++st) {
      spmv(N, rp, ci, v, y, t); /* t = D Y */
#pragma omp parallel for schedule(static)
      for (int64_t blk = 0; blk < ncell * (int64_t)n; ++blk) { /* k = M^-1 (h - D Y) */
        const double* mi = minv + (size_t)(blk / n) * nloc * nloc;
        const int64_t o = blk * nloc;
        for (int i = 0; i < nloc; ++i) {
          double s = 0.0;
          for (int j = 0; j < nloc; ++j) s += mi[i * nloc + j] * (h[o + j] - t[o + j]);
          k[o + i] = s;
        }
      }
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < N; ++i) {
        acc[i] += dt * b[st] * k[i];
        y[i] = z[i] + a[st] * dt * k[i];
      }
    }
    memcpy(z, acc, sizeof(double) * N);
  }
  free(t); free(y); free(k); free(acc);
  return omp_get_max_threads();
}
