/*
 * FP64 CPU oracle for GPSS (Algorithm GP + Algorithm SS, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA path is compared against.
 * It shares no code with the CUDA library and never calls it.
 *
 * The code follows the paper's steps in the paper's order:
 *   - the problem is eq. 2: f(x) = ||Kx - y||^2 on Omega = {||x||_1 <= rho},
 *     so grad f(x) = 2 K^T (Kx - y);
 *   - Algorithm GP (Steps 1-6) with the non-monotone Armijo rule of Step 5,
 *     where every trial value f(x_k + lambda d_k) is evaluated directly with a
 *     fresh product K(x_k + lambda d_k);
 *   - Algorithm SS for alpha_k, with s = x_k - x_{k-1} and z = g_k - g_{k-1}
 *     formed explicitly and the BB rules of eq. (bbrules);
 *   - the default parameters listed at the end of Sec. 3.
 * The projection onto Omega, which the paper uses without giving an algorithm,
 * is the sort-based method of Duchi, Shalev-Shwartz, Singer & Chandra (2008).
 */
#include "gpss_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- storage */

static double k_at(const void* K, int dtype, long ldk, long i, long j) {
  if (dtype == ORA_F64) return ((const double*)K)[i * ldk + j];
  if (dtype == ORA_F32) return (double)((const float*)K)[i * ldk + j];
  /* bfloat16: the 16 stored bits are the high half of an IEEE float32. */
  unsigned int bits = (unsigned int)((const unsigned short*)K)[i * ldk + j] << 16;
  float f;
  memcpy(&f, &bits, sizeof f);
  return (double)f;
}

void ora_set_threads(int n) {
  if (n > 0) omp_set_num_threads(n);
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------- products with K */

double ora_residual(const void* K, int dtype, long n, long p, long ldk,
                    const double* y, const double* x, double* r) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double acc = 0.0;
    for (long j = 0; j < p; ++j) acc += k_at(K, dtype, ldk, i, j) * x[j];
    r[i] = acc - y[i];
  }
  double f = 0.0;   /* summed in index order, so results do not depend on threads */
  for (long i = 0; i < n; ++i) f += r[i] * r[i];
  return f;
}

void ora_kt(const void* K, int dtype, long n, long p, long ldk, const double* r, double* out) {
  /* Each thread owns a contiguous block of columns and walks all rows. */
#pragma omp parallel
  {
    int nt = 1, t = 0;
#ifdef _OPENMP
    nt = omp_get_num_threads();
    t = omp_get_thread_num();
#endif
    long j0 = p * t / nt, j1 = p * (t + 1) / nt;
    for (long j = j0; j < j1; ++j) out[j] = 0.0;
    for (long i = 0; i < n; ++i) {
      double ri = r[i];
      for (long j = j0; j < j1; ++j) out[j] += k_at(K, dtype, ldk, i, j) * ri;
    }
  }
}

static void gradient(const void* K, int dtype, long n, long p, long ldk, const double* y,
                     const double* x, double* r, double* g, double* f) {
  *f = ora_residual(K, dtype, n, p, ldk, y, x, r);
  ora_kt(K, dtype, n, p, ldk, r, g);
  for (long j = 0; j < p; ++j) g[j] *= 2.0;
}

/* ------------------------------------------------------------ projection */

static int cmp_desc(const void* a, const void* b) {
  double u = *(const double*)a, w = *(const double*)b;
  return (u < w) - (u > w);
}

double ora_project_l1(const double* v, double* out, long p, double rho) {
  double l1 = 0.0;
  for (long i = 0; i < p; ++i) l1 += fabs(v[i]);
  if (l1 <= rho) {
    if (out != v) memcpy(out, v, (size_t)p * sizeof(double));
    return 0.0;
  }
  /* u = |v| sorted decreasingly; the active count is the largest j with
     u_j > (u_1 + ... + u_j - rho) / j, and tau = (u_1 + ... + u_j - rho) / j. */
  double* u = (double*)malloc((size_t)p * sizeof(double));
  for (long i = 0; i < p; ++i) u[i] = fabs(v[i]);
  qsort(u, (size_t)p, sizeof(double), cmp_desc);
  /* j = 1 always qualifies (u_1 - (u_1 - rho) = rho > 0); start from it so
     that a rho below the rounding unit of u_1 still gives a threshold. */
  double S = u[0], tau = u[0] - rho;
  for (long j = 2; j <= p; ++j) {
    S += u[j - 1];
    double t = (S - rho) / (double)j;
    if (u[j - 1] > t) tau = t;
  }
  free(u);
  for (long i = 0; i < p; ++i) {
    double a = fabs(v[i]) - tau;
    double s = (v[i] > 0.0) - (v[i] < 0.0);   /* sgn(0) = 0 */
    out[i] = a > 0.0 ? s * a : 0.0;
  }
  return tau;
}

/* --------------------------------------------------------------- params */

void ora_params_default(ora_params* prm) {
  /* Parameter setting listed at the end of Sec. 3. */
  prm->beta = 1e-4;
  prm->theta = 0.5;
  prm->M = 1;
  prm->alpha_min = 1e-10;
  prm->alpha_max = 1e10;
  prm->tau1 = 0.5;
  prm->M_alpha = 2;
  prm->tol = 1e-6;
  prm->f_star = -1.0;
  prm->stop_fw = 0;
  prm->max_iter = 100000;
  prm->max_backtracks = 100;
  prm->stagnation = 0;
  prm->alpha0_rule = 0;
}

static double clamp(double a, double lo, double hi) { return a < lo ? lo : (a > hi ? hi : a); }

static double norm_inf(const double* v, long p) {
  double m = 0.0;
  for (long i = 0; i < p; ++i) m = fabs(v[i]) > m ? fabs(v[i]) : m;
  return m;
}

void ora_certificates(const void* K, int dtype, long n, long p, long ldk, const double* y,
                      double rho, const double* x, double* f, double* lambda_reg,
                      double* fw, double* g_out) {
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* g = (double*)malloc((size_t)p * sizeof(double));
  double fx;
  gradient(K, dtype, n, p, ldk, y, x, r, g, &fx);
  double gx = 0.0;
  for (long j = 0; j < p; ++j) gx += g[j] * x[j];
  double gi = norm_inf(g, p);
  if (f) *f = fx;
  /* lambda = max|K^T (y - Kx)| = ||g||_inf / 2 (relation of Sec. 1). */
  if (lambda_reg) *lambda_reg = 0.5 * gi;
  /* Frank-Wolfe gap: max over w in Omega of g^T (x - w) = g^T x + rho ||g||_inf,
     an upper bound on f(x) - f* by convexity. */
  if (fw) *fw = gx + rho * gi;
  if (g_out) memcpy(g_out, g, (size_t)p * sizeof(double));
  free(r);
  free(g);
}

/* ----------------------------------------------------- Algorithm GP + SS */

int ora_gpss(const void* K, int dtype, long n, long p, long ldk, const double* y,
             double rho, double* x, const ora_params* prm, ora_result* res, double* trace) {
  const size_t P = (size_t)p * sizeof(double), N = (size_t)n * sizeof(double);
  double *r = malloc(N), *g = malloc(P), *g_old = malloc(P), *x_old = malloc(P);
  double *h = malloc(P), *d = malloc(P), *xt = malloc(P), *rt = malloc(N);
  const int M = prm->M > 0 ? prm->M : 1;
  const int Ma = prm->M_alpha >= 0 ? prm->M_alpha : 0;
  double* f_hist = malloc((size_t)M * sizeof(double));          /* f(x_{k-j}), j < M   */
  double* a2_hist = malloc((size_t)(Ma + 1) * sizeof(double));  /* alpha^(2)_j window  */
  int a2_count = 0;

  /* The starting point must lie in Omega (Alg. GP): project it if it does not. */
  ora_project_l1(x, x, p, rho);

  double f;
  gradient(K, dtype, n, p, ldk, y, x, r, g, &f);

  /* alpha_0 = max{alpha_min, min{1/||P(x0 - grad f(x0))||_inf, alpha_max}} (Sec. 3). */
  for (long j = 0; j < p; ++j) xt[j] = x[j] - g[j];
  ora_project_l1(xt, h, p, rho);
  if (prm->alpha0_rule == 1)
    for (long j = 0; j < p; ++j) h[j] -= x[j];
  double ninf = norm_inf(h, p);
  double alpha = ninf > 0.0 ? clamp(1.0 / ninf, prm->alpha_min, prm->alpha_max) : prm->alpha_max;
  double tau = prm->tau1;   /* tau_1 (Alg. SS, k = 0) */

  int stop = ORA_STOP_MAX_ITER, k = 0, backtracks = 0;
  double best_f = f;
  int since_best = 0;
  for (int j = 0; j < M; ++j) f_hist[j] = f;

  for (k = 0; k < prm->max_iter; ++k) {
    if (!isfinite(f)) { stop = ORA_STOP_NONFINITE; break; }
    if (prm->stop_fw) {
      double gx = 0.0;
      for (long j = 0; j < p; ++j) gx += g[j] * x[j];
      double fw = gx + rho * norm_inf(g, p);
      if (fw <= prm->tol * (f - fw)) { stop = ORA_STOP_FW; break; }
    }

    /* Step 1: choose alpha_k by Algorithm SS. */
    if (k >= 1) {
      double ss = 0.0, sz = 0.0, zz = 0.0;
      for (long j = 0; j < p; ++j) {
        double s = x[j] - x_old[j], z = g[j] - g_old[j];
        ss += s * s;
        sz += s * z;
        zz += z * z;
      }
      double a2_this;
      if (sz <= 0.0) {
        alpha = prm->alpha_max;
        a2_this = prm->alpha_max;          /* alpha^(2)_k undefined: does not lower the min */
      } else {
        double a1 = clamp(ss / sz, prm->alpha_min, prm->alpha_max);
        double a2 = clamp(sz / zz, prm->alpha_min, prm->alpha_max);
        a2_this = a2;
        /* window j = max(1, k - M_alpha), ..., k  includes the current value */
        double amin = a2;
        for (int q = 0; q < a2_count && q < Ma; ++q) amin = a2_hist[q] < amin ? a2_hist[q] : amin;
        if (a2 / a1 <= tau) {
          alpha = amin;
          tau *= 0.9;
        } else {
          alpha = a1;
          tau *= 1.1;
        }
      }
      /* push alpha^(2)_k into the window (most recent first) */
      for (int q = Ma - 1; q > 0; --q) a2_hist[q] = a2_hist[q - 1];
      if (Ma > 0) a2_hist[0] = a2_this;
      if (a2_count < Ma) ++a2_count;
    }

    /* Step 2: h = P(x - alpha g); stop if h == x. */
    for (long j = 0; j < p; ++j) xt[j] = x[j] - alpha * g[j];
    ora_project_l1(xt, h, p, rho);
    int same = 1;
    for (long j = 0; j < p; ++j) same &= (h[j] == x[j]);
    if (same) { stop = ORA_STOP_STATIONARY; break; }

    /* Step 3: d = h - x.  Step 4: lambda = 1, f_max over the last M values. */
    double gd = 0.0;
    for (long j = 0; j < p; ++j) {
      d[j] = h[j] - x[j];
      gd += g[j] * d[j];
    }
    double fmax = f_hist[0];
    for (int j = 1; j < M && j <= k; ++j) fmax = f_hist[j] > fmax ? f_hist[j] : fmax;

    /* Step 5: backtracking with f(x + lambda d) evaluated directly. */
    double lam = 1.0, ft = 0.0;
    int bt = 0, ls_ok = 0;
    for (;;) {
      for (long j = 0; j < p; ++j) xt[j] = x[j] + lam * d[j];
      ft = ora_residual(K, dtype, n, p, ldk, y, xt, rt);
      if (ft <= fmax + prm->beta * lam * gd) { ls_ok = 1; break; }
      if (bt >= prm->max_backtracks) break;
      lam *= prm->theta;
      ++bt;
    }
    backtracks += bt;
    if (trace) {
      trace[4 * k + 0] = f;
      trace[4 * k + 1] = alpha;
      trace[4 * k + 2] = lam;
      trace[4 * k + 3] = tau;
    }
    if (!ls_ok) { stop = ORA_STOP_LINESEARCH; break; }

    /* Step 6: x_{k+1} = x_k + lambda d; keep x_k and g_k for s and z. */
    memcpy(x_old, x, P);
    memcpy(g_old, g, P);
    memcpy(x, xt, P);
    gradient(K, dtype, n, p, ldk, y, x, r, g, &f);
    for (int j = M - 1; j > 0; --j) f_hist[j] = f_hist[j - 1];
    f_hist[0] = f;

    if (prm->f_star > 0.0 && (f - prm->f_star) <= prm->tol * prm->f_star) {
      ++k;
      stop = ORA_STOP_REL_GAP;
      break;
    }
    if (prm->stagnation > 0) {
      if (f < best_f) { best_f = f; since_best = 0; }
      else if (++since_best >= prm->stagnation) { ++k; stop = ORA_STOP_STAGNATION; break; }
    }
  }

  if (res) {
    res->stop = stop;
    res->iters = k;
    res->backtracks = backtracks;
    ora_certificates(K, dtype, n, p, ldk, y, rho, x, &res->f, &res->lambda_reg, &res->fw_gap, NULL);
    double l1 = 0.0;
    for (long j = 0; j < p; ++j) l1 += fabs(x[j]);
    res->l1 = l1;
  }
  free(r); free(g); free(g_old); free(x_old); free(h); free(d); free(xt); free(rt);
  free(f_hist); free(a2_hist);
  return stop;
}
