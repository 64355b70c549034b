/*
 * FP64 CPU oracle for GPSS: gradient projection onto the l1 ball with the
 * adaptive Barzilai-Borwein steplength selection (Algorithm GP + Algorithm SS,
 * Sec. 3 of Loris, Bertero, De Mol, Zanella, Zanni, "Accelerating gradient
 * projection methods for l1-constrained signal recovery by steplength
 * selection rules").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the reference that the CUDA path is
 * compared against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library, and it never calls it.
 *
 * Everything is computed in double precision.  K may be stored as float64,
 * float32 or bfloat16 bit patterns; every element is widened exactly to
 * double before use, so the oracle solves exactly the stored problem.
 */
#ifndef GPSS_ORACLE_H
#define GPSS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_F64 = 0, ORA_F32 = 1, ORA_BF16 = 2 };

/* Stop reasons reported in ora_result.stop. */
enum {
  ORA_STOP_REL_GAP = 0,     /* (f - f_star)/f_star <= tol                         */
  ORA_STOP_STATIONARY = 1,  /* h == x exactly (Alg. GP, Step 2)                   */
  ORA_STOP_FW = 2,          /* Frank-Wolfe certificate <= tol                     */
  ORA_STOP_MAX_ITER = 3,
  ORA_STOP_LINESEARCH = 4,  /* backtracking cap reached                           */
  ORA_STOP_NONFINITE = 5,
  ORA_STOP_STAGNATION = 6   /* f did not decrease for `stagnation` iterations     */
};

typedef struct {
  double beta, theta;        /* Armijo parameters (Alg. GP)                         */
  int M;                     /* non-monotone memory (Alg. GP, Step 4)               */
  double alpha_min, alpha_max, tau1;
  int M_alpha;               /* length of the BB2 window (Alg. SS)                  */
  double tol;                /* tolerance of the stop rule                          */
  double f_star;             /* > 0: stop on relative gap to f_star                 */
  int stop_fw;               /* 1: stop on the Frank-Wolfe certificate              */
  int max_iter, max_backtracks;
  int stagnation;            /* > 0: stop when f has not decreased for this many it */
  int alpha0_rule;           /* 0: literal ||P(x0 - g0)||_inf; 1: ||P(x0-g0) - x0||  */
} ora_params;

typedef struct {
  int stop, iters, backtracks;
  double f;                  /* f(x) = ||Kx - y||^2 at the returned x, fresh         */
  double lambda_reg;         /* max_i |(K^T (y - K x))_i|  (relation of Sec. 1)      */
  double l1;                 /* ||x||_1                                              */
  double fw_gap;             /* g^T x + rho ||g||_inf at the returned x              */
} ora_result;

void ora_params_default(ora_params* prm);

/* Euclidean projection onto {||w||_1 <= rho} by sorting (Duchi, Shalev-Shwartz,
 * Singer, Chandra, ICML 2008).  Returns the threshold tau (0 if v is inside). */
double ora_project_l1(const double* v, double* out, long p, double rho);

/* r = K x - y (length n); returns ||r||^2. */
double ora_residual(const void* K, int dtype, long n, long p, long ldk,
                    const double* y, const double* x, double* r);

/* out = K^T r (length p). */
void ora_kt(const void* K, int dtype, long n, long p, long ldk, const double* r, double* out);

/* Algorithm GP with Algorithm SS.  x holds x0 on entry (projected first if it
 * is infeasible) and the result on exit.  trace, if not NULL, receives
 * 4 doubles per iteration: f(x_k), alpha_k, lambda_k (line-search step), and
 * tau after Alg. SS at iteration k (tau_{k+1}). */
int ora_gpss(const void* K, int dtype, long n, long p, long ldk, const double* y,
             double rho, double* x, const ora_params* prm, ora_result* res, double* trace);

/* Certificates at a given x: lambda = max|K^T(y - Kx)|, fw = g^T x + rho||g||_inf,
 * f = ||Kx - y||^2.  g (length p, may be NULL) receives the gradient 2K^T(Kx-y). */
void ora_certificates(const void* K, int dtype, long n, long p, long ldk, const double* y,
                      double rho, const double* x, double* f, double* lambda_reg,
                      double* fw, double* g);

/* Number of OpenMP threads the oracle uses. */
int ora_num_threads(void);
/* Threads of the OpenMP loops (n > 0), e.g. 1 for a single-threaded timing. */
void ora_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
