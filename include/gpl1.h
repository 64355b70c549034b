/*
 * gpl1 -- gradient projection onto the l1 ball with adaptive Barzilai-Borwein
 * steplengths (GPSS), single GB300 GPU, C ABI.
 *
 * Problem (eq. 2, Sec. 1):   minimise f(x) = ||K x - y||^2   subject to ||x||_1 <= rho,
 * with K an n x p matrix.  The method is Algorithm GP (gradient projection with
 * a non-monotone Armijo line search along the feasible direction) with
 * Algorithm SS (adaptive alternation of the two Barzilai-Borwein rules of
 * eq. (bbrules)), both in Sec. 3; the default parameters are the ones listed at
 * the end of Sec. 3.
 *
 * Conventions shared by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller, unless a
 *     comment says otherwise.  The library never frees caller memory.
 *   - K is row-major: element (i, j) is at K[i * ldk + j], 0 <= i < n,
 *     0 <= j < p, ldk >= p.  The K pointer must be 16-byte aligned and
 *     ldk * sizeof(element) must be a multiple of 16 bytes (rows start on
 *     16-byte boundaries); columns p..ldk-1 are never read.
 *   - Element types: GPL1_F64 -> K, y, x are double.  GPL1_F32 -> K, y, x are
 *     float.  GPL1_BF16 -> K is bfloat16 (raw 16-bit patterns), y and x are
 *     float.  Products with K accumulate in float (double for GPL1_F64); the
 *     line-search test, the steplength rule and the projection threshold are
 *     decided in double precision.
 *   - Work is enqueued on the context's stream (gpl1_create / gpl1_set_stream)
 *     in stream order.  Calls that return results in host memory synchronise
 *     that stream before returning.
 *   - Every function returns a gpl1_status; nothing throws or aborts across
 *     the ABI.  On GPL1_ERR_INVALID_ARG / GPL1_ERR_UNSUPPORTED nothing was
 *     enqueued.  gpl1_last_error() returns a message for the last failure.
 *   - Device-side waits are bounded by gpl1_params.timeout_ns; a wait that runs
 *     out reports GPL1_ERR_TIMEOUT instead of hanging.
 */
#ifndef GPL1_H
#define GPL1_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpl1_ctx gpl1_ctx; /* opaque: stream, device workspace, cached plans */

typedef enum {
  GPL1_OK = 0,
  GPL1_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment, parameter           */
  GPL1_ERR_CUDA = 2,          /* a CUDA runtime call failed                         */
  GPL1_ERR_NOT_CONVERGED = 3, /* max_iter reached before the stop rule held         */
  GPL1_ERR_LINESEARCH = 4,    /* Armijo backtracking cap reached (Alg. GP, Step 5)  */
  GPL1_ERR_NONFINITE = 5,     /* f, a dot product or the steplength became NaN/inf  */
  GPL1_ERR_TIMEOUT = 6,       /* a device-side wait exceeded timeout_ns             */
  GPL1_ERR_UNSUPPORTED = 7    /* size or shape beyond what the library handles      */
} gpl1_status;

typedef enum { GPL1_F64 = 0, GPL1_F32 = 1, GPL1_BF16 = 2 } gpl1_dtype;

/* Why a solve stopped (gpl1_result.stop). */
typedef enum {
  GPL1_STOP_REL_GAP = 0,    /* f(x) - f_star <= tol max(f_star, tol ||y||^2)         */
  GPL1_STOP_STATIONARY = 1, /* P(x - alpha g) == x exactly: stationary (Alg. GP, Step 2) */
  GPL1_STOP_FW = 2,         /* Frank-Wolfe certificate (g^T x + rho ||g||_inf) <= tol (f - cert) */
  GPL1_STOP_MAX_ITER = 3,
  GPL1_STOP_ERROR = 4,      /* see gpl1_result.status                                */
  GPL1_STOP_STAGNATION = 5  /* float data (one-read single solve, shared-K form): f
                               stopped falling near the stop (by 1e-3 tol of the gap
                               denominator) for 64 (single solve) or 32 (shared-K)
                               iterations before the rule held: the precision floor of
                               the FP32 path; status GPL1_ERR_NOT_CONVERGED           */
} gpl1_stop;

/* Stop rules (gpl1_params.stop_rule, a bit set; the solve stops at the first that holds). */
#define GPL1_STOP_ON_REL_GAP 1 /* needs f_star >= 0                                    */
#define GPL1_STOP_ON_FW 2

#define GPL1_DEBUG_UNREACHABLE_BARRIER 1

typedef struct {
  /* Algorithm GP (Sec. 3): Armijo parameters beta, theta in (0,1), memory M >= 1. */
  double beta, theta;
  int M;
  /* Algorithm SS (Sec. 3): 0 < alpha_min < alpha_max, tau_1 in (0,1), M_alpha >= 0. */
  double alpha_min, alpha_max, tau1;
  int M_alpha;
  /* stop rule */
  double tol;          /* tolerance of the rules in stop_rule                          */
  double f_star;       /* optimal value for GPL1_STOP_ON_REL_GAP (< 0: unknown)        */
  int stop_rule;       /* GPL1_STOP_ON_* bits; h == x always stops                     */
  int max_iter;        /* iterations of Alg. GP                                        */
  int max_backtracks;  /* trials of Alg. GP Step 5 before GPL1_ERR_LINESEARCH          */
  int alpha0_rule;     /* 0: alpha_0 = 1/||P(x0 - g0)||_inf (Sec. 3, literal);
                          1: alpha_0 = 1/||P(x0 - g0) - x0||_inf                      */
  int x0_is_zero;      /* 1: ignore the contents of x and start from x0 = 0            */
  int debug;           /* 0.  Bit GPL1_DEBUG_UNREACHABLE_BARRIER makes the group barrier
                          of a multi-CTA solve wait for one arrival more than the group
                          has, so the solve must end with GPL1_ERR_TIMEOUT after
                          timeout_ns: a fault-free test of the bounded-wait path.      */
  long long timeout_ns; /* bound on every device-side wait                             */
  int engine;          /* which kernel runs a single solve (gpl1_solve, gpl1_solve_async):
                          GPL1_ENGINE_AUTO lets the autotuner pick among the kernels
                          that can take the instance (below); the batched calls and
                          gpl1_solve_noalloc always run the two-pass kernel          */
  int method;          /* GPL1_METHOD_GPSS (Alg. GP + SS, the default) or one of the
                          comparison methods of Sec. 2 below; those run only in single
                          solves (gpl1_solve, gpl1_solve_async) on the one-read kernel */
  double lambda_pen;   /* ISTA, FISTA: lambda > 0 of eq. 1                             */
  double step;         /* ISTA, FISTA: step s > 0 of x + s K^T (y - K x) thresholded at
                          s lambda; 1 is the paper's iteration (||K|| < 1), 1/||K||^2
                          (gpl1_spectral_norm_sq) admits any K                         */
  int tile;            /* box shape of the two-pass kernel (GPL1_TILE_*): AUTO lets the
                          batched calls tune it per batch (gpl1_batched_tuned) and
                          gives MEDIUM to single solves; gpl1_solve_noalloc always
                          runs MEDIUM                                                 */
  int tile_pad;        /* 0 */
} gpl1_params;

/* gpl1_params.tile: the two-pass kernel streams K in TMA boxes of RB rows x
 * 256 columns through a 120 KiB shared-memory ring; RB rows split evenly over
 * its 15 consumer warps.
 *   SMALL:  15 KiB boxes, 8 stages (RB = 15 F32, 30 BF16; no F64 shape)
 *   MEDIUM: 30 KiB boxes, 4 stages (RB = 15 F64, 30 F32, 60 BF16)
 *   LARGE:  60 KiB boxes, 2 stages (RB = 30 F64, 60 F32, 120 BF16)
 * Smaller boxes pad ragged row counts less and spread an instance over more
 * units; larger ones take fewer waits and reductions per byte.  AUTO: the
 * first time a context meets a batch (dtype and the list of instance shapes),
 * gpl1_solve_batched, gpl1_solve_batched_async and gpl1_plan_create time
 * every admissible shape on the batch itself (four iterations into scratch
 * copies of x, twice; the faster second run wins) and keep the choice for the
 * context; that first call synchronises the stream.  A shape given here is used
 * as is (GPL1_ERR_UNSUPPORTED for SMALL with F64 data). */
#define GPL1_TILE_AUTO 0
#define GPL1_TILE_SMALL 1
#define GPL1_TILE_MEDIUM 2
#define GPL1_TILE_LARGE 3

/* gpl1_params.method: the iterations of Sec. 2 on the one-read kernel's passes
 * (each pass forms K v and 2 K^T (K x - y), 2 K^T K v for the pass's direction v
 * in one read of K; the methods differ only in the scalar step between passes).
 *  ISTA:  x_{k+1} = S_{s lam}[x_k + s K^T (y - K x_k)]                  (eq. 1)
 *  FISTA: x_{k+1} = T(x_k + (t_k - 1)/t_{k+1} (x_k - x_{k-1})), T the ISTA map,
 *         t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2        (eq. fista; eq. 1)
 *  PSD:   x_{k+1} = P_Omega[x_k + beta_k r_k], r_k = K^T (y - K x_k),
 *         beta_k = ||r_k||^2 / ||K r_k||^2                                   (eq. 2)
 * One pass per iteration for ISTA and FISTA, two for PSD (beta_k needs K r_k
 * before the step).  For ISTA and FISTA, rho is not used (it must still be > 0),
 * x0 is not projected, f_star is the optimal value of eq. 1 (||K x - y||^2 +
 * 2 lam ||x||_1), GPL1_STOP_ON_REL_GAP compares that objective with it, and
 * GPL1_STOP_ON_FW is refused; gpl1_result.f is that objective at the returned x.
 * PSD keeps the conventions of Alg. GP (x0 projected, f and the stop rules of
 * eq. 2).  A step that leaves x unchanged stops with GPL1_STOP_STATIONARY. */
#define GPL1_METHOD_GPSS 0
#define GPL1_METHOD_ISTA 1
#define GPL1_METHOD_FISTA 2
#define GPL1_METHOD_PSD 3

/* gpl1_params.engine.
 *  ONE_READ: one persistent launch of thread-block clusters that reads K once
 *    per iteration.  The gradient is linear in the iterate, so the pass that
 *    forms K x_k and K d_k also forms 2 K^T (K x_k - y) and 2 K^T K d_k from
 *    the same tiles, and g_{k+1} is their combination with the Armijo step
 *    (Alg. GP, Steps 5-6).  A cluster of C CTAs covers the p columns, each CTA
 *    a slice of W columns held by its 256 consumer threads, each with two
 *    16-byte chunks of columns (W = 2048 F32, 4096 BF16, 1024 F64) or four
 *    (twice that, half the cluster), up to C = 16.  ONE_READ lets the
 *    autotuner pick the chunks per thread; ONE_READ_NCH2 and ONE_READ_NCH4 fix
 *    them.  GPL1_ERR_UNSUPPORTED when the instance does not fit.
 *  TWO_PASS: one persistent cooperative launch that reads K twice per
 *    iteration (K^T r, then [K d, K x]); p up to 16800 F32/BF16, 3840 F64.
 *  AUTO: the autotuner picks among all engines that fit.
 * The autotuner (AUTO, ONE_READ) times each admissible engine the first time
 * a context meets an instance shape (dtype, n, p): four iterations from
 * x0 = 0 into a scratch x, twice, on the caller's K and y; the faster wins and
 * is kept for the context (gpl1_solve_tuned lists the choices).  That first
 * call synchronises the stream, asynchronous or not. */
#define GPL1_ENGINE_AUTO 0
#define GPL1_ENGINE_ONE_READ 1
#define GPL1_ENGINE_TWO_PASS 2
#define GPL1_ENGINE_ONE_READ_NCH2 3
#define GPL1_ENGINE_ONE_READ_NCH4 4

typedef struct {
  int status;          /* gpl1_status of this instance                                 */
  int stop;            /* gpl1_stop                                                    */
  int iters;           /* completed iterations of Alg. GP                              */
  int backtracks;      /* total Armijo reductions lambda <- theta lambda               */
  double f;            /* f at the returned x (from the exact quadratic expansion)      */
  double rel_gap;      /* (f - f_star)/f_star if f_star > 0, else -1                    */
  double fw_gap;       /* last Frank-Wolfe certificate g^T x + rho ||g||_inf (or -1)    */
  double lambda;       /* last max|K^T (y - K x)| = ||g||_inf / 2 (relation of Sec. 1) */
  double alpha;        /* last steplength alpha_k                                      */
  double tau;          /* last projection threshold                                    */
  double kernel_ms;    /* device time of the solver launch that produced this result
                          (CUDA events on the context stream around the kernel)        */
  int fail_site;       /* GPL1_ERR_TIMEOUT: which bounded wait gave up first (1 pass A
                          box, 2 pass B box, 3 drain, 4 group barrier, 5 producer), or 0 */
  int fail_iter;       /* iteration at which the solve ended                            */
} gpl1_result;

/* One instance of eq. 2 (device pointers).  x holds x0 on entry (projected onto
 * the ball first if it lies outside, since Alg. GP starts in Omega) and the
 * solution on exit. */
typedef struct {
  const void* K;
  long long n, p, ldk;
  const void* y;
  double rho;     /* radius of the l1 ball, > 0                                        */
  void* x;
  double f_star;  /* optional per-instance optimal value (< 0: use gpl1_params.f_star) */
  double* trace;  /* optional device array of trace_cap rows of GPL1_TRACE_COLS doubles:
                     row k = (f(x_k), alpha_k, lambda_k (0 if the line search failed),
                     tau_{k+1} of Alg. SS, g_k^T d_k, ||K d_k||^2, ||d_k||^2,
                     projection threshold, then the nanoseconds from the start of
                     iteration k to the end of: pass A, its barrier, the projection
                     phase, pass B, its barrier, the phase-P reductions, Alg. SS, the
                     threshold search; then the number of threshold-search steps, six
                     clock stamps inside the search and the number of candidates it
                     kept; then, as raw globaltimer values (the bits of the double
                     slots), the earliest and latest end of pass A and of pass B over
                     all CTAs), written for k < trace_cap (the rows must start zeroed);
                     NULL for none                                                   */
  long long trace_cap;
} gpl1_problem;

#define GPL1_TRACE_COLS 28

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; 0 means the legacy default stream).  *out receives the
 * context (NULL on failure).  The context allocates device workspace lazily and
 * frees it in gpl1_destroy. */
gpl1_status gpl1_create(gpl1_ctx** out, int device, void* cuda_stream);
void gpl1_destroy(gpl1_ctx* ctx);
gpl1_status gpl1_set_stream(gpl1_ctx* ctx, void* cuda_stream);
const char* gpl1_last_error(const gpl1_ctx* ctx);

/* Defaults of Sec. 3: M = 1, theta = 0.5, beta = 1e-4, alpha_min = 1e-10,
 * alpha_max = 1e10, tau_1 = 0.5, M_alpha = 2, alpha_0 rule 0; plus tol = 1e-6,
 * stop on the FW certificate, max_iter = 100000, max_backtracks = 100,
 * timeout 10 s. */
void gpl1_params_default(gpl1_params* prm);

/* Euclidean projection onto {w : ||w||_1 <= rho_b} (the P_Omega of Alg. GP,
 * Step 2), for `batch` segments of length p.  Segment b reads v + b*stride and
 * writes out + b*stride (out may equal v).  rho points to `batch` doubles in
 * host memory (rho_on_device = 0) or device memory (1).  Inside the ball the
 * output equals the input bit for bit; otherwise out = sgn(v) max(|v| - tau, 0)
 * with sum max(|v| - tau, 0) = rho, tau found by a radix select on |v| with
 * exact fixed-point partial sums.  dtype GPL1_F64 or GPL1_F32.  tau_out, if not
 * NULL, receives the `batch` thresholds (device pointer, double). */
gpl1_status gpl1_project(gpl1_ctx* ctx, const void* v, void* out, gpl1_dtype dtype, long long p,
                         long long batch, long long stride, const double* rho, int rho_on_device,
                         double* tau_out);

/* Solve one instance with Alg. GP + SS.  k_dtype is the element type of K
 * (see the conventions above).  res: host pointer; the call synchronises the
 * stream and fills it. */
gpl1_status gpl1_solve(gpl1_ctx* ctx, const gpl1_problem* prob, gpl1_dtype k_dtype,
                       const gpl1_params* prm, gpl1_result* res);

/* Solve `count` independent instances of possibly different n, p in one
 * persistent launch.  probs: host array of descriptors (device pointers
 * inside).  res: host array of `count` results; the call synchronises. */
gpl1_status gpl1_solve_batched(gpl1_ctx* ctx, const gpl1_problem* probs, int count,
                               gpl1_dtype k_dtype, const gpl1_params* prm, gpl1_result* res);

/* Batched plans: repeated solves of the same instances without host work.
 * gpl1_plan_create checks the instances and parameters as gpl1_solve_batched
 * does, lays out a workspace owned by the plan, encodes the tensor maps,
 * orders the queue (largest n p first), and records everything one batched
 * solve enqueues (zeroing x when prm->x0_is_zero, zeroing the accumulation
 * buffers, the upload of the descriptors, the persistent launch, the read-back
 * of the results into pinned memory) as a CUDA graph.  gpl1_plan_run replays
 * the graph on the context's stream, synchronises, and fills res (host array
 * of `count` results, in the order of probs) with the same values
 * gpl1_solve_batched gives.  The instances' device arrays (K, y, x) must stay
 * allocated while the plan lives; their contents may change between runs
 * (new right-hand sides written into y, new K values); rho, f_star, the
 * sizes, the dtype and the parameters are fixed at creation.  A plan belongs
 * to its context: destroy it first.  Errors: as gpl1_solve_batched;
 * GPL1_ERR_CUDA if the capture or the graph fails. */
typedef struct gpl1_plan gpl1_plan;
gpl1_status gpl1_plan_create(gpl1_ctx* ctx, const gpl1_problem* probs, int count, gpl1_dtype k_dtype,
                             const gpl1_params* prm, gpl1_plan** out);
gpl1_status gpl1_plan_run(gpl1_plan* plan, gpl1_result* res);
void gpl1_plan_destroy(gpl1_plan* plan);

/* gpl1_solve and gpl1_solve_batched without host synchronisation: the
 * argument checks, workspace sizing and descriptor staging happen in the call,
 * everything else is enqueued on the context's stream, and the results (one
 * per instance, in the order of probs; kernel_ms reads 0) are written to
 * res_dev, a DEVICE array, when the solve completes.  The workspace is the
 * context's: successive calls on one context are ordered by its stream, so a
 * caller overlaps solves with its own copies on other streams (events), not
 * with other solves of the same context.  Status codes report argument and
 * launch errors only; an instance's outcome is in its result. */
gpl1_status gpl1_solve_async(gpl1_ctx* ctx, const gpl1_problem* prob, gpl1_dtype k_dtype,
                             const gpl1_params* prm, gpl1_result* res_dev);
gpl1_status gpl1_solve_batched_async(gpl1_ctx* ctx, const gpl1_problem* probs, int count,
                                     gpl1_dtype k_dtype, const gpl1_params* prm, gpl1_result* res_dev);

/* Tensor-core product used by the shared-K form of the method (many
 * right-hand sides on one K turn K^T r and K d into matrix products):
 *   out[n * ldo + m] = scale * sum_{k < Kd} A[m * lda + (k mod Ka)] * B[n * ldb + k]
 * for 0 <= m < M, 0 <= n < N.  A (M x Ka) and B (N x Kd) are bfloat16 (raw
 * 16-bit patterns), row-major with K contiguous; the products accumulate in
 * FP32 on the tcgen05 tensor cores.  Ka and Kd are positive multiples of 64
 * (a B longer than A along K multiplies A repeatedly: B = [b_hi | b_mid | b_lo]
 * against [A A A] is how an FP32 vector operand is carried in BF16 terms).
 * A, B and their row strides must be 16-byte aligned; out is FP32 (device),
 * written transposed (column n of the product is contiguous).  The call
 * synchronises the context stream. */
gpl1_status gpl1_gemm_bf16(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda,
                           const void* B, long long N, long long Kd, long long ldb, float* out,
                           long long ldo, float scale);

/* gpl1_gemm_bf16 with an explicit kernel configuration and a split of the
 * contraction.  config: 0 = 128 x 128 output tiles, 4-stage load ring (one CTA
 * per SM); 1 = 128 x 256 tiles, 4 stages; 2 = 128 x 128, 3 stages (two CTAs per
 * SM); 3 = 128 x 128, 6 stages.  splits in [1, Kd / 64]: part z sums the
 * 64-wide k-blocks [z KB / splits, (z+1) KB / splits) (KB = Kd / 64) and is
 * written, in the layout of gpl1_gemm_bf16, to out + z * split_stride (floats,
 * split_stride >= N * ldo when splits > 1); the parts add up to the product.
 * The shared-K solve uses this to fill the GPU when M x N has few tiles.
 * GPL1_ERR_INVALID_ARG for a config or split out of range. */
gpl1_status gpl1_gemm_bf16_ex(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda,
                              const void* B, long long N, long long Kd, long long ldb, float* out,
                              long long ldo, float scale, int config, int splits,
                              long long split_stride);

/* The autotuner's choices.  gpl1_solve_shared_k times every configuration and
 * admissible split of its two products on their operands the first time it
 * meets a shape, adds the cost of summing the extra partials, and keeps the
 * fastest per context.  Returns the number of tuned shapes (-1 for a NULL
 * ctx); for 0 <= index < that number it also writes shape[5] = {M, N, Kd, Ka,
 * max_splits}, the configuration, the split and the tuned time per product
 * (ms).  Any output pointer may be NULL. */
int gpl1_gemm_tuned(const gpl1_ctx* ctx, int index, long long* shape, int* config, int* splits,
                    float* ms);

/* The single-solve autotuner's choices (gpl1_params.engine AUTO / ONE_READ):
 * returns the number of tuned shapes (-1 for a NULL ctx); for 0 <= index <
 * that number it also writes shape[4] = {dtype, n, p, 0 for AUTO or 1 for
 * ONE_READ}, the engine chosen (GPL1_ENGINE_TWO_PASS, _ONE_READ_NCH2 or
 * _ONE_READ_NCH4) and its time for the tuning solve (ms).  Any output pointer
 * may be NULL. */
int gpl1_solve_tuned(const gpl1_ctx* ctx, int index, long long* shape, int* engine, float* ms);

/* The batched autotuner's choices (gpl1_params.tile AUTO): returns the number
 * of tuned batches (-1 for a NULL ctx); for 0 <= index < that number it also
 * writes key[4] = {dtype, instances, sum of n p over the instances, largest
 * n p}, the tile chosen (GPL1_TILE_*) and the time of each candidate's tuning
 * run in ms[3] (SMALL, MEDIUM, LARGE; -1 where a shape does not apply).  Any
 * output pointer may be NULL. */
int gpl1_batched_tuned(const gpl1_ctx* ctx, int index, long long* key, int* tile, float* ms);

/* Pins the choice for one product shape (shape[5] = {M, N, Kd, Ka, max_splits},
 * as listed by gpl1_gemm_tuned) in the context's cache, so that the solve uses
 * it without tuning: to reuse choices from an earlier run, or to reproduce a
 * configuration under a profiler (which distorts the tuner's timings).  The
 * tuned time of a pinned entry reads 0.  GPL1_ERR_INVALID_ARG for a config or
 * split out of range. */
gpl1_status gpl1_gemm_tuned_set(gpl1_ctx* ctx, const long long* shape, int config, int splits);

/* Solve nrhs instances of eq. 2 that share one K (GPL1_BF16, n x p, row
 * stride ldk) and differ in y and rho, with Alg. GP + SS per instance: the
 * gradients 2 K^T r and the products K d of all instances are formed as
 * tensor-core matrix products (gpl1_gemm_bf16_ex with autotuned configuration
 * and split, FP32 vectors carried as three BF16 terms), r is carried and
 * updated by lam K d (near the stop K x is summed exactly over the support of
 * x instead), the steplength, projection and line search run per instance.
 *   Y: device, nrhs rows of n floats (row stride ldy); X: device, nrhs rows of
 *   p floats (row stride ldx): x0 on entry (ignored when prm->x0_is_zero is
 *   set; projected onto its ball first if it lies outside), the solutions on
 *   exit.  rho, f_star: host arrays of nrhs doubles (f_star may be
 *   NULL; otherwise it enables GPL1_STOP_ON_REL_GAP per instance).  res: host
 *   array of nrhs results (kernel_ms = the whole solve).  n and p must be
 *   multiples of 64, n <= 4320, p <= 16800 (GPL1_ERR_UNSUPPORTED otherwise).
 *   The call synchronises the context stream. */
gpl1_status gpl1_solve_shared_k(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                const float* Y, long long ldy, const double* rho, const double* f_star,
                                float* X, long long ldx, int nrhs, const gpl1_params* prm,
                                gpl1_result* res);

/* ||K||_2^2, the largest eigenvalue of K^T K, by power iteration: `iters`
 * (1..100000) products with K^T K from a fixed start vector (signs from a
 * counter-based hash), each an HBM-bound pass of K v and K^T u.  *out (host)
 * receives the Rayleigh quotient ||K v||^2 of the last unit vector, which never
 * exceeds ||K||_2^2 and approaches it from below (1/out is then a step s a
 * little above 1/||K||^2, still inside ISTA's bound of 2/||K||^2).  K (device):
 * n x p of `dtype`, row stride ldk elements, aligned to its element size.
 * Uses the context workspace and stream; returns after the result is on the
 * host. */
gpl1_status gpl1_spectral_norm_sq(gpl1_ctx* ctx, const void* K, gpl1_dtype dtype, long long n, long long p,
                                  long long ldk, int iters, double* out);

/* Learned warm start: an unrolled, learned version of the ISTA iteration of
 * Sec. 2 (soft-thresholded Landweber steps),
 *   x^0 = 0,  x^{l+1} = S_{theta_l}(x^l + W_l (y - K x^l)),  l < layers,
 * for a batch of B right-hand sides (rows of Y, B x n, row stride ldy); its
 * output, projected onto the l1 ball, is a starting point x0 for Alg. GP.
 * K: GPL1_BF16 n x p (row stride ldk).  W: device FP32, layers x p x n (each
 * layer row-major p x n).  theta: device FP32, layers.  The products run on
 * the tensor cores in BF16 with FP32 accumulation (gpl1_gemm_bf16); n, p and
 * B must be multiples of 64.  All three calls synchronise the context stream.
 *   gpl1_lista_forward: X (device, B x p, row stride ldx) = x^layers.
 *   gpl1_lista_grad: the loss mean_b ||x^layers_b - Xt_b||^2 (host double) and
 *     its gradients dW (device FP32, like W) and dtheta (device FP32, layers);
 *     the soft threshold contributes the subgradient 1[|z| > theta].
 *   gpl1_lista_train: `steps` Adam updates (bias-corrected, beta 0.9/0.999,
 *     step numbers t0+1 ..) of W (rate lr) and theta (rate lr_theta), step s
 *     on rows (s mod (N / batch)) * batch .. + batch of (Y, Xt); adam_m,
 *     adam_v: device FP32 moments of layers*p*n + layers entries (W, then
 *     theta); losses: host array of `steps` doubles, the loss before each
 *     update. */
gpl1_status gpl1_lista_forward(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                               int layers, const float* W, const float* theta, const float* Y,
                               long long ldy, long long B, float* X, long long ldx);
gpl1_status gpl1_lista_grad(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                            int layers, const float* W, const float* theta, const float* Y, long long ldy,
                            long long B, const float* Xt, long long ldt, float* dW, float* dtheta,
                            double* loss);
gpl1_status gpl1_lista_train(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                             int layers, float* W, float* theta, float* adam_m, float* adam_v,
                             const float* Y, long long ldy, const float* Xt, long long ldt, long long N,
                             long long batch, int steps, int t0, float lr, float lr_theta,
                             double* losses);

/* The learned warm start as a product.
 *   gpl1_lista_init: the network's starting point, every layer one ISTA step
 *     of eq. 1 (Sec. 2) with step 1/L: W_l = K^T / L (device FP32, layers x p
 *     x n) with L = ||K||_2^2 from gpl1_spectral_norm_sq (`power_iters`
 *     products), theta_l = lam0 / L (device FP32, layers) with lam0 the median
 *     of the `count` >= 1 values `lambdas` (host; e.g. gpl1_result.lambda of
 *     the training solves: the lambda of the lambda-rho relation of Sec. 1);
 *     *L_out (host, may be NULL) receives L.  K as for gpl1_lista_forward.
 *   gpl1_solve_warm: nrhs instances of eq. 2 sharing the BF16 K, right-hand
 *     side b in row b of Y (device FP32, stride ldy), radius rho[b], optimal
 *     value f_star[b] (host arrays; f_star may be NULL), solution in row b of X
 *     (device FP32, stride ldx):
 *       1. x0 = the network's output (gpl1_lista_forward; any nrhs, a ragged
 *          tail of fewer than 64 rows goes through a zero-padded batch);
 *       2. Alg. GP + SS from the projection of x0 onto each ball (the shared-K
 *          form, alpha_0 by rule 1), at most warm_max_iter iterations
 *          (<= 0: prm->max_iter);
 *       3. the fallback: every instance whose warm solve did not end with
 *          GPL1_OK is solved again from x0 = 0 by gpl1_solve with prm, which
 *          thereby also judges the warm start: a network that does not help
 *          costs time, never the result.
 *     res (host, nrhs): the final result of each instance; fell_back (host,
 *     nrhs ints, may be NULL): 1 where the cold solve ran; *fallbacks (may be
 *     NULL): how many did.  prm: Alg. GP + SS only.  Uses the context
 *     workspace, a second buffer for the padded batch, and the stream; returns
 *     after the results are on the host. */
gpl1_status gpl1_lista_init(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk, int layers,
                            const double* lambdas, long long count, int power_iters, float* W, float* theta,
                            double* L_out);
gpl1_status gpl1_solve_warm(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk, int layers,
                            const float* W, const float* theta, const float* Y, long long ldy, const double* rho,
                            const double* f_star, float* X, long long ldx, int nrhs, const gpl1_params* prm,
                            int warm_max_iter, gpl1_result* res, int* fell_back, int* fallbacks);

/* ---- Solve without allocating (an addition of this library; the paper has
 * no counterpart).
 *
 * gpl1_solve_noalloc runs the same solver as gpl1_solve but needs no context
 * and allocates nothing, on the device or pinned on the host.  Its workspace
 * is one fixed array of GPL1_NOALLOC_SCRATCH_BYTES bytes built into the
 * library, one per device.  It is for callers that must not allocate at solve
 * time: code that runs under a device-memory budget fixed in advance, loops
 * with a latency bound where an allocation could stall on the driver, or
 * programs whose framework allocator owns all device memory and must not be
 * bypassed.
 *
 *  - Setup: the first call on a device, made with that device current, looks
 *    up the address of the array (which also loads the library's device code).
 *    Make that first call before any stream capture begins, e.g. at start-up.
 *  - Size limit: one instance needs about 12 p + 32 n bytes for F32 and BF16
 *    (24 p + 48 n for F64), plus about 20 KB.  A problem that needs more than
 *    GPL1_NOALLOC_SCRATCH_BYTES is rejected with GPL1_ERR_UNSUPPORTED and a
 *    message in err, before anything is enqueued.
 *  - Zero state: the call clears every part of the array that the kernel
 *    accumulates into (barrier counters, gradient and K-product buffers) before
 *    it launches, so nothing has to be zero on entry; x is cleared only when
 *    prm->x0_is_zero is set, exactly as in gpl1_solve.
 *  - Overlapping calls race: there is one array per device, so two calls that
 *    overlap on the same device (from two host threads, or on two streams)
 *    overwrite each other's workspace.  Serialise them.  Each call synchronises
 *    cuda_stream before it returns, so consecutive calls from one thread are
 *    safe.
 *  - Arguments and results as in gpl1_solve; res (host) gets kernel_ms = 0
 *    (no CUDA events are created).  cuda_stream: a cudaStream_t of the current
 *    device (0: the legacy default stream).  err: optional host buffer of
 *    err_len bytes that receives a message when the call fails. */
#define GPL1_NOALLOC_SCRATCH_BYTES (4u << 20)
gpl1_status gpl1_solve_noalloc(const gpl1_problem* prob, gpl1_dtype k_dtype, const gpl1_params* prm,
                               gpl1_result* res, void* cuda_stream, char* err, int err_len);

#ifdef __cplusplus
}
#endif
#endif
