// GPSS solver kernel: Algorithm GP (gradient projection with Armijo
// backtracking along the feasible direction) with Algorithm SS (adaptive
// alternation of the Barzilai-Borwein rules), Sec. 3, for
//     min f(x) = ||K x - y||^2   s.t.  ||x||_1 <= rho            (eq. 2).
//
// One persistent launch runs every iteration on the device.  Per iteration it
// reads K exactly twice, which is the minimum: the gradient needs K^T r and the
// line search needs K d, and d depends on the whole gradient.
//
//   pass A    g_k = 2 K^T r_k                  (TMA-streamed K, column strips)
//   --------- group barrier
//   phase P   z^T z, g^T x, ||g||_inf; Alg. SS -> alpha_k; v = x_k - alpha_k g_k
//             staged in shared memory; the projection threshold tau_k
//   pass B    [K d_k, K x_k] in one read of K (same tiles, reverse order), with
//             d_k = P(v)_j - x_j rebuilt per column, and g^T d, ||d||^2
//   --------- group barrier
//   phase L   f_k = ||K x_k - y||^2 and ||K d_k||^2; Armijo on
//             f(x + l d) = f_k + l g^T d + l^2 ||K d||^2, so every trial is
//             scalar work; x_{k+1} = x_k + l d_k; s^T s, s^T z for Alg. SS.
//
// Work split.  K is cut into units of RB rows x 256 columns (a TMA box of 15,
// 30 or 60 KiB, the tile; gpl1_params.tile picks it, the batched calls tune it);
// units are numbered strip-major and each CTA of a group owns one contiguous
// range.  Pass A walks the range forward, pass B backward, so the tail of
// pass A is still in L2 when pass B starts on it.  Partial products go to
// global buffers with fire-and-forget reductions.  Phase P and phase L are
// computed redundantly by every CTA of the group on the full vectors, with
// exact or fixed-order reductions, so all CTAs reach bit-identical scalars and
// decisions without a further barrier.
//
// GB300 issues FP64 at a small fraction of the FP32 rate and with long
// latency, so for float data the per-element work and the reductions stay on
// the FP32 and integer pipes (float pairs, exact fixed-point sums) and FP64 is
// used for the O(1) scalars of the line search and the stop test.
//
// A group is either all CTAs of the grid working on one instance (barriers
// through a global counter; the launch is cooperative, so all CTAs are
// resident) or a single CTA working through a queue of instances.
#pragma once

#include "common.cuh"
#include "project.cuh"

namespace gpl1 {

// Per-instance buffer of the pass-B products, two of them (iterations
// alternate): [(K d, K x) pairs: 2 nn values of the accumulation type]
// [K x: nn doubles].  Float data near the stop sum K x compensated into the
// FP64 array instead of the pair (r = K x - y cancels most of its digits near
// the solution); K d shrinks with d and always stays in the pair.
__host__ __device__ inline size_t kbuf_pair_bytes(long long nn, int acc_bytes) {
  return (static_cast<size_t>(nn) * 2 * acc_bytes + 255) & ~static_cast<size_t>(255);
}
__host__ __device__ inline size_t kbuf_stride(long long nn, int acc_bytes) {
  return kbuf_pair_bytes(nn, acc_bytes) + ((static_cast<size_t>(nn) * 8 + 255) & ~static_cast<size_t>(255));
}

struct InstDesc {
  const void* y;        // V[n]
  void* x;              // V[p]: x0 in, solution out
  double rho;
  double f_star;        // < 0: unknown
  int n, p;
  int x0_zero;
  int pad;
  void* gbuf;           // A[3][pp], zeroed before launch
  void* kbuf;           // 2 x kbuf_stride(nn) bytes, zeroed before launch
  gpl1_result* res;     // device result slot
  const void* tmap;     // CUtensorMap of K in global memory, or null for the kernel argument
  double* trace;        // optional per-iteration record (GPL1_TRACE_COLS doubles per row)
  long long trace_cap;
  void* pbuf;           // per-CTA pass-B partials: 4 doubles per CTA of the group
};

struct SolveParams {
  double beta, theta, alpha_min, alpha_max, tau1, tol;
  int M, M_alpha, stop_rule, max_iter, max_backtracks, alpha0_rule, debug;
  long long timeout_ns;
  int method, method_pad;   // GPL1_METHOD_* (the one-read kernel; the others run GPSS only)
  double lam_pen, step;     // ISTA / FISTA: lambda of eq. 1 and the step s
};

struct KArgs {
  const InstDesc* desc;
  int count;            // instances
  int group;            // CTAs per instance: gridDim.x (one instance) or 1 (queue)
  unsigned* queue;      // next instance (group == 1)
  unsigned* bar;        // group barrier counter (group > 1)
  int* err;             // sticky error flag of the launch (group > 1)
  SolveParams prm;
};

enum { CTL_STOP = 0, CTL_DONE = 1, CTL_ISSUED = 2, CTL_INST = 3, CTL_ERR = 4, CTL_BROKEN = 5, CTL_SITE = 6 };

// Where a bounded wait gave up (gpl1_result.fail_site).
enum { kSiteNone = 0, kSitePassA = 1, kSitePassB = 2, kSiteDrain = 3, kSiteGroup = 4, kSiteProducer = 5 };

// Bound on waits for TMA copies that are already in flight (drain, quiesce).
constexpr uint64_t kInflightNs = 2000000000ull;
// Pass B sums K x with compensated arithmetic once the distance to the
// requested stop is below this many times the tolerance (FP32 sums of K x
// carry about 1e-7 relative noise into f).
constexpr double kAccGapFactor = 100.0;
// ... and, whatever the stop rule, once an iteration decreases f by less than
// this fraction of f.
constexpr double kAccDecrease = 1e-5;

// SolveParams.debug bit: the group barrier waits for one arrival more than the
// group has, so every wait runs out.  Exercises the bounded-wait error path.
constexpr int kDebugUnreachableBarrier = 1;

// Columns per consumer thread held during phase P: p <= VMAX * kConsumers.
template <int DT> struct VMaxOf { static constexpr int value = 35; };    // p <= 16800
template <> struct VMaxOf<GPL1_F64> { static constexpr int value = 8; };   // p <= 3840

// Scalar state of Alg. GP + SS, identical in every thread of a group.
// State of Algorithm SS in the arithmetic of the path (FP32 for float data,
// FP64 for FP64 data): the steplength is a heuristic choice in
// [alpha_min, alpha_max] (Sec. 3), so float data need no FP64 here.
template <typename U>
struct SSState {
  U tau_ss, ss_prev, sz_prev;
  U a2win[kMaxMalpha];
  int a2cnt;
};

struct Uni {
  double alpha, tau, lam, f_cur, gd, dd, gmax;
  double gap_den;   // denominator of the relative-gap stop: max(f*, tol ||y||^2)
  // x_k as stored times this factor is the iterate: 1, or slightly below 1 when
  // rounding in the update x + lam d left ||x||_1 above rho (the iterate must
  // stay in the ball for d to be a descent direction)
  double xscale_d;
  float xscale_f;
  int acc_kx;       // pass B sums K x with compensated arithmetic (near the stop)
  int kmode[2];     // acc_kx of the pass B that filled each pass-B buffer
  SSState<float> ssf;
  SSState<double> ssd;
  float ah, al, th, tl, lf;   // alpha, tau as float pairs and lam as float, for the FP32 pipe
  float vbound;               // bound on |x - alpha g| (rho + alpha ||g||_inf: x is feasible)
  float gmaxf, ddf, kb2f;
  F2 rho_p;                   // rho as a float pair
  double fhist[kMaxM];
  int stop, iters, backtracks, inside, status, done;
  unsigned long long ts[9];   // phase-end timestamps of the current iteration (trace only)
  int psteps;                 // threshold-search steps of the current iteration (trace only)
  long long tt[8];
  // g^T x for the certificate: a float pair (float data) or a double
  union GX {
    F2 f;
    double d;
  } gx_u;
  __device__ void set_gx(const F2& v) { gx_u.f = v; }
  __device__ void set_gx(double v) { gx_u.d = v; }
};

template <int DT, int TL>
struct alignas(128) SolverSmem {
  static constexpr int kStages = Tile<DT, TL>::STAGES;
  uint8_t stage[kStages][Tile<DT, TL>::BOX];
  union {
    typename Traits<DT>::A red[kConsumerWarps][kBoxCols];
    ProjSmem proj;
  } u;
  // phase P: x_k, then v = x_k - alpha_k g_k; element e of thread t is
  // column t + e * kConsumers.
  typename Traits<DT>::V xs[VMaxOf<DT>::value * kConsumers];
  Scratch sc;
  Uni uni;
  uint64_t full[kStages];
  uint64_t empty[kStages];
  int ctl[8];
};

// Element accessor over the staged vector in shared memory (element e of this
// thread is column threadIdx.x + e * kConsumers).
template <typename V, int N>
struct SmemAcc {
  static constexpr int ne = N;
  const V* xs;
  int neu;
  __device__ V get(int e) const { return xs[e * kConsumers + threadIdx.x]; }
};

// d_j = P(x - alpha g)_j - x_j without forming P(.) first.  With v = x - alpha g:
//   inside the ball (tau = 0):  d = -alpha g
//   |v| <= tau (inactive):      d = -x
//   |v| >  tau (active):        d = -(alpha g + tau sgn v)
// The active form never subtracts x from a number of the same size, so d keeps
// its relative accuracy when it is small next to x (near convergence).  alpha
// and tau are carried as (hi, lo) pairs so the float path loses nothing to
// their rounding; the FP64 path uses doubles throughout.
struct Dir {
  double alpha, tau;
  float ah, al, th, tl;
  int inside;
  __device__ Dir(const Uni& u)
      : alpha(u.alpha), tau(u.tau), ah(u.ah), al(u.al), th(u.th), tl(u.tl), inside(u.inside) {}
  __device__ Dir(double t, float h, float l, int in) : alpha(0.0), tau(t), ah(0.f), al(0.f), th(h), tl(l), inside(in) {}
  __device__ __forceinline__ float d(float x, float g) const {
    const float v = fmaf(-ah, g, x);
    if (inside) return -fmaf(ah, g, al * g);
    if (!((fabsf(v) - th) > tl)) return -x;   // |v| <= tau, decided exactly (see TauPair)
    const float s = v > 0.f ? 1.f : -1.f;
    // alpha g + tau s with the product split exactly: p + e = ah * g
    const float p = __fmul_rn(ah, g);
    const float e = fmaf(ah, g, -p);
    const F2 q = two_sum(p, th * s);
    return -(q.hi + (q.lo + (e + fmaf(al, g, tl * s))));
  }
  __device__ __forceinline__ double d(double x, double g) const {
    const double v = fma(-alpha, g, x);
    if (inside) return -alpha * g;
    if (fabs(v) <= tau) return -x;
    return -fma(alpha, g, v > 0.0 ? tau : -tau);
  }
  // soft threshold S_tau(x) (the projection once tau is known)
  __device__ __forceinline__ float proj(float x) const {
    if (inside) return x;
    const float a = fabsf(x);
    return ((a - th) > tl) ? copysignf((a - th) - tl, x) : 0.f;
  }
  __device__ __forceinline__ double proj(double x) const {
    return inside ? x : copysign(fmax(fabs(x) - tau, 0.0), x);
  }
};

// ------------------------------------------------------------ producer
template <int DT, int TL>
__device__ void producer_run(const InstDesc& D, const void* tmap, SolverSmem<DT, TL>& sm, uint32_t& it,
                             int cta, int G, long long timeout_ns) {
  constexpr int RB = Tile<DT, TL>::RB, kStages = Tile<DT, TL>::STAGES, kBoxBytes = Tile<DT, TL>::BOX;
  const int NB = (D.n + RB - 1) / RB, TC = (D.p + kBoxCols - 1) / kBoxCols;
  const long long U = static_cast<long long>(NB) * TC;
  const int u0 = static_cast<int>(U * cta / G), u1 = static_cast<int>(U * (cta + 1) / G);
  volatile int* ctl = sm.ctl;
  if (u1 <= u0) goto done;
  for (int ph = D.x0_zero ? 1 : 0;; ++ph) {
    const bool fwd = (ph & 1) != 0;   // odd phases are pass A (forward), even ones pass B
    for (int q = 0; q < u1 - u0; ++q) {
      const int u = fwd ? u0 + q : u1 - 1 - q;
      const int st = static_cast<int>(it % kStages);
      const uint32_t par = ((it / kStages) & 1u) ^ 1u;
      uint64_t t0 = 0;
      while (!mbar_try_wait(&sm.empty[st], par)) {
        if (ctl[CTL_STOP]) goto done;
        const uint64_t t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > static_cast<uint64_t>(timeout_ns)) {
          if (!ctl[CTL_ERR]) ctl[CTL_SITE] = kSiteProducer;
          ctl[CTL_ERR] = GPL1_ERR_TIMEOUT;
          goto done;
        }
      }
      if (ctl[CTL_STOP]) goto done;
      mbar_arrive_expect_tx(&sm.full[st], kBoxBytes);
      tma_load_2d(sm.stage[st], tmap, &sm.full[st], (u / NB) * kBoxCols, (u % NB) * RB);
      ++it;
      ctl[CTL_ISSUED] = static_cast<int>(it);
    }
  }
done:
  __threadfence_block();
  ctl[CTL_DONE] = 1;
}

// ------------------------------------------------------------ consumers
template <int DT, int TL>
struct Consumer {
  using T = Traits<DT>;
  static constexpr int kStages = Tile<DT, TL>::STAGES;
  using A = typename T::A;
  using V = typename T::V;
  using S = typename std::conditional<DT == GPL1_F64, double, F2>::type;   // reduction type
  using LC = LaneCols<DT>;
  static constexpr int RB = Tile<DT, TL>::RB;          // rows of a box
  static constexpr int RPW = Tile<DT, TL>::RPW;        // rows of a box per warp
  static constexpr int VMAX = VMaxOf<DT>::value;      // p <= VMAX * kConsumers
  static constexpr bool kF64 = DT == GPL1_F64;

  const KArgs& a;
  const InstDesc& D;
  SolverSmem<DT, TL>& sm;
  uint32_t& it;
  unsigned& epoch;
  const int cta, G, tid, lane, warp, n, p, NB, TC, u0, u1, pp, nn;
  A* gbuf;
  uint8_t* kbuf;
  const V* y;
  V* x;
  int status = GPL1_OK;

  __device__ Consumer(const KArgs& a_, const InstDesc& D_, SolverSmem<DT, TL>& sm_, uint32_t& it_,
                      unsigned& ep_, int cta_, int G_)
      : a(a_), D(D_), sm(sm_), it(it_), epoch(ep_), cta(cta_), G(G_), tid(threadIdx.x), lane(threadIdx.x & 31),
        warp(threadIdx.x >> 5), n(D_.n), p(D_.p), NB((D_.n + RB - 1) / RB),
        TC((D_.p + kBoxCols - 1) / kBoxCols),
        u0(static_cast<int>(static_cast<long long>(NB) * TC * cta_ / G_)),
        u1(static_cast<int>(static_cast<long long>(NB) * TC * (cta_ + 1) / G_)),
        pp(TC * kBoxCols), nn(NB * RB), gbuf(static_cast<A*>(D_.gbuf)), kbuf(static_cast<uint8_t*>(D_.kbuf)),
        y(static_cast<const V*>(D_.y)), x(static_cast<V*>(D_.x)) {}

  __device__ A xscale() const {
    if constexpr (kF64) return sm.uni.xscale_d;
    else return sm.uni.xscale_f;
  }
  __device__ A* kp_of(int b) const { return reinterpret_cast<A*>(kbuf + b * kbuf_stride(nn, sizeof(A))); }
  __device__ double* kx_of(int b) const {
    return reinterpret_cast<double*>(kbuf + b * kbuf_stride(nn, sizeof(A)) + kbuf_pair_bytes(nn, sizeof(A)));
  }
  // r_i = (K x)_i - y_i from buffer b, in the working type (FP64 for the
  // compensated form, whose K x is in the FP64 array)
  template <bool COMP>
  __device__ A resid(const A* kp, const double* kx64, int i) const {
    if constexpr (kF64 || !COMP) return kp[2 * i + 1] - static_cast<A>(y[i]);
    else return static_cast<float>(kx64[i] - static_cast<double>(y[i]));
  }

  __device__ static S s_of(A v) {
    if constexpr (kF64) return v;
    else return F2{v, 0.f};
  }
  // acc + a*b; for float data the product is exact and the sum compensated
  __device__ static void s_fma(S& acc, A a, A b) {
    if constexpr (kF64) acc = fma(a, b, acc);
    else acc = f2_fma(acc, a, b);
  }

  // ---- pipeline
  // Wait for the box of stage `it`.  nullptr if the wait ran out or the CTA
  // has already failed (its error flag is then set; the caller skips the box
  // and does not release it).  The decision is the same for the whole warp:
  // lane 0 polls, broadcasts the outcome, and on success every lane takes the
  // (already complete) barrier phase for itself, which orders its reads of the
  // box after the TMA writes.
  __device__ const uint8_t* wait_full(uint64_t limit_ns, int site) {
    const int st = static_cast<int>(it % kStages);
    const uint32_t par = (it / kStages) & 1u;
    int ok = 1;
    if (lane == 0) {
      volatile int* ctl = sm.ctl;
      if (ctl[CTL_ERR] && site != kSiteDrain) {
        ok = 0;
      } else if (!mbar_try_wait(&sm.full[st], par)) {
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&sm.full[st], par)) {
          if (globaltimer() - t0 > limit_ns || (site != kSiteDrain && ctl[CTL_ERR])) {
            ok = 0;
            break;
          }
        }
      }
      if (!ok && !ctl[CTL_ERR]) {
        ctl[CTL_ERR] = GPL1_ERR_TIMEOUT;
        ctl[CTL_SITE] = site;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return nullptr;
    // the phase is complete and cannot advance before this warp releases the
    // stage, so this returns at once; the bound only keeps every spin finite
    for (int spin = 0; spin < (1 << 20) && !mbar_try_wait(&sm.full[st], par); ++spin) {
    }
    return sm.stage[st];
  }
  __device__ const uint8_t* wait_full(int site) { return wait_full(static_cast<uint64_t>(a.prm.timeout_ns), site); }
  __device__ void release() {
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[it % kStages]);
    ++it;
  }
  __device__ void skip() { ++it; }

  // Stop the producer and consume (without computing) every box it issued.
  // Boxes already in flight always land within microseconds, so these waits
  // use a fixed bound of their own, independent of the caller's timeout.
  __device__ void drain() {
    volatile int* ctl = sm.ctl;
    if (tid == 0) ctl[CTL_STOP] = 1;
    const uint64_t t0 = globaltimer();
    while (!ctl[CTL_DONE]) {
      if (globaltimer() - t0 > kInflightNs) {
        ctl[CTL_ERR] = GPL1_ERR_TIMEOUT;
        break;
      }
    }
    __threadfence_block();
    const uint32_t issued = static_cast<uint32_t>(ctl[CTL_ISSUED]);
    while (it < issued) {
      if (wait_full(kInflightNs, kSiteDrain)) release();
      else skip();
    }
    consumer_sync();
    // After an error some boxes may have been skipped: before the CTA moves on,
    // make sure the last box issued into every stage has landed.
    if (tid == 0 && ctl[CTL_ERR]) {
      for (uint32_t s = 0; s < kStages && s < issued; ++s) {
        const uint32_t last = issued - 1 - ((issued - 1 - s) % kStages);   // last index == s mod kStages
        const uint32_t par = (last / kStages) & 1u;
        const uint64_t t1 = globaltimer();
        while (!mbar_try_wait(&sm.full[s], par))
          if (globaltimer() - t1 > kInflightNs) break;
      }
    }
    consumer_sync();
  }

  // ---- group barrier.  Also folds in the CTA's own error flag (set by a
  // bounded wait that ran out), read once by thread 0 and broadcast, so all
  // consumer threads take the same branch.  Returns false once the launch has
  // failed.
  __device__ bool group_sync() {
    consumer_sync();
    if (tid == 0) {
      int e = reinterpret_cast<volatile int*>(sm.ctl)[CTL_ERR];
      if (G > 1) {
        if (e) atomicCAS(a.err, 0, e);
        ++epoch;
        __threadfence();
        red_release_add(a.bar, 1u);
        const unsigned target =
            epoch * static_cast<unsigned>(G) + ((a.prm.debug & kDebugUnreachableBarrier) ? 1u : 0u);
        // poll with relaxed loads (one round trip each; the fence after the
        // loop orders what follows); the error flag and the clock every 16th
        const uint64_t t0 = globaltimer();
        for (unsigned poll = 0; ld_relaxed(a.bar) < target; ++poll) {
          if ((poll & 15u) != 15u) continue;
          if (ld_volatile(a.err)) break;
          if (globaltimer() - t0 > static_cast<uint64_t>(a.prm.timeout_ns)) {
            atomicCAS(a.err, 0, GPL1_ERR_TIMEOUT);
            if (!sm.ctl[CTL_SITE]) sm.ctl[CTL_SITE] = kSiteGroup;
            break;
          }
        }
        __threadfence();
        e = ld_volatile(a.err);
      }
      sm.sc.flags[0] = e;
    }
    consumer_sync();
    const int e = sm.sc.flags[0];
    consumer_sync();
    if (e) status = e;
    return e == 0;
  }

  // ---- pass A: gout[j] += 2 sum_i K_ij r_i with r = Kx_prev - y + lam_prev Kd_prev
  __device__ void flush_a(int s, A (&acc)[8], A* gout) {
#pragma unroll
    for (int e = 0; e < 8; ++e) sm.u.red[warp][LC::col(lane, e)] = acc[e];
    consumer_sync();
    for (int c = tid; c < kBoxCols; c += kConsumers) {
      A v = 0;
#pragma unroll
      for (int w = 0; w < kConsumerWarps; ++w) v += sm.u.red[w][c];
      const int col = s * kBoxCols + c;
      if (col < p) atomicAdd(gout + col, v);
    }
    consumer_sync();
  }

  template <bool COMP>
  __device__ void pass_a(const A* kp, const double* kx64, A lp, A* gout) {
    A acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0;
    int cur = -1;
    for (int u = u0; u < u1; ++u) {
      const int s = u / NB, b = u % NB;
      if (s != cur) {
        if (cur >= 0) {
          flush_a(cur, acc, gout);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] = 0;
        }
        cur = s;
      }
      A rv = 0;
      if (lane < RPW) {
        const int i = b * RB + warp + kConsumerWarps * lane;
        if (i < n) rv = 2 * (resid<COMP>(kp, kx64, i) + lp * kp[2 * i]);
      }
      const uint8_t* st = wait_full(kSitePassA);
      if (!st) {
        skip();
        continue;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const A r = __shfl_sync(0xffffffffu, rv, q);
        A kv[8];
        load_row8<DT>(st + (warp + kConsumerWarps * q) * (kBoxCols * T::ES), lane, kv);
        if constexpr (!kF64) {
          // two columns per instruction (packed FP32 FMA; each half is the
          // same rounded fma as the scalar form)
          const float2 r2 = make_float2(r, r);
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            const float2 a2 = __ffma2_rn(make_float2(kv[e], kv[e + 1]), r2, make_float2(acc[e], acc[e + 1]));
            acc[e] = a2.x;
            acc[e + 1] = a2.y;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] = vfma(kv[e], r, acc[e]);
        }
      }
      release();
    }
    if (cur >= 0) flush_a(cur, acc, gout);
  }

  // ---- pass B: kd[i] += (K d)_i, kx[i] += (K x)_i, with
  // d_j = P(x - alpha g)_j - x_j rebuilt per strip from x, g (no d vector in
  // memory).  The CTA that owns row box 0 of a strip also accumulates
  // g^T d, ||d||^2 and "d != 0" over the strip's columns (each column counted
  // once in the group) and publishes its totals in part[cta].
  // setup (gk == null): d = 0 and x = S_tau(x_mem) (the projected x0).
  // (K x)_i is summed without rounding error on float data: each product
  // K_ij x_j is split exactly into a float pair (FMA), the lane's terms and
  // the warp's lanes are added with error-free two-sums, and the pair is
  // added to the FP64 total in global memory.
  template <bool ACC>
  __device__ void pass_b(const A* gk, const Dir& dir, A* kp, double* kx64, double* part) {
    A dv[8], xv[8];
    // g^T d is a sum of terms of both signs whose total goes to 0 as the
    // iteration converges, while the Armijo test needs its sign right: it is
    // accumulated compensated.  ||d||^2 has terms of one sign only.
    S sgd{};
    A sdd = 0;
    const A xsc = gk ? xscale() : A(1);
    constexpr bool acc = ACC;
    unsigned snz = 0;
    int cur = -1;
    for (int u = u1 - 1; u >= u0; --u) {
      const int s = u / NB, b = u % NB;
      if (s != cur) {
        cur = s;
        // every warp rebuilds the same columns (warps split the rows): warp 0 counts them
        const bool owns = gk && s * NB >= u0 && warp == 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int col = s * kBoxCols + LC::col(lane, e);
          A xj = 0, dj = 0;
          if (col < p) {
            xj = static_cast<A>(x[col]) * xsc;
            if (gk) {
              const A gj = gk[col];
              dj = dir.d(xj, gj);
              if (owns) {
                s_fma(sgd, gj, dj);
                sdd = vfma(dj, dj, sdd);
                snz |= dj != A(0) ? 1u : 0u;
              }
            } else {
              xj = dir.proj(xj);
            }
          }
          dv[e] = dj;
          xv[e] = xj;
        }
      }
      const uint8_t* st = wait_full(kSitePassB);
      if (!st) {
        skip();
        continue;
      }
      if constexpr (!kF64 && !acc) {
        // far from the stop, plain FP32 sums: the warp's RPW rows x (K d, K x)
        // reduced together (warp_sum_many), then one v2 add per row
        float vals[2 * RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          A kv[8];
          load_row8<DT>(st + (warp + kConsumerWarps * q) * (kBoxCols * T::ES), lane, kv);
          // even and odd columns in the two halves of packed FP32 FMAs
          float2 pd = make_float2(0.f, 0.f), sh = make_float2(0.f, 0.f);
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            const float2 k2 = make_float2(kv[e], kv[e + 1]);
            pd = __ffma2_rn(k2, make_float2(dv[e], dv[e + 1]), pd);
            sh = __ffma2_rn(k2, make_float2(xv[e], xv[e + 1]), sh);
          }
          vals[2 * q] = pd.x + pd.y;
          vals[2 * q + 1] = sh.x + sh.y;
        }
        const float tot = warp_sum_many<2 * RPW>(vals, lane);   // lane q * GL holds value q
        constexpr int GL = 32 / (2 * RPW);
        const float kx_tot = __shfl_down_sync(0xffffffffu, tot, GL);
        if (lane % (2 * GL) == 0) {
          const int i = b * RB + warp + kConsumerWarps * (lane / (2 * GL));
          if (i < n) red_add2(kp + 2 * i, tot, kx_tot);
        }
        release();
        continue;
      }
      if constexpr (!kF64 && acc) {
        // near the stop, K x without rounding error: the rows' (K d, K x) reduced
        // together as above, K x as exact float pairs (warp_sum_many_f2)
        float vd[RPW];
        F2 vx[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
          A kv[8];
          load_row8<DT>(st + (warp + kConsumerWarps * q) * (kBoxCols * T::ES), lane, kv);
          float pd = 0.f, sh = 0.f, sl = 0.f;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            pd = fmaf(kv[e], dv[e], pd);
            const float pr = __fmul_rn(kv[e], xv[e]);
            const float pe = fmaf(kv[e], xv[e], -pr);   // K_ij x_j - pr, exact
            const F2 t = two_sum(sh, pr);
            sh = t.hi;
            sl = __fadd_rn(sl, __fadd_rn(pe, t.lo));
          }
          vd[q] = pd;
          vx[q] = F2{sh, sl};
        }
        const float dtot = warp_sum_many<RPW>(vd, lane);       // lane q * GL holds row q
        const F2 xtot = warp_sum_many_f2<RPW>(vx, lane);
        constexpr int GL = 32 / RPW;
        if (lane % GL == 0) {
          const int i = b * RB + warp + kConsumerWarps * (lane / GL);
          if (i < n) {
            red_add(kp + 2 * i, dtot);
            red_add(kx64 + i, static_cast<double>(xtot.hi) + static_cast<double>(xtot.lo));
          }
        }
        release();
        continue;
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        A kv[8];
        load_row8<DT>(st + (warp + kConsumerWarps * q) * (kBoxCols * T::ES), lane, kv);
        const int i = b * RB + warp + kConsumerWarps * q;
        A pd = 0;
        if constexpr (kF64) {
          double px = 0;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            pd = fma(kv[e], dv[e], pd);
            px = fma(kv[e], xv[e], px);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            pd += __shfl_xor_sync(0xffffffffu, pd, o);
            px += __shfl_xor_sync(0xffffffffu, px, o);
          }
          if (lane == 0 && i < n) red_add2(kp + 2 * i, pd, px);
        } else {
          float sh = 0.f, sl = 0.f;   // (K x) partial as an unevaluated pair
          if constexpr (acc) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              pd = fmaf(kv[e], dv[e], pd);
              const float pr = __fmul_rn(kv[e], xv[e]);
              const float pe = fmaf(kv[e], xv[e], -pr);   // K_ij x_j - pr, exact
              const F2 t = two_sum(sh, pr);
              sh = t.hi;
              sl = __fadd_rn(sl, __fadd_rn(pe, t.lo));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              pd += __shfl_xor_sync(0xffffffffu, pd, o);
              const float oh = __shfl_xor_sync(0xffffffffu, sh, o);
              const float ol = __shfl_xor_sync(0xffffffffu, sl, o);
              const F2 t = two_sum(sh, oh);
              sh = t.hi;
              sl = __fadd_rn(__fadd_rn(sl, ol), t.lo);
            }
          } else {   // far from the stop: plain FP32 sums
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              pd = fmaf(kv[e], dv[e], pd);
              sh = fmaf(kv[e], xv[e], sh);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              pd += __shfl_xor_sync(0xffffffffu, pd, o);
              sh += __shfl_xor_sync(0xffffffffu, sh, o);
            }
          }
          if (lane == 0 && i < n) {
            if constexpr (acc) {
              red_add(kp + 2 * i, pd);
              red_add(kx64 + i, static_cast<double>(sh) + static_cast<double>(sl));
            } else {
              red_add2(kp + 2 * i, pd, sh);
            }
          }
        }
      }
      release();
    }
    if (part) {
      S v[2] = {sgd, s_of(sdd)};
      lead_reduce<2>(v, snz, sm.sc);
      if (tid == 0) {
        double* o = part + 4 * cta;
        if constexpr (kF64) {
          o[0] = v[0];
          o[1] = v[1];
        } else {
          reinterpret_cast<float*>(o)[0] = v[0].hi;
          reinterpret_cast<float*>(o)[1] = v[0].lo;
          reinterpret_cast<float*>(o)[2] = v[1].hi;
          reinterpret_cast<float*>(o)[3] = v[1].lo;
        }
        o[2] = static_cast<double>(snz);   // FP64 data only reads it as a flag; stored as 0/1
        reinterpret_cast<unsigned*>(o)[6] = snz;
      }
    }
  }

  // Sum of the group's pass-B partials in CTA order (warp 0; lane 0 gets it).
  __device__ void reduce_parts(const double* part, S& gd, S& dd, unsigned& nz) {
    gd = S{};
    dd = S{};
    nz = 0;
    for (int c = lane; c < G; c += 32) {
      const double* o = part + 4 * c;
      if constexpr (kF64) {
        gd += o[0];
        dd += o[1];
      } else {
        const float* f = reinterpret_cast<const float*>(o);
        gd = f2_add(gd, F2{f[0], f[1]});
        dd = f2_add(dd, F2{f[2], f[3]});
      }
      nz |= reinterpret_cast<const unsigned*>(o)[6];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      if constexpr (kF64) {
        gd += __shfl_xor_sync(0xffffffffu, gd, off);
        dd += __shfl_xor_sync(0xffffffffu, dd, off);
      } else {
        gd = f2_add(gd, F2{__shfl_xor_sync(0xffffffffu, gd.hi, off), __shfl_xor_sync(0xffffffffu, gd.lo, off)});
        dd = f2_add(dd, F2{__shfl_xor_sync(0xffffffffu, dd.hi, off), __shfl_xor_sync(0xffffffffu, dd.lo, off)});
      }
      nz |= __shfl_xor_sync(0xffffffffu, nz, off);
    }
  }

  // ---- phase L scalars: f = ||Kx - y||^2, a = r^T Kd, b = ||Kd||^2 (r = Kx - y),
  // summed into thread 0 (lead_reduce).
  template <bool COMP>
  __device__ void line_scalars(const A* kp, const double* kx64, S (&o)[3]) {
    if constexpr (kF64) {
      double v[3] = {0, 0, 0};
      for (int i = tid; i < n; i += kConsumers) {
        const double kd = kp[2 * i], r = kp[2 * i + 1] - y[i];
        v[0] = fma(r, r, v[0]);
        v[1] = fma(r, kd, v[1]);
        v[2] = fma(kd, kd, v[2]);
      }
      o[0] = v[0];
      o[1] = v[1];
      o[2] = v[2];
    } else {
      F2 v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      for (int i = tid; i < n; i += kConsumers) {
        const float kd = kp[2 * i];
        F2 r;
        if constexpr (COMP) {   // r_i in FP64, then as a float pair
          const double rd = kx64[i] - static_cast<double>(y[i]);
          const float rh = static_cast<float>(rd);
          r = F2{rh, static_cast<float>(rd - static_cast<double>(rh))};
        } else {
          r = two_sum(kp[2 * i + 1], -static_cast<float>(y[i]));
        }
        v[0] = f2_fma(v[0], r.hi, r.hi + 2.f * r.lo);
        v[1] = f2_fma(v[1], r.hi + r.lo, kd);
        v[2] = f2_fma(v[2], kd, kd);
      }
      o[0] = v[0];
      o[1] = v[1];
      o[2] = v[2];
    }
    unsigned dummy = 0;
    lead_reduce<3>(o, dummy, sm.sc);
  }

  __device__ void zero_slices(A* gz, int kb) {
    const int j0 = static_cast<int>(static_cast<long long>(pp) * cta / G);
    const int j1 = static_cast<int>(static_cast<long long>(pp) * (cta + 1) / G);
    for (int j = j0 + tid; j < j1; j += kConsumers) gz[j] = 0;
    A* const kz = kp_of(kb);
    double* const xz = kx_of(kb);
    const int i0 = static_cast<int>(static_cast<long long>(nn) * cta / G);
    const int i1 = static_cast<int>(static_cast<long long>(nn) * (cta + 1) / G);
    for (int i = i0 + tid; i < i1; i += kConsumers) {
      kz[2 * i] = 0;
      kz[2 * i + 1] = 0;
      xz[i] = 0.0;
    }
  }

  // Phase P's pass over x_k and g_k: z^T z (z = g_k - g_{k-1}), g^T x, max |g|
  // into the first two sums and mx; stores x_k into shared memory.  Near the
  // stop (L1) also ||x_k||_1, compensated, for the feasibility check.
  template <bool L1>
  __device__ void phase_p_sums(const A* gk, const A* gprev, int k, int neu, S (&red)[3], unsigned& mx, A& pm) {
    V* const xs = sm.xs;
    A part2[2] = {0, 0};
    pm = 0;
    S l1{};
    constexpr int CH = 7;   // loads of a chunk are issued together, then stored
#pragma unroll
    for (int c0 = 0; c0 < VMAX; c0 += CH) {
      A gv[CH], gp[CH];
      V xv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i, j = tid + e * kConsumers;
        const bool ok = e < VMAX && e < neu && j < p;
        gv[i] = ok ? gk[j] : A(0);
        xv[i] = ok ? x[j] : V(0);
        gp[i] = (ok && k > 0) ? gprev[j] : A(0);
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        if (e >= VMAX || e >= neu) break;
        if (k > 0) {
          const A z = gv[i] - gp[i];
          part2[0] = vfma(z, z, part2[0]);
        }
        xs[e * kConsumers + tid] = xv[i];
        part2[1] = vfma(gv[i], static_cast<A>(xv[i]), part2[1]);
        if constexpr (L1) {
          if constexpr (kF64) l1 += fabs(xv[i]);
          else l1 = f2_add(l1, fabsf(xv[i]));
        }
        pm = vmax(pm, vabs(gv[i]));
      }
    }
    red[0] = s_of(part2[0]);
    red[1] = s_of(part2[1]);
    red[2] = l1;
    mx = kF64 ? __float_as_uint(static_cast<float>(pm) * 1.0000002f) : __float_as_uint(static_cast<float>(pm));
  }

  // Float data near the stop: tau again, on the active set A the search found
  // (|v| > tau), from x and g themselves rather than from v = x - alpha g as
  // rounded into shared memory.  With s = sgn v, the direction of pass B gives
  // h = x + d with sum_A |h_j| = sum_A s_j x_j - alpha sum_A s_j g_j - |A| tau,
  // so this tau makes ||h||_1 = rho to float-pair accuracy.  The rounding of v
  // (half an ulp of each |v_j|) would otherwise leave ||h||_1 - rho of the
  // order of the decrease the Armijo test has to see near the solution.
  __device__ void refine_tau(const A* gk, int neu, float& th, float& tl) {
    const V* const xs = sm.xs;
    const TauPair tp{th, tl};
    const A xsc = xscale();
    S v[3] = {S{}, S{}, S{}};
#pragma unroll 4
    for (int e = 0; e < VMAX; ++e) {
      if (e >= neu) break;
      const int j = tid + e * kConsumers;
      const float vv = xs[e * kConsumers + tid];
      if (j < p && !tp.below(fabsf(vv))) {
        const float sg = vv > 0.f ? 1.f : -1.f;
        v[0] = f2_add(v[0], sg * (static_cast<A>(x[j]) * xsc));
        v[1] = f2_add(v[1], sg * gk[j]);
        v[2] = f2_add(v[2], 1.f);
      }
    }
    unsigned dummy = 0;
    lead_reduce<3>(v, dummy, sm.sc);
    if (tid == 0) {
      const Uni& u = sm.uni;
      const F2 sx = v[0], sgs = v[1];
      const float c = v[2].hi;   // |A| (an integer below 2^24: exact)
      // alpha * S_g with alpha = ah + al, the leading product split exactly
      const float ph = __fmul_rn(u.ah, sgs.hi);
      const float pl = fmaf(u.ah, sgs.hi, -ph) + fmaf(u.ah, sgs.lo, u.al * sgs.hi);
      F2 t = f2_add(sx, F2{-ph, -pl});
      t = f2_add(t, F2{-u.rho_p.hi, -u.rho_p.lo});
      // t / c as a float pair: the remainder of the leading quotient is exact
      const float q1 = __fdiv_rn(t.hi, c);
      const float rem = fmaf(-q1, c, t.hi) + t.lo;
      const F2 q = two_sum(q1, __fdiv_rn(rem, c));
      if (c > 0.f && q.hi > 0.f) {
        sm.sc.tp[2] = q.hi;
        sm.sc.tp[3] = q.lo;
      } else {   // keep the search's value
        sm.sc.tp[2] = th;
        sm.sc.tp[3] = tl;
      }
    }
    consumer_sync();
    th = sm.sc.tp[2];
    tl = sm.sc.tp[3];
    consumer_sync();
  }

  // xs := x - a g for every column this thread holds (x from shared memory
  // when from_smem, else from global; g from global, in chunks so the loads
  // of a chunk are in flight together).
  __device__ void stage_v(const A* gk, V av, bool from_smem, int neu) {
    const V xsc = static_cast<V>(xscale());
    V* const xs = sm.xs;
    constexpr int CH = 7;
#pragma unroll
    for (int c0 = 0; c0 < VMAX; c0 += CH) {
      V gv[CH], xv[CH];
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i, j = tid + e * kConsumers;
        const bool ok = e < VMAX && e < neu && j < p;
        gv[i] = ok ? static_cast<V>(gk[j]) : V(0);
        xv[i] = (ok && !from_smem) ? x[j] : V(0);
      }
#pragma unroll
      for (int i = 0; i < CH; ++i) {
        const int e = c0 + i;
        if (e >= VMAX || e >= neu) break;
        const V xe = (from_smem ? xs[e * kConsumers + tid] : xv[i]) * xsc;
        xs[e * kConsumers + tid] = vfma(-av, gv[i], xe);
      }
    }
  }

  // ---- scalar state of Alg. GP + SS.  It is the same in every thread, so it
  // lives in shared memory, is updated by consumer thread 0 between two
  // barriers, and is read by everyone after the second barrier.
  template <typename U>
  __device__ U ss_step(SSState<U>& st, U zz) {   // Algorithm SS: alpha_k for k >= 1
    const SolveParams& P = a.prm;
    const U amin_p = static_cast<U>(P.alpha_min), amax_p = static_cast<U>(P.alpha_max);
    U alpha, a2_this;
    if (st.sz_prev <= U(0)) {
      alpha = amax_p;
      a2_this = amax_p;   // alpha^(2)_k undefined: does not lower the window minimum
    } else {
      const U a1 = vmin(vmax(st.ss_prev / st.sz_prev, amin_p), amax_p);
      const U a2 = vmin(vmax(st.sz_prev / zz, amin_p), amax_p);
      a2_this = a2;
      U amin = a2;   // window j = max(1, k - M_alpha) .. k
      for (int q = 0; q < st.a2cnt && q < P.M_alpha; ++q) amin = vmin(amin, st.a2win[q]);
      if (a2 <= st.tau_ss * a1) {   // alpha^(2)/alpha^(1) <= tau_k
        alpha = amin;
        st.tau_ss *= U(0.9);
      } else {
        alpha = a1;
        st.tau_ss *= U(1.1);
      }
    }
    for (int q = P.M_alpha - 1; q > 0; --q) st.a2win[q] = st.a2win[q - 1];
    if (P.M_alpha > 0) st.a2win[0] = a2_this;
    if (st.a2cnt < P.M_alpha) ++st.a2cnt;
    return alpha;
  }

  // Feasibility of the stored x_k (lead thread).  In exact arithmetic every
  // iterate of Alg. GP lies in the ball (x_k + lam d_k with lam <= 1 is a
  // convex combination of feasible points); rounding in the update can leave
  // ||x||_1 a few ulps above rho.  The iterate is then x_k scaled back onto
  // the ball, with a factor rounded down so the scaled vector is feasible.
  __device__ void set_xscale(double l1) {   // FP64 data
    Uni& u = sm.uni;
    u.xscale_d = l1 > D.rho ? (D.rho / l1) * (1.0 - 0x1p-50) : 1.0;
  }
  __device__ void set_xscale(const F2& l1) {   // float data: float work only
    Uni& u = sm.uni;
    const F2 rp = u.rho_p;
    // l1 - rho, exact to a few ulps of rho (the high parts cancel exactly)
    const float ex = (l1.hi - rp.hi) + (l1.lo - rp.lo);
    u.xscale_f = ex > 0.f ? __fdiv_rd(rp.hi, l1.hi) * (1.f - 0x1p-21f) : 1.f;
  }

  // Publish alpha_k (lead thread): a float pair for the FP32 pipe and the bound
  // rho + alpha ||g||_inf on |x - alpha g| (x is feasible, so ||x||_inf <= rho).
  __device__ void set_alpha(double alpha) {   // FP64 data
    Uni& u = sm.uni;
    u.alpha = alpha;
    const F2 af = f2_of(alpha);
    u.ah = af.hi;
    u.al = af.lo;
    u.vbound = static_cast<float>((D.rho + alpha * u.gmax) * 1.000001);
    if (!isfinite(alpha)) {
      u.status = GPL1_ERR_NONFINITE;
      u.stop = GPL1_STOP_ERROR;
      u.done = 1;
    }
  }
  __device__ void set_alpha(float alpha) {    // float data: no FP64 work
    Uni& u = sm.uni;
    u.ah = alpha;
    u.al = 0.f;
    u.vbound = (u.rho_p.hi + alpha * u.gmaxf) * 1.00001f;
    if (!isfinite(alpha)) {
      u.status = GPL1_ERR_NONFINITE;
      u.stop = GPL1_STOP_ERROR;
      u.done = 1;
    }
  }

  // Columns c, c+1 of row k: the earliest and latest of every CTA's stamp t
  // (raw globaltimer bits in the double slots; the row starts zeroed).
  __device__ void trace_spread(int k, int c, unsigned long long t) {
    if (!D.trace || k >= D.trace_cap) return;
    unsigned long long* r = reinterpret_cast<unsigned long long*>(D.trace + static_cast<long long>(k) * GPL1_TRACE_COLS);
    atomicCAS(r + c, 0ull, ~0ull);   // the first CTA turns the "min" slot into +inf
    atomicMin(r + c, t);
    atomicMax(r + c + 1, t);
  }

  __device__ void trace_row(int k, double fk, double lam, double kb2) {
    Uni& u = sm.uni;
    if (D.trace && k < D.trace_cap && cta == 0) {
      double* t = D.trace + static_cast<long long>(k) * GPL1_TRACE_COLS;
      t[0] = fk;
      t[1] = kF64 ? u.alpha : static_cast<double>(u.ah);
      t[2] = lam;
      t[3] = kF64 ? u.ssd.tau_ss : static_cast<double>(u.ssf.tau_ss);
      t[4] = u.gd;
      t[5] = kb2;
      t[6] = u.dd;
      t[7] = kF64 ? u.tau : static_cast<double>(u.th) + static_cast<double>(u.tl);
      for (int q = 0; q < 5; ++q) t[8 + q] = static_cast<double>(u.ts[q] - u.ts[5]);
      for (int q = 6; q < 9; ++q) t[7 + q] = static_cast<double>(u.ts[q] - u.ts[5]);
      t[16] = u.psteps;
      for (int q = 1; q < 7; ++q) t[16 + q] = static_cast<double>(u.tt[q] - u.tt[0]);
      t[23] = static_cast<double>(u.tt[7]);   // candidates kept by the threshold search
    }
  }

  // Armijo backtracking (Alg. GP, Steps 4-6), in FP64, on the exact expansion
  // of the quadratic f:  f(x_k + l d) = f_k + l g_k^T d + l^2 ||K d||^2.  The
  // linear term is the product g_k^T d_k that the Armijo test itself uses; it
  // comes from the gradient and stays accurate when K d loses digits to
  // cancellation (d in small singular directions of an ill-conditioned K),
  // whereas 2 r^T K d would not.  Sets lam, f_cur and the stop state.
  __device__ void ls_step(int k, double fk, double kb2) {
    Uni& u = sm.uni;
    const SolveParams& P = a.prm;
    const double gd = u.gd, dd = u.dd;
    if (!isfinite(fk) || !isfinite(kb2) || !isfinite(gd)) {
      u.status = GPL1_ERR_NONFINITE;
      u.stop = GPL1_STOP_ERROR;
      u.iters = k;
      u.done = 1;
      return;
    }
    u.fhist[0] = fk;   // fresh f(x_k)
    double fmaxv = fk;
    for (int q = 1; q < P.M && q <= k; ++q) fmaxv = fmax(fmaxv, u.fhist[q]);
    double lam = 1.0;
    int bt = 0;
    bool ok = false;
    for (;;) {
      // f(x + lam d) - f_max = (f_k - f_max) + lam (g^T d + lam b)  vs  beta lam g^T d
      if ((fk - fmaxv) + lam * (gd + lam * kb2) <= P.beta * lam * gd) {
        ok = true;
        break;
      }
      if (bt >= P.max_backtracks) break;
      lam *= P.theta;
      ++bt;
    }
    u.backtracks += bt;
    trace_row(k, fk, ok ? lam : 0.0, kb2);
    if (!ok) {
      u.status = GPL1_ERR_LINESEARCH;
      u.stop = GPL1_STOP_ERROR;
      u.iters = k;
      u.f_cur = fk;
      u.done = 1;
      return;
    }
    const double fnext = fk + lam * (gd + lam * kb2);
    for (int q = kMaxM - 1; q > 0; --q) u.fhist[q] = u.fhist[q - 1];
    u.fhist[0] = fnext;
    u.lam = lam;
    u.lf = static_cast<float>(lam);
    // s^T s = lam^2 ||d||^2 and s^T z = s^T (2 K^T K s) = 2 lam^2 ||K d||^2 for this quadratic f
    if constexpr (kF64) {
      u.ssd.ss_prev = lam * lam * dd;
      u.ssd.sz_prev = 2.0 * lam * lam * kb2;
    } else {
      u.ssf.ss_prev = u.lf * u.lf * u.ddf;
      u.ssf.sz_prev = 2.f * u.lf * u.lf * u.kb2f;
    }
    u.f_cur = fnext;
    u.iters = k + 1;
    if ((P.stop_rule & GPL1_STOP_ON_REL_GAP) && D.f_star >= 0.0 &&
        fnext - D.f_star <= kAccGapFactor * P.tol * u.gap_den)
      u.acc_kx = 1;
    if (fk - fnext <= kAccDecrease * fk) u.acc_kx = 1;   // progress near the FP32 resolution of f
    if ((P.stop_rule & GPL1_STOP_ON_REL_GAP) && D.f_star >= 0.0 && fnext - D.f_star <= P.tol * u.gap_den) {
      u.stop = GPL1_STOP_REL_GAP;
      u.done = 1;
    } else if (u.iters >= P.max_iter) {
      u.stop = GPL1_STOP_MAX_ITER;
      u.status = GPL1_ERR_NOT_CONVERGED;
      u.done = 1;
    }
  }

  __device__ double sum_sq_y() {   // ||y||^2, into thread 0
    S v[1];
    if constexpr (kF64) {
      double t = 0.0;
      for (int i = tid; i < n; i += kConsumers) t = fma(y[i], y[i], t);
      v[0] = t;
    } else {
      F2 t = {0.f, 0.f};
      for (int i = tid; i < n; i += kConsumers) t = f2_fma(t, static_cast<float>(y[i]), static_cast<float>(y[i]));
      v[0] = t;
    }
    unsigned dummy = 0;
    lead_reduce<1>(v, dummy, sm.sc);
    return as_double(v[0]);
  }

  __device__ void run() {
    const SolveParams& P = a.prm;
    const double rho = D.rho;
    Uni& u = sm.uni;
    V* const xs = sm.xs;
    const int neu = (p + kConsumers - 1) / kConsumers;   // occupied slots per thread (uniform)
    double* const part = static_cast<double*>(D.pbuf);

    if (tid == 0) {
      u.alpha = u.tau = u.lam = 0.0;
      u.ah = u.al = u.th = u.tl = u.lf = 0.f;
      u.gd = u.dd = u.gmax = 0.0;
      u.gx_u.d = 0.0;
      u.ddf = u.kb2f = u.gmaxf = 0.f;
      u.rho_p = f2_of(rho);
      u.ssf.tau_ss = static_cast<float>(P.tau1);
      u.ssd.tau_ss = P.tau1;
      u.ssf.a2cnt = u.ssd.a2cnt = 0;
      u.ssf.ss_prev = u.ssf.sz_prev = 0.f;
      u.ssd.ss_prev = u.ssd.sz_prev = 0.0;
      u.stop = GPL1_STOP_MAX_ITER;
      u.iters = u.backtracks = 0;
      u.inside = 0;
      u.status = GPL1_OK;
      u.done = 0;
      u.psteps = 0;
      u.xscale_d = 1.0;
      u.xscale_f = 1.f;
      // with no target to approach, every pass B sums K x compensated
      u.acc_kx = (P.stop_rule & (GPL1_STOP_ON_REL_GAP | GPL1_STOP_ON_FW)) ? 0 : 1;
      u.kmode[0] = 0;
      u.kmode[1] = kF64 ? 0 : u.acc_kx;   // the setup pass B (x0 given) fills buffer 1
    }
    consumer_sync();

    // ---------------- setup: feasible x0, r0 = K x0 - y, f0
    if (!D.x0_zero) {
#pragma unroll
      for (int e = 0; e < VMAX; ++e) {
        if (e >= neu) break;
        const int j = tid + e * kConsumers;
        xs[e * kConsumers + tid] = j < p ? x[j] : V(0);
      }
      const SmemAcc<V, VMAX> acc0{xs, neu};
      const TauResult t0 = block_l1_tau_fixed_point<V>(acc0, rho, u.rho_p, 0.f, sm.u.proj, sm.sc);
      const Dir dir0(t0.tau, t0.th, t0.tl, t0.inside);
      if (u.kmode[1]) pass_b<true>(nullptr, dir0, kp_of(1), kx_of(1), nullptr);
      else pass_b<false>(nullptr, dir0, kp_of(1), kx_of(1), nullptr);
      if (!group_sync()) goto finish;
      if (!t0.inside) {   // write the projected x0 only after every CTA has read x0
        const int j0 = static_cast<int>(static_cast<long long>(p) * cta / G);
        const int j1 = static_cast<int>(static_cast<long long>(p) * (cta + 1) / G);
        for (int j = j0 + tid; j < j1; j += kConsumers) x[j] = static_cast<V>(dir0.proj(static_cast<A>(x[j])));
      }
      S o[3];
      if (u.kmode[1]) line_scalars<true>(kp_of(1), kx_of(1), o);
      else line_scalars<false>(kp_of(1), kx_of(1), o);
      if (tid == 0) u.f_cur = as_double(o[0]);
    }
    {
      // ||y||^2 = f(0).  With f* ~ 0 (an exact fit) a relative gap cannot be
      // resolved, so the gap is then measured against tol ||y||^2 instead.
      const double yy = sum_sq_y();
      if (tid == 0) {
        if (D.x0_zero) u.f_cur = yy;
        u.gap_den = fmax(D.f_star, P.tol * yy);
      }
    }
    if (tid == 0)
      for (int q = 0; q < kMaxM; ++q) u.fhist[q] = u.f_cur;
    consumer_sync();

    for (int k = 0;; ++k) {
      A* const gk = gbuf + (k % 3) * pp;
      A* const gprev = gbuf + ((k + 2) % 3) * pp;
      if (tid == 0 && D.trace) u.ts[5] = globaltimer();
      // ---------------- pass A: g_k = 2 K^T r_k
      {
        const A lp = kF64 ? static_cast<A>(u.lam) : static_cast<A>(u.lf);
        if (!kF64 && u.kmode[(k + 1) & 1]) pass_a<true>(kp_of((k + 1) & 1), kx_of((k + 1) & 1), lp, gk);
        else pass_a<false>(kp_of((k + 1) & 1), kx_of((k + 1) & 1), lp, gk);
      }
      if (tid == 0 && D.trace) {
        u.ts[0] = globaltimer();
        trace_spread(k, 24, u.ts[0]);
      }
      if (!group_sync()) break;
      if (tid == 0 && D.trace) u.ts[1] = globaltimer();

      // ---------------- phase P: z^T z, g^T x, ||g||_inf; Alg. SS; threshold
      {
        S red[3];
        unsigned mx;
        A pm;
        const bool near = u.acc_kx != 0;
        if (near) phase_p_sums<true>(gk, gprev, k, neu, red, mx, pm);
        else phase_p_sums<false>(gk, gprev, k, neu, red, mx, pm);
        lead_reduce<3>(red, mx, sm.sc);
        double gmax64 = 0.0;
        if constexpr (kF64) gmax64 = block_max_nonneg(static_cast<double>(pm), sm.sc);
        if (tid == 0 && D.trace) u.ts[6] = globaltimer();
        if (tid == 0) {
          u.gmaxf = __uint_as_float(mx);
          u.set_gx(red[1]);
          if (near) set_xscale(red[2]);
          if constexpr (kF64) u.gmax = gmax64;
          if (P.stop_rule & GPL1_STOP_ON_FW) {   // FP64 only when this rule is on
            const double gmax = kF64 ? gmax64 : static_cast<double>(u.gmaxf);
            const double fw = as_double(red[1]) + rho * gmax;
            if (fw <= kAccGapFactor * P.tol * (u.f_cur - fw)) u.acc_kx = 1;
            if (fw <= P.tol * (u.f_cur - fw)) {
              u.stop = GPL1_STOP_FW;
              u.iters = k;
              u.done = 1;
            }
          }
          u.kmode[k & 1] = u.acc_kx;   // the form of this iteration's pass B
          if (!u.done && k > 0) {
            if constexpr (kF64) set_alpha(ss_step(u.ssd, red[0]));
            else set_alpha(ss_step(u.ssf, red[0].hi + red[0].lo));
          }
          if (!u.done && k == 0) u.vbound = (u.rho_p.hi + u.gmaxf) * 1.00001f;
        }
        consumer_sync();
        if (u.done) break;
      }
      if (k == 0) {
        // alpha_0 = clamp(1 / ||P(x0 - g0)||_inf)   (rule 1: ||P(x0 - g0) - x0||_inf)
        stage_v(gk, V(1), true, neu);
        consumer_sync();
        const SmemAcc<V, VMAX> wacc{xs, neu};
        const TauResult tw = block_l1_tau_fixed_point<V>(wacc, rho, u.rho_p, 0.f, sm.u.proj, sm.sc, u.vbound);
        const Dir pw(tw.tau, tw.th, tw.tl, tw.inside);
        A m = 0;
#pragma unroll
        for (int e = 0; e < VMAX; ++e) {
          if (e >= neu) break;
          const int j = tid + e * kConsumers;
          const A h = pw.proj(static_cast<A>(wacc.get(e)));
          m = vmax(m, vabs(P.alpha0_rule == 1 ? h - (j < p ? static_cast<A>(x[j]) : A(0)) : h));
        }
        m = block_max_nonneg(m, sm.sc);
        if (tid == 0) {
          const double ninf = static_cast<double>(m);   // ||P(x0 - g0)||_inf (or of P(.) - x0)
          const double a0 = ninf > 0.0 ? fmin(fmax(1.0 / ninf, P.alpha_min), P.alpha_max) : P.alpha_max;
          if constexpr (kF64) set_alpha(a0);
          else set_alpha(static_cast<float>(a0));
        }
        consumer_sync();
        if (u.done) break;   // non-finite steplength
        stage_v(gk, kF64 ? static_cast<V>(u.alpha) : static_cast<V>(u.ah), false, neu);
      } else {
        stage_v(gk, kF64 ? static_cast<V>(u.alpha) : static_cast<V>(u.ah), true, neu);
      }
      consumer_sync();
      if (tid == 0 && D.trace) u.ts[7] = globaltimer();
      {
        // projection h = P(x - alpha g): its threshold (the direction d = h - x is formed in pass B)
        const SmemAcc<V, VMAX> vacc{xs, neu};
        const TauResult tv = block_l1_tau_fixed_point<V>(vacc, rho, u.rho_p, u.th, sm.u.proj, sm.sc, u.vbound);
        float th = tv.th, tl = tv.tl;
        if constexpr (!kF64) {
          if (u.acc_kx && !tv.inside) refine_tau(gk, neu, th, tl);
        }
        if (tid == 0) {
          if (D.trace) u.ts[8] = globaltimer();
          u.psteps = sm.sc.flags[2];
          for (int q = 0; q < 8; ++q) u.tt[q] = sm.sc.tt[q];
          u.tau = tv.inside ? 0.0 : (kF64 ? tv.tau : static_cast<double>(th) + static_cast<double>(tl));
          u.th = th;
          u.tl = tl;
          u.inside = tv.inside;
        }
      }
      // the pass-A reductions of k+1 and the pass-B ones of k+1 go to buffers
      // nobody reads any more: clear this CTA's slices
      zero_slices(gbuf + ((k + 1) % 3) * pp, (k + 1) & 1);
      consumer_sync();

      if (tid == 0 && D.trace) u.ts[2] = globaltimer();
      // ---------------- pass B: [K d_k, K x_k], g^T d, ||d||^2
      if (!kF64 && u.kmode[k & 1]) pass_b<true>(gk, Dir(u), kp_of(k & 1), kx_of(k & 1), part);
      else pass_b<false>(gk, Dir(u), kp_of(k & 1), kx_of(k & 1), part);
      if (tid == 0 && D.trace) {
        u.ts[3] = globaltimer();
        trace_spread(k, 26, u.ts[3]);
      }
      if (!group_sync()) break;
      if (tid == 0 && D.trace) u.ts[4] = globaltimer();

      // ---------------- phase L
      {
        S ls[3];
        if (!kF64 && u.kmode[k & 1]) line_scalars<true>(kp_of(k & 1), kx_of(k & 1), ls);
        else line_scalars<false>(kp_of(k & 1), kx_of(k & 1), ls);
        S gd, dd;
        unsigned nz;
        if (warp == 0) reduce_parts(part, gd, dd, nz);
        if (tid == 0) {
          u.gd = as_double(gd);
          u.dd = as_double(dd);
          if constexpr (!kF64) {
            u.ddf = dd.hi + dd.lo;
            u.kb2f = ls[2].hi + ls[2].lo;
          }
          if (!nz) {   // h == x: stationary point (Alg. GP, Step 2)
            u.stop = GPL1_STOP_STATIONARY;
            u.iters = k;
            u.f_cur = as_double(ls[0]);
            u.done = 1;
          } else {
            ls_step(k, as_double(ls[0]), as_double(ls[2]));
          }
        }
        consumer_sync();
        if (u.status == GPL1_ERR_NONFINITE || u.status == GPL1_ERR_LINESEARCH || u.stop == GPL1_STOP_STATIONARY)
          break;
        // x_{k+1} = x_k + lam d_k on this CTA's columns
        const A la = kF64 ? static_cast<A>(u.lam) : static_cast<A>(u.lf);
        const Dir dir(u);
        const int j0 = static_cast<int>(static_cast<long long>(p) * cta / G);
        const int j1 = static_cast<int>(static_cast<long long>(p) * (cta + 1) / G);
        const A xsc = xscale();
        for (int j = j0 + tid; j < j1; j += kConsumers) {
          const A xj = static_cast<A>(x[j]) * xsc;
          x[j] = static_cast<V>(vfma(la, dir.d(xj, gk[j]), xj));
        }
        if (u.done) break;
      }
    }
  finish:
    drain();
    if (cta == 0 && tid == 0) {
      int st = u.status;
      if (status != GPL1_OK) st = status;   // launch-level failure (timeout)
      const double gmax = kF64 ? u.gmax : static_cast<double>(u.gmaxf);
      gpl1_result r;
      r.status = st;
      r.stop = (st != GPL1_OK && st != GPL1_ERR_NOT_CONVERGED) ? GPL1_STOP_ERROR : u.stop;
      r.iters = u.iters;
      r.backtracks = u.backtracks;
      r.f = u.f_cur;
      r.rel_gap = D.f_star > 0.0 ? (u.f_cur - D.f_star) / D.f_star : -1.0;
      double gx;
      if constexpr (kF64) gx = u.gx_u.d;
      else gx = as_double(u.gx_u.f);
      r.fw_gap = gx + D.rho * gmax;
      r.lambda = 0.5 * gmax;
      r.alpha = kF64 ? u.alpha : static_cast<double>(u.ah);
      r.tau = kF64 ? u.tau : static_cast<double>(u.th) + static_cast<double>(u.tl);
      r.kernel_ms = 0.0;   // filled in by the host from events around the launch
      r.fail_site = sm.ctl[CTL_SITE];
      r.fail_iter = u.iters;
      *D.res = r;
    }
    if (tid == 0 && reinterpret_cast<volatile int*>(sm.ctl)[CTL_ERR]) sm.ctl[CTL_BROKEN] = 1;
  }
};

template <int DT, int TL>
__global__ void __launch_bounds__(kThreads, 1) gpss_kernel(const __grid_constant__ KArgs a,
                                                           const __grid_constant__ CUtensorMap tmap0) {
  constexpr int kStages = Tile<DT, TL>::STAGES;
  extern __shared__ uint8_t dyn_smem[];
  SolverSmem<DT, TL>& sm = *reinterpret_cast<SolverSmem<DT, TL>*>(
      (reinterpret_cast<uintptr_t>(dyn_smem) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kConsumerWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t it = 0;
  unsigned epoch = 0;
  const int G = a.group;
  const int cta = G == 1 ? 0 : static_cast<int>(blockIdx.x);
  for (int round = 0;; ++round) {
    if (tid == 0) {
      int inst;
      if (G == 1) inst = static_cast<int>(atomicAdd(a.queue, 1u));
      else inst = round == 0 ? 0 : a.count;
      sm.ctl[CTL_INST] = inst;
      sm.ctl[CTL_STOP] = 0;
      sm.ctl[CTL_DONE] = 0;
      sm.ctl[CTL_ERR] = 0;
      sm.ctl[CTL_SITE] = 0;
      sm.ctl[CTL_ISSUED] = static_cast<int>(it);
      if (round == 0) sm.ctl[CTL_BROKEN] = 0;
    }
    __syncthreads();
    const int inst = sm.ctl[CTL_INST];
    if (inst >= a.count) break;
    const InstDesc& D = a.desc[inst];
    const void* tmap = D.tmap ? D.tmap : static_cast<const void*>(&tmap0);
    if (tid >= kConsumers) {
      if (tid == kConsumers) producer_run<DT, TL>(D, tmap, sm, it, cta, G, a.prm.timeout_ns);
      // lane 0 of the producer warp ran the producer loop alone: reconverge the
      // warp before the aligned block barrier below
      __syncwarp();
    } else {
      Consumer<DT, TL> c(a, D, sm, it, epoch, cta, G);
      c.run();
      __syncwarp();
    }
    __syncthreads();
    if (sm.ctl[CTL_BROKEN]) break;   // its barriers are in an unknown state: take no more instances
  }
}

// Host side of one dtype's kernels (instantiated by gpss_<dtype>.cu): the
// dynamic shared memory, the kernel and its launch for a tile (GPL1_TILE_*).
template <int DT, int TL>
size_t gpss_smem_tl() {
  return sizeof(SolverSmem<DT, TL>) + 128;
}
template <int DT, int TL>
cudaError_t gpss_launch_tl(const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative, cudaStream_t stream) {
  const size_t smem = gpss_smem_tl<DT, TL>();
  const void* fn = reinterpret_cast<const void*>(gpss_kernel<DT, TL>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<KArgs*>(&a), const_cast<CUtensorMap*>(&tmap)};
  if (cooperative) return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, stream);
  return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, stream);
}
// tile -> (launch, shared memory, kernel); FP64 has no SMALL tile
template <int DT>
struct GpssHost {
  static constexpr bool kSmall = DT != GPL1_F64;
  static cudaError_t launch(int tile, const KArgs& a, const CUtensorMap& tmap, int grid, bool coop, cudaStream_t s) {
    if constexpr (kSmall)
      if (tile == GPL1_TILE_SMALL) return gpss_launch_tl<DT, GPL1_TILE_SMALL>(a, tmap, grid, coop, s);
    if (tile == GPL1_TILE_MEDIUM) return gpss_launch_tl<DT, GPL1_TILE_MEDIUM>(a, tmap, grid, coop, s);
    if (tile == GPL1_TILE_LARGE) return gpss_launch_tl<DT, GPL1_TILE_LARGE>(a, tmap, grid, coop, s);
    return cudaErrorInvalidValue;
  }
  static size_t smem(int tile) {
    if constexpr (kSmall)
      if (tile == GPL1_TILE_SMALL) return gpss_smem_tl<DT, GPL1_TILE_SMALL>();
    if (tile == GPL1_TILE_LARGE) return gpss_smem_tl<DT, GPL1_TILE_LARGE>();
    return gpss_smem_tl<DT, GPL1_TILE_MEDIUM>();
  }
  static const void* kernel(int tile) {
    if constexpr (kSmall)
      if (tile == GPL1_TILE_SMALL) return reinterpret_cast<const void*>(gpss_kernel<DT, GPL1_TILE_SMALL>);
    if (tile == GPL1_TILE_LARGE) return reinterpret_cast<const void*>(gpss_kernel<DT, GPL1_TILE_LARGE>);
    return reinterpret_cast<const void*>(gpss_kernel<DT, GPL1_TILE_MEDIUM>);
  }
};

}  // namespace gpl1
