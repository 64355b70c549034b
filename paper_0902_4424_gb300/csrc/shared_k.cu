// Shared-K form of Alg. GP + SS: nrhs instances of eq. 2 that share one K
// (BF16) and differ in y and rho, solved together.  Their gradients
// g_b = 2 K^T r_b and their products K d_b, K x_b are then the matrix products
//
//   G  = 2 R K      (nrhs x p)   on the tensor cores as  K^T R^T
//   KD = D K^T      (nrhs x n)   on the tensor cores as  K D^T
//
// (gemm_tc.cu), with the FP32 vectors carried as three BF16 terms
// (hi + mid + lo = the FP32 value to 2^-24), so a BF16 K gives FP32-accurate
// products.  Everything else of an iteration is per instance and runs in two
// "column" kernels, one CTA per instance:
//
//   mr_phase_p: z^T z, g^T x, ||g||_inf; Alg. SS; v = x - alpha g; the
//     projection threshold (block_l1_tau_fixed_point, as in the single solve);
//     d = P(v) - x; g^T d, ||d||^2; the BF16 terms of d for the second
//     product.
//   mr_phase_l: the sum of the second product's split-K partials; f,
//     r^T K d, ||K d||^2; the Armijo test of Alg. GP on the exact expansion
//     (FP64, lead thread); x += lam d, r += lam K d (the update of Alg. GP,
//     Step 6) and its BF16 terms for the next gradient; Alg. SS state; the
//     stop rules.
//
// r is carried from iteration to iteration (its BF16 terms hold the FP32
// value exactly), so the second product needs K d only: half the tensor work
// of forming K x again.  The carried r drifts from K x - y by the rounding of
// the updates and the FP32 accumulation error of each K d (about 1e-6 of
// lam |K d|); summed over the path from x0 that is about 1e-6 |K x|, and
// r^T dKx turns it into an error of f far above tol f* when f* << ||y||^2.
// So near the stop (estimated gap below 1000 tol, or progress below 1e-4 f)
// r restarts from an exact K x (mr_exact_kx, between the second product and
// mr_phase_l), on the first iteration there and every 8th after: the drift
// since a restart is 1e-6 of the few small steps near the optimum.  The
// relative-gap stop is only taken on an iteration whose r was restarted: met
// on a carried r, it schedules a restart for the next iteration and is
// decided there.  The iterate is sparse by then (the l1 ball), so K x = sum
// over the support of x_j (column j of K = row j of the stored K^T), with
// exact products and two-sums: the same compensated sum as the single
// solve's pass B near its stop.
//
// As in the single solve, x is kept inside the ball (an exact ||x||_1 check
// and a scale back onto the ball when rounding leaves it outside) and tau is
// recomputed on the active set from x and g, so d stays a descent direction.
#include <cudaTypedefs.h>

#include "launch.h"

namespace gpl1 {

constexpr int kMrVmax = 35;   // p <= 35 * 480

struct MrState {
  SSState<float> ss;
  float ah, th, tl, vbound, gmaxf, xscale;
  float rho_hi, rho_lo;
  int inside, nz, iters, backtracks, stop, status, done, acc, acc_age;
  double f_cur, gap_den, f_star, rho, lam, gd, dd, gx;
  double fhist[kMaxM];
  double f_best;   // lowest f so far, and the iterations since it last fell by a
  int stall;       // meaningful amount (the stagnation stop near the precision floor)
};

// Stagnation (with a stop rule to reach): near the stop (acc), an instance
// whose f has not fallen by more
// than 1e-3 tol of its gap denominator for this many iterations sits at the
// precision floor of the FP32 form (its carried and exact residuals disagree
// by about the tolerance) and stops, not converged, instead of running to
// max_iter and holding the whole batch.
constexpr int kMrStallIters = 32;

// The staged vector comes last: a launch allocates only its first
// ceil(p / 480) * 480 entries, so that for p = 8192 four CTAs share an SM.
struct MrSmem {
  ProjSmem ps;
  Scratch sc;
  int flag[4];
  float xs[2 * kMrVmax * kConsumers];
};

// Phase P stages two vectors there (x, later v, and g; each neu * 480
// floats); the other kernels use the first.
size_t mr_smem_bytes(int p, int vectors) {
  const size_t neu = (static_cast<size_t>(p) + kConsumers - 1) / kConsumers;
  return offsetof(MrSmem, xs) + static_cast<size_t>(vectors) * neu * kConsumers * sizeof(float);
}

size_t mr_state_bytes() { return sizeof(MrState); }

__device__ __forceinline__ void split3(float v, uint16_t& h, uint16_t& m, uint16_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(bh);   // exact
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);  // exact
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

// Alg. SS for k >= 1 (the same rule as the single solve): alpha from BB1/BB2
// with the ratio test against tau_k and the alpha^(2) window.
__device__ float mr_ss_step(SSState<float>& st, float zz, const SolveParams& P) {
  const float amin_p = static_cast<float>(P.alpha_min), amax_p = static_cast<float>(P.alpha_max);
  float alpha, a2_this;
  if (st.sz_prev <= 0.f) {
    alpha = amax_p;
    a2_this = amax_p;
  } else {
    const float a1 = fminf(fmaxf(st.ss_prev / st.sz_prev, amin_p), amax_p);
    const float a2 = fminf(fmaxf(st.sz_prev / zz, amin_p), amax_p);
    a2_this = a2;
    float amin = a2;
    for (int q = 0; q < st.a2cnt && q < P.M_alpha; ++q) amin = fminf(amin, st.a2win[q]);
    if (a2 <= st.tau_ss * a1) {
      alpha = amin;
      st.tau_ss *= 0.9f;
    } else {
      alpha = a1;
      st.tau_ss *= 1.1f;
    }
  }
  for (int q = P.M_alpha - 1; q > 0; --q) st.a2win[q] = st.a2win[q - 1];
  if (P.M_alpha > 0) st.a2win[0] = a2_this;
  if (st.a2cnt < P.M_alpha) ++st.a2cnt;
  return alpha;
}

// Initial state, x0 = 0, r0 = -y: its BF16 terms for the first gradient.
__global__ void __launch_bounds__(kConsumers) mr_init(const float* Y, long long ldy, float* X, long long ldx,
                                                      uint16_t* Rs, int n, int p, const double* rho,
                                                      const double* fstar, MrState* st, SolveParams prm) {
  const int b = blockIdx.x, tid = threadIdx.x;
  __shared__ Scratch sc;
  const float* y = Y + b * ldy;
  float* x = X + b * ldx;
  uint16_t* rs = Rs + static_cast<long long>(b) * 3 * n;
  for (int j = tid; j < p; j += kConsumers) x[j] = 0.f;
  F2 yy{0.f, 0.f};
  for (int i = tid; i < n; i += kConsumers) {
    const float r = -y[i];
    yy = f2_fma(yy, r, r);
    uint16_t h, m, l;
    split3(r, h, m, l);
    rs[i] = h;
    rs[n + i] = m;
    rs[2 * n + i] = l;
  }
  F2 v[1] = {yy};
  unsigned dummy = 0;
  lead_reduce<1>(v, dummy, sc);
  if (tid == 0) {
    MrState s;
    memset(&s, 0, sizeof s);
    s.ss.tau_ss = static_cast<float>(prm.tau1);
    const double y2 = as_double(v[0]);
    s.f_cur = y2;
    s.f_best = y2;
    for (int q = 0; q < kMaxM; ++q) s.fhist[q] = y2;
    s.rho = rho[b];
    const F2 rp = f2_of(rho[b]);
    s.rho_hi = rp.hi;
    s.rho_lo = rp.lo;
    s.f_star = fstar ? fstar[b] : -1.0;
    s.gap_den = fmax(s.f_star, prm.tol * y2);
    s.xscale = 1.f;
    s.stop = GPL1_STOP_MAX_ITER;
    st[b] = s;
  }
}

// Given x0 (rows of X): project it onto its ball where it lies outside (Alg.
// GP starts in Omega), then lay out its BF16 terms (in the rows of the d
// terms) for the product K x0.
__global__ void __launch_bounds__(kConsumers) mr_setup_x0(float* X, long long ldx, uint16_t* DXs, int p, int nrhs,
                                                          const double* rho) {
  const int b = blockIdx.x, tid = threadIdx.x;
  extern __shared__ uint8_t mr_raw[];
  MrSmem& sm = *reinterpret_cast<MrSmem*>(mr_raw);
  float* const xs = sm.xs;
  float* x = X + b * ldx;
  const int neu = (p + kConsumers - 1) / kConsumers;
  for (int e = 0; e < neu; ++e) {
    const int j = tid + e * kConsumers;
    xs[e * kConsumers + tid] = j < p ? x[j] : 0.f;
  }
  if (tid == 0) {
    const F2 rp = f2_of(rho[b]);
    sm.sc.tp[0] = rp.hi;
    sm.sc.tp[1] = rp.lo;
  }
  consumer_sync();
  const F2 rho_p{sm.sc.tp[0], sm.sc.tp[1]};
  consumer_sync();
  const SmemAcc<float, kMrVmax> acc{xs, neu};
  const TauResult t = block_l1_tau_fixed_point<float>(acc, rho[b], rho_p, 0.f, sm.ps, sm.sc);
  const TauPair tp{t.th, t.tl};
  uint16_t* xx_s = DXs + static_cast<long long>(b) * 3 * p;
  for (int e = 0; e < neu; ++e) {
    const int j = tid + e * kConsumers;
    if (j >= p) break;
    const float v = xs[e * kConsumers + tid];
    const float a = fabsf(v);
    const float xj = t.inside ? v : (tp.below(a) ? 0.f : copysignf((a - tp.hi) - tp.lo, v));
    x[j] = xj;
    uint16_t h, m, l;
    split3(xj, h, m, l);
    xx_s[j] = h;
    xx_s[p + j] = m;
    xx_s[2 * p + j] = l;
  }
}

// Initial state from r0 = K x0 - y (K x0 from the tensor-core product).
__global__ void __launch_bounds__(kConsumers) mr_setup_r(const float* KDX, const float* Y, long long ldy,
                                                         uint16_t* Rs, int n, int nrhs, const double* rho,
                                                         const double* fstar, MrState* st, SolveParams prm) {
  const int b = blockIdx.x, tid = threadIdx.x;
  __shared__ Scratch sc;
  const float* kx = KDX + static_cast<long long>(b) * n;
  const float* y = Y + b * ldy;
  uint16_t* rs = Rs + static_cast<long long>(b) * 3 * n;
  F2 ff{0.f, 0.f}, yy{0.f, 0.f};
  for (int i = tid; i < n; i += kConsumers) {
    const F2 r = two_sum(kx[i], -y[i]);
    ff = f2_fma(ff, r.hi, r.hi + 2.f * r.lo);
    yy = f2_fma(yy, y[i], y[i]);
    uint16_t h, m, l;
    split3(r.hi + r.lo, h, m, l);
    rs[i] = h;
    rs[n + i] = m;
    rs[2 * n + i] = l;
  }
  F2 v[2] = {ff, yy};
  unsigned dummy = 0;
  lead_reduce<2>(v, dummy, sc);
  if (tid == 0) {
    MrState s;
    memset(&s, 0, sizeof s);
    s.ss.tau_ss = static_cast<float>(prm.tau1);
    const double f0 = as_double(v[0]), y2 = as_double(v[1]);
    s.f_cur = f0;
    s.f_best = f0;
    for (int q = 0; q < kMaxM; ++q) s.fhist[q] = f0;
    s.rho = rho[b];
    const F2 rp = f2_of(rho[b]);
    s.rho_hi = rp.hi;
    s.rho_lo = rp.lo;
    s.f_star = fstar ? fstar[b] : -1.0;
    s.gap_den = fmax(s.f_star, prm.tol * y2);
    s.xscale = 1.f;
    s.stop = GPL1_STOP_MAX_ITER;
    st[b] = s;
  }
}

// d_j from the float pair of alpha (hi only here) and tau, as in pass B of the
// single solve: the active form never subtracts x from a number of its size.
__device__ __forceinline__ float mr_dir(float x, float g, float ah, float th, float tl, int inside) {
  const float v = fmaf(-ah, g, x);
  if (inside) return -ah * g;
  if (!((fabsf(v) - th) > tl)) return -x;
  const float s = v > 0.f ? 1.f : -1.f;
  const float pr = __fmul_rn(ah, g);
  const float e = fmaf(ah, g, -pr);
  const F2 q = two_sum(pr, th * s);
  return -(q.hi + (q.lo + (e + tl * s)));
}

// Restarts of r from the exact K x (see the file comment): on the first
// iteration near the stop, on the iteration after a relative-gap stop was met
// on a carried r, and every 8th iteration in between.  (Every 32nd saves
// restarts but lets the drift into the line search: c4 then took 51.5
// iterations on average instead of 47.2.)
constexpr int kMrExactEvery = 8;   // near the stop, r restarts from the exact K x every 8 iterations

__device__ __forceinline__ bool mr_restarts(const MrState& S) {
  return !S.done && S.acc && S.acc_age % kMrExactEvery == 0;
}

// The instances that restart in iteration k are listed by phase P of k in
// list[k & 1] (count cnt[k & 1]) for mr_exact_kx; phase P of k clears the
// other count, which mr_exact_kx of k - 1 has consumed.
struct MrRestartList {
  int* cnt;    // [2]
  int* list;   // [2][nrhs]
};

__global__ void __launch_bounds__(kConsumers) mr_phase_p(const float* G, const float* Gprev, const float* X,
                                                         long long ldx, float* D, uint16_t* DXs, int p, int nrhs,
                                                         int k, MrState* st, SolveParams prm, MrRestartList rl) {
  const int b = blockIdx.x, tid = threadIdx.x;
  pdl_wait();
  pdl_trigger();
  MrState& S = st[b];
  if (b == 0 && tid == 0) rl.cnt[(k + 1) & 1] = 0;
  if (S.done) return;   // the same value in every thread of the CTA
  extern __shared__ uint8_t mr_raw[];
  MrSmem& sm = *reinterpret_cast<MrSmem*>(mr_raw);
  const int neu = (p + kConsumers - 1) / kConsumers;
  // staged in shared memory, element e of this thread = column tid + e * 480:
  // xs (x, later v = x - alpha g) and gs (g)
  float* const xs = sm.xs;
  float* const gs = xs + neu * kConsumers;
  const float* g = G + static_cast<long long>(b) * p;
  const float* gp = Gprev + static_cast<long long>(b) * p;
  const float* x = X + b * ldx;
  // z^T z, g^T x, max |g|, ||x||_1.  z^T z (for a steplength) takes plain FP32
  // sums; g^T x (the Frank-Wolfe certificate, a difference of large terms near
  // the stop) and ||x||_1 (the feasibility check) float pairs.
  F2 gx{0.f, 0.f}, l1{0.f, 0.f};
  float zzf = 0.f;
  float pm = 0.f;
  constexpr int CH = 6;   // the loads of a chunk are issued together
  for (int e0 = 0; e0 < neu; e0 += CH) {
    float gv[CH], gq[CH], xv[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = tid + (e0 + c) * kConsumers;
      const bool in = e0 + c < neu && j < p;
      gv[c] = in ? g[j] : 0.f;
      xv[c] = in ? x[j] : 0.f;
      gq[c] = in && k > 0 ? gp[j] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (e0 + c >= neu) break;
      if (k > 0) {
        const float z = gv[c] - gq[c];
        zzf = fmaf(z, z, zzf);
      }
      gx = f2_fma(gx, gv[c], xv[c]);
      l1 = f2_add(l1, fabsf(xv[c]));
      pm = fmaxf(pm, fabsf(gv[c]));
      const int o = (e0 + c) * kConsumers + tid;
      xs[o] = xv[c];
      gs[o] = gv[c];
    }
  }
  F2 red[3] = {F2{zzf, 0.f}, gx, l1};
  unsigned mx = __float_as_uint(pm);
  lead_reduce<3>(red, mx, sm.sc);
  if (tid == 0) {
    S.gmaxf = __uint_as_float(mx);
    S.gx = as_double(red[1]);
    const F2 rp{S.rho_hi, S.rho_lo};
    const float ex = (red[2].hi - rp.hi) + (red[2].lo - rp.lo);   // ||x||_1 - rho
    S.xscale = ex > 0.f ? __fdiv_rd(rp.hi, red[2].hi) * (1.f - 0x1p-21f) : 1.f;
    int fin = 0;
    if (prm.stop_rule & GPL1_STOP_ON_FW) {
      const double fw = S.gx + S.rho * static_cast<double>(S.gmaxf);
      if (fw <= prm.tol * (S.f_cur - fw)) {
        S.stop = GPL1_STOP_FW;
        S.done = 1;
        fin = 1;
      }
    }
    if (!fin && k > 0) {
      S.ah = mr_ss_step(S.ss, red[0].hi + red[0].lo, prm);
      S.vbound = (S.rho_hi + S.ah * S.gmaxf) * 1.00001f;
    }
    if (!fin && k == 0) S.vbound = (S.rho_hi + S.gmaxf) * 1.00001f;
    sm.flag[0] = fin;
  }
  consumer_sync();
  if (sm.flag[0]) return;
  const float xsc = S.xscale;
  const F2 rho_p{S.rho_hi, S.rho_lo};
  if (k == 0) {   // alpha_0 = clamp(1 / ||P(x0 - g0)||_inf)  (rule 1: of P(.) - x0)
    for (int e = 0; e < neu; ++e) {
      const int o = e * kConsumers + tid;
      xs[o] = fmaf(-1.f, gs[o], xs[o] * xsc);   // 0 past p (g and x staged as 0 there)
    }
    consumer_sync();
    const SmemAcc<float, kMrVmax> acc{xs, neu};
    const TauResult tw = block_l1_tau_fixed_point<float>(acc, S.rho, rho_p, 0.f, sm.ps, sm.sc, S.vbound);
    const TauPair tp{tw.th, tw.tl};
    float m = 0.f;
    for (int e = 0; e < neu; ++e) {
      const int j = tid + e * kConsumers;
      if (j >= p) break;
      const float v = xs[e * kConsumers + tid];
      const float a = fabsf(v);
      float h = tw.inside ? v : (tp.below(a) ? 0.f : copysignf((a - tp.hi) - tp.lo, v));
      if (prm.alpha0_rule == 1) h -= x[j] * xsc;
      m = fmaxf(m, fabsf(h));
    }
    m = block_max_nonneg(m, sm.sc);
    if (tid == 0) {
      const double a0 = m > 0.f ? fmin(fmax(1.0 / static_cast<double>(m), prm.alpha_min), prm.alpha_max)
                                : prm.alpha_max;
      S.ah = static_cast<float>(a0);
      S.vbound = (S.rho_hi + S.ah * S.gmaxf) * 1.00001f;
    }
    consumer_sync();
  }
  const float ah = S.ah;
  if (k == 0) {   // xs holds x0 - g0 here: x from memory
    for (int e0 = 0; e0 < neu; e0 += CH) {
      float xv[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int j = tid + (e0 + c) * kConsumers;
        xv[c] = e0 + c < neu && j < p ? x[j] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        if (e0 + c >= neu) break;
        const int o = (e0 + c) * kConsumers + tid;
        xs[o] = fmaf(-ah, gs[o], xv[c] * xsc);
      }
    }
  } else {
    for (int e = 0; e < neu; ++e) {
      const int o = e * kConsumers + tid;
      xs[o] = fmaf(-ah, gs[o], xs[o] * xsc);
    }
  }
  consumer_sync();
  const SmemAcc<float, kMrVmax> vacc{xs, neu};
  const TauResult tv = block_l1_tau_fixed_point<float>(vacc, S.rho, rho_p, S.th, sm.ps, sm.sc, S.vbound);
  float th = tv.th, tl = tv.tl;
  if (!tv.inside) {
    // tau on the active set from x and g themselves (see the file comment)
    const TauPair tp{th, tl};
    F2 v3[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int e = 0; e < neu; ++e) {
      const int j = tid + e * kConsumers, o = e * kConsumers + tid;
      const float vv = xs[o];
      if (j < p && !tp.below(fabsf(vv))) {
        const float s = vv > 0.f ? 1.f : -1.f;
        v3[0] = f2_add(v3[0], s * (x[j] * xsc));
        v3[1] = f2_add(v3[1], s * gs[o]);
        v3[2] = f2_add(v3[2], 1.f);
      }
    }
    unsigned dummy = 0;
    lead_reduce<3>(v3, dummy, sm.sc);
    if (tid == 0) {
      const float c = v3[2].hi;
      const float ph = __fmul_rn(ah, v3[1].hi);
      const float pl = fmaf(ah, v3[1].hi, -ph) + ah * v3[1].lo;
      F2 t = f2_add(v3[0], F2{-ph, -pl});
      t = f2_add(t, F2{-rho_p.hi, -rho_p.lo});
      const float q1 = __fdiv_rn(t.hi, c);
      const float rem = fmaf(-q1, c, t.hi) + t.lo;
      const F2 q = two_sum(q1, __fdiv_rn(rem, c));
      sm.sc.tp[2] = (c > 0.f && q.hi > 0.f) ? q.hi : th;
      sm.sc.tp[3] = (c > 0.f && q.hi > 0.f) ? q.lo : tl;
    }
    consumer_sync();
    th = sm.sc.tp[2];
    tl = sm.sc.tp[3];
  }
  // direction, its sums, and the BF16 terms of d for K D^T
  float* d = D + static_cast<long long>(b) * p;
  uint16_t* dd_s = DXs + static_cast<long long>(b) * 3 * p;
  F2 sgd{0.f, 0.f};   // its sign decides the line search near the stop: float pairs
  float sddf = 0.f;
  unsigned nz = 0;
  for (int e0 = 0; e0 < neu; e0 += CH) {
    float xr[CH];   // x from memory: a chunk's loads are issued before its stores
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = tid + (e0 + c) * kConsumers;
      xr[c] = e0 + c < neu && j < p ? x[j] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int e = e0 + c, j = tid + e * kConsumers, o = e * kConsumers + tid;
      if (e >= neu || j >= p) break;
      const float xj = xr[c] * xsc, gj = gs[o];
      const float dj = mr_dir(xj, gj, ah, th, tl, tv.inside);
      d[j] = dj;
      sgd = f2_fma(sgd, gj, dj);
      sddf = fmaf(dj, dj, sddf);
      nz |= dj != 0.f ? 1u : 0u;
      uint16_t h, m, l;
      split3(dj, h, m, l);
      dd_s[j] = h;
      dd_s[p + j] = m;
      dd_s[2 * p + j] = l;
    }
  }
  F2 v2[2] = {sgd, F2{sddf, 0.f}};
  unsigned nzm = nz;
  lead_reduce<2>(v2, nzm, sm.sc);
  if (tid == 0) {
    S.gd = as_double(v2[0]);
    S.dd = as_double(v2[1]);
    S.nz = nzm ? 1 : 0;
    S.th = th;
    S.tl = tl;
    S.inside = tv.inside;
    if (mr_restarts(S)) rl.list[(k & 1) * nrhs + atomicAdd(&rl.cnt[k & 1], 1)] = b;
  }
}

constexpr int kMrRowsPerThread = 9; // n <= 9 * 480 rows for the accurate K x

// Exact K x for the instances that restart r this iteration, split over
// S = ceil(p / 1024) CTAs per instance by columns: CTA (b, s) takes the nonzero
// x_j (x scaled into the ball, as phase P used it) of columns
// [s p / S, (s+1) p / S) in increasing j, and sums x_j K_:j (row j of the
// stored K^T) into float pairs, exactly up to the pair's 2^-48: each product
// K_ij x_j is exact as (p, e) (FMA) and the running sum takes p by an
// error-free two-sum, its error and e accumulating in the low word.  A thread
// owns 8 consecutive rows (one 16-byte load of K^T per column).  Phase L sums
// the S partials of a row in order of s.
constexpr int kMrExactCols = 1024;   // columns per CTA of mr_exact_kx
constexpr int kMrExactThreads = 256;
constexpr int kMrExactGroups = 3;    // 8-row groups per thread: n <= 3 * 256 * 8 = 6144

int mr_exact_splits(int p) { return (p + kMrExactCols - 1) / kMrExactCols; }


// One (instance b, column range s) item of mr_exact_kx.
__device__ __forceinline__ void mr_exact_item(const uint16_t* __restrict__ Kt, const float* __restrict__ X,
                                              long long ldx, F2* __restrict__ part, int n, int p, int S,
                                              const MrState& M, int b, int s, int tid, int* sup_j, float* sup_x,
                                              int& sup_n) {
  const int j0 = static_cast<int>(static_cast<long long>(s) * p / S);
  const int j1 = static_cast<int>(static_cast<long long>(s + 1) * p / S);
  const float xsc = M.xscale;
  const float* x = X + b * ldx;
  if (tid < 32) {   // warp 0 lists the nonzeros in increasing j (ballot order)
    int cnt = 0;
    for (int c0 = j0; c0 < j1; c0 += 32) {
      const int j = c0 + tid;
      const float xv = j < j1 ? x[j] * xsc : 0.f;
      const unsigned nzm = __ballot_sync(0xffffffffu, xv != 0.f);
      if (xv != 0.f) {
        const int q = cnt + __popc(nzm & ((1u << tid) - 1u));
        sup_j[q] = j;
        sup_x[q] = xv;
      }
      cnt += __popc(nzm);
    }
    if (tid == 0) sup_n = cnt;
  }
  __syncthreads();
  const int ns = sup_n;
  F2 acc[kMrExactGroups][8];
#pragma unroll
  for (int m = 0; m < kMrExactGroups; ++m)
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[m][r] = F2{0.f, 0.f};
  for (int q = 0; q < ns; ++q) {
    const float xv = sup_x[q];
    const uint16_t* col = Kt + static_cast<long long>(sup_j[q]) * n;   // column j of K
#pragma unroll
    for (int m = 0; m < kMrExactGroups; ++m) {
      const int i0 = 8 * (tid + m * kMrExactThreads);
      if (i0 >= n) break;
      const uint4 w = *reinterpret_cast<const uint4*>(col + i0);
      const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float kv = __uint_as_float(r & 1 ? (u[r >> 1] & 0xffff0000u) : (u[r >> 1] << 16));
        const float pr = __fmul_rn(kv, xv);
        const float pe = fmaf(kv, xv, -pr);
        const F2 t = two_sum(acc[m][r].hi, pr);
        acc[m][r].hi = t.hi;
        acc[m][r].lo += t.lo + pe;
      }
    }
  }
  F2* out = part + (static_cast<long long>(b) * S + s) * n;
#pragma unroll
  for (int m = 0; m < kMrExactGroups; ++m) {
    const int i0 = 8 * (tid + m * kMrExactThreads);
    if (i0 >= n) break;
#pragma unroll
    for (int r = 0; r < 8; ++r) out[i0 + r] = two_sum(acc[m][r].hi, acc[m][r].lo);
  }
}

__global__ void __launch_bounds__(kMrExactThreads) mr_exact_kx(const uint16_t* __restrict__ Kt,
                                                              const float* __restrict__ X, long long ldx,
                                                              F2* __restrict__ part, int n, int p, int S,
                                                              const MrState* __restrict__ st, const int* cnt,
                                                              const int* list) {
  __shared__ int sup_j[kMrExactCols];
  __shared__ float sup_x[kMrExactCols];
  __shared__ int sup_n;
  pdl_wait();
  pdl_trigger();
  const int items = *cnt * S, tid = threadIdx.x;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {   // (listed instance, column range)
    const int b = list[item / S], s = item % S;
    mr_exact_item(Kt, X, ldx, part, n, p, S, st[b], b, s, tid, sup_j, sup_x, sup_n);
    __syncthreads();   // the lists in shared memory are reused by the next item
  }
}

// The carried r_i = K x - y: its three BF16 terms add up to the FP32 value
// exactly; on an iterate that phase P scaled back onto the ball (x -> c x),
// K (c x) - y = c r + (c - 1) y.
__device__ __forceinline__ F2 mr_carried_r(const uint16_t* rs, int n, int i, float xsc, float yi) {
  const float r = (__uint_as_float(static_cast<unsigned>(rs[i]) << 16) +
                   __uint_as_float(static_cast<unsigned>(rs[n + i]) << 16)) +
                  __uint_as_float(static_cast<unsigned>(rs[2 * n + i]) << 16);
  if (xsc == 1.f) return F2{r, 0.f};
  return two_sum(__fmul_rn(xsc, r), (xsc - 1.f) * yi);
}

__global__ void __launch_bounds__(kConsumers) mr_phase_l(float* KD, int splits, long long split_stride,
                                                         const F2* part, int xsplits, const float* Y, long long ldy,
                                                         float* X, long long ldx, const float* D, uint16_t* Rs, int n,
                                                         int p, int k, MrState* st, SolveParams prm,
                                                         gpl1_result* res, int* done_count) {
  const int b = blockIdx.x, tid = threadIdx.x;
  pdl_wait();
  pdl_trigger();
  MrState& S = st[b];
  __shared__ Scratch sc;
  __shared__ int flag[2];
  __shared__ float lamf;
  if (S.done) {   // stopped in phase P of this iteration (FW) or earlier
    if (tid == 0 && S.done == 1) {
      S.done = 2;   // record once
      gpl1_result r{};
      r.status = S.status;
      r.stop = S.stop;
      r.iters = S.iters;
      r.backtracks = S.backtracks;
      r.f = S.f_cur;
      r.rel_gap = S.f_star > 0.0 ? (S.f_cur - S.f_star) / S.f_star : -1.0;
      r.fw_gap = S.gx + S.rho * static_cast<double>(S.gmaxf);
      r.lambda = 0.5 * static_cast<double>(S.gmaxf);
      r.alpha = S.ah;
      r.tau = static_cast<double>(S.th) + static_cast<double>(S.tl);
      r.fail_iter = S.iters;
      res[b] = r;
      atomicAdd(done_count, 1);
    }
    return;
  }
  float* kd = KD + static_cast<long long>(b) * n;
  const float* y = Y + b * ldy;
  const uint16_t* rsc = Rs + static_cast<long long>(b) * 3 * n;
  const float xsc0 = S.xscale;
  // r = K x - y: carried, or on a restart the exact K x of mr_exact_kx (its
  // column partials summed in order)
  const bool exact = mr_restarts(S);
  F2 racc[kMrRowsPerThread];
#pragma unroll
  for (int m = 0; m < kMrRowsPerThread; ++m) racc[m] = F2{0.f, 0.f};
  if (exact) {
    const F2* pb = part + static_cast<long long>(b) * xsplits * n;
    for (int z = 0; z < xsplits; ++z) {
#pragma unroll
      for (int m = 0; m < kMrRowsPerThread; ++m) {
        const int i = tid + m * kConsumers;
        if (i < n) racc[m] = f2_add(racc[m], pb[static_cast<long long>(z) * n + i]);
      }
    }
  }
  // K d (the split-K partials summed in order, the sum kept in partial 0), y and r
  float kdv[kMrRowsPerThread], yv[kMrRowsPerThread];
  F2 rv[kMrRowsPerThread];
#pragma unroll
  for (int m = 0; m < kMrRowsPerThread; ++m) {
    const int i = tid + m * kConsumers;
    kdv[m] = i < n ? kd[i] : 0.f;
    yv[m] = i < n ? y[i] : 0.f;
  }
  for (int z = 1; z < splits; ++z) {
#pragma unroll
    for (int m = 0; m < kMrRowsPerThread; ++m) {
      const int i = tid + m * kConsumers;
      if (i < n) kdv[m] += kd[z * split_stride + i];
    }
  }
  F2 v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int m = 0; m < kMrRowsPerThread; ++m) {
    const int i = tid + m * kConsumers;
    if (i >= n) continue;
    if (splits > 1) kd[i] = kdv[m];
    if (exact) {
      const F2 t = two_sum(racc[m].hi, -yv[m]);
      rv[m] = two_sum(t.hi, t.lo + racc[m].lo);
    } else {
      rv[m] = mr_carried_r(rsc, n, i, xsc0, yv[m]);
    }
    v[0] = f2_fma(v[0], rv[m].hi, rv[m].hi + 2.f * rv[m].lo);
    v[1] = f2_fma(v[1], rv[m].hi + rv[m].lo, kdv[m]);
    v[2] = f2_fma(v[2], kdv[m], kdv[m]);
  }
  unsigned dummy = 0;
  lead_reduce<3>(v, dummy, sc);
  if (tid == 0) {
    // Alg. GP, Steps 4-6, on f(x + lam d) = f + lam g^T d + lam^2 ||K d||^2 (FP64)
    const double fk = as_double(v[0]), kb2 = as_double(v[2]), gd = S.gd;
    int acc = 0;
    double lam = 1.0, fnext = fk;
    if (!S.nz) {
      S.stop = GPL1_STOP_STATIONARY;
      S.f_cur = fk;
      S.done = 1;
    } else if (!isfinite(fk) || !isfinite(kb2) || !isfinite(gd)) {
      S.status = GPL1_ERR_NONFINITE;
      S.stop = GPL1_STOP_ERROR;
      S.done = 1;
    } else {
      S.fhist[0] = fk;
      double fmaxv = fk;
      for (int q = 1; q < prm.M && q <= k; ++q) fmaxv = fmax(fmaxv, S.fhist[q]);
      int bt = 0;
      for (;;) {
        if ((fk - fmaxv) + lam * (gd + lam * kb2) <= prm.beta * lam * gd) {
          acc = 1;
          break;
        }
        if (bt >= prm.max_backtracks) break;
        lam *= prm.theta;
        ++bt;
      }
      S.backtracks += bt;
      if (!acc) {
        S.status = GPL1_ERR_LINESEARCH;
        S.stop = GPL1_STOP_ERROR;
        S.f_cur = fk;
        S.done = 1;
      } else {
        fnext = fk + lam * (gd + lam * kb2);
        for (int q = kMaxM - 1; q > 0; --q) S.fhist[q] = S.fhist[q - 1];
        S.fhist[0] = fnext;
        S.lam = lam;
        const float lf = static_cast<float>(lam);
        S.ss.ss_prev = lf * lf * static_cast<float>(S.dd);
        S.ss.sz_prev = 2.f * lf * lf * static_cast<float>(kb2);
        S.f_cur = fnext;
        S.iters = k + 1;
        if (S.acc) ++S.acc_age;
        if ((S.f_star >= 0.0 && fnext - S.f_star <= 1e3 * prm.tol * S.gap_den) || fk - fnext <= 1e-4 * fk) S.acc = 1;
        const bool gap_met =
            (prm.stop_rule & GPL1_STOP_ON_REL_GAP) && S.f_star >= 0.0 && fnext - S.f_star <= prm.tol * S.gap_den;
        if (fnext < S.f_best - 1e-3 * prm.tol * S.gap_den) {
          S.f_best = fnext;
          S.stall = 0;
        } else {
          ++S.stall;
        }
        // f from the exact K x of this iterate
        if (gap_met && exact) {
          S.stop = GPL1_STOP_REL_GAP;
          S.done = 1;
        } else {
          if (gap_met) {   // f from the carried r: confirm on an exact K x next iteration
            S.acc = 1;
            S.acc_age = 0;
          }
          // the last iteration ends every instance still running, whatever its state
          if (S.iters >= prm.max_iter) {
            S.stop = GPL1_STOP_MAX_ITER;
            S.status = GPL1_ERR_NOT_CONVERGED;
            S.done = 1;
          } else if (S.acc && S.stall >= kMrStallIters &&
                     (prm.stop_rule & (GPL1_STOP_ON_REL_GAP | GPL1_STOP_ON_FW))) {
            S.stop = GPL1_STOP_STAGNATION;
            S.status = GPL1_ERR_NOT_CONVERGED;
            S.done = 1;
          }
        }
      }
    }
    if (!S.done) S.iters = k + 1;
    flag[0] = acc;
    flag[1] = S.done;
    lamf = static_cast<float>(lam);
  }
  __syncthreads();
  if (flag[0]) {   // x += lam d (on the iterate scaled into the ball), r += lam K d
    const float la = lamf, xsc = S.xscale;
    float* x = X + b * ldx;
    const float* d = D + static_cast<long long>(b) * p;
    constexpr int CH = 8;   // loads of a chunk are issued together, then the stores
    for (int j0 = tid; j0 < p; j0 += CH * kConsumers) {
      float dv[CH], xv[CH];
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int j = j0 + c * kConsumers;
        dv[c] = j < p ? d[j] : 0.f;
        xv[c] = j < p ? x[j] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int j = j0 + c * kConsumers;
        if (j < p) x[j] = fmaf(la, dv[c], xv[c] * xsc);
      }
    }
    uint16_t* rs = Rs + static_cast<long long>(b) * 3 * n;
#pragma unroll
    for (int m = 0; m < kMrRowsPerThread; ++m) {
      const int i = tid + m * kConsumers;
      if (i >= n) continue;
      const float rn = rv[m].hi + fmaf(la, kdv[m], rv[m].lo);
      uint16_t th3, tm3, tl3;
      split3(rn, th3, tm3, tl3);
      rs[i] = th3;
      rs[n + i] = tm3;
      rs[2 * n + i] = tl3;
    }
  }
  if (flag[1] && tid == 0) {
    S.done = 2;
    gpl1_result r{};
    r.status = S.status;
    r.stop = S.stop;
    r.iters = S.iters;
    r.backtracks = S.backtracks;
    r.f = S.f_cur;
    r.rel_gap = S.f_star > 0.0 ? (S.f_cur - S.f_star) / S.f_star : -1.0;
    r.fw_gap = S.gx + S.rho * static_cast<double>(S.gmaxf);
    r.lambda = 0.5 * static_cast<double>(S.gmaxf);
    r.alpha = S.ah;
    r.tau = static_cast<double>(S.th) + static_cast<double>(S.tl);
    r.fail_iter = S.iters;
    res[b] = r;
    atomicAdd(done_count, 1);
  }
}

// K^T (p x n) from K (n x ldk), BF16 bit patterns, 32 x 32 tiles.
__global__ void transpose_bf16(const uint16_t* K, long long ldk, uint16_t* Kt, int n, int p) {
  __shared__ uint16_t t[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    t[r][threadIdx.x] = (i < n && j < p) ? K[i * ldk + j] : 0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < p && i < n) Kt[static_cast<long long>(j) * n + i] = t[threadIdx.x][r];
  }
}

cudaError_t launch_mr_setup_x0(float* X, long long ldx, uint16_t* DXs, int p, int nrhs, const double* rho,
                               cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(mr_setup_x0, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sizeof(MrSmem)));
  if (e != cudaSuccess) return e;
  mr_setup_x0<<<nrhs, kConsumers, mr_smem_bytes(p, 1), s>>>(X, ldx, DXs, p, nrhs, rho);
  return cudaGetLastError();
}
cudaError_t launch_mr_setup_r(const float* KDX, const float* Y, long long ldy, uint16_t* Rs, int n, int nrhs,
                              const double* rho, const double* fstar, void* states, const SolveParams& prm,
                              cudaStream_t s) {
  mr_setup_r<<<nrhs, kConsumers, 0, s>>>(KDX, Y, ldy, Rs, n, nrhs, rho, fstar, static_cast<MrState*>(states), prm);
  return cudaGetLastError();
}

cudaError_t launch_mr_init(const float* Y, long long ldy, float* X, long long ldx, uint16_t* Rs, int n, int p,
                           const double* rho, const double* fstar, void* states, const SolveParams& prm, int nrhs,
                           cudaStream_t s) {
  mr_init<<<nrhs, kConsumers, 0, s>>>(Y, ldy, X, ldx, Rs, n, p, rho, fstar, static_cast<MrState*>(states), prm);
  return cudaGetLastError();
}
cudaError_t launch_mr_phase_p(const float* G, const float* Gprev, const float* X, long long ldx, float* D,
                              uint16_t* DXs, int p, int nrhs, int k, void* states, const SolveParams& prm,
                              int* restart_cnt, int* restart_list, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mr_phase_p, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sizeof(MrSmem)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return launch_pdl(mr_phase_p, dim3(nrhs), dim3(kConsumers), mr_smem_bytes(p, 2), s, G, Gprev, X, ldx, D, DXs, p,
                    nrhs, k, static_cast<MrState*>(states), prm, MrRestartList{restart_cnt, restart_list});
}
cudaError_t launch_mr_phase_l(float* KD, int splits, long long split_stride, const void* xpart, const float* Y,
                              long long ldy, float* X, long long ldx, const float* D, uint16_t* Rs, int n, int p,
                              int nrhs, int k, void* states, const SolveParams& prm, gpl1_result* res,
                              int* done_count, cudaStream_t s) {
  return launch_pdl(mr_phase_l, dim3(nrhs), dim3(kConsumers), 0, s, KD, splits, split_stride,
                    static_cast<const F2*>(xpart), mr_exact_splits(p), Y, ldy, X, ldx, D, Rs, n, p, k,
                    static_cast<MrState*>(states), prm, res, done_count);
}
size_t mr_exact_part_bytes(int n, int p, int nrhs) {
  return static_cast<size_t>(nrhs) * mr_exact_splits(p) * n * sizeof(F2);
}
cudaError_t launch_mr_exact_kx(const void* Kt, const float* X, long long ldx, void* xpart, int n, int p, int nrhs,
                               const void* states, const int* restart_cnt, const int* restart_list, int k, int num_sms,
                               cudaStream_t s) {
  // persistent over the (listed instance, column range) items of this iteration
  const int grid = std::min(3 * num_sms, nrhs * mr_exact_splits(p));
  return launch_pdl(mr_exact_kx, dim3(grid), dim3(kMrExactThreads), 0, s, static_cast<const uint16_t*>(Kt), X, ldx,
                    static_cast<F2*>(xpart), n, p, mr_exact_splits(p), static_cast<const MrState*>(states),
                    restart_cnt + (k & 1), restart_list + (k & 1) * nrhs);
}
cudaError_t launch_transpose_bf16(const void* K, long long ldk, void* Kt, int n, int p, cudaStream_t s) {
  const dim3 grid((p + 31) / 32, (n + 31) / 32), block(32, 8);
  transpose_bf16<<<grid, block, 0, s>>>(static_cast<const uint16_t*>(K), ldk, static_cast<uint16_t*>(Kt), n, p);
  return cudaGetLastError();
}

}  // namespace gpl1
