// Euclidean projection onto the l1 ball {w : ||w||_1 <= rho}: the P_Omega of
// Algorithm GP, Step 2 (Sec. 3).  The paper uses the projection without giving
// an algorithm; here it is a block-level parallel threshold search, in two
// forms that return the same threshold:
//
//  * block_l1_tau_fixed_point (used first): the fixed-point iteration of
//    Michelot (1986), tau <- (sum_{|v_i| > tau} |v_i| - rho) / #{|v_i| > tau},
//    started from a lower bound of the root.  It increases monotonically and
//    stops exactly when the active set no longer changes, so its result is
//    the exact threshold.  Each step is one block reduction (warp shuffles,
//    no atomics); a warm start from the previous iteration's threshold takes
//    3-5 steps on the solver's vectors.
//
//  * block_l1_tau (the fallback after a capped number of steps): the radix
//    select described next.
//
// The projection of v with ||v||_1 > rho is w = sgn(v) max(|v| - tau, 0) with
// tau > 0 the root of phi(t) = sum_i max(|v_i| - t, 0) = rho.  phi is
// decreasing and piecewise linear.  The search runs a radix select on the IEEE
// bit patterns of |v| (which order like the values): digit by digit, from the
// most significant 11 bits down, it builds a histogram of the candidates with
// counts and sums, evaluates phi at the lower edge of every bucket through a
// suffix scan, and keeps the highest bucket whose lower edge t still has
// phi(t) > rho.  After the last digit the largest bit pattern t* with
// phi(t*) > rho is known; the active set is {|v_i| > t*} and
// tau = (sum over the active set - rho) / (its size).  No sort, no global
// memory traffic beyond reading v.
//
// Every partial sum is an exact integer: |v_i| in fixed point with 2^F, F
// chosen from the largest exponent so that sums of up to 2^20 elements stay
// below 2^63.  Integer addition is associative, so the atomics that build the
// histograms give the same result in any order and every CTA that runs this
// routine on the same data selects the same threshold.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace gpl1 {

template <typename V> struct KeyT;
template <> struct KeyT<float> {
  using K = uint32_t;
  static constexpr int KBITS = 31, MANT = 23, BIAS = 127;
  __device__ static __forceinline__ K key(float v) { return __float_as_uint(v) & 0x7fffffffu; }
};
template <> struct KeyT<double> {
  using K = unsigned long long;
  static constexpr int KBITS = 63, MANT = 52, BIAS = 1023;
  __device__ static __forceinline__ K key(double v) {
    return static_cast<K>(__double_as_longlong(v)) & 0x7fffffffffffffffull;
  }
};

// Histogram of one digit: count and the exact 43-bit fixed-point sum of the
// elements in each bucket, the sum kept as three 32-bit components (bits
// 0-15, 16-31, 32-42) so every update is a native 32-bit shared-memory atomic
// and no component can overflow for up to 2^14.6 elements per block.
struct ProjSmem {
  unsigned cnt[kHistBins];
  unsigned s0[kHistBins];
  unsigned s1[kHistBins];
  unsigned s2[kHistBins];
};
static_assert(35 * kConsumers < (1 << 16), "bucket component sums must fit in 32 bits");

// floor(|v| * 2^F) for the value with bit pattern `key`, F = 42 + BIAS - emax.
template <typename V>
__device__ __forceinline__ unsigned long long to_fixed(typename KeyT<V>::K key, int emax) {
  using KT = KeyT<V>;
  const int e = static_cast<int>(key >> KT::MANT);
  const unsigned long long m =
      static_cast<unsigned long long>(key) & ((1ull << KT::MANT) - 1ull);
  const unsigned long long M = e ? (m | (1ull << KT::MANT)) : m;
  const int s = (e ? e : 1) - emax + (42 - KT::MANT);
  if (s > 62 - KT::MANT) return 0x7fffffffffffffffull;   // above the largest element: never weighed
  if (s >= 0) return M << s;
  return s > -64 ? (M >> (-s)) : 0ull;
}

// Element accessor over values held in registers: element e of this thread is
// global index threadIdx.x + e * kConsumers; missing elements read as 0.
template <typename V, int N>
struct RegAcc {
  static constexpr int ne = N;
  const V (&v)[N];
  int neu;   // slots e >= neu are empty in every thread (uniform bound)
  __device__ V get(int e) const { return v[e]; }
};

struct TauResult {
  double tau;     // threshold, 0 when the input lies inside the ball
  double tstar;   // largest |v| pattern with phi > rho: the active set is {|v| > tstar}
  int inside;     // ||v||_1 <= rho: the projection is the identity
  float th, tl;   // tau as a float pair (set by block_l1_tau_fixed_point)
};

template <typename V> __device__ __forceinline__ double key_value(typename KeyT<V>::K k);
template <> __device__ __forceinline__ double key_value<float>(uint32_t k) { return (double)__uint_as_float(k); }
template <> __device__ __forceinline__ double key_value<double>(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>(k));
}

// Threshold of the projection of the block-distributed vector `acc` onto the
// l1 ball of radius rho > 0.  Called by all kConsumers threads; every thread
// returns the same value.  Elements that are 0 (including padding) never enter
// the active set, so padding does not change the result.
template <typename V, class Acc>
__device__ __noinline__ TauResult block_l1_tau(const Acc& acc, double rho, ProjSmem& ps, Scratch& sc) {
  using KT = KeyT<V>;
  using K = typename KT::K;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  K kmax = 0;
#pragma unroll
  for (int e = 0; e < Acc::ne; ++e) {
    if (e >= acc.neu) break;
    const K k = KT::key(acc.get(e));
    kmax = k > kmax ? k : kmax;
  }
  kmax = static_cast<K>(block_max_u64(static_cast<unsigned long long>(kmax), sc));
  if (kmax == 0) return {0.0, 0.0, 1, 0.f, 0.f};
  int emax = static_cast<int>(kmax >> KT::MANT);
  emax = emax < 1 ? 1 : emax;
  const int F = 42 + KT::BIAS - emax;
  const double rf = ldexp(rho, F);
  const unsigned long long rho_fix =
      rf >= 9.0e18 ? 0x7fffffffffffffffull : static_cast<unsigned long long>(rf);

  K prefix = 0;
  unsigned long long s_above = 0;   // fixed-point sum of elements above the current bucket range
  unsigned c_above = 0;             // their count
  int hi = KT::KBITS;               // bits [hi, KBITS) of the threshold are fixed

  for (int round = 0; hi > 0; ++round) {
    const int bits = hi >= 11 ? 11 : hi;
    const int shift = hi - bits;
    const int nb = 1 << bits;
    for (int b = tid; b < nb; b += kConsumers) {
      ps.cnt[b] = 0;
      ps.s0[b] = 0;
      ps.s1[b] = 0;
      ps.s2[b] = 0;
    }
    consumer_sync();
#pragma unroll
    for (int e = 0; e < Acc::ne; ++e) {
      if (e >= acc.neu) break;
      const K k = KT::key(acc.get(e));
      const bool match = (hi == KT::KBITS) || ((k >> hi) == (prefix >> hi));
      if (match && k != 0) {
        const int b = static_cast<int>((k >> shift) & static_cast<K>(nb - 1));
        const unsigned long long fx = to_fixed<V>(k, emax);
        atomicAdd(&ps.cnt[b], 1u);
        atomicAdd(&ps.s0[b], static_cast<unsigned>(fx & 0xffffu));
        atomicAdd(&ps.s1[b], static_cast<unsigned>((fx >> 16) & 0xffffu));
        atomicAdd(&ps.s2[b], static_cast<unsigned>(fx >> 32));
      }
    }
    consumer_sync();

    // Suffix scan over buckets.  Thread t owns buckets BPT*t .. BPT*t + BPT-1.
    constexpr int BPT = kBinsPerThread;
    unsigned cs[BPT];
    unsigned long long ss[BPT];
    unsigned tc = 0;
    unsigned long long ts = 0;
#pragma unroll
    for (int q = BPT - 1; q >= 0; --q) {
      const int b = BPT * tid + q;
      if (b < nb) {
        tc += ps.cnt[b];
        ts += static_cast<unsigned long long>(ps.s0[b]) + (static_cast<unsigned long long>(ps.s1[b]) << 16) +
              (static_cast<unsigned long long>(ps.s2[b]) << 32);
      }
      cs[q] = tc;
      ss[q] = ts;
    }
    unsigned vc = tc;
    unsigned long long vs = ts;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned oc = __shfl_down_sync(0xffffffffu, vc, o);
      const unsigned long long os = __shfl_down_sync(0xffffffffu, vs, o);
      if (lane + o < 32) {
        vc += oc;
        vs += os;
      }
    }
    if (lane == 0) {
      sc.u[warp][0] = vs;
      sc.u[warp][1] = vc;
    }
    consumer_sync();
    unsigned long long es = vs - ts;   // sum over threads after this one, same warp
    unsigned ec = vc - tc;
    unsigned long long tot_s = 0;
    for (int w = 0; w < kConsumerWarps; ++w) {
      tot_s += sc.u[w][0];
      if (w > warp) {
        es += sc.u[w][0];
        ec += static_cast<unsigned>(sc.u[w][1]);
      }
    }
    if (round == 0 && tot_s <= rho_fix) {   // ||v||_1 <= rho
      consumer_sync();
      return {0.0, 0.0, 1, 0.f, 0.f};
    }
    // phi at the lower edge L_b of each bucket: elements >= L_b contribute (v - L_b).
    int ntrue = 0;
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = BPT * tid + q;
      if (b < nb) {
        const unsigned long long S = s_above + es + ss[q];
        const unsigned long long C = static_cast<unsigned long long>(c_above) + ec + cs[q];
        const K lkey = prefix | (static_cast<K>(b) << shift);
        const unsigned long long L = to_fixed<V>(lkey, emax);
        const unsigned long long phi = S - C * L;
        ntrue += (phi > rho_fix) ? 1 : 0;
      }
    }
    // bucket 0's lower edge always qualifies, so the chosen bucket is ntrue - 1
    int wt = ntrue;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wt += __shfl_xor_sync(0xffffffffu, wt, o);
    consumer_sync();
    if (lane == 0) sc.u[warp][0] = static_cast<unsigned long long>(wt);
    consumer_sync();
    int total = 0;
    for (int w = 0; w < kConsumerWarps; ++w) total += static_cast<int>(sc.u[w][0]);
    const int bstar = total - 1;
    // the suffix sums of bucket bstar + 1 (everything above the chosen bucket)
    if (bstar + 1 == nb) {
      if (tid == 0) {
        sc.ubcast[0] = 0;
        sc.ubcast[1] = 0;
      }
    } else if ((bstar + 1) / BPT == tid) {
      const int q = (bstar + 1) % BPT;
      sc.ubcast[0] = es + ss[q];
      sc.ubcast[1] = ec + cs[q];
    }
    consumer_sync();
    s_above += sc.ubcast[0];
    c_above += static_cast<unsigned>(sc.ubcast[1]);
    prefix |= static_cast<K>(bstar) << shift;
    hi = shift;
    consumer_sync();
  }
  // active set {key > prefix}: tau = (sum - rho) / count
  const double tau = ldexp(static_cast<double>(s_above - rho_fix), -F) / static_cast<double>(c_above);
  return {tau, key_value<V>(prefix), 0, 0.f, 0.f};
}

// FP64 input: recompute the active-set sum exactly in double over the set
// {|v| > tstar} selected above (the fixed-point sums keep 43 bits, enough to
// select the set but short of a 53-bit tau).  Fixed summation order.
template <class Acc>
__device__ double refine_tau_f64(const Acc& acc, double rho, const TauResult& t, Scratch& sc) {
  double s = 0.0, c = 0.0;
#pragma unroll
  for (int e = 0; e < Acc::ne; ++e) {
    if (e >= acc.neu) break;
    const double a = fabs(acc.get(e));
    if (a > t.tstar) {
      s += a;
      c += 1.0;
    }
  }
  double v[2] = {s, c}, o[2];
  block_sum_f64<2>(v, o, sc);
  return o[1] > 0.0 ? (o[0] - rho) / o[1] : t.tau;
}

// tau held as a float pair (hi + lo == tau to ~2^-48): |v| > tau is decided
// exactly as (|v| - hi) > lo, since |v| - hi is exact whenever |v| is within a
// factor 2 of hi (Sterbenz) and far from lo otherwise.
struct TauPair {
  float hi, lo;
  __device__ __forceinline__ bool below(float a) const { return !((a - hi) > lo); }   // a <= tau
};

constexpr int kFixedPointCap = 24;   // steps before falling back to the radix select

// Warp-sum N float pairs, publish the per-warp values, and return (in warp 0
// only, every lane) the block total.  Caller syncs and decides in lane 0.
template <int N>
__device__ __forceinline__ void warp_then_warp0_sum(F2 (&v)[N], Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      F2 t{__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
      v[q] = f2_add(v[q], t);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) sc.f2[warp][q] = v[q];
  consumer_sync();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = lane < kConsumerWarps ? sc.f2[lane][q] : F2{0.f, 0.f};
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < N; ++q) {
        F2 t{__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
        v[q] = f2_add(v[q], t);
      }
  }
}
template <int N>
__device__ __forceinline__ void warp_then_warp0_sum(double (&v)[N], Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) sc.d[warp][q] = v[q];
  consumer_sync();
  if (warp == 0 && lane == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double t = 0.0;
      for (int w = 0; w < kConsumerWarps; ++w) t += sc.d[w][q];
      v[q] = t;
    }
}
__device__ __forceinline__ double as_double(const F2& v) { return static_cast<double>(v.hi) + static_cast<double>(v.lo); }
__device__ __forceinline__ double as_double(double v) { return v; }

// Exact fixed-point value floor(a * 2^F) of a >= 0 with F = 42 + BIAS - eb,
// for eb >= the biased exponent of every value summed: each value is below
// 2^43, so up to 2^20 of them sum below 2^63.
__device__ __forceinline__ unsigned long long fixed43(float a, int eb) {
  const unsigned bits = __float_as_uint(a);
  const int e = static_cast<int>(bits >> 23);
  const unsigned long long M = (bits & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int s = (e ? e : 1) - eb + 19;
  return s >= 0 ? (M << s) : (s > -64 ? (M >> (-s)) : 0ull);
}
__device__ __forceinline__ unsigned long long fixed43(double a, int eb) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(a));
  const int e = static_cast<int>(bits >> 52);
  const unsigned long long M = (bits & 0xfffffffffffffull) | (e ? 0x10000000000000ull : 0ull);
  const int s = (e ? e : 1) - eb - 10;
  return s >= 0 ? (M << s) : (s > -64 ? (M >> (-s)) : 0ull);
}
template <typename V> struct FixedTraits;
template <> struct FixedTraits<float> { static constexpr int BIAS = 127; };
template <> struct FixedTraits<double> { static constexpr int BIAS = 1023; };

// Block sum of N (u64 sum, u32 count) pairs, finished by lane 0 of warp 0
// (the totals are returned there; other threads' values are partial).
template <int N>
__device__ __forceinline__ void warp_then_lead_sum(unsigned long long (&s)[N], unsigned (&c)[N], Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
      c[q] += __shfl_xor_sync(0xffffffffu, c[q], o);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      sc.u2[warp][q] = s[q];
      sc.c2[warp][q] = c[q];
    }
  consumer_sync();
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      s[q] = 0;
      c[q] = 0;
      for (int w = 0; w < kConsumerWarps; ++w) {
        s[q] += sc.u2[w][q];
        c[q] += sc.c2[w][q];
      }
    }
}

// 2^e as a float factor pair (exact; each factor a normal float) for |e| <= 252.
__device__ __forceinline__ void pow2_pair(int e, float& f1, float& f2) {
  const int e1 = e / 2, e2 = e - e1;
  f1 = __int_as_float((127 + e1) << 23);
  f2 = __int_as_float((127 + e2) << 23);
}

// t * 2^-F as a float pair (hi + lo carries ~48 bits), integer and FP32 work only.
__device__ __forceinline__ F2 fixed_to_pair(unsigned long long t, int F) {
  const float h = __ull2float_rz(t);                        // rounded toward zero
  const unsigned long long hi_int = __float2ull_rz(h);      // exact (h is an integer)
  const float l = __ll2float_rn(static_cast<long long>(t - hi_int));
  float f1, f2;
  pow2_pair(-F, f1, f2);
  return {(h * f1) * f2, (l * f1) * f2};
}

// floor-ish (within one unit) of (hi + lo) * 2^F as an unsigned fixed-point
// integer, clamped to 2^62.
__device__ __forceinline__ unsigned long long pair_to_fixed(F2 v, int F) {
  float f1, f2;
  pow2_pair(F, f1, f2);
  const float H = (v.hi * f1) * f2, L = (v.lo * f1) * f2;
  if (!(H < 4.0e18f)) return 1ull << 62;
  if (H <= 0.f) return 0ull;
  const long long r = static_cast<long long>(__float2ull_rn(H)) + __float2ll_rn(L);
  return r > 0 ? static_cast<unsigned long long>(r) : 0ull;
}

// Threshold of the projection of `acc` onto the l1 ball of radius rho by the
// fixed-point iteration (see the top of this file).  The sums that define each
// iterate are exact 43-bit fixed-point integers (so the same in every CTA
// whatever the order) and each iterate tau_fix = floor((S - rho)/C) is kept in
// that fixed point, so it never exceeds the root.  Classification uses tau as
// a float pair (exact, see TauPair); only the few elements above tau are
// converted to fixed point.  The leading lane does the integer division and
// publishes the pair.  Float data involve no FP64 instruction at all (GB300
// issues FP64 at a small fraction of the FP32 rate and with long latency);
// FP64 data get tau recomputed in FP64 over the final active set.
//
// rho is given as a double (FP64 data) and as a float pair (float data).
// vbound >= max |v| when the caller knows one (no extra reduction then);
// hint > 0 is a recent threshold, and 0.9 * hint starts the iteration when
// phi(0.9 hint) >= rho.  Every thread returns the same value; for float data
// only the pair (th, tl) is set, tau = 0.
template <typename V, class Acc>
__device__ __noinline__ TauResult block_l1_tau_fixed_point(const Acc& acc, double rho, F2 rho_p, float hint, ProjSmem& ps,
                                              Scratch& sc, float vbound = 0.f) {
  constexpr int BIAS = FixedTraits<V>::BIAS;
  constexpr bool kF64 = sizeof(V) == 8;
  const bool lead = threadIdx.x == 0;
  if (lead) sc.tt[0] = clock64();
  if (!(vbound > 0.f)) {
    float m = 0.f;
#pragma unroll 4
    for (int e = 0; e < Acc::ne; ++e) {
      if (e >= acc.neu) break;
      m = fmaxf(m, fminf(static_cast<float>(vabs(acc.get(e))), 3.0e38f));
    }
    vbound = block_max_nonneg(m, sc);
    if (vbound == 0.f) return {0.0, 0.0, 1, 0.f, 0.f};
  }
  if (lead) {
    // exponent bound: the float exponent of vbound, +1 for rounding, in V's bias
    const int ef = static_cast<int>(__float_as_uint(fminf(vbound, 3.0e38f)) >> 23) + 1;
    const int eb = ef - 127 + BIAS;
    const int F = 42 + BIAS - eb;
    sc.ub[0] = pair_to_fixed(rho_p, F);                                       // rho
    sc.ub[1] = hint > 0.f ? pair_to_fixed(F2{0.9f * hint, 0.f}, F) : 0ull;   // warm start t_w
    const F2 tp = fixed_to_pair(sc.ub[1], F);                                 // t_w as classified
    sc.tp[0] = tp.hi;
    sc.tp[1] = tp.lo;
    sc.flags[1] = eb;
    sc.flags[3] = F;
    sc.tt[1] = clock64();
  }
  consumer_sync();
  const int eb = sc.flags[1];
  const unsigned long long rho_fix = sc.ub[0];
  // step 0: sums over |v| > t_w (warm start); if that is not a valid start,
  // a second pass over all elements gives ||v||_1 and the cold start.
  for (int pass = 0; pass < 2; ++pass) {
    const TauPair tw{sc.tp[0], sc.tp[1]};
    const bool cold = kF64 || pass == 1 || sc.ub[1] == 0;
    unsigned long long sv[1] = {0};
    unsigned cv[1] = {0};
#pragma unroll 4
    for (int e = 0; e < Acc::ne; ++e) {
      if (e >= acc.neu) break;
      const V a = vabs(acc.get(e));
      if (cold ? a > V(0) : !tw.below(static_cast<float>(a))) {
        sv[0] += fixed43(a, eb);
        ++cv[0];
      }
    }
    if (lead) sc.tt[2] = clock64();
    warp_then_lead_sum<1>(sv, cv, sc);
    if (lead) {
      sc.tt[3] = clock64();
      int flag = 0;   // 0 continue, 1 inside, 4 retry cold
      const unsigned long long twf = cold ? 0ull : sc.ub[1];
      if (cold && sv[0] <= rho_fix) {
        flag = 1;
      } else if (!cold && (cv[0] == 0 || sv[0] - twf * cv[0] < rho_fix)) {
        flag = 4;     // phi(t_w) < rho: t_w is above the root
      } else {
        const unsigned long long t = (sv[0] - rho_fix) / cv[0];   // a Michelot iterate, <= the root
        const F2 tp = fixed_to_pair(t, sc.flags[3]);
        sc.tp[2] = tp.hi;
        sc.tp[3] = tp.lo;
        sc.cnt_prev = cv[0];
      }
      sc.tflag = flag;
      sc.tt[4] = clock64();
    }
    consumer_sync();
    if (sc.tflag != 4) break;
  }
  if (sc.tflag == 1) {
    consumer_sync();
    return {0.0, 0.0, 1, 0.f, 0.f};
  }
  // Later steps only look at elements above the current iterate, which bounds
  // the root from below, so they form a superset of the final active set.
  // Compact them into shared memory (the radix-select area, unused here) when
  // they fit; the sums stay exact integers, so the order of the list does not
  // matter.
  V* const cand = reinterpret_cast<V*>(&ps);
  constexpr int kCandCap = static_cast<int>(sizeof(ProjSmem) / sizeof(V));
  if (lead) sc.flags[2] = 0;   // candidate count
  consumer_sync();
  {
    const TauPair tp{sc.tp[2], sc.tp[3]};
    const V tdv = static_cast<V>(static_cast<double>(tp.hi) + static_cast<double>(tp.lo));
#pragma unroll 4
    for (int e = 0; e < Acc::ne; ++e) {
      if (e >= acc.neu) break;
      const V a = vabs(acc.get(e));
      const bool take = kF64 ? a > tdv : !tp.below(static_cast<float>(a));
      const unsigned m = __ballot_sync(0xffffffffu, take);   // e-loop bound is block-uniform
      if (m) {
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == 0) base = atomicAdd(&sc.flags[2], __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int slot = base + __popc(m & ((1u << lane) - 1u));
        if (take && slot < kCandCap) cand[slot] = a;
      }
    }
  }
  consumer_sync();
  const int ncand = sc.flags[2];
  const bool compact = ncand <= kCandCap;
  if (lead) {
    sc.tt[5] = clock64();
    sc.tt[7] = ncand;
  }
  consumer_sync();
  for (int step = 0; step < kFixedPointCap; ++step) {
    const TauPair tp{sc.tp[2], sc.tp[3]};
    const V tdv = static_cast<V>(static_cast<double>(tp.hi) + static_cast<double>(tp.lo));
    unsigned long long sa[1] = {0};
    unsigned ca[1] = {0};
    if (compact) {
      for (int c = threadIdx.x; c < ncand; c += kConsumers) {
        const V a = cand[c];
        if (kF64 ? a > tdv : !tp.below(static_cast<float>(a))) {
          sa[0] += fixed43(a, eb);
          ++ca[0];
        }
      }
    } else {
#pragma unroll 4
      for (int e = 0; e < Acc::ne; ++e) {
        if (e >= acc.neu) break;
        const V a = vabs(acc.get(e));
        if (kF64 ? a > tdv : !tp.below(static_cast<float>(a))) {
          sa[0] += fixed43(a, eb);
          ++ca[0];
        }
      }
    }
    warp_then_lead_sum<1>(sa, ca, sc);
    if (lead) {
      if (ca[0] == 0 || sa[0] <= rho_fix) {
        sc.tflag = 3;   // cannot happen in exact arithmetic; take the radix select
      } else if (ca[0] == sc.cnt_prev) {   // active set unchanged: converged
        sc.tflag = 2;
        const F2 t = fixed_to_pair((sa[0] - rho_fix) / ca[0], sc.flags[3]);
        sc.tp[2] = t.hi;
        sc.tp[3] = t.lo;
      } else {
        const F2 t = fixed_to_pair((sa[0] - rho_fix) / ca[0], sc.flags[3]);
        sc.tp[2] = t.hi;
        sc.tp[3] = t.lo;
        sc.cnt_prev = ca[0];
      }
      sc.flags[1] = step + 1;   // steps (eb is no longer needed by the lead)
    }
    consumer_sync();
    if (sc.tflag == 3) break;
    if (sc.tflag == 2) {
      double tau = 0.0;
      if constexpr (kF64) {   // FP64 data: tau in FP64 over the final set
        const double tcmp = static_cast<double>(tp.hi) + static_cast<double>(tp.lo);
        double v2[2] = {0.0, 0.0};
        if (compact) {
          for (int c = threadIdx.x; c < ncand; c += kConsumers) {
            const double a = static_cast<double>(cand[c]);
            if (a > tcmp) { v2[0] += a; v2[1] += 1.0; }
          }
        } else {
          for (int e = 0; e < acc.neu; ++e) {
            const double a = fabs(static_cast<double>(acc.get(e)));
            if (a > tcmp) { v2[0] += a; v2[1] += 1.0; }
          }
        }
        warp_then_warp0_sum<2>(v2, sc);
        if (lead) {
          sc.dtau = (v2[0] - rho) / v2[1];
          const F2 t = f2_of(sc.dtau);
          sc.tp[2] = t.hi;
          sc.tp[3] = t.lo;
        }
        consumer_sync();
        tau = sc.dtau;
      }
      const TauResult r{tau, 0.0, 0, sc.tp[2], sc.tp[3]};
      if (lead) {
        sc.flags[2] = sc.flags[1];   // report the step count
        sc.tt[6] = clock64();
      }
      consumer_sync();
      return r;
    }
  }
  // not settled after the cap (pathological spacing): exact radix select
  consumer_sync();
  TauResult r = block_l1_tau<V>(acc, rho, ps, sc);
  if constexpr (kF64) {
    if (!r.inside) r.tau = refine_tau_f64(acc, rho, r, sc);
  }
  if (lead) {
    const F2 t = f2_of(r.tau);
    sc.tp[2] = t.hi;
    sc.tp[3] = t.lo;
  }
  consumer_sync();
  r.th = sc.tp[2];
  r.tl = sc.tp[3];
  consumer_sync();
  return r;
}

}  // namespace gpl1
