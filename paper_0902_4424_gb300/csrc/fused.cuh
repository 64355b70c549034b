// One-read GPSS solver kernel: Algorithm GP with Algorithm SS (Sec. 3) for
//     min f(x) = ||K x - y||^2   s.t.  ||x||_1 <= rho          (eq. 2),
// reading K once per iteration.
//
// Why one read suffices.  The gradient is linear in the iterate: with
// x_{k+1} = x_k + lam_k d_k (Alg. GP, Step 6),
//     g_{k+1} = 2 K^T (K x_k - y) + lam_k 2 K^T (K d_k).
// Both K^T products can be formed in the same pass that forms K x_k and K d_k,
// row block by row block, while the block is still in shared memory: once the
// row sums (K x)_i, (K d)_i of a block are complete, the block's contribution
// 2 K_i^T (r_i, (K d)_i) to both gradients is accumulated from the same tile.
// The steplength lam_k (Armijo, Step 5) only scales the second vector, so the
// line search runs after the pass on scalars.
//
// Layout of the work.
//   * A cluster of C CTAs owns a contiguous range of row blocks (R rows each);
//     CTA rank r of every cluster owns the column slice [r W, r W + W), so the
//     C CTAs of a cluster together cover all p columns and every cluster holds
//     one copy of x, d and g, distributed over its CTAs.
//   * Thread t of a CTA owns NCH 16-byte chunks of the slice (chunk t + 256 m)
//     and keeps x, d, g and the two gradient accumulators of its columns in
//     registers for the whole solve.
//   * A row block arrives through TMA (boxes of 256 columns x R rows).  Each
//     thread forms its partial row sums, each consumer warp reduces them, the
//     sender warp adds the CTA's partials of a chunk of blocks and sends them
//     to every CTA of the cluster through distributed shared memory (bulk
//     copies with an mbarrier transaction count), and the totaler warp adds
//     the C messages in rank order, so all CTAs of a cluster hold
//     bit-identical row sums.  kLagC chunks later the same blocks arrive again
//     (from L2) and each thread accumulates K_i^T of them into its columns, so
//     the exchange of a chunk overlaps the next chunks' work.
//   * At the end of the pass every CTA adds its gradient accumulators into a
//     global buffer (vector reductions at L2) and its scalar partials into a
//     per-CTA record; one grid barrier follows.
//   * Then every CTA runs the line search on the summed scalars (all CTAs get
//     the same values: fixed summation order) and the next projection phase on
//     its own columns.  Block sums needed by Alg. SS and the projection
//     threshold are reduced over the CTA and then over the cluster through
//     distributed shared memory; the threshold search uses exact fixed-point
//     integer sums (Michelot's fixed-point iteration), so every cluster finds
//     the same threshold.
//
// Per iteration: one read of K, one grid barrier, a handful of cluster
// reductions.  Every wait is bounded by timeout_ns; a wait that runs out
// records its site, raises the launch's error flag and skips the remaining
// work, so the kernel returns an error status instead of hanging.
#pragma once

#include "gpss.cuh"   // SolveParams, Dir, the stop and error conventions of the two-pass kernel

namespace gpl1 {
namespace fz {

constexpr int kWarps = 8;               // consumer warps (two or four column chunks per thread:
                                        // fewer warps with more registers each beat 16 warps
                                        // of one chunk, 4.18 against 4.50 ms on c1)
constexpr int kCons = kWarps * 32;      // consumer threads
constexpr int kThr = kCons + 96;        // + TMA producer warp, sender warp, totaler warp
constexpr int kProd = kCons;            // first thread of the producer warp
constexpr int kSend = kCons + 32;       // ... of the sender warp
constexpr int kTot = kCons + 64;        // ... of the totaler warp
// The ring shape (stages, row-block bytes, blocks per chunk) is per dtype: see
// Cfg.  Float data: row blocks of 64 KB per CTA (8 rows FP32) through two HBM
// stages and one L2 stage; taller blocks halve the per-block waits and
// reductions (3.50 against 3.89 ms on c1 with 4-row blocks in a 3 + 2 ring).
// FP64 data (c0-sized, latency-bound solves): 32 KB blocks in a 3 + 2 ring.
constexpr int CTL_ISSUED_B = 7;         // (sm.ctl) loads issued into the B ring
constexpr int kBoxW = 256;              // TMA box width (elements)
constexpr int kCMax = 16;               // CTAs per cluster
constexpr int kLagC = 2;                // chunks between a chunk's row sums and its K^T step (3: 2.4 % slower on c1, 1: 17 %)
constexpr int kNRed = kLagC + 1;        // chunk slots of the warp partials
constexpr int kRNS = 5;                 // chunk slots of the row-sum channel (> kLagC + 1)
constexpr int kNTot = 3;                // chunk slots of the published row multipliers
constexpr int kRCW = 64;                // words per CTA of one chunk's row sums (at most)
constexpr uint32_t kSleepNs = 20000;    // suspend hint of a blocking mbarrier wait
constexpr int kSNS = 3;                 // slots of the scalar channel
constexpr int kRWMax = 16;              // words per CTA of one row-sum message
constexpr int kSWMax = 8;               // words per CTA of one scalar message
constexpr int kBW = 12;                 // words of a block reduction
constexpr int kPartW = 16;              // words of a CTA's record of pass scalars
constexpr int kTauCap = 400;            // threshold-search steps before giving up
constexpr int kStallIters = 64;         // iterations without progress near the stop (stagnation)

// Where a bounded wait gave up (gpl1_result.fail_site); 1-5 as the two-pass kernel.
enum { kSiteRowMsg = 6, kSiteScalarMsg = 7, kSiteRed = 8 };

template <int DT, int NCH>
struct Cfg {
  using T = Traits<DT>;
  using A = typename T::A;   // arithmetic of products with K and of x, d, g
  using V = typename T::V;   // element of x and y in memory
  static constexpr bool kF64 = DT == GPL1_F64;
  static constexpr int ES = T::ES;
  static constexpr int EPC = 16 / ES;                  // elements per 16-byte chunk
  static constexpr int NE = EPC * NCH;                 // columns per thread
  static constexpr int W = kCons * NE;                 // columns per CTA (slice)
  static constexpr int SB = kF64 ? 32768 : 65536;      // bytes of a row block of the slice
  static constexpr int NSA = kF64 ? 3 : 2;             // stages of the ring from HBM (A steps)
  static constexpr int NSB = kF64 ? 2 : 1;             // stages of the ring from L2 (B steps)
  static constexpr int NST = NSA + NSB;
  static constexpr int CB = kF64 ? 4 : 2;              // row blocks per chunk (one row-sum exchange each)
  static constexpr int R = SB / (W * ES);              // rows per block
  static constexpr int NBOX = W / kBoxW;               // TMA boxes per block
  static constexpr int BOXB = kBoxW * R * ES;          // bytes per box
  static constexpr int RWPR = kF64 ? 4 : 3;            // message words per row
  static constexpr int RW = RWPR * R;                  // row-sum words per block
  static constexpr int RC = R * CB;                    // rows per chunk
  static constexpr int RCW = RWPR * RC;                // row-sum words per chunk
  static constexpr int RCWP = (RCW + 3) & ~3;          // padded to 16 bytes
  static_assert(R >= 1 && R * W * ES == SB, "a stage holds whole rows");
  static_assert(RCWP <= kRCW, "row message too long");
  static_assert(RC <= 32, "a chunk's rows fit a warp");
  static_assert(kBoxW % EPC == 0, "a chunk never straddles two boxes");
};

// Kernel arguments.  U: [3][2][pp] gradient accumulators (A), rotating:
// the pass of iteration k adds into U[k % 3] and the buffer of k + 2 is
// cleared during iteration k + 1.  parts: [2][G][kPartW] words of per-CTA
// pass scalars (alternating).
struct FArgs {
  const void* y;
  void* x;
  double rho, f_star;
  int n, p, x0_zero, C;
  int NC;                   // clusters
  int pad_;
  void* U;
  long long pp;             // C * W
  unsigned* parts;
  unsigned* bar;            // grid barrier counter
  int* err;                 // sticky error flag of the launch
  gpl1_result* res;
  double* trace;
  long long trace_cap;
  SolveParams prm;
};

// ------------------------------------------------------------ PTX: clusters
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }
// shared::cluster address of `local` in the CTA of cluster rank `rank`
__device__ __forceinline__ uint32_t mapa(const void* local, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async4(uint32_t raddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                          uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   raddr),
               "r"(a), "r"(b), "r"(c), "r"(d), "r"(rbar)
               : "memory");
}
// bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to the
// shared memory of a CTA of the cluster, completing on that CTA's mbarrier
__device__ __forceinline__ void bulk_to_cluster(uint32_t rdst, const void* src, uint32_t bytes, uint32_t rbar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(rdst),
               "r"(smem_u32(src)), "r"(bytes), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_remote(uint32_t rbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// test_wait: never blocks (busy polling, for latency-critical waits).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend hint: the thread sleeps until the phase completes or
// the hint runs out, instead of spinning.
__device__ __forceinline__ bool mbar_wait_h(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSleepNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_h_cl(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSleepNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
// the consumer warps' barrier (named barrier 2; the producer warp never joins)
__device__ __forceinline__ void csync() { asm volatile("barrier.sync 2, %0;" ::"n"(kCons) : "memory"); }

// 16 bytes of a staged row, widened to the arithmetic type
template <int DT>
__device__ __forceinline__ void widen16(const uint8_t* p, typename Traits<DT>::A (&o)[16 / Traits<DT>::ES]);
template <>
__device__ __forceinline__ void widen16<GPL1_F32>(const uint8_t* p, float (&o)[4]) {
  const float4 c = *reinterpret_cast<const float4*>(p);
  o[0] = c.x;
  o[1] = c.y;
  o[2] = c.z;
  o[3] = c.w;
}
template <>
__device__ __forceinline__ void widen16<GPL1_BF16>(const uint8_t* p, float (&o)[8]) {
  const uint4 c = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[2 * q] = __uint_as_float(w[q] << 16);
    o[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
  }
}
template <>
__device__ __forceinline__ void widen16<GPL1_F64>(const uint8_t* p, double (&o)[2]) {
  const double2 c = *reinterpret_cast<const double2*>(p);
  o[0] = c.x;
  o[1] = c.y;
}

// x, y elements from global memory (bypassing L1: other CTAs write them)
__device__ __forceinline__ float ldg_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ float sum_pair(float a, float b) { return a + b; }
__device__ __forceinline__ double sum_pair(double a, double b) { return a + b; }

// Warp butterfly sums / maxima (every lane gets the result; fixed order).
__device__ __forceinline__ F2 wsum(F2 v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) {
    const F2 t{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = f2_add(v, t);
  }
  return v;
}
__device__ __forceinline__ double wsum(double v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long wsum(unsigned long long v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned wsumu(unsigned v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned wmaxu(unsigned v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned worr(unsigned v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sum of NV doubles at once (halving butterfly, as warp_sum_many).
template <int NV>
__device__ __forceinline__ double warp_sum_many_d(double (&v)[NV], int lane) {
  int o = 16;
#pragma unroll
  for (int n = NV; n > 1; n >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const double send = upper ? v[i] : v[i + n / 2];
      const double keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

// Scalar state of Alg. GP + SS (written by consumer thread 0 between two
// consumer barriers, read by every consumer thread after the second).
struct FState {
  double alpha, lam, f_cur, gd, dd, kb2, gmax, gx, gap_den, yy;
  double tau_ss, ss_prev, sz_prev;   // Alg. SS in FP64
  double a2win[kMaxMalpha];
  int a2cnt;
  float ah, al, th, tl, lf, vbound, gmaxf, xscale;
  double xscale_d;
  F2 rho_p;
  float hint;                        // previous threshold (warm start of the search)
  double tau64;                      // FP64 threshold (FP64 data)
  double fhist[kMaxM];
  int stop, iters, backtracks, inside, status, done, acc, nz;
  int tau_steps;
  unsigned long long ts[10];
  // comparison methods (Sec. 2): objective of the method's problem at x_k,
  // ||g_k||^2 and ||K g_k||^2 (PSD), and the coefficient of U2 in the next
  // gradient (1 after a pass along x_{k+1} - x_k, 0 after the setup or a probe)
  double F_cur, gg, kb2p;
  int cpass;
  // stagnation near the stop: the lowest f so far and the iterations since it
  // last fell by more than 1e-3 tol of the gap denominator
  double f_best;
  int stall;
};

template <int DT, int NCH>
struct alignas(128) FSmem {
  uint8_t stage[Cfg<DT, NCH>::NST][Cfg<DT, NCH>::SB];
  uint32_t red[kNRed][kWarps][kRCW];      // warp partials of a chunk's row sums
  uint32_t rx[kRNS][kCMax][kRCW];         // row-sum messages, one row per sender rank
  uint32_t xout[kRNS][kRCW];              // this CTA's outgoing messages (bulk-copied to the cluster)
  uint32_t sx[kSNS][kCMax][kSWMax];       // scalar messages
  uint32_t wred[kWarps][kBW];             // warp partials of block reductions
  uint32_t bc[2][kBW];                    // block/cluster reduction results (alternating)
  uint64_t full[Cfg<DT, NCH>::NST], empty[Cfg<DT, NCH>::NST];
  uint64_t redfull[kNRed];
  uint64_t rfull[kRNS], rempty[kRNS];
  uint64_t tfull[kNTot], tcons[kNTot];
  uint32_t tot[kNTot][128];               // per chunk: 2 K^T multipliers 2 r_i, 2 (K d)_i of its rows
  uint32_t ysm[kNRed][32][3];             // per chunk: y_i and "row i < n" of its rows
  uint32_t bmode[kNRed];                  // per chunk: compensated (1) or plain (0) sums
  uint32_t rowacc[32][6];                 // the pass's row scalars, rows q mod RC (cluster rank 0)
  uint64_t sfull[kSNS], sempty[kSNS];
  FState st;
  int ctl[8];
};

}  // namespace fz
}  // namespace gpl1

namespace gpl1 {
namespace fz {

// ------------------------------------------------------------ word packing
__device__ __forceinline__ void put(uint32_t* w, const F2& v) {
  w[0] = __float_as_uint(v.hi);
  w[1] = __float_as_uint(v.lo);
}
__device__ __forceinline__ void put(uint32_t* w, double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  w[0] = static_cast<uint32_t>(b);
  w[1] = static_cast<uint32_t>(b >> 32);
}
__device__ __forceinline__ void put(uint32_t* w, float v) {
  w[0] = __float_as_uint(v);
  w[1] = 0u;
}
__device__ __forceinline__ void put(uint32_t* w, unsigned long long v) {
  w[0] = static_cast<uint32_t>(v);
  w[1] = static_cast<uint32_t>(v >> 32);
}
__device__ __forceinline__ F2 get_f2(const uint32_t* w) { return F2{__uint_as_float(w[0]), __uint_as_float(w[1])}; }
__device__ __forceinline__ double get_d(const uint32_t* w) {
  return __longlong_as_double(static_cast<long long>(static_cast<unsigned long long>(w[0]) |
                                                     (static_cast<unsigned long long>(w[1]) << 32)));
}
__device__ __forceinline__ unsigned long long get_u64(const uint32_t* w) {
  return static_cast<unsigned long long>(w[0]) | (static_cast<unsigned long long>(w[1]) << 32);
}

// Combiners of packed words (a op= b).  Each op is commutative bit for bit
// (two-sum based pair addition, IEEE addition, integer addition, max, or), so a
// butterfly leaves the same value in every lane, and all-zero words are the
// identity.  NS sums (float pairs or doubles) followed by NM maxima of
// non-negative values given as their bits (32-bit words, or 64-bit words in
// two 32-bit halves when M64: doubles), then NO bitwise ors.
template <typename S, int NS, int NM, int NO, bool M64 = false>
struct Comb {
  static constexpr int MW = M64 ? 2 : 1;
  static constexpr int NW = 2 * NS + MW * NM + NO;
  __device__ static void op(uint32_t (&a)[NW], const uint32_t (&b)[NW]) {
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      if constexpr (std::is_same<S, F2>::value) put(a + 2 * i, f2_add(get_f2(a + 2 * i), get_f2(b + 2 * i)));
      else put(a + 2 * i, get_d(a + 2 * i) + get_d(b + 2 * i));
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      if constexpr (M64) {
        const unsigned long long x = get_u64(a + 2 * NS + 2 * i), y = get_u64(b + 2 * NS + 2 * i);
        put(a + 2 * NS + 2 * i, x > y ? x : y);
      } else {
        a[2 * NS + i] = max(a[2 * NS + i], b[2 * NS + i]);
      }
    }
#pragma unroll
    for (int i = 0; i < NO; ++i) a[2 * NS + MW * NM + i] |= b[2 * NS + MW * NM + i];
  }
};
// bits of a non-negative value (ordered like the values) for the maxima above
__device__ __forceinline__ void put_max(uint32_t* w, float v) { w[0] = __float_as_uint(v); }
__device__ __forceinline__ void put_max(uint32_t* w, double v) {
  put(w, static_cast<unsigned long long>(__double_as_longlong(v)));
}
__device__ __forceinline__ float get_max_f(const uint32_t* w) { return __uint_as_float(w[0]); }
__device__ __forceinline__ double get_max_d(const uint32_t* w) {
  return __longlong_as_double(static_cast<long long>(get_u64(w)));
}
// fixed-point threshold sums: (u64 sum, u32 count)
struct CombFix {
  static constexpr int NW = 3;
  __device__ static void op(uint32_t (&a)[3], const uint32_t (&b)[3]) {
    put(a, get_u64(a) + get_u64(b));
    a[2] += b[2];
  }
};

// ================================================================= consumers
template <int DT, int NCH>
struct FC {
  using CF = Cfg<DT, NCH>;
  using A = typename CF::A;
  using V = typename CF::V;
  static constexpr bool kF64 = CF::kF64;
  static constexpr int NE = CF::NE, EPC = CF::EPC, R = CF::R, W = CF::W, RWPR = CF::RWPR, RW = CF::RW,
                       RC = CF::RC, RCW = CF::RCW, RCWP = CF::RCWP, ES = CF::ES;
  using S = typename std::conditional<kF64, double, F2>::type;

  const FArgs& a;
  FSmem<DT, NCH>& sm;
  const int tid, lane, warp;
  const unsigned rank, cid;
  const int C, NC, G, cta, n, p;
  int bk0, bk1;
  uint32_t rseq = 0, sseq = 0;
  // stage and phase of the next block of each ring (A: from HBM, B: from L2)
  uint32_t sta = 0, pha = 0, stb = 0, phb = 0;
  unsigned epoch = 0;
  int bsl = 0;
  int status = GPL1_OK;

  A x[NE], d[NE], g[NE], u1[NE], u2[NE];
  double tk = 1.0;  // FISTA's t_k (every thread keeps the same sequence)
  bool cv[NCH];
  int gcol[NCH];    // global column of the chunk's first element
  int soff[NCH];    // byte offset of the chunk in row 0 of a stage

  // column partials of the direction (formed in the projection phase, used by
  // the line search after the next pass): g^T d, ||d||^2, d != 0
  S c_gd{}, c_dd{};
  unsigned c_nz = 0;

  __device__ FC(const FArgs& a_, FSmem<DT, NCH>& sm_)
      : a(a_), sm(sm_), tid(threadIdx.x), lane(threadIdx.x & 31), warp(threadIdx.x >> 5), rank(cl_rank()),
        cid(cl_id()), C(a_.C), NC(a_.NC), G(a_.C * a_.NC), cta(static_cast<int>(cl_id()) * a_.C + static_cast<int>(cl_rank())),
        n(a_.n), p(a_.p) {
    const int NBt = (n + R - 1) / R;
    bk0 = static_cast<int>(static_cast<long long>(NBt) * cid / NC);
    bk1 = static_cast<int>(static_cast<long long>(NBt) * (cid + 1) / NC);
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
      const int c = (tid + kCons * m) * EPC;   // slice column
      gcol[m] = static_cast<int>(rank) * W + c;
      cv[m] = gcol[m] < p;
      soff[m] = (c / kBoxW) * CF::BOXB + (c % kBoxW) * ES;
    }
  }

  __device__ FState& S_() { return sm.st; }
  __device__ bool failed() const { return reinterpret_cast<volatile const int*>(sm.ctl)[CTL_ERR] != 0; }
  __device__ void set_err(int site, int code = GPL1_ERR_TIMEOUT) {
    volatile int* ctl = sm.ctl;
    if (!ctl[CTL_ERR]) ctl[CTL_SITE] = site;
    ctl[CTL_ERR] = code;
    atomicCAS(a.err, 0, code);
  }

  // Bounded wait of a whole warp on an mbarrier phase.  Lane 0 polls (and gives
  // up after timeout_ns, or when this CTA or the launch has failed); on success
  // every lane then takes the completed phase itself, which orders its reads
  // after the writes the phase covers (acquire at cluster scope for barriers
  // that complete on other CTAs' messages).
  __device__ bool poll(uint64_t* bar, uint32_t par, bool cl, bool spin) {
    if (spin) return cl ? mbar_test_cl(bar, par) : mbar_test(bar, par);
    return cl ? mbar_wait_h_cl(bar, par) : mbar_wait_h(bar, par);
  }
  // spin: poll without sleeping (for the waits on the critical path of the
  // row-sum exchange, where the wake-up of a suspended warp would add latency)
  __device__ bool wwait(uint64_t* bar, uint32_t par, int site, bool cl, bool spin = false) {
    // fast path: the phase is already complete; every lane takes it itself
    if (__all_sync(0xffffffffu, poll(bar, par, cl, spin))) return true;
    int ok = 1;
    if (lane == 0) {
      if (failed()) {
        ok = 0;
      } else if (!poll(bar, par, cl, spin)) {
        const uint64_t t0 = globaltimer();
        for (unsigned it = 0;; ++it) {
          if (poll(bar, par, cl, spin)) break;
          if (spin && (it & 63u) != 63u) continue;
          if (failed() || ld_volatile(a.err)) {
            ok = 0;
            break;
          }
          if (globaltimer() - t0 > static_cast<uint64_t>(a.prm.timeout_ns)) {
            ok = 0;
            break;
          }
        }
        if (!ok) set_err(site, ld_volatile(a.err) ? ld_volatile(a.err) : GPL1_ERR_TIMEOUT);
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    for (int spin = 0; spin < (1 << 20) && !(cl ? mbar_try_wait_cl(bar, par) : mbar_try_wait(bar, par)); ++spin) {
    }
    return true;
  }

  // A wait of an exchange warp for its next piece of work: as wwait, but it
  // also ends (returning false) when the consumers stop the solve, and its
  // bound counts from the last piece of work.
  __device__ bool xwait(uint64_t* bar, uint32_t par, bool cl) {
    int ok = 1;
    if (lane == 0) {
      volatile int* ctl = sm.ctl;
      const uint64_t t0 = globaltimer();
      for (;;) {
        if (cl ? mbar_wait_h_cl(bar, par) : mbar_wait_h(bar, par)) break;
        if (ctl[CTL_STOP] || failed()) {
          ok = 0;
          break;
        }
        if (globaltimer() - t0 > static_cast<uint64_t>(a.prm.timeout_ns)) {
          set_err(kSiteRed);
          ok = 0;
          break;
        }
      }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    for (int spin = 0; spin < (1 << 20) && !(cl ? mbar_try_wait_cl(bar, par) : mbar_try_wait(bar, par)); ++spin) {
    }
    return true;
  }

  // ---------------------------------------------------- grid barrier
  // Thread 0 arrives on the launch's counter with release semantics after
  // the CTA's writes (the consumer barrier before it orders the other
  // threads' writes, the fence makes them visible at GPU scope) and polls
  // with a bound; the outcome (including another CTA's failure) is broadcast.
  __device__ bool gsync() {
    csync();
    if (tid == 0) {
      int e = reinterpret_cast<volatile int*>(sm.ctl)[CTL_ERR];
      if (G > 1) {
        if (e) atomicCAS(a.err, 0, e);
        ++epoch;
        __threadfence();
        red_release_add(a.bar, 1u);
        const unsigned target =
            epoch * static_cast<unsigned>(G) + ((a.prm.debug & kDebugUnreachableBarrier) ? 1u : 0u);
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
      if (e && !sm.ctl[CTL_ERR]) sm.ctl[CTL_ERR] = e;
      sm.bc[bsl][0] = static_cast<uint32_t>(e);
    }
    csync();
    const int e = static_cast<int>(sm.bc[bsl][0]);
    bsl ^= 1;
    if (e) status = e;
    return e == 0;
  }

  // ---------------------------------------------------- scalar channel
  // Warp 0 sends its NW words (identical in every lane) to every CTA of the
  // cluster and returns, in lane r < C, the words of rank r (zeros in the
  // other lanes).  Slot reuse is guarded by a handshake: a CTA writes into
  // its peers' slot only after all of them have released it.
  template <int NW>
  __device__ bool sx_exchange(uint32_t (&v)[NW]) {
    constexpr int NWP = (NW + 3) & ~3;
    static_assert(NWP <= kSWMax, "scalar message too long");
    const uint32_t slot = sseq % kSNS, use = sseq / kSNS;
    ++sseq;
    bool ok = true;
    if (use >= 1) ok = wwait(&sm.sempty[slot], (use - 1) & 1u, kSiteScalarMsg, true);
    if (ok) {
      if (lane == 0) mbar_arrive_expect_tx(&sm.sfull[slot], static_cast<uint32_t>(C * NWP * 4));
      if (lane < C) {
        const uint32_t raddr = mapa(&sm.sx[slot][rank][0], static_cast<unsigned>(lane));
        const uint32_t rbar = mapa(&sm.sfull[slot], static_cast<unsigned>(lane));
#pragma unroll
        for (int c = 0; c < NWP; c += 4) {
          uint32_t q[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) q[i] = c + i < NW ? v[c + i] : 0u;
          st_async4(raddr + 4 * c, q[0], q[1], q[2], q[3], rbar);
        }
      }
      ok = wwait(&sm.sfull[slot], use & 1u, kSiteScalarMsg, true);
    }
#pragma unroll
    for (int i = 0; i < NW; ++i) v[i] = (ok && lane < C) ? sm.sx[slot][lane][i] : 0u;
    __syncwarp();
    if (ok && lane < C) mbar_arrive_remote(mapa(&sm.sempty[slot], static_cast<unsigned>(lane)));
    return ok;
  }

  // Block (and, with cl, cluster) reduction of packed words; every consumer
  // thread gets the total.  The summation order is fixed (butterflies over
  // lanes, warps in lanes, ranks in lanes), so every CTA of a cluster, and
  // every cluster given the same inputs, gets bit-identical totals.
  template <class Cb>
  __device__ void reduce(uint32_t (&w)[Cb::NW], bool cl) {
    constexpr int NW = Cb::NW;
    static_assert(NW <= kBW, "too many words");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      uint32_t t[NW];
#pragma unroll
      for (int i = 0; i < NW; ++i) t[i] = __shfl_xor_sync(0xffffffffu, w[i], o);
      Cb::op(w, t);
    }
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < NW; ++i) sm.wred[warp][i] = w[i];
    csync();
    if (warp == 0) {
      uint32_t v[NW];
#pragma unroll
      for (int i = 0; i < NW; ++i) v[i] = lane < kWarps ? sm.wred[lane][i] : 0u;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        uint32_t t[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) t[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
        Cb::op(v, t);
      }
      if (cl && C > 1) {
        if constexpr (NW <= kSWMax) {
          sx_exchange<NW>(v);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            uint32_t t[NW];
#pragma unroll
            for (int i = 0; i < NW; ++i) t[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
            Cb::op(v, t);
          }
        }
      }
      if (lane == 0)
#pragma unroll
        for (int i = 0; i < NW; ++i) sm.bc[bsl][i] = v[i];
    }
    csync();
#pragma unroll
    for (int i = 0; i < NW; ++i) w[i] = sm.bc[bsl][i];
    bsl ^= 1;
  }

  // One step of the threshold search after the local sums: reduce (s, c) over
  // the cluster, then lane 0 of warp 0 alone takes the decision (64-bit
  // division and conversions are long instruction sequences) and publishes
  // it: w = {s lo, s hi, c, next iterate lo, hi, its float pair hi, lo}.
  __device__ void tau_reduce(unsigned long long& s, unsigned& c, unsigned long long rho_fix, int F,
                             unsigned long long& tn, F2& tp) {
    uint32_t w[3];
    put(w, s);
    w[2] = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      uint32_t t[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = __shfl_xor_sync(0xffffffffu, w[i], o);
      CombFix::op(w, t);
    }
    if (lane == 0)
#pragma unroll
      for (int i = 0; i < 3; ++i) sm.wred[warp][i] = w[i];
    csync();
    if (warp == 0) {
      uint32_t v[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] = lane < kWarps ? sm.wred[lane][i] : 0u;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        uint32_t t[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) t[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
        CombFix::op(v, t);
      }
      if (C > 1) {
        sx_exchange<3>(v);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          uint32_t t[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) t[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
          CombFix::op(v, t);
        }
      }
      if (lane == 0) {
        const unsigned long long S_ = get_u64(v);
        const unsigned C_ = v[2];
        const unsigned long long t = (C_ > 0 && S_ > rho_fix) ? (S_ - rho_fix) / C_ : 0ull;
        const F2 q = fixed_to_pair(t, F);
        uint32_t* o = sm.bc[bsl];
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
        put(o + 3, t);
        o[5] = __float_as_uint(q.hi);
        o[6] = __float_as_uint(q.lo);
      }
    }
    csync();
    const uint32_t* o = sm.bc[bsl];
    s = get_u64(o);
    c = o[2];
    tn = get_u64(o + 3);
    tp = F2{__uint_as_float(o[5]), __uint_as_float(o[6])};
    bsl ^= 1;
  }

  // ---------------------------------------------------- threshold search
  // tau of P_Omega(v) for the v held by the cluster (Michelot's fixed-point
  // iteration from a lower bound of the root, exact fixed-point sums); see
  // block_l1_tau_fixed_point for the arithmetic.  vbound >= max |v|.  hint:
  // the previous threshold (0.9 hint starts the iteration when it lies below
  // the root).  Sets th/tl (float pair), tau64 (FP64 data), inside.
  __device__ void tau_search(const A (&v)[NE], float hint, float vbound, float& th, float& tl, double& tau64,
                             int& inside) {
    constexpr int BIAS = FixedTraits<A>::BIAS;
    th = tl = 0.f;
    tau64 = 0.0;
    inside = 0;
    if (!(vbound > 0.f)) {
      inside = 1;
      return;
    }
    const FState& st = sm.st;
    const int ef = static_cast<int>(__float_as_uint(fminf(vbound, 3.0e38f)) >> 23) + 1;
    const int eb = ef - 127 + BIAS;
    const int F = 42 + BIAS - eb;
    const unsigned long long rho_fix = pair_to_fixed(st.rho_p, F);
    const unsigned long long tw_fix = hint > 0.f ? pair_to_fixed(F2{0.9f * hint, 0.f}, F) : 0ull;
    unsigned long long t = 0;
    F2 tpair{0.f, 0.f};
    unsigned cprev = 0;
    bool started = false;
    for (int pass = 0; pass < 2 && !started; ++pass) {
      const bool cold = kF64 || pass == 1 || tw_fix == 0;
      const F2 twp = fixed_to_pair(tw_fix, F);
      const TauPair tw{twp.hi, twp.lo};
      unsigned long long s = 0;
      unsigned c = 0;
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        const A av = vabs(v[j]);
        if (cold ? av > A(0) : !tw.below(static_cast<float>(av))) {
          s += fixed43(av, eb);
          ++c;
        }
      }
      tau_reduce(s, c, rho_fix, F, t, tpair);
      if (cold && s <= rho_fix) {
        inside = 1;
        return;
      }
      if (!cold && (c == 0 || s - tw_fix * c < rho_fix)) continue;   // 0.9 hint lies above the root
      cprev = c;
      started = true;
    }
    int steps = 0;
    for (; steps < kTauCap; ++steps) {
      const TauPair tp{tpair.hi, tpair.lo};
      const A tdv = static_cast<A>(static_cast<double>(tp.hi) + static_cast<double>(tp.lo));
      unsigned long long s = 0;
      unsigned c = 0;
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        const A av = vabs(v[j]);
        if (kF64 ? av > tdv : !tp.below(static_cast<float>(av))) {
          s += fixed43(av, eb);
          ++c;
        }
      }
      unsigned long long tn;
      F2 tpn;
      tau_reduce(s, c, rho_fix, F, tn, tpn);
      if (c == 0 || s <= rho_fix) break;   // not reachable from below the root; keep t
      t = tn;
      tpair = tpn;
      if (c == cprev) break;   // the active set no longer changes: t is the threshold
      cprev = c;
    }
    if (tid == 0) sm.st.tau_steps = steps;
    th = tpair.hi;
    tl = tpair.lo;
    if constexpr (kF64) {   // FP64 data: tau in FP64 over the final active set
      const double tcmp = static_cast<double>(th) + static_cast<double>(tl);
      double s2 = 0.0, c2 = 0.0;
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        const double av = fabs(static_cast<double>(v[j]));
        if (av > tcmp) {
          s2 += av;
          c2 += 1.0;
        }
      }
      uint32_t w[4];
      put(w, s2);
      put(w + 2, c2);
      reduce<Comb<double, 2, 0, 0>>(w, true);
      const double S2 = get_d(w), C2 = get_d(w + 2);
      tau64 = C2 > 0.0 ? (S2 - a.rho) / C2 : tcmp;
      const F2 tq = f2_of(tau64);
      th = tq.hi;
      tl = tq.lo;
    }
  }

  // ---------------------------------------------------- the pass over K
  // Warp partials of the block's row sums: (K d)_q and (K x)_q over this
  // warp's columns, written as RWPR words per row to out (one lane per value).
  template <bool ACC>
  __device__ void row_partials(const uint8_t* stg, uint32_t* out) {
    if constexpr (!kF64) {
      if constexpr (!ACC) {
        float vals[2 * R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          if constexpr (!kF64) {
            // even and odd columns in the two halves of packed FP32 FMAs
            float2 pd = make_float2(0.f, 0.f), px = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
              if (!cv[m]) continue;
              A kv[EPC];
              widen16<DT>(stg + soff[m] + q * kBoxW * ES, kv);
#pragma unroll
              for (int e = 0; e < EPC; e += 2) {
                const int j = m * EPC + e;
                const float2 k2 = make_float2(kv[e], kv[e + 1]);
                pd = __ffma2_rn(k2, make_float2(d[j], d[j + 1]), pd);
                px = __ffma2_rn(k2, make_float2(x[j], x[j + 1]), px);
              }
            }
            vals[2 * q] = pd.x + pd.y;
            vals[2 * q + 1] = px.x + px.y;
          } else {
            float pd = 0.f, px = 0.f;
#pragma unroll
            for (int m = 0; m < NCH; ++m) {
              if (!cv[m]) continue;
              A kv[EPC];
              widen16<DT>(stg + soff[m] + q * kBoxW * ES, kv);
#pragma unroll
              for (int e = 0; e < EPC; ++e) {
                pd = fmaf(kv[e], d[m * EPC + e], pd);
                px = fmaf(kv[e], x[m * EPC + e], px);
              }
            }
            vals[2 * q] = pd;
            vals[2 * q + 1] = px;
          }
        }
        const float tot = warp_sum_many<2 * R>(vals, lane);
        constexpr int GL = 32 / (2 * R);
        if (lane % GL == 0) {
          const int v = lane / GL, q = v >> 1;
          out[3 * q + (v & 1)] = __float_as_uint(tot);
          if (v & 1) out[3 * q + 2] = 0u;
        }
      } else {
        // near the stop: K x without rounding error (exact products, two-sums)
        float vd[R];
        F2 vx[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          float pd = 0.f, sh = 0.f, sl = 0.f;
#pragma unroll
          for (int m = 0; m < NCH; ++m) {
            if (!cv[m]) continue;
            A kv[EPC];
            widen16<DT>(stg + soff[m] + q * kBoxW * ES, kv);
#pragma unroll
            for (int e = 0; e < EPC; ++e) {
              pd = fmaf(kv[e], d[m * EPC + e], pd);
              const float pr = __fmul_rn(kv[e], x[m * EPC + e]);
              const float pe = fmaf(kv[e], x[m * EPC + e], -pr);
              const F2 t = two_sum(sh, pr);
              sh = t.hi;
              sl = __fadd_rn(sl, __fadd_rn(pe, t.lo));
            }
          }
          vd[q] = pd;
          vx[q] = F2{sh, sl};
        }
        const float dt = warp_sum_many<R>(vd, lane);
        const F2 xt = warp_sum_many_f2<R>(vx, lane);
        constexpr int GL = 32 / R;
        if (lane % GL == 0) {
          const int q = lane / GL;
          out[3 * q] = __float_as_uint(dt);
          out[3 * q + 1] = __float_as_uint(xt.hi);
          out[3 * q + 2] = __float_as_uint(xt.lo);
        }
      }
    } else {
      double vals[2 * R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        double pd = 0.0, px = 0.0;
#pragma unroll
        for (int m = 0; m < NCH; ++m) {
          if (!cv[m]) continue;
          A kv[EPC];
          widen16<DT>(stg + soff[m] + q * kBoxW * ES, kv);
#pragma unroll
          for (int e = 0; e < EPC; ++e) {
            pd = fma(kv[e], d[m * EPC + e], pd);
            px = fma(kv[e], x[m * EPC + e], px);
          }
        }
        vals[2 * q] = pd;
        vals[2 * q + 1] = px;
      }
      const double tot = warp_sum_many_d<2 * R>(vals, lane);
      constexpr int GL = 32 / (2 * R);
      if (lane % GL == 0) {
        const int v = lane / GL, q = v >> 1;
        put(out + 4 * q + 2 * (v & 1), tot);
      }
    }
  }

  // Lanes per row in the exchange warps: row q of a chunk is handled by lanes
  // q * LPR .. q * LPR + LPR - 1.
  static constexpr int LPR = 32 / RC;

  // Sender warp: the CTA's partial row sums of a chunk from the consumer warps'
  // partials.  Lane g of row q's group adds warps g, g + LPR, ...; a butterfly
  // over the group completes the sum (a fixed order), so every lane of the
  // group ends with the row's words (RWPR of them).
  __device__ void cta_rowsum(const uint32_t (*red)[kRCW], uint32_t (&wd)[RWPR], bool acc) {
    const int q = lane / LPR, g = lane % LPR;
    if constexpr (!kF64) {
      float kd = 0.f;
      F2 kx{0.f, 0.f};
      if (acc) {   // K x as float pairs (compensated)
        for (int w = g; w < kWarps; w += LPR) {
          kd += __uint_as_float(red[w][3 * q]);
          kx = f2_add(kx, F2{__uint_as_float(red[w][3 * q + 1]), __uint_as_float(red[w][3 * q + 2])});
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
          kd += __shfl_xor_sync(0xffffffffu, kd, o);
          kx = f2_add(kx, F2{__shfl_xor_sync(0xffffffffu, kx.hi, o), __shfl_xor_sync(0xffffffffu, kx.lo, o)});
        }
      } else {     // plain FP32 sums
        for (int w = g; w < kWarps; w += LPR) {
          kd += __uint_as_float(red[w][3 * q]);
          kx.hi += __uint_as_float(red[w][3 * q + 1]);
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) {
          kd += __shfl_xor_sync(0xffffffffu, kd, o);
          kx.hi += __shfl_xor_sync(0xffffffffu, kx.hi, o);
        }
      }
      wd[0] = __float_as_uint(kd);
      wd[1] = __float_as_uint(kx.hi);
      wd[2] = __float_as_uint(kx.lo);
    } else {
      double kd = 0.0, kx = 0.0;
      for (int w = g; w < kWarps; w += LPR) {
        kd += get_d(&red[w][4 * q]);
        kx += get_d(&red[w][4 * q + 2]);
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) {
        kd += __shfl_xor_sync(0xffffffffu, kd, o);
        kx += __shfl_xor_sync(0xffffffffu, kx, o);
      }
      put(wd, kd);
      put(wd + 2, kx);
    }
  }

  // Sender warp: send the CTA's row sums of chunk message `seq` to every CTA of
  // the cluster, one bulk copy per CTA (to itself too) from the outgoing slot.
  // The message goes into the slot of message seq - kRNS, which every CTA's
  // totaler must have read (it releases a slot on every CTA, remote arrive on
  // rempty, as soon as it has read it); that also means the bulk copies out of
  // this CTA's outgoing slot have completed.
  __device__ bool rx_send(uint32_t seq, const uint32_t (&wd)[RWPR]) {
    const uint32_t slot = seq % kRNS, use = seq / kRNS;
    if (use >= 1 && !wwait(&sm.rempty[slot], (use - 1) & 1u, kSiteRowMsg, true)) return false;
    if (lane % LPR == 0) {
      uint32_t* o = &sm.xout[slot][RWPR * (lane / LPR)];
#pragma unroll
      for (int i = 0; i < RWPR; ++i) o[i] = wd[i];
    }
    if (lane == 0)
      for (int i = RCW; i < RCWP; ++i) sm.xout[slot][i] = 0u;
    fence_proxy_async_smem();   // the bulk copies read these words through the async proxy
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(&sm.rfull[slot], static_cast<uint32_t>(C * RCWP * 4));
    if (lane < C)
      bulk_to_cluster(mapa(&sm.rx[slot][rank][0], static_cast<unsigned>(lane)), &sm.xout[slot][0],
                      static_cast<uint32_t>(RCWP * 4), mapa(&sm.rfull[slot], static_cast<unsigned>(lane)));
    return true;
  }

  // r = K x - y of one row: as a float pair (float data) or a double
  __device__ static S resid(const S& kx, A y) {
    if constexpr (!kF64) {
      const F2 t = two_sum(kx.hi, -y);
      return two_sum(t.hi, t.lo + kx.lo);
    } else {
      return kx - y;
    }
  }
  __device__ static A lead(const S& v) {
    if constexpr (!kF64) return v.hi;
    else return v;
  }
  __device__ static void acc_sq(S& acc, const S& v) {   // acc += v^2
    if constexpr (!kF64) acc = f2_fma(acc, v.hi, v.hi + 2.f * v.lo);
    else acc = fma(v, v, acc);
  }
  __device__ static void acc_mul(S& acc, A a_, A b_) {   // acc += a b
    if constexpr (!kF64) acc = f2_fma(acc, a_, b_);
    else acc = fma(a_, b_, acc);
  }

  // One pass over this cluster's row blocks (serpentine: even passes forward,
  // odd ones backward), chunk by chunk.  Step A(c): the blocks of chunk c
  // arrive from HBM; the warps' partial row sums go to the sender warp (with
  // y of the chunk's rows, from warp 0) and each block's stage is released at
  // once.  Step B(c - kLagC): the same blocks arrive again (now from L2) and,
  // with the multipliers the totaler published for that chunk,
  // u1 += 2 K^T (K x - y) and u2 += 2 K^T K d over this thread's columns.
  // Reading each block twice lets the row-sum exchange of a chunk take
  // kLagC chunks without holding the chunk in shared memory; HBM still
  // serves K once per pass.  SETUP: d = 0 and no u2; with x0 = 0 there are
  // no row sums (r = -y), and warp 0 of cluster rank 0 adds the row scalars.
  template <bool ACC, bool SETUP>
  __device__ void sweep(int s, S (&rowsc)[3]) {
    constexpr int AW = kF64 ? 2 : 1;
    const bool fwd = (s & 1) == 0;
    const int nb = bk1 - bk0;
    const int ncks = (nb + CF::CB - 1) / CF::CB;
    const bool dots = !(SETUP && a.x0_zero);
    const V* yg = static_cast<const V*>(a.y);
    const uint32_t rs0 = rseq;
#pragma unroll 1
    for (int c = 0; c < ncks + kLagC; ++c) {
      const bool hasA = c < ncks, hasB = c >= kLagC;
      const int cntA = hasA ? min(CF::CB, nb - c * CF::CB) : 0;
      const int cb = c - kLagC;
      const int cntB = hasB ? min(CF::CB, nb - cb * CF::CB) : 0;
      const uint32_t seq = rs0 + c, s3 = seq % kNRed;
      const uint32_t m = rs0 + cb, ts = m % kNTot;
      bool okt = true;
      // y of the chunk's rows (warp 0, lane = row of the chunk), loaded once
      // at the start of the chunk and handed to the totaler after its blocks
      A ych = 0;
      bool vch = false;
      if (hasA && dots && warp == 0 && lane < RC) {
        const int jj = lane / R;
        const int qb = c * CF::CB + jj;
        const int row = (fwd ? bk0 + qb : bk1 - 1 - qb) * R + lane % R;
        vch = jj < cntA && row < n;
        if (vch) ych = static_cast<A>(yg[row]);
      }
#pragma unroll 1
      for (int j = 0; j < CF::CB; ++j) {
        // ---- step A: block j of chunk c (from HBM): its row sums
        if (hasA) {
          if (j < cntA) {
            const uint32_t st = sta;
            const bool ok = wwait(&sm.full[st], pha, kSitePassA, false);
            if (dots && ok) row_partials<ACC>(sm.stage[st], &sm.red[s3][warp][RWPR * R * j]);
            __syncwarp();
            if (lane == 0 && ok) mbar_arrive(&sm.empty[st]);
            if (++sta == CF::NSA) {
              sta = 0;
              pha ^= 1u;
            }
          } else if (dots) {   // past the last block of the pass
            if (lane < RWPR * R) sm.red[s3][warp][RWPR * R * j + lane] = 0u;
          }
        }
        // ---- step B: block j of chunk c - kLagC (from L2): its K^T step
        if (hasB && j < cntB) {
          if (dots && j == 0) okt = wwait(&sm.tfull[ts], (m / kNTot) & 1u, kSiteRowMsg, false);
          const int qb = cb * CF::CB + j;
          const int b = fwd ? bk0 + qb : bk1 - 1 - qb;
          A m1[R], m2[R];
          if (dots) {
#pragma unroll
            for (int qq = 0; qq < R; ++qq) {
              if constexpr (!kF64) {
                m1[qq] = __uint_as_float(sm.tot[ts][j * R + qq]);
                m2[qq] = __uint_as_float(sm.tot[ts][RC + j * R + qq]);
              } else {
                m1[qq] = get_d(&sm.tot[ts][AW * (j * R + qq)]);
                m2[qq] = get_d(&sm.tot[ts][AW * (RC + j * R + qq)]);
              }
            }
          } else {   // x0 = 0: r = -y
            const int row = b * R + lane;
            const bool valid = lane < R && row < n;
            const A yv = valid ? static_cast<A>(yg[row]) : A(0);
            if (warp == 0 && rank == 0 && valid) {
              acc_mul(rowsc[0], yv, yv);
              acc_mul(rowsc[2], yv, yv);
            }
#pragma unroll
            for (int qq = 0; qq < R; ++qq) {
              m1[qq] = A(-2) * __shfl_sync(0xffffffffu, yv, qq);
              m2[qq] = A(0);
            }
          }
          const uint32_t st = CF::NSA + stb;
          const bool ok = wwait(&sm.full[st], phb, kSitePassB, false);
          if (ok && okt) {
            const uint8_t* stg = sm.stage[st];
#pragma unroll
            for (int qq = 0; qq < R; ++qq) {
              if constexpr (!kF64) {
                // two columns per instruction (packed FP32 FMA; each half is
                // the same rounded fma as the scalar form)
                const float2 w1 = make_float2(m1[qq], m1[qq]), w2 = make_float2(m2[qq], m2[qq]);
#pragma unroll
                for (int mm = 0; mm < NCH; ++mm) {
                  if (!cv[mm]) continue;
                  A kv[EPC];
                  widen16<DT>(stg + soff[mm] + qq * kBoxW * ES, kv);
#pragma unroll
                  for (int e = 0; e < EPC; e += 2) {
                    const int j = mm * EPC + e;
                    const float2 k2 = make_float2(kv[e], kv[e + 1]);
                    const float2 a1 = __ffma2_rn(k2, w1, make_float2(u1[j], u1[j + 1]));
                    u1[j] = a1.x;
                    u1[j + 1] = a1.y;
                    if constexpr (!SETUP) {
                      const float2 a2 = __ffma2_rn(k2, w2, make_float2(u2[j], u2[j + 1]));
                      u2[j] = a2.x;
                      u2[j + 1] = a2.y;
                    }
                  }
                }
              } else {
#pragma unroll
                for (int mm = 0; mm < NCH; ++mm) {
                  if (!cv[mm]) continue;
                  A kv[EPC];
                  widen16<DT>(stg + soff[mm] + qq * kBoxW * ES, kv);
#pragma unroll
                  for (int e = 0; e < EPC; ++e) {
                    u1[mm * EPC + e] = vfma(kv[e], m1[qq], u1[mm * EPC + e]);
                    if constexpr (!SETUP) u2[mm * EPC + e] = vfma(kv[e], m2[qq], u2[mm * EPC + e]);
                  }
                }
              }
            }
          }
          __syncwarp();
          if (lane == 0 && ok) mbar_arrive(&sm.empty[st]);
          if (++stb == CF::NSB) {
            stb = 0;
            phb ^= 1u;
          }
        }
      }
      if (hasA && dots) {
        if (warp == 0 && lane < RC) {
          uint32_t* yw = sm.ysm[s3][lane];
          put(yw, ych);   // a float occupies the first word, a double the first two
          yw[2] = vch ? 1u : 0u;
        }
        if (warp == 0 && lane == 0) sm.bmode[s3] = ACC ? 1u : 0u;
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.redfull[s3]);
      }
      if (hasB && dots) {
        __syncwarp();
        if (lane == 0 && okt) mbar_arrive(&sm.tcons[ts]);
      }
    }
    if (dots) {
      rseq = rs0 + ncks;
      // the row scalars the totaler added (cluster rank 0); cleared for the
      // next pass (the totaler's next update follows the next partials, which
      // warp 0 releases after this)
      if (tid == 0) {
        for (int qq = 0; qq < RC; ++qq) {
          const uint32_t* ra = sm.rowacc[qq];
          if constexpr (!kF64) {
            rowsc[0] = f2_add(rowsc[0], get_f2(ra));
            rowsc[1] = f2_add(rowsc[1], get_f2(ra + 2));
            rowsc[2] = f2_add(rowsc[2], get_f2(ra + 4));
          } else {
            rowsc[0] += get_d(ra);
            rowsc[1] += get_d(ra + 2);
            rowsc[2] += get_d(ra + 4);
          }
        }
        for (int qq = 0; qq < 32; ++qq)
          for (int i = 0; i < 6; ++i) sm.rowacc[qq][i] = 0u;
      }
    }
  }

  // End of a pass: add the gradient accumulators into U[s % 3] (vector
  // reductions at L2), clear them, and publish this CTA's record of pass
  // scalars: row scalars (f, ||K d||^2, ||y||^2) and the column partials of
  // the direction (g^T d, ||d||^2, d != 0).
  __device__ void finish_sweep(int s, const S (&rowsc)[3]) {
    A* const U1 = static_cast<A*>(a.U) + static_cast<long long>(s % 3) * 2 * a.pp;
    A* const U2 = U1 + a.pp;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
      if (!cv[m]) continue;
      const int c = gcol[m];
      if constexpr (!kF64) {
#pragma unroll
        for (int e = 0; e < EPC; e += 4) {
          red_add_v4(U1 + c + e, u1[m * EPC + e], u1[m * EPC + e + 1], u1[m * EPC + e + 2], u1[m * EPC + e + 3]);
          red_add_v4(U2 + c + e, u2[m * EPC + e], u2[m * EPC + e + 1], u2[m * EPC + e + 2], u2[m * EPC + e + 3]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < EPC; ++e) {
          red_add(U1 + c + e, u1[m * EPC + e]);
          red_add(U2 + c + e, u2[m * EPC + e]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) u1[j] = u2[j] = A(0);
    uint32_t w[11];
    put(w, rowsc[0]);
    put(w + 2, rowsc[1]);
    put(w + 4, rowsc[2]);
    put(w + 6, c_gd);
    put(w + 8, c_dd);
    w[10] = c_nz;
    reduce<Comb<S, 5, 0, 1>>(w, false);
    if (tid == 0) {
      unsigned* o = a.parts + (static_cast<long long>(s & 1) * G + cta) * kPartW;
#pragma unroll
      for (int i = 0; i < 11; ++i) o[i] = w[i];
    }
  }

  // Sum of the G records of pass s, in a fixed order (every CTA gets the
  // same totals): f, ||K d||^2, ||y||^2, g^T d, ||d||^2 (doubles) and d != 0.
  __device__ void read_parts(int s, double (&o)[5], unsigned& nz) {
    using Cb = Comb<S, 5, 0, 1>;
    if (warp == 0) {
      uint32_t v[11] = {};
      for (int c = lane; c < G; c += 32) {
        const unsigned* src = a.parts + (static_cast<long long>(s & 1) * G + c) * kPartW;
        uint32_t t[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) t[i] = __ldcg(src + i);
        Cb::op(v, t);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        uint32_t t[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) t[i] = __shfl_xor_sync(0xffffffffu, v[i], off);
        Cb::op(v, t);
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if constexpr (!kF64) o[q] = as_double(get_f2(v + 2 * q));
        else o[q] = get_d(v + 2 * q);
      }
      nz = v[10];
    }
  }

  // ---------------------------------------------------- the exchange warps
  // Sender: message after message (in the consumers' order), wait until the 16
  // consumer warps have left their partials of a block, add them and send the
  // CTA's row sums to the cluster.
  __device__ void send_loop() {
    for (uint32_t seq = 0;; ++seq) {
      const uint32_t s3 = seq % kNRed;
      if (!xwait(&sm.redfull[s3], (seq / kNRed) & 1u, false)) break;
      uint32_t wd[RWPR] = {};
      cta_rowsum(sm.red[s3], wd, sm.bmode[s3] != 0u);
      if (!rx_send(seq, wd)) break;
    }
  }

  // Totaler: message after message, wait for the C ranks' row sums of a chunk,
  // add them in rank order (every CTA of the cluster gets the same totals),
  // release the slot on every CTA, and publish for the consumers the K^T
  // multipliers 2 r_i = 2 ((K x)_i - y_i) and 2 (K d)_i of the chunk's rows.
  // On cluster rank 0 it also adds the rows' ||r||^2, ||K d||^2, ||y||^2 into
  // rowacc (slot q for row q of every chunk: a fixed summation order).
  __device__ void total_loop() {
    constexpr int AW = kF64 ? 2 : 1;   // words per value of the arithmetic type
    const int q = lane / LPR, g = lane % LPR;
    for (uint32_t m = 0;; ++m) {
      const uint32_t slot = m % kRNS, s3 = m % kNRed;
      if (!xwait(&sm.rfull[slot], (m / kRNS) & 1u, true)) break;
      // (the partials' phase of this chunk is complete: taking it orders the
      // reads of y and of the mode below after consumer warp 0 wrote them)
      for (int spin = 0; spin < (1 << 20) && !mbar_try_wait(&sm.redfull[s3], (m / kNRed) & 1u); ++spin) {
      }
      const bool acc = sm.bmode[s3] != 0u;
      A kd = 0;
      S kx{};
      for (int r = g; r < C; r += LPR) {
        const uint32_t* w = &sm.rx[slot][r][RWPR * q];
        if constexpr (!kF64) {
          kd += __uint_as_float(w[0]);
          if (acc) kx = f2_add(kx, F2{__uint_as_float(w[1]), __uint_as_float(w[2])});
          else kx.hi += __uint_as_float(w[1]);
        } else {
          kd += get_d(w);
          kx += get_d(w + 2);
        }
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) {
        if constexpr (!kF64) {
          kd += __shfl_xor_sync(0xffffffffu, kd, o);
          if (acc) kx = f2_add(kx, F2{__shfl_xor_sync(0xffffffffu, kx.hi, o), __shfl_xor_sync(0xffffffffu, kx.lo, o)});
          else kx.hi += __shfl_xor_sync(0xffffffffu, kx.hi, o);
        } else {
          kd += __shfl_xor_sync(0xffffffffu, kd, o);
          kx += __shfl_xor_sync(0xffffffffu, kx, o);
        }
      }
      A y = 0;
      bool valid = false;
      {
        const uint32_t* yw = sm.ysm[s3][q];
        if constexpr (!kF64) y = __uint_as_float(yw[0]);
        else y = get_d(yw);
        valid = yw[2] != 0u;
      }
      __syncwarp();
      if (lane < C) mbar_arrive_remote(mapa(&sm.rempty[slot], static_cast<unsigned>(lane)));
      S r;
      if constexpr (!kF64) r = acc ? resid(kx, y) : F2{kx.hi - y, 0.f};
      else r = resid(kx, y);
      if (!valid) {
        r = S{};
        kd = 0;
        y = 0;
      }
      const uint32_t ts = m % kNTot;
      if (m >= kNTot && !wwait(&sm.tcons[ts], ((m - kNTot) / kNTot) & 1u, kSiteRowMsg, false)) break;
      if (g == 0) {
        const A m1 = A(2) * lead(r), m2 = A(2) * kd;
        if constexpr (!kF64) {
          sm.tot[ts][q] = __float_as_uint(m1);
          sm.tot[ts][RC + q] = __float_as_uint(m2);
        } else {
          put(&sm.tot[ts][AW * q], m1);
          put(&sm.tot[ts][AW * (RC + q)], m2);
        }
        if (rank == 0) {
          uint32_t* ra = sm.rowacc[q];
          if constexpr (!kF64) {
            F2 f = get_f2(ra), k2 = get_f2(ra + 2), yy = get_f2(ra + 4);
            acc_sq(f, r);
            acc_mul(k2, kd, kd);
            acc_mul(yy, y, y);
            put(ra, f);
            put(ra + 2, k2);
            put(ra + 4, yy);
          } else {
            double f = get_d(ra), k2 = get_d(ra + 2), yy = get_d(ra + 4);
            acc_sq(f, r);
            acc_mul(k2, kd, kd);
            acc_mul(yy, y, y);
            put(ra, f);
            put(ra + 2, k2);
            put(ra + 4, yy);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.tfull[ts]);
    }
  }

  // ---------------------------------------------------- scalar steps (lead)
  // Algorithm SS for k >= 1 (FP64): BB1/BB2 from s^T s, s^T z (previous
  // iteration) and z^T z, the ratio test against tau_k, the alpha^(2) window.
  __device__ double ss_step(double zz) {
    FState& u = sm.st;
    const SolveParams& P = a.prm;
    double alpha, a2_this;
    if (u.sz_prev <= 0.0) {
      alpha = P.alpha_max;
      a2_this = P.alpha_max;   // alpha^(2)_k undefined: does not lower the window minimum
    } else {
      const double a1 = fmin(fmax(u.ss_prev / u.sz_prev, P.alpha_min), P.alpha_max);
      const double a2 = fmin(fmax(u.sz_prev / zz, P.alpha_min), P.alpha_max);
      a2_this = a2;
      double amin = a2;
      for (int q = 0; q < u.a2cnt && q < P.M_alpha; ++q) amin = fmin(amin, u.a2win[q]);
      if (a2 <= u.tau_ss * a1) {
        alpha = amin;
        u.tau_ss *= 0.9;
      } else {
        alpha = a1;
        u.tau_ss *= 1.1;
      }
    }
    for (int q = P.M_alpha - 1; q > 0; --q) u.a2win[q] = u.a2win[q - 1];
    if (P.M_alpha > 0) u.a2win[0] = a2_this;
    if (u.a2cnt < P.M_alpha) ++u.a2cnt;
    return alpha;
  }

  __device__ void set_alpha(double alpha) {
    FState& u = sm.st;
    u.alpha = alpha;
    const F2 af = f2_of(alpha);
    u.ah = af.hi;
    u.al = af.lo;
    u.vbound = static_cast<float>((a.rho + alpha * u.gmax) * 1.000001);
    if (!isfinite(alpha)) {
      u.status = GPL1_ERR_NONFINITE;
      u.stop = GPL1_STOP_ERROR;
      u.done = 1;
    }
  }

  __device__ void trace_row(int k, double fk, double lam, double kb2) {
    const FState& u = sm.st;
    if (!a.trace || k >= a.trace_cap || cta != 0) return;
    double* t = a.trace + static_cast<long long>(k) * GPL1_TRACE_COLS;
    t[0] = fk;
    t[1] = u.alpha;
    t[2] = lam;
    t[3] = u.tau_ss;
    t[4] = u.gd;
    t[5] = kb2;
    t[6] = u.dd;
    t[7] = kF64 ? u.tau64 : static_cast<double>(u.th) + static_cast<double>(u.tl);
    for (int q = 1; q < 8; ++q) t[7 + q] = static_cast<double>(u.ts[q] - u.ts[0]);
    t[16] = u.tau_steps;
    t[17] = C;
    t[18] = NC;
  }

  // Armijo backtracking (Alg. GP, Steps 4-6) in FP64 on the exact expansion of
  // the quadratic f: f(x_k + l d) = f_k + l g_k^T d_k + l^2 ||K d_k||^2.
  // Returns 0 (continue), 1 (stop after the update x + lam d), 2 (stop at x_k).
  __device__ int ls_step(int k, double fk, double kb2) {
    FState& u = sm.st;
    const SolveParams& P = a.prm;
    const double gd = u.gd, dd = u.dd;
    if (!isfinite(fk) || !isfinite(kb2) || !isfinite(gd)) {
      u.status = GPL1_ERR_NONFINITE;
      u.stop = GPL1_STOP_ERROR;
      u.iters = k;
      u.done = 1;
      return 2;
    }
    u.fhist[0] = fk;
    double fmaxv = fk;
    for (int q = 1; q < P.M && q <= k; ++q) fmaxv = fmax(fmaxv, u.fhist[q]);
    double lam = 1.0;
    int bt = 0;
    bool ok = false;
    for (;;) {
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
      return 2;
    }
    const double fnext = fk + lam * (gd + lam * kb2);
    for (int q = kMaxM - 1; q > 0; --q) u.fhist[q] = u.fhist[q - 1];
    u.fhist[0] = fnext;
    u.lam = lam;
    u.lf = static_cast<float>(lam);
    // s^T s = lam^2 ||d||^2 and s^T z = s^T 2 K^T K s = 2 lam^2 ||K d||^2 for this quadratic f
    u.ss_prev = lam * lam * dd;
    u.sz_prev = 2.0 * lam * lam * kb2;
    u.f_cur = fnext;
    u.iters = k + 1;
    const bool relgap = (P.stop_rule & GPL1_STOP_ON_REL_GAP) && a.f_star >= 0.0;
    if (relgap && fnext - a.f_star <= kAccGapFactor * P.tol * u.gap_den) u.acc = 1;
    if (fk - fnext <= kAccDecrease * fk) u.acc = 1;
    if (fnext < u.f_best - 1e-3 * P.tol * u.gap_den) {
      u.f_best = fnext;
      u.stall = 0;
    } else {
      ++u.stall;
    }
    if (relgap && fnext - a.f_star <= P.tol * u.gap_den) {
      u.stop = GPL1_STOP_REL_GAP;
      u.done = 1;
      return 1;
    }
    if (u.iters >= P.max_iter) {
      u.stop = GPL1_STOP_MAX_ITER;
      u.status = GPL1_ERR_NOT_CONVERGED;
      u.done = 1;
      return 1;
    }
    // float data at their precision floor: f no longer falls near the stop
    if (u.acc && u.stall >= kStallIters && (P.stop_rule & (GPL1_STOP_ON_REL_GAP | GPL1_STOP_ON_FW))) {
      u.stop = GPL1_STOP_STAGNATION;
      u.status = GPL1_ERR_NOT_CONVERGED;
      u.done = 1;
      return 1;
    }
    return 0;
  }

  // After the pass of iteration k (pass number s): the line search.
  __device__ int phase_l(int k, int s) {
    double o[5];
    unsigned nz = 0;
    read_parts(s, o, nz);
    if (tid == 0) {
      FState& u = sm.st;
      if (a.trace) u.ts[2] = globaltimer();
      u.kb2 = o[1];
      u.gd = o[3];
      u.dd = o[4];
      int act;
      if (!nz) {   // h == x: a stationary point (Alg. GP, Step 2)
        u.stop = GPL1_STOP_STATIONARY;
        u.iters = k;
        u.f_cur = o[0];
        u.done = 1;
        act = 2;
      } else {
        act = ls_step(k, o[0], o[1]);
      }
      sm.ctl[CTL_INST] = act;
    }
    csync();
    const int act = sm.ctl[CTL_INST];
    csync();
    return act;
  }

  // After the setup pass: f(x0), ||y||^2, the gap denominator.
  __device__ void phase_l0() {
    double o[5];
    unsigned nz = 0;
    read_parts(0, o, nz);
    if (tid == 0) {
      FState& u = sm.st;
      u.f_cur = o[0];
      u.yy = o[2];
      u.gap_den = fmax(a.f_star, a.prm.tol * o[2]);
      u.f_best = o[0];
      u.stall = 0;
      for (int q = 0; q < kMaxM; ++q) u.fhist[q] = o[0];
      if (!isfinite(o[0])) {
        u.status = GPL1_ERR_NONFINITE;
        u.stop = GPL1_STOP_ERROR;
        u.done = 1;
      }
    }
    csync();
  }

  __device__ Dir dir_of() const {
    const FState& u = sm.st;
    Dir dr(u.tau64, u.th, u.tl, u.inside);
    dr.alpha = u.alpha;
    dr.ah = u.ah;
    dr.al = u.al;
    return dr;
  }

  // Float data near the stop: tau again, on the active set {|v| > tau}, from x
  // and g themselves (float pairs) rather than from the rounded v, so that
  // ||x + d||_1 = rho to pair accuracy (as in the two-pass kernel).
  __device__ void refine_tau(const A (&v)[NE], float& th, float& tl) {
    const TauPair tp{th, tl};
    F2 sx{0.f, 0.f}, sg{0.f, 0.f}, sc{0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      if (!tp.below(fabsf(static_cast<float>(v[j]))) && v[j] != A(0)) {
        const float s_ = v[j] > A(0) ? 1.f : -1.f;
        sx = f2_add(sx, s_ * static_cast<float>(x[j]));
        sg = f2_add(sg, s_ * static_cast<float>(g[j]));
        sc = f2_add(sc, 1.f);
      }
    }
    uint32_t w[6];
    put(w, sx);
    put(w + 2, sg);
    put(w + 4, sc);
    reduce<Comb<F2, 3, 0, 0>>(w, true);
    const FState& u = sm.st;
    const F2 SX = get_f2(w), SG = get_f2(w + 2);
    const float c = get_f2(w + 4).hi;
    const float ph = __fmul_rn(u.ah, SG.hi);
    const float pl = fmaf(u.ah, SG.hi, -ph) + fmaf(u.ah, SG.lo, u.al * SG.hi);
    F2 t = f2_add(SX, F2{-ph, -pl});
    t = f2_add(t, F2{-u.rho_p.hi, -u.rho_p.lo});
    const float q1 = __fdiv_rn(t.hi, c);
    const float rem = fmaf(-q1, c, t.hi) + t.lo;
    const F2 q = two_sum(q1, __fdiv_rn(rem, c));
    if (c > 0.f && q.hi > 0.f) {
      th = q.hi;
      tl = q.lo;
    }
  }

  // Projection phase of iteration k after pass s: x_k (already updated),
  // g_k = u1 + lam_{k-1} u2 from U[s % 3]; z^T z, g^T x, ||g||_inf, ||x||_1;
  // the FW stop; Alg. SS (alpha_0 at k = 0); v = x - alpha g; the threshold;
  // d = P(v) - x and its column partials.  Returns false when the solve stops
  // here (x_k is the answer) or failed.
  __device__ bool phase_p(int k, int s) {
    FState& u = sm.st;
    const SolveParams& P = a.prm;
    const A* const U1 = static_cast<const A*>(a.U) + static_cast<long long>(s % 3) * 2 * a.pp;
    const A* const U2 = U1 + a.pp;
    const A lam = k == 0 ? A(0) : (kF64 ? static_cast<A>(u.lam) : static_cast<A>(u.lf));
    A zz = 0, gm = 0;
    S gx{}, l1{};
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
      if (!cv[m]) continue;
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = m * EPC + e;
        const A gn = vfma(lam, ldg_cg(U2 + gcol[m] + e), ldg_cg(U1 + gcol[m] + e));
        const A z = gn - g[j];
        zz = vfma(z, z, zz);
        g[j] = gn;
        acc_mul(gx, gn, x[j]);
        gm = vmax(gm, vabs(gn));
        if constexpr (!kF64) l1 = f2_add(l1, fabsf(x[j]));
        else l1 += fabs(x[j]);
      }
    }
    {   // clear this CTA's share of the buffer the pass after next adds into
      A* const Z = static_cast<A*>(a.U) + static_cast<long long>((s + 2) % 3) * 2 * a.pp;
      const long long tot = 2 * a.pp, j0 = tot * cta / G, j1 = tot * (cta + 1) / G;
      for (long long j = j0 + tid; j < j1; j += kCons) Z[j] = A(0);
    }
    using CbP = Comb<S, 3, 1, 0, kF64>;
    uint32_t w[CbP::NW];
    if constexpr (!kF64) put(w, F2{zz, 0.f});
    else put(w, zz);
    put(w + 2, gx);
    put(w + 4, l1);
    put_max(w + 6, gm);
    reduce<CbP>(w, true);
    if (tid == 0) {
      if (a.trace) u.ts[3] = globaltimer();
      double zzd, gxd, l1d;
      if constexpr (!kF64) {
        zzd = as_double(get_f2(w));
        gxd = as_double(get_f2(w + 2));
        const F2 l1p = get_f2(w + 4);
        l1d = as_double(l1p);
        // feasibility of x_k: rounding in x + lam d can leave ||x||_1 a few
        // ulps above rho; the iterate is then scaled back onto the ball
        const float ex = (l1p.hi - u.rho_p.hi) + (l1p.lo - u.rho_p.lo);
        u.xscale = ex > 0.f ? __fdiv_rd(u.rho_p.hi, l1p.hi) * (1.f - 0x1p-21f) : 1.f;
      } else {
        zzd = get_d(w);
        gxd = get_d(w + 2);
        l1d = get_d(w + 4);
        u.xscale = 1.f;
        u.xscale_d = l1d > a.rho ? (a.rho / l1d) * (1.0 - 0x1p-50) : 1.0;
      }
      if constexpr (!kF64) {
        u.gmaxf = get_max_f(w + 6);
        u.gmax = static_cast<double>(u.gmaxf);
      } else {
        u.gmax = get_max_d(w + 6);
        u.gmaxf = static_cast<float>(u.gmax) * 1.0000002f;   // an upper bound, for the float-side bound only
      }
      u.gx = gxd;
      (void)l1d;
      if (P.stop_rule & GPL1_STOP_ON_FW) {
        const double fw = gxd + a.rho * u.gmax;
        if (fw <= kAccGapFactor * P.tol * (u.f_cur - fw)) u.acc = 1;
        if (fw <= P.tol * (u.f_cur - fw)) {
          u.stop = GPL1_STOP_FW;
          u.iters = k;
          u.done = 1;
        }
      }
      if (!u.done && k > 0) set_alpha(ss_step(zzd));
      if (!u.done && k == 0) u.vbound = static_cast<float>((a.rho + u.gmax) * 1.000001);
      sm.ctl[CTL_INST] = u.done;
      if (a.trace) u.ts[4] = globaltimer();
    }
    csync();
    if (sm.ctl[CTL_INST]) return false;
    if constexpr (!kF64) {
      if (u.xscale != 1.f) {
        const float xs = u.xscale;
#pragma unroll
        for (int j = 0; j < NE; ++j) x[j] *= xs;
      }
    } else {
      if (u.xscale_d != 1.0) {
        const double xs = u.xscale_d;
#pragma unroll
        for (int j = 0; j < NE; ++j) x[j] *= xs;
      }
    }
    A v[NE];
    float th, tl;
    double t64;
    int inside;
    if (k == 0) {
      // alpha_0 = clamp(1 / ||P(x0 - g0)||_inf)   (rule 1: ||P(x0 - g0) - x0||_inf)
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = x[j] - g[j];
      tau_search(v, 0.f, u.vbound, th, tl, t64, inside);
      const Dir pw(t64, th, tl, inside);
      A mx = 0;
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        const A h = pw.proj(v[j]);
        mx = vmax(mx, vabs(P.alpha0_rule == 1 ? h - x[j] : h));
      }
      using CbM = Comb<S, 0, 1, 0, kF64>;
      uint32_t wm[CbM::NW];
      put_max(wm, mx);
      reduce<CbM>(wm, true);
      if (tid == 0) {
        double ninf;
        if constexpr (!kF64) ninf = static_cast<double>(get_max_f(wm));
        else ninf = get_max_d(wm);
        set_alpha(ninf > 0.0 ? fmin(fmax(1.0 / ninf, P.alpha_min), P.alpha_max) : P.alpha_max);
        sm.ctl[CTL_INST] = u.done;
      }
      csync();
      if (sm.ctl[CTL_INST]) return false;
    }
    // v = x - alpha g and the threshold of P(v)
    if constexpr (!kF64) {
      const float ah = u.ah;
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = fmaf(-ah, g[j], x[j]);
    } else {
      const double al = u.alpha;
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = fma(-al, g[j], x[j]);
    }
    tau_search(v, u.hint, u.vbound, th, tl, t64, inside);
    if constexpr (!kF64) {
      if (u.acc && !inside) refine_tau(v, th, tl);
    }
    csync();
    if (tid == 0) {
      u.th = th;
      u.tl = tl;
      u.tau64 = t64;
      u.inside = inside;
      if (!inside) u.hint = th;
      if (a.trace) u.ts[5] = globaltimer();
    }
    csync();
    // d = P(v) - x, and the direction's column partials (counted once: cluster 0)
    const Dir dr = dir_of();
    c_gd = S{};
    c_dd = S{};
    c_nz = 0;
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = m * EPC + e;
        d[j] = cv[m] ? dr.d(x[j], g[j]) : A(0);
        if (cid == 0) {
          acc_mul(c_gd, g[j], d[j]);
          acc_mul(c_dd, d[j], d[j]);
          c_nz |= d[j] != A(0) ? 1u : 0u;
        }
      }
    }
    return true;
  }

  // x0 given: project it onto the ball (Alg. GP starts in Omega).
  __device__ void project_x0() {
    A mx = 0;
#pragma unroll
    for (int j = 0; j < NE; ++j) mx = vmax(mx, vabs(x[j]));
    uint32_t wm[1] = {__float_as_uint(fminf(static_cast<float>(mx), 3.0e38f) * 1.0000002f)};
    reduce<Comb<S, 0, 1, 0>>(wm, true);
    float th, tl;
    double t64;
    int inside;
    tau_search(x, 0.f, __uint_as_float(wm[0]), th, tl, t64, inside);
    if (!inside) {
      const Dir pr(t64, th, tl, 0);
#pragma unroll
      for (int j = 0; j < NE; ++j) x[j] = pr.proj(x[j]);
    }
  }

  // Stop the producer and wait for every TMA copy it issued (copies in flight
  // land within microseconds; the waits have a fixed bound of their own).
  __device__ void drain() {
    volatile int* ctl = sm.ctl;
    if (tid == 0) ctl[CTL_STOP] = 1;
    const uint64_t t0 = globaltimer();
    while (!ctl[CTL_DONE]) {
      if (globaltimer() - t0 > kInflightNs) {
        if (tid == 0) set_err(kSiteDrain);
        break;
      }
    }
    __threadfence_block();
    if (tid == 0) {
      // the last copy issued into every stage of both rings (earlier ones
      // completed their phases before it could be issued)
      for (int ring = 0; ring < 2; ++ring) {
        const uint32_t issued = static_cast<uint32_t>(ctl[ring ? CTL_ISSUED_B : CTL_ISSUED]);
        const uint32_t ns = ring ? CF::NSB : CF::NSA, base = ring ? CF::NSA : 0;
        for (uint32_t s = 0; s < ns && s < issued; ++s) {
          const uint32_t last = issued - 1 - ((issued - 1 - s) % ns);
          const uint32_t par = (last / ns) & 1u;
          const uint64_t t1 = globaltimer();
          while (!mbar_try_wait(&sm.full[base + s], par))
            if (globaltimer() - t1 > kInflightNs) break;
        }
      }
    }
    csync();
  }

  // ---------------------------------------------------- comparison methods
  // ISTA, FISTA and PSD (Sec. 2) on the same passes.  After pass s the
  // gradient at x_k is g_k = U1 + c U2 with c = cpass.  FISTA evaluates the
  // gradient at z_k = x_k + w_k (x_k - x_{k-1}) instead, and since the pass
  // carried d_{k-1} = x_k - x_{k-1}, g(z_k) = g_k + w_k U2 (the gradient is
  // linear in the point).  mode 0: ISTA / FISTA step, d_k = S(v) - x_k with
  // v = z_k - (s/2) g(z_k) (= z_k + s K^T (y - K z_k)); mode 1: PSD probe, the
  // pass's direction is g_k (its ||K g_k||^2 gives beta_k); mode 2: PSD step,
  // d_k = P(x_k - (beta_k/2) g_k) - x_k (= P(x_k + beta_k r_k) - x_k).
  // Modes 0 and 1 open iteration k with its stop tests at x_k.  Returns false
  // when the solve stops here (x_k is the answer) or failed.
  __device__ bool phase_m(int k, int s, int mode) {
    FState& u = sm.st;
    const SolveParams& P = a.prm;
    const bool eq1 = P.method != GPL1_METHOD_PSD;
    const A* const U1 = static_cast<const A*>(a.U) + static_cast<long long>(s % 3) * 2 * a.pp;
    const A* const U2 = U1 + a.pp;
    const A c = u.cpass ? A(1) : A(0);
    double wk = 0.0;
    if (mode == 0 && P.method == GPL1_METHOD_FISTA) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
      wk = (tk - 1.0) / tn;
      tk = tn;
    }
    const A w = static_cast<A>(wk);
    A gz[NE];
    A gg = 0, gm = 0;
    S gx{}, l1{};
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = m * EPC + e;
        gz[j] = A(0);
        if (!cv[m]) continue;
        const A v2 = ldg_cg(U2 + gcol[m] + e);
        const A gn = vfma(c, v2, ldg_cg(U1 + gcol[m] + e));
        g[j] = gn;
        gz[j] = vfma(w, v2, gn);
        gg = vfma(gn, gn, gg);
        acc_mul(gx, gn, x[j]);
        gm = vmax(gm, vabs(gn));
        if constexpr (!kF64) l1 = f2_add(l1, fabsf(x[j]));
        else l1 += fabs(x[j]);
      }
    }
    {   // clear this CTA's share of the buffer the pass after next adds into
      A* const Z = static_cast<A*>(a.U) + static_cast<long long>((s + 2) % 3) * 2 * a.pp;
      const long long tot = 2 * a.pp, j0 = tot * cta / G, j1 = tot * (cta + 1) / G;
      for (long long j = j0 + tid; j < j1; j += kCons) Z[j] = A(0);
    }
    using CbP = Comb<S, 3, 1, 0, kF64>;
    uint32_t wr[CbP::NW];
    if constexpr (!kF64) put(wr, F2{gg, 0.f});
    else put(wr, gg);
    put(wr + 2, gx);
    put(wr + 4, l1);
    put_max(wr + 6, gm);
    reduce<CbP>(wr, true);
    if (tid == 0) {
      double ggd, gxd, l1d;
      if constexpr (!kF64) {
        ggd = as_double(get_f2(wr));
        gxd = as_double(get_f2(wr + 2));
        const F2 l1p = get_f2(wr + 4);
        l1d = as_double(l1p);
        u.gmaxf = get_max_f(wr + 6);
        u.gmax = static_cast<double>(u.gmaxf);
        // PSD iterates lie in the ball: rounding in x + d can leave ||x||_1 a
        // few ulps above rho, and the iterate is scaled back (as in Alg. GP)
        const float ex = (l1p.hi - u.rho_p.hi) + (l1p.lo - u.rho_p.lo);
        u.xscale = (!eq1 && mode == 1 && ex > 0.f) ? __fdiv_rd(u.rho_p.hi, l1p.hi) * (1.f - 0x1p-21f) : 1.f;
      } else {
        ggd = get_d(wr);
        gxd = get_d(wr + 2);
        l1d = get_d(wr + 4);
        u.gmax = get_max_d(wr + 6);
        u.gmaxf = static_cast<float>(u.gmax) * 1.0000002f;
        u.xscale = 1.f;
        u.xscale_d = (!eq1 && mode == 1 && l1d > a.rho) ? (a.rho / l1d) * (1.0 - 0x1p-50) : 1.0;
      }
      u.gx = gxd;
      if (mode != 2) {   // stop tests at x_k: the objective of the method's problem
        const double obj = eq1 ? u.f_cur + 2.0 * P.lam_pen * l1d : u.f_cur;
        u.F_cur = obj;
        if ((P.stop_rule & GPL1_STOP_ON_REL_GAP) && a.f_star >= 0.0) {
          if (obj - a.f_star <= kAccGapFactor * P.tol * u.gap_den) u.acc = 1;
          if (obj - a.f_star <= P.tol * u.gap_den) {
            u.stop = GPL1_STOP_REL_GAP;
            u.iters = k;
            u.done = 1;
          }
        }
        if (!eq1 && !u.done && (P.stop_rule & GPL1_STOP_ON_FW)) {
          const double fw = gxd + a.rho * u.gmax;
          if (fw <= kAccGapFactor * P.tol * (u.f_cur - fw)) u.acc = 1;
          if (fw <= P.tol * (u.f_cur - fw)) {
            u.stop = GPL1_STOP_FW;
            u.iters = k;
            u.done = 1;
          }
        }
        if (!isfinite(obj) && !u.done) {
          u.status = GPL1_ERR_NONFINITE;
          u.stop = GPL1_STOP_ERROR;
          u.iters = k;
          u.done = 1;
        }
      }
      if (!u.done) {
        if (eq1) {
          u.alpha = 0.5 * P.step;
          u.ah = static_cast<float>(u.alpha);
          u.tau64 = P.step * P.lam_pen;
          u.th = static_cast<float>(u.tau64);
          u.tl = 0.f;
        } else if (mode == 1) {
          u.gg = ggd;
          if (!(ggd > 0.0)) {   // g_k = 0: x_k minimises f outright
            u.stop = GPL1_STOP_STATIONARY;
            u.iters = k;
            u.done = 1;
          }
        } else if (!(u.kb2p > 0.0)) {   // K g_k = 0 with g_k != 0 cannot happen for g = 2 K^T r
          u.stop = GPL1_STOP_STATIONARY;
          u.iters = k;
          u.done = 1;
        } else {
          set_alpha(u.gg / (2.0 * u.kb2p));
        }
      }
      sm.ctl[CTL_INST] = u.done;
    }
    csync();
    if (sm.ctl[CTL_INST]) return false;
    if (mode == 1) {
      if constexpr (!kF64) {
        if (u.xscale != 1.f) {
          const float xs = u.xscale;
#pragma unroll
          for (int j = 0; j < NE; ++j) x[j] *= xs;
        }
      } else {
        if (u.xscale_d != 1.0) {
          const double xs = u.xscale_d;
#pragma unroll
          for (int j = 0; j < NE; ++j) x[j] *= xs;
        }
      }
    }
    c_gd = S{};
    c_dd = S{};
    c_nz = 0;
    if (mode == 1) {   // the probe pass runs along g_k
#pragma unroll
      for (int j = 0; j < NE; ++j) d[j] = g[j];
      return true;
    }
    if (mode == 0) {
      const A al = kF64 ? static_cast<A>(u.alpha) : static_cast<A>(u.ah);
      const A th = kF64 ? static_cast<A>(u.tau64) : static_cast<A>(u.th);
#pragma unroll
      for (int m = 0; m < NCH; ++m) {
#pragma unroll
        for (int e = 0; e < EPC; ++e) {
          const int j = m * EPC + e;
          A dn = A(0);
          if (cv[m]) {
            const A z = vfma(w, d[j], x[j]);
            const A v = vfma(-al, gz[j], z);
            const A mag = vabs(v) - th;
            const A xn = mag > A(0) ? (v > A(0) ? mag : -mag) : A(0);
            dn = xn - x[j];
          }
          d[j] = dn;
          if (cid == 0) {
            acc_mul(c_gd, g[j], dn);
            acc_mul(c_dd, dn, dn);
            c_nz |= dn != A(0) ? 1u : 0u;
          }
        }
      }
      return true;
    }
    // mode 2: v = x - alpha g and the threshold of P(v)
    A v[NE];
    float th, tl;
    double t64;
    int inside;
    if constexpr (!kF64) {
      const float ah = u.ah;
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = fmaf(-ah, g[j], x[j]);
    } else {
      const double al = u.alpha;
#pragma unroll
      for (int j = 0; j < NE; ++j) v[j] = fma(-al, g[j], x[j]);
    }
    tau_search(v, u.hint, u.vbound, th, tl, t64, inside);
    if constexpr (!kF64) {
      if (u.acc && !inside) refine_tau(v, th, tl);
    }
    csync();
    if (tid == 0) {
      u.th = th;
      u.tl = tl;
      u.tau64 = t64;
      u.inside = inside;
      if (!inside) u.hint = th;
    }
    csync();
    const Dir dr = dir_of();
#pragma unroll
    for (int m = 0; m < NCH; ++m) {
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = m * EPC + e;
        d[j] = cv[m] ? dr.d(x[j], g[j]) : A(0);
        if (cid == 0) {
          acc_mul(c_gd, g[j], d[j]);
          acc_mul(c_dd, d[j], d[j]);
          c_nz |= d[j] != A(0) ? 1u : 0u;
        }
      }
    }
    return true;
  }

  // After the pass of a comparison method's step (mode 0 or 2): the step is
  // taken whole, f_{k+1} = f_k + g_k^T d_k + ||K d_k||^2 (exact for the
  // quadratic f).  After a PSD probe (mode 1): ||K g_k||^2.  Returns 0
  // (continue), 1 (stop after the update x + d) or 2 (stop at x_k).
  __device__ int phase_lm(int k, int s, int mode) {
    double o[5];
    unsigned nz = 0;
    read_parts(s, o, nz);
    if (tid == 0) {
      FState& u = sm.st;
      const SolveParams& P = a.prm;
      int act = 0;
      if (!isfinite(o[0]) || !isfinite(o[1]) || !isfinite(o[3])) {
        u.status = GPL1_ERR_NONFINITE;
        u.stop = GPL1_STOP_ERROR;
        u.iters = k;
        u.done = 1;
        act = 2;
      } else if (mode == 1) {
        u.kb2p = o[1];
        u.cpass = 0;
      } else {
        const double fk = o[0], kb2 = o[1];
        u.kb2 = kb2;
        u.gd = o[3];
        u.dd = o[4];
        u.cpass = 1;
        if (!nz) {   // x_{k+1} = x_k: a fixed point of the iteration
          u.stop = GPL1_STOP_STATIONARY;
          u.iters = k;
          u.f_cur = fk;
          u.done = 1;
          act = 2;
        } else {
          const double fnext = fk + u.gd + kb2;
          if (P.method != GPL1_METHOD_PSD) u.tau_ss = u.F_cur;   // trace column 3: the objective of eq. 1
          trace_row(k, fk, 1.0, kb2);
          if (fabs(fk - fnext) <= kAccDecrease * fk) u.acc = 1;
          u.lam = 1.0;
          u.lf = 1.f;
          u.f_cur = fnext;
          u.iters = k + 1;
          if (u.iters >= P.max_iter) {
            u.stop = GPL1_STOP_MAX_ITER;
            u.status = GPL1_ERR_NOT_CONVERGED;
            u.done = 1;
            act = 1;
          }
        }
      }
      sm.ctl[CTL_INST] = act;
    }
    csync();
    const int act = sm.ctl[CTL_INST];
    csync();
    return act;
  }

  // The objective of eq. 1 at the returned x after a stop that followed a
  // whole ISTA / FISTA step (||x||_1 of the new iterate not yet summed).
  __device__ void eq1_objective_tail() {
    S l1{};
#pragma unroll
    for (int j = 0; j < NE; ++j) {
      if constexpr (!kF64) l1 = f2_add(l1, fabsf(x[j]));
      else l1 += fabs(x[j]);
    }
    uint32_t wl[2];
    put(wl, l1);
    reduce<Comb<S, 1, 0, 0>>(wl, true);
    if (tid == 0) {
      double l1d;
      if constexpr (!kF64) l1d = as_double(get_f2(wl));
      else l1d = get_d(wl);
      sm.st.F_cur = sm.st.f_cur + 2.0 * a.prm.lam_pen * l1d;
    }
    csync();
  }

  __device__ void init_state() {
    FState& u = sm.st;
    const SolveParams& P = a.prm;
    u.alpha = u.lam = u.f_cur = u.gd = u.dd = u.kb2 = u.gmax = u.gx = u.gap_den = u.yy = 0.0;
    u.tau_ss = P.tau1;
    u.ss_prev = u.sz_prev = 0.0;
    u.a2cnt = 0;
    u.ah = u.al = u.th = u.tl = u.lf = u.vbound = u.gmaxf = 0.f;
    u.xscale = 1.f;
    u.xscale_d = 1.0;
    u.rho_p = f2_of(a.rho);
    u.hint = 0.f;
    u.tau64 = 0.0;
    u.stop = GPL1_STOP_MAX_ITER;
    u.iters = u.backtracks = u.inside = 0;
    u.status = GPL1_OK;
    u.done = 0;
    u.nz = 0;
    u.tau_steps = 0;
    u.F_cur = u.gg = u.kb2p = 0.0;
    u.cpass = 0;
    // with no target to approach, every pass sums K x compensated
    u.acc = (P.stop_rule & (GPL1_STOP_ON_REL_GAP | GPL1_STOP_ON_FW)) ? 0 : 1;
    if (kF64) u.acc = 0;
    for (int q = 0; q < 10; ++q) u.ts[q] = 0;
  }

  template <bool SETUP>
  __device__ void pass(int s) {
    S rowsc[3] = {S{}, S{}, S{}};
    if (!kF64 && sm.st.acc) sweep<true, SETUP>(s, rowsc);
    else sweep<false, SETUP>(s, rowsc);
    finish_sweep(s, rowsc);
  }

  __device__ void run() {
    FState& u = sm.st;
    if (tid == 0) init_state();
    csync();
    const V* const xin = static_cast<const V*>(a.x);
#pragma unroll
    for (int m = 0; m < NCH; ++m)
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = m * EPC + e;
        x[j] = (cv[m] && !a.x0_zero && gcol[m] + e < p) ? static_cast<A>(xin[gcol[m] + e]) : A(0);
        d[j] = g[j] = u1[j] = u2[j] = A(0);
      }
    const bool eq1 = a.prm.method == GPL1_METHOD_ISTA || a.prm.method == GPL1_METHOD_FISTA;
    if (!a.x0_zero && !eq1) project_x0();   // Alg. GP and PSD start in Omega; eq. 1 has no ball
    int k = 0;
    // setup pass: g_0 = 2 K^T (K x0 - y), f(x0), ||y||^2
    pass<true>(0);
    if (gsync()) {
      phase_l0();
      int s = 0;
      // One pass per trip.  Alg. GP + SS: projection phase, pass, line search.
      // ISTA / FISTA: step phase, pass, whole step.  PSD: two trips per
      // iteration, a probe along g_k (mode 1) and the projected step (mode 2).
      const bool gpss = a.prm.method == GPL1_METHOD_GPSS;
      const bool psd = a.prm.method == GPL1_METHOD_PSD;
      int mode = psd ? 1 : 0;
      bool tail = false;   // eq. 1: stopped after a whole step (max_iter)
      if (!u.done) {
        for (k = 0;;) {
          if (tid == 0 && a.trace) u.ts[0] = globaltimer();
          // stop at x_k (a stop test or the FW certificate) or failure
          if (!(gpss ? phase_p(k, s) : phase_m(k, s, mode))) break;
          ++s;
          pass<false>(s);
          if (tid == 0 && a.trace) u.ts[1] = globaltimer();
          if (!gsync()) break;
          const int act = gpss ? phase_l(k, s) : phase_lm(k, s, mode);
          if (mode == 1) {   // PSD probe: x unchanged, the step follows
            if (act != 0) break;
            mode = 2;
            continue;
          }
          if (act != 2) {   // x_{k+1} = x_k + lam d_k (lam = 1 for the methods of Sec. 2)
            const A la = kF64 ? static_cast<A>(u.lam) : static_cast<A>(u.lf);
#pragma unroll
            for (int j = 0; j < NE; ++j) x[j] = vfma(la, d[j], x[j]);
          }
          if (act != 0) {
            tail = act == 1;   // the same decision in every CTA (identical scalars)
            break;
          }
          ++k;
          if (psd) mode = 1;
        }
      }
      if (eq1 && tail) eq1_objective_tail();
    }
    drain();
    // the solution: cluster 0 writes its copy
    if (cid == 0 && !failed()) {
      V* const xo = static_cast<V*>(a.x);
#pragma unroll
      for (int m = 0; m < NCH; ++m)
#pragma unroll
        for (int e = 0; e < EPC; ++e)
          if (cv[m] && gcol[m] + e < p) xo[gcol[m] + e] = static_cast<V>(x[m * EPC + e]);
    }
    if (cta == 0 && tid == 0) {
      int st = u.status;
      const int e = sm.ctl[CTL_ERR] ? sm.ctl[CTL_ERR] : status;
      if (e != GPL1_OK) st = e;
      gpl1_result r;
      r.status = st;
      r.stop = (st != GPL1_OK && st != GPL1_ERR_NOT_CONVERGED) ? GPL1_STOP_ERROR : u.stop;
      r.iters = u.iters;
      r.backtracks = u.backtracks;
      r.f = eq1 ? u.F_cur : u.f_cur;
      r.rel_gap = a.f_star > 0.0 ? (r.f - a.f_star) / a.f_star : -1.0;
      r.fw_gap = eq1 ? -1.0 : u.gx + a.rho * u.gmax;
      r.lambda = 0.5 * u.gmax;
      r.alpha = u.alpha;
      r.tau = kF64 ? u.tau64 : static_cast<double>(u.th) + static_cast<double>(u.tl);
      r.kernel_ms = 0.0;
      r.fail_site = sm.ctl[CTL_SITE];
      r.fail_iter = u.iters;
      *a.res = r;
    }
  }
};

// ================================================================= producer
// One lane streams the cluster's row blocks of this CTA's slice, pass after
// pass (serpentine order), into the stage ring until the consumers stop it.
template <int DT, int NCH>
__device__ void producer(const FArgs& a, const CUtensorMap* tmap, FSmem<DT, NCH>& sm) {
  using CF = Cfg<DT, NCH>;
  constexpr int R = CF::R;
  const unsigned rank = cl_rank(), cid = cl_id();
  const int NBt = (a.n + R - 1) / R;
  const int bk0 = static_cast<int>(static_cast<long long>(NBt) * cid / a.NC);
  const int bk1 = static_cast<int>(static_cast<long long>(NBt) * (cid + 1) / a.NC);
  const int nb = bk1 - bk0;
  const int c0 = static_cast<int>(rank) * CF::W;
  const int rest = a.p - c0;
  const int nbox = rest <= 0 ? 0 : min(CF::NBOX, (rest + kBoxW - 1) / kBoxW);
  volatile int* ctl = sm.ctl;
  // Two streams of the same block sequence (pass after pass, serpentine):
  // A into the A ring (the first read of a block, from HBM), B into the B
  // ring (the second read, normally served by L2).  A block's B load is issued
  // only after its A load.  The lane polls both rings' empty barriers and
  // issues into whichever has room.
  uint32_t ia = 0, ib = 0;   // loads issued per ring
  int pa = 0, qa = 0, pb = 0, qb = 0;   // (pass, position in the pass) of the next A and B block
  auto block_of = [&](int pass, int q) { return (pass & 1) == 0 ? bk0 + q : bk1 - 1 - q; };
  auto load = [&](int st, int b) {
    mbar_arrive_expect_tx(&sm.full[st], static_cast<uint32_t>(nbox * CF::BOXB));
    for (int i = 0; i < nbox; ++i)
      tma_load_2d(sm.stage[st] + i * CF::BOXB, tmap, &sm.full[st], c0 + i * kBoxW, b * R);
  };
  if (nb > 0) {
    uint64_t t0 = globaltimer();
    for (unsigned poll = 0;; ++poll) {
      bool did = false;
      if (mbar_test(&sm.empty[ia % CF::NSA], ((ia / CF::NSA) & 1u) ^ 1u)) {
        if (ctl[CTL_STOP]) goto done;
        load(static_cast<int>(ia % CF::NSA), block_of(pa, qa));
        ++ia;
        ctl[CTL_ISSUED] = static_cast<int>(ia);
        if (++qa == nb) {
          qa = 0;
          ++pa;
        }
        did = true;
      }
      if (ib < ia && mbar_test(&sm.empty[CF::NSA + ib % CF::NSB], ((ib / CF::NSB) & 1u) ^ 1u)) {
        if (ctl[CTL_STOP]) goto done;
        load(static_cast<int>(CF::NSA + ib % CF::NSB), block_of(pb, qb));
        ++ib;
        ctl[CTL_ISSUED_B] = static_cast<int>(ib);
        if (++qb == nb) {
          qb = 0;
          ++pb;
        }
        did = true;
      }
      if (did) {
        t0 = globaltimer();
        continue;
      }
      __nanosleep(128);   // nothing to issue: yield the issue slots to the consumer warps
      if ((poll & 15u) != 15u) continue;
      if (ctl[CTL_STOP]) goto done;
      if (globaltimer() - t0 > static_cast<uint64_t>(a.prm.timeout_ns)) {
        if (!ctl[CTL_ERR]) ctl[CTL_SITE] = kSiteProducer;
        ctl[CTL_ERR] = GPL1_ERR_TIMEOUT;
        goto done;
      }
    }
  }
done:
  __threadfence_block();
  ctl[CTL_DONE] = 1;
}

template <int DT, int NCH>
__global__ void __launch_bounds__(kThr, 1) fused_kernel(const __grid_constant__ FArgs a,
                                                         const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t fz_dyn[];
  FSmem<DT, NCH>& sm =
      *reinterpret_cast<FSmem<DT, NCH>*>((reinterpret_cast<uintptr_t>(fz_dyn) + 127) & ~static_cast<uintptr_t>(127));
  const int tid = threadIdx.x;
  // The launch must have the shape the arguments describe (clusters of C CTAs,
  // C x NC CTAs, kThr threads): every exchange below addresses the peers'
  // shared memory by cluster rank.  Otherwise report and leave untouched.
  if (cl_size() != static_cast<unsigned>(a.C) || gridDim.x != static_cast<unsigned>(a.C * a.NC) ||
      blockDim.x != static_cast<unsigned>(kThr)) {
    if (blockIdx.x == 0 && tid == 0) {
      atomicCAS(a.err, 0, GPL1_ERR_CUDA);
      a.res->status = GPL1_ERR_CUDA;
      a.res->stop = GPL1_STOP_ERROR;
    }
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < Cfg<DT, NCH>::NST; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], kWarps);
    }
    for (int s = 0; s < kNRed; ++s) mbar_init(&sm.redfull[s], kWarps);
    for (int s = 0; s < kRNS; ++s) {
      mbar_init(&sm.rfull[s], 1);
      mbar_init(&sm.rempty[s], static_cast<uint32_t>(a.C));
    }
    for (int s = 0; s < kNTot; ++s) {
      mbar_init(&sm.tfull[s], 1);
      mbar_init(&sm.tcons[s], kWarps);
    }
    // (shared memory keeps whatever the previous kernel on this SM left:
    // everything read before it is written starts cleared here)
    for (int q = 0; q < 32; ++q)
      for (int i = 0; i < 6; ++i) sm.rowacc[q][i] = 0u;
    for (int s = 0; s < kSNS; ++s) {
      mbar_init(&sm.sfull[s], 1);
      mbar_init(&sm.sempty[s], static_cast<uint32_t>(a.C));
    }
    for (int q = 0; q < 8; ++q) sm.ctl[q] = 0;
    mbar_fence_init();
  }
  __syncthreads();
  cl_arrive();   // every CTA of the cluster has initialised its barriers
  cl_wait();
  if (tid >= kTot) {   // the totaler warp
    FC<DT, NCH> c(a, sm);
    c.total_loop();
    __syncwarp();
  } else if (tid >= kSend) {   // the sender warp
    FC<DT, NCH> c(a, sm);
    c.send_loop();
    __syncwarp();
  } else if (tid >= kProd) {   // the producer warp (one lane)
    if (tid == kProd) producer<DT, NCH>(a, &tmap, sm);
    __syncwarp();
  } else {
    FC<DT, NCH> c(a, sm);
    c.run();
    __syncwarp();
  }
  __syncthreads();
  cl_arrive();   // no CTA leaves while a peer may still address its shared memory
  cl_wait();
}

template <int DT, int NCH>
constexpr size_t fused_smem_bytes() {
  return sizeof(FSmem<DT, NCH>) + 128;
}

}  // namespace fz
}  // namespace gpl1
