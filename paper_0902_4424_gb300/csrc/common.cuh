// Device-side building blocks shared by the gpl1 kernels (sm_103a).
//
//  * element traits for the three storage types of K;
//  * mbarrier / TMA (cp.async.bulk.tensor) wrappers in inline PTX;
//  * consumer-only named barriers and a bounded grid barrier;
//  * deterministic block reductions for the 512 consumer threads.
//
// Every wait in this file is bounded by a deadline on %globaltimer; a wait that
// runs out sets the kernel's error flag and returns instead of spinning.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/gpl1.h"

namespace gpl1 {

// ------------------------------------------------------------------ layout
constexpr int kBoxCols = 256;                 // columns of K per TMA box (one "strip")
constexpr int kConsumerWarps = 15;            // + 1 producer = 16 warps: 128 registers/thread
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;     // + one TMA producer warp
constexpr int kRingBytes = 122880;            // the two-pass kernel's smem ring (120 KiB, every tile)
constexpr int kHistBins = 2048;               // radix-select digit of 11 bits
constexpr int kBinsPerThread = (kHistBins + kConsumers - 1) / kConsumers;
constexpr int kMaxM = 16;                     // non-monotone memory supported
constexpr int kMaxMalpha = 8;                 // BB2 window supported

// Storage traits: E = element of K, A = accumulator of products with K,
// V = element of x and y.  RB = rows per TMA box of the default tile (a box
// of 30 KiB whose rows split evenly over the consumer warps).
template <int DT> struct Traits;
template <> struct Traits<GPL1_F64> {
  using E = double; using A = double; using V = double;
  static constexpr int ES = 8, RB = 15;
};
template <> struct Traits<GPL1_F32> {
  using E = float; using A = float; using V = float;
  static constexpr int ES = 4, RB = 30;
};
template <> struct Traits<GPL1_BF16> {
  using E = __nv_bfloat16; using A = float; using V = float;
  static constexpr int ES = 2, RB = 60;
};

// Box shapes of the two-pass kernel (gpl1_params.tile): a TMA box is RB rows
// x 256 columns with RB = RPW rows per consumer warp x kConsumerWarps, and the
// ring holds kRingBytes in every shape:
//   GPL1_TILE_SMALL   15 KiB boxes, 8 stages (F32: RB 15, BF16: RB 30)
//   GPL1_TILE_MEDIUM  30 KiB boxes, 4 stages (F64: 15, F32: 30, BF16: 60)
//   GPL1_TILE_LARGE   60 KiB boxes, 2 stages (F64: 30, F32: 60, BF16: 120)
// FP64 has no SMALL shape (a warp takes at least one row of a box).
template <int DT, int TL>
struct Tile {
  static constexpr int BOX = 15360 << (TL - GPL1_TILE_SMALL);      // bytes per box
  static constexpr int STAGES = kRingBytes / BOX;
  static constexpr int RB = BOX / (kBoxCols * Traits<DT>::ES);      // rows per box
  static constexpr int RPW = RB / kConsumerWarps;                   // rows per warp
  static_assert(TL >= GPL1_TILE_SMALL && TL <= GPL1_TILE_LARGE, "tile");
  static_assert(RPW >= 1 && RPW * kConsumerWarps == RB && RPW <= 8, "rows of a box split over the warps");
};
__host__ __device__ constexpr bool tile_valid(int dt, int tl) {
  return tl >= GPL1_TILE_SMALL && tl <= GPL1_TILE_LARGE && !(dt == GPL1_F64 && tl == GPL1_TILE_SMALL);
}
__host__ __device__ constexpr int tile_rows(int dt, int tl) {
  return (15360 << (tl - GPL1_TILE_SMALL)) / (kBoxCols * (dt == GPL1_F64 ? 8 : dt == GPL1_F32 ? 4 : 2));
}

// Each lane owns 8 columns of a 256-column strip: NCH 16-byte chunks, chunk m
// of lane l starting at element (l + 32 m) * EPC.
template <int DT> struct LaneCols {
  static constexpr int ES = Traits<DT>::ES;
  static constexpr int EPC = 16 / ES;   // elements per 16-byte chunk
  static constexpr int NCH = 8 / EPC;   // chunks per lane
  __device__ static __forceinline__ int col(int lane, int e) {
    return (lane + 32 * (e / EPC)) * EPC + (e % EPC);
  }
};

template <int DT>
__device__ __forceinline__ void load_row8(const uint8_t* row, int lane, typename Traits<DT>::A (&o)[8]);

template <>
__device__ __forceinline__ void load_row8<GPL1_F64>(const uint8_t* row, int lane, double (&o)[8]) {
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const double2 c = *reinterpret_cast<const double2*>(row + (lane + 32 * m) * 16);
    o[2 * m] = c.x;
    o[2 * m + 1] = c.y;
  }
}
template <>
__device__ __forceinline__ void load_row8<GPL1_F32>(const uint8_t* row, int lane, float (&o)[8]) {
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const float4 c = *reinterpret_cast<const float4*>(row + (lane + 32 * m) * 16);
    o[4 * m] = c.x; o[4 * m + 1] = c.y; o[4 * m + 2] = c.z; o[4 * m + 3] = c.w;
  }
}
template <>
__device__ __forceinline__ void load_row8<GPL1_BF16>(const uint8_t* row, int lane, float (&o)[8]) {
  const uint4 c = *reinterpret_cast<const uint4*>(row + lane * 16);
  const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[2 * q] = __uint_as_float(w[q] << 16);
    o[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
  }
}

// Typed math helpers for templated code: a bare fabs/fma/fmax on a float can
// resolve to the double overload, which on GB300 means conversions plus
// FP64-pipe instructions of ~75-cycle latency for every element.
__device__ __forceinline__ float vabs(float x) { return fabsf(x); }
__device__ __forceinline__ double vabs(double x) { return fabs(x); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }

// ------------------------------------------------------------------- PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Warp sum of NV values at once (NV a power of two, at most 32): at each of the
// first log2 NV butterfly levels a lane keeps half of its values and adds the
// partner's copy of that half, so the warp exchanges NV - 1 + (5 - log2 NV)
// values instead of 5 NV.  On return every lane of the group of 32 / NV lanes
// starting at lane q * (32 / NV) holds the warp total of v[q].
template <int NV>
__device__ __forceinline__ float warp_sum_many(float (&v)[NV], int lane) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  int o = 16;
#pragma unroll
  for (int n = NV; n > 1; n >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = upper ? v[i] : v[i + n / 2];
      const float keep = upper ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute may start (block scheduling, prologue) while
// its predecessor in the stream still runs; pdl_wait() blocks until the
// predecessor has completed and its memory is visible (a no-op for a kernel
// launched without the attribute), pdl_trigger() lets the successor launch.
// Every kernel of the shared-K iteration waits before its first global access.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with the programmatic stream-serialization attribute (host side).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// c0 = column (innermost), c1 = row.  Out-of-range elements are zero-filled.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
// Named barrier 1 over the consumer warps (the producer warp never joins).
// The non-aligned form: it is defined when the threads of a warp reach it at
// different times (lead-only sections, loops with uneven trip counts right
// before it), which the aligned bar.sync leaves undefined; with bar.sync the
// FP64 solver stalled in such a section.
__device__ __forceinline__ void consumer_sync() { asm volatile("barrier.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Reductions into global memory (no return value: compiled as red, not atom).
__device__ __forceinline__ void red_add(float* addr, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}
__device__ __forceinline__ void red_add(double* addr, double a) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(a) : "memory");
}
__device__ __forceinline__ void red_add2(float* addr, float a, float b) {   // 8-byte aligned pair
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add2(double* addr, double a, double b) {
  red_add(addr, a);
  red_add(addr + 1, b);
}

// ------------------------------------------------------- shared scratch

// Error-free transformations (Knuth two-sum, FMA two-product): a float pair
// (hi, lo) carries a sum with about 48 significant bits while every operation
// stays on the FP32 pipe.  GB300 runs FP64 at a small fraction of the FP32
// rate, so bulk reductions use these and only O(1) scalars use FP64.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ F2 f2_add(F2 x, float y) {
  F2 s = two_sum(x.hi, y);
  s.lo += x.lo;
  return two_sum(s.hi, s.lo);
}
__device__ __forceinline__ F2 f2_fma(F2 acc, float a, float b) {   // acc + a*b, product exact
  float p = __fmul_rn(a, b);   // not contracted into the following add
  float e = fmaf(a, b, -p);
  F2 s = two_sum(acc.hi, p);
  s.lo += acc.lo + e;
  return two_sum(s.hi, s.lo);
}

// warp_sum_many for float pairs: the same halving butterfly, each combine an
// error-free two-sum of the high words with the low words and the rounding
// error added to the low word.
template <int NV>
__device__ __forceinline__ F2 warp_sum_many_f2(F2 (&v)[NV], int lane) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two <= 32");
  int o = 16;
#pragma unroll
  for (int n = NV; n > 1; n >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const F2 send = upper ? v[i] : v[i + n / 2];
      const F2 keep = upper ? v[i + n / 2] : v[i];
      const float oh = __shfl_xor_sync(0xffffffffu, send.hi, o);
      const float ol = __shfl_xor_sync(0xffffffffu, send.lo, o);
      const F2 t = two_sum(keep.hi, oh);
      v[i] = F2{t.hi, __fadd_rn(__fadd_rn(keep.lo, ol), t.lo)};
    }
  }
#pragma unroll
  for (; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, v[0].hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, v[0].lo, o);
    const F2 t = two_sum(v[0].hi, oh);
    v[0] = F2{t.hi, __fadd_rn(__fadd_rn(v[0].lo, ol), t.lo)};
  }
  return v[0];
}

struct Scratch {
  double d[kConsumerWarps][8];   // per-warp partials of block reductions (FP64 data)
  F2 f2[kConsumerWarps][8];      // per-warp partials of block reductions (float data)
  unsigned long long u[kConsumerWarps][2];
  double bcast[8];
  unsigned long long ubcast[4];
  int flags[4];
  unsigned long long u2[kConsumerWarps][2];
  unsigned c2[kConsumerWarps][2];
  // threshold search state published by one lane
  unsigned long long ub[4];
  long long tt[8];   // lead-lane clock stamps inside the threshold search (trace only)
  unsigned cnt_prev;
  double dtau, cprev;
  float tp[4];
  int tflag;
};

// Block reductions over the kConsumers threads.  Each warp reduces with
// shuffles, lane 0 stores the warp value, warp 0 combines the (at most 16)
// warp values in a fixed order and publishes the result; every thread then
// reads the same value.  Only warp 0's lane 0 touches FP64, so the slow FP64
// pipe of GB300 sees O(1) work per reduction instead of O(threads).
static_assert(kConsumerWarps <= 16, "warp 0 combines at most 16 warp values");

template <int N>
__device__ __forceinline__ void block_sum_f2(F2 (&v)[N], double (&out)[N], Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      F2 t{__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
      v[q] = f2_add(v[q], t);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) sc.f2[warp][q] = v[q];
  }
  consumer_sync();
  if (warp == 0) {
    F2 w[N];
#pragma unroll
    for (int q = 0; q < N; ++q) w[q] = lane < kConsumerWarps ? sc.f2[lane][q] : F2{0.f, 0.f};
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        F2 t{__shfl_xor_sync(0xffffffffu, w[q].hi, o), __shfl_xor_sync(0xffffffffu, w[q].lo, o)};
        w[q] = f2_add(w[q], t);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < N; ++q) sc.bcast[q] = static_cast<double>(w[q].hi) + static_cast<double>(w[q].lo);
    }
  }
  consumer_sync();
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = sc.bcast[q];
}

// Same for double partials (the FP64 storage path).
template <int N>
__device__ __forceinline__ void block_sum_f64(double (&v)[N], double (&out)[N], Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) sc.d[warp][q] = v[q];
  }
  consumer_sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      double s = 0.0;
      for (int w = 0; w < kConsumerWarps; ++w) s += sc.d[w][q];
      sc.bcast[q] = s;
    }
  }
  consumer_sync();
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = sc.bcast[q];
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if (lane == 0) sc.u[warp][0] = v;
  consumer_sync();
  unsigned long long m = sc.u[0][0];
#pragma unroll
  for (int w = 1; w < kConsumerWarps; ++w) m = sc.u[w][0] > m ? sc.u[w][0] : m;
  consumer_sync();
  return m;
}

// Maximum of non-negative values through their bit patterns (which order
// like the values): integer work only.
__device__ __forceinline__ double block_max_nonneg(double v, Scratch& sc) {
  const unsigned long long m = block_max_u64(static_cast<unsigned long long>(__double_as_longlong(v)), sc);
  return __longlong_as_double(static_cast<long long>(m));
}
__device__ __forceinline__ float block_max_nonneg(float v, Scratch& sc) {
  const unsigned long long m = block_max_u64(static_cast<unsigned long long>(__float_as_uint(v)), sc);
  return __uint_as_float(static_cast<unsigned>(m));
}

// (hi, lo) float pair of a double, for broadcasting FP64 scalars to threads
// that then work on the FP32 pipe.  Called by one thread.
__device__ __forceinline__ F2 f2_of(double t) {
  const float h = static_cast<float>(t);
  return {h, static_cast<float>(t - static_cast<double>(h))};
}

__device__ __forceinline__ int block_or(int v, Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = __any_sync(0xffffffffu, v);
  if (lane == 0) sc.u[warp][1] = static_cast<unsigned long long>(v);
  consumer_sync();
  int r = 0;
#pragma unroll
  for (int w = 0; w < kConsumerWarps; ++w) r |= static_cast<int>(sc.u[w][1]);
  consumer_sync();
  return r;
}

// Block reduction finished by the leading thread only: N sums (float pairs or
// doubles) and one unsigned max, returned in thread 0's arguments.  The caller
// lets thread 0 decide, then publishes the decision with one consumer_sync.
template <int N, typename S>
__device__ __forceinline__ void lead_reduce(S (&v)[N], unsigned& mx, Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if constexpr (sizeof(S) == 8 && !std::is_same<S, F2>::value) {
        v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
      } else {
        F2 t{__shfl_xor_sync(0xffffffffu, v[q].hi, o), __shfl_xor_sync(0xffffffffu, v[q].lo, o)};
        v[q] = f2_add(v[q], t);
      }
    }
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if constexpr (std::is_same<S, F2>::value) sc.f2[warp][q] = v[q];
      else sc.d[warp][q] = v[q];
    }
    sc.c2[warp][0] = mx;
  }
  consumer_sync();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if constexpr (std::is_same<S, F2>::value) {
        F2 t = sc.f2[0][q];
        for (int w = 1; w < kConsumerWarps; ++w) t = f2_add(t, sc.f2[w][q]);
        v[q] = t;
      } else {
        double t = sc.d[0][q];
        for (int w = 1; w < kConsumerWarps; ++w) t += sc.d[w][q];
        v[q] = t;
      }
    }
    unsigned m = sc.c2[0][0];
    for (int w = 1; w < kConsumerWarps; ++w) m = max(m, sc.c2[w][0]);
    mx = m;
  }
}

// Exact sum of unsigned 64-bit integers over the block (associative: the same
// in every CTA whatever the order).
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, Scratch& sc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sc.u[warp][0] = v;
  consumer_sync();
  unsigned long long s = 0;
#pragma unroll
  for (int w = 0; w < kConsumerWarps; ++w) s += sc.u[w][0];
  consumer_sync();
  return s;
}

}  // namespace gpl1
