// BF16 tensor-core GEMM for sm_103a (tcgen05, TMA, tensor memory): the
// products K^T R and K [D X] of the shared-K multi-right-hand-side form of
// Alg. GP, where many instances of eq. 2 share one K and the gradient and the
// K-products of all of them become matrix products.
//
//   C (M x N, FP32) = A (M x Kd) * B (N x Kd)^T,
//   out[n * ldo + m] = scale * C[m][n]   (transposed store), or
//   out[m * ldo + n] = scale * C[m][n]   (row-major store)
//
// A and B are BF16, row-major with K contiguous (K-major).  A may be shorter
// along K than B (Ka < Kd): its K coordinate wraps modulo Ka, so the split
// vector operand [hi | mid | lo] of B multiplies the same A three times in one
// accumulation.  The transposed store makes each right-hand side's vector
// contiguous; the row-major one keeps batch-major activations batch-major.
//
// One CTA per 128 x BN tile and split of the contraction, 128 threads: thread 0
// issues the TMA loads of an ST-stage ring (128-byte swizzle), thread 32 issues
// the MMAs (128 x BN x 16 per instruction, FP32 accumulator in tensor memory),
// and all four warps read the accumulator back (warp w owns tensor-memory
// lanes 32w .. 32w+31, i.e. rows m0 + 32w ..) and store it.  Every wait is
// bounded; a wait that runs out sets *err and the CTA still releases its
// tensor memory.
//
// Split-K: with S splits, CTA (x, y, z) sums k-blocks [z KB / S, (z+1) KB / S)
// and writes its partial product to out + z * split_stride; the S partials
// add up to the product (the consumer sums them in a fixed order, so results
// do not depend on scheduling).  This fills the 152 SMs when M x N has few
// tiles and the contraction is long.
//
// Configurations (the autotuner of the shared-K solve picks one per shape):
//   0: BN 128, 4 stages (132 KB shared memory, one CTA per SM)
//   1: BN 256, 4 stages (193 KB, one CTA per SM)
//   2: BN 128, 3 stages (97 KB, two CTAs per SM: one's epilogue overlaps the
//      other's main loop)
//   3: BN 128, 6 stages (193 KB, one CTA per SM: deeper load pipeline)
#include <cudaTypedefs.h>

#include "launch.h"
#include "tcgen05.cuh"

namespace gpl1 {

constexpr int kTcBM = 128, kTcBK = 64;

struct GemmArgs {
  int M, N, Kd, Ka;
  float* out;
  long long ldo;
  float scale;
  int* err;
  long long timeout_ns;
  int trans_out;
  int splits;
  long long split_stride;
};

template <int BN, int ST>
struct GemmLayout {
  static constexpr int kA = kTcBM * kTcBK * 2;   // 16 KB
  static constexpr int kB = BN * kTcBK * 2;      // 16 or 32 KB
  static constexpr int kStage = kA + kB;         // a multiple of 1024 (swizzle atoms)
  static constexpr size_t kBytes = static_cast<size_t>(ST) * kStage + 128 + 1024;
};

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

template <int BN, int ST>
__global__ void __launch_bounds__(128, 1) gemm_bf16_tn(const __grid_constant__ CUtensorMap ta,
                                                       const __grid_constant__ CUtensorMap tb, const GemmArgs g) {
  constexpr int kTcStages = ST;
  using L = GemmLayout<BN, ST>;
  extern __shared__ uint8_t gemm_raw[];
  uint8_t* const base =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gemm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* const full = reinterpret_cast<uint64_t*>(base + kTcStages * L::kStage);
  uint64_t* const empty = full + kTcStages;
  uint64_t* const done = empty + kTcStages;
  uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* const state = reinterpret_cast<int*>(tmem_slot + 1);   // [0] error, [1] loads issued, [2] stages consumed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
  // this CTA's k-blocks: [kb0, kb0 + KB) of the Kd / 64 in all
  const int KT = g.Kd / kTcBK, z = blockIdx.z;
  const int kb0 = static_cast<int>(static_cast<long long>(z) * KT / g.splits);
  const int KB = static_cast<int>(static_cast<long long>(z + 1) * KT / g.splits) - kb0;
  float* const out = g.out + static_cast<long long>(z) * g.split_stride;
  const uint64_t lim = static_cast<uint64_t>(g.timeout_ns);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    state[0] = state[1] = state[2] = 0;
    mbar_fence_init();
  }
  if (warp == 2) {
    tc::tmem_alloc(tmem_slot, BN);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();   // the operands come from the previous kernel of the stream
  pdl_trigger();

  if (warp == 0 && lane == 0) {   // TMA producer
    int kb = 0;
    for (; kb < KB; ++kb) {
      const int s = kb % kTcStages;
      if (kb >= kTcStages && !wait_bounded(&empty[s], static_cast<uint32_t>((kb / kTcStages - 1) & 1), lim)) {
        state[0] = 1;
        break;
      }
      uint8_t* const sa = base + s * L::kStage;
      mbar_arrive_expect_tx(&full[s], L::kStage);
      tma_load_2d(sa, &ta, &full[s], ((kb0 + kb) * kTcBK) % g.Ka, m0);
      tma_load_2d(sa + L::kA, &tb, &full[s], (kb0 + kb) * kTcBK, n0);
    }
    state[1] = kb;
  } else if (warp == 1 && lane == 0) {   // MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcBM, BN);
    int kb = 0;
    for (; kb < KB; ++kb) {
      const int s = kb % kTcStages;
      if (!wait_bounded(&full[s], static_cast<uint32_t>((kb / kTcStages) & 1), lim)) {
        state[0] = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t sa = smem_u32(base + s * L::kStage);
      const uint64_t ad = tc::sdesc_kmajor_sw128(sa);
      const uint64_t bd = tc::sdesc_kmajor_sw128(sa + L::kA);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk)   // 16 BF16 = 32 bytes = 2 descriptor units per step
        tc::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
      tc::commit(&empty[s]);   // the stage is free once these MMAs have read it
    }
    state[2] = kb;
    tc::commit(done);          // arrives when every MMA issued above has completed
  }
  __syncwarp();
  __syncthreads();
  const bool failed = reinterpret_cast<volatile int*>(state)[0] != 0;
  const bool ready = wait_bounded(done, 0, lim);
  tc::fence_after_sync();
  if (ready && !failed) {
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tc::ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c0), v);
      if (m < g.M) {
        if (g.trans_out) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int n = n0 + c0 + q;
            if (n < g.N) out[static_cast<long long>(n) * g.ldo + m] = g.scale * v[q];
          }
        } else {
          float* row = out + static_cast<long long>(m) * g.ldo + n0 + c0;
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (n0 + c0 + q < g.N) row[q] = g.scale * v[q];
        }
      }
    }
  }
  if (threadIdx.x == 0 && (failed || !ready)) {
    atomicCAS(g.err, 0, static_cast<int>(GPL1_ERR_TIMEOUT));
    // loads issued but never consumed land within microseconds: let them
    // complete before the CTA (and its shared memory) goes away
    for (int kb = state[2]; kb < state[1]; ++kb)
      wait_bounded(&full[kb % kTcStages], static_cast<uint32_t>((kb / kTcStages) & 1), 2000000000ull);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, BN);
}

namespace {

CUresult encode_kmajor(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map, const void* ptr, long long rows,
                       long long cols, long long ld, int box_rows) {
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcBK), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int BN, int ST>
cudaError_t launch_cfg(const CUtensorMap& ta, const CUtensorMap& tb, const GemmArgs& g, cudaStream_t stream) {
  const size_t smem = GemmLayout<BN, ST>::kBytes;
  // the attribute is set once per instantiation and device (the context is bound to one device)
  static int set_for = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (set_for != dev) {
    e = cudaFuncSetAttribute(gemm_bf16_tn<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    set_for = dev;
  }
  const dim3 grid((g.M + kTcBM - 1) / kTcBM, (g.N + BN - 1) / BN, g.splits);
  return launch_pdl(gemm_bf16_tn<BN, ST>, grid, dim3(128), smem, stream, ta, tb, g);
}

}  // namespace

int gemm_cfg_bn(int cfg) { return cfg == 1 ? 256 : 128; }

int launch_gemm_bf16_cfg(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda,
                         const void* B, int N, int Kd, long long ldb, float* out, long long ldo, float scale,
                         int* err, long long timeout_ns, int cfg, int splits, long long split_stride,
                         cudaStream_t stream, int trans_out) {
  if (cfg < 0 || cfg >= kGemmConfigs || splits < 1 || splits > Kd / kTcBK) return static_cast<int>(cudaErrorInvalidValue);
  CUtensorMap ta, tb;
  if (encode_kmajor(enc, &ta, A, M, Ka, lda, kTcBM) != CUDA_SUCCESS) return -1;
  if (encode_kmajor(enc, &tb, B, N, Kd, ldb, gemm_cfg_bn(cfg)) != CUDA_SUCCESS) return -1;
  GemmArgs g{M, N, Kd, Ka, out, ldo, scale, err, timeout_ns, trans_out, splits, split_stride};
  cudaError_t e;
  switch (cfg) {
    case 1: e = launch_cfg<256, 4>(ta, tb, g, stream); break;
    case 2: e = launch_cfg<128, 3>(ta, tb, g, stream); break;
    case 3: e = launch_cfg<128, 6>(ta, tb, g, stream); break;
    default: e = launch_cfg<128, 4>(ta, tb, g, stream); break;
  }
  return static_cast<int>(e);
}

int launch_gemm_bf16(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda,
                     const void* B, int N, int Kd, long long ldb, float* out, long long ldo, float scale, int* err,
                     long long timeout_ns, int bn, cudaStream_t stream, int trans_out) {
  return launch_gemm_bf16_cfg(enc, A, M, Ka, lda, B, N, Kd, ldb, out, ldo, scale, err, timeout_ns, bn == 256 ? 1 : 0,
                              1, 0, stream, trans_out);
}

}  // namespace gpl1
