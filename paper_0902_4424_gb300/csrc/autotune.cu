// Autotuner for the tensor-core products of the shared-K form.
//
// A product's best tile shape and split of the contraction depend on its
// shape: C = A B^T with M x N output tiles of 128 x BN fills the 152 SMs only
// when M N / (128 BN) is large, while a long contraction over few tiles needs
// a split-K to use the machine.  autotune_gemm times every configuration of
// gemm_tc.cu and every admissible split on the product's real operands (CUDA
// events on the caller's stream), adds the cost of summing the extra partials
// in the consumer kernel, and returns the fastest.  The caller caches the
// result per shape, so a shape is tuned once per context.
#include <cudaTypedefs.h>

#include "launch.h"

namespace gpl1 {

int autotune_gemm(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda, const void* B,
                  int N, int Kd, long long ldb, float* out, long long ldo, float scale, int* err, long long timeout_ns,
                  int max_splits, long long split_stride, double sum_gbs, cudaStream_t stream, GemmChoice* best) {
  constexpr int kReps = 3;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = static_cast<int>(cudaEventCreate(&e0));
  if (rc) return rc;
  rc = static_cast<int>(cudaEventCreate(&e1));
  if (rc) {
    cudaEventDestroy(e0);
    return rc;
  }
  const int kt = Kd / 64;
  best->cfg = 0;
  best->splits = 1;
  best->ms = -1.f;
  float best_cost = 0.f;
  for (int cfg = 0; cfg < kGemmConfigs && rc == 0; ++cfg) {
    for (int s = 1; s <= max_splits && rc == 0; ++s) {
      if (s > 1 && kt / s < 8) break;   // splits of fewer than 8 k-blocks are all prologue and epilogue
      auto launch = [&] {
        return launch_gemm_bf16_cfg(enc, A, M, Ka, lda, B, N, Kd, ldb, out, ldo, scale, err, timeout_ns, cfg, s,
                                    split_stride, stream);
      };
      if ((rc = launch()) != 0) break;   // warm-up (and the one-time attribute setting)
      if ((rc = static_cast<int>(cudaEventRecord(e0, stream))) != 0) break;
      for (int r = 0; r < kReps && rc == 0; ++r) rc = launch();
      if (rc) break;
      if ((rc = static_cast<int>(cudaEventRecord(e1, stream))) != 0) break;
      if ((rc = static_cast<int>(cudaEventSynchronize(e1))) != 0) break;
      float ms = 0.f;
      if ((rc = static_cast<int>(cudaEventElapsedTime(&ms, e0, e1))) != 0) break;
      ms /= kReps;
      // the consumer reads s partial slices instead of one and writes the sum back
      const double extra = s > 1 ? static_cast<double>(s) * M * N * 4.0 / (sum_gbs * 1e9) * 1e3 : 0.0;
      const float cost = ms + static_cast<float>(extra);
      if (best->ms < 0.f || cost < best_cost) {
        best->cfg = cfg;
        best->splits = s;
        best->ms = ms;
        best_cost = cost;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace gpl1
