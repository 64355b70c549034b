// Instantiation of the GPSS kernel for K stored as GPL1_BF16.
#include "gpss.cuh"

namespace gpl1 {

cudaError_t launch_gpss_bf16(const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative, cudaStream_t stream,
                           int tile) {
  return GpssHost<GPL1_BF16>::launch(tile, a, tmap, grid, cooperative, stream);
}
size_t gpss_smem_bytes_bf16(int tile) { return GpssHost<GPL1_BF16>::smem(tile); }
const void* gpss_kernel_ptr_bf16(int tile) { return GpssHost<GPL1_BF16>::kernel(tile); }

}  // namespace gpl1
