// Instantiation of the GPSS kernel for K stored as GPL1_F32.
#include "gpss.cuh"

namespace gpl1 {

cudaError_t launch_gpss_f32(const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative, cudaStream_t stream,
                           int tile) {
  return GpssHost<GPL1_F32>::launch(tile, a, tmap, grid, cooperative, stream);
}
size_t gpss_smem_bytes_f32(int tile) { return GpssHost<GPL1_F32>::smem(tile); }
const void* gpss_kernel_ptr_f32(int tile) { return GpssHost<GPL1_F32>::kernel(tile); }

}  // namespace gpl1
