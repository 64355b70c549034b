// Instantiation of the GPSS kernel for K stored as GPL1_F64.
#include "gpss.cuh"

namespace gpl1 {

cudaError_t launch_gpss_f64(const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative, cudaStream_t stream,
                           int tile) {
  return GpssHost<GPL1_F64>::launch(tile, a, tmap, grid, cooperative, stream);
}
size_t gpss_smem_bytes_f64(int tile) { return GpssHost<GPL1_F64>::smem(tile); }
const void* gpss_kernel_ptr_f64(int tile) { return GpssHost<GPL1_F64>::kernel(tile); }

}  // namespace gpl1
