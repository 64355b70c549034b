// Instantiation of the GPSS kernel for K stored as GPL1_BF16.
#include "gpss.cuh"

namespace gpl1 {

cudaError_t launch_gpss_bf16(const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative,
                              cudaStream_t stream) {
  const size_t smem = sizeof(SolverSmem<GPL1_BF16>) + 128;
  cudaError_t e = cudaFuncSetAttribute(gpss_kernel<GPL1_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<KArgs*>(&a), const_cast<CUtensorMap*>(&tmap)};
  if (cooperative)
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(gpss_kernel<GPL1_BF16>), dim3(grid),
                                       dim3(kThreads), args, smem, stream);
  return cudaLaunchKernel(reinterpret_cast<const void*>(gpss_kernel<GPL1_BF16>), dim3(grid), dim3(kThreads),
                          args, smem, stream);
}
size_t gpss_smem_bytes_bf16() { return sizeof(SolverSmem<GPL1_BF16>) + 128; }
const void* gpss_kernel_ptr_bf16() { return reinterpret_cast<const void*>(gpss_kernel<GPL1_BF16>); }

}  // namespace gpl1
