// Host-side entry points of the kernel translation units (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "gpss.cuh"

namespace gpl1 {

// Persistent GPSS kernel for element type `dtype` (GPL1_*): grid CTAs of
// kThreads threads; cooperative launches are used when a group spans CTAs.
cudaError_t launch_gpss(int dtype, const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative,
                        cudaStream_t stream);
size_t gpss_smem_bytes(int dtype);
const void* gpss_kernel_ptr(int dtype);
int gpss_vmax(int dtype);

// Batched projection onto l1 balls, one CTA per segment.
cudaError_t launch_project(int dtype, const void* v, void* out, long long p, long long batch,
                           long long stride, const double* rho, double* tau, cudaStream_t stream);
long long project_max_p(int dtype);

}  // namespace gpl1
