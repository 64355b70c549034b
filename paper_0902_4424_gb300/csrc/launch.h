// Host-side entry points of the kernel translation units (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

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

// BF16 tensor-core GEMM (gemm_tc.cu): out[n * ldo + m] = scale * sum_k A[m][k % Ka] B[n][k],
// A M x Ka (row stride lda), B N x Kd (row stride ldb), Kd a multiple of 64, Ka of 64.
// bn: 128 or 256 (tile width along N).  Returns a cudaError_t, or -1 if a tensor map
// could not be encoded.
int launch_gemm_bf16(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda,
                     const void* B, int N, int Kd, long long ldb, float* out, long long ldo, float scale, int* err,
                     long long timeout_ns, int bn, cudaStream_t stream);

}  // namespace gpl1
