// Host-side entry points of the kernel translation units (internal to the library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include "gpss.cuh"

namespace gpl1 {

// Persistent GPSS kernel for element type `dtype` (GPL1_*) and box shape
// `tile` (GPL1_TILE_SMALL / MEDIUM / LARGE, valid for the dtype): grid CTAs
// of kThreads threads; cooperative launches are used when a group spans CTAs.
cudaError_t launch_gpss(int dtype, const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative,
                        cudaStream_t stream, int tile);
size_t gpss_smem_bytes(int dtype, int tile);
const void* gpss_kernel_ptr(int dtype, int tile);
int gpss_vmax(int dtype);

// Batched projection onto l1 balls, one CTA per segment.
cudaError_t launch_project(int dtype, const void* v, void* out, long long p, long long batch,
                           long long stride, const double* rho, double* tau, cudaStream_t stream);
long long project_max_p(int dtype);

// BF16 tensor-core GEMM (gemm_tc.cu): C[m][n] = scale * sum_k A[m][k % Ka] B[n][k],
// stored out[n * ldo + m] (trans_out = 1) or out[m * ldo + n] (trans_out = 0);
// A M x Ka (row stride lda), B N x Kd (row stride ldb), Kd a multiple of 64, Ka of 64.
// bn: 128 or 256 (tile width along N).  Returns a cudaError_t, or -1 if a tensor map
// could not be encoded.
int launch_gemm_bf16(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda,
                     const void* B, int N, int Kd, long long ldb, float* out, long long ldo, float scale, int* err,
                     long long timeout_ns, int bn, cudaStream_t stream, int trans_out = 1);
// The same with a kernel configuration (0..kGemmConfigs-1, see gemm_tc.cu) and a
// split of the contraction into `splits` parts: part z goes to out + z * split_stride.
constexpr int kGemmConfigs = 4;
int gemm_cfg_bn(int cfg);
int launch_gemm_bf16_cfg(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda,
                         const void* B, int N, int Kd, long long ldb, float* out, long long ldo, float scale,
                         int* err, long long timeout_ns, int cfg, int splits, long long split_stride,
                         cudaStream_t stream, int trans_out = 1);

// Autotuner (autotune.cu): the fastest configuration and split (<= max_splits,
// partial z at out + z * split_stride) of one product, timed on its operands;
// sum_gbs is the bandwidth at which the consumer sums the partials (its cost is
// added).  Returns a cudaError_t or -1 (tensor map).
struct GemmChoice {
  int cfg, splits;
  float ms;
};
int autotune_gemm(PFN_cuTensorMapEncodeTiled_v12000 enc, const void* A, int M, int Ka, long long lda, const void* B,
                  int N, int Kd, long long ldb, float* out, long long ldo, float scale, int* err, long long timeout_ns,
                  int max_splits, long long split_stride, double sum_gbs, cudaStream_t stream, GemmChoice* best);

// One-read kernel (fused.cu): columns per CTA (W) and rows per block (R) of a
// configuration, its dynamic shared memory, the number of clusters of C CTAs
// that stay resident together, and the launch (args: a fz::FArgs).
int fused_rows(int dt, int nch);
int fused_width(int dt, int nch);
size_t fused_smem(int dt, int nch);
cudaError_t fused_max_clusters(int dt, int nch, int C, int* out);
cudaError_t launch_fused(int dt, int nch, const void* args, const CUtensorMap& tmap, int clusters, int C,
                         bool cooperative, cudaStream_t stream);

}  // namespace gpl1

namespace gpl1 {
// Shared-K multi-right-hand-side form (shared_k.cu).
size_t mr_state_bytes();
cudaError_t launch_mr_init(const float* Y, long long ldy, float* X, long long ldx, uint16_t* Rs, int n, int p,
                           const double* rho, const double* fstar, void* states, const SolveParams& prm, int nrhs,
                           cudaStream_t s);
cudaError_t launch_mr_phase_p(const float* G, const float* Gprev, const float* X, long long ldx, float* D,
                              uint16_t* DXs, int p, int nrhs, int k, void* states, const SolveParams& prm,
                              int* restart_cnt, int* restart_list, cudaStream_t s);
cudaError_t launch_mr_phase_l(float* KD, int splits, long long split_stride, const void* xpart, const float* Y,
                              long long ldy, float* X, long long ldx, const float* D, uint16_t* Rs, int n, int p,
                              int nrhs, int k, void* states, const SolveParams& prm, gpl1_result* res,
                              int* done_count, cudaStream_t s);
size_t mr_exact_part_bytes(int n, int p, int nrhs);
// restart_cnt: 2 ints (zero at the start of a solve); restart_list: 2 x nrhs ints.
cudaError_t launch_mr_exact_kx(const void* Kt, const float* X, long long ldx, void* xpart, int n, int p, int nrhs,
                               const void* states, const int* restart_cnt, const int* restart_list, int k, int num_sms,
                               cudaStream_t s);
cudaError_t launch_transpose_bf16(const void* K, long long ldk, void* Kt, int n, int p, cudaStream_t s);
cudaError_t launch_mr_setup_x0(float* X, long long ldx, uint16_t* DXs, int p, int nrhs, const double* rho,
                               cudaStream_t s);
cudaError_t launch_mr_setup_r(const float* KDX, const float* Y, long long ldy, uint16_t* Rs, int n, int nrhs,
                              const double* rho, const double* fstar, void* states, const SolveParams& prm,
                              cudaStream_t s);
}  // namespace gpl1

namespace gpl1 {
// Learned warm start (lista.cu).
size_t lista_ws_bytes(int L, long long n, long long p, long long B);
int lista_pass(PFN_cuTensorMapEncodeTiled_v12000 enc, uint8_t* ws, int* gerr, const void* K, long long n, long long p,
               long long ldk, int L, const float* W, bool convert_w, const float* theta, const float* Y,
               long long ldy, long long B, const float* Xt, long long ldt, float* Xout, long long ldx, float* dW,
               float* dtheta, double* loss_out, cudaStream_t s);
cudaError_t lista_adam_step(float* w, const float* g, float* m, float* v, long long count, float lr, int t,
                            cudaStream_t s);
// W_l = scale K^T for l < L (W: L x p x n FP32; K BF16 n x ldk).
cudaError_t lista_init_weights(const void* K, long long ldk, int n, int p, int L, float scale, float* W,
                               cudaStream_t s);
}  // namespace gpl1

namespace gpl1 {
// ||K||_2^2 by power iteration (power.cu): `iters` products with K^T K from a
// fixed start vector; *out (host) receives the Rayleigh quotient of the last
// unit vector.  ws: power_ws_bytes(n, p, iters) bytes of device memory.
size_t power_ws_bytes(long long n, long long p, int iters);
cudaError_t launch_power(int dtype, const void* K, long long ldk, int n, int p, int iters, void* ws, double* out,
                         cudaStream_t s);
}  // namespace gpl1
