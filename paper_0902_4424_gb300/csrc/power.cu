// ||K||_2^2 by power iteration on K^T K (the step 1/||K||^2 that makes ISTA and
// FISTA of Sec. 2 admissible for any K, and the scaling of the learned warm
// start's W = K^T / L).  Both products are HBM-bound matrix-vector products:
//   u = K v      one warp per row, lanes stride along the row (coalesced),
//   w = K^T u    one thread per column, a CTA per (256 columns x 256 rows)
//                tile, FP64 partial sums added into w with atomics;
// then one CTA forms ||w|| and v = w / ||w||.  The estimate returned is the
// Rayleigh quotient ||K v||^2 of the last unit vector (never above ||K||^2).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.h"

namespace gpl1 {
namespace {

constexpr int kPwThreads = 256;
constexpr int kPwRows = 256;   // rows per K^T tile

__device__ __forceinline__ double elem(const double* K, long long i) { return K[i]; }
__device__ __forceinline__ double elem(const float* K, long long i) { return static_cast<double>(K[i]); }
__device__ __forceinline__ double elem(const uint16_t* K, long long i) {
  return static_cast<double>(__uint_as_float(static_cast<uint32_t>(K[i]) << 16));
}

// u = K v and uu += ||u||^2 (one warp per row).
template <typename T>
__global__ void __launch_bounds__(kPwThreads) pw_kv(const T* K, long long ldk, int n, int p, const double* v, double* u,
                                                     double* uu) {
  const int lane = threadIdx.x & 31;
  const long long row = static_cast<long long>(blockIdx.x) * (kPwThreads / 32) + (threadIdx.x >> 5);
  if (row >= n) return;
  const T* Kr = K + row * ldk;
  double s = 0.0;
  for (int j = lane; j < p; j += 32) s = fma(elem(Kr, j), v[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    u[row] = s;
    atomicAdd(uu, s * s);
  }
}

// w += K^T u over one tile of 256 columns x 256 rows.
template <typename T>
__global__ void __launch_bounds__(kPwThreads) pw_ktu(const T* K, long long ldk, int n, int p, const double* u,
                                                      double* w) {
  const int col = blockIdx.x * kPwThreads + threadIdx.x;
  const int r0 = blockIdx.y * kPwRows;
  const int r1 = min(n, r0 + kPwRows);
  if (col >= p) return;
  double s = 0.0;
  for (int r = r0; r < r1; ++r) s = fma(elem(K, static_cast<long long>(r) * ldk + col), u[r], s);
  atomicAdd(w + col, s);
}

// v = w / ||w|| (w cleared for the next product); one CTA.
__global__ void __launch_bounds__(kPwThreads) pw_normalize(double* w, double* v, int p) {
  __shared__ double part[kPwThreads / 32];
  double s = 0.0;
  for (int j = threadIdx.x; j < p; j += kPwThreads) s = fma(w[j], w[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < kPwThreads / 32; ++q) t += part[q];
  const double inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  for (int j = threadIdx.x; j < p; j += kPwThreads) {
    v[j] = w[j] * inv;
    w[j] = 0.0;
  }
}

// A start vector with no structure K could be orthogonal to: +-1/sqrt(p)
// with signs from a counter-based hash of the index (SplitMix64's finaliser).
__global__ void pw_start(double* v, double* w, int p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  uint64_t z = static_cast<uint64_t>(j) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[j] = ((z & 1ull) ? 1.0 : -1.0) * rsqrt(static_cast<double>(p));
  w[j] = 0.0;
}

template <typename T>
cudaError_t run_power(const T* K, long long ldk, int n, int p, int iters, double* ws, double* out, cudaStream_t s) {
  double* v = ws;
  double* w = v + p;
  double* u = w + p;
  double* uu = u + n;   // iters + 1 slots
  cudaMemsetAsync(uu, 0, sizeof(double) * (iters + 1), s);
  pw_start<<<(p + 255) / 256, 256, 0, s>>>(v, w, p);
  const dim3 gkv((n + kPwThreads / 32 - 1) / (kPwThreads / 32));
  const dim3 gkt((p + kPwThreads - 1) / kPwThreads, (n + kPwRows - 1) / kPwRows);
  for (int it = 0; it < iters; ++it) {
    pw_kv<T><<<gkv, kPwThreads, 0, s>>>(K, ldk, n, p, v, u, uu + it);
    pw_ktu<T><<<gkt, kPwThreads, 0, s>>>(K, ldk, n, p, u, w);
    pw_normalize<<<1, kPwThreads, 0, s>>>(w, v, p);
  }
  pw_kv<T><<<gkv, kPwThreads, 0, s>>>(K, ldk, n, p, v, u, uu + iters);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(out, uu + iters, sizeof(double), cudaMemcpyDeviceToHost, s);
}

}  // namespace

size_t power_ws_bytes(long long n, long long p, int iters) {
  return sizeof(double) * static_cast<size_t>(2 * p + n + iters + 1);
}

cudaError_t launch_power(int dtype, const void* K, long long ldk, int n, int p, int iters, void* ws, double* out,
                         cudaStream_t s) {
  double* w = static_cast<double*>(ws);
  switch (dtype) {
    case GPL1_F64: return run_power(static_cast<const double*>(K), ldk, n, p, iters, w, out, s);
    case GPL1_F32: return run_power(static_cast<const float*>(K), ldk, n, p, iters, w, out, s);
    case GPL1_BF16: return run_power(static_cast<const uint16_t*>(K), ldk, n, p, iters, w, out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpl1
