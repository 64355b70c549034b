// Learned warm start for Alg. GP: an unrolled, learned ISTA (the soft-
// thresholded Landweber iteration of Sec. 2),
//
//   x^0 = 0,  z^l = x^l + W_l (y - K x^l),  x^{l+1} = S_{theta_l}(z^l),  l < L,
//
// over a batch of B right-hand sides, batch-major (row b = sample b).  Every
// product is a BF16 tensor-core GEMM (gemm_tc.cu) with FP32 accumulation:
//
//   forward   U  = X^l K^T      (B x n),   C = R W_l^T   (B x p),  R = Y - U
//   backward  dW_l = delta^T R  (p x n),   H = delta W_l (B x n),  HK = H K (B x p)
//
// with delta = g^{l+1} 1[|z^l| > theta_l], dtheta_l = -sum delta sgn(z^l),
// g^l = delta - HK, g^L = (2/B)(x^L - x_target) (loss = mean ||x^L - xt||^2).
// The elementwise steps (residual, soft threshold, its subgradient), the
// conversions to BF16, the transposes the backward products need and the Adam
// update of the FP32 master weights are the kernels below.
#include <cudaTypedefs.h>

#include "launch.h"

namespace gpl1 {

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

__global__ void lista_to_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[i] = bf16_bits(src[i]);
}

// dst (cols x rows, BF16) = src (rows x cols, FP32, row stride lds) transposed.
__global__ void lista_transpose_bf16(const float* __restrict__ src, long long lds, uint16_t* __restrict__ dst, int rows,
                                     int cols) {
  __shared__ float t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    t[r][threadIdx.x] = (i < rows && j < cols) ? src[i * lds + j] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = c0 + r, i = r0 + threadIdx.x;
    if (j < cols && i < rows) dst[static_cast<long long>(j) * rows + i] = bf16_bits(t[threadIdx.x][r]);
  }
}

// R = Y - U (B x n), FP32 and its BF16 copy.
__global__ void lista_residual(const float* __restrict__ Y, long long ldy, const float* __restrict__ U,
                               float* __restrict__ R, uint16_t* __restrict__ Rb, int B, int n) {
  const long long count = static_cast<long long>(B) * n;
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = q / n, i = q % n;
    const float r = Y[b * ldy + i] - U[q];
    R[q] = r;
    Rb[q] = bf16_bits(r);
  }
}

// Z = X + C, X' = S_theta(Z) (B x p), X' also in BF16.
__global__ void lista_activate(const float* __restrict__ X, const float* __restrict__ C, const float* __restrict__ theta,
                               int l, float* __restrict__ Z, float* __restrict__ Xn, uint16_t* __restrict__ Xnb,
                               long long count) {
  const float t = theta[l];
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float z = X[q] + C[q];
    const float a = fabsf(z) - t;
    const float x = a > 0.f ? copysignf(a, z) : 0.f;
    Z[q] = z;
    Xn[q] = x;
    Xnb[q] = bf16_bits(x);
  }
}

// G = (2/B)(X - Xt), loss += sum (X - Xt)^2 / B  (FP64 accumulation of block sums).
__global__ void lista_loss_grad(const float* __restrict__ X, const float* __restrict__ Xt, long long ldt,
                                float* __restrict__ G, int B, int p, double* loss) {
  __shared__ double part[32];
  const long long count = static_cast<long long>(B) * p;
  double s = 0.0;
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long b = q / p, j = q % p;
    const float d = X[q] - Xt[b * ldt + j];
    G[q] = 2.f / static_cast<float>(B) * d;
    s += static_cast<double>(d) * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(loss, t / B);
  }
}

// delta = G 1[|Z| > theta] (FP32 and BF16), dtheta -= sum delta sgn(Z).
__global__ void lista_delta(const float* __restrict__ G, const float* __restrict__ Z, const float* __restrict__ theta,
                            int l, float* __restrict__ D, uint16_t* __restrict__ Db, long long count,
                            double* dtheta) {
  __shared__ double part[32];
  const float t = theta[l];
  double s = 0.0;
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float z = Z[q];
    const float d = fabsf(z) > t ? G[q] : 0.f;
    D[q] = d;
    Db[q] = bf16_bits(d);
    if (d != 0.f) s -= static_cast<double>(d) * (z > 0.f ? 1.0 : -1.0);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) u += part[w];
    atomicAdd(dtheta + l, u);
  }
}

// G = delta - HK (the gradient with respect to x^l).
__global__ void lista_back_x(const float* __restrict__ D, const float* __restrict__ HK, float* __restrict__ G,
                             long long count) {
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x)
    G[q] = D[q] - HK[q];
}

// Adam (bias-corrected) on FP32 masters: w -= lr mhat / (sqrt(vhat) + eps).
__global__ void lista_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, long long count, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  for (long long q = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; q < count;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

__global__ void lista_d2f(const double* __restrict__ a, float* __restrict__ b, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) b[i] = static_cast<float>(a[i]);
}

namespace {
int grid_for(long long count) {
  const long long g = (count + 255) / 256;
  return static_cast<int>(g < 152LL * 16 ? (g < 1 ? 1 : g) : 152LL * 16);
}
}  // namespace

// ------------------------------------------------------------- host driver
// Workspace (bytes at ws, see lista_ws_bytes): BF16 W (L p n), BF16 W^T (L n p),
// K^T (p n), per layer X^l (FP32 + BF16), Z^l, R^l (FP32 + BF16), scratch.

size_t lista_ws_bytes(int L, long long n, long long p, long long B) {
  const size_t pn = static_cast<size_t>(p) * n, Bp = static_cast<size_t>(B) * p, Bn = static_cast<size_t>(B) * n;
  size_t s = 0;
  s += 2 * static_cast<size_t>(L) * pn * 2;            // W, W^T (BF16)
  s += pn * 2;                                         // K^T
  s += static_cast<size_t>(L + 1) * Bp * (4 + 2);      // X^l
  s += static_cast<size_t>(L) * Bp * 4;                // Z^l
  s += static_cast<size_t>(L) * Bn * (4 + 2);          // R^l
  s += Bp * 4 * 4 + Bn * 4 * 2 + Bp * 2 + Bn * 2 + Bp * 2 + Bn * 2 + 4096;   // U, C/HK, G, D (+BF16), H
  s += static_cast<size_t>(L) * 8 + 64 + 64 * 256;     // dtheta, loss, alignment
  return s;
}

struct ListaPtrs {
  uint16_t *Wb, *Wtb, *Kt;
  float* X;      // (L + 1) x B x p
  uint16_t* Xb;  // (L + 1) x B x p
  float* Z;      // L x B x p
  float* R;      // L x B x n
  uint16_t* Rb;  // L x B x n
  float *U, *C, *G, *D, *HK, *H;
  uint16_t *Db, *Hb, *DTb, *RTb;
  double *dtheta, *loss;
};

static ListaPtrs lista_carve(uint8_t* ws, int L, long long n, long long p, long long B) {
  const size_t pn = static_cast<size_t>(p) * n, Bp = static_cast<size_t>(B) * p, Bn = static_cast<size_t>(B) * n;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* q = ws + off;
    off = (off + bytes + 255) & ~static_cast<size_t>(255);
    return q;
  };
  ListaPtrs P;
  P.Wb = reinterpret_cast<uint16_t*>(take(static_cast<size_t>(L) * pn * 2));
  P.Wtb = reinterpret_cast<uint16_t*>(take(static_cast<size_t>(L) * pn * 2));
  P.Kt = reinterpret_cast<uint16_t*>(take(pn * 2));
  P.X = reinterpret_cast<float*>(take(static_cast<size_t>(L + 1) * Bp * 4));
  P.Xb = reinterpret_cast<uint16_t*>(take(static_cast<size_t>(L + 1) * Bp * 2));
  P.Z = reinterpret_cast<float*>(take(static_cast<size_t>(L) * Bp * 4));
  P.R = reinterpret_cast<float*>(take(static_cast<size_t>(L) * Bn * 4));
  P.Rb = reinterpret_cast<uint16_t*>(take(static_cast<size_t>(L) * Bn * 2));
  P.U = reinterpret_cast<float*>(take(Bn * 4));
  P.C = reinterpret_cast<float*>(take(Bp * 4));
  P.G = reinterpret_cast<float*>(take(Bp * 4));
  P.D = reinterpret_cast<float*>(take(Bp * 4));
  P.HK = reinterpret_cast<float*>(take(Bp * 4));
  P.H = reinterpret_cast<float*>(take(Bn * 4));
  P.Db = reinterpret_cast<uint16_t*>(take(Bp * 2));
  P.Hb = reinterpret_cast<uint16_t*>(take(Bn * 2));
  P.DTb = reinterpret_cast<uint16_t*>(take(Bp * 2));
  P.RTb = reinterpret_cast<uint16_t*>(take(Bn * 2));
  P.dtheta = reinterpret_cast<double*>(take(static_cast<size_t>(L) * 8));
  P.loss = reinterpret_cast<double*>(take(64));
  return P;
}

// One forward (and, with Xt, backward) pass.  W: FP32 masters (L x p x n),
// theta: device (L).  With Xt != null the gradients go to dW (FP32, L x p x n),
// dtheta (FP32, L) and the loss to *loss_dev (FP64).  Returns a cudaError_t,
// -1 (tensor map) or -2 (GEMM wait ran out, *gerr set).
int lista_pass(PFN_cuTensorMapEncodeTiled_v12000 enc, uint8_t* ws, int* gerr, const void* K, long long n, long long p,
               long long ldk, int L, const float* W, bool convert_w, const float* theta, const float* Y,
               long long ldy, long long B, const float* Xt, long long ldt, float* Xout, long long ldx, float* dW,
               float* dtheta, double* loss_out, cudaStream_t s) {
  ListaPtrs P = lista_carve(ws, L, n, p, B);
  const long long pn = p * n, Bp = B * p, Bn = B * n;
  const long long tmo = 10LL * 1000 * 1000 * 1000;
  cudaError_t e;
  if (convert_w) {   // BF16 copies of W and W^T, and K^T
    lista_to_bf16<<<grid_for(L * pn), 256, 0, s>>>(W, P.Wb, L * pn);
    for (int l = 0; l < L; ++l)
      lista_transpose_bf16<<<dim3((n + 31) / 32, (p + 31) / 32), dim3(32, 8), 0, s>>>(W + l * pn, n, P.Wtb + l * pn,
                                                                                       static_cast<int>(p),
                                                                                       static_cast<int>(n));
    if ((e = launch_transpose_bf16(K, ldk, P.Kt, static_cast<int>(n), static_cast<int>(p), s)) != cudaSuccess)
      return static_cast<int>(e);
  }
  // x^0 = 0
  if ((e = cudaMemsetAsync(P.X, 0, Bp * 4, s)) != cudaSuccess) return static_cast<int>(e);
  if ((e = cudaMemsetAsync(P.Xb, 0, Bp * 2, s)) != cudaSuccess) return static_cast<int>(e);
  auto gemm = [&](const void* A, long long M, long long Ka, long long lda, const void* Bm, long long N, long long Kd,
                  long long ldb, float* out, long long ldo) {
    const int bn = ((M + 127) / 128) * ((N + 255) / 256) < 152 ? 128 : 256;
    return launch_gemm_bf16(enc, A, static_cast<int>(M), static_cast<int>(Ka), lda, Bm, static_cast<int>(N),
                            static_cast<int>(Kd), ldb, out, ldo, 1.f, gerr, tmo, bn, s, 0);
  };
  int r;
  for (int l = 0; l < L; ++l) {
    float* Xl = P.X + l * Bp;
    uint16_t* Xlb = P.Xb + l * Bp;
    float* Rl = P.R + l * Bn;
    uint16_t* Rlb = P.Rb + l * Bn;
    // U = X^l K^T (B x n); R = Y - U
    if ((r = gemm(Xlb, B, p, p, K, n, p, ldk, P.U, n)) != 0) return r;
    lista_residual<<<grid_for(Bn), 256, 0, s>>>(Y, ldy, P.U, Rl, Rlb, static_cast<int>(B), static_cast<int>(n));
    // C = R W_l^T (B x p); Z = X + C; X^{l+1} = S(Z)
    if ((r = gemm(Rlb, B, n, n, P.Wb + l * pn, p, n, n, P.C, p)) != 0) return r;
    lista_activate<<<grid_for(Bp), 256, 0, s>>>(Xl, P.C, theta, l, P.Z + l * Bp, P.X + (l + 1) * Bp,
                                                P.Xb + (l + 1) * Bp, Bp);
  }
  if (Xout) {
    if ((e = cudaMemcpy2DAsync(Xout, ldx * 4, P.X + L * Bp, p * 4, p * 4, B, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
      return static_cast<int>(e);
  }
  if (!Xt) return static_cast<int>(cudaGetLastError());
  // backward
  if ((e = cudaMemsetAsync(P.dtheta, 0, L * 8, s)) != cudaSuccess) return static_cast<int>(e);
  if ((e = cudaMemsetAsync(P.loss, 0, 8, s)) != cudaSuccess) return static_cast<int>(e);
  lista_loss_grad<<<grid_for(Bp), 256, 0, s>>>(P.X + L * Bp, Xt, ldt, P.G, static_cast<int>(B), static_cast<int>(p),
                                               P.loss);
  for (int l = L - 1; l >= 0; --l) {
    lista_delta<<<grid_for(Bp), 256, 0, s>>>(P.G, P.Z + l * Bp, theta, l, P.D, P.Db, Bp, P.dtheta);
    // dW_l = delta^T R (p x n): K-dimension = the batch
    lista_transpose_bf16<<<dim3((p + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s>>>(P.D, p, P.DTb,
                                                                                   static_cast<int>(B),
                                                                                   static_cast<int>(p));
    lista_transpose_bf16<<<dim3((n + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s>>>(P.R + l * Bn, n, P.RTb,
                                                                                   static_cast<int>(B),
                                                                                   static_cast<int>(n));
    if ((r = gemm(P.DTb, p, B, B, P.RTb, n, B, B, dW + l * pn, n)) != 0) return r;
    if (l == 0) break;   // x^0 is fixed
    // H = delta W_l (B x n) = delta (W_l^T)^T; HK = H K (B x p); g^l = delta - HK
    if ((r = gemm(P.Db, B, p, p, P.Wtb + l * pn, n, p, p, P.H, n)) != 0) return r;
    lista_to_bf16<<<grid_for(Bn), 256, 0, s>>>(P.H, P.Hb, Bn);
    if ((r = gemm(P.Hb, B, n, n, P.Kt, p, n, n, P.HK, p)) != 0) return r;
    lista_back_x<<<grid_for(Bp), 256, 0, s>>>(P.D, P.HK, P.G, Bp);
  }
  lista_d2f<<<1, 64, 0, s>>>(P.dtheta, dtheta, L);
  if (loss_out) {
    if ((e = cudaMemcpyAsync(loss_out, P.loss, 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return static_cast<int>(e);
  }
  return static_cast<int>(cudaGetLastError());
}

// W (p x n, FP32) = scale * K^T for BF16 K (n rows, stride ldk): 32 x 32 tiles
// through shared memory, coalesced on both sides.
__global__ void lista_init_w(const uint16_t* __restrict__ K, long long ldk, int n, int p, float scale,
                             float* __restrict__ W) {
  __shared__ float t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;   // rows of K, columns of K
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = r0 + r, j = c0 + threadIdx.x;
    t[r][threadIdx.x] = (i < n && j < p) ? __uint_as_float(static_cast<uint32_t>(K[i * ldk + j]) << 16) : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = c0 + r, i = r0 + threadIdx.x;
    if (j < p && i < n) W[static_cast<long long>(j) * n + i] = scale * t[threadIdx.x][r];
  }
}

cudaError_t lista_init_weights(const void* K, long long ldk, int n, int p, int L, float scale, float* W,
                               cudaStream_t s) {
  const dim3 grid((p + 31) / 32, (n + 31) / 32), block(32, 8);
  lista_init_w<<<grid, block, 0, s>>>(static_cast<const uint16_t*>(K), ldk, n, p, scale, W);
  cudaError_t e = cudaGetLastError();
  const size_t layer = static_cast<size_t>(p) * n * sizeof(float);
  for (int l = 1; l < L && e == cudaSuccess; ++l)
    e = cudaMemcpyAsync(reinterpret_cast<uint8_t*>(W) + l * layer, W, layer, cudaMemcpyDeviceToDevice, s);
  return e;
}

cudaError_t lista_adam_step(float* w, const float* g, float* m, float* v, long long count, float lr, int t,
                            cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, static_cast<float>(t)), c2 = 1.f - powf(b2, static_cast<float>(t));
  lista_adam<<<grid_for(count), 256, 0, s>>>(w, g, m, v, count, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

}  // namespace gpl1
