// Batched projection onto l1 balls (gpl1_project), plus the dtype dispatch of
// the GPSS launchers.
#include "launch.h"
#include "project.cuh"

namespace gpl1 {

// elements per thread kept in registers: p <= 16800 (float), 7680 (double)
template <typename V> struct ProjVmax { static constexpr int value = 35; };
template <> struct ProjVmax<double> { static constexpr int value = 16; };

// Shared-memory accessor (element e of thread t is index t + e * kConsumers).
template <typename V, int N>
struct SegAcc {
  static constexpr int ne = N;
  const V* vs;
  int neu;
  __device__ V get(int e) const { return vs[e * kConsumers + threadIdx.x]; }
};

template <typename V>
__global__ void __launch_bounds__(kConsumers) project_kernel(const V* __restrict__ v, V* out, long long p,
                                                             long long stride, const double* __restrict__ rho,
                                                             double* tau_out) {
  constexpr int kProjVmax = ProjVmax<V>::value;
  extern __shared__ uint8_t proj_dyn[];
  V* vsm = reinterpret_cast<V*>(proj_dyn);
  ProjSmem& ps = *reinterpret_cast<ProjSmem*>(proj_dyn + sizeof(V) * kProjVmax * kConsumers);
  Scratch& sc = *reinterpret_cast<Scratch*>(proj_dyn + sizeof(V) * kProjVmax * kConsumers + sizeof(ProjSmem));
  const long long seg = blockIdx.x;
  const V* vs = v + seg * stride;
  V* os = out + seg * stride;
  const int neu = static_cast<int>((p + kConsumers - 1) / kConsumers);
  for (int e = 0; e < neu; ++e) {
    const long long j = threadIdx.x + static_cast<long long>(e) * kConsumers;
    vsm[e * kConsumers + threadIdx.x] = j < p ? vs[j] : V(0);
  }
  const double rh = rho[seg];
  if (threadIdx.x == 0) {
    const F2 rp = f2_of(rh);
    sc.tp[0] = rp.hi;
    sc.tp[1] = rp.lo;
  }
  consumer_sync();
  const F2 rho_p{sc.tp[0], sc.tp[1]};
  consumer_sync();
  const SegAcc<V, kProjVmax> acc{vsm, neu};
  const TauResult t = block_l1_tau_fixed_point<V>(acc, rh, rho_p, 0.f, ps, sc);
  const double tau = t.inside ? 0.0 : t.tau;
  for (int e = 0; e < neu; ++e) {
    const long long j = threadIdx.x + static_cast<long long>(e) * kConsumers;
    if (j >= p) break;
    const V r = vsm[e * kConsumers + threadIdx.x];
    if (t.inside) {
      os[j] = r;
    } else if constexpr (sizeof(V) == 8) {
      os[j] = copysign(fmax(fabs(r) - tau, 0.0), r);
    } else {
      const TauPair tp{t.th, t.tl};   // |v| - tau = (|v| - hi) - lo, the first difference exact near tau
      const float a = fabsf(static_cast<float>(r));
      os[j] = tp.below(a) ? 0.f : copysignf((a - tp.hi) - tp.lo, static_cast<float>(r));
    }
  }
  if (tau_out && threadIdx.x == 0)
    tau_out[seg] = t.inside ? 0.0 : (sizeof(V) == 8 ? tau : static_cast<double>(t.th) + static_cast<double>(t.tl));
}

template <typename V>
size_t project_smem() {
  return sizeof(V) * ProjVmax<V>::value * kConsumers + sizeof(ProjSmem) + sizeof(Scratch);
}

long long project_max_p(int dtype) {
  return static_cast<long long>(dtype == GPL1_F64 ? ProjVmax<double>::value : ProjVmax<float>::value) * kConsumers;
}

cudaError_t launch_project(int dtype, const void* v, void* out, long long p, long long batch, long long stride,
                           const double* rho, double* tau, cudaStream_t stream) {
  if (dtype == GPL1_F64) {
    const size_t sm = project_smem<double>();
    cudaError_t e = cudaFuncSetAttribute(project_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    project_kernel<double><<<static_cast<unsigned>(batch), kConsumers, sm, stream>>>(
        static_cast<const double*>(v), static_cast<double*>(out), p, stride, rho, tau);
  } else {
    const size_t sm = project_smem<float>();
    cudaError_t e = cudaFuncSetAttribute(project_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    project_kernel<float><<<static_cast<unsigned>(batch), kConsumers, sm, stream>>>(
        static_cast<const float*>(v), static_cast<float*>(out), p, stride, rho, tau);
  }
  return cudaGetLastError();
}

cudaError_t launch_gpss_f64(const KArgs&, const CUtensorMap&, int, bool, cudaStream_t, int);
cudaError_t launch_gpss_f32(const KArgs&, const CUtensorMap&, int, bool, cudaStream_t, int);
cudaError_t launch_gpss_bf16(const KArgs&, const CUtensorMap&, int, bool, cudaStream_t, int);
size_t gpss_smem_bytes_f64(int);
size_t gpss_smem_bytes_f32(int);
size_t gpss_smem_bytes_bf16(int);
const void* gpss_kernel_ptr_f64(int);
const void* gpss_kernel_ptr_f32(int);
const void* gpss_kernel_ptr_bf16(int);

cudaError_t launch_gpss(int dtype, const KArgs& a, const CUtensorMap& tmap, int grid, bool cooperative,
                        cudaStream_t stream, int tile) {
  switch (dtype) {
    case GPL1_F64: return launch_gpss_f64(a, tmap, grid, cooperative, stream, tile);
    case GPL1_F32: return launch_gpss_f32(a, tmap, grid, cooperative, stream, tile);
    default: return launch_gpss_bf16(a, tmap, grid, cooperative, stream, tile);
  }
}
size_t gpss_smem_bytes(int dtype, int tile) {
  return dtype == GPL1_F64 ? gpss_smem_bytes_f64(tile)
         : dtype == GPL1_F32 ? gpss_smem_bytes_f32(tile)
                             : gpss_smem_bytes_bf16(tile);
}
const void* gpss_kernel_ptr(int dtype, int tile) {
  return dtype == GPL1_F64 ? gpss_kernel_ptr_f64(tile)
         : dtype == GPL1_F32 ? gpss_kernel_ptr_f32(tile)
                             : gpss_kernel_ptr_bf16(tile);
}
int gpss_vmax(int dtype) {
  return dtype == GPL1_F64 ? VMaxOf<GPL1_F64>::value : dtype == GPL1_F32 ? VMaxOf<GPL1_F32>::value
                                                                         : VMaxOf<GPL1_BF16>::value;
}

}  // namespace gpl1
