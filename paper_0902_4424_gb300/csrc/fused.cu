// Instantiations and launches of the one-read GPSS kernel (fused.cuh).
#include "fused.cuh"
#include "launch.h"

namespace gpl1 {

namespace {

template <int DT, int NCH>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(fz::fused_kernel<DT, NCH>);
}

const void* fused_ptr(int dt, int nch) {
  switch (dt * 8 + nch) {
    case GPL1_F64 * 8 + 2: return kernel_ptr<GPL1_F64, 2>();
    case GPL1_F64 * 8 + 4: return kernel_ptr<GPL1_F64, 4>();
    case GPL1_F32 * 8 + 2: return kernel_ptr<GPL1_F32, 2>();
    case GPL1_F32 * 8 + 4: return kernel_ptr<GPL1_F32, 4>();
    case GPL1_BF16 * 8 + 2: return kernel_ptr<GPL1_BF16, 2>();
    case GPL1_BF16 * 8 + 4: return kernel_ptr<GPL1_BF16, 4>();
    default: return nullptr;
  }
}

size_t smem_of(int dt, int nch) {
  switch (dt * 8 + nch) {
    case GPL1_F64 * 8 + 2: return fz::fused_smem_bytes<GPL1_F64, 2>();
    case GPL1_F64 * 8 + 4: return fz::fused_smem_bytes<GPL1_F64, 4>();
    case GPL1_F32 * 8 + 2: return fz::fused_smem_bytes<GPL1_F32, 2>();
    case GPL1_F32 * 8 + 4: return fz::fused_smem_bytes<GPL1_F32, 4>();
    case GPL1_BF16 * 8 + 2: return fz::fused_smem_bytes<GPL1_BF16, 2>();
    case GPL1_BF16 * 8 + 4: return fz::fused_smem_bytes<GPL1_BF16, 4>();
    default: return 0;
  }
}

cudaError_t prepare(const void* fn, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

}  // namespace

int fused_rows(int dt, int nch) {
  switch (dt * 8 + nch) {
    case GPL1_F64 * 8 + 2: return fz::Cfg<GPL1_F64, 2>::R;
    case GPL1_F64 * 8 + 4: return fz::Cfg<GPL1_F64, 4>::R;
    case GPL1_F32 * 8 + 2: return fz::Cfg<GPL1_F32, 2>::R;
    case GPL1_F32 * 8 + 4: return fz::Cfg<GPL1_F32, 4>::R;
    case GPL1_BF16 * 8 + 2: return fz::Cfg<GPL1_BF16, 2>::R;
    case GPL1_BF16 * 8 + 4: return fz::Cfg<GPL1_BF16, 4>::R;
    default: return 0;
  }
}
int fused_width(int dt, int nch) {
  const int es = dt == GPL1_F64 ? 8 : dt == GPL1_F32 ? 4 : 2;
  return fz::kCons * (16 / es) * nch;
}
size_t fused_smem(int dt, int nch) { return smem_of(dt, nch); }
size_t fused_args_size() { return sizeof(fz::FArgs); }

cudaError_t fused_max_clusters(int dt, int nch, int C, int* out) {
  *out = 0;
  const void* fn = fused_ptr(dt, nch);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = smem_of(dt, nch);
  cudaError_t e = prepare(fn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(fz::kThr);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(out, fn, &cfg);
}

// clusters x C CTAs, all co-resident (the kernel's grid barrier needs it):
// the caller launches at most the clusters the occupancy query reports
// resident together; `cooperative` adds the cooperative attribute.
cudaError_t launch_fused(int dt, int nch, const void* args, const CUtensorMap& tmap, int clusters, int C,
                         bool cooperative, cudaStream_t stream) {
  const void* fn = fused_ptr(dt, nch);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = smem_of(dt, nch);
  cudaError_t e = prepare(fn, smem);
  if (e != cudaSuccess) return e;
  const fz::FArgs& a = *static_cast<const fz::FArgs*>(args);
  void* kargs[] = {const_cast<fz::FArgs*>(&a), const_cast<CUtensorMap*>(&tmap)};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * C);
  cfg.blockDim = dim3(fz::kThr);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeCooperative;
  attr[1].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cooperative ? 2 : 1;
  return cudaLaunchKernelExC(&cfg, fn, kargs);
}

}  // namespace gpl1
