// C ABI of the gpl1 library: context, argument checks, device workspace,
// TMA descriptors, launches.  See include/gpl1.h for the contract.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "fused.cuh"
#include "launch.h"

using namespace gpl1;

struct gpl1_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  char err[512] = {0};
  void* ws = nullptr;               // device workspace
  size_t ws_bytes = 0;
  gpl1_result* host_res = nullptr;  // pinned staging for results
  size_t host_res_count = 0;
  std::vector<uint8_t> host_stage;  // staging of descriptors (kept alive across async copies)
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};   // around the solver launch
  // autotuned tensor-core products: (M, N, Kd, Ka, max_splits) -> configuration and split
  std::map<std::vector<long long>, gpl1::GemmChoice> gemm_tuned;
  // one-read kernel: resident clusters per (dtype, chunks per thread, cluster size)
  std::map<std::vector<int>, int> fused_resident;
  void* aux = nullptr;              // second device buffer (the warm-start call's padded rows)
  size_t aux_bytes = 0;
  // single-solve autotuner: (dtype, n, p, engine class) -> engine and tuned ms
  std::map<std::vector<long long>, std::pair<int, float>> solve_tuned;
  // batched autotuner: (dtype, count, sum of n p, largest n p, hash of the
  // shapes) -> tile and the tuning time of each tile (-1: not a candidate)
  struct TileTune {
    int tile;
    float ms[3];
  };
  std::map<std::vector<long long>, TileTune> tile_tuned;
};

namespace {

gpl1_status fail(gpl1_ctx* c, gpl1_status st, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
  }
  return st;
}

gpl1_status cuda_fail(gpl1_ctx* c, cudaError_t e, const char* what) {
  return fail(c, GPL1_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GPL1_CUDA(call, what)                         \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_size(int dt) { return dt == GPL1_F64 ? 8 : dt == GPL1_F32 ? 4 : 2; }
int acc_size(int dt) { return dt == GPL1_F64 ? 8 : 4; }
// rows of a TMA box of the two-pass kernel (the tile's shape)
int rows_per_box(int dt, int tile = GPL1_TILE_MEDIUM) { return tile_rows(dt, tile); }

gpl1_status ensure_ws(gpl1_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return GPL1_OK;
  if (ctx->ws) {
    GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  const size_t want = align_up(bytes + bytes / 4, 1 << 20);
  GPL1_CUDA(cudaMalloc(&ctx->ws, want), "cudaMalloc(workspace)");
  ctx->ws_bytes = want;
  return GPL1_OK;
}

// A second device buffer of the context (scratch that must not share the workspace).
gpl1_status ensure_aux(gpl1_ctx* ctx, size_t bytes) {
  if (ctx->aux_bytes >= bytes) return GPL1_OK;
  if (ctx->aux) {
    GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    cudaFree(ctx->aux);
    ctx->aux = nullptr;
    ctx->aux_bytes = 0;
  }
  GPL1_CUDA(cudaMalloc(&ctx->aux, bytes), "cudaMalloc(aux)");
  ctx->aux_bytes = bytes;
  return GPL1_OK;
}

gpl1_status ensure_host_res(gpl1_ctx* ctx, size_t count) {
  if (count <= ctx->host_res_count) return GPL1_OK;
  if (ctx->host_res) cudaFreeHost(ctx->host_res);
  ctx->host_res = nullptr;
  GPL1_CUDA(cudaMallocHost(&ctx->host_res, count * sizeof(gpl1_result)), "cudaMallocHost");
  ctx->host_res_count = count;
  return GPL1_OK;
}

// methods: whether the caller runs the comparison methods of Sec. 2 (single
// solves on the one-read kernel); every other entry point runs Alg. GP + SS only.
gpl1_status check_params(gpl1_ctx* ctx, const gpl1_params* p, bool methods = false) {
  if (!p) return fail(ctx, GPL1_ERR_INVALID_ARG, "params is NULL");
  if (p->method < GPL1_METHOD_GPSS || p->method > GPL1_METHOD_PSD)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "method must be GPL1_METHOD_GPSS, _ISTA, _FISTA or _PSD");
  if (p->method != GPL1_METHOD_GPSS) {
    if (!methods)
      return fail(ctx, GPL1_ERR_UNSUPPORTED, "ISTA, FISTA and PSD run in gpl1_solve and gpl1_solve_async only");
    if (p->engine == GPL1_ENGINE_TWO_PASS)
      return fail(ctx, GPL1_ERR_UNSUPPORTED, "ISTA, FISTA and PSD run on the one-read engine only");
    const bool eq1 = p->method == GPL1_METHOD_ISTA || p->method == GPL1_METHOD_FISTA;
    if (eq1 && (!(p->lambda_pen > 0) || !std::isfinite(p->lambda_pen)))
      return fail(ctx, GPL1_ERR_INVALID_ARG, "ISTA and FISTA need a finite lambda_pen > 0");
    if (eq1 && (!(p->step > 0) || !std::isfinite(p->step)))
      return fail(ctx, GPL1_ERR_INVALID_ARG, "ISTA and FISTA need a finite step > 0");
    if (eq1 && (p->stop_rule & GPL1_STOP_ON_FW))
      return fail(ctx, GPL1_ERR_INVALID_ARG, "GPL1_STOP_ON_FW is a certificate of eq. 2, not of ISTA/FISTA's eq. 1");
  }
  if (!(p->beta > 0 && p->beta < 1) || !(p->theta > 0 && p->theta < 1))
    return fail(ctx, GPL1_ERR_INVALID_ARG, "beta and theta must lie in (0,1)");
  if (p->M < 1 || p->M > kMaxM) return fail(ctx, GPL1_ERR_INVALID_ARG, "M must lie in [1,%d]", kMaxM);
  if (p->M_alpha < 0 || p->M_alpha > kMaxMalpha)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "M_alpha must lie in [0,%d]", kMaxMalpha);
  if (!(p->alpha_min > 0 && p->alpha_min < p->alpha_max) || !std::isfinite(p->alpha_max))
    return fail(ctx, GPL1_ERR_INVALID_ARG, "need 0 < alpha_min < alpha_max < inf");
  if (!(p->tau1 > 0 && p->tau1 < 1)) return fail(ctx, GPL1_ERR_INVALID_ARG, "tau1 must lie in (0,1)");
  if (!(p->tol >= 0) || !std::isfinite(p->tol)) return fail(ctx, GPL1_ERR_INVALID_ARG, "tol must be finite, >= 0");
  if (p->max_iter < 1 || p->max_backtracks < 0) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad max_iter/max_backtracks");
  if (p->timeout_ns <= 0) return fail(ctx, GPL1_ERR_INVALID_ARG, "timeout_ns must be > 0");
  if (p->alpha0_rule != 0 && p->alpha0_rule != 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "alpha0_rule is 0 or 1");
  if (p->engine < GPL1_ENGINE_AUTO || p->engine > GPL1_ENGINE_ONE_READ_NCH4)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "engine must be one of GPL1_ENGINE_*");
  if (p->tile < GPL1_TILE_AUTO || p->tile > GPL1_TILE_LARGE)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "tile must be one of GPL1_TILE_*");
  return GPL1_OK;
}

gpl1_status check_problem(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, int idx, bool two_pass = true) {
  if (!pr) return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d is NULL", idx);
  if (!pr->K || !pr->y || !pr->x) return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: NULL K, y or x", idx);
  if (pr->n < 1 || pr->p < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: n and p must be >= 1", idx);
  if (pr->ldk < pr->p) return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: ldk < p", idx);
  if (!(pr->rho > 0) || !std::isfinite(pr->rho))
    return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: rho must be finite and > 0", idx);
  const int es = elem_size(dt);
  if (reinterpret_cast<uintptr_t>(pr->K) % 16 != 0)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: K must be 16-byte aligned", idx);
  if ((pr->ldk * es) % 16 != 0)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: ldk * sizeof(element) must be a multiple of 16", idx);
  const int vs = dt == GPL1_F64 ? 8 : 4;
  if (reinterpret_cast<uintptr_t>(pr->y) % vs || reinterpret_cast<uintptr_t>(pr->x) % vs)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "problem %d: x and y must be aligned to their element size", idx);
  if (two_pass && pr->p > static_cast<long long>(gpss_vmax(dt)) * kConsumers)
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "problem %d: p = %lld exceeds %d for this dtype", idx, pr->p,
                gpss_vmax(dt) * kConsumers);
  if (pr->n > (1LL << 30) || pr->ldk > (1LL << 31))
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "problem %d: n or ldk too large", idx);
  return GPL1_OK;
}

gpl1_status encode_tmap(gpl1_ctx* ctx, CUtensorMap* map, const gpl1_problem* pr, int dt, int box_rows = 0) {
  if (!ctx->encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    GPL1_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q),
              "cudaGetDriverEntryPointByVersion");
    if (q != cudaDriverEntryPointSuccess || !fn)
      return fail(ctx, GPL1_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const CUtensorMapDataType t = dt == GPL1_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                : dt == GPL1_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(pr->p), static_cast<cuuint64_t>(pr->n)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pr->ldk) * elem_size(dt)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(kBoxCols),
                             static_cast<cuuint32_t>(box_rows > 0 ? box_rows : rows_per_box(dt))};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode(map, t, 2, const_cast<void*>(pr->K), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, GPL1_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return GPL1_OK;
}

SolveParams to_kernel_params(const gpl1_params* p) {
  SolveParams s;
  s.beta = p->beta;
  s.theta = p->theta;
  s.alpha_min = p->alpha_min;
  s.alpha_max = p->alpha_max;
  s.tau1 = p->tau1;
  s.tol = p->tol;
  s.M = p->M;
  s.M_alpha = p->M_alpha;
  s.stop_rule = p->stop_rule;
  s.max_iter = p->max_iter;
  s.max_backtracks = p->max_backtracks;
  s.alpha0_rule = p->alpha0_rule;
  s.timeout_ns = p->timeout_ns;
  s.debug = p->debug;
  s.method = p->method;
  s.method_pad = 0;
  s.lam_pen = p->lambda_pen;
  s.step = p->step;
  return s;
}

struct Sizes {
  int NB, TC;
  long long pp, nn, units;
};
Sizes sizes_of(const gpl1_problem* pr, int dt, int tile = GPL1_TILE_MEDIUM) {
  Sizes s;
  const int RB = rows_per_box(dt, tile);
  s.NB = static_cast<int>((pr->n + RB - 1) / RB);
  s.TC = static_cast<int>((pr->p + kBoxCols - 1) / kBoxCols);
  s.pp = static_cast<long long>(s.TC) * kBoxCols;
  s.nn = static_cast<long long>(s.NB) * RB;
  s.units = static_cast<long long>(s.NB) * s.TC;
  return s;
}

}  // namespace

extern "C" {

void gpl1_params_default(gpl1_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->beta = 1e-4;
  p->theta = 0.5;
  p->M = 1;
  p->alpha_min = 1e-10;
  p->alpha_max = 1e10;
  p->tau1 = 0.5;
  p->M_alpha = 2;
  p->tol = 1e-6;
  p->f_star = -1.0;
  p->stop_rule = GPL1_STOP_ON_REL_GAP | GPL1_STOP_ON_FW;
  p->max_iter = 100000;
  p->max_backtracks = 100;
  p->alpha0_rule = 0;
  p->x0_is_zero = 0;
  p->timeout_ns = 10LL * 1000 * 1000 * 1000;
  p->method = GPL1_METHOD_GPSS;
  p->lambda_pen = 0.0;
  p->step = 1.0;
}

gpl1_status gpl1_create(gpl1_ctx** out, int device, void* stream) {
  if (!out) return GPL1_ERR_INVALID_ARG;
  *out = nullptr;
  gpl1_ctx* ctx = new (std::nothrow) gpl1_ctx();
  if (!ctx) return GPL1_ERR_CUDA;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete ctx;
    return GPL1_ERR_CUDA;
  }
  *out = ctx;
  return GPL1_OK;
}

void gpl1_destroy(gpl1_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
  }
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->host_res) cudaFreeHost(ctx->host_res);
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

gpl1_status gpl1_set_stream(gpl1_ctx* ctx, void* stream) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return GPL1_OK;
}

const char* gpl1_last_error(const gpl1_ctx* ctx) { return ctx ? ctx->err : "null context"; }

gpl1_status gpl1_project(gpl1_ctx* ctx, const void* v, void* out, gpl1_dtype dtype, long long p, long long batch,
                         long long stride, const double* rho, int rho_on_device, double* tau_out) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!v || !out || !rho) return fail(ctx, GPL1_ERR_INVALID_ARG, "NULL pointer");
  if (dtype != GPL1_F64 && dtype != GPL1_F32) return fail(ctx, GPL1_ERR_INVALID_ARG, "dtype must be F64 or F32");
  if (p < 1 || batch < 1 || stride < p) return fail(ctx, GPL1_ERR_INVALID_ARG, "need p >= 1, batch >= 1, stride >= p");
  if (batch > 2147483647LL) return fail(ctx, GPL1_ERR_UNSUPPORTED, "batch too large");
  if (p > project_max_p(dtype))
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "p = %lld exceeds %lld", p, project_max_p(dtype));
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  const double* rho_dev = rho;
  if (!rho_on_device) {
    for (long long b = 0; b < batch; ++b)
      if (!(rho[b] > 0) || !std::isfinite(rho[b])) return fail(ctx, GPL1_ERR_INVALID_ARG, "rho[%lld] must be > 0", b);
    gpl1_status st = ensure_ws(ctx, static_cast<size_t>(batch) * sizeof(double));
    if (st) return st;
    GPL1_CUDA(cudaMemcpyAsync(ctx->ws, rho, static_cast<size_t>(batch) * sizeof(double), cudaMemcpyHostToDevice,
                              ctx->stream),
              "cudaMemcpyAsync(rho)");
    rho_dev = static_cast<const double*>(ctx->ws);
  }
  GPL1_CUDA(launch_project(dtype, v, out, p, batch, stride, rho_dev, tau_out, ctx->stream), "project kernel");
  if (!rho_on_device) GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return GPL1_OK;
}

namespace {

// Launch `count` instances.  group > 1: one instance over `group` CTAs
// (cooperative); group == 1: persistent CTAs pulling instances from a queue.
// Workspace layout of one launch of `count` instances:
// [counters 256][descs][results][tmaps][gbuf/kbuf/pbuf per instance].
struct BatchLayout {
  std::vector<int> order;   // queue order: largest n p first (the longest instances start first)
  size_t off_desc = 256, off_res = 0, off_tmap = 0, off_bufs = 0, total = 0;
  std::vector<size_t> off_g, off_k, off_p;
  bool batched = false;
  int tile = GPL1_TILE_MEDIUM;   // box shape of the launch
};

BatchLayout batch_layout(const gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, int tile) {
  BatchLayout L;
  L.tile = tile;
  L.order.resize(count);
  std::iota(L.order.begin(), L.order.end(), 0);
  if (count > 1)
    std::stable_sort(L.order.begin(), L.order.end(), [&](int a, int b) {
      return probs[a].n * probs[a].p > probs[b].n * probs[b].p;
    });
  const int as = acc_size(dt);
  L.batched = count > 1;
  L.off_res = align_up(L.off_desc + sizeof(InstDesc) * count, 256);
  L.off_tmap = align_up(L.off_res + sizeof(gpl1_result) * count, 256);
  L.off_bufs = align_up(L.off_tmap + (L.batched ? sizeof(CUtensorMap) * count : 0), 256);
  L.off_g.resize(count);
  L.off_k.resize(count);
  L.off_p.resize(count);
  const int max_group = L.batched ? 1 : ctx->num_sms * 4;
  size_t cur = L.off_bufs;
  for (int q = 0; q < count; ++q) {
    const Sizes sz = sizes_of(&probs[q], dt, tile);
    L.off_g[q] = cur;
    cur = align_up(cur + 3 * sz.pp * as, 256);
    L.off_k[q] = cur;
    cur = align_up(cur + 2 * kbuf_stride(sz.nn, as), 256);
    L.off_p[q] = cur;   // pass-B partials: 4 doubles per CTA of the group
    cur = align_up(cur + 32 * static_cast<size_t>(max_group), 256);
  }
  L.total = cur;
  return L;
}

// Host image of [descs][results][tmaps] (off_bufs - off_desc bytes at `host`)
// for a workspace at `ws`; the single solve's tensor map goes to *tmap0.
gpl1_status stage_batch(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                        const BatchLayout& L, uint8_t* ws, uint8_t* host, CUtensorMap* tmap0) {
  std::memset(host, 0, L.off_bufs - L.off_desc);
  InstDesc* hd = reinterpret_cast<InstDesc*>(host);
  CUtensorMap* ht = reinterpret_cast<CUtensorMap*>(host + (L.off_tmap - L.off_desc));
  gpl1_result* hr = reinterpret_cast<gpl1_result*>(host + (L.off_res - L.off_desc));
  for (int q = 0; q < count; ++q) {   // overwritten by the kernel; stays if an instance never ran
    hr[q].status = GPL1_ERR_TIMEOUT;
    hr[q].stop = GPL1_STOP_ERROR;
  }
  std::memset(tmap0, 0, sizeof *tmap0);
  for (int q = 0; q < count; ++q) {
    const int src = L.order[q];
    const gpl1_problem& pr = probs[src];
    InstDesc& d = hd[q];
    d.y = pr.y;
    d.x = pr.x;
    d.rho = pr.rho;
    d.f_star = pr.f_star >= 0 ? pr.f_star : prm->f_star;
    d.n = static_cast<int>(pr.n);
    d.p = static_cast<int>(pr.p);
    d.x0_zero = prm->x0_is_zero ? 1 : 0;
    d.pad = 0;
    d.gbuf = ws + L.off_g[src];
    d.kbuf = ws + L.off_k[src];
    d.res = reinterpret_cast<gpl1_result*>(ws + L.off_res) + src;
    d.trace = pr.trace;
    d.trace_cap = pr.trace ? pr.trace_cap : 0;
    d.pbuf = ws + L.off_p[src];
    gpl1_status st;
    if (L.batched) {
      st = encode_tmap(ctx, &ht[q], &pr, dt, rows_per_box(dt, L.tile));
      d.tmap = ws + L.off_tmap + sizeof(CUtensorMap) * q;
    } else {
      st = encode_tmap(ctx, tmap0, &pr, dt, rows_per_box(dt, L.tile));
      d.tmap = nullptr;
    }
    if (st) return st;
  }
  return GPL1_OK;
}

// Everything one solve puts on `stream`: zero x (x0 = 0), the counters and the
// accumulation buffers, upload the host image, launch, read the results back
// into host_res.  No host synchronisation, so a stream capture can record it.
gpl1_status enqueue_batch(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                          const BatchLayout& L, uint8_t* ws, const uint8_t* host, const CUtensorMap& tmap0,
                          cudaStream_t stream, gpl1_result* host_res, cudaEvent_t ev0, cudaEvent_t ev1,
                          bool capture = false, cudaMemcpyKind res_kind = cudaMemcpyDeviceToHost) {
  // under stream capture the events become event-record nodes of the graph
  const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (prm->x0_is_zero)   // x0 = 0: the iterate buffer must start at zero
    for (int q = 0; q < count; ++q)
      GPL1_CUDA(cudaMemsetAsync(probs[q].x, 0, static_cast<size_t>(probs[q].p) * (dt == GPL1_F64 ? 8 : 4), stream),
                "cudaMemsetAsync(x)");
  GPL1_CUDA(cudaMemsetAsync(ws, 0, 256, stream), "cudaMemsetAsync");
  GPL1_CUDA(cudaMemsetAsync(ws + L.off_bufs, 0, L.total - L.off_bufs, stream), "cudaMemsetAsync");
  GPL1_CUDA(cudaMemcpyAsync(ws + L.off_desc, host, L.off_bufs - L.off_desc, cudaMemcpyHostToDevice, stream),
            "cudaMemcpyAsync(desc)");
  KArgs ka;
  ka.desc = reinterpret_cast<const InstDesc*>(ws + L.off_desc);
  ka.count = count;
  ka.queue = reinterpret_cast<unsigned*>(ws + 0);
  ka.bar = reinterpret_cast<unsigned*>(ws + 64);
  ka.err = reinterpret_cast<int*>(ws + 128);
  ka.prm = to_kernel_params(prm);
  int occ = 0;
  GPL1_CUDA(cudaFuncSetAttribute(gpss_kernel_ptr(dt, L.tile), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(gpss_smem_bytes(dt, L.tile))),
            "cudaFuncSetAttribute");
  GPL1_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gpss_kernel_ptr(dt, L.tile), kThreads,
                                                          gpss_smem_bytes(dt, L.tile)),
            "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) return fail(ctx, GPL1_ERR_CUDA, "solver kernel does not fit on an SM");
  GPL1_CUDA(cudaEventRecordWithFlags(ev0, stream, evf), "cudaEventRecord");
  if (!L.batched) {
    const Sizes sz = sizes_of(&probs[0], dt, L.tile);
    const long long G = std::min<long long>(static_cast<long long>(ctx->num_sms) * occ, sz.units);
    ka.group = static_cast<int>(G);
    GPL1_CUDA(launch_gpss(dt, ka, tmap0, ka.group, G > 1, stream, L.tile), "solver launch");
  } else {
    ka.group = 1;
    const int grid = std::min(ctx->num_sms * occ, count);
    GPL1_CUDA(launch_gpss(dt, ka, tmap0, grid, false, stream, L.tile), "solver launch");
  }
  GPL1_CUDA(cudaEventRecordWithFlags(ev1, stream, evf), "cudaEventRecord");
  GPL1_CUDA(cudaMemcpyAsync(host_res, ws + L.off_res, sizeof(gpl1_result) * count, res_kind, stream),
            "cudaMemcpyAsync(result)");
  return GPL1_OK;
}

// After the stream has synchronised: results out, kernel time, worst status.
gpl1_status finish_batch(gpl1_ctx* ctx, int count, const gpl1_result* host_res, gpl1_result* res, cudaEvent_t ev0,
                         cudaEvent_t ev1) {
  std::memcpy(res, host_res, sizeof(gpl1_result) * count);
  float ms = 0.f;
  GPL1_CUDA(cudaEventElapsedTime(&ms, ev0, ev1), "cudaEventElapsedTime");
  for (int q = 0; q < count; ++q) res[q].kernel_ms = ms;
  int worst = GPL1_OK;
  for (int q = 0; q < count; ++q)
    if (res[q].status != GPL1_OK && res[q].status != GPL1_ERR_NOT_CONVERGED) worst = res[q].status;
  if (worst != GPL1_OK) return fail(ctx, static_cast<gpl1_status>(worst), "an instance failed (status %d)", worst);
  return GPL1_OK;
}

// Enqueue only: the results go to res_dev (device memory), nothing waits.
gpl1_status run_async(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                      gpl1_result* res_dev, int tile) {
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  const BatchLayout L = batch_layout(ctx, probs, count, dt, tile);
  gpl1_status st = ensure_ws(ctx, L.total);
  if (st) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  ctx->host_stage.assign(L.off_bufs - L.off_desc, 0);   // pageable: copied before cudaMemcpyAsync returns
  CUtensorMap tmap0;
  st = stage_batch(ctx, probs, count, dt, prm, L, ws, ctx->host_stage.data(), &tmap0);
  if (st) return st;
  if (!ctx->ev[0]) {
    GPL1_CUDA(cudaEventCreate(&ctx->ev[0]), "cudaEventCreate");
    GPL1_CUDA(cudaEventCreate(&ctx->ev[1]), "cudaEventCreate");
  }
  return enqueue_batch(ctx, probs, count, dt, prm, L, ws, ctx->host_stage.data(), tmap0, ctx->stream, res_dev,
                       ctx->ev[0], ctx->ev[1], false, cudaMemcpyDeviceToDevice);
}

gpl1_status run(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                gpl1_result* res, int tile) {
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  const BatchLayout L = batch_layout(ctx, probs, count, dt, tile);
  gpl1_status st = ensure_ws(ctx, L.total);
  if (st) return st;
  st = ensure_host_res(ctx, count);
  if (st) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  ctx->host_stage.assign(L.off_bufs - L.off_desc, 0);
  CUtensorMap tmap0;
  st = stage_batch(ctx, probs, count, dt, prm, L, ws, ctx->host_stage.data(), &tmap0);
  if (st) return st;
  if (!ctx->ev[0]) {
    GPL1_CUDA(cudaEventCreate(&ctx->ev[0]), "cudaEventCreate");
    GPL1_CUDA(cudaEventCreate(&ctx->ev[1]), "cudaEventCreate");
  }
  st = enqueue_batch(ctx, probs, count, dt, prm, L, ws, ctx->host_stage.data(), tmap0, ctx->stream, ctx->host_res,
                     ctx->ev[0], ctx->ev[1]);
  if (st) return st;
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "solver");
  return finish_batch(ctx, count, ctx->host_res, res, ctx->ev[0], ctx->ev[1]);
}

// The batched autotuner (gpl1_params.tile AUTO): every admissible box shape
// solves the batch for kTuneIters iterations from x0 = 0 into scratch copies
// of x, twice; the faster second run wins, per batch (dtype and the list of
// instance shapes) and context.
constexpr int kTileTuneIters = 4;

std::vector<long long> tile_key(const gpl1_problem* probs, int count, int dt) {
  long long sum = 0, mx = 0;
  unsigned long long h = 1469598103934665603ull;   // FNV-1a over the (n, p) list
  for (int q = 0; q < count; ++q) {
    const long long np = probs[q].n * probs[q].p;
    sum += np;
    mx = std::max(mx, np);
    for (long long v : {probs[q].n, probs[q].p})
      for (int b = 0; b < 8; ++b) {
        h ^= static_cast<unsigned long long>(v >> (8 * b)) & 0xffull;
        h *= 1099511628211ull;
      }
  }
  return {dt, count, sum, mx, static_cast<long long>(h & 0x7fffffffffffffffull)};
}

gpl1_status tune_tile(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                      const std::vector<long long>& key, int* best) {
  const size_t vs = dt == GPL1_F64 ? 8 : 4;
  std::vector<size_t> off(count);
  size_t tot = 0;
  for (int q = 0; q < count; ++q) {
    off[q] = tot;
    tot = align_up(tot + static_cast<size_t>(probs[q].p) * vs, 256);
  }
  gpl1_status st = ensure_aux(ctx, tot + 256);
  if (st) return st;
  std::vector<gpl1_problem> tp(probs, probs + count);
  for (int q = 0; q < count; ++q) {
    tp[q].x = static_cast<uint8_t*>(ctx->aux) + off[q];
    tp[q].trace = nullptr;
    tp[q].trace_cap = 0;
  }
  gpl1_params tq = *prm;
  tq.stop_rule = 0;
  tq.max_iter = kTileTuneIters;
  tq.x0_is_zero = 1;
  std::vector<gpl1_result> r(count);
  gpl1_ctx::TileTune rec{GPL1_TILE_MEDIUM, {-1.f, -1.f, -1.f}};
  float best_ms = 0.f;
  *best = -1;
  for (int tl = GPL1_TILE_SMALL; tl <= GPL1_TILE_LARGE; ++tl) {
    if (!tile_valid(dt, tl)) continue;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      st = run(ctx, tp.data(), count, dt, &tq, r.data(), tl);
      if (st != GPL1_OK && st != GPL1_ERR_NOT_CONVERGED && st != GPL1_ERR_LINESEARCH) return st;
      ms = static_cast<float>(r[0].kernel_ms);
    }
    rec.ms[tl - GPL1_TILE_SMALL] = ms;
    if (*best < 0 || ms < best_ms) {
      *best = tl;
      best_ms = ms;
    }
  }
  rec.tile = *best;
  ctx->tile_tuned[key] = rec;
  return GPL1_OK;
}

// The box shape of a two-pass launch: the caller's, else MEDIUM for a single
// instance, else the batched autotuner's choice for this batch.
gpl1_status pick_tile(gpl1_ctx* ctx, const gpl1_problem* probs, int count, int dt, const gpl1_params* prm,
                      int* tile) {
  if (prm->tile != GPL1_TILE_AUTO) {
    if (!tile_valid(dt, prm->tile)) return fail(ctx, GPL1_ERR_UNSUPPORTED, "tile %d does not apply to this dtype", prm->tile);
    *tile = prm->tile;
    return GPL1_OK;
  }
  *tile = GPL1_TILE_MEDIUM;
  if (count < 2) return GPL1_OK;
  const std::vector<long long> key = tile_key(probs, count, dt);
  auto it = ctx->tile_tuned.find(key);
  if (it != ctx->tile_tuned.end()) {
    *tile = it->second.tile;
    return GPL1_OK;
  }
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  return tune_tile(ctx, probs, count, dt, prm, key, tile);
}

// ---------------------------------------------------------------------------
// The one-read engine (fused.cuh): shape choice, workspace, launch.

struct OneRead {
  int nch = 1, C = 1, NC = 0, R = 1, W = 0;
  long long pp = 0;
  size_t off_res = 256, off_U = 512, off_parts = 0, total = 0;
};

// Chunks per thread and cluster size for p columns (the smallest cluster that
// covers p with two chunks per thread, else with four; portable sizes first),
// and the number of clusters that stay resident together.
gpl1_status one_read_choose(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, OneRead* o, int want_nch = 0) {
  const long long p = pr->p;
  int nch = 0, C = 0;
  if (want_nch) {   // a given number of chunks per thread (the autotuner's candidates)
    const long long w = fused_width(dt, want_nch);
    const long long c = (p + w - 1) / w;
    if (c > fz::kCMax)
      return fail(ctx, GPL1_ERR_UNSUPPORTED, "p = %lld needs clusters of more than %d CTAs", p, fz::kCMax);
    nch = want_nch;
    C = static_cast<int>(c);
  }
  for (int cand : {2, 4}) {
    if (nch) break;
    const long long w = fused_width(dt, cand);
    const long long c = (p + w - 1) / w;
    if (c <= 8) {
      nch = cand;
      C = static_cast<int>(c);
      break;
    }
  }
  if (!nch) {
    const long long w = fused_width(dt, 4);
    const long long c = (p + w - 1) / w;
    if (c > fz::kCMax)
      return fail(ctx, GPL1_ERR_UNSUPPORTED, "p = %lld exceeds the one-read kernel's %lld columns", p,
                  static_cast<long long>(fz::kCMax) * w);
    nch = 4;
    C = static_cast<int>(c);
  }
  const std::vector<int> key = {dt, nch, C};
  auto it = ctx->fused_resident.find(key);
  int resident = 0;
  if (it == ctx->fused_resident.end()) {
    cudaError_t e = fused_max_clusters(dt, nch, C, &resident);
    if (e != cudaSuccess) {
      cudaGetLastError();
      resident = 0;
    }
    ctx->fused_resident[key] = resident;
  } else {
    resident = it->second;
  }
  if (resident < 1)
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "clusters of %d CTAs of the one-read kernel do not fit this GPU", C);
  o->nch = nch;
  o->C = C;
  o->R = fused_rows(dt, nch);
  o->W = fused_width(dt, nch);
  const long long nbt = (pr->n + o->R - 1) / o->R;
  o->NC = static_cast<int>(std::min<long long>(resident, nbt));
  o->pp = static_cast<long long>(C) * o->W;
  const size_t as = static_cast<size_t>(acc_size(dt));
  o->off_parts = align_up(o->off_U + 3 * 2 * static_cast<size_t>(o->pp) * as, 256);
  o->total = align_up(o->off_parts + 2 * static_cast<size_t>(o->NC) * C * fz::kPartW * 4, 256);
  return GPL1_OK;
}

// Everything one single solve puts on `stream` with the one-read kernel:
// clear the workspace, launch, copy the result to `res_dst` (kind).
gpl1_status one_read_enqueue(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, const gpl1_params* prm,
                             const OneRead& o, uint8_t* ws, cudaStream_t stream, void* res_dst, cudaMemcpyKind kind,
                             cudaEvent_t ev0, cudaEvent_t ev1) {
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof tmap);
  gpl1_status st = encode_tmap(ctx, &tmap, pr, dt, o.R);
  if (st) return st;
  fz::FArgs fa;
  std::memset(&fa, 0, sizeof fa);
  fa.y = pr->y;
  fa.x = pr->x;
  fa.rho = pr->rho;
  fa.f_star = pr->f_star >= 0 ? pr->f_star : prm->f_star;
  fa.n = static_cast<int>(pr->n);
  fa.p = static_cast<int>(pr->p);
  fa.x0_zero = prm->x0_is_zero ? 1 : 0;
  fa.C = o.C;
  fa.NC = o.NC;
  fa.U = ws + o.off_U;
  fa.pp = o.pp;
  fa.parts = reinterpret_cast<unsigned*>(ws + o.off_parts);
  fa.bar = reinterpret_cast<unsigned*>(ws + 64);
  fa.err = reinterpret_cast<int*>(ws + 128);
  fa.res = reinterpret_cast<gpl1_result*>(ws + o.off_res);
  fa.trace = pr->trace;
  fa.trace_cap = pr->trace ? pr->trace_cap : 0;
  fa.prm = to_kernel_params(prm);
  GPL1_CUDA(cudaMemsetAsync(ws, 0, o.total, stream), "cudaMemsetAsync");
  gpl1_result init;
  std::memset(&init, 0, sizeof init);
  init.status = GPL1_ERR_TIMEOUT;   // overwritten by the kernel
  init.stop = GPL1_STOP_ERROR;
  GPL1_CUDA(cudaMemcpyAsync(ws + o.off_res, &init, sizeof init, cudaMemcpyHostToDevice, stream),
            "cudaMemcpyAsync(result)");
  if (ev0) GPL1_CUDA(cudaEventRecord(ev0, stream), "cudaEventRecord");
  // a cluster launch of at most the clusters the occupancy query reports
  // resident together (the kernel's grid barrier waits for all of them, with
  // a bound)
  const cudaError_t e = launch_fused(dt, o.nch, &fa, tmap, o.NC, o.C, false, stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "one-read solver launch");
  if (ev1) GPL1_CUDA(cudaEventRecord(ev1, stream), "cudaEventRecord");
  GPL1_CUDA(cudaMemcpyAsync(res_dst, ws + o.off_res, sizeof(gpl1_result), kind, stream), "cudaMemcpyAsync(result)");
  return GPL1_OK;
}

gpl1_status run_one_read(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, const gpl1_params* prm, const OneRead& o,
                         gpl1_result* res, gpl1_result* res_dev);

constexpr int kTuneIters = 4;   // Alg. GP iterations of a timed candidate solve

// The autotuner of the single solve: each admissible engine (the one-read
// kernel with one or two column chunks per thread, which changes the cluster
// size and the rows per block, and, for GPL1_ENGINE_AUTO, the two-pass
// kernel) solves the instance for kTuneIters iterations from x0 = 0 into a
// scratch x, twice; the faster second run wins, per (dtype, n, p, engine
// class) and context.
gpl1_status tune_engine(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, const gpl1_params* prm,
                        const std::vector<int>& cands, int* best) {
  const size_t vs = dt == GPL1_F64 ? 8 : 4;
  gpl1_status st = ensure_aux(ctx, static_cast<size_t>(pr->p) * vs + 256);
  if (st) return st;
  gpl1_problem tp = *pr;
  tp.x = ctx->aux;
  tp.trace = nullptr;
  tp.trace_cap = 0;
  gpl1_params tq = *prm;
  tq.stop_rule = 0;
  tq.max_iter = kTuneIters;
  tq.x0_is_zero = 1;
  float best_ms = 0.f;
  *best = -1;
  for (int eng : cands) {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      gpl1_result r;
      if (eng == GPL1_ENGINE_TWO_PASS) {
        st = run(ctx, &tp, 1, dt, &tq, &r, GPL1_TILE_MEDIUM);
      } else {
        OneRead o;
        if ((st = one_read_choose(ctx, &tp, dt, &o, eng == GPL1_ENGINE_ONE_READ_NCH4 ? 4 : 2))) return st;
        st = run_one_read(ctx, &tp, dt, &tq, o, &r, nullptr);
      }
      if (st != GPL1_OK && st != GPL1_ERR_NOT_CONVERGED && st != GPL1_ERR_LINESEARCH) return st;
      ms = static_cast<float>(r.kernel_ms);
    }
    if (*best < 0 || ms < best_ms) {
      *best = eng;
      best_ms = ms;
    }
  }
  const std::vector<long long> key = {dt, pr->n, pr->p, prm->engine == GPL1_ENGINE_AUTO ? 0 : 1};
  ctx->solve_tuned[key] = {*best, best_ms};
  return GPL1_OK;
}

// Which engine runs this single solve (GPL1_OK with *use_one_read set and *o
// filled for the one-read kernel, or an error when the engine asked for cannot
// take the instance).
gpl1_status pick_engine(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, const gpl1_params* prm, OneRead* o,
                        bool* use_one_read) {
  *use_one_read = false;
  if (prm->engine == GPL1_ENGINE_TWO_PASS) return check_problem(ctx, pr, dt, 0, true);
  gpl1_status st = check_problem(ctx, pr, dt, 0, false);
  if (st) return st;
  if (pr->n > (1LL << 30) || pr->p > (1LL << 30)) return fail(ctx, GPL1_ERR_UNSUPPORTED, "n or p too large");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (prm->engine == GPL1_ENGINE_ONE_READ_NCH2 || prm->engine == GPL1_ENGINE_ONE_READ_NCH4) {
    if ((st = one_read_choose(ctx, pr, dt, o, prm->engine == GPL1_ENGINE_ONE_READ_NCH4 ? 4 : 2))) return st;
    *use_one_read = true;
    return GPL1_OK;
  }
  // the admissible candidates
  std::vector<int> cands;
  gpl1_status last = GPL1_OK;
  for (int nch : {2, 4}) {
    OneRead t;
    const gpl1_status s1 = one_read_choose(ctx, pr, dt, &t, nch);
    if (s1 == GPL1_OK) cands.push_back(nch == 2 ? GPL1_ENGINE_ONE_READ_NCH2 : GPL1_ENGINE_ONE_READ_NCH4);
    else last = s1;
  }
  const bool two_ok = prm->engine == GPL1_ENGINE_AUTO && prm->method == GPL1_METHOD_GPSS &&
                      pr->p <= static_cast<long long>(gpss_vmax(dt)) * kConsumers;
  if (two_ok) cands.push_back(GPL1_ENGINE_TWO_PASS);
  if (cands.empty()) return last ? last : check_problem(ctx, pr, dt, 0, true);
  int eng = cands[0];
  if (cands.size() > 1) {
    const std::vector<long long> key = {dt, pr->n, pr->p, prm->engine == GPL1_ENGINE_AUTO ? 0 : 1};
    auto it = ctx->solve_tuned.find(key);
    if (it != ctx->solve_tuned.end()) {
      eng = it->second.first;
    } else if ((st = tune_engine(ctx, pr, dt, prm, cands, &eng))) {
      return st;
    }
  }
  if (eng == GPL1_ENGINE_TWO_PASS) return check_problem(ctx, pr, dt, 0, true);
  if ((st = one_read_choose(ctx, pr, dt, o, eng == GPL1_ENGINE_ONE_READ_NCH4 ? 4 : 2))) return st;
  *use_one_read = true;
  return GPL1_OK;
}

gpl1_status run_one_read(gpl1_ctx* ctx, const gpl1_problem* pr, int dt, const gpl1_params* prm, const OneRead& o,
                         gpl1_result* res, gpl1_result* res_dev) {
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  gpl1_status st = ensure_ws(ctx, o.total);
  if (st) return st;
  if (!ctx->ev[0]) {
    GPL1_CUDA(cudaEventCreate(&ctx->ev[0]), "cudaEventCreate");
    GPL1_CUDA(cudaEventCreate(&ctx->ev[1]), "cudaEventCreate");
  }
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  if (res_dev)
    return one_read_enqueue(ctx, pr, dt, prm, o, ws, ctx->stream, res_dev, cudaMemcpyDeviceToDevice, nullptr,
                            nullptr);
  st = ensure_host_res(ctx, 1);
  if (st) return st;
  st = one_read_enqueue(ctx, pr, dt, prm, o, ws, ctx->stream, ctx->host_res, cudaMemcpyDeviceToHost, ctx->ev[0],
                        ctx->ev[1]);
  if (st) return st;
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "solver");
  return finish_batch(ctx, 1, ctx->host_res, res, ctx->ev[0], ctx->ev[1]);
}

}  // namespace

gpl1_status gpl1_solve(gpl1_ctx* ctx, const gpl1_problem* prob, gpl1_dtype dt, const gpl1_params* prm,
                       gpl1_result* res) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!res) return fail(ctx, GPL1_ERR_INVALID_ARG, "result is NULL");
  gpl1_status st = check_params(ctx, prm, true);
  if (st) return st;
  OneRead o;
  bool one = false;
  st = pick_engine(ctx, prob, dt, prm, &o, &one);
  if (st) return st;
  if (one) return run_one_read(ctx, prob, dt, prm, o, res, nullptr);
  int tile = GPL1_TILE_MEDIUM;
  if ((st = pick_tile(ctx, prob, 1, dt, prm, &tile))) return st;
  return run(ctx, prob, 1, dt, prm, res, tile);
}

gpl1_status gpl1_solve_async(gpl1_ctx* ctx, const gpl1_problem* prob, gpl1_dtype dt, const gpl1_params* prm,
                             gpl1_result* res_dev) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!res_dev) return fail(ctx, GPL1_ERR_INVALID_ARG, "result is NULL");
  gpl1_status st = check_params(ctx, prm, true);
  if (st) return st;
  OneRead o;
  bool one = false;
  st = pick_engine(ctx, prob, dt, prm, &o, &one);
  if (st) return st;
  if (one) return run_one_read(ctx, prob, dt, prm, o, nullptr, res_dev);
  int tile = GPL1_TILE_MEDIUM;
  if ((st = pick_tile(ctx, prob, 1, dt, prm, &tile))) return st;
  return run_async(ctx, prob, 1, dt, prm, res_dev, tile);
}

gpl1_status gpl1_solve_batched_async(gpl1_ctx* ctx, const gpl1_problem* probs, int count, gpl1_dtype dt,
                                     const gpl1_params* prm, gpl1_result* res_dev) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!probs || !res_dev || count < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "need probs, res and count >= 1");
  gpl1_status st = check_params(ctx, prm);
  if (st) return st;
  for (int q = 0; q < count; ++q) {
    st = check_problem(ctx, &probs[q], dt, q);
    if (st) return st;
  }
  int tile = GPL1_TILE_MEDIUM;
  if ((st = pick_tile(ctx, probs, count, dt, prm, &tile))) return st;
  return run_async(ctx, probs, count, dt, prm, res_dev, tile);
}

gpl1_status gpl1_solve_batched(gpl1_ctx* ctx, const gpl1_problem* probs, int count, gpl1_dtype dt,
                               const gpl1_params* prm, gpl1_result* res) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!probs || !res || count < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "need probs, res and count >= 1");
  gpl1_status st = check_params(ctx, prm);
  if (st) return st;
  for (int q = 0; q < count; ++q) {
    st = check_problem(ctx, &probs[q], dt, q);
    if (st) return st;
  }
  int tile = GPL1_TILE_MEDIUM;
  if ((st = pick_tile(ctx, probs, count, dt, prm, &tile))) return st;
  return run(ctx, probs, count, dt, prm, res, tile);
}

int gpl1_batched_tuned(const gpl1_ctx* ctx, int index, long long* key, int* tile, float* ms) {
  if (!ctx) return -1;
  const int n = static_cast<int>(ctx->tile_tuned.size());
  if (index >= 0 && index < n) {
    auto it = ctx->tile_tuned.begin();
    std::advance(it, index);
    if (key)
      for (int i = 0; i < 4; ++i) key[i] = it->first[i];
    if (tile) *tile = it->second.tile;
    if (ms)
      for (int i = 0; i < 3; ++i) ms[i] = it->second.ms[i];
  }
  return n;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched plans: the enqueue of gpl1_solve_batched captured once into a CUDA
// graph and replayed (declaration and contract in gpl1.h).

struct gpl1_plan {
  gpl1_ctx* ctx = nullptr;
  int device = 0;
  int count = 0, dt = 0;
  gpl1_params prm{};
  std::vector<gpl1_problem> probs;
  BatchLayout layout;
  void* ws = nullptr;                 // the plan's own workspace
  uint8_t* host_img = nullptr;        // pinned: descriptors, initial results, tensor maps
  gpl1_result* host_res = nullptr;    // pinned: results read back by the graph
  CUtensorMap tmap0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" void gpl1_plan_destroy(gpl1_plan* pl) {
  if (!pl) return;
  cudaSetDevice(pl->device);
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  for (cudaEvent_t e : pl->ev)
    if (e) cudaEventDestroy(e);
  if (pl->ws) cudaFree(pl->ws);
  if (pl->host_img) cudaFreeHost(pl->host_img);
  if (pl->host_res) cudaFreeHost(pl->host_res);
  delete pl;
}

extern "C" gpl1_status gpl1_plan_create(gpl1_ctx* ctx, const gpl1_problem* probs, int count, gpl1_dtype dt,
                                        const gpl1_params* prm, gpl1_plan** out) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!out) return fail(ctx, GPL1_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!probs || count < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "need probs and count >= 1");
  gpl1_status st = check_params(ctx, prm);
  if (st) return st;
  for (int q = 0; q < count; ++q) {
    st = check_problem(ctx, &probs[q], dt, q);
    if (st) return st;
  }
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  int tile = GPL1_TILE_MEDIUM;
  st = pick_tile(ctx, probs, count, dt, prm, &tile);
  if (st) return st;
  gpl1_plan* pl = new gpl1_plan;
  pl->ctx = ctx;
  pl->device = ctx->device;
  pl->count = count;
  pl->dt = dt;
  pl->prm = *prm;
  pl->probs.assign(probs, probs + count);
  pl->layout = batch_layout(ctx, probs, count, dt, tile);
  const BatchLayout& L = pl->layout;
  cudaStream_t cap = nullptr;
  auto bail = [&](gpl1_status code) {
    if (cap) cudaStreamDestroy(cap);
    gpl1_plan_destroy(pl);
    return code;
  };
  cudaError_t e = cudaMalloc(&pl->ws, L.total);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&pl->host_img), L.off_bufs - L.off_desc);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&pl->host_res), sizeof(gpl1_result) * count);
  if (e == cudaSuccess) e = cudaEventCreate(&pl->ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&pl->ev[1]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "plan allocation"));
  st = stage_batch(ctx, probs, count, dt, prm, L, static_cast<uint8_t*>(pl->ws), pl->host_img, &pl->tmap0);
  if (st) return bail(st);
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaStreamBeginCapture"));
  st = enqueue_batch(ctx, pl->probs.data(), count, dt, &pl->prm, L, static_cast<uint8_t*>(pl->ws), pl->host_img,
                     pl->tmap0, cap, pl->host_res, pl->ev[0], pl->ev[1], true);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cap, &g);
  pl->graph = g;
  if (st) return bail(st);
  if (ee != cudaSuccess) return bail(cuda_fail(ctx, ee, "cudaStreamEndCapture"));
  e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGraphInstantiate"));
  cudaStreamDestroy(cap);
  *out = pl;
  return GPL1_OK;
}

extern "C" gpl1_status gpl1_plan_run(gpl1_plan* pl, gpl1_result* res) {
  if (!pl) return GPL1_ERR_INVALID_ARG;
  gpl1_ctx* ctx = pl->ctx;
  if (!res) return fail(ctx, GPL1_ERR_INVALID_ARG, "res is NULL");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  GPL1_CUDA(cudaGraphLaunch(pl->exec, ctx->stream), "cudaGraphLaunch");
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "plan");
  return finish_batch(ctx, pl->count, pl->host_res, res, pl->ev[0], pl->ev[1]);
}

// ---------------------------------------------------------------------------
// gpl1_solve_noalloc: gpl1_solve with its workspace in a fixed static device
// array instead of context memory (declaration and contract in gpl1.h).

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GPL1_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Per device: the scratch address and the CUDA context it was taken in.  A
// cudaDeviceReset (by the caller or a framework) destroys the primary context
// with the module; the next context loads the module again and the array may
// sit elsewhere, so the address is looked up again whenever the current
// context differs from the one recorded.
struct NoallocSlot {
  void* addr = nullptr;
  CUcontext ctx = nullptr;
};
NoallocSlot g_noalloc_slot[kNoallocMaxDevices];
using PFN_ctxGetCurrent = CUresult (*)(CUcontext*);
PFN_ctxGetCurrent g_ctx_get_current = nullptr;

gpl1_status noalloc_fail(char* err, int err_len, gpl1_status st, const char* msg) {
  if (err && err_len > 0) std::snprintf(err, static_cast<size_t>(err_len), "%s", msg);
  return st;
}

}  // namespace

extern "C" gpl1_status gpl1_solve_noalloc(const gpl1_problem* prob, gpl1_dtype dt, const gpl1_params* prm,
                                          gpl1_result* res, void* cuda_stream, char* err, int err_len) {
  if (err && err_len > 0) err[0] = 0;
  gpl1_ctx c;   // on the stack: argument checks and their messages only
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16)
    return noalloc_fail(err, err_len, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!res) return noalloc_fail(err, err_len, GPL1_ERR_INVALID_ARG, "result is NULL");
  gpl1_status st = check_params(&c, prm);
  if (st == GPL1_OK) st = check_problem(&c, prob, dt, 0);
  if (st != GPL1_OK) return noalloc_fail(err, err_len, st, c.err);

  // workspace layout of a single solve: [counters][desc][result][gbuf][kbuf][pbuf]
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int num_sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoallocMaxDevices) return noalloc_fail(err, err_len, GPL1_ERR_UNSUPPORTED, "device index too large");
  const Sizes s = sizes_of(prob, dt);
  const int as = acc_size(dt);
  const size_t off_desc = 256;
  const size_t off_res = align_up(off_desc + sizeof(InstDesc), 256);
  const size_t off_g = align_up(off_res + sizeof(gpl1_result), 256);
  const size_t off_k = align_up(off_g + 3 * s.pp * as, 256);
  const size_t off_p = align_up(off_k + 2 * kbuf_stride(s.nn, as), 256);
  const size_t total = align_up(off_p + 32 * static_cast<size_t>(num_sms) * 4, 256);
  if (total > GPL1_NOALLOC_SCRATCH_BYTES) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch; the static scratch holds %u (GPL1_NOALLOC_SCRATCH_BYTES)",
                  total, static_cast<unsigned>(GPL1_NOALLOC_SCRATCH_BYTES));
    return noalloc_fail(err, err_len, GPL1_ERR_UNSUPPORTED, msg);
  }

  // per-device setup: the scratch address (the first lookup also loads the
  // module), taken again after the device's context has been replaced
  uint8_t* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_ctx_get_current) {
      cudaDriverEntryPointQueryResult q;
      void* fn = nullptr;
      e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return noalloc_fail(err, err_len, GPL1_ERR_CUDA, "cuCtxGetCurrent is not available");
      g_ctx_get_current = reinterpret_cast<PFN_ctxGetCurrent>(fn);
    }
    // make the device's primary context current (since CUDA 12 cudaSetDevice
    // initialises it; the device is already the current one)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, cudaGetErrorString(e));
    CUcontext cur = nullptr;
    if (g_ctx_get_current(&cur) != CUDA_SUCCESS || !cur)
      return noalloc_fail(err, err_len, GPL1_ERR_CUDA, "no current CUDA context");
    NoallocSlot& slot = g_noalloc_slot[dev];
    if (!slot.addr || slot.ctx != cur) {
      void* a = nullptr;
      e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, cudaGetErrorString(e));
      if (!a) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, "cudaGetSymbolAddress returned a null scratch address");
      slot.addr = a;
      slot.ctx = cur;
    }
    ws = static_cast<uint8_t*>(slot.addr);
  }

  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof tmap);
  st = encode_tmap(&c, &tmap, prob, dt);
  if (st != GPL1_OK) return noalloc_fail(err, err_len, st, c.err);
  struct {
    InstDesc d;
    gpl1_result r;
  } host;   // staged by value (pageable copies complete before cudaMemcpyAsync returns)
  std::memset(&host, 0, sizeof host);
  InstDesc& d = host.d;
  d.y = prob->y;
  d.x = prob->x;
  d.rho = prob->rho;
  d.f_star = prob->f_star >= 0 ? prob->f_star : prm->f_star;
  d.n = static_cast<int>(prob->n);
  d.p = static_cast<int>(prob->p);
  d.x0_zero = prm->x0_is_zero ? 1 : 0;
  d.gbuf = ws + off_g;
  d.kbuf = ws + off_k;
  d.res = reinterpret_cast<gpl1_result*>(ws + off_res);
  d.tmap = nullptr;
  d.trace = prob->trace;
  d.trace_cap = prob->trace ? prob->trace_cap : 0;
  d.pbuf = ws + off_p;
  host.r.status = GPL1_ERR_TIMEOUT;   // overwritten by the kernel
  host.r.stop = GPL1_STOP_ERROR;

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const void* fn = gpss_kernel_ptr(dt, GPL1_TILE_MEDIUM);
  const size_t smem = gpss_smem_bytes(dt, GPL1_TILE_MEDIUM);
  int occ = 0;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
  if (e == cudaSuccess && occ < 1) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, "solver kernel does not fit on an SM");
  // zero what the kernel accumulates into: counters, gbuf, kbuf, pbuf; then x0 = 0 if asked
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, off_desc, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + off_g, 0, total - off_g, stream);
  if (e == cudaSuccess && prm->x0_is_zero)
    e = cudaMemsetAsync(prob->x, 0, static_cast<size_t>(prob->p) * (dt == GPL1_F64 ? 8 : 4), stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + off_desc, &host.d, sizeof(InstDesc), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + off_res, &host.r, sizeof(gpl1_result), cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, cudaGetErrorString(e));

  KArgs ka;
  ka.desc = reinterpret_cast<const InstDesc*>(ws + off_desc);
  ka.count = 1;
  ka.queue = reinterpret_cast<unsigned*>(ws + 0);
  ka.bar = reinterpret_cast<unsigned*>(ws + 64);
  ka.err = reinterpret_cast<int*>(ws + 128);
  ka.prm = to_kernel_params(prm);
  const long long G = std::min<long long>(static_cast<long long>(num_sms) * occ, s.units);
  ka.group = static_cast<int>(G);
  e = launch_gpss(dt, ka, tmap, ka.group, G > 1, stream, GPL1_TILE_MEDIUM);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host.r, ws + off_res, sizeof(gpl1_result), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return noalloc_fail(err, err_len, GPL1_ERR_CUDA, cudaGetErrorString(e));
  *res = host.r;
  res->kernel_ms = 0.0;   // no events: timing is left to the caller
  if (res->status != GPL1_OK && res->status != GPL1_ERR_NOT_CONVERGED) {
    char msg[64];
    std::snprintf(msg, sizeof msg, "the solve failed (status %d)", res->status);
    return noalloc_fail(err, err_len, static_cast<gpl1_status>(res->status), msg);
  }
  return GPL1_OK;
}

// ---------------------------------------------------------------------------
// gpl1_gemm_bf16: the tensor-core product of the shared-K form (gemm_tc.cu).

namespace {

gpl1_status gemm_impl(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda, const void* B,
                      long long N, long long Kd, long long ldb, float* out, long long ldo, float scale, int cfg,
                      int splits, long long split_stride) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!A || !B || !out) return fail(ctx, GPL1_ERR_INVALID_ARG, "NULL pointer");
  if (M < 1 || N < 1 || Ka < 64 || Kd < 64 || Ka % 64 || Kd % 64)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "need M, N >= 1 and Ka, Kd positive multiples of 64");
  if (lda < Ka || ldb < Kd || ldo < M) return fail(ctx, GPL1_ERR_INVALID_ARG, "need lda >= Ka, ldb >= Kd, ldo >= M");
  if ((lda * 2) % 16 || (ldb * 2) % 16 || reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(B) % 16)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "A, B and their row strides must be 16-byte aligned");
  if (M > (1LL << 30) || N > (1LL << 30) || Kd > (1LL << 30))
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "dimension too large");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!ctx->encode) {   // the driver's tensor-map encoder (as for the solver)
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    GPL1_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q),
              "cudaGetDriverEntryPointByVersion");
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(ctx, GPL1_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  gpl1_status st = ensure_ws(ctx, 256);
  if (st) return st;
  int* err = static_cast<int*>(ctx->ws);
  GPL1_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream), "cudaMemsetAsync");
  if (cfg < 0 || cfg >= kGemmConfigs) return fail(ctx, GPL1_ERR_INVALID_ARG, "config must lie in [0, %d)", kGemmConfigs);
  if (splits < 1 || splits > Kd / 64) return fail(ctx, GPL1_ERR_INVALID_ARG, "splits must lie in [1, Kd / 64]");
  if (splits > 1 && split_stride < ldo * N)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "split_stride must hold a whole N x ldo output");
  const int e = launch_gemm_bf16_cfg(ctx->encode, A, static_cast<int>(M), static_cast<int>(Ka), lda, B,
                                     static_cast<int>(N), static_cast<int>(Kd), ldb, out, ldo, scale, err,
                                     10LL * 1000 * 1000 * 1000, cfg, splits, split_stride, ctx->stream);
  if (e == -1) return fail(ctx, GPL1_ERR_CUDA, "tensor map encoding failed");
  if (e != 0) return cuda_fail(ctx, static_cast<cudaError_t>(e), "gemm launch");
  int herr = 0;
  GPL1_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "gemm");
  if (herr) return fail(ctx, static_cast<gpl1_status>(herr), "a bounded wait in the GEMM ran out");
  return GPL1_OK;
}

}  // namespace

extern "C" gpl1_status gpl1_gemm_bf16(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda,
                                      const void* B, long long N, long long Kd, long long ldb, float* out,
                                      long long ldo, float scale) {
  return gemm_impl(ctx, A, M, Ka, lda, B, N, Kd, ldb, out, ldo, scale, N > 128 ? 1 : 0, 1, 0);
}

extern "C" gpl1_status gpl1_gemm_bf16_ex(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda,
                                         const void* B, long long N, long long Kd, long long ldb, float* out,
                                         long long ldo, float scale, int config, int splits,
                                         long long split_stride) {
  return gemm_impl(ctx, A, M, Ka, lda, B, N, Kd, ldb, out, ldo, scale, config, splits, split_stride);
}

extern "C" gpl1_status gpl1_gemm_tuned_set(gpl1_ctx* ctx, const long long* shape, int config, int splits) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!shape) return fail(ctx, GPL1_ERR_INVALID_ARG, "shape is NULL");
  if (config < 0 || config >= kGemmConfigs) return fail(ctx, GPL1_ERR_INVALID_ARG, "config must lie in [0, %d)", kGemmConfigs);
  if (shape[2] < 64 || shape[2] % 64 || shape[4] < 1 || splits < 1 || splits > shape[4] || splits > shape[2] / 64)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "need Kd a multiple of 64 and 1 <= splits <= min(max_splits, Kd / 64)");
  ctx->gemm_tuned[std::vector<long long>(shape, shape + 5)] = GemmChoice{config, splits, 0.f};
  return GPL1_OK;
}

extern "C" int gpl1_solve_tuned(const gpl1_ctx* ctx, int index, long long* shape, int* engine, float* ms) {
  if (!ctx) return -1;
  const int count = static_cast<int>(ctx->solve_tuned.size());
  if (index < 0 || index >= count) return count;
  auto it = ctx->solve_tuned.begin();
  std::advance(it, index);
  if (shape)
    for (int q = 0; q < 4; ++q) shape[q] = it->first[q];
  if (engine) *engine = it->second.first;
  if (ms) *ms = it->second.second;
  return count;
}

extern "C" int gpl1_gemm_tuned(const gpl1_ctx* ctx, int index, long long* shape, int* config, int* splits,
                               float* ms) {
  if (!ctx) return -1;
  const int count = static_cast<int>(ctx->gemm_tuned.size());
  if (index < 0 || index >= count) return count;
  auto it = ctx->gemm_tuned.begin();
  std::advance(it, index);
  if (shape)
    for (int q = 0; q < 5; ++q) shape[q] = it->first[q];
  if (config) *config = it->second.cfg;
  if (splits) *splits = it->second.splits;
  if (ms) *ms = it->second.ms;
  return count;
}

// ---------------------------------------------------------------------------
// gpl1_solve_shared_k: nrhs instances sharing one BF16 K (shared_k.cu).

namespace {

constexpr int kMaxSplits = 8;   // split-K partial slices of the second product

// The configuration of one product of the shared-K form: from the context's
// cache, else tuned on the given operands (autotune.cu) and cached.
gpl1_status tuned_gemm(gpl1_ctx* ctx, const void* A, long long M, long long Ka, long long lda, const void* B,
                       long long Nc, long long Kd, long long ldb, float* out, long long ldo, float scale, int* err,
                       long long tmo, int max_splits, long long split_stride, GemmChoice* c) {
  const std::vector<long long> key{M, Nc, Kd, Ka, max_splits};
  const auto it = ctx->gemm_tuned.find(key);
  if (it != ctx->gemm_tuned.end()) {
    *c = it->second;
    return GPL1_OK;
  }
  const int e = autotune_gemm(ctx->encode, A, static_cast<int>(M), static_cast<int>(Ka), lda, B, static_cast<int>(Nc),
                              static_cast<int>(Kd), ldb, out, ldo, scale, err, tmo, max_splits, split_stride, 6000.0,
                              ctx->stream, c);
  if (e == -1) return fail(ctx, GPL1_ERR_CUDA, "tensor map");
  if (e) return cuda_fail(ctx, static_cast<cudaError_t>(e), "autotune");
  int ge = 0;
  GPL1_CUDA(cudaMemcpy(&ge, err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (ge) return fail(ctx, static_cast<gpl1_status>(ge), "a bounded wait in a GEMM ran out while tuning");
  ctx->gemm_tuned[key] = *c;
  return GPL1_OK;
}

}  // namespace

extern "C" gpl1_status gpl1_solve_shared_k(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                           const float* Y, long long ldy, const double* rho, const double* f_star,
                                           float* X, long long ldx, int nrhs, const gpl1_params* prm,
                                           gpl1_result* res) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!K || !Y || !rho || !X || !res || nrhs < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "NULL pointer or nrhs < 1");
  gpl1_status st = check_params(ctx, prm);
  if (st) return st;
  if (n < 64 || p < 64 || n % 64 || p % 64)
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "the shared-K form needs n and p to be multiples of 64");
  if (p > static_cast<long long>(35) * kConsumers) return fail(ctx, GPL1_ERR_UNSUPPORTED, "p exceeds %d", 35 * kConsumers);
  if (n > static_cast<long long>(9) * kConsumers) return fail(ctx, GPL1_ERR_UNSUPPORTED, "n exceeds %d", 9 * kConsumers);
  if (ldk < p || (ldk * 2) % 16 || reinterpret_cast<uintptr_t>(K) % 16)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "K rows must be 16-byte aligned, ldk >= p");
  if (ldy < n || ldx < p) return fail(ctx, GPL1_ERR_INVALID_ARG, "need ldy >= n and ldx >= p");
  for (int b = 0; b < nrhs; ++b)
    if (!(rho[b] > 0) || !std::isfinite(rho[b])) return fail(ctx, GPL1_ERR_INVALID_ARG, "rho[%d] must be > 0", b);
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (!ctx->encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    GPL1_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q),
              "cudaGetDriverEntryPointByVersion");
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(ctx, GPL1_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // workspace
  const size_t N = static_cast<size_t>(nrhs), nn = static_cast<size_t>(n), pp = static_cast<size_t>(p);
  size_t off = 256;   // [0] done count, [64] gemm error flag, [128] restart counts
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_kt = take(pp * nn * 2), o_g0 = take(N * pp * 4), o_g1 = take(N * pp * 4), o_d = take(N * pp * 4);
  const size_t o_dx = take(N * 3 * pp * 2), o_kdx = take(kMaxSplits * N * nn * 4), o_rs = take(N * 3 * nn * 2);
  const size_t o_st = take(N * mr_state_bytes()), o_res = take(N * sizeof(gpl1_result));
  const size_t o_rho = take(N * 8), o_fs = take(N * 8);
  const size_t o_xp = take(mr_exact_part_bytes(static_cast<int>(n), static_cast<int>(p), nrhs));
  const size_t o_rl = take(2 * N * sizeof(int));
  st = ensure_ws(ctx, off);
  if (st) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  int* done_count = reinterpret_cast<int*>(ws);
  int* gerr = reinterpret_cast<int*>(ws + 64);
  uint16_t* Kt = reinterpret_cast<uint16_t*>(ws + o_kt);
  float* G[2] = {reinterpret_cast<float*>(ws + o_g0), reinterpret_cast<float*>(ws + o_g1)};
  float* D = reinterpret_cast<float*>(ws + o_d);
  uint16_t* DXs = reinterpret_cast<uint16_t*>(ws + o_dx);
  float* KD = reinterpret_cast<float*>(ws + o_kdx);   // kMaxSplits partial slices of N x n
  uint16_t* Rs = reinterpret_cast<uint16_t*>(ws + o_rs);
  void* states = ws + o_st;
  gpl1_result* rdev = reinterpret_cast<gpl1_result*>(ws + o_res);
  double* rho_d = reinterpret_cast<double*>(ws + o_rho);
  double* fs_d = reinterpret_cast<double*>(ws + o_fs);
  void* xpart = ws + o_xp;   // column partials of the exact K x
  int* restart_cnt = reinterpret_cast<int*>(ws + 128);   // [2], zeroed with the counters
  int* restart_list = reinterpret_cast<int*>(ws + o_rl);
  cudaStream_t s = ctx->stream;
  GPL1_CUDA(cudaMemsetAsync(ws, 0, 256, s), "cudaMemsetAsync");
  GPL1_CUDA(cudaMemsetAsync(G[1], 0, N * pp * 4, s), "cudaMemsetAsync");
  GPL1_CUDA(cudaMemcpyAsync(rho_d, rho, N * 8, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(rho)");
  if (f_star) GPL1_CUDA(cudaMemcpyAsync(fs_d, f_star, N * 8, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(f*)");
  {   // every result slot starts as "not converged"; phase L overwrites it when its instance stops
    std::vector<gpl1_result> init(N);
    for (gpl1_result& r : init) {
      std::memset(&r, 0, sizeof r);
      r.status = GPL1_ERR_NOT_CONVERGED;
      r.stop = GPL1_STOP_MAX_ITER;
    }
    GPL1_CUDA(cudaMemcpyAsync(rdev, init.data(), N * sizeof(gpl1_result), cudaMemcpyHostToDevice, s),
              "cudaMemcpyAsync(results)");   // pageable source: staged before the call returns
  }
  const SolveParams sp = to_kernel_params(prm);
  if (!ctx->ev[0]) {
    GPL1_CUDA(cudaEventCreate(&ctx->ev[0]), "cudaEventCreate");
    GPL1_CUDA(cudaEventCreate(&ctx->ev[1]), "cudaEventCreate");
  }
  GPL1_CUDA(cudaEventRecord(ctx->ev[0], s), "cudaEventRecord");
  GPL1_CUDA(launch_transpose_bf16(K, ldk, Kt, static_cast<int>(n), static_cast<int>(p), s), "transpose");
  const long long tmo = prm->timeout_ns;
  if (prm->x0_is_zero) {
    GPL1_CUDA(launch_mr_init(Y, ldy, X, ldx, Rs, static_cast<int>(n), static_cast<int>(p), rho_d,
                             f_star ? fs_d : nullptr, states, sp, nrhs, s),
              "init");
  } else {   // x0 given: into the balls, K x0 on the tensor cores, then r0 and f0
    GPL1_CUDA(launch_mr_setup_x0(X, ldx, DXs, static_cast<int>(p), nrhs, rho_d, s), "setup x0");
    const int e0 = launch_gemm_bf16(ctx->encode, K, static_cast<int>(n), static_cast<int>(p), ldk, DXs, nrhs,
                                    static_cast<int>(3 * p), 3 * p, KD, n, 1.f, gerr, tmo, 128, s);
    if (e0) return e0 == -1 ? fail(ctx, GPL1_ERR_CUDA, "tensor map") : cuda_fail(ctx, static_cast<cudaError_t>(e0), "K x0");
    GPL1_CUDA(launch_mr_setup_r(KD, Y, ldy, Rs, static_cast<int>(n), nrhs, rho_d, f_star ? fs_d : nullptr, states,
                                sp, s),
              "setup r0");
  }
  // the two products' configurations, tuned once per shape and context on these operands
  GemmChoice c1, c2;
  if ((st = tuned_gemm(ctx, Kt, p, n, n, Rs, nrhs, 3 * n, 3 * n, G[0], p, 2.f, gerr, tmo, 1, 0, &c1))) return st;
  if ((st = tuned_gemm(ctx, K, n, p, ldk, DXs, nrhs, 3 * p, 3 * p, KD, n, 1.f, gerr, tmo, kMaxSplits,
                       static_cast<long long>(N * nn), &c2)))
    return st;
  for (int k = 0; k < prm->max_iter; ++k) {
    float* Gc = G[k & 1];
    float* Gp = G[(k + 1) & 1];
    int e = launch_gemm_bf16_cfg(ctx->encode, Kt, static_cast<int>(p), static_cast<int>(n), n, Rs, nrhs,
                                 static_cast<int>(3 * n), 3 * n, Gc, p, 2.f, gerr, tmo, c1.cfg, 1, 0, s);
    if (e) return e == -1 ? fail(ctx, GPL1_ERR_CUDA, "tensor map") : cuda_fail(ctx, static_cast<cudaError_t>(e), "gemm 1");
    GPL1_CUDA(launch_mr_phase_p(Gc, Gp, X, ldx, D, DXs, static_cast<int>(p), nrhs, k, states, sp, restart_cnt,
                                restart_list, s),
              "phase P");
    e = launch_gemm_bf16_cfg(ctx->encode, K, static_cast<int>(n), static_cast<int>(p), ldk, DXs, nrhs,
                             static_cast<int>(3 * p), 3 * p, KD, n, 1.f, gerr, tmo, c2.cfg, c2.splits,
                             static_cast<long long>(N * nn), s);
    if (e) return e == -1 ? fail(ctx, GPL1_ERR_CUDA, "tensor map") : cuda_fail(ctx, static_cast<cudaError_t>(e), "gemm 2");
    GPL1_CUDA(launch_mr_exact_kx(Kt, X, ldx, xpart, static_cast<int>(n), static_cast<int>(p), nrhs, states,
                                 restart_cnt, restart_list, k, ctx->num_sms, s),
              "exact K x");
    GPL1_CUDA(launch_mr_phase_l(KD, c2.splits, static_cast<long long>(N * nn), xpart, Y, ldy, X, ldx, D, Rs,
                                static_cast<int>(n), static_cast<int>(p), nrhs, k, states, sp, rdev, done_count, s),
              "phase L");
    if ((k & 3) == 3 || k + 1 == prm->max_iter) {
      int hd[2] = {0, 0};
      GPL1_CUDA(cudaMemcpyAsync(hd, ws, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
      GPL1_CUDA(cudaStreamSynchronize(s), "shared-K iteration");
      if (hd[0] >= nrhs) break;
      int ge = 0;
      GPL1_CUDA(cudaMemcpy(&ge, gerr, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
      if (ge) return fail(ctx, static_cast<gpl1_status>(ge), "a bounded wait in a GEMM ran out");
    }
  }
  GPL1_CUDA(cudaEventRecord(ctx->ev[1], s), "cudaEventRecord");
  GPL1_CUDA(cudaMemcpyAsync(res, rdev, N * sizeof(gpl1_result), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(res)");
  GPL1_CUDA(cudaStreamSynchronize(s), "shared-K solve");
  float ms = 0.f;
  GPL1_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]), "cudaEventElapsedTime");
  int worst = GPL1_OK;
  for (int b = 0; b < nrhs; ++b) {
    res[b].kernel_ms = ms;
    if (res[b].status != GPL1_OK && res[b].status != GPL1_ERR_NOT_CONVERGED) worst = res[b].status;
  }
  if (worst != GPL1_OK) return fail(ctx, static_cast<gpl1_status>(worst), "an instance failed (status %d)", worst);
  return GPL1_OK;
}

// ---------------------------------------------------------------------------
// Learned warm start (lista.cu).

namespace {

gpl1_status ensure_encode(gpl1_ctx* ctx) {
  if (ctx->encode) return GPL1_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  GPL1_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q),
            "cudaGetDriverEntryPointByVersion");
  if (q != cudaDriverEntryPointSuccess || !fn) return fail(ctx, GPL1_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  ctx->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return GPL1_OK;
}

gpl1_status check_lista(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk, int layers,
                        long long B) {
  if (!K) return fail(ctx, GPL1_ERR_INVALID_ARG, "K is NULL");
  if (layers < 1 || layers > 64) return fail(ctx, GPL1_ERR_INVALID_ARG, "layers must lie in [1, 64]");
  if (n < 64 || p < 64 || B < 64 || n % 64 || p % 64 || B % 64)
    return fail(ctx, GPL1_ERR_UNSUPPORTED, "n, p and the batch must be multiples of 64");
  if (ldk < p || (ldk * 2) % 16 || reinterpret_cast<uintptr_t>(K) % 16)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "K rows must be 16-byte aligned, ldk >= p");
  if (n > (1LL << 20) || p > (1LL << 20) || B > (1LL << 20)) return fail(ctx, GPL1_ERR_UNSUPPORTED, "too large");
  return GPL1_OK;
}

gpl1_status lista_status(gpl1_ctx* ctx, int r, int* gerr) {
  if (r == -1) return fail(ctx, GPL1_ERR_CUDA, "tensor map encoding failed");
  if (r != 0) return cuda_fail(ctx, static_cast<cudaError_t>(r), "learned warm start");
  int ge = 0;
  GPL1_CUDA(cudaMemcpyAsync(&ge, gerr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "learned warm start");
  if (ge) return fail(ctx, static_cast<gpl1_status>(ge), "a bounded wait in a GEMM ran out");
  return GPL1_OK;
}

}  // namespace

// gpl1_spectral_norm_sq: power iteration on K^T K (power.cu).
extern "C" gpl1_status gpl1_spectral_norm_sq(gpl1_ctx* ctx, const void* K, gpl1_dtype dt, long long n, long long p,
                                             long long ldk, int iters, double* out) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (dt != GPL1_F64 && dt != GPL1_F32 && dt != GPL1_BF16) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad dtype");
  if (!K || !out) return fail(ctx, GPL1_ERR_INVALID_ARG, "K and out must not be NULL");
  if (n < 1 || p < 1 || ldk < p) return fail(ctx, GPL1_ERR_INVALID_ARG, "need n, p >= 1 and ldk >= p");
  if (n > (1LL << 30) || p > (1LL << 30)) return fail(ctx, GPL1_ERR_UNSUPPORTED, "n or p too large");
  if (iters < 1 || iters > 100000) return fail(ctx, GPL1_ERR_INVALID_ARG, "iters must lie in [1, 100000]");
  if (reinterpret_cast<uintptr_t>(K) % elem_size(dt) != 0)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "K must be aligned to its element size");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  gpl1_status st = ensure_ws(ctx, power_ws_bytes(n, p, iters));
  if (st) return st;
  GPL1_CUDA(launch_power(dt, K, ldk, static_cast<int>(n), static_cast<int>(p), iters, ctx->ws, out, ctx->stream),
            "power iteration");
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "power iteration");
  if (!std::isfinite(*out)) return fail(ctx, GPL1_ERR_NONFINITE, "power iteration: non-finite estimate");
  return GPL1_OK;
}

extern "C" gpl1_status gpl1_lista_forward(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                          int layers, const float* W, const float* theta, const float* Y,
                                          long long ldy, long long B, float* X, long long ldx) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  gpl1_status st = check_lista(ctx, K, n, p, ldk, layers, B);
  if (st) return st;
  if (!W || !theta || !Y || !X || ldy < n || ldx < p) return fail(ctx, GPL1_ERR_INVALID_ARG, "bad pointer or stride");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((st = ensure_encode(ctx))) return st;
  if ((st = ensure_ws(ctx, 256 + lista_ws_bytes(layers, n, p, B)))) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  int* gerr = reinterpret_cast<int*>(ws);
  GPL1_CUDA(cudaMemsetAsync(gerr, 0, sizeof(int), ctx->stream), "cudaMemsetAsync");
  const int r = lista_pass(ctx->encode, ws + 256, gerr, K, n, p, ldk, layers, W, true, theta, Y, ldy, B, nullptr, 0,
                           X, ldx, nullptr, nullptr, nullptr, ctx->stream);
  return lista_status(ctx, r, gerr);
}

extern "C" gpl1_status gpl1_lista_grad(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                       int layers, const float* W, const float* theta, const float* Y, long long ldy,
                                       long long B, const float* Xt, long long ldt, float* dW, float* dtheta,
                                       double* loss) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  gpl1_status st = check_lista(ctx, K, n, p, ldk, layers, B);
  if (st) return st;
  if (!W || !theta || !Y || !Xt || !dW || !dtheta || ldy < n || ldt < p)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "bad pointer or stride");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((st = ensure_encode(ctx))) return st;
  if ((st = ensure_ws(ctx, 256 + lista_ws_bytes(layers, n, p, B)))) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  int* gerr = reinterpret_cast<int*>(ws);
  double* dloss = reinterpret_cast<double*>(ws + 64);
  GPL1_CUDA(cudaMemsetAsync(ws, 0, 128, ctx->stream), "cudaMemsetAsync");
  const int r = lista_pass(ctx->encode, ws + 256, gerr, K, n, p, ldk, layers, W, true, theta, Y, ldy, B, Xt, ldt,
                           nullptr, 0, dW, dtheta, dloss, ctx->stream);
  if (r == 0 && loss)
    GPL1_CUDA(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "cudaMemcpyAsync");
  return lista_status(ctx, r, gerr);
}

extern "C" gpl1_status gpl1_lista_train(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                        int layers, float* W, float* theta, float* adam_m, float* adam_v,
                                        const float* Y, long long ldy, const float* Xt, long long ldt, long long N,
                                        long long batch, int steps, int t0, float lr, float lr_theta,
                                        double* losses) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  gpl1_status st = check_lista(ctx, K, n, p, ldk, layers, batch);
  if (st) return st;
  if (!W || !theta || !adam_m || !adam_v || !Y || !Xt || ldy < n || ldt < p || N < batch || steps < 1 || t0 < 0)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "bad pointer, stride or count");
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((st = ensure_encode(ctx))) return st;
  const size_t wcount = static_cast<size_t>(layers) * p * n;
  const size_t grads = align_up((wcount + layers) * 4, 256);
  const size_t lbytes = align_up(static_cast<size_t>(steps) * 8, 256);
  if ((st = ensure_ws(ctx, 256 + grads + lbytes + lista_ws_bytes(layers, n, p, batch)))) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  int* gerr = reinterpret_cast<int*>(ws);
  float* dW = reinterpret_cast<float*>(ws + 256);
  float* dth = dW + wcount;
  double* dloss = reinterpret_cast<double*>(ws + 256 + grads);
  uint8_t* pass_ws = ws + 256 + grads + lbytes;
  GPL1_CUDA(cudaMemsetAsync(gerr, 0, sizeof(int), ctx->stream), "cudaMemsetAsync");
  const long long nb = N / batch;
  for (int s = 0; s < steps; ++s) {
    const long long b0 = (s % nb) * batch;
    const int r = lista_pass(ctx->encode, pass_ws, gerr, K, n, p, ldk, layers, W, true, theta, Y + b0 * ldy, ldy,
                             batch, Xt + b0 * ldt, ldt, nullptr, 0, dW, dth, dloss + s, ctx->stream);
    if (r != 0) return lista_status(ctx, r, gerr);
    GPL1_CUDA(lista_adam_step(W, dW, adam_m, adam_v, static_cast<long long>(wcount), lr, t0 + s + 1, ctx->stream),
              "adam");
    GPL1_CUDA(lista_adam_step(theta, dth, adam_m + wcount, adam_v + wcount, layers, lr_theta, t0 + s + 1, ctx->stream),
              "adam");
  }
  if (losses)
    GPL1_CUDA(cudaMemcpyAsync(losses, dloss, static_cast<size_t>(steps) * 8, cudaMemcpyDeviceToHost, ctx->stream),
              "cudaMemcpyAsync");
  return lista_status(ctx, 0, gerr);
}

// ---------------------------------------------------------------------------
// The learned warm start as a product: the network's initial weights, and
// warm-started solves with the plain cold solve as the fallback.

namespace {

bool solver_outcome(gpl1_status st) {
  return st == GPL1_OK || st == GPL1_ERR_NOT_CONVERGED || st == GPL1_ERR_LINESEARCH || st == GPL1_ERR_NONFINITE ||
         st == GPL1_ERR_TIMEOUT;
}

constexpr long long kWarmChunk = 4096;   // right-hand sides per network pass and per shared-K call

// x^L of rows [b0, b0 + m) of Y into the same rows of X: whole batches of 64
// directly, a ragged tail through a zero-padded 64-row buffer.
gpl1_status warm_forward(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk, int layers,
                         const float* W, const float* theta, const float* Y, long long ldy, float* X, long long ldx,
                         long long b0, long long m) {
  const long long full = m / 64 * 64;
  gpl1_status st;
  if (full > 0) {
    if ((st = ensure_ws(ctx, 256 + lista_ws_bytes(layers, n, p, full)))) return st;
    uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
    int* gerr = reinterpret_cast<int*>(ws);
    GPL1_CUDA(cudaMemsetAsync(gerr, 0, sizeof(int), ctx->stream), "cudaMemsetAsync");
    const int r = lista_pass(ctx->encode, ws + 256, gerr, K, n, p, ldk, layers, W, true, theta, Y + b0 * ldy, ldy,
                             full, nullptr, 0, X + b0 * ldx, ldx, nullptr, nullptr, nullptr, ctx->stream);
    if ((st = lista_status(ctx, r, gerr))) return st;
  }
  const long long t = m - full;
  if (t == 0) return GPL1_OK;
  if ((st = ensure_aux(ctx, static_cast<size_t>(64) * (n + p) * sizeof(float)))) return st;
  float* Yp = static_cast<float*>(ctx->aux);
  float* Xp = Yp + 64 * n;
  GPL1_CUDA(cudaMemsetAsync(Yp, 0, static_cast<size_t>(64) * n * sizeof(float), ctx->stream), "cudaMemsetAsync");
  GPL1_CUDA(cudaMemcpy2DAsync(Yp, n * sizeof(float), Y + (b0 + full) * ldy, ldy * sizeof(float), n * sizeof(float),
                              t, cudaMemcpyDeviceToDevice, ctx->stream),
            "cudaMemcpy2DAsync");
  if ((st = ensure_ws(ctx, 256 + lista_ws_bytes(layers, n, p, 64)))) return st;
  uint8_t* ws = static_cast<uint8_t*>(ctx->ws);
  int* gerr = reinterpret_cast<int*>(ws);
  GPL1_CUDA(cudaMemsetAsync(gerr, 0, sizeof(int), ctx->stream), "cudaMemsetAsync");
  const int r = lista_pass(ctx->encode, ws + 256, gerr, K, n, p, ldk, layers, W, true, theta, Yp, n, 64, nullptr, 0,
                           Xp, p, nullptr, nullptr, nullptr, ctx->stream);
  if ((st = lista_status(ctx, r, gerr))) return st;
  GPL1_CUDA(cudaMemcpy2DAsync(X + (b0 + full) * ldx, ldx * sizeof(float), Xp, p * sizeof(float), p * sizeof(float), t,
                              cudaMemcpyDeviceToDevice, ctx->stream),
            "cudaMemcpy2DAsync");
  return GPL1_OK;
}

}  // namespace

extern "C" gpl1_status gpl1_lista_init(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                       int layers, const double* lambdas, long long count, int power_iters, float* W,
                                       float* theta, double* L_out) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  gpl1_status st = check_lista(ctx, K, n, p, ldk, layers, 64);
  if (st) return st;
  if (!W || !theta || !lambdas || count < 1) return fail(ctx, GPL1_ERR_INVALID_ARG, "need W, theta and lambdas");
  std::vector<double> lam(lambdas, lambdas + count);
  for (double v : lam)
    if (!(v >= 0) || !std::isfinite(v)) return fail(ctx, GPL1_ERR_INVALID_ARG, "lambdas must be finite, >= 0");
  double L = 0.0;
  if ((st = gpl1_spectral_norm_sq(ctx, K, GPL1_BF16, n, p, ldk, power_iters, &L))) return st;
  if (!(L > 0)) return fail(ctx, GPL1_ERR_INVALID_ARG, "K is zero");
  // the median of the lambdas (the mean of the two middle values for an even count)
  std::sort(lam.begin(), lam.end());
  const size_t c = lam.size();
  const double med = c % 2 ? lam[c / 2] : 0.5 * (lam[c / 2 - 1] + lam[c / 2]);
  GPL1_CUDA(lista_init_weights(K, ldk, static_cast<int>(n), static_cast<int>(p), layers, static_cast<float>(1.0 / L), W,
                               ctx->stream),
            "network initialisation");
  std::vector<float> th(static_cast<size_t>(layers), static_cast<float>(med / L));
  GPL1_CUDA(cudaMemcpyAsync(theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
            "cudaMemcpyAsync(theta)");
  GPL1_CUDA(cudaStreamSynchronize(ctx->stream), "network initialisation");
  if (L_out) *L_out = L;
  return GPL1_OK;
}

extern "C" gpl1_status gpl1_solve_warm(gpl1_ctx* ctx, const void* K, long long n, long long p, long long ldk,
                                       int layers, const float* W, const float* theta, const float* Y, long long ldy,
                                       const double* rho, const double* f_star, float* X, long long ldx, int nrhs,
                                       const gpl1_params* prm, int warm_max_iter, gpl1_result* res, int* fell_back,
                                       int* fallbacks) {
  if (!ctx) return GPL1_ERR_INVALID_ARG;
  if (!W || !theta || !Y || !rho || !X || !res || nrhs < 1 || ldy < n || ldx < p)
    return fail(ctx, GPL1_ERR_INVALID_ARG, "NULL pointer, nrhs < 1 or bad stride");
  gpl1_status st = check_params(ctx, prm);
  if (st) return st;
  if ((st = check_lista(ctx, K, n, p, ldk, layers, 64))) return st;
  GPL1_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
  if ((st = ensure_encode(ctx))) return st;
  // 1. the network's output for every right-hand side (the warm start x0)
  for (long long b0 = 0; b0 < nrhs; b0 += kWarmChunk)
    if ((st = warm_forward(ctx, K, n, p, ldk, layers, W, theta, Y, ldy, X, ldx, b0,
                           std::min<long long>(kWarmChunk, nrhs - b0))))
      return st;
  // 2. Alg. GP + SS from its projection onto each ball (shared-K form; alpha_0
  //    from the projected-gradient step at x0, rule 1)
  gpl1_params pw = *prm;
  pw.x0_is_zero = 0;
  pw.alpha0_rule = 1;
  if (warm_max_iter > 0) pw.max_iter = warm_max_iter;
  for (long long b0 = 0; b0 < nrhs; b0 += kWarmChunk) {
    const int m = static_cast<int>(std::min<long long>(kWarmChunk, nrhs - b0));
    st = gpl1_solve_shared_k(ctx, K, n, p, ldk, Y + b0 * ldy, ldy, rho + b0, f_star ? f_star + b0 : nullptr,
                             X + b0 * ldx, ldx, m, &pw, res + b0);
    if (!solver_outcome(st)) return st;
  }
  // 3. the fallback: every instance the warm solve did not bring to the stop is
  //    solved again from x0 = 0 by the plain solver with the caller's parameters
  gpl1_params pc = *prm;
  pc.x0_is_zero = 1;
  pc.engine = GPL1_ENGINE_AUTO;
  int nfb = 0;
  for (int b = 0; b < nrhs; ++b) {
    if (fell_back) fell_back[b] = 0;
    if (res[b].status == GPL1_OK) continue;
    gpl1_problem pr;
    std::memset(&pr, 0, sizeof pr);
    pr.K = K;
    pr.n = n;
    pr.p = p;
    pr.ldk = ldk;
    pr.y = Y + b * ldy;
    pr.rho = rho[b];
    pr.x = X + b * ldx;
    pr.f_star = f_star ? f_star[b] : -1.0;
    gpl1_result r;
    st = gpl1_solve(ctx, &pr, GPL1_BF16, &pc, &r);
    if (!solver_outcome(st)) return st;
    res[b] = r;
    if (fell_back) fell_back[b] = 1;
    ++nfb;
  }
  if (fallbacks) *fallbacks = nfb;
  return GPL1_OK;
}
