// fovea_render_noalloc: the single-frame render path for callers that cannot
// allocate GPU memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where the
// allocator is owned by someone else (a host framework with its own memory
// pool and a fixed budget, an inference server that has reserved the device
// up front), and code that must not allocate while the device is being driven
// by a latency-critical loop. For them this entry point takes device input and
// output buffers and renders with the same kernels as fovea_render, but keeps
// all of its working memory (the per-block sigma/radius records, their ranks,
// the radius-ordered work list and the counters) in one statically sized
// array that is part of the loaded library image. It calls no cudaMalloc,
// cudaFree or other allocating routine.
//
// Every call shares that array, so calls whose GPU work overlaps (several
// streams, or several host threads) race and must be serialised by the
// caller. The array keeps the last call's contents; the counters that must
// start at zero are cleared at the start of every call (an asynchronous
// memset on the call's stream), the fault word among them, so
// fovea_noalloc_check reports on the latest call only.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fovea_host.h"
#include "fovea_internal.cuh"

using namespace fovea;

namespace {

constexpr long long kMaxItems = FOVEA_NOALLOC_MAX_BLOCKS;
constexpr size_t kItemsBytes = (size_t)kMaxItems * sizeof(ItemInfo);
constexpr size_t kRankBytes = (size_t)kMaxItems * sizeof(int);
constexpr size_t kOrderBytes = (size_t)kMaxItems * sizeof(int);
constexpr size_t kCounterBytes = (size_t)CNT_TOTAL * sizeof(unsigned int);
constexpr size_t kScratchBytes = kItemsBytes + kRankBytes + kOrderBytes + kCounterBytes;

// Zero at load; held by every GPU that loads the library until process exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to

// Unique id of the current device's CUDA context (0 if the driver cannot
// say). cudaDeviceReset destroys a device's primary context, and the module
// (with the array) is loaded again, possibly elsewhere, in the next one.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    cudaGetLastError();
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Device address of the scratch array on the current device. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress, once per device (with that device current), and
// again only if the device's context has been replaced since (after a
// cudaDeviceReset).
int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_cuda_failure(e);
  if (dev < 0 || dev >= kMaxDevices) return FOVEA_EUNSUPPORTED;
  e = cudaSetDevice(dev);  // makes the device's primary context current on this thread
  if (e != cudaSuccess) return record_cuda_failure(e);
  const unsigned long long ctx_id = current_context_id();
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return record_cuda_failure(e);
    if (!p) return FOVEA_ECUDA;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx_id;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return FOVEA_OK;
}

unsigned int* counters_of(unsigned char* base) {
  return reinterpret_cast<unsigned int*>(base + kItemsBytes + kRankBytes + kOrderBytes);
}

}  // namespace

extern "C" int fovea_render_noalloc(const void* in_dev, void* out_dev, int width, int height, int channels,
                                    int format, int block, double sigma0, double k, float fix_x, float fix_y,
                                    void* stream) {
  if (!in_dev || !out_dev) return FOVEA_EINVAL;
  FrameLaw law;
  law.sigma0 = sigma0;
  law.k = k;
  int st = check_frame(width, height, channels, format, block, law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  if (block > 32) return FOVEA_EUNSUPPORTED;  // one work item per block here
  const size_t nb = frame_bytes(width, height, channels, format);
  const char* a = static_cast<const char*>(in_dev);
  const char* b = static_cast<const char*>(out_dev);
  if (a < b + nb && b < a + nb) return FOVEA_EINVAL;
  const long long items = (long long)((width + block - 1) / block) * ((height + block - 1) / block);
  if (items > kMaxItems) return FOVEA_EUNSUPPORTED;  // more blocks than the static scratch holds

  unsigned char* base = nullptr;
  st = scratch_for_current_device(&base);
  if (st != FOVEA_OK) return st;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return record_cuda_failure(e);

  Workspace ws;
  ws.items = reinterpret_cast<ItemInfo*>(base);
  ws.rank = reinterpret_cast<int*>(base + kItemsBytes);
  ws.order = reinterpret_cast<int*>(base + kItemsBytes + kRankBytes);
  ws.counters = counters_of(base);
  ws.capacity = kMaxItems;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The counters (ticket, done flags, radius histogram) must start at zero.
  e = cudaMemsetAsync(ws.counters, 0, kCounterBytes, s);
  if (e != cudaSuccess) return record_cuda_failure(e);

  FrameSource src;
  std::memset(&src, 0, sizeof(src));
  src.one.in = in_dev;
  src.one.out = out_dev;
  src.one.W = width; src.one.H = height; src.one.C = channels; src.one.fmt = format;
  src.one.B = block;
  src.one.T = block;
  src.one.nbx = (width + block - 1) / block;
  src.one.nbxb = src.one.nbx;
  src.one.nby = (height + block - 1) / block;
  src.one.fx = fix_x; src.one.fy = fix_y;
  src.one.sigma0 = sigma0; src.one.k = k;
  src.one_total = items;

  const int rmax = radius_bound(width, height, block, fix_x, fix_y, law);
  const int sg = (int)((items + 255) / 256);
  e = launch_sigma_order(src, ws, sg < 1 ? 1 : (sg > 4 * sms ? 4 * sms : sg), nullptr, nullptr, s);
  if (e != cudaSuccess) return record_cuda_failure(e);
  const FwdConfig cfg{256, 0, 32, 0};
  const int fmt_mask = format == FOVEA_F32_CHW ? 2 : 1;
  const int per = forward_max_ctas_per_sm(cfg, rmax, fmt_mask);
  if (per <= 0) return FOVEA_EUNSUPPORTED;
  e = launch_forward(src, ws, cfg, rmax, fmt_mask, per * sms, s);
  if (e != cudaSuccess) return record_cuda_failure(e);
  return FOVEA_OK;
}

extern "C" int fovea_noalloc_check(void* stream, unsigned int* faults) {
  if (faults) *faults = 0u;
  unsigned char* base = nullptr;
  int st = scratch_for_current_device(&base);
  if (st != FOVEA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int word = 0u;
  cudaError_t e = cudaMemcpyAsync(&word, counters_of(base) + CNT_ERROR, sizeof(word), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return record_cuda_failure(e);
  if (faults) *faults = word;
  return fault_status(word);
}
