// C ABI of libfovea: contexts, argument checks, workspace, launches, graphs.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fovea_internal.cuh"
#include "fovea_host.h"

using namespace fovea;

namespace {

thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return e == cudaErrorMemoryAllocation ? FOVEA_ENOMEM : FOVEA_ECUDA;
}

#define FOVEA_CUDA(call)                      \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

}  // namespace

namespace fovea {

int fault_status(unsigned int word) {
  if (!word) return FOVEA_OK;
  if (word & kFaultWait) return FOVEA_ETIMEOUT;
  if (word & ~(kFaultSigmaRange | kFaultValueRange)) return FOVEA_ECUDA;
  return FOVEA_EINVAL;
}

}  // namespace fovea

namespace {

constexpr int kBatchSlots = 4;
constexpr double kPi = 3.14159265358979323846;

// Zero the output planes of every frame of a device-resident batch (the
// adjoint accumulates into them).
// Zeroes every frame's float32 output (the adjoint scatter-adds into it).
// The launch is captured once for any batch size, so the grid is fixed: CTA
// row y takes frames y, y + gridDim.y, ...; the CTAs of a row split a frame
// with 16-byte stores where its alignment allows.
__global__ void zero_outputs_kernel(const BatchHeader* hdr, const FrameDesc* frames) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = hdr->nframes;
  for (int f = blockIdx.y; f < nf; f += gridDim.y) {
    const FrameDesc fd = frames[f];
    const size_t n = (size_t)fd.W * fd.H * fd.C;
    float* out = static_cast<float*>(fd.out);
    size_t head = 0;
    if ((reinterpret_cast<uintptr_t>(out) & 15) == 0) {
      const size_t n4 = n / 4;
      float4* o4 = reinterpret_cast<float4*>(out);
      for (size_t i = t0; i < n4; i += stride) o4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      head = 4 * n4;
    }
    for (size_t i = head + t0; i < n; i += stride) out[i] = 0.0f;
  }
}

}  // namespace

struct fovea_ctx {
  int W = 0, H = 0, C = 0, B = 32, fmt = 0;
  fovea::FrameLaw law;
  bool batch_only = false;
  int device = 0, num_sms = 0;
  FwdConfig cfg{256, 0, 32, 1};
  bool cfg_tuned = false;
  // set by fovea_set_config: batches then run ctx->cfg instead of the
  // configuration tuned for their kind of batch
  bool cfg_explicit = false;
  Workspace ws{};
  cudaStream_t capture_stream = nullptr;
  // device-resident batch (header + descriptors)
  void* batch_dev = nullptr;
  size_t batch_dev_cap = 0;
  void* batch_host[kBatchSlots] = {};
  cudaEvent_t batch_ev[kBatchSlots] = {};
  size_t batch_host_cap = 0;
  int batch_slot = 0;
  // CUDA graphs of the batch launch sequence, keyed by the launch (adjoint,
  // format mask, tensor-core channel count, radius bound) and the
  // configuration it was captured with
  std::map<std::pair<long long, long long>, cudaGraphExec_t> graphs;
  // Batch buffers replaced by larger ones while queued work may still read
  // them: freed by fovea_destroy, so growing never waits for the device.
  std::vector<void*> retired_dev, retired_host;
  // optional events bracketing the persistent blur kernel (measurement)
  cudaEvent_t kev_start = nullptr, kev_stop = nullptr;
  // per-radius item lists of the single-frame path
  int* blist = nullptr;
  size_t blist_cap = 0;  // ints
  // fovea_render_host: two staging slots and three internal streams, so that
  // the copies of one call overlap the kernels of the next
  struct HostSlot {
    void* in_dev = nullptr;
    void* out_dev = nullptr;
    cudaEvent_t ev_h2d = nullptr, ev_comp = nullptr, ev_d2h = nullptr;
    bool used = false;
  } hslot[2];
  int hslot_next = 0;
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_entry = nullptr;
  size_t host_io_bytes = 0;
  // Gaussian-pyramid levels (fovea_render_pyramid)
  float* pyr = nullptr;
  size_t pyr_bytes = 0;
  // set by every call that enqueues workspace use on the caller's stream;
  // the next fovea_render_host orders its kernels after that work
  bool caller_stream_used = false;
  // fovea_check_async: pinned copy of the device fault word and the event
  // that marks its arrival
  unsigned int* fault_host = nullptr;
  cudaEvent_t fault_ev = nullptr;
  bool fault_copy_pending = false;
  // tensor maps of the last two input buffers of the single-frame path
  // (fovea_render_host alternates two staging buffers); a map depends only on
  // the buffer, the context's fixed frame shape and the rows per box
  struct MapEntry {
    alignas(kTensorMapAlign) unsigned char map[kTensorMapBytes] = {};
    const void* in = nullptr;
    int rows = 0;
    bool ok = false;
  } maps[2];
  int map_next = 0;
};

namespace fovea {

double block_centre_host(int b, int B) { return (double)B * (double)b + 0.5 * (double)B; }

int grid_origin(float f, int B, int grid) {
  if (grid != FOVEA_GRID_CENTRED) return 0;
  const long long c = (long long)std::floor((double)f + 0.5);
  long long o = ((long long)(B / 2) - c) % B;
  if (o < 0) o += B;
  return (int)o;
}

void grid_dims(int W, int H, int B, int ox, int oy, int* nbx, int* nby) {
  *nbx = (W + ox + B - 1) / B;
  *nby = (H + oy + B - 1) / B;
}

int radius_bound(int W, int H, int B, float fxf, float fyf, const FrameLaw& law) {
  if (law.smap) {
    const double s3 = 3.0 * law.smap_max;
    return s3 > 1e9 ? 1000000000 : (int)std::ceil(s3);
  }
  // The largest eccentricity over the block grid is reached at one of its
  // four corner blocks; every step is rounded on its own (this file is
  // compiled without floating-point contraction), so the result equals the
  // device's radius of that block.
  const double fx = fxf, fy = fyf, sigma0 = law.sigma0, k = law.k;
  const int ox = grid_origin(fxf, B, law.grid), oy = grid_origin(fyf, B, law.grid);
  int nbx, nby;
  grid_dims(W, H, B, ox, oy, &nbx, &nby);
  const int bxs[2] = {0, nbx - 1}, bys[2] = {0, nby - 1};
  int rmax = 0;
  for (int bx : bxs)
    for (int by : bys) {
      volatile double cx = block_centre_host(bx, B) - (double)ox;
      volatile double cy = block_centre_host(by, B) - (double)oy;
      volatile double dx = cx - fx;
      volatile double dy = cy - fy;
      volatile double dx2 = dx * dx;
      volatile double dy2 = dy * dy;
      volatile double e = std::sqrt(dx2 + dy2);
      volatile double ke = k * e;
      volatile double s = sigma0 + ke;
      volatile double s3 = 3.0 * s;
      double rc = std::ceil(s3);
      int r = rc > 1e9 ? 1000000000 : (int)rc;
      rmax = std::max(rmax, r);
    }
  return rmax;
}

int check_frame(int W, int H, int C, int fmt, int B, const FrameLaw& law, float fx, float fy) {
  if (W <= 0 || H <= 0 || B <= 0) return FOVEA_EINVAL;
  if (B > kMaxBlock || (B > 32 && B % 32 != 0)) return FOVEA_EUNSUPPORTED;
  if (C < 1 || C > 4) return FOVEA_EINVAL;
  if (fmt != FOVEA_U8_HWC && fmt != FOVEA_F32_CHW) return FOVEA_EINVAL;
  if (law.grid != FOVEA_GRID_ANCHORED && law.grid != FOVEA_GRID_CENTRED) return FOVEA_EINVAL;
  if (law.smap) {
    if (!finite_nonneg(law.smap_max)) return FOVEA_EINVAL;
  } else if (!finite_nonneg(law.sigma0) || !finite_nonneg(law.k)) {
    return FOVEA_EINVAL;
  }
  if (!std::isfinite(fx) || !std::isfinite(fy)) return FOVEA_EINVAL;
  if ((long long)W * H * C > (1ll << 31) - 1) return FOVEA_EUNSUPPORTED;
  if (radius_bound(W, H, B, fx, fy, law) > kMaxRadius) return FOVEA_EUNSUPPORTED;
  return FOVEA_OK;
}

size_t frame_bytes(int W, int H, int C, int fmt) {
  return (size_t)W * H * C * (fmt == FOVEA_U8_HWC ? 1 : 4);
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

// Items are tiles of side min(B, 32) (per_block: one item per block, for
// sigma tables only).
FrameDesc make_desc(int W, int H, int C, int fmt, int B, const void* in, void* out, float fx, float fy,
                    const FrameLaw& law, long long item0, bool per_block = false) {
  FrameDesc d;
  std::memset(&d, 0, sizeof(d));
  d.in = in;
  d.out = out;
  d.W = W; d.H = H; d.C = C; d.fmt = fmt;
  d.B = B;
  d.ox = grid_origin(fx, B, law.grid);
  d.oy = grid_origin(fy, B, law.grid);
  d.T = (per_block || B <= 32) ? B : 32;
  grid_dims(W, H, d.T, d.ox, d.oy, &d.nbx, &d.nby);
  int nbyb = 0;
  grid_dims(W, H, B, d.ox, d.oy, &d.nbxb, &nbyb);
  d.fx = fx; d.fy = fy;
  d.sigma0 = law.sigma0; d.k = law.k;
  d.smap = law.smap;
  d.smap_max = law.smap ? law.smap_max : 0.0;
  d.item0 = item0;
  return d;
}

}  // namespace fovea

namespace {

void drop_graphs(fovea_ctx* ctx) {
  // An executable graph destroyed while a launch of it is in flight is
  // released when that launch completes.
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

// Item workspace for `items` items. Grows at least twofold, so a stream of
// ever larger batches reallocates (and recaptures its graphs) a logarithmic
// number of times; the old buffers may still be read by queued work and are
// retired rather than freed, so growing does not wait for the device.
int ensure_workspace(fovea_ctx* ctx, long long items) {
  if (ctx->ws.capacity >= items && ctx->ws.counters) return FOVEA_OK;
  long long cap = std::max<long long>({items, 2 * ctx->ws.capacity, 1024});
  if (ctx->ws.items) {
    ctx->retired_dev.push_back(ctx->ws.items);
    ctx->retired_dev.push_back(ctx->ws.rank);
    ctx->retired_dev.push_back(ctx->ws.order);
    ctx->ws.items = nullptr;
    ctx->ws.rank = ctx->ws.order = nullptr;
    ctx->ws.capacity = 0;
    drop_graphs(ctx);
  }
  FOVEA_CUDA(cudaMalloc(&ctx->ws.items, cap * sizeof(ItemInfo)));
  FOVEA_CUDA(cudaMalloc(&ctx->ws.rank, cap * sizeof(int)));
  FOVEA_CUDA(cudaMalloc(&ctx->ws.order, cap * sizeof(int)));
  if (!ctx->ws.counters) {
    FOVEA_CUDA(cudaMalloc(&ctx->ws.counters, CNT_TOTAL * sizeof(unsigned int)));
    FOVEA_CUDA(cudaMemset(ctx->ws.counters, 0, CNT_TOTAL * sizeof(unsigned int)));
    FOVEA_CUDA(cudaDeviceSynchronize());
  }
  ctx->ws.capacity = cap;
  return FOVEA_OK;
}

int sigma_grid(long long items, int num_sms) {
  long long g = (items + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, 4ll * num_sms));
}

// The tensor-core kernels serve launches whose frames are all uint8 with one
// channel count (tc_c = that count, 0 otherwise). Returns the kernel a
// launch runs on: 0 the fp32 FMA kernel, 1 the mma.sync kernel, 2 the
// kernel with pass 1 on tcgen05, 3 the kernel with both passes on tcgen05
// (2 and 3 where the radius bound, row chunk and channel count permit, and
// for 3 when every frame's rows can be loaded by TMA (all_tma); else the
// mma.sync kernel); 4 float32-only launches on the tensor cores (every
// frame TMA-loadable; else the fp32 kernel).
int tc_kind(const FwdConfig& cfg, int fmt_mask, int tc_c, int rmax, bool all_tma = true) {
  if (cfg.tc && fmt_mask == 2) return all_tma && tcf_supports(rmax) ? 4 : 0;  // float32 frames
  if (!cfg.tc || fmt_mask != 1 || tc_c <= 0) return 0;
  if (cfg.tc == 2 && rmax <= kUmmaMaxRadius && cfg.rows_per_chunk <= 32) return 2;
  if (cfg.tc == 3 && all_tma && tc05_supports(rmax, tc_c) && cfg.rows_per_chunk == 16) return 3;
  return 1;
}

int forward_grid(const fovea_ctx* ctx, const FwdConfig& cfg, int rmax, int fmt_mask, int tc_c, bool all_tma = true) {
  const int kind = tc_kind(cfg, fmt_mask, tc_c, rmax, all_tma);
  int per = kind == 4   ? tcf_forward_max_ctas_per_sm(rmax, tc_c)
            : kind == 3 ? tc05_forward_max_ctas_per_sm(cfg, rmax)
            : kind == 2 ? umma_forward_max_ctas_per_sm(cfg, rmax, tc_c)
            : kind == 1 ? tc_forward_max_ctas_per_sm(cfg, rmax, tc_c)
                        : forward_max_ctas_per_sm(cfg, rmax, fmt_mask);
  if (per <= 0) return 0;
  if (cfg.ctas_per_sm > 0) per = std::min(per, cfg.ctas_per_sm);
  return per * ctx->num_sms;
}

FwdConfig to_fwd(const fovea_config& c) {
  return FwdConfig{c.threads, c.ctas_per_sm, c.rows_per_chunk, c.tensor_cores};
}

// A configuration as one number (part of the batch graphs' key).
long long config_code(const FwdConfig& c) {
  return (((long long)c.threads * 128 + c.rows_per_chunk) * 4 + c.tc) * 16 + c.ctas_per_sm;
}

// tc: the tensor-core adjoint (tensor_cores = 2; measured slower than the
// fp32 adjoint, which every other setting runs), else the fp32 one
int adjoint_grid(fovea_ctx* ctx, int rmax, bool tc) {
  int per = tc ? tca_adjoint_max_ctas_per_sm(rmax) : adjoint_max_ctas_per_sm(rmax);
  if (per <= 0) return 0;
  return per * ctx->num_sms;
}

// Stage n frame descriptors into the pinned slot ring and copy them to the
// device-resident batch buffer on `s`. Returns total items in *total.
// Bytes of the batch table for n frames: header, descriptors, then one
// tensor map per frame on its alignment.
size_t batch_table_maps_offset(int n) {
  return (sizeof(BatchHeader) + (size_t)n * sizeof(FrameDesc) + kTensorMapAlign - 1) & ~(kTensorMapAlign - 1);
}
size_t batch_table_bytes(int n) { return batch_table_maps_offset(n) + (size_t)n * kTensorMapBytes; }

// Device batch table and its pinned host staging slots for `bytes` bytes.
// Replaced buffers are retired (queued copies and kernels may still use
// them), so growing waits for nothing.
int ensure_batch_tables(fovea_ctx* ctx, size_t bytes) {
  if (bytes > ctx->batch_dev_cap) {
    if (ctx->batch_dev) {
      ctx->retired_dev.push_back(ctx->batch_dev);
      ctx->batch_dev = nullptr;
      ctx->batch_dev_cap = 0;
      drop_graphs(ctx);
    }
    size_t cap = std::max<size_t>(bytes * 2, 64 * 1024);
    FOVEA_CUDA(cudaMalloc(&ctx->batch_dev, cap));
    ctx->batch_dev_cap = cap;
  }
  if (bytes > ctx->batch_host_cap) {
    for (int i = 0; i < kBatchSlots; ++i) {
      if (ctx->batch_host[i]) ctx->retired_host.push_back(ctx->batch_host[i]);
      ctx->batch_host[i] = nullptr;
    }
    ctx->batch_host_cap = 0;
    size_t cap = std::max<size_t>(bytes * 2, 64 * 1024);
    for (int i = 0; i < kBatchSlots; ++i) {
      FOVEA_CUDA(cudaHostAlloc(&ctx->batch_host[i], cap, cudaHostAllocDefault));
      if (!ctx->batch_ev[i]) FOVEA_CUDA(cudaEventCreateWithFlags(&ctx->batch_ev[i], cudaEventDisableTiming));
    }
    ctx->batch_host_cap = cap;
  }
  return FOVEA_OK;
}

FrameLaw law_of(const fovea_frame& f) {
  FrameLaw fl;
  fl.sigma0 = f.sigma0; fl.k = f.k; fl.smap = f.sigma_map; fl.smap_max = f.sigma_map_max; fl.grid = f.grid;
  return fl;
}

// Whether p is device memory (not page-locked host memory mapped into the
// device's address space, nor an address CUDA does not know).
bool in_device_memory(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int upload_batch(fovea_ctx* ctx, const FwdConfig& cfg, const fovea_frame* frames, int n, bool adjoint, cudaStream_t s,
                 long long* total, int* rmax, int* fmt_mask, int* tc_c, bool* all_tma) {
  if (n <= 0 || !frames) return FOVEA_EINVAL;
  std::vector<FrameDesc> descs((size_t)n);
  long long item0 = 0;
  int rm = 0;
  int mask = 0, cc = -1;
  for (int i = 0; i < n; ++i) {
    const fovea_frame& f = frames[i];
    const FrameLaw fl = law_of(f);
    int st = check_frame(f.width, f.height, f.channels, f.format, ctx->B, fl, f.fix_x, f.fix_y);
    if (st != FOVEA_OK) return st;
    if (adjoint && f.format != FOVEA_F32_CHW) return FOVEA_EINVAL;
    if (!f.in || !f.out) return FOVEA_EINVAL;
    const size_t nb = frame_bytes(f.width, f.height, f.channels, f.format);
    if (overlaps(f.in, nb, f.out, nb)) return FOVEA_EINVAL;
    descs[(size_t)i] = make_desc(f.width, f.height, f.channels, f.format, ctx->B, f.in, f.out, f.fix_x,
                                 f.fix_y, fl, item0);
    item0 += (long long)descs[(size_t)i].nbx * descs[(size_t)i].nby;
    rm = std::max(rm, radius_bound(f.width, f.height, ctx->B, f.fix_x, f.fix_y, fl));
    mask |= f.format == FOVEA_F32_CHW ? 2 : 1;
    cc = cc == -1 ? f.channels : (cc == f.channels ? cc : 0);
  }
  if (item0 > (1ll << 31) - 1) return FOVEA_EUNSUPPORTED;
  int st = ensure_workspace(ctx, item0);
  if (st != FOVEA_OK) return st;
  // tensor maps of the uint8 frames for the tensor-core kernel's row loads
  const size_t maps_off = batch_table_maps_offset(n);
  const size_t bytes = batch_table_bytes(n);
  if (maps_off > (size_t)0x7fffffff) return FOVEA_EUNSUPPORTED;
  st = ensure_batch_tables(ctx, bytes);
  if (st != FOVEA_OK) return st;
  const int slot = ctx->batch_slot;
  ctx->batch_slot = (slot + 1) % kBatchSlots;
  FOVEA_CUDA(cudaEventSynchronize(ctx->batch_ev[slot]));  // copy from this slot finished
  BatchHeader hdr;
  hdr.nframes = n;
  hdr.maps_offset = (int)maps_off;
  hdr.total_items = item0;
  char* hbuf = static_cast<char*>(ctx->batch_host[slot]);
  bool every_tma = true;
  for (int i = 0; i < n; ++i) {
    FrameDesc& d = descs[(size_t)i];
    void* map = hbuf + maps_off + (size_t)i * kTensorMapBytes;
    // rows are loaded by TMA only from device memory (a frame in mapped host
    // memory is staged with plain loads)
    d.tma = 0;
    if (!adjoint && in_device_memory(d.in)) {
      if (d.fmt == FOVEA_U8_HWC) d.tma = make_u8_tensor_map(map, d.in, d.W, d.H, d.C, cfg.rows_per_chunk) ? 1 : 0;
      else if (cfg.tc) d.tma = make_f32_tensor_map(map, d.in, d.W, d.H, d.C, 16) ? 1 : 0;
    }
    if (!d.tma) std::memset(map, 0, kTensorMapBytes);
    every_tma = every_tma && d.tma;
  }
  *all_tma = every_tma;
  std::memcpy(hbuf, &hdr, sizeof(hdr));
  std::memcpy(hbuf + sizeof(hdr), descs.data(), (size_t)n * sizeof(FrameDesc));
  FOVEA_CUDA(cudaMemcpyAsync(ctx->batch_dev, hbuf, bytes, cudaMemcpyHostToDevice, s));
  FOVEA_CUDA(cudaEventRecord(ctx->batch_ev[slot], s));
  *total = item0;
  *rmax = rm;
  *fmt_mask = mask;
  *tc_c = cc > 0 ? cc : 0;
  return FOVEA_OK;
}

FrameSource batch_source(fovea_ctx* ctx) {
  FrameSource src;
  std::memset(&src, 0, sizeof(src));
  src.hdr = static_cast<const BatchHeader*>(ctx->batch_dev);
  src.frames = reinterpret_cast<const FrameDesc*>(static_cast<const char*>(ctx->batch_dev) + sizeof(BatchHeader));
  return src;
}

// Enqueue (or capture) the batch launch sequence for the current batch buffer.
int enqueue_batch_kernels(fovea_ctx* ctx, const FwdConfig& cfg, bool adjoint, int rbound, int fmt_mask, int tc_c,
                          bool all_tma, cudaStream_t s) {
  const FrameSource src = batch_source(ctx);
  const int sg = 4 * ctx->num_sms;
  if (adjoint) {
    cudaError_t e;
    zero_outputs_kernel<<<dim3(16, 64), 256, 0, s>>>(src.hdr, src.frames);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  }
  cudaError_t e = launch_sigma_order(src, ctx->ws, sg, nullptr, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (adjoint) {
    const bool tca = cfg.tc == 2;
    int grid = adjoint_grid(ctx, rbound, tca);
    if (grid <= 0) return FOVEA_EUNSUPPORTED;
    e = tca ? launch_tca_adjoint(src, ctx->ws, rbound, grid, s) : launch_adjoint(src, ctx->ws, rbound, grid, s);
  } else {
    int grid = forward_grid(ctx, cfg, rbound, fmt_mask, tc_c, all_tma);
    if (grid <= 0) return FOVEA_EUNSUPPORTED;
    switch (tc_kind(cfg, fmt_mask, tc_c, rbound, all_tma)) {
      case 4:
        e = launch_tcf_forward(src, ctx->ws, rbound, tc_c, grid, s, BucketList{nullptr, 0, 0}, false, nullptr);
        break;
      case 3:
        e = launch_tc05_forward(src, ctx->ws, cfg, rbound, grid, s, BucketList{nullptr, 0, 0}, false, nullptr);
        break;
      case 2:
        e = launch_umma_forward(src, ctx->ws, cfg, rbound, tc_c, grid, s, BucketList{nullptr, 0, 0}, false, nullptr);
        break;
      case 1:
        e = launch_tc_forward(src, ctx->ws, cfg, rbound, tc_c, grid, s, BucketList{nullptr, 0, 0}, false, nullptr);
        break;
      default:
        e = launch_forward(src, ctx->ws, cfg, rbound, fmt_mask, grid, s);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

// The configuration a batch runs with: the context's own after
// fovea_set_config, else the one fovea_autotune_batch chose for batches of
// this kind (see batch_tune_key), else the context's default.
FwdConfig batch_config(fovea_ctx* ctx, const fovea_frame* frames, int n, bool adjoint) {
  if (ctx->cfg_explicit || adjoint || n <= 0 || !frames) return ctx->cfg;
  BatchSummary bs;
  if (summarize_batch(ctx, frames, n, &bs) != FOVEA_OK) return ctx->cfg;
  fovea_config c;
  return lookup_batch_config(ctx, bs, &c) ? to_fwd(c) : ctx->cfg;
}

int run_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, bool adjoint, cudaStream_t s,
              const FwdConfig* forced = nullptr) {
  const FwdConfig cfg = forced ? *forced : batch_config(ctx, frames, n, adjoint);
  long long total = 0;
  int rmax = 0;
  int fmt_mask = 0, tc_c = 0;
  bool all_tma = true;
  int st = upload_batch(ctx, cfg, frames, n, adjoint, s, &total, &rmax, &fmt_mask, &tc_c, &all_tma);
  if (st != FOVEA_OK) return st;
  // Radius bound of the graph: next multiple of 64 (shared-memory size of
  // the persistent kernel depends on it).
  const int rbound = std::min(kMaxRadius, ((rmax + 63) / 64) * 64);
  const auto key = std::make_pair((long long)((adjoint ? 1 : 0) + 2 * fmt_mask + 8 * tc_c + 64 * (all_tma ? 1 : 0)) *
                                      2048 + rbound,
                                  config_code(cfg));
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (!ctx->capture_stream) FOVEA_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    FOVEA_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue_batch_kernels(ctx, cfg, adjoint, rbound, fmt_mask, tc_c, all_tma, ctx->capture_stream);
    cudaError_t ee = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (st != FOVEA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ee != cudaSuccess) return cuda_fail(ee);
    cudaGraphExec_t ex = nullptr;
    ee = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ee != cudaSuccess) return cuda_fail(ee);
    it = ctx->graphs.emplace(key, ex).first;
  }
  FOVEA_CUDA(cudaGraphLaunch(it->second, s));
  return FOVEA_OK;
}

}  // namespace

extern "C" {

int fovea_create(int width, int height, int channels, int block, const fovea_sigma_law* law, int format,
                 fovea_ctx** out) {
  if (!out || !law) return FOVEA_EINVAL;
  *out = nullptr;
  FrameLaw fl;
  fl.grid = law->grid;
  if (fl.grid != FOVEA_GRID_ANCHORED && fl.grid != FOVEA_GRID_CENTRED) return FOVEA_EINVAL;
  switch (law->kind) {
    case FOVEA_LAW_LINEAR:
      if (!finite_nonneg(law->sigma0) || !finite_nonneg(law->k)) return FOVEA_EINVAL;
      fl.sigma0 = law->sigma0;
      fl.k = law->k;
      break;
    case FOVEA_LAW_GEISLER_PERRY: {
      if (width <= 0 || height <= 0) return FOVEA_EINVAL;  // the law depends on the frame diagonal
      const int st = fovea_gp_law(width, height, law->e_corner_deg, &fl.sigma0, &fl.k);
      if (st != FOVEA_OK) return st;
      break;
    }
    case FOVEA_LAW_MAP:
      if (!law->sigma_map || !finite_nonneg(law->sigma_map_max)) return FOVEA_EINVAL;
      fl.smap = law->sigma_map;
      fl.smap_max = law->sigma_map_max;
      break;
    default:
      return FOVEA_EINVAL;
  }
  if (block <= 0) return FOVEA_EINVAL;
  if (block > kMaxBlock || (block > 32 && block % 32 != 0)) return FOVEA_EUNSUPPORTED;
  if (format != FOVEA_U8_HWC && format != FOVEA_F32_CHW) return FOVEA_EINVAL;
  const bool batch_only = width == 0 && height == 0;
  if (!batch_only) {
    if (width <= 0 || height <= 0) return FOVEA_EINVAL;
    if (channels < 1 || channels > 4) return FOVEA_EINVAL;
  }
  fovea_ctx* ctx = new (std::nothrow) fovea_ctx();
  if (!ctx) return FOVEA_ENOMEM;
  ctx->W = width; ctx->H = height; ctx->C = channels; ctx->B = block; ctx->fmt = format;
  ctx->law = fl;
  ctx->batch_only = batch_only;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e);
  }
  // work items are tiles of side min(B, 32); a shifted grid may start up to
  // B - 1 pixels before the frame
  const int tile = block <= 32 ? block : 32, shift = fl.grid == FOVEA_GRID_CENTRED ? block - 1 : 0;
  long long items = batch_only ? 1024
                               : (long long)((width + shift + tile - 1) / tile) * ((height + shift + tile - 1) / tile);
  int st = ensure_workspace(ctx, items);
  if (st != FOVEA_OK) {
    fovea_destroy(ctx);
    return st;
  }
  fovea_apply_cached_config(ctx);
  *out = ctx;
  return FOVEA_OK;
}

// The tensor map of a single frame at in_dev (the context's shape and
// format), from the context's two-entry cache; nullptr where TMA cannot load
// the frame's rows (as in batches, only device memory is loaded by TMA).
static const void* frame_tensor_map(fovea_ctx* ctx, const void* in_dev, int fmt_mask) {
  const int rows = fmt_mask == 1 ? ctx->cfg.rows_per_chunk : 16;
  for (const auto& m : ctx->maps)
    if (m.in == in_dev && m.rows == rows) return m.ok ? m.map : nullptr;
  auto& m = ctx->maps[ctx->map_next];
  ctx->map_next ^= 1;
  m.ok = in_device_memory(in_dev) &&
         (fmt_mask == 1 ? make_u8_tensor_map(m.map, in_dev, ctx->W, ctx->H, ctx->C, rows)
                        : make_f32_tensor_map(m.map, in_dev, ctx->W, ctx->H, ctx->C, rows));
  m.in = in_dev;
  m.rows = rows;
  return m.ok ? m.map : nullptr;
}

static int render_one(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                      cudaStream_t s) {
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  const size_t nb = frame_bytes(ctx->W, ctx->H, ctx->C, ctx->fmt);
  if (overlaps(in_dev, nb, out_dev, nb)) return FOVEA_EINVAL;
  FrameSource src;
  std::memset(&src, 0, sizeof(src));
  src.one = make_desc(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, in_dev, out_dev, fix_x, fix_y, ctx->law, 0);
  src.one_total = (long long)src.one.nbx * src.one.nby;
  const int rmax = radius_bound(ctx->W, ctx->H, ctx->B, fix_x, fix_y, ctx->law);
  const int fmt_mask = ctx->fmt == FOVEA_F32_CHW ? 2 : 1;
  const int tc_c = ctx->C;
  // A float32 frame that fits one wave of the fp32 kernel takes its
  // one-launch path (no sigma kernel) even with the tensor cores enabled.
  bool f32_one_wave = false;
  int grid = 0;
  if (fmt_mask == 2 && ctx->cfg.tc) {
    FwdConfig c0 = ctx->cfg;
    c0.tc = 0;
    grid = forward_grid(ctx, c0, rmax, fmt_mask, tc_c);
    f32_one_wave = grid > 0 && src.one_total <= grid;
  }
  // the tensor map of the frame's rows (the tensor-core kernels load rows by TMA where it exists)
  const void* map = ctx->cfg.tc && !f32_one_wave ? frame_tensor_map(ctx, src.one.in, fmt_mask) : nullptr;
  src.one.tma = map ? 1 : 0;
  if (!f32_one_wave) grid = forward_grid(ctx, ctx->cfg, rmax, fmt_mask, tc_c, src.one.tma != 0);
  if (grid <= 0) return FOVEA_EUNSUPPORTED;
  const int kind = tc_kind(ctx->cfg, fmt_mask, tc_c, rmax, src.one.tma != 0);
  if (kind == 0 && src.one_total <= grid) {
    // every block fits in one wave: one launch, one CTA per block, each
    // evaluating its own sigma (no sigma kernel, no work list)
    if (ctx->kev_start) FOVEA_CUDA(cudaEventRecord(ctx->kev_start, s));
    cudaError_t e = launch_forward_direct(src.one, src.one_total, ctx->ws, ctx->cfg, rmax, fmt_mask, s, !ctx->kev_start);
    if (e != cudaSuccess) return cuda_fail(e);
    if (ctx->kev_stop) FOVEA_CUDA(cudaEventRecord(ctx->kev_stop, s));
    return FOVEA_OK;
  }
  // no more persistent CTAs than items (small frames start fewer CTAs)
  grid = (int)std::min<long long>(grid, src.one_total);
  // Single frame: the sigma kernel also files every block under its radius
  // and the blur kernel orders its own work (largest radius first) from the
  // histogram, so no ordering kernel runs in between.
  const size_t need = (size_t)(rmax + 1) * (size_t)src.one_total;
  BucketList bl{nullptr, 0, 0};
  if (need <= ((size_t)64 << 20)) {
    if (ctx->blist_cap < need) {
      if (ctx->blist) {
        FOVEA_CUDA(cudaDeviceSynchronize());
        cudaFree(ctx->blist);
        ctx->blist = nullptr;
        ctx->blist_cap = 0;
      }
      FOVEA_CUDA(cudaMalloc(&ctx->blist, need * sizeof(int)));
      ctx->blist_cap = need;
    }
    bl = BucketList{ctx->blist, (int)src.one_total, rmax + 1};
  }
  const int sg = (int)std::min<long long>((src.one_total + sigma_threads() - 1) / sigma_threads(), 8ll * ctx->num_sms);
  cudaError_t e = bl.list ? launch_sigma_buckets(src, ctx->ws, std::max(sg, 1), bl, s)
                          : launch_sigma_order(src, ctx->ws, sigma_grid(src.one_total, ctx->num_sms), nullptr, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (ctx->kev_start) FOVEA_CUDA(cudaEventRecord(ctx->kev_start, s));
  // Programmatic dependent launch lets the blur kernel's prologue overlap the
  // sigma kernel (not when its launch is bracketed by timing events).
  const bool pdl = bl.list && !ctx->kev_start;
  if (kind) {
    e = kind == 4   ? launch_tcf_forward(src, ctx->ws, rmax, tc_c, grid, s, bl, pdl, map)
        : kind == 3 ? launch_tc05_forward(src, ctx->ws, ctx->cfg, rmax, grid, s, bl, pdl, map)
        : kind == 2 ? launch_umma_forward(src, ctx->ws, ctx->cfg, rmax, tc_c, grid, s, bl, pdl, map)
                    : launch_tc_forward(src, ctx->ws, ctx->cfg, rmax, tc_c, grid, s, bl, pdl, map);
  } else {
    e = launch_forward(src, ctx->ws, ctx->cfg, rmax, fmt_mask, grid, s, bl, pdl);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (ctx->kev_stop) FOVEA_CUDA(cudaEventRecord(ctx->kev_stop, s));
  return FOVEA_OK;
}

int fovea_render(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y, void* stream) {
  fovea::TraceRange trace("fovea_render");
  if (!ctx || !in_dev || !out_dev || ctx->batch_only) return FOVEA_EINVAL;
  ctx->caller_stream_used = true;
  return render_one(ctx, in_dev, out_dev, fix_x, fix_y, static_cast<cudaStream_t>(stream));
}

int fovea_render_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, void* stream) {
  fovea::TraceRange trace("fovea_render_batch");
  if (!ctx) return FOVEA_EINVAL;
  ctx->caller_stream_used = true;
  return run_batch(ctx, frames, n, false, static_cast<cudaStream_t>(stream));
}

int fovea_backward_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, void* stream) {
  fovea::TraceRange trace("fovea_backward_batch");
  if (!ctx) return FOVEA_EINVAL;
  ctx->caller_stream_used = true;
  return run_batch(ctx, frames, n, true, static_cast<cudaStream_t>(stream));
}

int fovea_render_host(fovea_ctx* ctx, const void* in_host, void* out_host, float fix_x, float fix_y,
                      void* stream) {
  fovea::TraceRange trace("fovea_render_host");
  if (!ctx || !in_host || !out_host || ctx->batch_only) return FOVEA_EINVAL;
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  const size_t nb = frame_bytes(ctx->W, ctx->H, ctx->C, ctx->fmt);
  if (overlaps(in_host, nb, out_host, nb)) return FOVEA_EINVAL;
  if (!ctx->s_h2d) {
    FOVEA_CUDA(cudaStreamCreateWithFlags(&ctx->s_h2d, cudaStreamNonBlocking));
    FOVEA_CUDA(cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking));
    FOVEA_CUDA(cudaStreamCreateWithFlags(&ctx->s_d2h, cudaStreamNonBlocking));
    FOVEA_CUDA(cudaEventCreateWithFlags(&ctx->ev_entry, cudaEventDisableTiming));
    for (auto& sl : ctx->hslot) {
      FOVEA_CUDA(cudaEventCreateWithFlags(&sl.ev_h2d, cudaEventDisableTiming));
      FOVEA_CUDA(cudaEventCreateWithFlags(&sl.ev_comp, cudaEventDisableTiming));
      FOVEA_CUDA(cudaEventCreateWithFlags(&sl.ev_d2h, cudaEventDisableTiming));
    }
  }
  if (ctx->host_io_bytes < nb) {
    FOVEA_CUDA(cudaDeviceSynchronize());
    for (auto& sl : ctx->hslot) {
      if (sl.in_dev) cudaFree(sl.in_dev);
      if (sl.out_dev) cudaFree(sl.out_dev);
      sl.in_dev = sl.out_dev = nullptr;
      sl.used = false;
    }
    ctx->host_io_bytes = 0;
    for (auto& sl : ctx->hslot) {
      FOVEA_CUDA(cudaMalloc(&sl.in_dev, nb));
      FOVEA_CUDA(cudaMalloc(&sl.out_dev, nb));
    }
    ctx->host_io_bytes = nb;
  }
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  if (ctx->caller_stream_used) {
    // earlier calls of this context on the caller's stream use the workspace
    FOVEA_CUDA(cudaEventRecord(ctx->ev_entry, caller));
    FOVEA_CUDA(cudaStreamWaitEvent(ctx->s_comp, ctx->ev_entry, 0));
    ctx->caller_stream_used = false;
  }
  auto& sl = ctx->hslot[ctx->hslot_next];
  ctx->hslot_next ^= 1;
  // H2D once the slot's previous kernel has read its input
  if (sl.used) FOVEA_CUDA(cudaStreamWaitEvent(ctx->s_h2d, sl.ev_comp, 0));
  FOVEA_CUDA(cudaMemcpyAsync(sl.in_dev, in_host, nb, cudaMemcpyHostToDevice, ctx->s_h2d));
  FOVEA_CUDA(cudaEventRecord(sl.ev_h2d, ctx->s_h2d));
  // kernels once the input is there and the slot's previous result is copied out
  FOVEA_CUDA(cudaStreamWaitEvent(ctx->s_comp, sl.ev_h2d, 0));
  if (sl.used) FOVEA_CUDA(cudaStreamWaitEvent(ctx->s_comp, sl.ev_d2h, 0));
  st = render_one(ctx, sl.in_dev, sl.out_dev, fix_x, fix_y, ctx->s_comp);
  if (st != FOVEA_OK) return st;
  FOVEA_CUDA(cudaEventRecord(sl.ev_comp, ctx->s_comp));
  FOVEA_CUDA(cudaStreamWaitEvent(ctx->s_d2h, sl.ev_comp, 0));
  FOVEA_CUDA(cudaMemcpyAsync(out_host, sl.out_dev, nb, cudaMemcpyDeviceToHost, ctx->s_d2h));
  FOVEA_CUDA(cudaEventRecord(sl.ev_d2h, ctx->s_d2h));
  sl.used = true;
  // the caller's stream completes this call's work (so later calls on it are
  // ordered after these kernels, and synchronising it means out_host is ready)
  FOVEA_CUDA(cudaStreamWaitEvent(caller, sl.ev_d2h, 0));
  return FOVEA_OK;
}

int fovea_backward(fovea_ctx* ctx, const float* grad_out_dev, float* grad_in_dev, float fix_x, float fix_y,
                   void* stream) {
  fovea::TraceRange trace("fovea_backward");
  if (!ctx || !grad_out_dev || !grad_in_dev || ctx->batch_only) return FOVEA_EINVAL;
  if (ctx->fmt != FOVEA_F32_CHW) return FOVEA_EINVAL;
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  const size_t nb = frame_bytes(ctx->W, ctx->H, ctx->C, ctx->fmt);
  if (overlaps(grad_out_dev, nb, grad_in_dev, nb)) return FOVEA_EINVAL;
  ctx->caller_stream_used = true;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FrameSource src;
  std::memset(&src, 0, sizeof(src));
  src.one = make_desc(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, grad_out_dev, grad_in_dev, fix_x, fix_y,
                      ctx->law, 0);
  src.one_total = (long long)src.one.nbx * src.one.nby;
  const int rmax = radius_bound(ctx->W, ctx->H, ctx->B, fix_x, fix_y, ctx->law);
  FOVEA_CUDA(cudaMemsetAsync(grad_in_dev, 0, nb, s));
  cudaError_t e = launch_sigma_order(src, ctx->ws, sigma_grid(src.one_total, ctx->num_sms), nullptr, nullptr, s);
  if (e != cudaSuccess) return cuda_fail(e);
  const bool tc = ctx->cfg.tc == 2;
  const int grid = adjoint_grid(ctx, rmax, tc);
  if (grid <= 0) return FOVEA_EUNSUPPORTED;
  e = tc ? launch_tca_adjoint(src, ctx->ws, rmax, grid, s) : launch_adjoint(src, ctx->ws, rmax, grid, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

int fovea_sigma_table(fovea_ctx* ctx, float fix_x, float fix_y, float* sigma_dev, int* radius_dev, void* stream) {
  fovea::TraceRange trace("fovea_sigma_table");
  if (!ctx || !sigma_dev || !radius_dev || ctx->batch_only) return FOVEA_EINVAL;
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  FrameSource src;
  std::memset(&src, 0, sizeof(src));
  src.one = make_desc(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, nullptr, nullptr, fix_x, fix_y, ctx->law, 0, true);
  src.one_total = (long long)src.one.nbx * src.one.nby;
  ctx->caller_stream_used = true;
  cudaError_t e = launch_sigma_order(src, ctx->ws, sigma_grid(src.one_total, ctx->num_sms), sigma_dev, radius_dev,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

namespace {

// Largest per-pixel radius of a W x H frame: the farthest pixel centre from
// the fixation is a corner pixel's; every step rounded on its own, as the
// device computes it.
int pixel_radius_bound(int W, int H, double fx, double fy, double sigma0, double k) {
  const int xs[2] = {0, W - 1}, ys[2] = {0, H - 1};
  int rmax = 0;
  for (int x : xs)
    for (int y : ys) {
      volatile double cx = (double)x + 0.5;
      volatile double cy = (double)y + 0.5;
      volatile double dx = cx - fx;
      volatile double dy = cy - fy;
      volatile double dx2 = dx * dx;
      volatile double dy2 = dy * dy;
      volatile double e = std::sqrt(dx2 + dy2);
      volatile double ke = k * e;
      volatile double sg = sigma0 + ke;
      volatile double s3 = 3.0 * sg;
      const double rc = std::ceil(s3);
      rmax = std::max(rmax, rc > 1e9 ? 1000000000 : (int)rc);
    }
  return rmax;
}

}  // namespace

int fovea_render_pixelwise(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                           void* stream) {
  fovea::TraceRange trace("fovea_render_pixelwise");
  if (!ctx || !in_dev || !out_dev || ctx->batch_only) return FOVEA_EINVAL;
  if (ctx->law.smap) return FOVEA_EINVAL;  // a per-block map gives no per-pixel law
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  const size_t nb = frame_bytes(ctx->W, ctx->H, ctx->C, ctx->fmt);
  if (overlaps(in_dev, nb, out_dev, nb)) return FOVEA_EINVAL;
  const int rmax = pixel_radius_bound(ctx->W, ctx->H, fix_x, fix_y, ctx->law.sigma0, ctx->law.k);
  if (rmax > kPixelMaxRadius) return FOVEA_EUNSUPPORTED;
  const bool isu8 = ctx->fmt == FOVEA_U8_HWC;
  const bool tc = isu8 && ctx->cfg.tc != 0 && pixel_tc_fits(rmax, ctx->C);
  if (!tc && pixel_fp32_rows(rmax, ctx->C) <= 0) return FOVEA_EUNSUPPORTED;
  ctx->caller_stream_used = true;
  PixelParams pp;
  pp.in = in_dev;
  pp.out = out_dev;
  pp.W = ctx->W; pp.H = ctx->H; pp.C = ctx->C; pp.isu8 = isu8 ? 1 : 0;
  pp.fx = fix_x; pp.fy = fix_y; pp.sigma0 = ctx->law.sigma0; pp.k = ctx->law.k;
  pp.rmax = rmax;
  pp.words = ((size_t)ctx->W * ctx->C) % 4 == 0 && reinterpret_cast<uintptr_t>(in_dev) % 4 == 0;
  pp.err = ctx->ws.counters ? ctx->ws.counters + CNT_ERROR : nullptr;
  if (!pp.err) return FOVEA_EINVAL;
  cudaError_t e = launch_pixel_forward(pp, tc, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

int fovea_render_pyramid(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                         void* stream) {
  fovea::TraceRange trace("fovea_render_pyramid");
  if (!ctx || !in_dev || !out_dev || ctx->batch_only) return FOVEA_EINVAL;
  if (ctx->law.smap) return FOVEA_EINVAL;
  int st = check_frame(ctx->W, ctx->H, ctx->C, ctx->fmt, ctx->B, ctx->law, fix_x, fix_y);
  if (st != FOVEA_OK) return st;
  const size_t nb = frame_bytes(ctx->W, ctx->H, ctx->C, ctx->fmt);
  if (overlaps(in_dev, nb, out_dev, nb)) return FOVEA_EINVAL;
  // levels down to 1 x 1, of which those up to the largest fractional level
  // any pixel reads (the farthest corner pixel's sigma) are built
  PyramidLevels lv;
  std::memset(&lv, 0, sizeof(lv));
  lv.w[0] = ctx->W;
  lv.h[0] = ctx->H;
  int nl = 1;
  while ((lv.w[nl - 1] > 1 || lv.h[nl - 1] > 1) && nl < kMaxPyramidLevels) {
    lv.w[nl] = (lv.w[nl - 1] + 1) / 2;
    lv.h[nl] = (lv.h[nl - 1] + 1) / 2;
    ++nl;
  }
  double smax = 0.0;
  for (int x : {0, ctx->W - 1})
    for (int y : {0, ctx->H - 1}) {
      const double dx = (double)x + 0.5 - fix_x, dy = (double)y + 0.5 - fix_y;
      smax = std::max(smax, ctx->law.sigma0 + ctx->law.k * std::sqrt(dx * dx + dy * dy));
    }
  const double lmax = std::log(3.0 * smax * smax + 1.0) / std::log(4.0);
  lv.top = std::min(nl - 1, (int)std::ceil(lmax));
  size_t need = 0;
  for (int l = 1; l <= lv.top; ++l) need += (size_t)lv.w[l] * lv.h[l] * ctx->C * sizeof(float);
  if (need > ctx->pyr_bytes) {
    if (ctx->pyr) {
      FOVEA_CUDA(cudaDeviceSynchronize());
      cudaFree(ctx->pyr);
      ctx->pyr = nullptr;
      ctx->pyr_bytes = 0;
    }
    FOVEA_CUDA(cudaMalloc(&ctx->pyr, need));
    ctx->pyr_bytes = need;
  }
  size_t off = 0;
  for (int l = 1; l <= lv.top; ++l) {
    lv.ptr[l] = ctx->pyr + off / sizeof(float);
    off += (size_t)lv.w[l] * lv.h[l] * ctx->C * sizeof(float);
  }
  ctx->caller_stream_used = true;
  cudaError_t e = launch_pyramid(in_dev, out_dev, ctx->W, ctx->H, ctx->C, ctx->fmt == FOVEA_U8_HWC ? 1 : 0, fix_x,
                                 fix_y, (float)ctx->law.sigma0, (float)ctx->law.k, lv,
                                 static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

int fovea_ssim(int width, int height, int channels, int format, const void* a_dev, const void* b_dev,
               double data_range, float* map_dev, double* sum_dev, void* stream) {
  fovea::TraceRange trace("fovea_ssim");
  if (!a_dev || !b_dev || width <= 0 || height <= 0) return FOVEA_EINVAL;
  if (channels < 1 || channels > 4) return FOVEA_EINVAL;
  if (format != FOVEA_U8_HWC && format != FOVEA_F32_CHW) return FOVEA_EINVAL;
  if (!map_dev && !sum_dev) return FOVEA_EINVAL;
  if ((long long)width * height * channels > (1ll << 31) - 1) return FOVEA_EUNSUPPORTED;
  double L = data_range;
  if (L <= 0.0) L = format == FOVEA_U8_HWC ? 255.0 : 1.0;
  if (!std::isfinite(L)) return FOVEA_EINVAL;
  cudaError_t e = launch_ssim(a_dev, b_dev, width, height, channels, format == FOVEA_U8_HWC ? 1 : 0, (float)L,
                              map_dev, sum_dev, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return FOVEA_OK;
}

int fovea_gp_law(int width, int height, double e_corner_deg, double* sigma0, double* k) {
  if (width <= 0 || height <= 0 || !sigma0 || !k || !finite_nonneg(e_corner_deg)) return FOVEA_EINVAL;
  const double e2 = 2.3;
  volatile double w2 = (double)width * (double)width;
  volatile double h2 = (double)height * (double)height;
  volatile double d_corner = 0.5 * std::sqrt(w2 + h2);
  volatile double pe2 = kPi * e2;
  *sigma0 = 1.0 / kPi;
  *k = e_corner_deg / (pe2 * d_corner);
  return FOVEA_OK;
}

int fovea_grid(const fovea_ctx* ctx, float fix_x, float fix_y, int* nbx, int* nby, int* ox, int* oy) {
  if (!ctx || !nbx || !nby || !ox || !oy || ctx->batch_only) return FOVEA_EINVAL;
  if (!std::isfinite(fix_x) || !std::isfinite(fix_y)) return FOVEA_EINVAL;
  *ox = grid_origin(fix_x, ctx->B, ctx->law.grid);
  *oy = grid_origin(fix_y, ctx->B, ctx->law.grid);
  grid_dims(ctx->W, ctx->H, ctx->B, *ox, *oy, nbx, nby);
  return FOVEA_OK;
}

int fovea_get_config(const fovea_ctx* ctx, fovea_config* cfg) {
  if (!ctx || !cfg) return FOVEA_EINVAL;
  cfg->threads = ctx->cfg.threads;
  cfg->ctas_per_sm = ctx->cfg.ctas_per_sm;
  cfg->rows_per_chunk = ctx->cfg.rows_per_chunk;
  cfg->tensor_cores = ctx->cfg.tc;
  return FOVEA_OK;
}

int fovea_set_config(fovea_ctx* ctx, const fovea_config* cfg) {
  if (!ctx || !cfg) return FOVEA_EINVAL;
  const int st = fovea::apply_config(ctx, cfg);
  if (st == FOVEA_OK) ctx->cfg_explicit = true;
  return st;
}

int fovea_reserve(fovea_ctx* ctx, int max_frames, long long max_items) {
  if (!ctx || max_frames < 0 || max_items < 0 || max_frames > (1 << 24) || max_items > (1ll << 31) - 1)
    return FOVEA_EINVAL;
  if (max_items > 0) {
    int st = ensure_workspace(ctx, max_items);
    if (st != FOVEA_OK) return st;
  }
  if (max_frames > 0) {
    int st = ensure_batch_tables(ctx, batch_table_bytes(max_frames));
    if (st != FOVEA_OK) return st;
  }
  return FOVEA_OK;
}

int fovea_set_kernel_events(fovea_ctx* ctx, void* ev_start, void* ev_stop) {
  if (!ctx || (ev_start == nullptr) != (ev_stop == nullptr)) return FOVEA_EINVAL;
  ctx->kev_start = static_cast<cudaEvent_t>(ev_start);
  ctx->kev_stop = static_cast<cudaEvent_t>(ev_stop);
  return FOVEA_OK;
}

void fovea_destroy(fovea_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  cudaFree(ctx->ws.items);
  cudaFree(ctx->ws.rank);
  cudaFree(ctx->ws.order);
  cudaFree(ctx->ws.counters);
  cudaFree(ctx->batch_dev);
  for (int i = 0; i < kBatchSlots; ++i) {
    if (ctx->batch_host[i]) cudaFreeHost(ctx->batch_host[i]);
    if (ctx->batch_ev[i]) cudaEventDestroy(ctx->batch_ev[i]);
  }
  for (auto& sl : ctx->hslot) {
    if (sl.in_dev) cudaFree(sl.in_dev);
    if (sl.out_dev) cudaFree(sl.out_dev);
    if (sl.ev_h2d) cudaEventDestroy(sl.ev_h2d);
    if (sl.ev_comp) cudaEventDestroy(sl.ev_comp);
    if (sl.ev_d2h) cudaEventDestroy(sl.ev_d2h);
  }
  if (ctx->pyr) cudaFree(ctx->pyr);
  for (void* p : ctx->retired_dev) cudaFree(p);
  for (void* p : ctx->retired_host) cudaFreeHost(p);
  if (ctx->ev_entry) cudaEventDestroy(ctx->ev_entry);
  if (ctx->s_h2d) cudaStreamDestroy(ctx->s_h2d);
  if (ctx->s_comp) cudaStreamDestroy(ctx->s_comp);
  if (ctx->s_d2h) cudaStreamDestroy(ctx->s_d2h);
  cudaFree(ctx->blist);
  if (ctx->fault_host) cudaFreeHost(ctx->fault_host);
  if (ctx->fault_ev) cudaEventDestroy(ctx->fault_ev);
  delete ctx;
}

int fovea_check(fovea_ctx* ctx, void* stream, unsigned int* faults) {
  if (faults) *faults = 0u;
  if (!ctx || !ctx->ws.counters) return FOVEA_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int word = 0u;
  FOVEA_CUDA(cudaMemcpyAsync(&word, ctx->ws.counters + CNT_ERROR, sizeof(word), cudaMemcpyDeviceToHost, s));
  FOVEA_CUDA(cudaStreamSynchronize(s));
  if (word) {
    FOVEA_CUDA(cudaMemsetAsync(ctx->ws.counters + CNT_ERROR, 0, sizeof(unsigned int), s));
    FOVEA_CUDA(cudaStreamSynchronize(s));
  }
  if (faults) *faults = word;
  return fault_status(word);
}

int fovea_check_async(fovea_ctx* ctx, void* stream, unsigned int* faults) {
  if (faults) *faults = 0u;
  if (!ctx || !ctx->ws.counters) return FOVEA_EINVAL;
  if (!ctx->fault_host) {
    FOVEA_CUDA(cudaHostAlloc(&ctx->fault_host, sizeof(unsigned int), cudaHostAllocDefault));
    *ctx->fault_host = 0u;
    FOVEA_CUDA(cudaEventCreateWithFlags(&ctx->fault_ev, cudaEventDisableTiming));
  }
  if (ctx->fault_copy_pending) {
    const cudaError_t q = cudaEventQuery(ctx->fault_ev);
    if (q == cudaErrorNotReady) return FOVEA_OK;  // the last copy is still on its way: nothing new to report
    if (q != cudaSuccess) return cuda_fail(q);
    ctx->fault_copy_pending = false;
    if (*ctx->fault_host) return fovea_check(ctx, stream, faults);  // the word is sticky: read and clear it
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FOVEA_CUDA(cudaMemcpyAsync(ctx->fault_host, ctx->ws.counters + CNT_ERROR, sizeof(unsigned int),
                             cudaMemcpyDeviceToHost, s));
  FOVEA_CUDA(cudaEventRecord(ctx->fault_ev, s));
  ctx->fault_copy_pending = true;
  return FOVEA_OK;
}

const char* fovea_strerror(int status) {
  switch (status) {
    case FOVEA_OK: return "ok";
    case FOVEA_EINVAL: return "invalid argument";
    case FOVEA_ENOMEM: return "out of memory";
    case FOVEA_ECUDA: return "CUDA error";
    case FOVEA_EBUSY: return "busy";
    case FOVEA_ETIMEOUT: return "timed out";
    case FOVEA_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int fovea_last_cuda_error(void) { return g_last_cuda_error; }

int fovea_build_flags(void) {
#if defined(FOVEA_BOUNDS)
  return FOVEA_BUILD_BOUNDS;
#else
  return 0;
#endif
}

}  // extern "C"

// ---------------------------------------------------------------- internals used by other units
namespace fovea {

int ctx_shape(const fovea_ctx* ctx, int* W, int* H, int* C, int* fmt, int* B) {
  *W = ctx->W; *H = ctx->H; *C = ctx->C; *fmt = ctx->fmt; *B = ctx->B;
  return ctx->batch_only ? FOVEA_EINVAL : FOVEA_OK;
}

int ctx_centre_radius_bound(const fovea_ctx* ctx) {
  if (ctx->batch_only || ctx->W <= 0 || ctx->H <= 0) return 0;
  return radius_bound(ctx->W, ctx->H, ctx->B, 0.5f * (float)ctx->W, 0.5f * (float)ctx->H, ctx->law);
}

int check_config(const fovea_config* cfg) {
  if (cfg->threads != 128 && cfg->threads != 256 && cfg->threads != 512) return FOVEA_EUNSUPPORTED;
  if (cfg->rows_per_chunk != 16 && cfg->rows_per_chunk != 32 && cfg->rows_per_chunk != 64) return FOVEA_EUNSUPPORTED;
  if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 8) return FOVEA_EINVAL;
  if (cfg->tensor_cores < 0 || cfg->tensor_cores > 3) return FOVEA_EINVAL;
  return FOVEA_OK;
}

int apply_config(fovea_ctx* ctx, const fovea_config* cfg) {
  const int st = check_config(cfg);
  if (st != FOVEA_OK) return st;
  ctx->cfg = to_fwd(*cfg);  // batch graphs are keyed by configuration: nothing to drop
  return FOVEA_OK;
}

int summarize_batch(const fovea_ctx* ctx, const fovea_frame* frames, int n, BatchSummary* out) {
  if (!ctx || !frames || n <= 0 || !out) return FOVEA_EINVAL;
  BatchSummary bs{0, -1, 0, 0, n};
  for (int i = 0; i < n; ++i) {
    const fovea_frame& f = frames[i];
    if (f.width <= 0 || f.height <= 0 || f.channels < 1 || f.channels > 4) return FOVEA_EINVAL;
    if (!std::isfinite(f.fix_x) || !std::isfinite(f.fix_y)) return FOVEA_EINVAL;
    bs.fmt_mask |= f.format == FOVEA_F32_CHW ? 2 : 1;
    bs.channels = bs.channels == -1 ? f.channels : (bs.channels == f.channels ? bs.channels : 0);
    bs.rmax = std::max(bs.rmax, radius_bound(f.width, f.height, ctx->B, f.fix_x, f.fix_y, law_of(f)));
    bs.blocks += (long long)((f.width + ctx->B - 1) / ctx->B) * ((f.height + ctx->B - 1) / ctx->B);
  }
  *out = bs;
  return FOVEA_OK;
}

int render_batch_with(fovea_ctx* ctx, const fovea_frame* frames, int n, const fovea_config* cfg, void* stream) {
  if (!ctx || !cfg) return FOVEA_EINVAL;
  const int st = check_config(cfg);
  if (st != FOVEA_OK) return st;
  const FwdConfig c = to_fwd(*cfg);
  ctx->caller_stream_used = true;
  return run_batch(ctx, frames, n, false, static_cast<cudaStream_t>(stream), &c);
}

int ctx_fault_word(const fovea_ctx* ctx, unsigned int** word) {
  if (!ctx->ws.counters) return FOVEA_EINVAL;
  *word = ctx->ws.counters + CNT_ERROR;
  return FOVEA_OK;
}

int ctx_device_info(const fovea_ctx* ctx, int* device, int* num_sms) {
  *device = ctx->device;
  *num_sms = ctx->num_sms;
  return FOVEA_OK;
}

int record_cuda_failure(int cuda_error) { return cuda_fail((cudaError_t)cuda_error); }

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cudaGetLastError();
  });
  return encode;
}

// Float32 CHW frame as a 3D tensor (x, y, channel plane): boxes of 32
// elements (128 bytes, 128-byte swizzle) x `rows` rows of one plane, zero
// outside the frame, so a row above or below a plane reads zeros (never the
// neighbouring plane). Needs a 16-byte aligned base and W a multiple of 4.
bool make_f32_tensor_map(void* map, const void* base, int W, int H, int C, int rows) {
  std::memset(map, 0, kTensorMapBytes);
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  const unsigned long long pitch = (unsigned long long)W * 4ull;
  if (!encode || !base || ((uintptr_t)base & 15) || (pitch & 15) || W <= 0 || H <= 0 || C <= 0 || rows <= 0 ||
      rows > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)C};
  const cuuint64_t strides[2] = {pitch, pitch * (cuuint64_t)H};
  const cuuint32_t box[3] = {32, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::memset(map, 0, kTensorMapBytes);
    return false;
  }
  return true;
}

bool make_u8_tensor_map(void* map, const void* base, int W, int H, int C, int rows) {
  std::memset(map, 0, kTensorMapBytes);
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  const unsigned long long pitch = (unsigned long long)W * (unsigned long long)C;
  if (!encode || !base || ((uintptr_t)base & 15) || (pitch & 15) || W <= 0 || H <= 0 || rows <= 0 || rows > 256)
    return false;
  const cuuint64_t dims[2] = {pitch, (cuuint64_t)H};
  const cuuint64_t strides[1] = {pitch};
  const cuuint32_t box[2] = {128, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base),
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::memset(map, 0, kTensorMapBytes);
    return false;
  }
  return true;
}

}  // namespace fovea
