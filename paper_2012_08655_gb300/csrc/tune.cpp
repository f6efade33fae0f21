// Autotuner of the forward kernel configuration (not in the paper, which
// fixes one CUDA block per fragment and 32 x 32 fragments of one thread
// layout).
//
// Candidates: the kernel (fp32 FMA; tensor cores on mma.sync with 128, 256
// or 512 threads per CTA, whose staged tile is a row chunk of 112, 240 or
// 496 bytes of the halo rows; tensor cores with the vertical pass on
// tcgen05) and the rows staged per chunk (16, 32, 64), each with as many
// persistent CTAs per SM as fit; then, for the fastest, 1 and 2 CTAs per SM.
// Each is timed with CUDA events and the fastest is kept in a process-wide
// cache, which can be persisted as a small JSON file (one entry per line).
//  - fovea_autotune times a synthetic frame of the context's own shape
//    (fixation at the centre) and keys its choice by device name, SM count,
//    frame shape, format, block side and radius bucket (the radius bound at
//    that fixation rounded up to a multiple of 64).
//  - fovea_autotune_batch times the caller's own batch and keys its choice by
//    device, SM count, block side, formats and channel count of the frames,
//    the largest radius (bucket of 64) and the numbers of blocks and frames
//    (powers of two); fovea_render_batch then uses the configuration chosen
//    for batches with the same key.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "fovea.h"
#include "fovea_host.h"

namespace {

struct Choice {
  fovea_config cfg;
  double ms;
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;
std::map<int, std::string> g_dev_names;  // device -> "name|SMs" (looked up once)

std::string device_tag(const fovea_ctx* ctx) {
  int dev, sms;
  fovea::ctx_device_info(ctx, &dev, &sms);
  auto it = g_dev_names.find(dev);
  if (it != g_dev_names.end()) return it->second;
  cudaDeviceProp p;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
  else cudaGetLastError();
  std::ostringstream os;
  os << name << "|" << sms;
  return g_dev_names[dev] = os.str();
}

// Key of a sized context (caller holds g_mu).
std::string frame_key(const fovea_ctx* ctx) {
  int W, H, C, fmt, B;
  fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B);
  const int rbucket = (fovea::ctx_centre_radius_bound(ctx) + 63) / 64 * 64;
  std::ostringstream os;
  os << device_tag(ctx) << "|" << W << "x" << H << "x" << C << "|f" << fmt << "|b" << B << "|r" << rbucket;
  return os.str();
}

int log2_bucket(long long v) {
  int b = 0;
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b;
}

// Key of a batch (caller holds g_mu).
std::string batch_key(const fovea_ctx* ctx, const fovea::BatchSummary& bs) {
  int W, H, C, fmt, B;
  fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B);
  std::ostringstream os;
  os << device_tag(ctx) << "|batch|b" << B << "|f" << bs.fmt_mask << "|c" << bs.channels << "|r"
     << (bs.rmax + 63) / 64 * 64 << "|i" << log2_bucket(bs.blocks) << "|n" << log2_bucket(bs.frames);
  return os.str();
}

void load_file(const char* path) {
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    // "key": {"threads": T, "ctas_per_sm": N, "rows_per_chunk": R, "tensor_cores": K, "ms": M},
    size_t a = line.find('"');
    size_t b = a == std::string::npos ? a : line.find('"', a + 1);
    if (b == std::string::npos) continue;
    std::string key = line.substr(a + 1, b - a - 1);
    Choice c{};
    if (std::sscanf(line.c_str() + b + 1,
                    ": {\"threads\": %d, \"ctas_per_sm\": %d, \"rows_per_chunk\": %d, \"tensor_cores\": %d, "
                    "\"ms\": %lf",
                    &c.cfg.threads, &c.cfg.ctas_per_sm, &c.cfg.rows_per_chunk, &c.cfg.tensor_cores, &c.ms) == 5 &&
        fovea::check_config(&c.cfg) == FOVEA_OK)
      g_cache[key] = c;
  }
}

void save_file(const char* path) {
  std::ofstream f(path, std::ios::trunc);
  f << "{\n";
  size_t i = 0;
  for (const auto& kv : g_cache) {
    const fovea_config& c = kv.second.cfg;
    f << "  \"" << kv.first << "\": {\"threads\": " << c.threads << ", \"ctas_per_sm\": " << c.ctas_per_sm
      << ", \"rows_per_chunk\": " << c.rows_per_chunk << ", \"tensor_cores\": " << c.tensor_cores
      << ", \"ms\": " << kv.second.ms << "}"
      << (++i < g_cache.size() ? ",\n" : "\n");
  }
  f << "}\n";
}

// Candidate configurations for frames of the given formats (fmt_mask bit 0
// uint8, bit 1 float32) and channel count (0: mixed): the uint8 tensor-core
// kernels serve launches whose frames are all uint8 with one channel count,
// the float32 one (16-row chunks whatever rows_per_chunk says) launches whose
// frames are all float32.
std::vector<fovea_config> candidates(int fmt_mask, int channels) {
  std::vector<fovea_config> v;
  const int rbs[3] = {16, 32, 64};
  for (int rb : rbs) v.push_back(fovea_config{256, 0, rb, 0});
  if (fmt_mask == 2) v.push_back(fovea_config{256, 0, 16, 1});
  if (fmt_mask == 1 && channels > 0) {
    for (int nt : {128, 256, 512})
      for (int rb : rbs) v.push_back(fovea_config{nt, 0, rb, 1});
    for (int rb : {16, 32}) v.push_back(fovea_config{256, 0, rb, 2});
    if (channels == 3)
      v.push_back(fovea_config{256, 0, 16, 3});
  }
  return v;
}

// Times `run` (a launch sequence on stream s) for every candidate, then the
// best with 1 and 2 CTAs per SM; returns the fastest (ms < 0: none ran).
template <typename Run>
Choice search(const std::vector<fovea_config>& cands, int iters, cudaStream_t s, Run&& run, int* status) {
  Choice best{fovea_config{256, 0, 32, 1}, -1.0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    *status = FOVEA_ENOMEM;
    cudaGetLastError();
  }
  auto time_one = [&](const fovea_config& c) {
    int st = run(c);  // warm-up (and graph capture for batches)
    if (st != FOVEA_OK) return;  // configuration does not fit: skip it
    cudaEventRecord(e0, s);
    for (int i = 0; i < iters && st == FOVEA_OK; ++i) st = run(c);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *status = FOVEA_ECUDA;
      return;
    }
    if (st != FOVEA_OK) return;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / iters;
    if (best.ms < 0 || per < best.ms) best = Choice{c, per};
  };
  for (const fovea_config& c : cands) {
    if (*status != FOVEA_OK) break;
    time_one(c);
  }
  if (*status == FOVEA_OK && best.ms >= 0) {
    const fovea_config base = best.cfg;
    for (int n : {1, 2}) {
      fovea_config c = base;
      c.ctas_per_sm = n;
      if (*status == FOVEA_OK) time_one(c);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return best;
}

}  // namespace

void fovea_apply_cached_config(fovea_ctx* ctx) {
  int W, H, C, fmt, B;
  if (fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B) != FOVEA_OK) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(frame_key(ctx));
  if (it == g_cache.end()) return;
  fovea::apply_config(ctx, &it->second.cfg);
}

namespace fovea {

bool lookup_batch_config(const fovea_ctx* ctx, const BatchSummary& bs, fovea_config* cfg) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_cache.empty()) return false;
  auto it = g_cache.find(batch_key(ctx, bs));
  if (it == g_cache.end()) return false;
  *cfg = it->second.cfg;
  return true;
}

}  // namespace fovea

extern "C" int fovea_autotune(fovea_ctx* ctx, int iters, const char* cache_path) {
  fovea::TraceRange trace("fovea_autotune");
  if (!ctx || iters <= 0) return FOVEA_EINVAL;
  int W, H, C, fmt, B;
  if (fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B) != FOVEA_OK) return FOVEA_EINVAL;
  std::string key;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    key = frame_key(ctx);
    if (cache_path) load_file(cache_path);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return fovea::apply_config(ctx, &it->second.cfg);
  }
  const size_t nb = fovea::frame_bytes(W, H, C, fmt);
  void* in = nullptr;
  void* out = nullptr;
  cudaStream_t s = nullptr;
  int status = FOVEA_OK;
  fovea_config saved;
  fovea_get_config(ctx, &saved);
  if (cudaMalloc(&in, nb) != cudaSuccess || cudaMalloc(&out, nb) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    status = FOVEA_ENOMEM;
  }
  if (status == FOVEA_OK && cudaMemsetAsync(in, 0x5A, nb, s) != cudaSuccess) status = FOVEA_ECUDA;
  const float fx = 0.5f * (float)W, fy = 0.5f * (float)H;
  Choice best{saved, -1.0};
  if (status == FOVEA_OK) {
    best = search(candidates(fmt == FOVEA_U8_HWC ? 1 : 2, C), iters, s,
                  [&](const fovea_config& c) {
                    const int st = fovea::apply_config(ctx, &c);
                    return st != FOVEA_OK ? st : fovea_render(ctx, in, out, fx, fy, s);
                  },
                  &status);
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(in);
  cudaFree(out);
  cudaGetLastError();
  if (status != FOVEA_OK || best.ms < 0) {
    fovea::apply_config(ctx, &saved);
    return status != FOVEA_OK ? status : FOVEA_EUNSUPPORTED;
  }
  fovea::apply_config(ctx, &best.cfg);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best;
  if (cache_path) save_file(cache_path);
  return FOVEA_OK;
}

extern "C" int fovea_autotune_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, int iters,
                                    const char* cache_path, fovea_config* chosen) {
  fovea::TraceRange trace("fovea_autotune_batch");
  if (!ctx || !frames || n <= 0 || iters <= 0) return FOVEA_EINVAL;
  fovea::BatchSummary bs;
  int status = fovea::summarize_batch(ctx, frames, n, &bs);
  if (status != FOVEA_OK) return status;
  std::string key;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    key = batch_key(ctx, bs);
    if (cache_path) load_file(cache_path);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      if (chosen) *chosen = it->second.cfg;
      return FOVEA_OK;
    }
  }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return FOVEA_ENOMEM;
  }
  // The timing runs write the caller's outputs (with the values any
  // configuration gives); they are ordered after the caller's earlier work
  // on the legacy stream only by the device synchronisation below.
  if (cudaDeviceSynchronize() != cudaSuccess) status = FOVEA_ECUDA;
  Choice best{fovea_config{256, 0, 32, 1}, -1.0};
  if (status == FOVEA_OK)
    best = search(candidates(bs.fmt_mask, bs.channels), iters, s,
                  [&](const fovea_config& c) { return fovea::render_batch_with(ctx, frames, n, &c, s); }, &status);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaGetLastError();
  if (status != FOVEA_OK) return status;
  if (best.ms < 0) return FOVEA_EUNSUPPORTED;
  if (chosen) *chosen = best.cfg;
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best;
  if (cache_path) save_file(cache_path);
  return FOVEA_OK;
}
