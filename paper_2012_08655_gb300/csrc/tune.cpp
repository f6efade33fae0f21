// Autotuner of the forward kernel configuration.
//
// Candidates: rows staged per chunk (16, 32, 64) x persistent CTAs per SM
// (1, 2, as many as fit). Each is timed with CUDA events on a synthetic frame
// of the context's own shape (fixation at the centre), and the fastest is
// kept in a process-wide cache keyed by device name, SM count, frame shape,
// format, block side and radius bucket (the radius bound at that fixation,
// rounded up to a multiple of 64: contexts of one shape whose sigma laws
// differ that much get their own choice); the cache can be persisted as a
// small JSON file (one entry per line).
#include <cuda_runtime.h>

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
  int rows_per_chunk;
  int ctas_per_sm;
  int tc;
  double ms;
};

std::mutex g_mu;
std::map<std::string, Choice> g_cache;

std::string make_key(const fovea_ctx* ctx) {
  int W, H, C, fmt, B, dev, sms;
  fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B);
  fovea::ctx_device_info(ctx, &dev, &sms);
  cudaDeviceProp p;
  std::string name = "unknown";
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) name = p.name;
  else cudaGetLastError();
  const int rbucket = (fovea::ctx_centre_radius_bound(ctx) + 63) / 64 * 64;
  std::ostringstream os;
  os << name << "|" << sms << "|" << W << "x" << H << "x" << C << "|f" << fmt << "|b" << B << "|r" << rbucket;
  return os.str();
}

void load_file(const char* path) {
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    // "key": {"rows_per_chunk": R, "ctas_per_sm": N, "tensor_cores": T, "ms": M},
    size_t a = line.find('"');
    size_t b = a == std::string::npos ? a : line.find('"', a + 1);
    if (b == std::string::npos) continue;
    std::string key = line.substr(a + 1, b - a - 1);
    Choice c{0, 0, 0, 0.0};
    if (std::sscanf(line.c_str() + b + 1, ": {\"rows_per_chunk\": %d, \"ctas_per_sm\": %d, \"tensor_cores\": %d, \"ms\": %lf",
                    &c.rows_per_chunk, &c.ctas_per_sm, &c.tc, &c.ms) == 4)
      g_cache[key] = c;
  }
}

void save_file(const char* path) {
  std::ofstream f(path, std::ios::trunc);
  f << "{\n";
  size_t i = 0;
  for (const auto& kv : g_cache) {
    f << "  \"" << kv.first << "\": {\"rows_per_chunk\": " << kv.second.rows_per_chunk
      << ", \"ctas_per_sm\": " << kv.second.ctas_per_sm << ", \"tensor_cores\": " << kv.second.tc
      << ", \"ms\": " << kv.second.ms << "}"
      << (++i < g_cache.size() ? ",\n" : "\n");
  }
  f << "}\n";
}

}  // namespace

void fovea_apply_cached_config(fovea_ctx* ctx) {
  int W, H, C, fmt, B;
  if (fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B) != FOVEA_OK) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(make_key(ctx));
  if (it == g_cache.end()) return;
  fovea_config cfg{256, it->second.ctas_per_sm, it->second.rows_per_chunk, it->second.tc};
  fovea_set_config(ctx, &cfg);
}

extern "C" int fovea_autotune(fovea_ctx* ctx, int iters, const char* cache_path) {
  if (!ctx || iters <= 0) return FOVEA_EINVAL;
  int W, H, C, fmt, B;
  if (fovea::ctx_shape(ctx, &W, &H, &C, &fmt, &B) != FOVEA_OK) return FOVEA_EINVAL;
  const std::string key = make_key(ctx);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cache_path) load_file(cache_path);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      fovea_config cfg{256, it->second.ctas_per_sm, it->second.rows_per_chunk, it->second.tc};
      return fovea_set_config(ctx, &cfg);
    }
  }
  const size_t nb = fovea::frame_bytes(W, H, C, fmt);
  void* in = nullptr;
  void* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = FOVEA_OK;
  Choice best{0, 0, 0, 1e30};
  fovea_config saved;
  fovea_get_config(ctx, &saved);
  if (cudaMalloc(&in, nb) != cudaSuccess || cudaMalloc(&out, nb) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    status = FOVEA_ENOMEM;
  }
  if (status == FOVEA_OK && cudaMemsetAsync(in, 0x5A, nb, s) != cudaSuccess) status = FOVEA_ECUDA;
  const float fx = 0.5f * (float)W, fy = 0.5f * (float)H;
  const int rbs[3] = {16, 32, 64};
  const int ctas[3] = {1, 2, 0};
  const int ntc = fmt == FOVEA_U8_HWC ? 3 : 1;
  for (int tcv = 0; tcv < ntc && status == FOVEA_OK; ++tcv)
  for (int a = 0; a < 3 && status == FOVEA_OK; ++a) {
    for (int b = 0; b < 3 && status == FOVEA_OK; ++b) {
      if (tcv == 2 && rbs[a] > 32) continue;  // the tcgen05 kernel stages 16 or 32 rows
      fovea_config cfg{256, ctas[b], rbs[a], tcv};
      if (fovea_set_config(ctx, &cfg) != FOVEA_OK) continue;
      int st = FOVEA_OK;
      for (int w = 0; w < 2 && st == FOVEA_OK; ++w) st = fovea_render(ctx, in, out, fx, fy, s);
      if (st != FOVEA_OK) continue;  // configuration does not fit: skip it
      cudaEventRecord(e0, s);
      for (int i = 0; i < iters && st == FOVEA_OK; ++i) st = fovea_render(ctx, in, out, fx, fy, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { status = FOVEA_ECUDA; break; }
      if (st != FOVEA_OK) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = (double)ms / iters;
      if (per < best.ms) best = Choice{rbs[a], ctas[b], tcv, per};
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(in);
  cudaFree(out);
  if (status != FOVEA_OK || best.rows_per_chunk == 0) {
    fovea_set_config(ctx, &saved);
    return status != FOVEA_OK ? status : FOVEA_EUNSUPPORTED;
  }
  fovea_config cfg{256, best.ctas_per_sm, best.rows_per_chunk, best.tc};
  fovea_set_config(ctx, &cfg);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best;
  if (cache_path) save_file(cache_path);
  return FOVEA_OK;
}
