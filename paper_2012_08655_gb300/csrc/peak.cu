// FP32 FMA throughput probe: the roof against which the blur kernels'
// arithmetic is reported. Each thread runs kChains independent packed
// two-lane FMA chains (fma.rn.f32x2, the instruction the FP32 blur kernel's
// inner loops use), so the FMA pipe, not a dependency, sets the rate.
#include <cuda_runtime.h>

#include "fovea_host.h"
#include "fovea_internal.cuh"

using namespace fovea;

namespace {

constexpr int kChains = 16;
constexpr int kIters = 2048;
constexpr int kThreadsPerCta = 256;
constexpr int kCtasPerSm = 8;

__global__ void __launch_bounds__(kThreadsPerCta) fma_rate_kernel(float* out, float seed) {
  float2 acc[kChains];
  #pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = make_float2(seed + i, seed - i);
  const float2 m = make_float2(0.999f, 1.001f), a = make_float2(seed * 1e-3f, -seed * 1e-3f);
  for (int it = 0; it < kIters; ++it) {
    #pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = ffma2(acc[i], m, a);
  }
  float s = 0.f;
  #pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i].x + acc[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int fovea_measure_fma_rate(double* fma_per_s, void* stream) {
  if (!fma_per_s) return FOVEA_EINVAL;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return record_cuda_failure(e);
  const int grid = sms * kCtasPerSm;
  float* out = nullptr;
  e = cudaMalloc(&out, (size_t)grid * kThreadsPerCta * sizeof(float));
  if (e != cudaSuccess) return record_cuda_failure(e);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = FOVEA_OK;
  float ms = 0.f;
  const int reps = 10;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    st = record_cuda_failure(e);
  } else {
    for (int w = 0; w < 3; ++w) fma_rate_kernel<<<grid, kThreadsPerCta, 0, s>>>(out, 1.0f + w);
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) fma_rate_kernel<<<grid, kThreadsPerCta, 0, s>>>(out, 2.0f + i);
    cudaEventRecord(e1, s);
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms <= 0.f) e = cudaErrorUnknown;
    if (e != cudaSuccess) st = record_cuda_failure(e);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != FOVEA_OK) return st;
  const double lanes = (double)grid * kThreadsPerCta * kChains * 2.0 * kIters * reps;
  *fma_per_s = lanes / (ms * 1e-3);
  return FOVEA_OK;
}
