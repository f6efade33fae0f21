// Gaussian-pyramid (mipmap) foveation: the earlier approach the paper
// compares its block-wise blur against (Section 3.2, Fig. 4, and its
// appendix on previous foveated rendering), here in CUDA instead of the
// graphics pipeline:
//
//  - a Burt-Adelson pyramid: level l+1 is level l convolved with the 5-tap
//    generating kernel (1, 4, 6, 4, 1) / 16 in each axis (clamp-to-edge) and
//    subsampled at the even indices, W_{l+1} = (W_l + 1) / 2;
//  - sample i of level l sits on original pixel 2^l i, and level l carries a
//    blur of variance (4^l - 1) / 3, so pixel p is read at the fractional
//    level L = log4(3 sigma_p^2 + 1) (sigma_p: the per-pixel law at the
//    pixel centre): bilinear interpolation in levels floor(L) and floor(L)+1
//    (neighbours clamped to the level), blended linearly by the fraction.
//
// pyramid_reduce_kernel builds one level (a CTA stages its 67 x 19 input
// footprint, filters horizontally into shared memory, then vertically);
// pyramid_sample_kernel writes the output, one thread per pixel. Levels
// above 0 are float32 planes in the context's workspace; level 0 is the
// frame itself.
#include "fovea_internal.cuh"

namespace fovea {
namespace {

constexpr int kRx = 32, kRy = 8;                         // outputs per reduce CTA
constexpr int kRinX = 2 * kRx + 3, kRinY = 2 * kRy + 3;  // its input footprint

__device__ __forceinline__ unsigned char quant8(float v) {
  int q = __float2int_rd(v + 0.5f);
  return (unsigned char)(q < 0 ? 0 : (q > 255 ? 255 : q));
}

template <int SRC>  // 0: uint8 HWC frame, 1: float32 CHW frame, 2: float32 level plane
__device__ __forceinline__ float level_at(const void* base, int W, int H, int C, int x, int y, int c) {
  if (SRC == 0) return (float)static_cast<const unsigned char*>(base)[((size_t)y * W + x) * C + c];
  if (SRC == 1) return static_cast<const float*>(base)[((size_t)c * H + y) * W + x];
  return static_cast<const float*>(base)[((size_t)c * H + y) * W + x];
}

template <int SRC>
__global__ void __launch_bounds__(kRx * kRy)
pyramid_reduce_kernel(const void* src, int W, int H, int C, float* dst, int W2, int H2) {
  __shared__ float sin[kRinY][kRinX + 1];
  __shared__ float sh[kRinY][kRx + 1];
  const float w[5] = {1.0f / 16.0f, 4.0f / 16.0f, 6.0f / 16.0f, 4.0f / 16.0f, 1.0f / 16.0f};
  const int tid = threadIdx.x, tx = tid % kRx, ty = tid / kRx;
  const int i0 = blockIdx.x * kRx, j0 = blockIdx.y * kRy, c = blockIdx.z;
  for (int idx = tid; idx < kRinY * kRinX; idx += kRx * kRy) {
    const int rr = idx / kRinX, cc = idx - rr * kRinX;
    const int y = min(max(2 * j0 - 2 + rr, 0), H - 1), x = min(max(2 * i0 - 2 + cc, 0), W - 1);
    sin[rr][cc] = level_at<SRC>(src, W, H, C, x, y, c);
  }
  __syncthreads();
  for (int idx = tid; idx < kRinY * kRx; idx += kRx * kRy) {
    const int rr = idx / kRx, cc = idx - rr * kRx;
    float a = 0.0f;
    #pragma unroll
    for (int m = 0; m < 5; ++m) a = fmaf(w[m], sin[rr][2 * cc + m], a);
    sh[rr][cc] = a;
  }
  __syncthreads();
  const int i = i0 + tx, j = j0 + ty;
  if (i >= W2 || j >= H2) return;
  float a = 0.0f;
  #pragma unroll
  for (int n = 0; n < 5; ++n) a = fmaf(w[n], sh[2 * ty + n][tx], a);
  dst[((size_t)c * H2 + j) * W2 + i] = a;
}

template <int SRC>
__device__ __forceinline__ float bilinear(const void* g, int Wl, int Hl, int C, int c, float u, float v) {
  const float fu0 = floorf(u), fv0 = floorf(v);
  const float fu = u - fu0, fv = v - fv0;
  int i0 = (int)fu0, j0 = (int)fv0;
  const int i1 = min(i0 + 1, Wl - 1), j1 = min(j0 + 1, Hl - 1);
  i0 = min(i0, Wl - 1);
  j0 = min(j0, Hl - 1);
  const float a = level_at<SRC>(g, Wl, Hl, C, i0, j0, c), b = level_at<SRC>(g, Wl, Hl, C, i1, j0, c);
  const float d = level_at<SRC>(g, Wl, Hl, C, i0, j1, c), e = level_at<SRC>(g, Wl, Hl, C, i1, j1, c);
  return (1.0f - fu) * (1.0f - fv) * a + fu * (1.0f - fv) * b + (1.0f - fu) * fv * d + fu * fv * e;
}

template <bool U8>
__global__ void __launch_bounds__(256)
pyramid_sample_kernel(const void* in, void* out, int W, int H, int C, float fx, float fy, float sigma0, float k,
                      PyramidLevels lv) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31), y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  const float dx = ((float)x + 0.5f) - fx, dy = ((float)y + 0.5f) - fy;
  const float sigma = sigma0 + k * sqrtf(dx * dx + dy * dy);
  float L = 0.5f * log2f(3.0f * sigma * sigma + 1.0f);
  L = fminf(fmaxf(L, 0.0f), (float)lv.top);
  const int l0 = min((int)floorf(L), lv.top);
  const float f = L - (float)l0;
  const int l1 = min(l0 + 1, lv.top);
  const float s0 = 1.0f / (float)(1 << l0), s1 = 1.0f / (float)(1 << l1);
  for (int c = 0; c < C; ++c) {
    float a;
    if (l0 == 0) a = U8 ? (float)static_cast<const unsigned char*>(in)[((size_t)y * W + x) * C + c]
                        : static_cast<const float*>(in)[((size_t)c * H + y) * W + x];
    else a = bilinear<2>(lv.ptr[l0], lv.w[l0], lv.h[l0], C, c, x * s0, y * s0);
    float v = a;
    if (f > 0.0f && l1 > l0) {
      const float b = bilinear<2>(lv.ptr[l1], lv.w[l1], lv.h[l1], C, c, x * s1, y * s1);
      v = fmaf(f, b - a, a);
    }
    if (U8) {
      static_cast<unsigned char*>(out)[((size_t)y * W + x) * C + c] = quant8(v);
    } else {
      static_cast<float*>(out)[((size_t)c * H + y) * W + x] = v;
    }
  }
}

}  // namespace

cudaError_t launch_pyramid(const void* in, void* out, int W, int H, int C, int isu8, float fx, float fy,
                           float sigma0, float k, const PyramidLevels& lv, cudaStream_t s) {
  for (int l = 1; l <= lv.top; ++l) {
    const dim3 grid((lv.w[l] + kRx - 1) / kRx, (lv.h[l] + kRy - 1) / kRy, C);
    if (l == 1) {
      if (isu8) pyramid_reduce_kernel<0><<<grid, kRx * kRy, 0, s>>>(in, W, H, C, lv.ptr[1], lv.w[1], lv.h[1]);
      else pyramid_reduce_kernel<1><<<grid, kRx * kRy, 0, s>>>(in, W, H, C, lv.ptr[1], lv.w[1], lv.h[1]);
    } else {
      pyramid_reduce_kernel<2><<<grid, kRx * kRy, 0, s>>>(lv.ptr[l - 1], lv.w[l - 1], lv.h[l - 1], C, lv.ptr[l],
                                                          lv.w[l], lv.h[l]);
    }
  }
  const dim3 grid((W + 31) / 32, (H + 7) / 8);
  if (isu8) pyramid_sample_kernel<true><<<grid, 256, 0, s>>>(in, out, W, H, C, fx, fy, sigma0, k, lv);
  else pyramid_sample_kernel<false><<<grid, 256, 0, s>>>(in, out, W, H, C, fx, fy, sigma0, k, lv);
  return cudaGetLastError();
}

}  // namespace fovea
