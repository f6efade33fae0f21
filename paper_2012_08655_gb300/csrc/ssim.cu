// SSIM map of two images (the quality measure of Section 3.1; Wang, Bovik,
// Sheikh and Simoncelli 2004 with their standard settings): local means,
// variances and covariance under an 11 x 11 Gaussian window of standard
// deviation 1.5 normalised to unit sum, clamp-to-edge at the border,
//
//   SSIM = (2 mu_a mu_b + C1)(2 cov + C2) / ((mu_a^2 + mu_b^2 + C1)(var_a + var_b + C2)),
//
// C1 = (0.01 L)^2, C2 = (0.03 L)^2; the map value of a pixel is the mean
// over its channels. The window is separable, so each CTA stages its tile
// with a 5-pixel halo, filters the five products (a, b, a^2, b^2, ab)
// horizontally into shared memory, then vertically. Values are taken
// relative to L / 2 before squaring, which keeps the single-pass moments
// E[a^2] - mu^2 well conditioned in fp32.
#include "fovea_internal.cuh"

namespace fovea {
namespace {

constexpr int kSx = 32, kSy = 8, kSr = 5;
constexpr int kSthreads = kSx * kSy;
constexpr int kSRows = kSy + 2 * kSr, kSCols = kSx + 2 * kSr;

template <bool U8>
__device__ __forceinline__ float load_px(const void* p, int W, int H, int C, int x, int y, int c) {
  if (U8) return (float)static_cast<const unsigned char*>(p)[((size_t)y * W + x) * C + c];
  return static_cast<const float*>(p)[((size_t)c * H + y) * W + x];
}

template <bool U8>
__global__ void __launch_bounds__(kSthreads)
ssim_kernel(const void* a, const void* b, int W, int H, int C, float L, float* map, double* sum) {
  __shared__ float sa[kSRows][kSCols + 1], sb[kSRows][kSCols + 1];
  __shared__ float hm[5][kSRows][kSx + 1];
  __shared__ float gw[2 * kSr + 1];
  __shared__ float red[32];
  const int tid = threadIdx.x, tx = tid % kSx, ty = tid / kSx;
  const int x0 = blockIdx.x * kSx, y0 = blockIdx.y * kSy;
  if (tid == 0) {
    float s = 0.0f;
    for (int i = -kSr; i <= kSr; ++i) {
      gw[i + kSr] = expf(-(float)(i * i) / (2.0f * 1.5f * 1.5f));
      s += gw[i + kSr];
    }
    for (int i = 0; i <= 2 * kSr; ++i) gw[i] /= s;
  }
  const float off = 0.5f * L;
  const float C1 = (0.01f * L) * (0.01f * L), C2 = (0.03f * L) * (0.03f * L);
  const int x = x0 + tx, y = y0 + ty;
  float total = 0.0f;
  for (int c = 0; c < C; ++c) {
    __syncthreads();  // previous channel consumed (and gw written)
    for (int idx = tid; idx < kSRows * kSCols; idx += kSthreads) {
      const int rr = idx / kSCols, cc = idx - rr * kSCols;
      const int yy = min(max(y0 - kSr + rr, 0), H - 1), xx = min(max(x0 - kSr + cc, 0), W - 1);
      sa[rr][cc] = load_px<U8>(a, W, H, C, xx, yy, c) - off;
      sb[rr][cc] = load_px<U8>(b, W, H, C, xx, yy, c) - off;
    }
    __syncthreads();
    for (int idx = tid; idx < kSRows * kSx; idx += kSthreads) {
      const int rr = idx / kSx, cc = idx - rr * kSx;
      float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
      #pragma unroll
      for (int i = 0; i <= 2 * kSr; ++i) {
        const float w = gw[i], va = sa[rr][cc + i], vb = sb[rr][cc + i];
        m0 = fmaf(w, va, m0);
        m1 = fmaf(w, vb, m1);
        m2 = fmaf(w, va * va, m2);
        m3 = fmaf(w, vb * vb, m3);
        m4 = fmaf(w, va * vb, m4);
      }
      hm[0][rr][cc] = m0; hm[1][rr][cc] = m1; hm[2][rr][cc] = m2; hm[3][rr][cc] = m3; hm[4][rr][cc] = m4;
    }
    __syncthreads();
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    #pragma unroll
    for (int j = 0; j <= 2 * kSr; ++j) {
      const float w = gw[j];
      #pragma unroll
      for (int q = 0; q < 5; ++q) m[q] = fmaf(w, hm[q][ty + j][tx], m[q]);
    }
    const float va = m[2] - m[0] * m[0], vb = m[3] - m[1] * m[1], cv = m[4] - m[0] * m[1];
    const float mua = m[0] + off, mub = m[1] + off;
    total += ((2.0f * mua * mub + C1) * (2.0f * cv + C2)) / ((mua * mua + mub * mub + C1) * (va + vb + C2));
  }
  const bool live = x < W && y < H;
  const float v = live ? total / (float)C : 0.0f;
  if (live && map) map[(size_t)y * W + x] = v;
  if (sum) {
    float s = v;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid < 32) {
      float t = tid < kSthreads / 32 ? red[tid] : 0.0f;
      #pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (tid == 0) atomicAdd(sum, (double)t);
    }
  }
}

}  // namespace

cudaError_t launch_ssim(const void* a, const void* b, int W, int H, int C, int isu8, float data_range,
                        float* map, double* sum, cudaStream_t s) {
  const dim3 grid((W + kSx - 1) / kSx, (H + kSy - 1) / kSy);
  if (sum) {
    cudaError_t e = cudaMemsetAsync(sum, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
  }
  if (isu8) {
    ssim_kernel<true><<<grid, kSthreads, 0, s>>>(a, b, W, H, C, data_range, map, sum);
  } else {
    ssim_kernel<false><<<grid, kSthreads, 0, s>>>(a, b, W, H, C, data_range, map, sum);
  }
  return cudaGetLastError();
}

}  // namespace fovea
