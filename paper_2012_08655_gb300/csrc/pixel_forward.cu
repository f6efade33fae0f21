// Per-pixel ("perfect") foveation: the quality reference of Section 3.1
// (Fig. 3), which the paper scores its block-wise output against. Every
// pixel is blurred with the Gaussian of its OWN eccentricity,
//
//   sigma_p = sigma0 + k |(x + 1/2, y + 1/2) - f|,  r_p = ceil(3 sigma_p),
//   out(p, c) = sum_{|i|,|j| <= r_p} u_p(i) u_p(j) in(clamp(x + i), clamp(y + j), c),
//
// with the taps u_p of Eq. 1 (truncated at r_p, normalised) and the
// clamp-to-edge border of the block-wise map; it equals the block-wise map
// with 1 x 1 blocks. No two output pixels share a filter, so the separable
// passes of the block-wise kernels do not apply: per pixel the work is
// (2 r_p + 1)^2 products.
//
// Two kernels:
//  - pixel_tc_kernel<C> (uint8 HWC): a 16 x 16 output tile per CTA, one warp
//    per output column x. The warp computes G[m][n] = sum_k A_x[m][k] B[k][n]
//    on the tensor cores (mma.sync m16n8k16, fp16 x fp16 -> fp32), where m
//    indexes the column's 16 output rows, k the staged (clamped) input rows,
//    n the staged input bytes, A_x[m][k] the vertical tap of pixel (x, y0+m)
//    at row offset k - R - m (hi + lo fp16 parts, as in the block-wise
//    kernels), and B the staged bytes entered as fp16 subnormals. Each
//    output is then the dot product of its row of G with its own horizontal
//    taps, on the FP32 units.
//  - pixel_fp32_kernel<C, U8> (both formats, any radius up to 255): one
//    thread per output pixel, the direct separable sum for that pixel with
//    its taps in shared memory.
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace fovea {
namespace {

using tcc::kWScale;
using tcc::mma16816;
using fwd::quant_u8;

// Sigma and radius of pixel (x, y): the block law's operations in the same
// order, at the pixel centre (x + 1/2, y + 1/2), binary64, no contraction.
__device__ __forceinline__ void pixel_sigma(int x, int y, double fx, double fy, double sigma0, double k,
                                            double& sigma, int& r) {
  const double dx = __dsub_rn(__dadd_rn((double)x, 0.5), fx);
  const double dy = __dsub_rn(__dadd_rn((double)y, 0.5), fy);
  const double e = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  sigma = __dadd_rn(sigma0, __dmul_rn(k, e));
  r = (int)ceil(__dmul_rn(3.0, sigma));
}

__device__ __forceinline__ float neg_half_inv_s2(double sigma) {
  return sigma > 0.0 ? (float)__ddiv_rn(-0.5, __dmul_rn(sigma, sigma)) : -INFINITY;
}

__device__ __forceinline__ float tap_w(int d, float c) { return d == 0 ? 1.0f : expf(c * (float)(d * d)); }

// ---------------------------------------------------------------- tensor-core kernel

constexpr int kTcM = 16;            // output rows per tile (the MMA's M)
constexpr int kTcN = 16;            // output columns per tile
constexpr int kTcWarps = 16;        // warp w takes output columns w, w + kTcWarps, ...
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kTcPix = kTcM * kTcN;
constexpr int kTcGroups = 3;        // 32-pixel groups (4 n-tiles each) accumulated at a time

template <int C>
__global__ void __launch_bounds__(kTcThreads, 1)
pixel_tc_kernel(PixelParams pp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PixelTcLayout L = pixel_tc_layout(pp.rmax, C);
  unsigned char* tile = smem;                                                   // C planes
  unsigned int* taps = reinterpret_cast<unsigned int*>(smem + L.tile_bytes);   // (hi, lo) fp16 per entry
  float* tc_c = reinterpret_cast<float*>(smem + L.tile_bytes + L.tap_bytes);
  int* tc_r = reinterpret_cast<int*>(tc_c + kTcPix);
  int* s_R = reinterpret_cast<int*>(tc_r + kTcPix);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * kTcN, y0 = blockIdx.y * kTcM;
  const int W = pp.W, H = pp.H, TP = L.tp;
  const unsigned char* in = static_cast<const unsigned char*>(pp.in);
  unsigned char* out = static_cast<unsigned char*>(pp.out);

  // ---- per-pixel sigma, radius, tap exponent (pixel p = row * 16 + column); tile radius
  if (tid == 0) *s_R = 0;
  __syncthreads();
  if (tid < kTcPix) {
    const int lx = tid & (kTcN - 1), ly = tid / kTcN;
    const int x = x0 + lx, y = y0 + ly;
    int r = 0;
    float c = -INFINITY;
    if (x < W && y < H) {
      double sigma;
      pixel_sigma(x, y, pp.fx, pp.fy, pp.sigma0, pp.k, sigma, r);
      if (r > pp.rmax || r < 0) {  // cannot happen with the host's bound; flagged, not run
        atomicOr(pp.err, kFaultPixelRadius);
        r = 0;
      } else {
        c = neg_half_inv_s2(sigma);
      }
      atomicMax(s_R, r);
    }
    tc_c[tid] = c;
    tc_r[tid] = r;
  }
  __syncthreads();
  const int R = *s_R;

  // ---- stage rows y0-R .. y0+15+R and pixels x0-R .. x0+15+R (clamped) as
  // one byte plane per channel; pair row P interleaves rows 2P and 2P+1:
  // 8-byte word w holds (row 2P, row 2P+1) of pixels 4w .. 4w+3
  {
    const int npr = 8 + R, nw = (16 + 2 * R + 3) / 4;
    for (int idx = tid; idx < C * npr * nw; idx += kTcThreads) {
      const int c = idx / (npr * nw), rem = idx - c * npr * nw;
      const int P = rem / nw, wi = rem - P * nw;
      const unsigned char* r0 = in + (size_t)min(max(y0 - R + 2 * P, 0), H - 1) * W * C + c;
      const unsigned char* r1 = in + (size_t)min(max(y0 - R + 2 * P + 1, 0), H - 1) * W * C + c;
      unsigned int lo = 0, hi = 0;
      #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const size_t xo = (size_t)min(max(x0 - R + 4 * wi + q, 0), W - 1) * C;
        const unsigned int v = (unsigned int)__ldg(r0 + xo) | ((unsigned int)__ldg(r1 + xo) << 8);
        if (q < 2) lo |= v << (16 * q);
        else hi |= v << (16 * (q - 2));
      }
      *reinterpret_cast<uint2*>(tile + c * L.plane_bytes + (size_t)P * L.pp + 8 * wi) = make_uint2(lo, hi);
    }
  }

  // ---- tap tables: entry d of pixel (row, column) = 2^12 u_p(d) as (hi, lo)
  // fp16, zero for d > r_p (the last entry is always zero); tables in
  // column-major pixel order (column * 16 + row)
  {
    // threads 2b and 2b+1 build table b (even and odd offsets)
    static_assert(kTcThreads == 2 * kTcPix, "two threads per tap table");
    const int tb = tid >> 1, h = tid & 1;
    const int pr = (tb & (kTcM - 1)) * kTcN + tb / kTcM;
    const int r = tc_r[pr];
    const float c = tc_c[pr];
    unsigned int* tw = taps + tb * TP;
    float* twf = reinterpret_cast<float*>(tw);
    float s = 0.0f;
    for (int d = h; d < TP; d += 2) {
      const float w = d <= r ? tap_w(d, c) : 0.0f;
      twf[d] = w;
      if (d >= 1) s += w;
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    const float inv = kWScale / (1.0f + 2.0f * s);
    for (int d = h; d < TP; d += 2) {
      const float w = twf[d] * inv;
      const __half hh = __float2half_rn(w);
      const __half ll = __float2half_rn(w - __half2float(hh));
      tw[d] = (unsigned int)__half_as_ushort(hh) | ((unsigned int)__half_as_ushort(ll) << 16);
    }
  }
  __syncthreads();

  // ---- per warp, output columns warp, warp + kTcWarps, ...: for each channel plane,
  // G[m][n] = sum_k A_x[m][k] B[k][n] over the column's window (32-pixel
  // groups from pixel 0), then out[m][c] = sum_n u_m(n - x - R) G[m][n]
  const int g = lane >> 2, t = lane & 3;
  const int KS = (16 + 2 * R + 15) >> 4;
  #pragma unroll 1
  for (int half = 0; half < kTcN / kTcWarps; ++half) {
    const int lx = warp + kTcWarps * half, x = x0 + lx;
    if (x >= W) break;  // warp-uniform; no barrier follows
    const unsigned int* TA = taps + (lx * kTcM + g) * TP;          // pixel (x, y0 + g)
    const unsigned int* TB = taps + (lx * kTcM + g + 8) * TP;      // pixel (x, y0 + g + 8)
    const int ng = (lx + 2 * R + 1 + 31) >> 5;                     // groups holding the window
    float o[2][C];
    #pragma unroll
    for (int h = 0; h < 2; ++h)
      #pragma unroll
      for (int c = 0; c < C; ++c) o[h][c] = 0.0f;
    #pragma unroll
    for (int c = 0; c < C; ++c) {
      const unsigned char* plane = tile + c * L.plane_bytes;
      for (int g0 = 0; g0 < ng; g0 += kTcGroups) {
        const int nc = min(kTcGroups, ng - g0);
        float acc[4 * kTcGroups][4];
        #pragma unroll
        for (int q = 0; q < 4 * kTcGroups; ++q)
          #pragma unroll
          for (int i = 0; i < 4; ++i) acc[q][i] = 0.0f;
        // A fragment: rows g (pixel A) and g + 8 (pixel B), columns
        // kb + 2t + {0, 1, 8, 9}; tap offset j = k - R - m. The taps of the
        // next k-step are loaded while this one's MMAs run.
        const int tl = TP - 1;
        unsigned int e[8];
        {
          const int jA = 2 * t - R - g;
          e[0] = TA[min(abs(jA), tl)]; e[1] = TA[min(abs(jA + 1), tl)];
          e[2] = TA[min(abs(jA + 8), tl)]; e[3] = TA[min(abs(jA + 9), tl)];
          e[4] = TB[min(abs(jA - 8), tl)]; e[5] = TB[min(abs(jA - 7), tl)];
          e[6] = TB[min(abs(jA), tl)]; e[7] = TB[min(abs(jA + 1), tl)];
        }
        for (int ks = 0; ks < KS; ++ks) {
          const int kb = 16 * ks;
          const unsigned int ah[4] = {__byte_perm(e[0], e[1], 0x5410), __byte_perm(e[4], e[5], 0x5410),
                                      __byte_perm(e[2], e[3], 0x5410), __byte_perm(e[6], e[7], 0x5410)};
          const unsigned int al[4] = {__byte_perm(e[0], e[1], 0x7632), __byte_perm(e[4], e[5], 0x7632),
                                      __byte_perm(e[2], e[3], 0x7632), __byte_perm(e[6], e[7], 0x7632)};
          if (ks + 1 < KS) {
            const int jA = kb + 16 + 2 * t - R - g;
            e[0] = TA[min(abs(jA), tl)]; e[1] = TA[min(abs(jA + 1), tl)];
            e[2] = TA[min(abs(jA + 8), tl)]; e[3] = TA[min(abs(jA + 9), tl)];
            e[4] = TB[min(abs(jA - 8), tl)]; e[5] = TB[min(abs(jA - 7), tl)];
            e[6] = TB[min(abs(jA), tl)]; e[7] = TB[min(abs(jA + 1), tl)];
          }
          // B: pair rows kb/2 + t (rows 2t, 2t+1) and kb/2 + t + 4 (rows
          // 2t+8, 2t+9); the lane's word g of a group holds column n = g of
          // n-tiles 0..3 (pixels 4g .. 4g+3)
          const unsigned char* bp = plane + (size_t)((kb >> 1) + t) * L.pp + (8 * g0 + g) * 8;
          // all hi products, then all lo products: the two MMAs into one
          // accumulator are 4 nc MMAs apart
          uint2 u[kTcGroups][2];
          #pragma unroll
          for (int grp = 0; grp < kTcGroups; ++grp) {
            if (grp >= nc) break;
            u[grp][0] = *reinterpret_cast<const uint2*>(bp + 64 * grp);
            u[grp][1] = *reinterpret_cast<const uint2*>(bp + 64 * grp + 4 * L.pp);
          }
          #pragma unroll
          for (int part = 0; part < 2; ++part) {
            #pragma unroll
            for (int grp = 0; grp < kTcGroups; ++grp) {
              if (grp >= nc) break;
              const uint2 u0 = u[grp][0], u8 = u[grp][1];
              unsigned int b[4][2];
              b[0][0] = __byte_perm(u0.x, 0u, 0x4140); b[1][0] = __byte_perm(u0.x, 0u, 0x4342);
              b[2][0] = __byte_perm(u0.y, 0u, 0x4140); b[3][0] = __byte_perm(u0.y, 0u, 0x4342);
              b[0][1] = __byte_perm(u8.x, 0u, 0x4140); b[1][1] = __byte_perm(u8.x, 0u, 0x4342);
              b[2][1] = __byte_perm(u8.y, 0u, 0x4140); b[3][1] = __byte_perm(u8.y, 0u, 0x4342);
              #pragma unroll
              for (int q = 0; q < 4; ++q) mma16816(acc[4 * grp + q], part ? al : ah, b[q][0], b[q][1]);
            }
          }
        }
        // horizontal taps: accumulator (n-tile q of group grp, column
        // 2t + hc, row g + 8 rh) is staged pixel 32 (g0 + grp) + 8t + 4hc + q
        #pragma unroll
        for (int grp = 0; grp < kTcGroups; ++grp) {
          if (grp >= nc) break;
          #pragma unroll
          for (int hc = 0; hc < 2; ++hc)
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int s = 32 * (g0 + grp) + 8 * t + 4 * hc + q;
              const int d = min(abs(s - lx - R), TP - 1);
              const unsigned int ea = TA[d], eb = TB[d];
              const float wa = __half2float(__ushort_as_half((unsigned short)(ea & 0xFFFFu))) +
                               __half2float(__ushort_as_half((unsigned short)(ea >> 16)));
              const float wb = __half2float(__ushort_as_half((unsigned short)(eb & 0xFFFFu))) +
                               __half2float(__ushort_as_half((unsigned short)(eb >> 16)));
              o[0][c] = fmaf(wa, acc[4 * grp + q][hc], o[0][c]);
              o[1][c] = fmaf(wb, acc[4 * grp + q][2 + hc], o[1][c]);
            }
        }
      }
    }
    // sum over the four lanes of a row, then store
    #pragma unroll
    for (int rh = 0; rh < 2; ++rh)
      #pragma unroll
      for (int c = 0; c < C; ++c) {
        float v = o[rh][c];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        o[rh][c] = v;
      }
    if (t == 0) {
      #pragma unroll
      for (int rh = 0; rh < 2; ++rh) {
        const int y = y0 + g + 8 * rh;
        if (y >= H) continue;
        unsigned char* op = out + ((size_t)y * W + x) * C;
        #pragma unroll
        for (int c = 0; c < C; ++c)
          if (in_bounds(op + c, 1, out, (size_t)W * H * C, pp.err)) op[c] = quant_u8(o[rh][c]);
      }
    }
  }
}

// ---------------------------------------------------------------- fp32 kernel

constexpr int kFpX = 16, kFpY = 8, kFpThreads = kFpX * kFpY;

template <int C, bool U8>
__global__ void __launch_bounds__(kFpThreads)
pixel_fp32_kernel(PixelParams pp, int rb) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Rl = pp.rmax;
  float* T = reinterpret_cast<float*>(smem);                    // T[d * 128 + tid], d <= R
  float* V = T + (size_t)(Rl + 1) * kFpThreads;                  // V[c][row][col], rb rows
  const int SP = kFpX + 2 * Rl + 1;                              // staged row pitch (floats)
  int* s_R = reinterpret_cast<int*>(V + (size_t)C * rb * SP);
  const int tid = threadIdx.x, tx = tid % kFpX, ty = tid / kFpX;
  const int x0 = blockIdx.x * kFpX, y0 = blockIdx.y * kFpY;
  const int W = pp.W, H = pp.H;
  const int x = x0 + tx, y = y0 + ty;
  const bool live = x < W && y < H;

  if (tid == 0) *s_R = 0;
  __syncthreads();
  int r = 0;
  float c = -INFINITY;
  if (live) {
    double sigma;
    pixel_sigma(x, y, pp.fx, pp.fy, pp.sigma0, pp.k, sigma, r);
    if (r > Rl || r < 0) {
      atomicOr(pp.err, kFaultPixelRadius);
      r = 0;
    } else {
      c = neg_half_inv_s2(sigma);
    }
    atomicMax(s_R, r);
  }
  // own taps, normalised
  float S = 1.0f;
  for (int d = 1; d <= r; ++d) S += 2.0f * tap_w(d, c);
  const float invS = 1.0f / S;
  for (int d = 0; d <= r; ++d) T[d * kFpThreads + tid] = tap_w(d, c) * invS;
  __syncthreads();
  const int R = *s_R;
  const int nrows = kFpY + 2 * R, ncols = kFpX + 2 * R;
  float acc[C];
  #pragma unroll
  for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;

  for (int r0 = 0; r0 < nrows; r0 += rb) {
    const int nr = min(rb, nrows - r0);
    __syncthreads();  // the previous chunk is consumed
    for (int idx = tid; idx < C * nr * ncols; idx += kFpThreads) {
      const int ch = idx / (nr * ncols), rem = idx - ch * nr * ncols;
      const int rr = rem / ncols, s = rem - rr * ncols;
      const int yy = min(max(y0 - R + r0 + rr, 0), H - 1);
      const int xx = min(max(x0 - R + s, 0), W - 1);
      float v;
      if (U8) {
        v = (float)static_cast<const unsigned char*>(pp.in)[((size_t)yy * W + xx) * C + ch];
      } else {
        v = static_cast<const float*>(pp.in)[((size_t)ch * H + yy) * W + xx];
      }
      V[((size_t)ch * rb + rr) * SP + s] = v;
    }
    __syncthreads();
    if (!live) continue;
    for (int rr = 0; rr < nr; ++rr) {
      const int j = r0 + rr - R - ty;  // row offset of staged row r0 + rr for this pixel
      if (j < -r || j > r) continue;
      const float wj = T[abs(j) * kFpThreads + tid];
      #pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        const float* vr = V + ((size_t)ch * rb + rr) * SP + tx + R;
        float h = T[tid] * vr[0];
        for (int i = 1; i <= r; ++i) h = fmaf(T[i * kFpThreads + tid], vr[-i] + vr[i], h);
        acc[ch] = fmaf(wj, h, acc[ch]);
      }
    }
  }
  if (!live) return;
  #pragma unroll
  for (int ch = 0; ch < C; ++ch) {
    if (U8) {
      unsigned char* o = static_cast<unsigned char*>(pp.out) + ((size_t)y * W + x) * C + ch;
      if (in_bounds(o, 1, pp.out, (size_t)W * H * C, pp.err)) *o = quant_u8(acc[ch]);
    } else {
      float* o = static_cast<float*>(pp.out) + ((size_t)ch * H + y) * W + x;
      if (in_bounds(o, 4, pp.out, (size_t)W * H * C * 4, pp.err)) *o = acc[ch];
    }
  }
}

template <int C>
cudaError_t launch_tc(const PixelParams& pp, cudaStream_t s) {
  const PixelTcLayout L = pixel_tc_layout(pp.rmax, C);
  const auto kern = pixel_tc_kernel<C>;
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(kern), L.total);
  if (e != cudaSuccess) return e;
  const dim3 grid((pp.W + kTcN - 1) / kTcN, (pp.H + kTcM - 1) / kTcM);
  kern<<<grid, kTcThreads, L.total, s>>>(pp);
  return cudaGetLastError();
}

template <int C, bool U8>
cudaError_t launch_fp32(const PixelParams& pp, cudaStream_t s) {
  const int rb = pixel_fp32_rows(pp.rmax, C);
  if (rb <= 0) return cudaErrorInvalidValue;
  const size_t smem = pixel_fp32_smem(pp.rmax, C, rb);
  const auto kern = pixel_fp32_kernel<C, U8>;
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((pp.W + kFpX - 1) / kFpX, (pp.H + kFpY - 1) / kFpY);
  kern<<<grid, kFpThreads, smem, s>>>(pp, rb);
  return cudaGetLastError();
}

}  // namespace

int pixel_fp32_rows(int rmax, int C) {
  const size_t taps = (size_t)(rmax + 1) * kFpThreads * 4;
  const size_t row = (size_t)C * (kFpX + 2 * rmax + 1) * 4;
  const size_t budget = kPixelSmemBudget;
  if (taps + row + 16 > budget) return 0;
  const int rows = (int)((budget - taps - 16) / row);
  const int need = kFpY + 2 * rmax;
  return rows < need ? rows : need;
}

size_t pixel_fp32_smem(int rmax, int C, int rb) {
  return (size_t)(rmax + 1) * kFpThreads * 4 + (size_t)C * rb * (kFpX + 2 * rmax + 1) * 4 + 16;
}

bool pixel_tc_fits(int rmax, int C) { return pixel_tc_layout(rmax, C).total <= kPixelSmemBudget; }

cudaError_t launch_pixel_forward(const PixelParams& pp, bool tensor_cores, cudaStream_t s) {
  if (pp.isu8 && tensor_cores) {
    switch (pp.C) {
      case 1: return launch_tc<1>(pp, s);
      case 2: return launch_tc<2>(pp, s);
      case 3: return launch_tc<3>(pp, s);
      case 4: return launch_tc<4>(pp, s);
    }
    return cudaErrorInvalidValue;
  }
  if (pp.isu8) {
    switch (pp.C) {
      case 1: return launch_fp32<1, true>(pp, s);
      case 2: return launch_fp32<2, true>(pp, s);
      case 3: return launch_fp32<3, true>(pp, s);
      case 4: return launch_fp32<4, true>(pp, s);
    }
  } else {
    switch (pp.C) {
      case 1: return launch_fp32<1, false>(pp, s);
      case 2: return launch_fp32<2, false>(pp, s);
      case 3: return launch_fp32<3, false>(pp, s);
      case 4: return launch_fp32<4, false>(pp, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace fovea
