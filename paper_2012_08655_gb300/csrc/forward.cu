// Forward foveation kernel: one persistent CTA loop over (frame, block) items.
//
// For one block (paper Section 2 and Algorithm 1: "place padded fragment into
// shared memory", "horizontal convolution", "place result into shared
// memory", "vertical convolution", "write result"):
//   * taps: the block's normalised 1D Gaussian, generated in the CTA and
//     summed with warp shuffles (no constant-memory filter bank);
//   * halo tile: rows y0-r .. y0+bh-1+r and columns x0-r .. x0+bw-1+r of the
//     input, clamped to the frame; uint8 is unpacked to float while staging;
//   * pass 1 (vertical): V[yo][e] = sum_ty u[ty - yo] * T[ty][e] for the 32
//     output rows and every tile element column e (pixel column x channel);
//   * pass 2 (horizontal): O[yo][x][c] = sum_tx u[tx - x] * V[yo][tx][c];
//   * round/pack and store.
// Running the vertical pass first lets the tile stream through shared memory
// in row chunks (each thread keeps its accumulators and a sliding window of
// taps in registers), so shared memory does not grow with the radius; wide
// tiles are cut into column slabs and pass 2 accumulates across slabs. All
// products are fp32 FMAs, two lanes per instruction (fma.rn.f32x2); each
// thread produces 8 outputs per input value it loads (the register data reuse
// of the paper's "Data Reuse" subsection, generalised).
#include "fovea_internal.cuh"

namespace fovea {

namespace {

constexpr int kThreads = 256;
constexpr int kSlab = 256;        // max element columns per slab
constexpr int kVVPitch = kSlab + 1;  // float2 pitch of the row-pair buffer (odd: no bank conflicts)

struct SmemLayout {
  size_t ring, vv, taps, coloff, red, total;
};

__host__ __device__ inline SmemLayout smem_layout(int rb, int ulen) {
  SmemLayout L;
  L.ring = 0;                                            // float [rb][kSlab]
  L.vv = L.ring + (size_t)rb * kSlab * sizeof(float);    // float2 [16][kVVPitch]
  L.taps = L.vv + (size_t)16 * kVVPitch * sizeof(float2);// float2 [ulen]
  L.coloff = L.taps + (size_t)ulen * sizeof(float2);     // int [kSlab]
  L.red = L.coloff + (size_t)kSlab * sizeof(int);        // float [32]
  L.total = L.red + 32 * sizeof(float);
  return L;
}

__device__ __forceinline__ unsigned char quant_u8(float v) {
  int q = __float2int_rd(v + 0.5f);
  q = q < 0 ? 0 : (q > 255 ? 255 : q);
  return (unsigned char)q;
}

template <int RB>
__global__ void __launch_bounds__(kThreads, 2)
forward_kernel(FrameSource src, Workspace ws, int ulen_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(RB, ulen_max);
  float4* ring4 = reinterpret_cast<float4*>(smem + L.ring);
  float2* VV = reinterpret_cast<float2*>(smem + L.vv);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  int* colOff = reinterpret_cast<int*>(smem + L.coloff);
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_ticket;

  const int tid = threadIdx.x;
  const int n_items = (int)ws.counters[CNT_NITEMS];
  // pass-1 identity: quad q1 of 4 element columns, row group G1 of 8 output rows
  const int q1 = tid & 63, G1 = tid >> 6;
  // pass-2 identity: row pair p2, channel c2, group g2 of 8 output columns
  const int g2 = tid >> 6, c2 = (tid >> 4) & 3, p2 = tid & 15;

  for (;;) {
    if (tid == 0) s_ticket = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
    __syncthreads();
    const int t = s_ticket;
    __syncthreads();  // s_ticket may be rewritten once every thread has read it
    if (t >= n_items) break;
    const int item = ws.order[t];
    if ((unsigned)item >= (unsigned)n_items) {  // work list out of step: skip, flag
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], 16u);
      continue;
    }
    const ItemInfo inf = ws.items[item];
    const FrameDesc fd = load_frame(src, inf.frame);
    const int r = inf.r;
    const int ulen = tap_len(r);
    if (ulen > ulen_max) {  // launch sized for a smaller radius: refuse the item
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], 2u);
      continue;
    }
    const int W = fd.W, H = fd.H, C = fd.C, B = fd.B;
    const bool u8 = fd.fmt == FOVEA_U8_HWC;
    const int bx = inf.block % fd.nbx, by = inf.block / fd.nbx;
    const int x0 = bx * B, y0 = by * B;
    const int bw = min(B, W - x0), bh = min(B, H - y0);

    make_taps(U, ulen, r, inf.neg_half_inv_s2, red);

    const int SW = (kSlab / (8 * C)) * (8 * C);  // slab width: whole pixels, 8-pixel aligned
    const int tileW = bw + 2 * r;
    const int E = tileW * C;                      // element columns of the tile
    const int nslabs = (E + SW - 1) / SW;
    const int steps = 1 + ((2 * r + 7) >> 3);     // 8-row (8-column) steps covering 2r+8 taps
    const int groups1 = (bh + 7) >> 3;
    const int groups2 = (bw + 7) >> 3;
    const int Rows = 8 * (groups1 - 1 + steps);   // tile rows that pass 1 reads
    const int nchunks = (Rows + RB - 1) / RB;
    const size_t rowPitch = u8 ? (size_t)W * C : (size_t)W;
    const int planePitch = W * H;

    const bool act2 = g2 < groups2 && c2 < C && 2 * p2 < bh;
    const int xg = 8 * g2;
    float2 acc2[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) acc2[j] = make_float2(0.f, 0.f);

    for (int sl = 0; sl < nslabs; ++sl) {
      const int s0 = sl * SW;
      const int SWs = min(SW, E - s0);
      const int P0 = s0 / C, P1 = P0 + SWs / C;
      for (int e = tid; e < SWs; e += kThreads) {
        const int eg = s0 + e;
        const int tx = eg / C, c = eg - tx * C;
        const int gx = clampi(x0 - r + tx, 0, W - 1);
        colOff[e] = u8 ? gx * C + c : c * planePitch + gx;
      }
      const bool act1 = G1 < groups1 && 4 * q1 < SWs;
      const int rlo = 8 * G1, rhi = 8 * (G1 + steps);
      float2 a1[8][2];
      float2 w1[8];
      #pragma unroll
      for (int j = 0; j < 8; ++j) {
        a1[j][0] = a1[j][1] = w1[j] = make_float2(0.f, 0.f);
      }
      for (int k = 0; k < nchunks; ++k) {
        const int R0 = k * RB;
        __syncthreads();  // ring free; colOff visible
        for (int idx = tid; idx < RB * (kSlab / 4); idx += kThreads) {
          const int row = idx / (kSlab / 4), q = idx % (kSlab / 4);
          const int e = 4 * q;
          if (R0 + row < Rows && e < SWs) {
            const int gy = clampi(y0 - r + R0 + row, 0, H - 1);
            float v[4];
            if (u8) {
              const unsigned char* base = static_cast<const unsigned char*>(fd.in) + (size_t)gy * rowPitch;
              #pragma unroll
              for (int u = 0; u < 4; ++u) v[u] = (e + u < SWs) ? u8_to_f32(__ldg(base + colOff[e + u])) : 0.f;
            } else {
              const float* base = static_cast<const float*>(fd.in) + (size_t)gy * rowPitch;
              #pragma unroll
              for (int u = 0; u < 4; ++u) v[u] = (e + u < SWs) ? __ldg(base + colOff[e + u]) : 0.f;
            }
            ring4[row * (kSlab / 4) + q] = make_float4(v[0], v[1], v[2], v[3]);
          }
        }
        __syncthreads();
        if (act1) {
          const int lo = max(R0, rlo), hi = min(min(R0 + RB, rhi), Rows);
          for (int ty0 = lo; ty0 < hi; ty0 += 8) {
            #pragma unroll
            for (int s = 0; s < 8; ++s) {
              const int ty = ty0 + s;
              w1[s] = U[kTapPad + ty - rlo];
              const float4 d = ring4[(ty - R0) * (kSlab / 4) + q1];
              const float2 dlo = make_float2(d.x, d.y), dhi = make_float2(d.z, d.w);
              #pragma unroll
              for (int j = 0; j < 8; ++j) {
                a1[j][0] = ffma2(w1[(s - j) & 7], dlo, a1[j][0]);
                a1[j][1] = ffma2(w1[(s - j) & 7], dhi, a1[j][1]);
              }
            }
          }
        }
      }
      if (act1) {  // V rows 8G1..8G1+7 -> row-pair buffer
        #pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          float2* dst = VV + (4 * G1 + pp) * kVVPitch + 4 * q1;
          dst[0] = make_float2(a1[2 * pp][0].x, a1[2 * pp + 1][0].x);
          dst[1] = make_float2(a1[2 * pp][0].y, a1[2 * pp + 1][0].y);
          dst[2] = make_float2(a1[2 * pp][1].x, a1[2 * pp + 1][1].x);
          dst[3] = make_float2(a1[2 * pp][1].y, a1[2 * pp + 1][1].y);
        }
      }
      __syncthreads();
      if (act2) {
        const int lo = max(P0, xg), hi = min(P1, xg + 8 * steps);
        if (lo < hi) {
          float2 w2[8];
          #pragma unroll
          for (int s = 0; s < 8; ++s) w2[s] = U[kTapPad + lo - 8 + s - xg];
          const float2* vrow = VV + p2 * kVVPitch + c2;
          for (int tx0 = lo; tx0 < hi; tx0 += 8) {
            #pragma unroll
            for (int s = 0; s < 8; ++s) {
              const int tx = tx0 + s;
              w2[s] = U[kTapPad + tx - xg];
              float2 d = make_float2(0.f, 0.f);
              if (tx < hi) d = vrow[(tx - P0) * C];
              #pragma unroll
              for (int j = 0; j < 8; ++j) acc2[j] = ffma2(w2[(s - j) & 7], d, acc2[j]);
            }
          }
        }
      }
    }

    if (!u8) {
      if (act2) {
        float* out = static_cast<float*>(fd.out) + (size_t)c2 * planePitch + (size_t)(y0 + 2 * p2) * W + x0;
        const bool second = 2 * p2 + 1 < bh;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = xg + j;
          if (x < bw) {
            out[x] = acc2[j].x;
            if (second) out[W + x] = acc2[j].y;
          }
        }
      }
    } else {
      // Stage the 8-bit block in shared memory (the ring is free after the
      // last pass 1) and write it out with coalesced byte runs.
      unsigned char* ost = smem + L.ring;
      const int opitch = 32 * C;
      if (act2) {
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = xg + j;
          ost[(2 * p2) * opitch + x * C + c2] = quant_u8(acc2[j].x);
          ost[(2 * p2 + 1) * opitch + x * C + c2] = quant_u8(acc2[j].y);
        }
      }
      __syncthreads();
      const int rowBytes = bw * C;
      unsigned char* out = static_cast<unsigned char*>(fd.out) + (size_t)y0 * rowPitch + (size_t)x0 * C;
      for (int idx = tid; idx < bh * rowBytes; idx += kThreads) {
        const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
        out[(size_t)yo * rowPitch + rem] = ost[yo * opitch + rem];
      }
    }
  }
}

template <int RB>
void* kernel_ptr() { return reinterpret_cast<void*>(&forward_kernel<RB>); }

void* pick_kernel(int rb) {
  switch (rb) {
    case 16: return kernel_ptr<16>();
    case 64: return kernel_ptr<64>();
    default: return kernel_ptr<32>();
  }
}

}  // namespace

size_t forward_smem_bytes(const FwdConfig& cfg, int rmax) {
  return smem_layout(cfg.rows_per_chunk, tap_len(rmax)).total;
}

int forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax) {
  const size_t smem = forward_smem_bytes(cfg, rmax);
  void* k = pick_kernel(cfg.rows_per_chunk);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg,
                           int rmax, int grid, cudaStream_t s) {
  const int ulen = tap_len(rmax);
  const size_t smem = forward_smem_bytes(cfg, rmax);
  void* k = pick_kernel(cfg.rows_per_chunk);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), const_cast<int*>(&ulen)};
  return cudaLaunchKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace fovea
