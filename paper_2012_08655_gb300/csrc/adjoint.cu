// Adjoint (transpose) of the foveation map for float32 CHW frames.
//
// The forward map of block b is out_b = Uv * T_b * Uh^T restricted to the
// block, where T_b is the clamped halo tile and Uv, Uh are banded Toeplitz
// matrices of the block's taps. Its transpose spreads each block's output
// gradient back over the block's halo tile and folds the clamped tile
// positions onto the edge pixels they were read from:
//   Z[yo][tx]  = sum_xo u[tx - xo] * g[yo][xo]      (horizontal, transposed)
//   gT[ty][tx] = sum_yo u[ty - yo] * Z[yo][tx]      (vertical, transposed)
//   g_in[clamp(y0-r+ty)][clamp(x0-r+tx)] += gT[ty][tx]
// Tiles of neighbouring blocks overlap, so the last step is a global atomic
// add (fp32; the summation order is not fixed, so results are reproducible to
// rounding, not bit for bit). Not in the paper: it exists so the blur can sit
// inside network training (a torch.autograd.Function uses it).
#include "fovea_internal.cuh"

namespace fovea {

namespace {

constexpr int kThreads = 256;
constexpr int kSlabPx = 256;           // tile pixel columns per slab (one channel at a time)
constexpr int kZPitch = kSlabPx + 4;   // float pitch of Z (multiple of 4 for float4 reads)
constexpr int kGPitch = 33;            // float2 pitch of the row-pair gradient block (odd)

struct SmemLayout {
  size_t gg, z, taps, red, total;
};

__host__ __device__ inline SmemLayout smem_layout(int ulen) {
  SmemLayout L;
  L.gg = 0;                                                // float2 [4][16][kGPitch]
  L.z = L.gg + (size_t)4 * 16 * kGPitch * sizeof(float2);  // float [32][kZPitch]
  L.taps = L.z + (size_t)32 * kZPitch * sizeof(float);     // float2 [ulen]
  L.red = L.taps + (size_t)ulen * sizeof(float2);          // float [32]
  L.total = L.red + 32 * sizeof(float);
  return L;
}

__global__ void __launch_bounds__(kThreads, 2)
adjoint_kernel(FrameSource src, Workspace ws, int ulen_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(ulen_max);
  float2* GG = reinterpret_cast<float2*>(smem + L.gg);
  float* Z = reinterpret_cast<float*>(smem + L.z);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_ticket;

  const int tid = threadIdx.x;
  const int n_items = (int)ws.counters[CNT_NITEMS];

  for (;;) {
    if (tid == 0) s_ticket = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
    __syncthreads();
    const int t = s_ticket;
    __syncthreads();
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
    if (ulen > ulen_max || fd.fmt != FOVEA_F32_CHW || fd.C > 4) {
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], 4u);
      continue;
    }
    const int W = fd.W, H = fd.H, C = fd.C, B = fd.B;
    const int bx = inf.block % fd.nbx, by = inf.block / fd.nbx;
    const int x0 = bx * B, y0 = by * B;
    const int bw = min(B, W - x0), bh = min(B, H - y0);
    const int planePitch = W * H;
    const float* gout = static_cast<const float*>(fd.in);
    float* gin = static_cast<float*>(fd.out);

    make_taps(U, ulen, r, inf.neg_half_inv_s2, red);

    // Output-gradient block as row pairs, zero outside the block.
    float* GGf = reinterpret_cast<float*>(GG);
    for (int idx = tid; idx < C * 32 * 32; idx += kThreads) {
      const int c = idx >> 10, yo = (idx >> 5) & 31, xo = idx & 31;
      float v = 0.f;
      if (yo < bh && xo < bw) v = __ldg(gout + (size_t)c * planePitch + (size_t)(y0 + yo) * W + x0 + xo);
      GGf[((c * 16 + (yo >> 1)) * kGPitch + xo) * 2 + (yo & 1)] = v;
    }
    __syncthreads();

    const int tileW = bw + 2 * r, tileH = bh + 2 * r;
    const int nh = (tileH + 7) >> 3;
    for (int c = 0; c < C; ++c) {
      for (int X0 = 0; X0 < tileW; X0 += kSlabPx) {
        const int SWx = min(kSlabPx, tileW - X0);
        // ---- pass A: Z[yo][tx - X0] for the slab, items (row pair p, 8-column group)
        const int ngA = (SWx + 7) >> 3;
        for (int it = tid; it < 16 * ngA; it += kThreads) {
          const int p = it & 15, g = it >> 4;
          const int txg = X0 + 8 * g;
          // k = txg - xo; data needs xo in [0, bw); taps need k + j in [0, 2r].
          const int klo = max(txg - bw + 1, -7), khi = min(txg, 2 * r);
          float2 acc[8];
          #pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
          if (klo <= khi) {
            const int k0 = klo >= 0 ? (klo & ~7) : -8;
            float2 w[8];
            #pragma unroll
            for (int s = 0; s < 7; ++s) w[s] = U[kTapPad + k0 + s];
            const float2* grow = GG + (c * 16 + p) * kGPitch;
            for (int kb = k0; kb <= khi; kb += 8) {
              #pragma unroll
              for (int s = 0; s < 8; ++s) {
                const int kk = kb + s;
                w[(s + 7) & 7] = U[kTapPad + kk + 7];
                float2 d = make_float2(0.f, 0.f);
                if (kk >= klo && kk <= khi) d = grow[txg - kk];
                #pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = ffma2(w[(s + j) & 7], d, acc[j]);
              }
            }
          }
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = 8 * g + j;
            if (col < SWx) {
              Z[(2 * p) * kZPitch + col] = acc[j].x;
              Z[(2 * p + 1) * kZPitch + col] = acc[j].y;
            }
          }
        }
        __syncthreads();
        // ---- pass B: gT rows for the slab, items (4-column quad, 8-row group)
        const int nq = (SWx + 3) >> 2;
        for (int it = tid; it < nq * nh; it += kThreads) {
          const int q = it % nq, h = it / nq;
          const int tyg = 8 * h;
          const int klo = max(tyg - bh + 1, -7), khi = min(tyg, 2 * r);
          if (klo > khi) continue;
          float2 acc[8][2];
          #pragma unroll
          for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
          const int k0 = klo >= 0 ? (klo & ~7) : -8;
          float2 w[8];
          #pragma unroll
          for (int s = 0; s < 7; ++s) w[s] = U[kTapPad + k0 + s];
          for (int kb = k0; kb <= khi; kb += 8) {
            #pragma unroll
            for (int s = 0; s < 8; ++s) {
              const int kk = kb + s;
              w[(s + 7) & 7] = U[kTapPad + kk + 7];
              float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
              if (kk >= klo && kk <= khi) d = *reinterpret_cast<const float4*>(Z + (tyg - kk) * kZPitch + 4 * q);
              const float2 dlo = make_float2(d.x, d.y), dhi = make_float2(d.z, d.w);
              #pragma unroll
              for (int j = 0; j < 8; ++j) {
                acc[j][0] = ffma2(w[(s + j) & 7], dlo, acc[j][0]);
                acc[j][1] = ffma2(w[(s + j) & 7], dhi, acc[j][1]);
              }
            }
          }
          float* plane = gin + (size_t)c * planePitch;
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ty = tyg + j;
            if (ty >= tileH) break;
            const int gy = clampi(y0 - r + ty, 0, H - 1);
            float* rowp = plane + (size_t)gy * W;
            const float v[4] = {acc[j][0].x, acc[j][0].y, acc[j][1].x, acc[j][1].y};
            #pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int col = 4 * q + e;
              if (col < SWx && v[e] != 0.f) {
                const int gx = clampi(x0 - r + X0 + col, 0, W - 1);
                atomicAdd(rowp + gx, v[e]);
              }
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

}  // namespace

size_t adjoint_smem_bytes(int rmax) { return smem_layout(tap_len(rmax)).total; }

int adjoint_max_ctas_per_sm(int rmax) {
  const size_t smem = adjoint_smem_bytes(rmax);
  if (cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_adjoint(const FrameSource& src, const Workspace& ws, int rmax, int grid,
                           cudaStream_t s) {
  const int ulen = tap_len(rmax);
  const size_t smem = adjoint_smem_bytes(rmax);
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adjoint_kernel<<<grid, kThreads, smem, s>>>(src, ws, ulen);
  return cudaGetLastError();
}

}  // namespace fovea
