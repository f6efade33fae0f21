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
// The tile is folded as in the forward kernel: only in-frame rows and columns
// are formed, and the clamped taps of the edge row / column are summed into
// one prefix-summed weight, so every frame pixel receives exactly one
// contribution per block. Tiles of neighbouring blocks overlap, so that
// contribution is a global atomic add (fp32; the summation order is not
// fixed, so results are reproducible to rounding, not bit for bit). Not in the paper: it exists so the blur can sit
// inside network training (a torch.autograd.Function uses it).
#include "fovea_internal.cuh"

namespace fovea {

namespace {

constexpr int kThreads = 256;
constexpr int kGPitch = 33;            // float2 pitch of the row-pair gradient block (odd)
// Every plane of the tile goes through each pass together (more independent
// work per phase, one pair of barriers per slab instead of per plane): Z
// holds the planes one after the other, slabs of 256 tile columns for one
// or two planes, 128 for three or four; a Z row has 4 spare floats (the
// column shift of the vector reductions, float4 reads).
__host__ __device__ constexpr int adj_slab(int C) { return C <= 2 ? 256 : 128; }
__host__ __device__ constexpr int adj_zpitch(int C) { return adj_slab(C) + 4; }
constexpr int kZFloats = 4 * 32 * (128 + 4);  // the largest C x 32 x pitch (C = 4; C = 2 needs 16,640)
static_assert(2 * 32 * (256 + 4) <= kZFloats && 1 * 32 * (256 + 4) <= kZFloats && 3 * 32 * (128 + 4) <= kZFloats,
              "every channel count's Z fits");

struct SmemLayout {
  size_t gg, z, taps, cum, red, total;
};

__host__ __device__ inline SmemLayout smem_layout(int rmax) {
  SmemLayout L;
  L.gg = 0;                                                // float2 [4][16][kGPitch]
  L.z = L.gg + (size_t)4 * 16 * kGPitch * sizeof(float2);  // float [C][32][zpitch]
  L.taps = L.z + (size_t)kZFloats * sizeof(float);         // float2 [tap_len]
  L.cum = L.taps + (size_t)tap_len(rmax) * sizeof(float2); // float [cum_len]
  L.red = L.cum + (size_t)cum_len(rmax) * sizeof(float);   // float [32]
  L.total = L.red + 32 * sizeof(float);
  return L;
}

__global__ void __launch_bounds__(kThreads, 2)
adjoint_kernel(FrameSource src, Workspace ws, int rmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(rmax);
  float2* GG = reinterpret_cast<float2*>(smem + L.gg);
  float* Z = reinterpret_cast<float*>(smem + L.z);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
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
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], kFaultWorklist);
      continue;
    }
    const ItemInfo inf = ws.items[item];
    const FrameDesc fd = load_frame(src, inf.frame);
    const int r = inf.r;
    if (r > rmax || fd.fmt != FOVEA_F32_CHW || fd.C > 4) {
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], kFaultAdjBound);
      continue;
    }
    const int W = fd.W, H = fd.H, C = fd.C, T = fd.T;
    const int tx = inf.block % fd.nbx, ty = inf.block / fd.nbx;  // tile
    const int xs = tx * T - fd.ox, ys = ty * T - fd.oy;          // unclipped tile start
    const int x0 = max(0, xs), y0 = max(0, ys);
    const int bw = min(xs + T, W) - x0, bh = min(ys + T, H) - y0;
    // Folded tile: frame columns gx0 .. gx0+EW-1 and rows gy0 .. gy0+EH-1; the
    // tap index of (tile column ex, block column xo) is offx + ex - xo.
    const int gx0 = max(0, x0 - r), EW = min(W - 1, x0 + bw - 1 + r) - gx0 + 1, offx = gx0 - (x0 - r);
    const int gy0 = max(0, y0 - r), EH = min(H - 1, y0 + bh - 1 + r) - gy0 + 1, offy = gy0 - (y0 - r);
    const bool foldL = x0 - r < 0, foldR = x0 + bw - 1 + r > W - 1;
    const bool foldT = y0 - r < 0, foldB = y0 + bh - 1 + r > H - 1;
    const size_t planePitch = (size_t)W * H;
    const float* gout = static_cast<const float*>(fd.in);
    float* gin = static_cast<float*>(fd.out);
    // rows of grad_in start on 16-byte boundaries: four consecutive columns
    // from a multiple of 4 take one vector reduction
    const bool vec_ok = (((uintptr_t)gin) & 15) == 0 && (W & 3) == 0;

    make_taps(U, tap_len(r), r, inf.neg_half_inv_s2, red);
    make_cumulative(U, CU, r);

    // Output-gradient block as row pairs, zero outside the block.
    float* GGf = reinterpret_cast<float*>(GG);
    for (int idx = tid; idx < C * 32 * 32; idx += kThreads) {
      const int c = idx >> 10, yo = (idx >> 5) & 31, xo = idx & 31;
      float v = 0.f;
      if (yo < bh && xo < bw) v = __ldg(gout + (size_t)c * planePitch + (size_t)(y0 + yo) * W + x0 + xo);
      GGf[((c * 16 + (yo >> 1)) * kGPitch + xo) * 2 + (yo & 1)] = v;
    }
    __syncthreads();

    const int nh = (EH + 7) >> 3;
    const int slab = adj_slab(C), kZPitch = adj_zpitch(C);
    {
      for (int X0 = 0; X0 < EW; X0 += slab) {
        const int SWx = min(slab, EW - X0);
        // Z column of slab column col is col + sh: pass B's groups of four Z
        // columns then cover frame columns from a multiple of 4
        const int sh = (gx0 + X0) & 3;
        // ---- pass A: Z[c][yo][ex - X0] = sum_xo w(ex, xo) g[c][yo][xo], every plane
        const int ngA = (SWx + 7) >> 3;
        for (int it = tid; it < C * 16 * ngA; it += kThreads) {
          const int c = it / (16 * ngA), rem = it - c * 16 * ngA;
          const int p = rem & 15, g = rem >> 4;
          float* Zc = Z + (size_t)c * 32 * kZPitch;
          const int tg = offx + X0 + 8 * g;   // tap index of (ex = X0 + 8g, xo = 0)
          const int klo = max(tg - bw + 1, -7), khi = min(tg, 2 * r);
          float2 acc[8];
          #pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
          const float2* grow = GG + (c * 16 + p) * kGPitch;
          if (klo <= khi) {
            const int k0 = klo >= 0 ? (klo & ~7) : -8;
            float2 w[8];
            #pragma unroll
            for (int s = 0; s < 7; ++s) w[s] = U[kTapPad + k0 + s];
            for (int kb = k0; kb <= khi; kb += 8) {
              #pragma unroll
              for (int s = 0; s < 8; ++s) {
                const int kk = kb + s;
                w[(s + 7) & 7] = U[kTapPad + kk + 7];
                float2 d = make_float2(0.f, 0.f);
                if (kk >= klo && kk <= khi) d = grow[tg - kk];
                #pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = ffma2(w[(s + j) & 7], d, acc[j]);
              }
            }
          }
          // Folded edge columns collect the clamped taps (prefix sums).
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ex = X0 + 8 * g + j;
            const bool fl = foldL && ex == 0, fr = foldR && ex == EW - 1;
            if (fl || fr) {
              for (int xo = 0; xo < bw; ++xo) {
                float cw = 0.f;
                if (fl) cw += cum_at(CU, offx - xo, r);
                if (fr) cw += cum_at(CU, 2 * r + 1 - (offx + EW - xo), r);
                acc[j] = ffma2(make_float2(cw, cw), grow[xo], acc[j]);
              }
            }
          }
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = 8 * g + j;
            if (col < SWx) {
              Zc[(2 * p) * kZPitch + col + sh] = acc[j].x;
              Zc[(2 * p + 1) * kZPitch + col + sh] = acc[j].y;
            }
          }
        }
        __syncthreads();
        // ---- pass B: g_in[gy0 + ey][gx0 + ex] += sum_yo w(ey, yo) Z[yo][ex]
        const int nq = (SWx + sh + 3) >> 2;  // groups of four Z columns (slab columns 4q - sh ..)
        for (int it = tid; it < C * nq * nh; it += kThreads) {
          const int c = it / (nq * nh), rem = it - c * nq * nh;
          const int q = rem % nq, h = rem / nq;
          const float* Zc = Z + (size_t)c * 32 * kZPitch;
          const int tg = offy + 8 * h;        // tap index of (ey = 8h, yo = 0)
          const int klo = max(tg - bh + 1, -7), khi = min(tg, 2 * r);
          float2 acc[8][2];
          #pragma unroll
          for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = make_float2(0.f, 0.f);
          if (klo <= khi) {
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
                if (kk >= klo && kk <= khi) d = *reinterpret_cast<const float4*>(Zc + (tg - kk) * kZPitch + 4 * q);
                const float2 dlo = make_float2(d.x, d.y), dhi = make_float2(d.z, d.w);
                #pragma unroll
                for (int j = 0; j < 8; ++j) {
                  acc[j][0] = ffma2(w[(s + j) & 7], dlo, acc[j][0]);
                  acc[j][1] = ffma2(w[(s + j) & 7], dhi, acc[j][1]);
                }
              }
            }
          }
          // Folded edge rows.
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ey = 8 * h + j;
            const bool ft = foldT && ey == 0, fb = foldB && ey == EH - 1;
            if (ft || fb) {
              for (int yo = 0; yo < bh; ++yo) {
                float cw = 0.f;
                if (ft) cw += cum_at(CU, offy - yo, r);
                if (fb) cw += cum_at(CU, 2 * r + 1 - (offy + EH - yo), r);
                const float4 d = *reinterpret_cast<const float4*>(Zc + yo * kZPitch + 4 * q);
                acc[j][0] = ffma2(make_float2(cw, cw), make_float2(d.x, d.y), acc[j][0]);
                acc[j][1] = ffma2(make_float2(cw, cw), make_float2(d.z, d.w), acc[j][1]);
              }
            }
          }
          float* plane = gin + (size_t)c * planePitch;
          const int col0 = 4 * q - sh;  // slab column of the group's first value
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int ey = 8 * h + j;
            if (ey >= EH) break;
            float* rowp = plane + (size_t)(gy0 + ey) * W + gx0 + X0;
            const float v[4] = {acc[j][0].x, acc[j][0].y, acc[j][1].x, acc[j][1].y};
            if (vec_ok && col0 >= 0 && col0 + 3 < SWx) {
              if (in_bounds(rowp + col0, 16, gin, planePitch * C * 4, ws.counters + CNT_ERROR))
                red_add_f32x4(rowp + col0, v[0], v[1], v[2], v[3]);
            } else {
              #pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int col = col0 + e;
                if (col >= 0 && col < SWx && v[e] != 0.f &&
                    in_bounds(rowp + col, 4, gin, planePitch * C * 4, ws.counters + CNT_ERROR))
                  red_add_f32(rowp + col, v[e]);
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

size_t adjoint_smem_bytes(int rmax) { return smem_layout(rmax).total; }

int adjoint_max_ctas_per_sm(int rmax) {
  const size_t smem = adjoint_smem_bytes(rmax);
  if (set_smem_attrs(reinterpret_cast<const void*>(adjoint_kernel), smem) != cudaSuccess) {
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
  const size_t smem = adjoint_smem_bytes(rmax);
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(adjoint_kernel), smem);
  if (e != cudaSuccess) return e;
  adjoint_kernel<<<grid, kThreads, smem, s>>>(src, ws, rmax);
  return cudaGetLastError();
}

}  // namespace fovea
