// Forward foveation kernel: one persistent CTA loop over (frame, block) items.
//
// For one block (paper Section 2 and Algorithm 1: "place padded fragment into
// shared memory", "horizontal convolution", "place result into shared
// memory", "vertical convolution", "write result"):
//   * taps: the block's normalised 1D Gaussian (Eq. 1, truncated at
//     r = ceil(3 sigma)), generated in the CTA and summed with warp shuffles,
//     plus their exclusive prefix sums;
//   * folded halo tile: only the in-frame rows y0-r .. y0+bh-1+r and columns
//     x0-r .. x0+bw-1+r are staged; the taps that clamp-to-edge sends to a
//     position outside the frame are folded onto the edge row / column with
//     one prefix-summed weight (exact in real arithmetic);
//   * staging: rows stream through a 3-stage shared-memory ring filled with
//     16-byte cp.async copies, so the loads of later rows overlap the
//     arithmetic on earlier ones; uint8 is unpacked exactly in registers;
//   * pass 1 (vertical, halo rows): V[yo][e] = sum_y u[y - yo] T[y][e] for the
//     32 output rows and every tile element column e (pixel x channel);
//   * pass 2 (horizontal): O[yo][x][c] = sum_x' u[x' - x] V[yo][x'][c];
//   * round/pack and store.
// The vertical pass runs first so the tile can stream by rows: shared memory
// does not grow with the radius. Wide tiles are cut into column slabs and
// pass 2 accumulates across slabs. All products are fp32 FMAs, two lanes per
// instruction (fma.rn.f32x2); a thread keeps 8 outputs per value it loads and
// a sliding window of 8 taps in registers (the register data reuse of the
// paper's "Data Reuse" subsection, generalised).
#include "fovea_internal.cuh"

namespace fovea {

namespace {

constexpr int kThreads = 256;
constexpr int kSlabMax = 240;           // elements per slab (ring row <= 15 + 240 + pad)
constexpr int kVVPitch = kSlabMax + 1;  // float2 pitch of the row-pair buffer (odd: conflict-free)
constexpr int kStages = 3;
constexpr int kRowBytesU8 = 256;        // ring row: 64 words of 4 bytes
constexpr int kRowBytesF32 = 1024;      // ring row: 64 quads of 4 floats

struct SmemLayout {
  size_t ring, vv, taps, cum, red, total;
};

__host__ __device__ inline SmemLayout smem_layout(int rb, int row_bytes, int rmax) {
  SmemLayout L;
  L.ring = 0;
  L.vv = L.ring + (size_t)kStages * rb * row_bytes;
  L.taps = L.vv + (size_t)16 * kVVPitch * sizeof(float2);
  L.cum = L.taps + (size_t)tap_len(rmax) * sizeof(float2);
  L.red = L.cum + (size_t)cum_len(rmax) * sizeof(float);
  L.total = L.red + 32 * sizeof(float);
  return L;
}

__device__ __forceinline__ unsigned char quant_u8(float v) {
  int q = __float2int_rd(v + 0.5f);
  q = q < 0 ? 0 : (q > 255 ? 255 : q);
  return (unsigned char)q;
}

// Geometry of one item (identical in every thread).
struct Item {
  const unsigned char* in;
  unsigned char* out;
  int W, H, C;
  bool u8;
  int r, x0, y0, bw, bh;
  int gx0, EW, offx;          // folded columns: frame columns gx0 .. gx0+EW-1, tap offset
  int gy0, EH, offy;          // folded rows
  bool foldL, foldR, foldT, foldB;
  int ph;                     // virtual-row phase: virtual row v holds folded row v - ph
  int vrows;                  // virtual rows staged (multiple of 8)
  int steps;                  // 8-tap steps covering 2r + 8 taps
  int nsl, sw, nchunks;       // slabs (per channel for f32), slab width, row chunks per slab
  size_t pitch;               // bytes per frame row (u8: W*C, f32: 4*W)
  bool fast;                  // 16-byte aligned rows: cp.async staging
};

struct Slab {
  int c;       // f32: channel of the slab; u8: -1
  int e0, sws; // first element (relative to the folded row) and width
  int ph;      // elements of alignment padding before e0 in the ring row
  size_t src;  // byte offset of element e0 within frame row 0 (plane c for f32)
};

__device__ __forceinline__ Slab slab_of(const Item& it, int s) {
  Slab sl;
  const int E = it.u8 ? it.EW * it.C : it.EW;
  const int ss = it.u8 ? s : s % it.nsl;
  sl.c = it.u8 ? -1 : s / it.nsl;
  sl.e0 = ss * it.sw;
  sl.sws = min(it.sw, E - sl.e0);
  if (it.u8) {
    sl.src = (size_t)it.gx0 * it.C + sl.e0;
  } else {
    sl.src = ((size_t)sl.c * it.H * it.W + it.gx0 + sl.e0) * 4;
  }
  sl.ph = it.fast ? (int)(((size_t)it.in + sl.src) & 15) / (it.u8 ? 1 : 4) : 0;
  return sl;
}

// Stage rows [k*RB, (k+1)*RB) (virtual) of slab `sl` into one ring stage.
template <int RB>
__device__ __forceinline__ void stage_rows(const Item& it, const Slab& sl, int k, unsigned char* ring,
                                           int row_bytes, size_t frame_bytes) {
  const int esz = it.u8 ? 1 : 4;
  if (it.fast) {
    const int nch = (sl.ph * esz + sl.sws * esz + 15) >> 4;  // 16-byte copies per row
    for (int idx = threadIdx.x; idx < RB * nch; idx += kThreads) {
      const int row = idx / nch, ch = idx - row * nch;
      const int v = k * RB + row;
      const int ey = v - it.ph;
      unsigned char* dst = ring + (size_t)row * row_bytes + ch * 16;
      if (v < it.vrows && ey >= 0 && ey < it.EH) {
        const size_t off = (size_t)(it.gy0 + ey) * it.pitch + sl.src - (size_t)sl.ph * esz + (size_t)ch * 16;
        const size_t rem = off < frame_bytes ? frame_bytes - off : 0;
        const int nbytes = rem >= 16 ? 16 : (int)rem;
        cp_async16(dst, nbytes > 0 ? it.in + off : it.in, nbytes);
      } else {
        cp_async16(dst, it.in, 0);
      }
    }
  } else {
    // Rows not 16-byte aligned: plain loads, element e at ring position e.
    const int n = RB * sl.sws;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
      const int row = idx / sl.sws, e = idx - row * sl.sws;
      const int v = k * RB + row;
      const int ey = v - it.ph;
      const bool ok = v < it.vrows && ey >= 0 && ey < it.EH;
      const size_t off = (size_t)(it.gy0 + (ok ? ey : 0)) * it.pitch + sl.src + (size_t)e * esz;
      unsigned char* dst = ring + (size_t)row * row_bytes + (size_t)e * esz;
      if (it.u8) {
        *dst = ok ? __ldg(it.in + off) : (unsigned char)0;
      } else {
        *reinterpret_cast<float*>(dst) = ok ? __ldg(reinterpret_cast<const float*>(it.in + off)) : 0.0f;
      }
    }
    // zero the tail of each row so whole words/quads read as zeros
    const int tail0 = sl.sws * esz, tailn = ((tail0 + 15) & ~15) - tail0;
    for (int idx = threadIdx.x; idx < RB * tailn; idx += kThreads) {
      const int row = idx / tailn, b = idx - row * tailn;
      ring[(size_t)row * row_bytes + tail0 + b] = 0;
    }
  }
}

template <int RB>
__global__ void __launch_bounds__(kThreads, 2)
forward_kernel(FrameSource src, Workspace ws, int rmax, int row_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(RB, row_bytes, rmax);
  unsigned char* ring = smem + L.ring;
  float2* VV = reinterpret_cast<float2*>(smem + L.vv);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_ticket;

  const int tid = threadIdx.x;
  const int n_items = (int)ws.counters[CNT_NITEMS];
  const size_t stage_bytes = (size_t)RB * row_bytes;
  // pass-1 identity: ring word/quad w1i, row group G1 of 8 output rows
  const int w1i = tid & 63, G1 = tid >> 6;
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
    if (inf.r > rmax || (fd.fmt != FOVEA_U8_HWC && row_bytes < kRowBytesF32)) {
      if (tid == 0) atomicOr(&ws.counters[CNT_ERROR], 2u);
      continue;
    }
    Item it;
    it.in = static_cast<const unsigned char*>(fd.in);
    it.out = static_cast<unsigned char*>(fd.out);
    it.W = fd.W; it.H = fd.H; it.C = fd.C;
    it.u8 = fd.fmt == FOVEA_U8_HWC;
    it.r = inf.r;
    const int r = it.r;
    {
      const int bx = inf.block % fd.nbx, by = inf.block / fd.nbx;
      it.x0 = bx * fd.B; it.y0 = by * fd.B;
      it.bw = min(fd.B, it.W - it.x0); it.bh = min(fd.B, it.H - it.y0);
    }
    it.gx0 = max(0, it.x0 - r);
    it.EW = min(it.W - 1, it.x0 + it.bw - 1 + r) - it.gx0 + 1;
    it.offx = it.gx0 - (it.x0 - r);
    it.foldL = it.x0 - r < 0; it.foldR = it.x0 + it.bw - 1 + r > it.W - 1;
    it.gy0 = max(0, it.y0 - r);
    it.EH = min(it.H - 1, it.y0 + it.bh - 1 + r) - it.gy0 + 1;
    it.offy = it.gy0 - (it.y0 - r);
    it.foldT = it.y0 - r < 0; it.foldB = it.y0 + it.bh - 1 + r > it.H - 1;
    it.ph = it.offy & 7;
    it.vrows = (it.EH + it.ph + 7) & ~7;
    it.steps = 1 + ((2 * r + 7) >> 3);
    it.pitch = it.u8 ? (size_t)it.W * it.C : (size_t)it.W * 4;
    it.fast = (((size_t)it.in & 15) == 0) && ((it.pitch & 15) == 0);
    {
      const int E = it.u8 ? it.EW * it.C : it.EW;
      const int cap = it.u8 ? (kSlabMax / it.C) * it.C : kSlabMax;
      const int nsl = (E + cap - 1) / cap;
      int sw = (E + nsl - 1) / nsl;
      if (it.u8) sw = ((sw + it.C - 1) / it.C) * it.C;
      it.nsl = nsl;
      it.sw = sw;
    }
    it.nchunks = (it.vrows + RB - 1) / RB;
    const int nslabs = it.u8 ? it.nsl : it.nsl * it.C;
    const int Q = nslabs * it.nchunks;
    const size_t frame_bytes = (size_t)it.H * it.pitch * (it.u8 ? 1 : it.C);

    // Start staging before the taps are ready: the copies do not need them.
    #pragma unroll
    for (int q = 0; q < kStages - 1; ++q) {
      if (q < Q) stage_rows<RB>(it, slab_of(it, q / it.nchunks), q % it.nchunks, ring + (size_t)q * stage_bytes,
                                row_bytes, frame_bytes);
      cp_async_commit();
    }
    make_taps(U, tap_len(r), r, inf.neg_half_inv_s2, red);
    make_cumulative(U, CU, r);
    __syncthreads();

    const int groups1 = (it.bh + 7) >> 3, groups2 = (it.bw + 7) >> 3;
    // pass-1 row range of this thread's group in virtual rows (8-aligned)
    const int vs1 = 8 * G1 - it.offy + it.ph;
    const int v1lo = max(0, vs1), v1hi = min(it.vrows, vs1 + 8 * it.steps);
    const bool grp1 = G1 < groups1;
    const int xg = 8 * g2;
    const bool act2base = g2 < groups2 && c2 < it.C && 2 * p2 < it.bh;
    float2 acc2[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) acc2[j] = make_float2(0.f, 0.f);
    float2 a1[8][2];
    float2 wv[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) wv[j] = make_float2(0.f, 0.f);

    for (int q = 0; q < Q; ++q) {
      cp_async_wait<kStages - 2>();
      __syncthreads();  // chunk q landed for every thread; chunk q-1 fully consumed
      {
        const int qn = q + kStages - 1;
        if (qn < Q) stage_rows<RB>(it, slab_of(it, qn / it.nchunks), qn % it.nchunks,
                                   ring + (size_t)(qn % kStages) * stage_bytes, row_bytes, frame_bytes);
        cp_async_commit();
      }
      const int s = q / it.nchunks, k = q - s * it.nchunks;
      const Slab sl = slab_of(it, s);
      const unsigned char* st = ring + (size_t)(q % kStages) * stage_bytes;
      // ring word/quad w1i holds slab elements 4*w1i - ph .. +3
      const int e_first = 4 * w1i - sl.ph;
      const bool act1 = grp1 && e_first + 3 >= 0 && e_first < sl.sws;
      if (k == 0) {
        #pragma unroll
        for (int j = 0; j < 8; ++j) a1[j][0] = a1[j][1] = make_float2(0.f, 0.f);
      }
      if (act1) {
        const int R0 = k * RB;
        const int lo = max(R0, v1lo), hi = min(R0 + RB, v1hi);
        if (lo < hi && lo == v1lo) {  // first row of the group: preload the tap window
          #pragma unroll
          for (int u = 1; u < 8; ++u) wv[u] = U[kTapPad + (lo - vs1) - 8 + u];
        }
        for (int v0 = lo; v0 < hi; v0 += 8) {
          #pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int v = v0 + u;
            wv[u] = U[kTapPad + v - vs1];
            float2 dlo, dhi;
            if (it.u8) {
              const unsigned int wd = *reinterpret_cast<const unsigned int*>(st + (size_t)(v - R0) * row_bytes + 4 * w1i);
              u8x4_to_f32(wd, dlo, dhi);
            } else {
              const float4 d = *reinterpret_cast<const float4*>(st + (size_t)(v - R0) * row_bytes + 16 * w1i);
              dlo = make_float2(d.x, d.y);
              dhi = make_float2(d.z, d.w);
            }
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
              a1[j][0] = ffma2(wv[(u - j) & 7], dlo, a1[j][0]);
              a1[j][1] = ffma2(wv[(u - j) & 7], dhi, a1[j][1]);
            }
          }
        }
        // Folded edge rows: the taps clamped onto the first / last frame row.
        #pragma unroll
        for (int f = 0; f < 2; ++f) {
          const bool on = f == 0 ? it.foldT : it.foldB;
          const int v = f == 0 ? it.ph : it.ph + it.EH - 1;
          if (on && v >= R0 && v < R0 + RB) {
            float2 dlo, dhi;
            if (it.u8) {
              const unsigned int wd = *reinterpret_cast<const unsigned int*>(st + (size_t)(v - R0) * row_bytes + 4 * w1i);
              u8x4_to_f32(wd, dlo, dhi);
            } else {
              const float4 d = *reinterpret_cast<const float4*>(st + (size_t)(v - R0) * row_bytes + 16 * w1i);
              dlo = make_float2(d.x, d.y);
              dhi = make_float2(d.z, d.w);
            }
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int yo = 8 * G1 + j;
              const float cw = f == 0 ? cum_at(CU, it.offy - yo, r) : cum_at(CU, 2 * r + 1 - (it.offy + it.EH - yo), r);
              const float2 w2 = make_float2(cw, cw);
              a1[j][0] = ffma2(w2, dlo, a1[j][0]);
              a1[j][1] = ffma2(w2, dhi, a1[j][1]);
            }
          }
        }
      }
      if (k != it.nchunks - 1) continue;

      // ---- slab complete: V rows -> row-pair buffer, then pass 2 over the slab
      if (act1) {
        #pragma unroll
        for (int pp = 0; pp < 4; ++pp) {
          float2* dst = VV + (4 * G1 + pp) * kVVPitch;
          const float v0[4] = {a1[2 * pp][0].x, a1[2 * pp][0].y, a1[2 * pp][1].x, a1[2 * pp][1].y};
          const float v1[4] = {a1[2 * pp + 1][0].x, a1[2 * pp + 1][0].y, a1[2 * pp + 1][1].x, a1[2 * pp + 1][1].y};
          #pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e_first + u;
            if (e >= 0 && e < sl.sws) dst[e] = make_float2(v0[u], v1[u]);
          }
        }
      }
      __syncthreads();
      const bool act2 = act2base && (it.u8 || c2 == sl.c);
      if (act2) {
        const int Cs = it.u8 ? it.C : 1;
        const int P0 = sl.e0 / Cs, P1 = P0 + sl.sws / Cs;  // folded columns of the slab
        const int xs = xg - it.offx;                         // column whose tap index is 0 for x = xg
        const int lo = max(P0, xs), hi = min(P1, xs + 8 * it.steps);
        const float2* vrow = VV + p2 * kVVPitch + (it.u8 ? c2 : 0);
        if (lo < hi) {
          const int la = lo - ((lo - xs) & 7);
          float2 w2[8];
          #pragma unroll
          for (int u = 1; u < 8; ++u) w2[u] = U[kTapPad + (la - xs) - 8 + u];
          for (int x0c = la; x0c < hi; x0c += 8) {
            #pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int ex = x0c + u;
              w2[u] = U[kTapPad + ex - xs];
              float2 d = make_float2(0.f, 0.f);
              if (ex >= lo && ex < hi) d = vrow[(ex - P0) * Cs];
              #pragma unroll
              for (int j = 0; j < 8; ++j) acc2[j] = ffma2(w2[(u - j) & 7], d, acc2[j]);
            }
          }
        }
        // Folded edge columns.
        #pragma unroll
        for (int f = 0; f < 2; ++f) {
          const bool on = f == 0 ? it.foldL : it.foldR;
          const int ex = f == 0 ? 0 : it.EW - 1;
          if (on && ex >= P0 && ex < P1) {
            const float2 d = vrow[(ex - P0) * Cs];
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int x = xg + j;
              const float cw = f == 0 ? cum_at(CU, it.offx - x, r) : cum_at(CU, 2 * r + 1 - (it.offx + it.EW - x), r);
              acc2[j] = ffma2(make_float2(cw, cw), d, acc2[j]);
            }
          }
        }
      }
    }
    cp_async_wait<0>();
    __syncthreads();  // ring no longer read; it becomes the output stage

    if (!it.u8) {
      if (act2base) {
        float* out = reinterpret_cast<float*>(it.out) + (size_t)c2 * it.W * it.H +
                     (size_t)(it.y0 + 2 * p2) * it.W + it.x0;
        const bool second = 2 * p2 + 1 < it.bh;
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = xg + j;
          if (x < it.bw) {
            out[x] = acc2[j].x;
            if (second) out[it.W + x] = acc2[j].y;
          }
        }
      }
    } else {
      unsigned char* ost = ring;
      const int opitch = 32 * it.C;
      if (act2base) {
        #pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int x = xg + j;
          ost[(2 * p2) * opitch + x * it.C + c2] = quant_u8(acc2[j].x);
          ost[(2 * p2 + 1) * opitch + x * it.C + c2] = quant_u8(acc2[j].y);
        }
      }
      __syncthreads();
      const int rowBytes = it.bw * it.C;
      unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * it.C;
      for (int idx = tid; idx < it.bh * rowBytes; idx += kThreads) {
        const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
        out[(size_t)yo * it.pitch + rem] = ost[yo * opitch + rem];
      }
    }
  }
  cp_async_wait<0>();
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

size_t forward_smem_bytes(const FwdConfig& cfg, int rmax, bool any_f32) {
  return smem_layout(cfg.rows_per_chunk, any_f32 ? kRowBytesF32 : kRowBytesU8, rmax).total;
}

int forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, bool any_f32) {
  const size_t smem = forward_smem_bytes(cfg, rmax, any_f32);
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
                           int rmax, bool any_f32, int grid, cudaStream_t s) {
  const size_t smem = forward_smem_bytes(cfg, rmax, any_f32);
  int row_bytes = any_f32 ? kRowBytesF32 : kRowBytesU8;
  void* k = pick_kernel(cfg.rows_per_chunk);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &row_bytes};
  return cudaLaunchKernel(k, dim3(grid), dim3(kThreads), args, smem, s);
}

}  // namespace fovea
