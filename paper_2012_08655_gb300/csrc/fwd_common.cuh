// Helpers shared by the two forward kernels (fp32 CUDA-core and tensor-core):
// constants, per-item geometry of the folded halo tile, column slabs, the
// cp.async row ring, and the work-list order of single-frame launches.
#pragma once

#include "fovea_internal.cuh"

namespace fovea {
namespace fwd {

constexpr int kThreads = 256;
constexpr int kSlabMax = 240;                 // elements per slab (ring row <= 15 + 240 + pad)
constexpr int kVVPad = 32;                    // zero columns on each side of a VV row (8 px x 4 ch)
constexpr int kVVPitch = kVVPad + kSlabMax + kVVPad + 1;  // odd pitch: conflict-free row pairs
constexpr int kStages = 3;
constexpr int kRowBytesU8 = 256;              // ring row: 128 pairs of bytes
constexpr int kRowBytesF32 = 1024;            // ring row: 128 pairs of floats
constexpr int kN1 = 16;                       // pass-1 output rows per thread (tap window)

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
  int r, x0, y0, bw, bh;
  int gx0, EW, offx;          // folded columns: frame columns gx0 .. gx0+EW-1, tap offset
  int gy0, EH, offy;          // folded rows
  bool foldL, foldR, foldT, foldB;
  int ph;                     // virtual-row phase: virtual row v holds folded row v - ph
  int vrows;                  // virtual rows staged (multiple of kN1)
  int nsl, sw, nchunks;       // slabs (per channel for f32), slab width, row chunks per slab
  size_t pitch;               // bytes per frame row (u8: W*C, f32: 4*W)
  bool fast;                  // 16-byte aligned rows: cp.async staging
  bool isu8;                  // uint8 HWC (else float32 CHW)
};

struct Slab {
  int c;       // f32: channel of the slab; u8: -1
  int e0, sws; // first element (relative to the folded row) and width
  int ph;      // elements of alignment padding before e0 in the ring row
  size_t src;  // byte offset of element e0 within frame row 0 (plane c for f32)
};

template <bool U8>
__device__ __forceinline__ Slab slab_of(const Item& it, int s) {
  Slab sl;
  const int E = U8 ? it.EW * it.C : it.EW;
  const int ss = U8 ? s : s % it.nsl;
  sl.c = U8 ? -1 : s / it.nsl;
  sl.e0 = ss * it.sw;
  sl.sws = min(it.sw, E - sl.e0);
  if (U8) {
    sl.src = (size_t)it.gx0 * it.C + sl.e0;
  } else {
    sl.src = ((size_t)sl.c * it.H * it.W + it.gx0 + sl.e0) * 4;
  }
  sl.ph = it.fast ? (int)(((size_t)it.in + sl.src) & 15) / (U8 ? 1 : 4) : 0;
  return sl;
}

// Stage rows [k*RB, (k+1)*RB) (virtual) of slab `sl` into one ring stage
// whose rows are ROWB bytes apart.
template <bool U8, int RB, int ROWB = (U8 ? kRowBytesU8 : kRowBytesF32)>
__device__ __forceinline__ void stage_rows(const Item& it, const Slab& sl, int k, unsigned char* ring,
                                           size_t frame_bytes) {
  constexpr int esz = U8 ? 1 : 4;
  constexpr int row_bytes = ROWB;
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
      if (U8) {
        *dst = ok ? __ldg(it.in + off) : (unsigned char)0;
      } else {
        *reinterpret_cast<float*>(dst) = ok ? __ldg(reinterpret_cast<const float*>(it.in + off)) : 0.0f;
      }
    }
    // zero the tail of each row so whole pairs read as zeros
    const int tail0 = sl.sws * esz, tailn = ((tail0 + 15) & ~15) - tail0;
    for (int idx = threadIdx.x; idx < RB * tailn; idx += kThreads) {
      const int row = idx / tailn, b = idx - row * tailn;
      ring[(size_t)row * row_bytes + tail0 + b] = 0;
    }
  }
}

// Per-item geometry from the item record (computed by one thread).
// full_slabs: every slab but the last is as wide as allowed (otherwise the
// slabs share the width evenly); slab_max: elements a slab may hold.
__device__ __forceinline__ void item_geometry(Item& it, const ItemInfo& inf, const FrameDesc& fd, int rb,
                                              bool full_slabs = false, int slab_max = kSlabMax) {
  const bool u8 = fd.fmt == FOVEA_U8_HWC;
  it.in = static_cast<const unsigned char*>(fd.in);
  it.out = static_cast<unsigned char*>(fd.out);
  it.W = fd.W; it.H = fd.H; it.C = fd.C;
  it.isu8 = u8;
  it.r = inf.r;
  const int r = it.r;
  const int tx = inf.block % fd.nbx, ty = inf.block / fd.nbx;  // tile
  const int xs = tx * fd.T - fd.ox, ys = ty * fd.T - fd.oy;    // unclipped tile start
  it.x0 = max(0, xs); it.y0 = max(0, ys);
  it.bw = min(xs + fd.T, it.W) - it.x0; it.bh = min(ys + fd.T, it.H) - it.y0;
  it.gx0 = max(0, it.x0 - r);
  it.EW = min(it.W - 1, it.x0 + it.bw - 1 + r) - it.gx0 + 1;
  it.offx = it.gx0 - (it.x0 - r);
  it.foldL = it.x0 - r < 0; it.foldR = it.x0 + it.bw - 1 + r > it.W - 1;
  it.gy0 = max(0, it.y0 - r);
  it.EH = min(it.H - 1, it.y0 + it.bh - 1 + r) - it.gy0 + 1;
  it.offy = it.gy0 - (it.y0 - r);
  it.foldT = it.y0 - r < 0; it.foldB = it.y0 + it.bh - 1 + r > it.H - 1;
  it.ph = it.offy & (kN1 - 1);
  it.vrows = (it.EH + it.ph + kN1 - 1) & ~(kN1 - 1);
  it.pitch = u8 ? (size_t)it.W * it.C : (size_t)it.W * 4;
  it.fast = (((size_t)it.in & 15) == 0) && ((it.pitch & 15) == 0);
  const int E = u8 ? it.EW * it.C : it.EW;
  const int cap = u8 ? (slab_max / it.C) * it.C : slab_max;
  const int nsl = (E + cap - 1) / cap;
  int sw = full_slabs && nsl > 1 ? cap : (E + nsl - 1) / nsl;
  if (u8) sw = ((sw + it.C - 1) / it.C) * it.C;
  it.nsl = nsl;
  it.sw = sw;
  it.nchunks = (it.vrows + rb - 1) / rb;
}

// Descending exclusive prefix of the radius histogram: start[b] is the first
// ticket of radius b when tickets are handed out largest radius first. NT:
// threads of the CTA (wsum holds NT / 32 ints).
template <int NT = kThreads>
__device__ __forceinline__ void bucket_starts(const unsigned int* hist, int nb, int* start, int* wsum) {
  constexpr int per = kBuckets / NT;  // positions per thread
  unsigned int v[per], run = 0;
  #pragma unroll
  for (int j = 0; j < per; ++j) {
    const int pos = threadIdx.x * per + j, b = nb - 1 - pos;
    v[j] = b >= 0 ? hist[b] : 0u;
    run += v[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int incl = run;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) wsum[warp] = (int)incl;
  __syncthreads();
  unsigned int acc = incl - run;
  for (int w = 0; w < warp; ++w) acc += (unsigned int)wsum[w];
  #pragma unroll
  for (int j = 0; j < per; ++j) {
    const int pos = threadIdx.x * per + j, b = nb - 1 - pos;
    if (b >= 0) start[b] = (int)acc;
    acc += v[j];
  }
  __syncthreads();
}

}  // namespace fwd
}  // namespace fovea
