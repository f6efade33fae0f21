// Pieces shared by the tensor-core forward kernels (tc_forward.cu: both
// passes on mma.sync; umma_forward.cu: pass 1 on tcgen05 with its
// accumulator in tensor memory): scaling constants of the fp16 hi/lo split,
// the TMA row ring (tensor-map boxes, 128-byte swizzle, mbarriers with
// bounded waits), the per-item tap tables, the mma.sync helpers, and the
// persistent item loop with its one-item lookahead.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "fwd_common.cuh"

namespace fovea {
namespace tcc {

using namespace fwd;

constexpr float kWScale = 4096.0f;          // taps scaled by 2^12
constexpr float kWInv = 1.0f / 4096.0f;
constexpr float kDScale = 1.0f / 16777216.0f;  // a staged byte b enters pass 1 as b * 2^-24
constexpr float kVScale = 4096.0f;          // V = pass-1 accumulator * 2^12 (= 2^24 / 2^12)
constexpr int kRingRow = 256;               // bytes per staged row of the 8-warp kernels: two 128-byte boxes
constexpr int kPairPad = 32;                // tap index -kPairPad is pair entry 0

// Shapes of the mma.sync kernel with NW warps (NW = 4, 8 or 16): in pass 1
// warp w owns staged bytes 32w .. 32w+31, so a staged row is 32 NW bytes
// (NW / 4 tensor-map boxes of 128 bytes) and a slab holds up to 32 NW - 16
// bytes (the row also holds up to 15 bytes of alignment padding).
template <int NW>
struct TcDims {
  static_assert(NW == 4 || NW == 8 || NW == 16, "4, 8 or 16 warps");
  static constexpr int NT = 32 * NW;
  static constexpr int ROW = 32 * NW;
  static constexpr int BOXES = NW / 4;
  static constexpr int SLAB = ROW - 16;
};

// Pitch (halves) of the pass-2 operand rows V[(c, yo)][p] for C channels and
// NW warps: the slab's pixels rounded up to 16, then to an odd multiple of 8
// halves (16 bytes), so the 8 rows an ldmatrix reads fall in distinct banks.
__host__ __device__ constexpr int tc_vp(int C, int NW) {
  return ((((32 * NW - 16) / C + 15) / 16 * 16) / 8) % 2 ? (((32 * NW - 16) / C + 15) / 16 * 16)
                                                          : (((32 * NW - 16) / C + 15) / 16 * 16) + 8;
}
__host__ __device__ constexpr int tc_vmax(int a, int b) { return a > b ? a : b; }
// Halves of one V array: the largest 32 C x VP over C = 1 .. 4.
__host__ __device__ constexpr int tc_vhalves(int NW) {
  return tc_vmax(tc_vmax(32 * tc_vp(1, NW), 64 * tc_vp(2, NW)), tc_vmax(96 * tc_vp(3, NW), 128 * tc_vp(4, NW)));
}
// Pass-2 units (16-row m-tile x 8-column n-tile) per warp: the 2C x 4 units
// of an item dealt to NW warps, unit u to warp u mod NW.
__host__ __device__ constexpr int tc_units(int C, int NW) { return (8 * C + NW - 1) / NW; }

__host__ __device__ inline int npair(int rmax) { return rmax + 56; }

// Raw uint8 row chunks staged or in flight: about 160 rows (at least three
// chunks), so that a chunk's load has several chunks' worth of work to hide
// behind.
__host__ __device__ constexpr int tc_stages(int rb) { return 160 / rb > 3 ? 160 / rb : 3; }
constexpr int kMaxTcStages = 10;

// Byte b (0..255) of staged row rho of a ring stage: box b / 128, 128-byte
// rows, 16-byte chunk index XOR (rho mod 8).
template <int RB>
__device__ __forceinline__ int ring_off(int rho, int b) {
  return (((b >> 7) * RB + rho) << 7) + ((((b >> 4) & 7) ^ (rho & 7)) << 4) + (b & 15);
}

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the given phase parity of an mbarrier, at most kWaitLimit polls
// (each poll may suspend for a short, hardware-chosen time). False: gave up.
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One 2D tensor-map box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// A tensor map in global memory is rewritten (by a host copy) between
// launches: order those generic writes before its use by the tensor-map
// proxy, which may otherwise hold the previous contents.
__device__ __forceinline__ void fence_tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(map) : "memory");
}

__device__ __forceinline__ unsigned int pack_half2(__half a, __half b) {
  return (unsigned int)__half_as_ushort(a) | ((unsigned int)__half_as_ushort(b) << 16);
}


// No side effects: left to the compiler to schedule (independent chains interleave).
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned int (&a)[4], unsigned int b0, unsigned int b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned int (&r)[4], const void* p) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

// Unnormalised tap of offset d: exp(c d^2) (c = -1 / (2 sigma^2)), 1 at d = 0.
__device__ __forceinline__ float tap_w(int d, float c) { return d == 0 ? 1.0f : expf(c * (float)(d * d)); }

// Sum S of the unnormalised taps over |d| <= r, computed by every warp on
// its own in one fixed order (lane-strided partial sums, then a butterfly,
// which leaves the same value in every lane), so every warp holds the same S
// without a block-wide barrier.
__device__ __forceinline__ float warp_tap_sum(int r, float c) {
  const int lane = threadIdx.x & 31;
  float s = 0.0f;
  for (int d = -r + lane; d <= r; d += 32) s += tap_w(d, c);
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Normalised tap of index m (offset m - r), zero outside [0, 2r].
__device__ __forceinline__ float tap_u(int m, int r, float c, float S) {
  return (m >= 0 && m <= 2 * r) ? tap_w(m - r, c) / S : 0.0f;
}

// Tap-pair tables: entry j of the even table holds (w(m), w(m+1)) with
// m = 2j - kPairPad, the odd table the pair starting one tap later; hi and lo
// parts of the scaled taps w = u * 2^12. NT: threads of the CTA.
template <int NT = kThreads>
__device__ __forceinline__ void make_pairs(unsigned int* P, int r, float c, float S, int np) {
  unsigned int* PEh = P;
  unsigned int* POh = P + np;
  unsigned int* PEl = P + 2 * np;
  unsigned int* POl = P + 3 * np;
  for (int j = threadIdx.x; j < np; j += NT) {
    __half h[3], l[3];
    #pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float w = tap_u(2 * j - kPairPad + q, r, c, S) * kWScale;
      h[q] = __float2half_rn(w);
      l[q] = __float2half_rn(w - __half2float(h[q]));
    }
    PEh[j] = pack_half2(h[0], h[1]);
    POh[j] = pack_half2(h[1], h[2]);
    PEl[j] = pack_half2(l[0], l[1]);
    POl[j] = pack_half2(l[1], l[2]);
  }
}

// Exclusive prefix sums of the normalised taps, CU[m] = sum_{m' < m} u(m')
// for m in [0, 2r+1] (used to fold clamped taps onto edge rows/columns, as
// in the fp32 kernel). One warp: contiguous lane segments, then a scan.
__device__ __forceinline__ void make_cumulative_tc(float* CU, int r, float c, float S) {
  const int lane = threadIdx.x & 31;
  const int n = 2 * r + 1;
  const int seg = (n + 31) >> 5;
  const int b = lane * seg, e = min(n, b + seg);
  float sum = 0.0f;
  for (int m = b; m < e; ++m) sum += tap_u(m, r, c, S);
  float incl = sum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  float run = incl - sum;
  for (int m = b; m < e; ++m) {
    CU[m] = run;
    run += tap_u(m, r, c, S);
  }
  if (lane == 31) CU[n] = incl;
}

// Everything the tensor-core kernel does for one item with C channels.
// Pass 2 of one slab on mma.sync: O[(c,yo)][x] += sum_p V[(c,yo)][p] Wh[p][x]
// over the slab's pixels, V as hi/lo fp16 (Vhi Whi + Vhi Wlo + Vlo Whi), the tap pairs from the tables P; the folded
// left column (first slab) is added before and the folded right column after
// the products. Warp w owns units u = w + 8i (row tile u / 4, column tile
// u % 4) and accumulates them in acc2[i] across slabs.
//
// Two layouts of V: VT = false, row (c, yo) = 32 c + yo of pitch VP, pixels
// contiguous; VT = true, row (px, c) = C px + c of kVtPitch halves, the 32
// output rows contiguous (fragments then come from ldmatrix.trans).
constexpr int kVtPitch = 40;  // 32 rows + 8: row starts 20 words apart, conflict-free for odd C

__device__ __forceinline__ void ldsm_x4_t(unsigned int (&r)[4], const void* p) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

template <int C, bool VT, int NW = 8>
__device__ __forceinline__ size_t v_index(int c, int yo, int px) {
  return VT ? (size_t)(px * C + c) * kVtPitch + yo : (size_t)(c * 32 + yo) * tc_vp(C, NW) + px;
}

// Unit i of a warp (u = warp + NW i) exists: 8 C units are dealt to NW warps.
template <int C, int NW>
__device__ __forceinline__ bool tc_unit_exists(int warp, int i) {
  return (8 * C) % NW == 0 ? true : warp + NW * i < 8 * C;
}

// FLUSH: each k-step's products go into a zeroed fragment that is added to
// acc2 in fp32 (round to nearest) instead of accumulating in the MMA, whose
// adds truncate; needed where the result is not rounded to 8 bits.
template <int C, bool VT = false, int NW = 8, bool FLUSH = false>
__device__ __forceinline__ void tc_pass2_slab(const Item& it, const Slab& sl, const __half* Vh, const __half* Vl,
                                              const float* CU, const unsigned int* P, int np,
                                              float (&acc2)[tc_units(C, NW)][4]) {
  constexpr int VP = tc_vp(C, NW);
  constexpr int U = tc_units(C, NW);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r = it.r;
  const int npx = sl.sws / C;
  const int npx16 = (npx + 15) & ~15;
  const int P0 = sl.e0 / C;  // first folded pixel of the slab
  // tap index of this lane's B registers has the parity of offx + P0 - g
  const int par2 = (it.offx + P0 + g) & 1;
  const unsigned int* Qh = P + (par2 ? np : 0);
  const unsigned int* Ql = P + 2 * np + (par2 ? np : 0);
  if (it.foldL && P0 == 0) {  // folded left column first: fixed summation order
    #pragma unroll
    for (int i = 0; i < U; ++i) {
      const int u = warp + NW * i;
      if (!tc_unit_exists<C, NW>(warp, i)) continue;
      const int mt2 = u >> 2, nt2 = u & 3;
      #pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = 16 * mt2 + g + 8 * h;
        const size_t o = v_index<C, VT, NW>(row >> 5, row & 31, 0);
        const float v = __half2float(Vh[o]) + __half2float(Vl[o]);
        #pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int x = 8 * nt2 + 2 * t + cc;
          acc2[i][2 * h + cc] = fmaf(cum_at(CU, it.offx - x, r) * kWScale, v, acc2[i][2 * h + cc]);
        }
      }
    }
  }
  // this warp's n-tile: u = warp + NW i has u & 3 = warp & 3 for every i (NW
  // is a multiple of 4), so the tap fragments of a k-step are shared by the
  // warp's m-tiles
  const int nt2w = warp & 3;
  for (int kk = 0; kk < npx16; kk += 16) {
    unsigned int a_h[U][4], a_l[U][4], bh[2], bl[2];
    {
      const int jb = (it.offx + P0 + kk + 2 * t - 8 * nt2w - g + kPairPad) >> 1;
      bh[0] = Qh[jb]; bh[1] = Qh[jb + 4];
      bl[0] = Ql[jb]; bl[1] = Ql[jb + 4];
    }
    #pragma unroll
    for (int i = 0; i < U; ++i) {
      if (!tc_unit_exists<C, NW>(warp, i)) continue;
      const int u = warp + NW * i;
      const int mt2 = u >> 2;
      if (VT) {  // stored rows are pixels: transpose on load
        const int m0 = 16 * mt2 + ((lane >> 3) & 1) * 8;
        const int krow = kk + (lane & 7) + ((lane >> 4) & 1) * 8;
        const size_t o = v_index<C, true, NW>(m0 >> 5, m0 & 31, krow);
        ldsm_x4_t(a_h[i], Vh + o);
        ldsm_x4_t(a_l[i], Vl + o);
      } else {
        const int arow = 16 * mt2 + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int acol = kk + ((lane >> 4) & 1) * 8;
        ldsm_x4(a_h[i], Vh + (size_t)arow * VP + acol);
        ldsm_x4(a_l[i], Vl + (size_t)arow * VP + acol);
      }
    }
    if (FLUSH) {
      #pragma unroll
      for (int i = 0; i < U; ++i) {
        if (!tc_unit_exists<C, NW>(warp, i)) continue;
        float tmp[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(tmp, a_h[i], bh[0], bh[1]);
        mma16816(tmp, a_h[i], bl[0], bl[1]);
        mma16816(tmp, a_l[i], bh[0], bh[1]);
        #pragma unroll
        for (int e = 0; e < 4; ++e) acc2[i][e] += tmp[e];
      }
    } else {
      #pragma unroll
      for (int i = 0; i < U; ++i)
        if (tc_unit_exists<C, NW>(warp, i)) mma16816(acc2[i], a_h[i], bh[0], bh[1]);
      #pragma unroll
      for (int i = 0; i < U; ++i)
        if (tc_unit_exists<C, NW>(warp, i)) mma16816(acc2[i], a_h[i], bl[0], bl[1]);
      #pragma unroll
      for (int i = 0; i < U; ++i)
        if (tc_unit_exists<C, NW>(warp, i)) mma16816(acc2[i], a_l[i], bh[0], bh[1]);
    }
  }
  {
    const int pr = it.EW - 1 - P0;  // folded right column after the last slab's products
    if (it.foldR && pr >= 0 && pr < npx) {
      #pragma unroll
      for (int i = 0; i < U; ++i) {
        if (!tc_unit_exists<C, NW>(warp, i)) continue;
        const int u = warp + NW * i;
        const int mt2 = u >> 2, nt2 = u & 3;
        #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = 16 * mt2 + g + 8 * h;
          const size_t o = v_index<C, VT, NW>(row >> 5, row & 31, pr);
          const float v = __half2float(Vh[o]) + __half2float(Vl[o]);
          #pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int x = 8 * nt2 + 2 * t + cc;
            acc2[i][2 * h + cc] = fmaf(cum_at(CU, 2 * r + 1 - (it.offx + it.EW - x), r) * kWScale, v, acc2[i][2 * h + cc]);
          }
        }
      }
    }
  }
}

// Rounds the item's outputs (acc2, scaled by 2^12) to uint8, stages them in
// ost (32 rows of 32 C bytes) and writes the block's rows with 16-byte
// stores where the frame's alignment allows. fault: the fault word that
// bounds-checked builds report stray stores in.
template <int C, int NW = 8>
__device__ __forceinline__ void tc_write_output(const Item& it, unsigned char* ost,
                                                const float (&acc2)[tc_units(C, NW)][4], unsigned int* fault) {
  constexpr int NT = TcDims<NW>::NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  constexpr int opitch = 32 * C;
  #pragma unroll
  for (int i = 0; i < tc_units(C, NW); ++i) {
    const int u = warp + NW * i;
    if (u >= 8 * C) continue;
    const int mt2 = u >> 2, nt2 = u & 3;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = 16 * mt2 + g + ((e >> 1) << 3);
      const int c = row >> 5, yo = row & 31;
      const int x = 8 * nt2 + 2 * t + (e & 1);
      unsigned char* o = ost + yo * opitch + x * C + c;
      if (smem_in_bounds(o, 1, fault)) *o = quant_u8(acc2[i][e] * kWInv);
    }
  }
  __syncthreads();
  const int rowBytes = it.bw * C;
  const size_t frame_bytes = (size_t)it.H * it.pitch;
  unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * C;
  if (((((size_t)out) | it.pitch | (size_t)rowBytes) & 15) == 0) {
    const int nv = rowBytes >> 4;  // 16-byte pieces per row
    for (int idx = tid; idx < it.bh * nv; idx += NT) {
      const int yo = idx / nv, v = idx - yo * nv;
      uint4* o = reinterpret_cast<uint4*>(out + (size_t)yo * it.pitch + 16 * v);
      if (in_bounds(o, 16, it.out, frame_bytes, fault)) *o = *reinterpret_cast<const uint4*>(ost + yo * opitch + 16 * v);
    }
  } else {
    for (int idx = tid; idx < it.bh * rowBytes; idx += NT) {
      const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
      unsigned char* o = out + (size_t)yo * it.pitch + rem;
      if (in_bounds(o, 1, it.out, frame_bytes, fault)) *o = ost[yo * opitch + rem];
    }
  }
}

// Persistent item loop of the tensor-core kernels. Thread 0 takes tickets
// (largest radius first: the frame's own bucket order, or the batch work
// list), checks the item and derives its geometry; item_fn(it, c, map,
// map_in_global, lookahead) then processes it with the whole CTA and
// returns false to stop (staging failure, flag already set). Thread 0 looks
// one item ahead: it holds the next item's ticket, and lookahead(0) /
// lookahead(1), called by item_fn at two points of the current item, load
// the next item's index and record, so the work list's dependent loads
// overlap the current item. Ends with the single-frame counter reset.
// s_start: shared memory for rmax + 1 bucket starts (single frames).
template <int RB, int C, bool FULL_SLABS = false, int NW = 8, int SLAB = TcDims<NW>::SLAB, bool F32 = false,
          typename ItemFn>
__device__ __forceinline__ void tc_item_loop(const FrameSource& src, const CUtensorMap& tmap1, const Workspace& ws,
                                             int rmax, const BucketList& bl, int* s_start, ItemFn&& item_fn) {
  constexpr int NT = TcDims<NW>::NT;
  __shared__ int s_state;
  __shared__ Item s_it;
  __shared__ float s_c;
  __shared__ const void* s_map;
  __shared__ int s_wsum[NW];
  const int tid = threadIdx.x;

  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool own_order = bl.list != nullptr;
  const int n_items = own_order ? (int)src.one_total : (int)ws.counters[CNT_NITEMS];
  if (own_order) bucket_starts<NT>(ws.counters + CNT_HIST, bl.nb, s_start, s_wsum);
  const CUtensorMap* batch_maps =
      src.hdr ? reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(src.hdr) + src.hdr->maps_offset)
              : nullptr;

  // Thread 0 looks one item ahead: it holds the next item's ticket, and
  // during the current item it loads the next item's index and record, so
  // the work list's dependent loads overlap the current item.
  int next_tk = 0;
  int nx_item = -1;        // next item's index (lookahead step 0)
  ItemInfo nx_inf;         // next item's record (lookahead step 1)
  bool nx_have = false;
  auto lookup = [&](int tk) -> int {
    if (!own_order) return ws.order[tk];
    int lo = 0, hi = bl.nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_start[mid] <= tk) hi = mid; else lo = mid + 1;
    }
    return bl.list[(size_t)lo * bl.cap + (tk - s_start[lo])];
  };
  auto lookahead = [&](int step) {
    if (step == 0) {
      nx_have = false;
      nx_item = next_tk < n_items ? lookup(next_tk) : -1;
    } else if ((unsigned)nx_item < (unsigned)n_items) {
      nx_inf = ws.items[nx_item];
      nx_have = true;
    }
  };
  if (tid == 0) next_tk = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (tid == 0) {
      const int tk = next_tk;
      int state = 0;
      if (tk >= n_items) {
        state = 2;
      } else {
        next_tk = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
        const int item = nx_have ? nx_item : lookup(tk);
        if ((unsigned)item >= (unsigned)n_items) {
          atomicOr(&ws.counters[CNT_ERROR], kFaultWorklist);
          state = 1;
        } else {
          const ItemInfo inf = nx_have ? nx_inf : ws.items[item];
          const FrameDesc fd = load_frame(src, inf.frame);
          const bool fmt_ok = F32 ? (fd.fmt == FOVEA_F32_CHW && (C == 1 || fd.C == C)) : (fd.fmt == FOVEA_U8_HWC && fd.C == C);
          if (inf.r > rmax || !fmt_ok) {
            atomicOr(&ws.counters[CNT_ERROR], kFaultRadiusBound);
            state = 1;
          } else {
            item_geometry(s_it, inf, fd, RB, FULL_SLABS, SLAB);
            s_c = inf.neg_half_inv_s2;
            s_map = !fd.tma ? nullptr : (batch_maps ? static_cast<const void*>(batch_maps + inf.frame)
                                                    : static_cast<const void*>(&tmap1));
          }
        }
      }
      nx_have = false;
      s_state = state;
    }
    __syncthreads();
    if (s_state == 2) break;
    if (s_state == 1) continue;
    if (!item_fn(s_it, s_c, s_map, batch_maps != nullptr, lookahead)) break;
  }
  if (own_order) {
    __threadfence();
    __syncthreads();
    if (tid == 0) s_state = atomicAdd(&ws.counters[CNT_DONE_SIGMA], 1u) == gridDim.x - 1 ? 3 : 0;
    __syncthreads();
    if (s_state == 3) {
      for (int j = tid; j < kBuckets; j += NT) ws.counters[CNT_HIST + j] = 0u;
      if (tid == 0) {
        ws.counters[CNT_TICKET] = 0u;
        ws.counters[CNT_DONE_SIGMA] = 0u;
      }
    }
  }
}

}  // namespace tcc
}  // namespace fovea
