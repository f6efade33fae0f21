// Tensor-core forward kernel for float32 CHW frames (any non-zero
// tensor_cores on a launch of float32 frames whose rows TMA can load; the
// fp32 CUDA-core kernel otherwise).
//
// The block-wise separable blur of paper Section 2 and Algorithm 1 (taps of
// Eq. 1 truncated at r = ceil(3 sigma)) as the banded Toeplitz contractions
// of tc_forward.cu, on mma.sync.m16n8k16 (fp16 x fp16 -> fp32), per channel
// plane:
//   pass 1 (vertical):   V[yo][e] = sum_v Wv[yo][v] T[v][e]
//   pass 2 (horizontal): O[yo][x] = sum_p V[yo][p] Wh[p][x]
// Each float32 value x is split into fp16 parts x_hi = fp16(x) and x_lo =
// fp16(x - x_hi), the taps (scaled by 2^12) into w_hi + w_lo, and pass 1
// computes W_hi X_hi + W_lo X_hi + W_hi X_lo (the dropped W_lo X_lo is about
// 2^-22 relative); V is split again for pass 2 as in the uint8 kernel. Every
// product of two fp16 values is exact in fp32, so the result carries fp32
// accumulation error plus a representation error of about 2^-21 of |x| (for
// |x| >= 2^-14; an absolute 2^-25 below, where the parts are fp16
// subnormals). The split needs |x| < 32760 (fp16 rounds larger values to
// 2^15 or more): a staged value beyond that, or one that is not finite, is
// recorded as FOVEA_FAULT_VALUE_RANGE and its block is not trustworthy.
// The tensor cores truncate (round toward zero) when they add products into
// an accumulator, about an ulp of the accumulator per MMA; summing a whole
// window in the MMA accumulators biased outputs toward zero by ~2e-6 of
// their value at r ~ 100. So each k-step's products go into a zeroed
// fragment, which is added to the running sums with a rounded fp32 add.
//
// Planes per pass: a launch whose frames all have C = 2 to 4 planes and whose
// radius bound is at most 128 takes all C planes of a tile in each slab
// pass, each plane on 8 / C warps side by side (slabs of up to 125 columns
// for two planes, 61 for three or four), so a narrow halo still keeps most
// warps busy in pass 1; other launches take one plane per pass on all eight
// warps (slabs of up to 240 columns). V holds the pass's planes one after
// the other (32 rows each) and pass 2 takes them as the uint8 kernel takes
// interleaved channels.
//
// Staging: per 16-row chunk of a slab, one thread issues one 32-element
// (128-byte) box per warp column of a 3D tensor map over (x, y, plane)
// (128-byte swizzle; rows outside the plane read zeros) into a four-stage
// ring with a full and an empty mbarrier per stage (bounded waits). Warp w
// owns staged elements 32 b .. 32 b + 31 of its plane (b = w mod warps per
// plane); lane (g, t) reads the four consecutive elements 32 b + 4g .. 4g + 3
// of staged rows 2t, 2t + 1, 2t + 8, 2t + 9 as four 16-byte loads and feeds
// element 32 b + 4g + j to n-tile j. The folded edge rows and columns, the
// tap-pair tables, pass 2 and the work list are those of the uint8 kernel
// (tc_common.cuh); a plane's outputs are stored once its last slab is done.
#include <cstring>

#include "tc_common.cuh"

namespace fovea {

namespace {

using namespace fwd;
using namespace tcc;

constexpr int kNWF = 8;                     // warps
constexpr int kNTF = 32 * kNWF;
constexpr int kRBF = 16;                    // staged rows per chunk (one k-step)
constexpr int kStagesF = 4;                 // ring stages
constexpr int kBoxesF = kNWF;               // one 32-element box per warp column
constexpr int kStageBF = kBoxesF * kRBF * 128;
constexpr float kRangeF = 32768.0f;         // an fp16 hi part this large (or not finite) flags the value range
constexpr float kVScaleF = 1.0f / 4096.0f;  // V = pass-1 accumulator * 2^-12 (taps x 2^12, data x 1)

// CP channel planes per slab pass: CP = 1 takes one plane at a time (any
// channel count); CP = C (2 to 4, launches whose frames all have C planes)
// gives each plane WPP warps side by side.
__host__ __device__ constexpr int tcf_min(int a, int b) { return a < b ? a : b; }
template <int CP>
struct TcfDims {
  static constexpr int WPP = kNWF / CP;    // warps (32-element boxes) per plane
  static constexpr int VP = tc_vp(CP, kNWF);  // V row pitch (halves), the one pass 2 addresses V with
  // elements per plane and slab: alignment padding (up to 3) and slab fit the
  // plane's warps, and the slab rounded up to whole k-steps fits the pitch
  static constexpr int SLAB = tcf_min(32 * WPP - 3, VP / 16 * 16);
  static_assert((SLAB + 15) / 16 * 16 <= VP, "a slab's V row, rounded up to whole k-steps, fits the pitch");
  static_assert(SLAB + 3 <= 32 * WPP, "a slab and its alignment padding fit the plane's warps");
};

struct TcfLayout {
  size_t ring, vh, vl, cum, pairs, starts, total;
};

// V halves (per hi or lo array) of CP planes per pass
__host__ __device__ constexpr int tcf_vhalves(int cp, int vp) { return 32 * cp * vp; }

__host__ __device__ inline TcfLayout tcf_layout(int rmax, int vhalves) {
  TcfLayout L;
  L.ring = 0;                                                 // [stage][box][16 rows][128 B], swizzled
  L.vh = L.ring + (size_t)kStagesF * kStageBF;                // half [planes][32][pitch]
  L.vl = L.vh + (size_t)vhalves * 2;                          // half [planes][32][pitch]
  L.cum = L.vl + (size_t)vhalves * 2;                         // float [cum_len]
  L.pairs = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;   // uint32 [4][npair]
  L.starts = L.pairs + (size_t)4 * npair(rmax) * 4;          // int [rmax + 1] bucket starts
  L.total = L.starts + (size_t)(rmax + 1) * 4 + 1024;         // + alignment slack
  return L;
}

// 16-byte piece q (elements 4q .. 4q + 3) of staged row rho of box bx
// (128-byte swizzle: the piece index XOR rho mod 8).
__device__ __forceinline__ int fpiece(int bx, int rho, int q) { return (bx * kRBF + rho) * 128 + ((q ^ (rho & 7)) << 4); }

__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ unsigned int h2_bits(__half2 h) {
  unsigned int u;
  memcpy(&u, &h, sizeof(u));
  return u;
}

// One item (a halo tile of all channel planes). Chunk gq of the CTA (counted
// over its items) sits in ring stage gq mod 4: full[stage] completes when its
// boxes land, empty[stage] when all eight warps have read it (one arrival per
// warp per chunk, whatever the warp did with it). Thread 0 issues a chunk
// once its stage's previous chunk is released, three chunks ahead of its own
// warp, so warps are not held in step chunk by chunk; block-wide barriers
// remain only where the warps share V (slab ends) and the tables (item start).
// A wait that runs out marks the warp dead (warp-uniform): it stops waiting
// but keeps arriving and passing the same barriers, so every thread leaves
// the item together, which then reports FOVEA_FAULT_WAIT.
template <int CP, typename LookAhead>
__device__ __forceinline__ bool tcf_item(const Item& it, float c_tap, unsigned char* ring, __half* Vh, __half* Vl,
                                         float* CU, unsigned int* P, int np, unsigned long long* full,
                                         unsigned long long* empty, const void* map, bool map_in_global, int& gq0,
                                         unsigned int* err, LookAhead&& lookahead) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r = it.r;
  using D = TcfDims<CP>;
  // CP = 1: slab s is plane s / nsl, columns of slab s % nsl; else slab s is
  // columns of slab s in every plane
  const int nslabs = CP == 1 ? it.nsl * it.C : it.nsl;
  const int Q = nslabs * it.nchunks;

  int issued = 0;      // thread 0: chunks of this item issued
  bool pdead = false;  // thread 0: a wait for a stage to be released ran out
  auto issue = [&](int qq) {  // thread 0: the chunk's boxes that hold slab elements
    const int gq = gq0 + qq, stg = gq % kStagesF;
    if (!pdead && gq >= kStagesF && !mbar_wait(empty + stg, (unsigned int)((gq - kStagesF) / kStagesF) & 1u))
      pdead = true;
    if (pdead) return;
    const Slab cs = slab_of<false>(it, qq / it.nchunks);
    unsigned char* dst = ring + (size_t)stg * kStageBF;
    const int x = it.gx0 + cs.e0 - cs.ph;  // element column, a multiple of 4
    const int y = it.gy0 - it.ph + (qq % it.nchunks) * kRBF;
    const int nbox = (cs.ph + cs.sws + 31) >> 5;  // per plane
    mbar_expect_tx(full + stg, (unsigned int)(CP * nbox) * 128u * kRBF);
    for (int p = 0; p < CP; ++p)  // plane p's boxes feed warps p WPP .. p WPP + nbox - 1
      for (int bx = 0; bx < nbox; ++bx)
        tma_load_3d(dst + (p * D::WPP + bx) * kRBF * 128, map, x + 32 * bx, y, CP == 1 ? cs.c : p, full + stg);
    ++issued;
  };
  if (tid == 0) {
    if (map_in_global) fence_tensormap_acquire(map);
    fence_proxy_async();
    for (int q = 0; q < kStagesF - 1 && q < Q; ++q) issue(q);
  }
  {
    const float S = warp_tap_sum(r, c_tap);
    make_pairs<kNTF>(P, r, c_tap, S, np);
    if ((it.foldT || it.foldB || it.foldL || it.foldR) && warp == kNWF - 1) make_cumulative_tc(CU, r, c_tap, S);
  }
  if (tid == 0) lookahead(0);
  __syncthreads();  // tables ready

  const unsigned int* Ph = P + ((g & 1) ? np : 0);
  const unsigned int* Pl = P + 2 * np + ((g & 1) ? np : 0);
  const int D0 = it.offy - it.ph;  // tap(v, yo) = v + D0 - yo
  const int wplane = warp / D::WPP;           // this warp's plane within the pass
  const int colw = 32 * (warp % D::WPP);      // and its first staged element
  const bool inplane = warp < CP * D::WPP;
  float acc1[2][4][4];
  float acc2[tc_units(CP, kNWF)][4];
  #pragma unroll
  for (int i = 0; i < tc_units(CP, kNWF); ++i)
    #pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = 0.f;
  // largest |x_hi| this thread converted, NaN sticking: x_hi = fp16(x) is
  // at least 2^15 (or infinite) for every |x| >= 32760
  __half2 hmax = __float2half2_rn(0.0f);
  bool dead = false;  // warp-uniform: a wait of this warp ran out

  for (int q = 0; q < Q; ++q) {
    const int gq = gq0 + q;
    if (tid == 0) {
      if (q + kStagesF - 1 < Q) issue(q + kStagesF - 1);
      if (q == 0) lookahead(1);
    }
    const int s = q / it.nchunks, k = q - s * it.nchunks;
    const Slab sl = slab_of<false>(it, s);
    const int R0 = k * kRBF;
    const unsigned char* st = ring + (size_t)(gq % kStagesF) * kStageBF;
    const bool wact = inplane && colw < sl.ph + sl.sws && colw + 32 > sl.ph;  // warp holds slab elements
    // every warp waits for the chunk, also one that holds none of the slab's
    // elements: a warp must not arrive for chunk gq + 4 (same stage) before
    // the chunk is issued, or its arrival would count toward chunk gq's phase
    if (!dead) dead = !__all_sync(0xffffffffu, mbar_wait(full + gq % kStagesF, (unsigned int)(gq / kStagesF) & 1u));
    if (k == 0) {
      #pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          #pragma unroll
          for (int i = 0; i < 4; ++i) acc1[mt][nt][i] = 0.f;
      if (it.foldT && wact) {  // folded top row first: fixed summation order
        const float4 a = *reinterpret_cast<const float4*>(st + fpiece(warp, it.ph, 2 * t));
        const float4 b = *reinterpret_cast<const float4*>(st + fpiece(warp, it.ph, 2 * t + 1));
        const float d0[4] = {a.x, a.y, a.z, a.w}, d1[4] = {b.x, b.y, b.z, b.w};
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const float c0 = cum_at(CU, it.offy - (16 * mt + g), r) * kWScale;
          const float c1 = cum_at(CU, it.offy - (16 * mt + g + 8), r) * kWScale;
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc1[mt][j][0] = fmaf(c0, d0[j], acc1[mt][j][0]);
            acc1[mt][j][1] = fmaf(c0, d1[j], acc1[mt][j][1]);
            acc1[mt][j][2] = fmaf(c1, d0[j], acc1[mt][j][2]);
            acc1[mt][j][3] = fmaf(c1, d1[j], acc1[mt][j][3]);
          }
        }
      }
    }
    // ---- pass 1 on the chunk (one 16-row k-step)
    if (wact) {
      const int k0 = R0;
      const bool on0 = k0 + 15 >= -D0 && k0 <= 15 - D0 + 2 * r;
      const bool on1 = k0 + 15 >= 16 - D0 && k0 <= 31 - D0 + 2 * r;
      if (on0 || on1) {
        const int j0 = (k0 + D0 + 2 * t - g + kPairPad) >> 1;
        unsigned int ah[2][4], al[2][4];
        {
          const unsigned int h_m12 = Ph[j0 - 12], h_m8 = Ph[j0 - 8], h_m4 = Ph[j0 - 4], h_0 = Ph[j0], h_p4 = Ph[j0 + 4];
          const unsigned int l_m12 = Pl[j0 - 12], l_m8 = Pl[j0 - 8], l_m4 = Pl[j0 - 4], l_0 = Pl[j0], l_p4 = Pl[j0 + 4];
          ah[0][0] = h_0; ah[0][1] = h_m4; ah[0][2] = h_p4; ah[0][3] = h_0;
          ah[1][0] = h_m8; ah[1][1] = h_m12; ah[1][2] = h_m4; ah[1][3] = h_m8;
          al[0][0] = l_0; al[0][1] = l_m4; al[0][2] = l_p4; al[0][3] = l_0;
          al[1][0] = l_m8; al[1][1] = l_m12; al[1][2] = l_m4; al[1][3] = l_m8;
        }
        // B fragments of the four n-tiles from rows 2t, 2t+1, 2t+8, 2t+9:
        // element 32w + 4g + j of each, split into fp16 hi and lo parts
        const float4 x0 = *reinterpret_cast<const float4*>(st + fpiece(warp, 2 * t, g));
        const float4 x1 = *reinterpret_cast<const float4*>(st + fpiece(warp, 2 * t + 1, g));
        const float4 x8 = *reinterpret_cast<const float4*>(st + fpiece(warp, 2 * t + 8, g));
        const float4 x9 = *reinterpret_cast<const float4*>(st + fpiece(warp, 2 * t + 9, g));
        const float v0[4] = {x0.x, x0.y, x0.z, x0.w}, v1[4] = {x1.x, x1.y, x1.z, x1.w};
        const float v8[4] = {x8.x, x8.y, x8.z, x8.w}, v9[4] = {x9.x, x9.y, x9.z, x9.w};
        unsigned int bh[4][2], bl[4][2];
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __half2 h01 = __floats2half2_rn(v0[j], v1[j]), h89 = __floats2half2_rn(v8[j], v9[j]);
          hmax = __hmax2_nan(hmax, __hmax2_nan(__habs2(h01), __habs2(h89)));
          const float2 f01 = __half22float2(h01), f89 = __half22float2(h89);
          bh[j][0] = h2_bits(h01);
          bh[j][1] = h2_bits(h89);
          bl[j][0] = h2_bits(__floats2half2_rn(v0[j] - f01.x, v1[j] - f01.y));
          bl[j][1] = h2_bits(__floats2half2_rn(v8[j] - f89.x, v9[j] - f89.y));
        }
        // W_hi X_hi, W_lo X_hi and W_hi X_lo of the k-step go into a zeroed
        // fragment that is then added to acc1 in fp32 (the MMA's own adds
        // truncate)
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (!(mt == 0 ? on0 : on1)) continue;
          float tmp[4][4];
          #pragma unroll
          for (int j = 0; j < 4; ++j)
            #pragma unroll
            for (int i = 0; i < 4; ++i) tmp[j][i] = 0.f;
          #pragma unroll
          for (int part = 0; part < 3; ++part)
            #pragma unroll
            for (int j = 0; j < 4; ++j)
              mma16816(tmp[j], part == 1 ? al[mt] : ah[mt], part == 2 ? bl[j][0] : bh[j][0],
                       part == 2 ? bl[j][1] : bh[j][1]);
          #pragma unroll
          for (int j = 0; j < 4; ++j)
            #pragma unroll
            for (int i = 0; i < 4; ++i) acc1[mt][j][i] += tmp[j][i];
        }
      }
    }
    const bool last = k == it.nchunks - 1;
    // folded bottom row (in the slab's last chunk), the stage's last read
    const int vb = it.ph + it.EH - 1;
    if (last && it.foldB && vb >= R0 && vb < R0 + kRBF && wact) {
      const float4 a = *reinterpret_cast<const float4*>(st + fpiece(warp, vb - R0, 2 * t));
      const float4 b = *reinterpret_cast<const float4*>(st + fpiece(warp, vb - R0, 2 * t + 1));
      const float d0[4] = {a.x, a.y, a.z, a.w}, d1[4] = {b.x, b.y, b.z, b.w};
      #pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const float c0 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g)), r) * kWScale;
        const float c1 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g + 8)), r) * kWScale;
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc1[mt][j][0] = fmaf(c0, d0[j], acc1[mt][j][0]);
          acc1[mt][j][1] = fmaf(c0, d1[j], acc1[mt][j][1]);
          acc1[mt][j][2] = fmaf(c1, d0[j], acc1[mt][j][2]);
          acc1[mt][j][3] = fmaf(c1, d1[j], acc1[mt][j][3]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + gq % kStagesF);  // this warp is done with the stage
    if (!last) continue;

    // ---- slab complete: V -> hi/lo fp16 for pass 2
    const int npx = sl.sws;
    const int npx16 = (npx + 15) & ~15;
    __syncthreads();  // every warp is done with the previous slab's V
    // V[yo][px] = acc * 2^-12 as hi + lo fp16; staged element 32w + 8t + e8
    // is slab pixel 32w + 8t + e8 - ph
    if (wact) {
      #pragma unroll
      for (int e8 = 0; e8 < 8; ++e8) {
        const int e = colw + 8 * t + e8 - sl.ph;
        if (e < 0 || e >= npx) continue;
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          #pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const float v = acc1[mt][e8 & 3][2 * hh + (e8 >> 2)] * kVScaleF;
            const __half h = __float2half_rn(v);
            const __half l = __float2half_rn(v - __half2float(h));
            const size_t o = (size_t)(32 * wplane + 16 * mt + g + 8 * hh) * D::VP + e;
            if (smem_in_bounds(Vh + o, 2, err) && smem_in_bounds(Vl + o, 2, err)) {
              Vh[o] = h;
              Vl[o] = l;
            }
          }
        }
      }
    }
    // zero the columns px in [npx, npx16) that pass 2 reads
    const int zc = npx16 - npx;
    for (int idx = tid; idx < 32 * CP * zc; idx += kNTF) {
      const int row = idx / zc, px = npx + (idx - row * zc);
      const size_t o = (size_t)row * D::VP + px;
      if (smem_in_bounds(Vh + o, 2, err) && smem_in_bounds(Vl + o, 2, err)) {
        Vh[o] = __ushort_as_half(0);
        Vl[o] = __ushort_as_half(0);
      }
    }
    __syncthreads();  // V complete
    {
      // pass 2 counts a slab in interleaved elements: pixels x planes
      Slab s2 = sl;
      s2.e0 = sl.e0 * CP;
      s2.sws = sl.sws * CP;
      tc_pass2_slab<CP, false, kNWF, true>(it, s2, Vh, Vl, CU, P, np, acc2);
    }

    if (s % it.nsl == it.nsl - 1) {
      // the last slab of the pass's planes: their outputs (x 2^-12) go
      // straight to the frame; unit u holds rows of m-tile u / 4 of V, whose
      // plane is (u / 4) / 2 (the slab's plane when CP = 1)
      const size_t plane = (size_t)it.W * it.H;
      const size_t frame_bytes = plane * it.C * 4;
      #pragma unroll
      for (int i = 0; i < tc_units(CP, kNWF); ++i) {
        const int u = warp + kNWF * i;
        if (u >= 8 * CP) continue;
        const int mt2 = u >> 2, nt2 = u & 3;
        float* outp = reinterpret_cast<float*>(it.out) + (size_t)(CP == 1 ? sl.c : mt2 >> 1) * plane;
        #pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int yo = 16 * (mt2 & 1) + g + ((e >> 1) << 3), x = 8 * nt2 + 2 * t + (e & 1);
          if (yo < it.bh && x < it.bw) {
            float* o = outp + (size_t)(it.y0 + yo) * it.W + it.x0 + x;
            if (in_bounds(o, 4, it.out, frame_bytes, err)) *o = acc2[i][e] * kWInv;
          }
          acc2[i][e] = 0.f;
        }
      }
    }
  }
  gq0 += Q;
  const bool fail = __syncthreads_or(dead || pdead) != 0;
  if (fail) {
    // a wait ran out: flag it, let this item's boxes still in flight land
    // (bounded) and give up
    if (tid == 0) {
      atomicOr(err, kFaultWait);
      const int first = gq0 - Q;
      for (int qq = issued > kStagesF ? issued - kStagesF : 0; qq < issued; ++qq) {
        const int c = first + qq;
        mbar_wait(full + c % kStagesF, (unsigned int)(c / kStagesF) & 1u);
      }
    }
    __syncthreads();
    return false;
  }
  const float2 hm = __half22float2(hmax);
  if (__syncthreads_or(!(hm.x < kRangeF && hm.y < kRangeF)) && tid == 0) atomicOr(err, kFaultValueRange);
  fence_proxy_async();  // the next item's TMA boxes overwrite the ring
  return true;
}

template <int CP>
__global__ void __launch_bounds__(kNTF, 2)
tcf_forward_kernel(const __grid_constant__ FrameSource src, Workspace ws, int rmax, BucketList bl,
                   const __grid_constant__ CUtensorMap tmap1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const TcfLayout L = tcf_layout(rmax, tcf_vhalves(CP, TcfDims<CP>::VP));
  unsigned char* ring = smem + L.ring;
  __half* Vh = reinterpret_cast<__half*>(smem + L.vh);
  __half* Vl = reinterpret_cast<__half*>(smem + L.vl);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  unsigned int* P = reinterpret_cast<unsigned int*>(smem + L.pairs);
  __shared__ __align__(8) unsigned long long s_full[kStagesF], s_empty[kStagesF];
  const int np = npair(rmax);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStagesF; ++i) {
      mbar_init(&s_full[i], 1);
      mbar_init(&s_empty[i], kNWF);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  int gq0 = 0;  // chunks this CTA has loaded so far (identical in every thread)
  tc_item_loop<kRBF, CP, true, kNWF, TcfDims<CP>::SLAB, true>(
      src, tmap1, ws, rmax, bl, reinterpret_cast<int*>(smem + L.starts),
      [&](const Item& it, float c, const void* map, bool map_global, auto& lookahead) {
        if (!map) {  // rows TMA cannot address: the host runs the fp32 kernel for such launches
          if (threadIdx.x == 0) atomicOr(ws.counters + CNT_ERROR, kFaultRadiusBound);
          return true;
        }
        return tcf_item<CP>(it, c, ring, Vh, Vl, CU, P, np, s_full, s_empty, map, map_global, gq0,
                            ws.counters + CNT_ERROR, lookahead);
      });
}

// Planes per pass for a launch whose frames all have `channels` planes (0:
// mixed counts) and whose radius bound is rmax. Packed passes pay off while
// halos are narrow; from a radius bound of 129 on (halos beyond 290 columns)
// one plane per pass on all eight warps measured faster (1920 x 1080 x 3
// float32, sigma = 0.5 + 0.08 e, radii up to 262: 1.24 ms against 1.34 ms
// packed; at radii up to 67, 0.248 ms packed against 0.267 ms).
constexpr int kTcfPackedRadius = 128;
int tcf_planes(int channels, int rmax) {
  return channels >= 2 && channels <= 4 && rmax <= kTcfPackedRadius ? channels : 1;
}

const void* tcf_kernel_fn(int channels, int rmax) {
  switch (tcf_planes(channels, rmax)) {
    case 2: return reinterpret_cast<const void*>(&tcf_forward_kernel<2>);
    case 3: return reinterpret_cast<const void*>(&tcf_forward_kernel<3>);
    case 4: return reinterpret_cast<const void*>(&tcf_forward_kernel<4>);
    default: return reinterpret_cast<const void*>(&tcf_forward_kernel<1>);
  }
}

int tcf_vpitch(int cp) {
  return cp == 2 ? TcfDims<2>::VP : cp == 3 ? TcfDims<3>::VP : cp == 4 ? TcfDims<4>::VP : TcfDims<1>::VP;
}

}  // namespace

bool tcf_supports(int rmax) { return rmax <= kMaxRadius; }

size_t tcf_forward_smem_bytes(int rmax, int channels) {
  const int cp = tcf_planes(channels, rmax);
  return tcf_layout(rmax, tcf_vhalves(cp, tcf_vpitch(cp))).total;
}

int tcf_forward_max_ctas_per_sm(int rmax, int channels) {
  const size_t smem = tcf_forward_smem_bytes(rmax, channels);
  const void* k = tcf_kernel_fn(channels, rmax);
  if (set_smem_attrs(k, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kNTF, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_tcf_forward(const FrameSource& src, const Workspace& ws, int rmax, int channels, int grid,
                               cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one) {
  const size_t smem = tcf_forward_smem_bytes(rmax, channels);
  void* k = const_cast<void*>(tcf_kernel_fn(channels, rmax));
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (tmap_one) std::memcpy(&map, tmap_one, sizeof(map));
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &b, &map};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(kNTF);
  lc.dynamicSmemBytes = smem;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelExC(&lc, k, args);
}

}  // namespace fovea
