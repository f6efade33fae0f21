// Forward kernel for uint8 HWC RGB frames with both separable passes on the
// 5th-generation tensor cores (tcgen05): the block-wise blur of paper
// Section 2 and Algorithm 1 (taps of Eq. 1 truncated at r = ceil(3 sigma)),
// as the two banded Toeplitz contractions of tc_forward.cu, each issued by one
// thread as asynchronous tcgen05.mma with its fp32 accumulator in tensor
// memory (TMEM):
//
//   pass 1 (vertical):   D1[e][n] = sum_v T[v][e] u(v + D0 - (31 - n))
//                        M = 128 element columns e of a tile, N = 32 output
//                        rows (reversed) x {hi, lo} taps, K = 16 staged rows;
//   pass 2 (horizontal): D2[(c, yo)][n] = sum_p V[(c, yo)][p] u(offx + p - (31 - n))
//                        M = 128 rows (c, yo) (96 used), N = 32 output
//                        columns (reversed) x {hi, lo} taps, K = 16 pixels.
//
// Both A operands are MN-major (their M index contiguous), which is the
// order the data arrives in: pass 1 reads the staged rows widened from bytes
// to fp16 (a byte b in the low bits of an fp16 is the exact subnormal
// b * 2^-24) without any transpose, and pass 2 reads V with the 32 output
// rows of one (pixel, channel) contiguous, which is how a thread holds them
// after reading its TMEM lane. Both B operands are the taps as Hankel strips
// (tc05_common.cuh): no weight matrix is built. Accuracy is that of the
// mma.sync kernel: taps and V split into fp16 hi + lo parts (one N = 64
// instruction computes the hi and lo tap products), fp32 accumulation.
//
// Work split (one 32 x 32 block = one item; columns in slabs of 96 pixels =
// three tiles of 32 pixels, each tile 128 staged bytes; rows in chunks of RB):
//   warp 0, lane 0: the producer. It issues the TMA row boxes of each chunk
//     into a 4-stage ring as stages are released, and, polling, the pass-2
//     MMAs of each tile as its V operand becomes ready, accumulating the
//     item's output in TMEM.
//   warps 1..3, one per tile: convert the tile's 128 staged bytes of each
//     chunk (ring bytes -> fp16 A1, two buffers per tile) and issue and commit
//     the tile's own pass-1 MMAs, so a chunk needs no hand-over between warps.
//     A converted row is indexed by staged byte, alignment padding included,
//     so every 16-byte piece converts in place; the padding is skipped when
//     the tile is read back (TMEM lane = staged byte).
//   warps 4..7 (tensor-memory lane quarters 0..3): after a slab, read each
//     tile's D1 back, add the folded top / bottom rows (clamp-to-edge, as in
//     the other kernels), and write V as fp16 hi / lo into one of two A2
//     buffers; warps 4..6, after the item, read D2, add the folded left /
//     right columns, round to uint8 and stage the block by channel planes.
// Every frame of a launch must be TMA-loadable (the host uses the mma.sync
// kernel otherwise). Every wait is bounded; a wait that gives up flags
// FOVEA_FAULT_WAIT, the CTA drains what it issued and stops.
#include <algorithm>
#include <cstring>

#include "tc05_common.cuh"

namespace fovea {

namespace {

using namespace fwd;
using namespace tcc;

constexpr int kC5 = 3;                      // channels this kernel serves
constexpr int kPxT = 32;                    // pixels per tile
constexpr int kElT = kPxT * kC5;            // 96 element columns per tile
constexpr int kTiles = 3;                   // tiles per slab
constexpr int kSlabEl5 = kTiles * kElT;     // 288 elements per slab
constexpr int kBoxes5 = 3;                  // 128-byte tensor-map boxes per staged row
constexpr int kStages5 = 4;                 // ring stages
constexpr int kA1Bufs5 = 2;                 // converted chunks in flight per tile
constexpr int kA2Part = 16 * 4 * 128;       // one V part (hi or lo) of a tile: 16 M cores x 4 K groups
constexpr int kThreads5 = 256;
constexpr unsigned int kTmemCols5 = 256;    // D1: 3 tiles x 64 columns; D2 at column 192
constexpr int kMaxRadius5 = 511;            // tap strips grow with r
// f32 accumulator, f16 A and B, A MN-major (bit 15), B K-major, N = 64, M = 128
constexpr unsigned int kIdesc5 = (1u << 4) | (1u << 15) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// One tile's converted chunk (pass-1 A operand, MN-major, 128 staged bytes x
// RB rows): core matrix (K group kg, M core mg) at mg * RB * 16 + kg * 128
// bytes, i.e. adjacent K groups 128 bytes apart (the descriptor's leading
// offset) and adjacent M cores RB * 16 bytes apart (its stride offset); the
// K groups of one M core side by side, so either reading of the two strides
// stays inside the buffer.
__host__ __device__ constexpr int a1_tile_bytes5(int rb) { return 16 * rb * 16; }

struct T5Layout {
  size_t ring, a1, a2, s1, s2, taps, cum, edge, foldw, vfold, ost, starts, total;
};

__host__ __device__ inline T5Layout t5_layout(int rb, int rmax) {
  T5Layout L;
  const size_t strip = (size_t)strip_entries(rmax) * 256;
  L.ring = 0;                                                        // u8 [stages][boxes][rb][128], swizzled
  L.a1 = L.ring + (size_t)kStages5 * kBoxes5 * rb * 128;             // [tile][buffer][a1_tile_bytes5]
  L.a2 = L.a1 + (size_t)kTiles * kA1Bufs5 * a1_tile_bytes5(rb);      // [2 buffers][hi, lo][kA2Part]
  L.s1 = L.a2 + (size_t)2 * 2 * kA2Part;                             // pass-1 strip
  L.s2 = L.s1 + strip;                                               // pass-2 strip
  L.taps = L.s2 + strip;                                             // float [2 rmax + 1] normalised taps
  L.cum = L.taps + (size_t)((2 * rmax + 1 + 3) & ~3) * 4;            // float [cum_len]
  L.edge = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;           // u8 [3 slabs][top, bottom][320 staged bytes]
  L.foldw = L.edge + (size_t)6 * 320;                                // float [top, bottom by yo; left, right by x][32]
  L.vfold = L.foldw + 128 * 4;                                       // float [2][96]
  L.ost = L.vfold + 2 * 96 * 4;                                      // u8 [C][32 rows][32 columns]
  L.starts = L.ost + 32 * 96;                                        // int [rmax + 1]
  L.total = L.starts + (size_t)(rmax + 1) * 4 + 1024;                // + alignment slack
  return L;
}

struct T5Smem {
  unsigned char* ring;
  unsigned char* a1;
  unsigned char* a2;
  __half* s1;
  __half* s2;
  float* U;
  float* CU;
  unsigned char* edge;
  float* foldw;
  float* vfold;
  unsigned char* ost;
};

struct T5Bars {
  unsigned long long ring[kStages5];            // TMA bytes of a ring stage landed (count 1 + tx)
  unsigned long long ringfree[kStages5];        // the three tile warps read a stage (3)
  unsigned long long a1free[kTiles][kA1Bufs5];  // the MMAs that read a tile's A1 buffer finished (commit)
  unsigned long long tdone[kTiles];             // a tile's pass-1 MMAs of a slab finished (commit + arrive; 2)
  unsigned long long d1free[kTiles];            // the read-back warps read a tile's D1 (4)
  unsigned long long a2full[2];                 // a tile's V written (4 warps)
  unsigned long long a2free[2];                 // the pass-2 MMAs that read an A2 buffer finished (commit)
  unsigned long long d2;                        // every pass-2 MMA of an item finished (commit)
};

// Phase counters (identical in every thread): ring chunks, A1 chunks (per
// tile, all tiles alike), pass-2 tiles (A2 buffers), slabs, items.
struct T5Count {
  int gr, gc, gtile, gslab, gitem;
};

__device__ __forceinline__ bool t5_wait(unsigned long long* bar, int use, volatile int* abort, unsigned int* err) {
  if (*abort) return false;
  if (mbar_wait(bar, (unsigned int)use & 1u)) return true;
  atomicOr(err, kFaultWait);
  *abort = 1;
  return false;
}

// Non-blocking: has the phase of the given use completed?
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, int use) {
  unsigned int ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"((unsigned int)use & 1u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld64(unsigned int taddr, float (&d)[64]) {
  float a[32], b[32];
  tmem_ld32(taddr, a);
  tmem_ld32(taddr + 32, b);
  #pragma unroll
  for (int i = 0; i < 32; ++i) {
    d[i] = a[i];
    d[32 + i] = b[i];
  }
}

template <int RB, typename LookAhead>
__device__ __forceinline__ bool t5_item(const Item& it, float c_tap, const T5Smem& sm, T5Bars* bars, int nent,
                                        unsigned int tmem, volatile int* abort, const void* map, bool map_in_global,
                                        T5Count& k, unsigned int* err, LookAhead&& lookahead) {
  constexpr size_t stage_bytes = (size_t)kBoxes5 * RB * 128;
  constexpr int a1t = a1_tile_bytes5(RB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = it.r;
  const int Q = it.nsl * it.nchunks;
  const int D0 = it.offy - it.ph;        // tap(v, yo) = v + D0 - yo; a multiple of 16, >= 0
  const int delta1 = (D0 + 1) & 7;       // (D0 - 31) mod 8
  const int delta2 = (it.offx + 1) & 7;  // (offx - 31) mod 8
  const bool prod = tid == 0;            // TMA producer and pass-2 MMA issuer
  const bool tilew = warp >= 1 && warp <= kTiles;
  const bool epi = warp >= 4;            // tile read-back: TMEM lane quarters 0..3
  const bool epi2 = warp >= 4 && warp <= 6;  // output: the channel quarters 0..2
  const int gr_base = k.gr;

  // ---- producer state: it walks the item's chunks (slab by slab) with counters
  int issued = 0, is_slab = 0, is_chunk = 0, is_x = 0;
  const int y_first = it.gy0 - it.ph;
  auto issue = [&]() {  // the next chunk's three TMA boxes into its ring stage
    if (is_chunk == 0) {
      const Slab cs = slab_of<true>(it, is_slab);
      is_x = (int)cs.src - cs.ph;  // 16-byte aligned byte column
    }
    const int g = gr_base + issued, stg = g % kStages5;
    unsigned char* dst = sm.ring + (size_t)stg * stage_bytes;
    const int y = y_first + is_chunk * RB;
    mbar_expect_tx(&bars->ring[stg], (unsigned int)kBoxes5 * 128u * RB);
    #pragma unroll
    for (int bx = 0; bx < kBoxes5; ++bx) tma_load_2d(dst + 128 * RB * bx, map, is_x + 128 * bx, y, &bars->ring[stg]);
    ++issued;
    if (++is_chunk == it.nchunks) {
      is_chunk = 0;
      ++is_slab;
    }
  };
  if (prod) {
    if (map_in_global) fence_tensormap_acquire(map);
    fence_proxy_async();
    while (issued < kStages5 && issued < Q) issue();  // the stages were released by the previous item
  }
  // ---- tables of the item: the taps once, then the two tap strips and the
  // folds' weights from them
  {
    const float S = warp_tap_sum(r, c_tap);
    make_tap_table<kThreads5>(sm.U, r, c_tap, S);
    __syncthreads();
    make_strips_tab<kThreads5>(sm.s1, nent, sm.U, r, delta1);
    make_strips_tab<kThreads5>(sm.s2, nent, sm.U, r, delta2);
    if ((it.foldT || it.foldB || it.foldL || it.foldR) && warp == 7) {
      make_cumulative_tab(sm.CU, sm.U, r);
      __syncwarp();
      // rows: weight of the folded top / bottom row for output row yo = lane
      // (in pass-1 accumulator units); columns: of the folded left / right
      // column for output column x = lane (in pass-2 accumulator units)
      sm.foldw[lane] = cum_at(sm.CU, it.offy - lane, r) * (kWScale * kDScale);
      sm.foldw[32 + lane] = cum_at(sm.CU, 2 * r + 1 - (it.offy + it.EH - lane), r) * (kWScale * kDScale);
      sm.foldw[64 + lane] = it.foldL ? cum_at(sm.CU, it.offx - lane, r) * kWScale : 0.0f;
      sm.foldw[96 + lane] = it.foldR ? cum_at(sm.CU, 2 * r + 1 - (it.offx + it.EW - lane), r) * kWScale : 0.0f;
    }
  }
  fence_proxy_async();  // the strips are read by the tensor cores
  __syncthreads();
  const int vb = it.ph + it.EH - 1;  // virtual row of the folded bottom row

  if (prod) {
    // ------------------------------------------------------------ producer
    lookahead(0);
    int total_tiles = 0;
    for (int s2 = 0; s2 < it.nsl; ++s2) total_tiles += (slab_of<true>(it, s2).sws / kC5 + kPxT - 1) / kPxT;
    const unsigned long long a2d = umma_desc(sm.a2, 128, 512);
    int done_tiles = 0, tslab = 0, ttile = 0, tslab_tiles = 0, tP0 = 0, tnpx = 0;
    unsigned long long s2d = 0;
    int d2_started = 0, idle = 0;
    bool looked = false;
    while ((issued < Q || done_tiles < total_tiles) && !*abort) {
      bool progress = false;
      if (issued < Q) {  // refill a released stage (its previous chunk, 4 back, was read by every tile warp)
        const int g = gr_base + issued;
        if (mbar_test(&bars->ringfree[g % kStages5], g / kStages5 - 1)) {
          issue();
          progress = true;
        }
      }
      if (done_tiles < total_tiles) {
        const int gtl = k.gtile + done_tiles, buf = gtl & 1;
        if (mbar_test(&bars->a2full[buf], gtl >> 1)) {
          if (ttile == 0) {  // first tile of a slab: its geometry and strip base
            const Slab cs = slab_of<true>(it, tslab);
            tnpx = cs.sws / kC5;
            tslab_tiles = (tnpx + kPxT - 1) / kPxT;
            tP0 = cs.e0 / kC5;
            // strip entry of pixel p0 of the slab: (offx + P0 + p0 - 31 - delta2) / 8 + kXOff
            s2d = umma_desc(sm.s2, 256, 128) + (unsigned long long)(16 * ((it.offx + tP0 - 31 - delta2) / 8 + kXOff));
          }
          tc05_fence_after();
          #pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const int p0 = kPxT * ttile + 16 * ks;
            if (p0 >= tnpx) break;
            const unsigned long long bd = s2d + (unsigned long long)(32 * (p0 >> 4));
            #pragma unroll
            for (int part = 0; part < 2; ++part) {
              umma_f16(tmem + 192, a2d + (unsigned long long)((buf * 2 + part) * (kA2Part >> 4) + 16 * ks), bd, kIdesc5,
                       d2_started);
              d2_started = 1;
            }
          }
          umma_commit(&bars->a2free[buf]);
          ++done_tiles;
          if (++ttile == tslab_tiles) {
            ttile = 0;
            ++tslab;
          }
          progress = true;
        }
      }
      if (!looked) {
        lookahead(1);
        looked = true;
      }
      if (progress) {
        idle = 0;
      } else if (++idle > kWaitLimit) {
        atomicOr(err, kFaultWait);
        *abort = 1;
      } else {
        __nanosleep(20);
      }
    }
    umma_commit(&bars->d2);
  } else if (tilew) {
    // ------------------------------------------------------------ tile warps
    const int t = warp - 1;
    const int k_end = min(it.vrows, 32 - D0 + 2 * r);  // K steps with a tap of the 32 output rows
    const unsigned long long s1d = umma_desc(sm.s1, 256, 128) + (unsigned long long)(16 * (D0 / 8 + 4));
    const unsigned long long a1d = umma_desc(sm.a1 + (size_t)t * kA1Bufs5 * a1t, 128, RB * 16);
    unsigned char* a1base = sm.a1 + (size_t)t * kA1Bufs5 * a1t;
    int g = k.gc;  // this tile's A1 chunk counter (the same in every tile warp)
    for (int s = 0; s < it.nsl; ++s) {
      const Slab sl = slab_of<true>(it, s);
      const int ntiles = (sl.sws / kC5 + kPxT - 1) / kPxT;
      const bool active = t < ntiles;
      const int gs = k.gslab + s;
      unsigned char* edge = sm.edge + (gs % 3) * 640;
      int started = 0;
      for (int kq = 0; kq < it.nchunks; ++kq, ++g) {
        const int gq = gr_base + s * it.nchunks + kq, stg = gq % kStages5;
        t5_wait(&bars->ring[stg], gq / kStages5, abort, err);
        const unsigned char* st = sm.ring + (size_t)stg * stage_bytes;
        const int buf = g % kA1Bufs5;
        // every tile warp commits once per chunk (an inactive tile with no
        // MMA at all), so the buffers' phases stay in step
        if (g >= kA1Bufs5) t5_wait(&bars->a1free[t][buf], g / kA1Bufs5 - 1, abort, err);
        if (active) {
          // convert: unit = (row rho, 16-byte group ge) of the tile's 128 staged bytes
          unsigned char* a1 = a1base + (size_t)buf * a1t;
          #pragma unroll
          for (int i = 0; i < RB / 4; ++i) {
            const int u = lane + 32 * i, rho = u % RB, ge = u / RB;
            const int b = kElT * t + 16 * ge;  // staged byte
            const uint4 w = *reinterpret_cast<const uint4*>(st + ring_off<RB>(rho, b));
            const int vv = kq * RB + rho;
            if ((kq == 0 && vv == it.ph) || vv == vb) {  // folded edge rows (both, if EH = 1)
              #pragma unroll
              for (int part = 0; part < 2; ++part) {
                if (part == 0 ? !(kq == 0 && vv == it.ph) : vv != vb) continue;
                *reinterpret_cast<uint4*>(edge + 320 * part + b) = w;
              }
            }
            const uint4 lo = make_uint4(__byte_perm(w.x, 0u, 0x4140), __byte_perm(w.x, 0u, 0x4342),
                                        __byte_perm(w.y, 0u, 0x4140), __byte_perm(w.y, 0u, 0x4342));
            const uint4 hi = make_uint4(__byte_perm(w.z, 0u, 0x4140), __byte_perm(w.z, 0u, 0x4342),
                                        __byte_perm(w.w, 0u, 0x4140), __byte_perm(w.w, 0u, 0x4342));
            unsigned char* o = a1 + (size_t)(2 * ge) * (RB * 16) + (rho >> 3) * 128 + (rho & 7) * 16;
            if (smem_in_bounds(o, 16, err) && smem_in_bounds(o + RB * 16, 16, err)) {
              *reinterpret_cast<uint4*>(o) = lo;
              *reinterpret_cast<uint4*>(o + RB * 16) = hi;
            }
          }
          fence_proxy_async();  // the converted chunk is read by the tensor cores
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bars->ringfree[stg]);  // this warp is done with the stage
          // the read-back of the tile's previous slab is done (also when the
          // tile is inactive: otherwise its slab commits could run two phases
          // ahead of the read-back warps' parity waits on tdone)
          if (kq == 0 && gs > 0) t5_wait(&bars->d1free[t], gs - 1, abort, err);
          if (active) {
            tc05_fence_after();
            #pragma unroll
            for (int ks = 0; ks < RB / 16; ++ks) {
              const int k0 = kq * RB + 16 * ks;
              if (k0 >= k_end || *abort) break;
              // strip entry 2 kidx + D0 / 8 + 4 for K step kidx = k0 / 16 (delta1 = 1)
              umma_f16(tmem + 64 * t, a1d + (unsigned long long)(buf * (a1t >> 4) + 16 * ks),
                       s1d + (unsigned long long)(32 * (k0 >> 4)), kIdesc5, started);
              started = 1;
            }
          }
          umma_commit(&bars->a1free[t][buf]);
        }
        __syncwarp();
      }
      __syncwarp();
      if (lane == 0) {
        umma_commit(&bars->tdone[t]);  // the tile's pass-1 MMAs of the slab (none if inactive)
        mbar_arrive(&bars->tdone[t]);  // and (release) the warp's edge-row stash
      }
      __syncwarp();
    }
  }
  // ------------------------------------------------------------ V (read-back warps)
  int tile_base = 0;
  if (epi) {
    const int q = warp - 4;                  // TMEM lane quarter
    const int lane_t = 32 * q + lane;        // TMEM lane = staged byte of the tile
    for (int s = 0; s < it.nsl; ++s) {
      const Slab sl = slab_of<true>(it, s);
      const int npx = sl.sws / kC5;
      const int ntiles = (npx + kPxT - 1) / kPxT;
      const int P0 = sl.e0 / kC5;
      const int gs = k.gslab + s;
      const unsigned char* edge = sm.edge + (gs % 3) * 640;
      const int el = lane_t - sl.ph;          // element of the tile (0 .. 95 for its 32 pixels)
      const bool mine = el >= 0 && el < kElT;
      const int px = mine ? el / kC5 : 0, c = mine ? el - px * kC5 : 0;
      for (int t = 0; t < kTiles; ++t) {
        t5_wait(&bars->tdone[t], gs, abort, err);
        if (t >= ntiles) {  // keep the tile's D1 phase in step
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->d1free[t]);
          continue;
        }
        tc05_fence_after();
        const int gtl = k.gtile + tile_base + t, buf = gtl & 1;
        if (gtl >= 2) t5_wait(&bars->a2free[buf], (gtl >> 1) - 1, abort, err);
        float d[64];
        __syncwarp();  // tcgen05.ld is warp-collective
        tmem_ld64(tmem + ((unsigned int)(32 * q) << 16) + 64 * t, d);
        tc05_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->d1free[t]);  // D1 of the tile is read: its next slab may start
        const int b = kElT * t + lane_t;      // staged byte
        const int spx = kPxT * t + px;        // slab pixel
        const int pg = P0 + spx;              // folded pixel
        const bool live = mine && spx < npx;
        const float et = it.foldT ? (float)edge[b] : 0.0f, eb = it.foldB ? (float)edge[320 + b] : 0.0f;
        float v[32];
        #pragma unroll
        for (int yo = 0; yo < 32; ++yo) {
          // column 16 a + 8 p + i holds part p of output row 31 - (8 a + i)
          const int n = 31 - yo, a = n >> 3, i = n & 7;
          float x = d[16 * a + i] + d[16 * a + 8 + i];
          if (it.foldT) x = fmaf(sm.foldw[yo], et, x);
          if (it.foldB) x = fmaf(sm.foldw[32 + yo], eb, x);
          v[yo] = x * kVScale;
        }
        if (live && it.foldL && pg == 0) {
          #pragma unroll
          for (int yo = 0; yo < 32; ++yo) sm.vfold[32 * c + yo] = v[yo];
        }
        if (live && it.foldR && pg == it.EW - 1) {
          #pragma unroll
          for (int yo = 0; yo < 32; ++yo) sm.vfold[96 + 32 * c + yo] = v[yo];
        }
        unsigned char* a2 = sm.a2 + (size_t)buf * 2 * kA2Part + (px >> 3) * 128 + (px & 7) * 16;
        #pragma unroll
        for (int j = 0; j < 4 && mine; ++j) {
          unsigned int hw[4], lw[4];
          #pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float v0 = live ? v[8 * j + 2 * m] : 0.0f, v1 = live ? v[8 * j + 2 * m + 1] : 0.0f;
            const __half2 h2 = __floats2half2_rn(v0, v1);
            const float2 f2 = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(v0 - f2.x, v1 - f2.y);
            hw[m] = *reinterpret_cast<const unsigned int*>(&h2);
            lw[m] = *reinterpret_cast<const unsigned int*>(&l2);
          }
          unsigned char* oh = a2 + (size_t)(4 * c + j) * 512;
          if (smem_in_bounds(oh, 16, err) && smem_in_bounds(oh + kA2Part, 16, err)) {
            *reinterpret_cast<uint4*>(oh) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(oh + kA2Part) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        fence_proxy_async();  // V is read by the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->a2full[buf]);
      }
      tile_base += ntiles;
    }
  } else {
    for (int s = 0; s < it.nsl; ++s) tile_base += (slab_of<true>(it, s).sws / kC5 + kPxT - 1) / kPxT;
  }
  // ------------------------------------------------------------ output
  if (epi) asm volatile("bar.sync 2, 128;" ::: "memory");  // the folded V columns of every slab are visible
  if (epi2) {
    t5_wait(&bars->d2, k.gitem, abort, err);
    tc05_fence_after();
    const int c = warp - 4, yo = lane;
    float d[64];
    __syncwarp();
    tmem_ld64(tmem + ((unsigned int)(32 * c) << 16) + 192, d);
    const float vl = it.foldL ? sm.vfold[32 * c + yo] : 0.0f, vr = it.foldR ? sm.vfold[96 + 32 * c + yo] : 0.0f;
    // the row's 32 outputs of channel c, contiguous in a channel plane
    unsigned int pk[8];
    #pragma unroll
    for (int x = 0; x < 32; ++x) {
      const int n = 31 - x, a = n >> 3, i = n & 7;
      float o = d[16 * a + i] + d[16 * a + 8 + i];
      if (it.foldL) o = fmaf(sm.foldw[64 + x], vl, o);
      if (it.foldR) o = fmaf(sm.foldw[96 + x], vr, o);
      const unsigned int qv = quant_u8(o * kWInv);
      pk[x >> 2] = (x & 3) ? (pk[x >> 2] | (qv << (8 * (x & 3)))) : qv;
    }
    unsigned char* orow = sm.ost + c * 1024 + yo * 32;
    if (smem_in_bounds(orow, 32, err)) {
      reinterpret_cast<uint4*>(orow)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      reinterpret_cast<uint4*>(orow)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    tc05_fence_before();
  }
  k.gr += Q;
  k.gc += it.nsl * it.nchunks;
  k.gtile += tile_base;
  k.gslab += it.nsl;
  k.gitem += 1;
  __syncthreads();  // the staged block is complete; D1, D2 and the tables are no longer read
  if (*abort) {
    // a wait gave up: let the row loads still in flight land and every MMA
    // issued finish (bounded waits) before the CTA stops
    if (prod) {
      // requested chunks whose stage was not released yet: one pending phase each
      for (int qq = 0; qq < issued; ++qq) {
        const int g2 = gr_base + qq;
        if (!mbar_test(&bars->ringfree[g2 % kStages5], g2 / kStages5))
          mbar_wait(&bars->ring[g2 % kStages5], (unsigned int)(g2 / kStages5) & 1u);
      }
      mbar_wait(&bars->d2, (unsigned int)(k.gitem - 1) & 1u);  // the item's commit follows its pass-2 MMAs
    }
    if (tilew && lane == 0) mbar_wait(&bars->tdone[warp - 1], (unsigned int)(k.gslab - 1) & 1u);
    __syncthreads();
    return false;
  }
  tc05_fence_after();
  // write the block's rows, interleaving the channel planes (16-byte stores
  // where the frame's alignment allows)
  const int rowBytes = it.bw * kC5;
  const size_t frame_bytes = (size_t)it.H * it.pitch;
  unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * kC5;
  auto staged = [&](int yo, int l) { return (unsigned int)sm.ost[(l % kC5) * 1024 + yo * 32 + l / kC5]; };
  if (((((size_t)out) | it.pitch | (size_t)rowBytes) & 15) == 0) {
    const int nv = rowBytes >> 4;
    for (int idx = tid; idx < it.bh * nv; idx += kThreads5) {
      const int yo = idx / nv, v = idx - yo * nv;
      unsigned int w[4];
      #pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = 16 * v + 4 * j;
        w[j] = staged(yo, l) | (staged(yo, l + 1) << 8) | (staged(yo, l + 2) << 16) | (staged(yo, l + 3) << 24);
      }
      uint4* o = reinterpret_cast<uint4*>(out + (size_t)yo * it.pitch + 16 * v);
      if (in_bounds(o, 16, it.out, frame_bytes, err)) *o = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int idx = tid; idx < it.bh * rowBytes; idx += kThreads5) {
      const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
      unsigned char* o = out + (size_t)yo * it.pitch + rem;
      if (in_bounds(o, 1, it.out, frame_bytes, err)) *o = (unsigned char)staged(yo, rem);
    }
  }
  return true;
}

template <int RB>
__global__ void __launch_bounds__(kThreads5, 2)
tc05_forward_kernel(const __grid_constant__ FrameSource src, Workspace ws, int rmax, BucketList bl,
                    const __grid_constant__ CUtensorMap tmap1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const T5Layout L = t5_layout(RB, rmax);
  T5Smem sm;
  sm.ring = smem + L.ring;
  sm.a1 = smem + L.a1;
  sm.a2 = smem + L.a2;
  sm.s1 = reinterpret_cast<__half*>(smem + L.s1);
  sm.s2 = reinterpret_cast<__half*>(smem + L.s2);
  sm.U = reinterpret_cast<float*>(smem + L.taps);
  sm.CU = reinterpret_cast<float*>(smem + L.cum);
  sm.edge = smem + L.edge;
  sm.foldw = reinterpret_cast<float*>(smem + L.foldw);
  sm.vfold = reinterpret_cast<float*>(smem + L.vfold);
  sm.ost = smem + L.ost;
  __shared__ __align__(8) T5Bars bars;
  __shared__ int s_abort;
  __shared__ unsigned int s_tmem;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages5; ++i) {
      mbar_init(&bars.ring[i], 1);
      mbar_init(&bars.ringfree[i], kTiles);
    }
    for (int t = 0; t < kTiles; ++t) {
      for (int i = 0; i < kA1Bufs5; ++i) mbar_init(&bars.a1free[t][i], 1);
      mbar_init(&bars.tdone[t], 2);
      mbar_init(&bars.d1free[t], 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars.a2full[i], 4);
      mbar_init(&bars.a2free[i], 1);
    }
    mbar_init(&bars.d2, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 0) {  // tensor memory for D1 and D2 (two CTAs per SM take 256 of 512 columns each)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols5)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const unsigned int tmem = s_tmem;
  const int nent = strip_entries(rmax);
  T5Count k{0, 0, 0, 0, 0};
  tc_item_loop<RB, kC5, true, 8, kSlabEl5>(
      src, tmap1, ws, rmax, bl, reinterpret_cast<int*>(smem + L.starts),
      [&](const Item& it, float c, const void* map, bool map_global, auto& lookahead) {
        if (!map) {  // rows TMA cannot address: the host runs the mma.sync kernel for such launches
          if (threadIdx.x == 0) atomicOr(ws.counters + CNT_ERROR, kFaultRadiusBound);
          return true;
        }
        return t5_item<RB>(it, c, sm, &bars, nent, tmem, &s_abort, map, map_global, k, ws.counters + CNT_ERROR,
                           lookahead);
      });
  tc05_fence_before();
  __syncthreads();  // every MMA was waited for before its accumulator was read
  if (warp == 0) {
    tc05_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols5) : "memory");
  }
}

int t5_rb(const FwdConfig& cfg) { return cfg.rows_per_chunk == 16 ? 16 : 32; }

void* pick_t5(const FwdConfig& cfg) {
  return t5_rb(cfg) == 16 ? reinterpret_cast<void*>(&tc05_forward_kernel<16>)
                          : reinterpret_cast<void*>(&tc05_forward_kernel<32>);
}

}  // namespace

bool tc05_supports(int rmax, int C) { return C == kC5 && rmax <= kMaxRadius5; }

size_t tc05_forward_smem_bytes(const FwdConfig& cfg, int rmax) { return t5_layout(t5_rb(cfg), rmax).total; }

int tc05_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax) {
  if (rmax > kMaxRadius5) return 0;
  const size_t smem = tc05_forward_smem_bytes(cfg, rmax);
  void* k = pick_t5(cfg);
  if (set_smem_attrs(reinterpret_cast<const void*>(k), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // CTAs per SM from shared memory, registers and tensor memory (each CTA
  // takes kTmemCols5 of the SM's 512 columns; the occupancy calculator does
  // not count tensor memory).
  int dev = 0, smem_sm = 0, reserved = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
  const int by_smem = (int)((size_t)smem_sm / per_cta);
  const int regs = ((fa.numRegs + 7) & ~7) * kThreads5;
  const int by_regs = regs > 0 ? 65536 / regs : 0;
  const int by_tmem = (int)(512 / kTmemCols5);
  return std::min(std::min(by_smem, by_regs), by_tmem);
}

cudaError_t launch_tc05_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int grid,
                                cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one) {
  const size_t smem = tc05_forward_smem_bytes(cfg, rmax);
  void* k = pick_t5(cfg);
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (tmap_one) std::memcpy(&map, tmap_one, sizeof(map));
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &b, &map};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(kThreads5);
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
