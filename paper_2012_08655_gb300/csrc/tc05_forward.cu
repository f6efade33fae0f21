// Forward kernel for uint8 HWC RGB frames with both separable passes on the
// 5th-generation tensor cores (tcgen05): the block-wise blur of paper
// Section 2 and Algorithm 1 (taps of Eq. 1 truncated at r = ceil(3 sigma)),
// as the two banded Toeplitz contractions of tc_forward.cu, each issued by a
// single thread as asynchronous tcgen05.mma with its fp32 accumulator in
// tensor memory (TMEM):
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
// One CTA per SM (it takes all 512 TMEM columns), 14 warps in four roles that
// each walk the CTA's items at their own pace, so that the tables and the
// output of one item overlap the passes of its neighbours. An item is one
// block; its folded halo columns are cut into slabs of 160 pixels (five
// tiles of 32 pixels, each tile 128 staged bytes), its rows into chunks of 16.
//   warp 0, lane 0 (control): issues the TMA row boxes of every chunk into a
//     six-stage ring, running ahead into the next item as stages are
//     released, and, polling, the pass-2 MMAs of each tile as its V operand
//     becomes ready, accumulating an item's output in one of two D2 slots.
//   warps 1..5, one per tile: convert the tile's staged bytes of each chunk
//     to fp16 (two A1 buffers per tile) and issue that chunk's pass-1 MMA
//     into the tile's D1 columns. A converted row is indexed by staged byte,
//     alignment padding included, so every 16-byte piece converts in place;
//     the padding is skipped when the tile is read back (TMEM lane = byte).
//   warps 6..9 (TMEM lane quarters 2, 3, 0, 1): after a slab, read each
//     tile's D1 back, add the folded top / bottom rows (clamp-to-edge, as in
//     the other kernels) and write V as fp16 hi / lo into one of two A2
//     buffers.
//   warps 10..13: take the next item from the work list and build its tables
//     (taps, the two tap strips, the fold weights) in one of two table
//     slots, then read the previous item's D2, add the folded left / right
//     columns, round to uint8 and store the block.
// Every frame of a launch must be TMA-loadable (the host uses the mma.sync
// kernel otherwise). Every wait is bounded; a wait that gives up flags
// FOVEA_FAULT_WAIT, every role stops, and the CTA lets its row loads and
// MMAs in flight finish before it exits.
#include <algorithm>
#include <cstring>

#include "tc05_common.cuh"

namespace fovea {

namespace {

using namespace fwd;
using namespace tcc;

constexpr int kC5 = 3;                      // channels this kernel serves
constexpr int kRB5 = 16;                    // staged rows per chunk (one K step)
constexpr int kPxT = 32;                    // pixels per tile
constexpr int kElT = kPxT * kC5;            // 96 element columns per tile
constexpr int kTiles = 5;                   // tiles per slab
constexpr int kSlabEl5 = kTiles * kElT;     // 480 elements per slab
constexpr int kBoxes5 = 4;                  // 128-byte tensor-map boxes per staged row
constexpr int kRowB5 = kBoxes5 * 128;       // staged bytes per row
constexpr int kA1T = 16 * kRB5 * 16;        // one tile's converted chunk (128 bytes x 16 rows, fp16)
constexpr int kA2Part = 16 * 4 * 128;       // one V part (hi or lo) of a tile: 16 M cores x 4 K groups
constexpr int kEdge5 = 2 * kRowB5;          // folded top / bottom staged row of one slab
constexpr int kWarps5 = 14;
constexpr int kThreads5 = 32 * kWarps5;
constexpr int kTileW0 = 1;                  // tile warps 1..5
constexpr int kBackW0 = 6;                  // read-back warps 6..9
constexpr int kTabW0 = 10;                  // table / output warps 10..13
constexpr int kTabThreads = 128;
constexpr int kTabBar = 1;                  // named barrier of the table warps
constexpr unsigned int kTmemCols5 = 512;    // D1: 5 tiles x 64 columns; D2: two slots of 64 at 320
constexpr int kD2Col = kTiles * 64;
constexpr int kSlots5 = 3;                  // items published ahead (table slots)
constexpr int kMaxRadius5 = 192;            // tap strips (two per table slot) grow with r
// f32 accumulator, f16 A and B, A MN-major (bit 15), B K-major, N = 64, M = 128
constexpr unsigned int kIdesc5 = (1u << 4) | (1u << 15) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// A tile's converted chunk (pass-1 A operand, MN-major, 128 staged bytes x 16
// rows): core matrix (K group kg, M core mg) at mg * 256 + kg * 128 bytes,
// i.e. adjacent K groups 128 bytes apart (the descriptor's leading offset)
// and adjacent M cores 256 bytes apart (its stride offset).

// Per-item tables (one of kSlots5 slots): the two tap strips the MMAs read
// and the fold weights and edge-column V the read-back and output use.
struct T5Tab {
  size_t s1, s2, foldw, vfold, bytes;
};

__host__ __device__ inline T5Tab t5_tab(int rmax) {
  T5Tab T;
  const size_t strip = (size_t)strip_entries(rmax) * 256;
  T.s1 = 0;                                                  // pass-1 strip
  T.s2 = T.s1 + strip;                                       // pass-2 strip
  T.foldw = T.s2 + strip;                                    // float [top, bottom by yo; left, right by x][32]
  T.vfold = T.foldw + 128 * 4;                               // float [left, right][c][yo]: V of the edge columns
  T.bytes = (T.vfold + 192 * 4 + 127) & ~(size_t)127;
  return T;
}

struct T5Layout {
  size_t ring, a1, a2, tab, U, CU, edge, ost, starts, total;
  T5Tab T;
};

// stages: ring stages; nb: converted chunks in flight per tile (A1 buffers)
__host__ __device__ inline T5Layout t5_layout(int rmax, int stages, int nb) {
  T5Layout L;
  L.T = t5_tab(rmax);
  L.ring = 0;                                                // u8 [stages][boxes][16][128], swizzled
  L.a1 = L.ring + (size_t)stages * kBoxes5 * kRB5 * 128;     // [tile][buffer][kA1T]
  L.a2 = L.a1 + (size_t)kTiles * nb * kA1T;                  // [2 buffers][hi, lo][kA2Part]
  L.tab = L.a2 + (size_t)2 * 2 * kA2Part;                    // [kSlots5][T5Tab]
  L.U = L.tab + kSlots5 * L.T.bytes;                         // float [2 rmax + 1] taps of the item in hand
  L.CU = L.U + (size_t)((2 * rmax + 1 + 3) & ~3) * 4;        // float [cum_len] their prefix sums
  L.edge = L.CU + (size_t)((cum_len(rmax) + 3) & ~3) * 4;    // u8 [3 slabs][top, bottom][512 staged bytes]
  L.ost = L.edge + (size_t)3 * kEdge5;                       // u8 [C][32 rows][32 columns]
  L.starts = L.ost + 32 * 96;                                // int [rmax + 1] work-list bucket starts
  L.total = L.starts + (size_t)(rmax + 1) * 4 + 1024;        // + alignment slack
  return L;
}

// An item as every role sees it (written by the table warps).
struct T5Slot {
  Item it;
  float c;            // -1 / (2 sigma^2)
  const void* map;    // the frame's tensor map
  int end;            // 1: no more items
};

constexpr int kMaxStages5 = 6, kMaxA1Bufs5 = 3;

struct T5Bars {
  unsigned long long ring[kMaxStages5];           // TMA bytes of a ring stage landed (count 1 + tx)
  unsigned long long ringfree[kMaxStages5];       // the tile warps read a stage (5)
  unsigned long long a1free[kTiles][kMaxA1Bufs5]; // the MMAs that read a tile's A1 buffer finished (commit)
  unsigned long long tdone[kTiles];             // a tile's pass-1 MMAs of a slab finished, edge rows stashed (2)
  unsigned long long d1free[kTiles];            // the read-back warps read a tile's D1 (4)
  unsigned long long a2full[2];                 // a tile's V written (4 warps)
  unsigned long long a2free[2];                 // the pass-2 MMAs that read an A2 buffer finished (commit)
  unsigned long long itemfull[kSlots5];         // an item slot and its tables are ready (1)
  unsigned long long vready[kSlots5];           // the read-back warps finished an item (its V columns) (4)
  unsigned long long d2full[2];                 // every pass-2 MMA of an item finished (commit)
  unsigned long long d2free[2];                 // the output warps read a D2 slot (4)
  unsigned long long drain[kTiles + 1];         // the MMAs a thread issued finished (abandoned launches)
};

__device__ __forceinline__ bool t5_wait(unsigned long long* bar, int use, volatile int* abort, unsigned int* err) {
  if (*abort) return false;
  if (mbar_wait(bar, (unsigned int)use & 1u)) return true;
  atomicOr(err, kFaultWait);
  *abort = 1;
  return false;
}

// Every lane of a warp waits; the warp goes on only if every lane's wait
// succeeded (so the lanes never part ways).
__device__ __forceinline__ bool warp_wait(unsigned long long* bar, int use, volatile int* abort, unsigned int* err) {
  const bool ok = t5_wait(bar, use, abort, err);
  return __all_sync(0xffffffffu, ok);
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

__device__ __forceinline__ void tab_sync() { asm volatile("bar.sync %0, %1;" ::"n"(kTabBar), "n"(kTabThreads) : "memory"); }

// Tiles of a slab of `sws` elements.
__device__ __forceinline__ int slab_tiles(int sws) { return (sws / kC5 + kPxT - 1) / kPxT; }

struct T5Args {
  FrameSource src;
  Workspace ws;
  int rmax;
  BucketList bl;
  const CUtensorMap* tmap1;
  unsigned char* smem;
  T5Layout L;
  T5Slot* slots;
  T5Bars* bars;
  volatile int* abort;
  volatile int* tab_stop;   // the table warps' common view of abort
  unsigned int* err;
  unsigned int tmem;
  int n_items;
  const CUtensorMap* batch_maps;
  const int* starts;
};

__device__ __forceinline__ unsigned char* tab_base(const T5Args& A, int j) {
  return A.smem + A.L.tab + (size_t)(j % kSlots5) * A.L.T.bytes;
}

// ------------------------------------------------------------------ control
// Warp 0, lane 0: TMA producer and pass-2 MMA issuer in one polling loop.
// Returns the number of chunks it requested.
template <int S>
__device__ int t5_control(const T5Args& A) {
  T5Bars* bars = A.bars;
  constexpr size_t stage_bytes = (size_t)kBoxes5 * kRB5 * 128;
  const unsigned long long a2d = umma_desc(A.smem + A.L.a2, 128, 512);
  // producer: item pj, its chunks issued so far; gq chunks in all
  int pj = 0, gq = 0, p_issued = 0, p_slab = 0, p_chunk = 0, p_x = 0, p_q = 0;
  bool p_have = false, p_end = false;
  // issuer: item ij, its tiles done so far; gtl tiles in all
  int ij = 0, gtl = 0, i_done = 0, i_total = 0, i_tslab = 0, i_ttile = 0, i_tiles = 0, i_npx = 0, d2_started = 0;
  bool i_have = false, i_end = false, i_d2ok = false;
  unsigned long long s2d = 0;
  int idle = 0;
  while (!(p_end && i_end) && !*A.abort) {
    bool progress = false;
    // ---- producer: the next chunk's four TMA boxes into its ring stage
    if (!p_end) {
      if (!p_have && mbar_test(&bars->itemfull[pj % kSlots5], pj / kSlots5)) {
        const T5Slot& P = A.slots[pj % kSlots5];
        if (P.end) {
          p_end = true;
        } else {
          p_have = true;
          p_issued = p_slab = p_chunk = 0;
          p_q = P.it.nsl * P.it.nchunks;
          if (A.batch_maps) fence_tensormap_acquire(P.map);
        }
        progress = true;
      }
      if (p_have && (gq < S || mbar_test(&bars->ringfree[gq % S], gq / S - 1))) {
        const T5Slot& P = A.slots[pj % kSlots5];
        if (p_chunk == 0) {
          const Slab cs = slab_of<true>(P.it, p_slab);
          p_x = (int)cs.src - cs.ph;  // 16-byte aligned byte column
        }
        const int stg = gq % S;
        unsigned char* dst = A.smem + A.L.ring + (size_t)stg * stage_bytes;
        const int y = P.it.gy0 - P.it.ph + p_chunk * kRB5;
        mbar_expect_tx(&bars->ring[stg], (unsigned int)kBoxes5 * 128u * kRB5);
        #pragma unroll
        for (int bx = 0; bx < kBoxes5; ++bx)
          tma_load_2d(dst + 128 * kRB5 * bx, P.map, p_x + 128 * bx, y, &bars->ring[stg]);
        ++gq;
        if (++p_chunk == P.it.nchunks) {
          p_chunk = 0;
          ++p_slab;
        }
        if (++p_issued == p_q) {
          p_have = false;
          ++pj;
        }
        progress = true;
      }
    }
    // ---- issuer: the pass-2 MMAs of the next tile whose V is written
    if (!i_end) {
      if (!i_have && mbar_test(&bars->itemfull[ij % kSlots5], ij / kSlots5)) {
        const T5Slot& I = A.slots[ij % kSlots5];
        if (I.end) {
          i_end = true;
        } else {
          i_have = true;
          i_done = i_tslab = i_ttile = 0;
          i_total = 0;
          for (int s = 0; s < I.it.nsl; ++s) i_total += slab_tiles(slab_of<true>(I.it, s).sws);
          i_d2ok = ij < 2;
          d2_started = 0;
        }
        progress = true;
      }
      if (i_have && !i_d2ok && mbar_test(&bars->d2free[ij & 1], (ij >> 1) - 1)) {
        i_d2ok = true;  // the output warps read the slot's previous item
        progress = true;
      }
      if (i_have && i_d2ok && mbar_test(&bars->a2full[gtl & 1], gtl >> 1)) {
        const T5Slot& I = A.slots[ij % kSlots5];
        const int buf = gtl & 1;
        if (i_ttile == 0) {  // first tile of a slab: its geometry and strip base
          const Slab cs = slab_of<true>(I.it, i_tslab);
          i_npx = cs.sws / kC5;
          i_tiles = slab_tiles(cs.sws);
          const int P0 = cs.e0 / kC5, delta2 = (I.it.offx + 1) & 7;
          // strip entry of pixel p0 of the slab: (offx + P0 + p0 - 31 - delta2) / 8 + kXOff
          s2d = umma_desc(tab_base(A, ij) + A.L.T.s2, 256, 128) +
                (unsigned long long)(16 * ((I.it.offx + P0 - 31 - delta2) / 8 + kXOff));
        }
        tc05_fence_after();
        const unsigned int d2 = A.tmem + kD2Col + 64 * (ij & 1);
        #pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int p0 = kPxT * i_ttile + 16 * ks;
          if (p0 >= i_npx) break;
          const unsigned long long bd = s2d + (unsigned long long)(32 * (p0 >> 4));
          #pragma unroll
          for (int part = 0; part < 2; ++part) {
            umma_f16(d2, a2d + (unsigned long long)((buf * 2 + part) * (kA2Part >> 4) + 16 * ks), bd, kIdesc5,
                     d2_started);
            d2_started = 1;
          }
        }
        umma_commit(&bars->a2free[buf]);
        ++gtl;
        if (++i_ttile == i_tiles) {
          i_ttile = 0;
          ++i_tslab;
        }
        if (++i_done == i_total) {
          umma_commit(&bars->d2full[ij & 1]);
          i_have = false;
          ++ij;
        }
        progress = true;
      }
    }
    if (progress) {
      idle = 0;
    } else if (++idle > kWaitLimit) {
      atomicOr(A.err, kFaultWait);
      *A.abort = 1;
    } else {
      __nanosleep(20);
    }
  }
  return gq;
}

// ------------------------------------------------------------------ tile warps
template <int S, int NB>
__device__ void t5_tiles(const T5Args& A, int t) {
  T5Bars* bars = A.bars;
  const int lane = threadIdx.x & 31;
  constexpr size_t stage_bytes = (size_t)kBoxes5 * kRB5 * 128;
  unsigned char* a1base = A.smem + A.L.a1 + (size_t)t * NB * kA1T;
  const unsigned long long a1d = umma_desc(a1base, 128, kRB5 * 16);
  // this lane's units (row rho, 16-byte group ge) of the tile's 128 staged
  // bytes: rho = lane % 16 and ge = lane / 16 + 2 i, the same in every chunk,
  // so their ring and A1 offsets are worked out once
  const int rho = lane & 15;
  int roff[kRB5 / 4], aoff[kRB5 / 4], boff[kRB5 / 4];
  #pragma unroll
  for (int i = 0; i < kRB5 / 4; ++i) {
    const int ge = (lane >> 4) + 2 * i;
    boff[i] = kElT * t + 16 * ge;  // staged byte
    roff[i] = ring_off<kRB5>(rho, boff[i]);
    aoff[i] = (2 * ge) * (kRB5 * 16) + (rho >> 3) * 128 + (rho & 7) * 16;
  }
  int g = 0, gs = 0;  // chunks (ring and A1 alike) and slabs so far
  for (int j = 0;; ++j) {
    if (!warp_wait(&bars->itemfull[j % kSlots5], j / kSlots5, A.abort, A.err)) return;
    const T5Slot& sl = A.slots[j % kSlots5];
    if (sl.end) return;
    const Item& it = sl.it;
    const int r = it.r, nsl = it.nsl, nchunks = it.nchunks, ph = it.ph;
    const int D0 = it.offy - ph;  // tap(v, yo) = v + D0 - yo; a multiple of 16, >= 0
    const int k_end = min(it.vrows, 32 - D0 + 2 * r);  // K steps with a tap of the 32 output rows
    const int vb = ph + it.EH - 1;                     // virtual row of the folded bottom row
    const int kq_b = vb / kRB5;                        // its chunk (the top row's is chunk 0)
    // strip entry 2 kidx + D0 / 8 + 4 for K step kidx (delta1 = (D0 + 1) & 7 = 1)
    const unsigned long long s1d =
        umma_desc(tab_base(A, j) + A.L.T.s1, 256, 128) + (unsigned long long)(16 * (D0 / 8 + 4));
    for (int s = 0; s < nsl; ++s, ++gs) {
      const bool active = t < slab_tiles(slab_of<true>(it, s).sws);
      unsigned char* edge = A.smem + A.L.edge + (size_t)(gs % 3) * kEdge5;
      int started = 0;
      for (int kq = 0; kq < nchunks; ++kq, ++g) {
        const int stg = g % S, buf = g % NB;
        if (!warp_wait(&bars->ring[stg], g / S, A.abort, A.err)) return;
        // every tile warp commits once per chunk (an inactive tile with no
        // MMA at all), so the buffers' phases stay in step
        if (g >= NB && !warp_wait(&bars->a1free[t][buf], g / NB - 1, A.abort, A.err)) return;
        if (active) {
          // all the loads first, then the conversions and stores
          const unsigned char* st = A.smem + A.L.ring + (size_t)stg * stage_bytes;
          uint4 w[kRB5 / 4];
          #pragma unroll
          for (int i = 0; i < kRB5 / 4; ++i) w[i] = *reinterpret_cast<const uint4*>(st + roff[i]);
          if (kq == 0 || kq == kq_b) {  // the folded edge rows (both, if EH = 1)
            const int vv = kq * kRB5 + rho;
            #pragma unroll
            for (int i = 0; i < kRB5 / 4; ++i) {
              if (kq == 0 && vv == ph && smem_in_bounds(edge + boff[i], 16, A.err))
                *reinterpret_cast<uint4*>(edge + boff[i]) = w[i];
              if (vv == vb && smem_in_bounds(edge + kRowB5 + boff[i], 16, A.err))
                *reinterpret_cast<uint4*>(edge + kRowB5 + boff[i]) = w[i];
            }
          }
          unsigned char* a1 = a1base + (size_t)buf * kA1T;
          #pragma unroll
          for (int i = 0; i < kRB5 / 4; ++i) {
            const uint4 lo = make_uint4(__byte_perm(w[i].x, 0u, 0x4140), __byte_perm(w[i].x, 0u, 0x4342),
                                        __byte_perm(w[i].y, 0u, 0x4140), __byte_perm(w[i].y, 0u, 0x4342));
            const uint4 hi = make_uint4(__byte_perm(w[i].z, 0u, 0x4140), __byte_perm(w[i].z, 0u, 0x4342),
                                        __byte_perm(w[i].w, 0u, 0x4140), __byte_perm(w[i].w, 0u, 0x4342));
            unsigned char* o = a1 + aoff[i];
            if (smem_in_bounds(o, 16, A.err) && smem_in_bounds(o + kRB5 * 16, 16, A.err)) {
              *reinterpret_cast<uint4*>(o) = lo;
              *reinterpret_cast<uint4*>(o + kRB5 * 16) = hi;
            }
          }
          fence_proxy_async();  // the converted chunk is read by the tensor cores
        }
        __syncwarp();
        bool ok = true;
        if (lane == 0) {
          mbar_arrive(&bars->ringfree[stg]);  // this warp is done with the stage
          // the read-back of the tile's previous slab is done (also when the
          // tile is inactive: otherwise its slab commits could run two phases
          // ahead of the read-back warps' parity waits on tdone)
          if (kq == 0 && gs > 0) ok = t5_wait(&bars->d1free[t], gs - 1, A.abort, A.err);
          const int k0 = kq * kRB5;
          if (ok && active && k0 < k_end) {
            tc05_fence_after();
            umma_f16(A.tmem + 64 * t, a1d + (unsigned long long)(buf * (kA1T >> 4)),
                     s1d + (unsigned long long)(32 * (k0 >> 4)), kIdesc5, started);
            started = 1;
          }
          umma_commit(&bars->a1free[t][buf]);
        }
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) return;
      }
      if (lane == 0) {
        umma_commit(&bars->tdone[t]);  // the tile's pass-1 MMAs of the slab (none if inactive)
        mbar_arrive(&bars->tdone[t]);  // and (release) the warp's edge-row stash
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------ read-back warps
__device__ void t5_readback(const T5Args& A, int q) {
  T5Bars* bars = A.bars;
  const int lane = threadIdx.x & 31;
  const int lane_t = 32 * q + lane;  // TMEM lane = staged byte of the tile
  int gs = 0, gtl = 0;
  for (int j = 0;; ++j) {
    if (!warp_wait(&bars->itemfull[j % kSlots5], j / kSlots5, A.abort, A.err)) return;
    const T5Slot& sl0 = A.slots[j % kSlots5];
    if (sl0.end) return;
    const Item& it = sl0.it;
    unsigned char* tb = tab_base(A, j);
    const float* foldw = reinterpret_cast<const float*>(tb + A.L.T.foldw);
    float* vfold = reinterpret_cast<float*>(tb + A.L.T.vfold);
    for (int s = 0; s < it.nsl; ++s, ++gs) {
      const Slab sl = slab_of<true>(it, s);
      const int npx = sl.sws / kC5;
      const int ntiles = slab_tiles(sl.sws);
      const int P0 = sl.e0 / kC5;
      const unsigned char* edge = A.smem + A.L.edge + (size_t)(gs % 3) * kEdge5;
      const int el = lane_t - sl.ph;  // element of the tile (0 .. 95 for its 32 pixels)
      const bool mine = el >= 0 && el < kElT;
      const int px = mine ? el / kC5 : 0, c = mine ? el - px * kC5 : 0;
      for (int t = 0; t < kTiles; ++t) {
        if (!warp_wait(&bars->tdone[t], gs, A.abort, A.err)) return;
        if (t >= ntiles) {  // keep the tile's D1 phase in step
          if (lane == 0) mbar_arrive(&bars->d1free[t]);
          continue;
        }
        tc05_fence_after();
        const int buf = gtl & 1;
        if (gtl >= 2 && !warp_wait(&bars->a2free[buf], (gtl >> 1) - 1, A.abort, A.err)) return;
        float d[64];
        tmem_ld64(A.tmem + ((unsigned int)(32 * q) << 16) + 64 * t, d);
        tc05_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->d1free[t]);  // D1 of the tile is read: its next slab may start
        const int b = kElT * t + lane_t;  // staged byte
        const int spx = kPxT * t + px;    // slab pixel
        const int pg = P0 + spx;          // folded pixel
        const bool live = mine && spx < npx;
        const float et = it.foldT ? (float)edge[b] : 0.0f, eb = it.foldB ? (float)edge[kRowB5 + b] : 0.0f;
        float v[32];
        #pragma unroll
        for (int yo = 0; yo < 32; ++yo) {
          // column 16 a + 8 p + i holds part p of output row 31 - (8 a + i)
          const int n = 31 - yo, a = n >> 3, i = n & 7;
          float x = d[16 * a + i] + d[16 * a + 8 + i];
          if (it.foldT) x = fmaf(foldw[yo], et, x);
          if (it.foldB) x = fmaf(foldw[32 + yo], eb, x);
          v[yo] = x * kVScale;
        }
        if (live && it.foldL && pg == 0) {
          #pragma unroll
          for (int yo = 0; yo < 32; ++yo) vfold[32 * c + yo] = v[yo];
        }
        if (live && it.foldR && pg == it.EW - 1) {
          #pragma unroll
          for (int yo = 0; yo < 32; ++yo) vfold[96 + 32 * c + yo] = v[yo];
        }
        unsigned char* a2 = A.smem + A.L.a2 + (size_t)buf * 2 * kA2Part + (px >> 3) * 128 + (px & 7) * 16;
        #pragma unroll
        for (int jj = 0; jj < 4 && mine; ++jj) {
          unsigned int hw[4], lw[4];
          #pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float v0 = live ? v[8 * jj + 2 * m] : 0.0f, v1 = live ? v[8 * jj + 2 * m + 1] : 0.0f;
            const __half2 h2 = __floats2half2_rn(v0, v1);
            const float2 f2 = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(v0 - f2.x, v1 - f2.y);
            hw[m] = *reinterpret_cast<const unsigned int*>(&h2);
            lw[m] = *reinterpret_cast<const unsigned int*>(&l2);
          }
          unsigned char* oh = a2 + (size_t)(4 * c + jj) * 512;
          if (smem_in_bounds(oh, 16, A.err) && smem_in_bounds(oh + kA2Part, 16, A.err)) {
            *reinterpret_cast<uint4*>(oh) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(oh + kA2Part) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        fence_proxy_async();  // V is read by the tensor cores
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->a2full[buf]);
        ++gtl;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&bars->vready[j % kSlots5]);  // the item's folded V columns are written
  }
}

// ------------------------------------------------------------------ table / output warps
struct T5Fetch {
  int next_tk;   // ticket taken ahead
  int nx_item;   // its item (once looked up)
  ItemInfo nx_inf;
  int stage;     // 0: ticket only, 1: item looked up, 2: record loaded
};

__device__ __forceinline__ int t5_lookup(const T5Args& A, int tk) {
  if (!A.bl.list) return A.ws.order[tk];
  int lo = 0, hi = A.bl.nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (A.starts[mid] <= tk) hi = mid; else lo = mid + 1;
  }
  return A.bl.list[(size_t)lo * A.bl.cap + (tk - A.starts[lo])];
}

// Thread 0 of the table warps: the next valid item into slot `sl` (or the
// end mark). Items the kernel cannot serve are flagged and skipped.
__device__ void t5_fetch(const T5Args& A, T5Fetch& F, T5Slot& sl) {
  for (;;) {
    if (F.next_tk >= A.n_items) {
      sl.end = 1;
      return;
    }
    if (F.stage < 1) F.nx_item = t5_lookup(A, F.next_tk);
    const int item = F.nx_item;
    if ((unsigned)item >= (unsigned)A.n_items) {
      atomicOr(A.err, kFaultWorklist);
      F.next_tk = (int)atomicAdd(&A.ws.counters[CNT_TICKET], 1u);
      F.stage = 0;
      continue;
    }
    const ItemInfo inf = F.stage >= 2 ? F.nx_inf : A.ws.items[item];
    F.next_tk = (int)atomicAdd(&A.ws.counters[CNT_TICKET], 1u);
    F.stage = 0;
    const FrameDesc fd = load_frame(A.src, inf.frame);
    const void* map = !fd.tma ? nullptr
                              : (A.batch_maps ? static_cast<const void*>(A.batch_maps + inf.frame)
                                              : static_cast<const void*>(A.tmap1));
    if (inf.r > A.rmax || fd.fmt != FOVEA_U8_HWC || fd.C != kC5 || !map) {
      // rows TMA cannot address: the host runs the mma.sync kernel for such launches
      atomicOr(A.err, kFaultRadiusBound);
      continue;
    }
    item_geometry(sl.it, inf, fd, kRB5, true, kSlabEl5);
    sl.c = inf.neg_half_inv_s2;
    sl.map = map;
    sl.end = 0;
    return;
  }
}

// Item j (or the end mark) into slot j % kSlots5, with its tables. The
// slot's previous item (j - kSlots5) was output by these warps before, so
// every role is done with it. Returns false at the end mark (the same in every thread).
__device__ bool t5_publish(const T5Args& A, T5Fetch& F, int j, int nent) {
  const int tt = threadIdx.x - 32 * kTabW0, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T5Slot& sl = A.slots[j % kSlots5];
  if (tt == 0) t5_fetch(A, F, sl);
  tab_sync();
  const bool end = sl.end != 0;
  if (!end) {
    const Item& it = sl.it;
    const int r = it.r;
    const float c = sl.c;
    unsigned char* tb = tab_base(A, j);
    float* U = reinterpret_cast<float*>(A.smem + A.L.U);
    float* CU = reinterpret_cast<float*>(A.smem + A.L.CU);
    float* foldw = reinterpret_cast<float*>(tb + A.L.T.foldw);
    __half* s1 = reinterpret_cast<__half*>(tb + A.L.T.s1);
    __half* s2 = reinterpret_cast<__half*>(tb + A.L.T.s2);
    // the taps once, then the two tap strips and the folds' weights from them
    const float S = warp_tap_sum(r, c);
    for (int m = tt; m <= 2 * r; m += kTabThreads) U[m] = tap_u(m, r, c, S);
    tab_sync();
    const int D0 = it.offy - it.ph;
    const int delta1 = (D0 + 1) & 7, delta2 = (it.offx + 1) & 7;
    for (int idx = tt; idx < 2 * nent * 8; idx += kTabThreads) {
      // one (strip, entry, row): the row's 8 taps as one 16-byte store each
      // of the hi and the lo parts (the layout of make_strips_tab)
      const int which = idx >= nent * 8, e = which ? idx - nent * 8 : idx;
      const int jj = e >> 3, rho = e & 7;
      const int m0 = 8 * (jj - kXOff) + rho + (which ? delta2 : delta1);
      unsigned int hw[4], lw[4];
      #pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float w0 = tap_at(U, m0 + 2 * i, r) * kWScale, w1 = tap_at(U, m0 + 2 * i + 1, r) * kWScale;
        const __half h0 = __float2half_rn(w0), h1 = __float2half_rn(w1);
        hw[i] = pack_half2(h0, h1);
        lw[i] = pack_half2(__float2half_rn(w0 - __half2float(h0)), __float2half_rn(w1 - __half2float(h1)));
      }
      __half* o = (which ? s2 : s1) + jj * 128 + rho * 8;
      *reinterpret_cast<uint4*>(o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(o + 64) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    if ((it.foldT || it.foldB || it.foldL || it.foldR) && warp == kTabW0) {
      make_cumulative_tab(CU, U, r);
      __syncwarp();
      // rows: weight of the folded top / bottom row for output row yo = lane
      // (in pass-1 accumulator units); columns: of the folded left / right
      // column for output column x = lane (in pass-2 accumulator units)
      foldw[lane] = cum_at(CU, it.offy - lane, r) * (kWScale * kDScale);
      foldw[32 + lane] = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - lane), r) * (kWScale * kDScale);
      foldw[64 + lane] = it.foldL ? cum_at(CU, it.offx - lane, r) * kWScale : 0.0f;
      foldw[96 + lane] = it.foldR ? cum_at(CU, 2 * r + 1 - (it.offx + it.EW - lane), r) * kWScale : 0.0f;
    }
    fence_proxy_async();  // the strips are read by the tensor cores
  }
  tab_sync();
  if (tt == 0) mbar_arrive(&A.bars->itemfull[j % kSlots5]);
  return !end;
}

// Item j's output: D2 (with the folded left / right columns) rounded to
// uint8, staged by channel planes, then stored row by row. Returns false
// (in every thread alike) once a wait gave up.
__device__ bool t5_output(const T5Args& A, int j) {
  T5Bars* bars = A.bars;
  const int tt = threadIdx.x - 32 * kTabW0, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp & 3;  // TMEM lane quarter = channel (quarter 3 unused)
  const T5Slot& sl = A.slots[j % kSlots5];
  const Item& it = sl.it;
  unsigned char* tb = tab_base(A, j);
  const float* foldw = reinterpret_cast<const float*>(tb + A.L.T.foldw);
  const float* vfold = reinterpret_cast<const float*>(tb + A.L.T.vfold);
  unsigned char* ost = A.smem + A.L.ost;
  const bool ok = warp_wait(&bars->vready[j % kSlots5], j / kSlots5, A.abort, A.err) &&
                  warp_wait(&bars->d2full[j & 1], j >> 1, A.abort, A.err);
  if (ok && c < kC5) {
    tc05_fence_after();
    const int yo = lane;
    float d[64];
    tmem_ld64(A.tmem + ((unsigned int)(32 * c) << 16) + kD2Col + 64 * (j & 1), d);
    tc05_fence_before();
    const float vl = it.foldL ? vfold[32 * c + yo] : 0.0f, vr = it.foldR ? vfold[96 + 32 * c + yo] : 0.0f;
    // the row's 32 outputs of channel c, contiguous in a channel plane
    unsigned int pk[8];
    #pragma unroll
    for (int x = 0; x < 32; ++x) {
      const int n = 31 - x, a = n >> 3, i = n & 7;
      float o = d[16 * a + i] + d[16 * a + 8 + i];
      if (it.foldL) o = fmaf(foldw[64 + x], vl, o);
      if (it.foldR) o = fmaf(foldw[96 + x], vr, o);
      const unsigned int qv = quant_u8(o * kWInv);
      pk[x >> 2] = (x & 3) ? (pk[x >> 2] | (qv << (8 * (x & 3)))) : qv;
    }
    unsigned char* orow = ost + c * 1024 + yo * 32;
    if (smem_in_bounds(orow, 32, A.err)) {
      reinterpret_cast<uint4*>(orow)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      reinterpret_cast<uint4*>(orow)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&bars->d2free[j & 1]);  // the D2 slot may take the item after next
  if (tt == 0) *A.tab_stop = *A.abort;
  tab_sync();
  if (*A.tab_stop) return false;
  // write the block's rows, interleaving the channel planes (16-byte stores
  // where the frame's alignment allows)
  const int rowBytes = it.bw * kC5;
  const size_t frame_bytes = (size_t)it.H * it.pitch;
  unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * kC5;
  auto staged = [&](int yo, int l) { return (unsigned int)ost[(l % kC5) * 1024 + yo * 32 + l / kC5]; };
  if (((((size_t)out) | it.pitch | (size_t)rowBytes) & 15) == 0) {
    const int nv = rowBytes >> 4;
    for (int idx = tt; idx < it.bh * nv; idx += kTabThreads) {
      const int yo = idx / nv, v = idx - yo * nv;
      unsigned int w[4];
      #pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int l = 16 * v + 4 * k;
        w[k] = staged(yo, l) | (staged(yo, l + 1) << 8) | (staged(yo, l + 2) << 16) | (staged(yo, l + 3) << 24);
      }
      uint4* o = reinterpret_cast<uint4*>(out + (size_t)yo * it.pitch + 16 * v);
      if (in_bounds(o, 16, it.out, frame_bytes, A.err)) *o = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int idx = tt; idx < it.bh * rowBytes; idx += kTabThreads) {
      const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
      unsigned char* o = out + (size_t)yo * it.pitch + rem;
      if (in_bounds(o, 1, it.out, frame_bytes, A.err)) *o = (unsigned char)staged(yo, rem);
    }
  }
  tab_sync();  // the staging buffer is free for the next item
  return true;
}

__device__ void t5_tables(const T5Args& A) {
  const int tt = threadIdx.x - 32 * kTabW0;
  const int nent = strip_entries(A.rmax);
  T5Fetch F;
  F.stage = 0;
  F.nx_item = -1;
  F.next_tk = 0;
  if (tt == 0) F.next_tk = (int)atomicAdd(&A.ws.counters[CNT_TICKET], 1u);
  // keep kSlots5 - 1 items published ahead of the one being output; `pub`
  // is the next index to publish, `ended` once the end mark went out (at
  // index pub - 1). All of it is the same in every table thread.
  int pub = 0;
  bool ended = false;
  while (pub < kSlots5 - 1 && !ended) ended = !t5_publish(A, F, pub++, nent);
  for (int j = 0; !ended || j < pub - 1; ++j) {
    if (!ended) ended = !t5_publish(A, F, pub++, nent);  // item j + kSlots5 - 1 into the slot of item j - 1
    // look the following ticket's item up now, and load its record after the
    // output, so the work list's dependent loads overlap the output
    if (tt == 0 && F.stage == 0 && F.next_tk < A.n_items) {
      F.nx_item = t5_lookup(A, F.next_tk);
      F.stage = 1;
    }
    if (!t5_output(A, j)) return;
    if (tt == 0 && F.stage == 1 && (unsigned)F.nx_item < (unsigned)A.n_items) {
      F.nx_inf = A.ws.items[F.nx_item];
      F.stage = 2;
    }
  }
}

template <int S, int NB>
__global__ void __launch_bounds__(kThreads5, 1)
tc05_forward_kernel(const __grid_constant__ FrameSource src, Workspace ws, int rmax, BucketList bl,
                    const __grid_constant__ CUtensorMap tmap1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) T5Bars bars;
  __shared__ __align__(16) T5Slot slots[kSlots5];
  __shared__ int s_abort, s_tab_stop, s_last;
  __shared__ unsigned int s_tmem;
  __shared__ int s_wsum[kWarps5];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&bars.ring[i], 1);
      mbar_init(&bars.ringfree[i], kTiles);
    }
    for (int t = 0; t < kTiles; ++t) {
      for (int i = 0; i < NB; ++i) mbar_init(&bars.a1free[t][i], 1);
      mbar_init(&bars.tdone[t], 2);
      mbar_init(&bars.d1free[t], 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars.a2full[i], 4);
      mbar_init(&bars.a2free[i], 1);
      mbar_init(&bars.d2full[i], 1);
      mbar_init(&bars.d2free[i], 4);
    }
    for (int i = 0; i < kSlots5; ++i) {
      mbar_init(&bars.itemfull[i], 1);
      mbar_init(&bars.vready[i], 4);
    }
    for (int i = 0; i <= kTiles; ++i) mbar_init(&bars.drain[i], 1);
    s_abort = 0;
    s_tab_stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 0) {  // all 512 tensor-memory columns (one CTA per SM)
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols5)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  T5Args A;
  A.src = src;
  A.ws = ws;
  A.rmax = rmax;
  A.bl = bl;
  A.tmap1 = &tmap1;
  A.smem = smem;
  A.L = t5_layout(rmax, S, NB);
  A.slots = slots;
  A.bars = &bars;
  A.abort = &s_abort;
  A.tab_stop = &s_tab_stop;
  A.err = ws.counters + CNT_ERROR;
  A.n_items = bl.list != nullptr ? (int)src.one_total : (int)ws.counters[CNT_NITEMS];
  A.batch_maps = src.hdr ? reinterpret_cast<const CUtensorMap*>(reinterpret_cast<const char*>(src.hdr) +
                                                                src.hdr->maps_offset)
                         : nullptr;
  int* starts = reinterpret_cast<int*>(smem + A.L.starts);
  A.starts = starts;
  // the work list's bucket starts (kBuckets positions over the first 256
  // threads; the others see none but join the block barriers)
  if (bl.list) bucket_starts<256>(ws.counters + CNT_HIST, bl.nb, starts, s_wsum);
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  A.tmem = s_tmem;

  int gq = 0;
  if (tid == 0) {
    gq = t5_control<S>(A);
  } else if (warp >= kTileW0 && warp < kTileW0 + kTiles) {
    t5_tiles<S, NB>(A, warp - kTileW0);
  } else if (warp >= kBackW0 && warp < kBackW0 + 4) {
    t5_readback(A, warp & 3);
  } else if (warp >= kTabW0) {
    t5_tables(A);
  }
  __syncwarp();
  tc05_fence_before();
  __syncthreads();  // every role is done (every MMA was waited for, unless a wait gave up)
  if (s_abort) {
    // a wait gave up: let the row loads still in flight land and every MMA
    // issued finish (bounded waits) before the CTA stops
    if (tid == 0) {
      for (int s = 0; s < S && s < gq; ++s) {
        const int last = s + S * ((gq - 1 - s) / S);  // the stage's last chunk
        mbar_wait(&bars.ring[s], (unsigned int)(last / S) & 1u);
      }
    }
    const int k = tid == 0 ? 0 : (warp >= kTileW0 && warp < kTileW0 + kTiles && lane == 0 ? warp : -1);
    if (k >= 0) {
      umma_commit(&bars.drain[k]);
      mbar_wait(&bars.drain[k], 0u);
    }
  }
  tc05_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc05_fence_after();
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(A.tmem), "r"(kTmemCols5)
                 : "memory");
  }
  if (bl.list) {  // the last CTA resets the work list's counters for the next launch
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(&ws.counters[CNT_DONE_SIGMA], 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
      for (int j = tid; j < kBuckets; j += kThreads5) ws.counters[CNT_HIST + j] = 0u;
      if (tid == 0) {
        ws.counters[CNT_TICKET] = 0u;
        ws.counters[CNT_DONE_SIGMA] = 0u;
      }
    }
  }
}


// The variants by depth: (ring stages, A1 buffers per tile), deepest first;
// a launch runs the deepest whose shared memory fits.
struct T5Variant {
  int stages, nb;
  void* fn;
};

const T5Variant* t5_variants(int* n) {
  static const T5Variant v[] = {{6, 3, reinterpret_cast<void*>(&tc05_forward_kernel<6, 3>)},
                                {5, 3, reinterpret_cast<void*>(&tc05_forward_kernel<5, 3>)},
                                {5, 2, reinterpret_cast<void*>(&tc05_forward_kernel<5, 2>)},
                                {4, 2, reinterpret_cast<void*>(&tc05_forward_kernel<4, 2>)}};
  *n = 4;
  return v;
}

size_t t5_smem(const T5Variant& v, int rmax) {
  // at least half an SM's shared memory, so that two CTAs (each taking all
  // 512 TMEM columns) never share an SM
  return std::max(t5_layout(rmax, v.stages, v.nb).total, (size_t)120 * 1024);
}

// The deepest variant whose shared memory the device grants (nullptr: none).
const T5Variant* t5_pick(int rmax) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  int n = 0;
  const T5Variant* v = t5_variants(&n);
  for (int i = 0; i < n; ++i) {
    // the kernel's static shared memory (barriers, item slots) also counts
    if (t5_smem(v[i], rmax) + 2048 <= (size_t)optin) return &v[i];
  }
  return nullptr;
}

}  // namespace

bool tc05_supports(int rmax, int C) { return C == kC5 && rmax <= kMaxRadius5; }

size_t tc05_forward_smem_bytes(const FwdConfig&, int rmax) {
  const T5Variant* v = t5_pick(rmax);
  return v ? t5_smem(*v, rmax) : 0;
}

int tc05_forward_max_ctas_per_sm(const FwdConfig&, int rmax) {
  if (rmax > kMaxRadius5) return 0;
  const T5Variant* v = t5_pick(rmax);
  if (!v || set_smem_attrs(reinterpret_cast<const void*>(v->fn), t5_smem(*v, rmax)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return 1;  // a CTA takes all of the SM's tensor memory
}

cudaError_t launch_tc05_forward(const FrameSource& src, const Workspace& ws, const FwdConfig&, int rmax, int grid,
                                cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one) {
  const T5Variant* v = t5_pick(rmax);
  if (!v) return cudaErrorInvalidConfiguration;
  const size_t smem = t5_smem(*v, rmax);
  void* k = v->fn;
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
