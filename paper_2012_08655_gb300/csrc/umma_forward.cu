// Tensor-core forward kernel for uint8 HWC frames with pass 1 on the
// 5th-generation tensor cores (tcgen05): the same block-wise separable blur
// (paper Section 2, Algorithm 1; taps of Eq. 1 truncated at r = ceil(3 sigma))
// and the same two banded Toeplitz contractions as tc_forward.cu, but the
// vertical pass, the larger of the two, is issued by one thread as
// asynchronous tcgen05.mma instructions with its accumulator in tensor memory:
//
//   D1[e][n] = sum_v T[v][e] * u(v + n - 31 + D0),    n = 31 - yo,
//
// M = 128 staged byte columns e (two M tiles cover a 256-byte slab row),
// N = 32 output rows (reversed), K = 16 staged rows per instruction, fp16
// operands, fp32 accumulation. A (the tile, M x K) is converted from the TMA
// row ring into fp16 K-major core matrices (a byte b becomes the exact fp16
// subnormal b * 2^-24). B (the taps) is a Hankel matrix once its N index is
// reversed: element (n, k) depends on n + k only, so the 8 x 8 core matrix of
// N group a and K group b is entry a + b of one strip of 128-byte core
// matrices, and a matrix descriptor with both strides 128 bytes reads it
// directly; the strip holds the taps scaled by 2^12 split into fp16 hi and
// lo parts, one instruction each. The accumulator is read back with
// tcgen05.ld, the clamp-to-edge folds of the top and bottom rows are added,
// and V = D1 * 2^12 goes to shared memory as fp16 hi/lo rows for pass 2,
// which runs on mma.sync exactly as in tc_forward.cu (tc_common.cuh).
#include <algorithm>
#include <cstring>

#include "tc05_common.cuh"

namespace fovea {

namespace {

using namespace fwd;
using namespace tcc;

constexpr int kTmemCols = 128;     // D1: two M tiles x 64 fp32 columns (hi and lo parts)
constexpr unsigned int kIdescM128N64 =
    (1u << 4)                      // D format: f32
    | (0u << 7) | (0u << 10)       // A, B format: f16
    | (0u << 15) | (0u << 16)      // A, B K-major
    | ((64u >> 3) << 17)           // N = 64
    | ((128u >> 4) << 24);         // M = 128

__host__ __device__ constexpr int um_stages(int rb) { return 96 / rb; }   // 96 staged rows
constexpr int kMaxUmStages = 6;
// A1 buffers: converted chunks waiting for (or read by) their MMAs; the
// converting warps may run this many chunks ahead of the tensor core.
constexpr int kA1Bufs = 4;
// A1 (pass-1 A operand), one M tile: 16 groups of 8 columns x RB/8 groups of
// 8 rows; K-adjacent core matrices 128 bytes apart, M-adjacent ones
// 16 RB + 16 bytes apart (the 16-byte skew keeps the conversion's 8-byte
// stores free of bank conflicts).
__host__ __device__ constexpr int a1_sbo(int rb) { return 16 * rb + 16; }
__host__ __device__ constexpr int a1_tile_bytes(int rb) { return 16 * a1_sbo(rb); }

struct UmLayout {
  size_t ring, a1, vh, vl, strip, cum, pairs, edge, foldw, starts, total;
};

// Rows (pixel, channel) of the transposed V arrays: the slab's pixels
// rounded up to 16, times C.
__host__ __device__ constexpr int vt_rows(int C) { return C == 1 ? 240 : C == 2 ? 256 : C == 3 ? 240 : 256; }

// Offsets from the 1024-byte aligned start of the dynamic shared memory.
__host__ __device__ inline UmLayout um_layout(int rb, int rmax, int C) {
  UmLayout L;
  const size_t vbytes = (size_t)vt_rows(C) * kVtPitch * 2;
  L.ring = 0;                                                        // u8 [stages][2][rb][128] (swizzled)
  L.a1 = L.ring + (size_t)um_stages(rb) * rb * kRingRow;             // half: [2 buffers][2 tiles] A1
  // V is written after a slab's last MMA has finished and read until the
  // slab's end, when no chunk of the next slab has been converted yet: it
  // shares its space with A1
  L.vh = L.a1;                                                       // half [C px + c][kVtPitch]
  L.vl = L.vh + vbytes;
  const size_t a1b = (size_t)2 * kA1Bufs * a1_tile_bytes(rb);
  const size_t a1v = a1b > 2 * vbytes ? a1b : 2 * vbytes;
  L.strip = L.a1 + a1v;                                              // half [2][entries][8][8]
  L.cum = L.strip + (size_t)2 * strip_entries(rmax) * 128;           // float [cum_len]
  L.pairs = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;          // uint32 [4][npair]
  L.edge = L.pairs + (size_t)4 * npair(rmax) * 4;                    // float [2][256]
  L.foldw = L.edge + (size_t)2 * 256 * 4;                            // float [2][32]
  L.starts = L.foldw + (size_t)2 * 32 * 4;                           // int [rmax + 1]
  L.total = L.starts + (size_t)(rmax + 1) * 4 + 1024;                // + alignment slack
  return L;
}

// One item. bars: TMA ring stages; mbar_mma / conv_full[kA1Bufs]: MMA
// completion and conversion completion per A1 buffer. gq0: chunks this CTA
// has staged so far, gt0: those of them loaded by TMA (identical in all
// threads). The conversion and MMA barriers complete a phase for every
// chunk; a ring stage's barrier only for chunks loaded by TMA, so its phase
// parity follows gt0 (items of frames that TMA cannot address stage their
// rows with plain loads).
template <int RB, int C, typename LookAhead>
__device__ __forceinline__ bool um_item(const Item& it, float c_tap, unsigned char* ring, __half* A1, __half* Vh,
                                        __half* Vl, __half* Sh, float* CU, unsigned int* P,
                                        float* edge, float* foldw, int np, int nent, unsigned int tmem,
                                        int* s_tile_has, volatile int* s_abort,
                                        unsigned long long* bars, unsigned long long* mbar_mma,
                                        unsigned long long* conv_full, const void* map,
                                        bool map_in_global, int& gq0, int& gt0, unsigned int* err,
                                        LookAhead&& lookahead) {
  constexpr size_t stage_bytes = (size_t)RB * kRingRow;
  constexpr int kStages = um_stages(RB);
  constexpr int kTileBytes = a1_tile_bytes(RB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = it.r;
  const int Q = it.nsl * it.nchunks;
  const int D0 = it.offy - it.ph;      // tap(v, yo) = v + D0 - yo
  const int delta1 = (D0 + 1) & 7;      // (D0 - 31) mod 8

  auto issue = [&](int qq) {  // one thread: the chunk's two TMA boxes
    const Slab cs = slab_of<true>(it, qq / it.nchunks);
    const int gt = gt0 + qq, stg = gt % kStages;
    unsigned char* dst = ring + (size_t)stg * stage_bytes;
    const int x = (int)cs.src - cs.ph;
    const int y = it.gy0 - it.ph + (qq % it.nchunks) * RB;
    mbar_expect_tx(bars + stg, 2u * 128u * RB);
    tma_load_2d(dst, map, x, y, bars + stg);
    tma_load_2d(dst + 128 * RB, map, x + 128, y, bars + stg);
  };
  auto load_plain_conv = [&](int qq, int ct) {  // converter threads: rows that TMA cannot load
    const Slab cs = slab_of<true>(it, qq / it.nchunks);
    unsigned char* dst = ring + (size_t)((gq0 + qq) % kStages) * stage_bytes;
    const long long x0 = (long long)cs.src - cs.ph;
    const int nb = min(256, (cs.ph + cs.sws + 31) & ~31);
    const int y0 = it.gy0 - it.ph + (qq % it.nchunks) * RB;
    for (int idx = ct; idx < RB * nb; idx += kThreads - 32) {
      const int rho = idx / nb, b = idx - rho * nb;
      const int y = y0 + rho;
      const long long xb = x0 + b;
      unsigned char v = 0;
      if (y >= 0 && y < it.H && xb < (long long)it.pitch) v = it.in[(size_t)y * it.pitch + (size_t)xb];
      dst[ring_off<RB>(rho, b)] = v;
    }
  };
  int issued = 0;  // thread 0: chunks of this item whose rows were requested
  if (map && tid == 0) {
    if (map_in_global) fence_tensormap_acquire(map);
    fence_proxy_async();
    for (; issued < kStages && issued < Q; ++issued) issue(issued);
  }
  {
    const float S = warp_tap_sum(r, c_tap);
    make_pairs(P, r, c_tap, S, np);
    make_strips(Sh, nent, r, c_tap, S, delta1);
    if ((it.foldT || it.foldB || it.foldL || it.foldR) && warp == kThreads / 32 - 1) {
      make_cumulative_tc(CU, r, c_tap, S);
      __syncwarp();
      // weights of the folded top / bottom rows for output row yo = lane
      foldw[lane] = cum_at(CU, it.offy - lane, r) * (kWScale * kDScale);
      foldw[32 + lane] = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - lane), r) * (kWScale * kDScale);
    }
  }
  if (tid == 0) lookahead(0);

  float acc2[C][4];
  #pragma unroll
  for (int i = 0; i < C; ++i)
    #pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = 0.f;

  // Within a slab the warps split roles: warps 1..7 convert chunks (wait for
  // the chunk's rows, wait until the MMAs of two chunks back have released
  // the A1 buffer, convert, arrive on conv_full), lane 0 of warp 0 issues
  // (wait conv_full, refill the chunk's ring stage, issue its MMAs, commit to
  // mma_done). Nobody waits for the slowest warp at every chunk; the CTA
  // meets once per slab to read the accumulator back. Every wait is bounded;
  // a timeout sets s_abort and the protocol continues (arrivals, commits) so
  // that no one waits forever, and the item is abandoned at the slab's end.
  const int vb = it.ph + it.EH - 1;
  bool ok = true;
  int q = 0;
  for (int s = 0; s < it.nsl && ok; ++s) {
    const Slab sl = slab_of<true>(it, s);
    const int qs = s * it.nchunks;  // first chunk of the slab
    if (warp == 0) {
      if (lane == 0) {
        int started[2] = {0, 0};
        for (int k = 0; k < it.nchunks; ++k) {
          const int qq = qs + k, gq = gq0 + qq;
          if (!mbar_wait(&conv_full[gq % kA1Bufs], (unsigned int)(gq / kA1Bufs) & 1u)) *s_abort = 1;
          tc05_fence_after();
          if (map && qq + kStages < Q) {  // this chunk's stage is converted: refill it
            issue(qq + kStages);
            issued = qq + kStages + 1;
          }
          const int R0 = k * RB;
          __half* a1b = A1 + (size_t)(gq % kA1Bufs) * kTileBytes;
          for (int ks = 0; ks < RB / 16 && !*s_abort; ++ks) {
            const int k0 = R0 + 16 * ks;
            if (k0 >= it.vrows) break;
            if (k0 + 15 < -D0 || k0 > 31 - D0 + 2 * r) continue;  // no tap of the 32 rows here
            const int j0 = (k0 + D0 - 31 - delta1) / 8 + kXOff;
            const unsigned long long bd = umma_desc(Sh + (size_t)j0 * 128, 256, 128);
            #pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (128 * h >= sl.ph + sl.sws || 128 * h + 128 <= sl.ph) continue;
              const unsigned long long ad = umma_desc(reinterpret_cast<unsigned char*>(a1b) +
                                                          (size_t)h * kTileBytes + ks * 256, 128, a1_sbo(RB));
              umma_f16(tmem + 64 * h, ad, bd, kIdescM128N64, started[h]);
              started[h] = 1;
            }
          }
          umma_commit(&mbar_mma[gq % kA1Bufs]);
        }
        s_tile_has[0] = started[0];
        s_tile_has[1] = started[1];
        if (s == 0) lookahead(1);  // idle until the slab's MMAs finish anyway
      }
      __syncwarp();
    } else {
      const int ct = tid - 32;  // converter thread 0..223
      for (int k = 0; k < it.nchunks; ++k) {
        const int qq = qs + k, gq = gq0 + qq;
        const int R0 = k * RB;
        if (map) {
          const int gt = gt0 + qq;
          if (!mbar_wait(bars + gt % kStages, (unsigned int)(gt / kStages) & 1u)) *s_abort = 1;
        } else {
          asm volatile("bar.sync 1, 224;" ::: "memory");  // converters done with this stage's old rows
          load_plain_conv(qq, ct);
          asm volatile("bar.sync 1, 224;" ::: "memory");
        }
        // the MMAs of chunk gq - kA1Bufs read the A1 buffer this chunk is converted into
        if (gq >= kA1Bufs && !mbar_wait(&mbar_mma[gq % kA1Bufs], (unsigned int)((gq - kA1Bufs) / kA1Bufs) & 1u))
          *s_abort = 1;
        const unsigned char* st = ring + (size_t)(((map ? gt0 : gq0) + qq) % kStages) * stage_bytes;
        __half* a1b = A1 + (size_t)(gq % kA1Bufs) * kTileBytes;
        // ---- convert: 8 columns x 4 rows per work unit, transposed into
        // K-major core matrices; stash the folded edge rows as floats
        for (int idx = ct; idx < 8 * RB; idx += kThreads - 32) {
          const int mi = (idx & 7) + ((idx >> 4) & 1) * 8;  // column group 0..15
          const int half = (idx >> 3) & 1;                    // rows 0-3 or 4-7 of a core matrix
          const int rest = idx >> 5;
          const int ki = rest % (RB / 8), h = rest / (RB / 8);
          const int b = 128 * h + 8 * mi;                     // first ring byte
          if (b >= sl.ph + sl.sws || b + 8 <= sl.ph) continue;  // no slab byte here
          const int v0 = 8 * ki + 4 * half;
          uint2 w[4];
          #pragma unroll
          for (int j = 0; j < 4; ++j) w[j] = *reinterpret_cast<const uint2*>(st + ring_off<RB>(v0 + j, b));
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int vv = R0 + v0 + j;
            if ((k == 0 && vv == it.ph) || vv == vb) {  // both stashes when the tile is one row high
              #pragma unroll
              for (int part = 0; part < 2; ++part) {
                if (part == 0 ? !(k == 0 && vv == it.ph) : vv != vb) continue;
                float* ed = edge + 256 * part + b;
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                  ed[i] = (float)((w[j].x >> (8 * i)) & 0xFFu);
                  ed[4 + i] = (float)((w[j].y >> (8 * i)) & 0xFFu);
                }
              }
            }
          }
          // rows (v0, v0+1) and (v0+2, v0+3) of column i -> two fp16 subnormal pairs
          unsigned int o[8][2];
          {
            const unsigned int p01 = __byte_perm(w[0].x, w[1].x, 0x5140), p23 = __byte_perm(w[0].x, w[1].x, 0x7362);
            const unsigned int q01 = __byte_perm(w[2].x, w[3].x, 0x5140), q23 = __byte_perm(w[2].x, w[3].x, 0x7362);
            const unsigned int p45 = __byte_perm(w[0].y, w[1].y, 0x5140), p67 = __byte_perm(w[0].y, w[1].y, 0x7362);
            const unsigned int q45 = __byte_perm(w[2].y, w[3].y, 0x5140), q67 = __byte_perm(w[2].y, w[3].y, 0x7362);
            o[0][0] = __byte_perm(p01, 0u, 0x4140); o[0][1] = __byte_perm(q01, 0u, 0x4140);
            o[1][0] = __byte_perm(p01, 0u, 0x4342); o[1][1] = __byte_perm(q01, 0u, 0x4342);
            o[2][0] = __byte_perm(p23, 0u, 0x4140); o[2][1] = __byte_perm(q23, 0u, 0x4140);
            o[3][0] = __byte_perm(p23, 0u, 0x4342); o[3][1] = __byte_perm(q23, 0u, 0x4342);
            o[4][0] = __byte_perm(p45, 0u, 0x4140); o[4][1] = __byte_perm(q45, 0u, 0x4140);
            o[5][0] = __byte_perm(p45, 0u, 0x4342); o[5][1] = __byte_perm(q45, 0u, 0x4342);
            o[6][0] = __byte_perm(p67, 0u, 0x4140); o[6][1] = __byte_perm(q67, 0u, 0x4140);
            o[7][0] = __byte_perm(p67, 0u, 0x4342); o[7][1] = __byte_perm(q67, 0u, 0x4342);
          }
          unsigned char* dst = reinterpret_cast<unsigned char*>(a1b) + (size_t)h * kTileBytes + mi * a1_sbo(RB) +
                               ki * 128 + half * 8;
          #pragma unroll
          for (int i = 0; i < 8; ++i) *reinterpret_cast<uint2*>(dst + i * 16) = make_uint2(o[i][0], o[i][1]);
        }
        fence_proxy_async();  // the converted chunk is read by the tensor cores
        mbar_arrive(&conv_full[gq % kA1Bufs]);
      }
    }
    q = qs + it.nchunks - 1;
    // ---- slab complete: read D1 back, add the folded rows, V -> hi/lo fp16
    const int gl = gq0 + q;  // the slab's last chunk
    const bool done =
        __all_sync(0xffffffffu, mbar_wait(&mbar_mma[gl % kA1Bufs], (unsigned int)(gl / kA1Bufs) & 1u));
    if (!done) *s_abort = 1;
    __syncthreads();  // s_tile_has, edge rows, abort flag visible
    tc05_fence_after();
    if (*s_abort) {
      ok = false;
      break;
    }
    const int npx = sl.sws / C;
    const int npx16 = (npx + 15) & ~15;
    {
      const int h = warp >> 2;                 // M tile of this warp
      const int e = 32 * (warp & 3) + lane;    // its tensor-memory lane
      const int b = 128 * h + e;               // ring byte = slab element + ph
      const int ee = b - sl.ph;
      const bool tile_on = s_tile_has[h] != 0;
      float d[32];
      if (tile_on) {  // column 16 a' + 8 p + rho: part p of output row 31 - (8 a' + rho)
        float dd[32];
        tmem_ld32(tmem + ((unsigned int)(32 * (warp & 3)) << 16) + 64 * h, d);
        tmem_ld32(tmem + ((unsigned int)(32 * (warp & 3)) << 16) + 64 * h + 32, dd);
        float t[32];
        #pragma unroll
        for (int a = 0; a < 2; ++a)
          #pragma unroll
          for (int rho = 0; rho < 8; ++rho) {
            t[8 * a + rho] = d[16 * a + rho] + d[16 * a + 8 + rho];
            t[16 + 8 * a + rho] = dd[16 * a + rho] + dd[16 * a + 8 + rho];
          }
        #pragma unroll
        for (int n = 0; n < 32; ++n) d[n] = t[n];
      }
      if (tile_on && ee >= 0 && ee < sl.sws) {
        // V row (px, c), the 32 output rows contiguous: 4 x 16 bytes of hi
        // and of lo fp16 parts
        const float et = it.foldT ? edge[b] : 0.0f, eb = it.foldB ? edge[256 + b] : 0.0f;
        const int px = ee / C, c = ee - px * C;
        uint4* vh = reinterpret_cast<uint4*>(Vh + v_index<C, true>(c, 0, px));
        uint4* vl = reinterpret_cast<uint4*>(Vl + v_index<C, true>(c, 0, px));
        #pragma unroll
        for (int q8 = 0; q8 < 4; ++q8) {
          unsigned int hw[4], lw[4];
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int yo = 8 * q8 + 2 * j;
            float a0v = d[31 - yo], a1v = d[30 - yo];
            if (it.foldT) {
              a0v = fmaf(foldw[yo], et, a0v);
              a1v = fmaf(foldw[yo + 1], et, a1v);
            }
            if (it.foldB) {
              a0v = fmaf(foldw[32 + yo], eb, a0v);
              a1v = fmaf(foldw[33 + yo], eb, a1v);
            }
            const float v0 = a0v * kVScale, v1 = a1v * kVScale;
            const __half2 h2 = __floats2half2_rn(v0, v1);
            const float2 f2 = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(v0 - f2.x, v1 - f2.y);
            hw[j] = *reinterpret_cast<const unsigned int*>(&h2);
            lw[j] = *reinterpret_cast<const unsigned int*>(&l2);
          }
          vh[q8] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          vl[q8] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      // zero the pixels px in [npx, npx16) that pass 2 reads
      for (int idx = tid; idx < (npx16 - npx) * C * 4; idx += kThreads) {
        const int row = npx * C + (idx >> 2), q8 = idx & 3;
        reinterpret_cast<uint4*>(Vh + (size_t)row * kVtPitch)[q8] = make_uint4(0u, 0u, 0u, 0u);
        reinterpret_cast<uint4*>(Vl + (size_t)row * kVtPitch)[q8] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    tc05_fence_before();
    __syncthreads();  // V complete; D1 read everywhere before the next slab's MMAs
    tc_pass2_slab<C, true>(it, sl, Vh, Vl, CU, P, np, acc2);
    __syncthreads();  // V (the A1 space) read everywhere before the next slab's chunks are converted
  }
  if (!ok) {
    // a chunk never arrived or an MMA never finished: flag it, let the row
    // loads still in flight land (bounded) and give up on the item; every
    // arrival and commit was still made, so nobody else is left waiting
    if (tid == 0) {
      atomicOr(err, kFaultWait);
      for (int qq = q + 1; qq < issued; ++qq) {
        const int g2 = gt0 + qq;
        mbar_wait(bars + g2 % kStages, (unsigned int)(g2 / kStages) & 1u);
      }
    }
    __syncthreads();
    return false;
  }
  gq0 += Q;
  if (map) gt0 += Q;
  __syncthreads();  // the ring is no longer read: it becomes the output stage
  tc_write_output<C>(it, ring, acc2, err);
  fence_proxy_async();  // the next item's TMA boxes overwrite the output stage
  return true;
}

template <int RB, int C>
__global__ void __launch_bounds__(kThreads, 2)
umma_forward_kernel(const __grid_constant__ FrameSource src, Workspace ws, int rmax, BucketList bl,
                    const __grid_constant__ CUtensorMap tmap1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const UmLayout L = um_layout(RB, rmax, C);
  unsigned char* ring = smem + L.ring;
  __half* A1 = reinterpret_cast<__half*>(smem + L.a1);
  __half* Vh = reinterpret_cast<__half*>(smem + L.vh);
  __half* Vl = reinterpret_cast<__half*>(smem + L.vl);
  const int nent = strip_entries(rmax);
  __half* Sh = reinterpret_cast<__half*>(smem + L.strip);  // interleaved hi / lo strip
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  unsigned int* P = reinterpret_cast<unsigned int*>(smem + L.pairs);
  float* edge = reinterpret_cast<float*>(smem + L.edge);
  float* foldw = reinterpret_cast<float*>(smem + L.foldw);
  __shared__ __align__(8) unsigned long long s_bar[kMaxUmStages];
  __shared__ __align__(8) unsigned long long s_mma[kA1Bufs];
  __shared__ __align__(8) unsigned long long s_conv[kA1Bufs];
  __shared__ int s_abort;
  __shared__ unsigned int s_tmem;
  __shared__ int s_tile_has[2];
  const int np = npair(rmax);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kMaxUmStages; ++i) mbar_init(&s_bar[i], 1);
    for (int i = 0; i < kA1Bufs; ++i) {
      mbar_init(&s_mma[i], 1);
      mbar_init(&s_conv[i], kThreads - 32);  // every converter thread arrives once per chunk
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 0) {  // tensor memory for D1 (two CTAs per SM take 128 of 512 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"((unsigned int)kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc05_fence_before();
  __syncthreads();
  tc05_fence_after();
  const unsigned int tmem = s_tmem;
  int gq0 = 0, gt0 = 0;
  tc_item_loop<RB, C>(src, tmap1, ws, rmax, bl, reinterpret_cast<int*>(smem + L.starts),
                      [&](const Item& it, float c, const void* map, bool map_global, auto& lookahead) {
                        return um_item<RB, C>(it, c, ring, A1, Vh, Vl, Sh, CU, P, edge, foldw, np, nent, tmem,
                                              s_tile_has, &s_abort, s_bar, s_mma, s_conv, map, map_global, gq0,
                                              gt0, ws.counters + CNT_ERROR, lookahead);
                      });
  tc05_fence_before();
  __syncthreads();  // every MMA was waited for before its accumulator was read
  if (warp == 0) {
    tc05_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((unsigned int)kTmemCols)
                 : "memory");
  }
}

template <int RB, int C>
void* um_kernel_ptr() { return reinterpret_cast<void*>(&umma_forward_kernel<RB, C>); }

template <int C>
void* pick_um_rb(int rb) {
  return rb == 16 ? um_kernel_ptr<16, C>() : um_kernel_ptr<32, C>();
}

void* pick_um(int rb, int C) {
  switch (C) {
    case 1: return pick_um_rb<1>(rb);
    case 2: return pick_um_rb<2>(rb);
    case 3: return pick_um_rb<3>(rb);
    default: return pick_um_rb<4>(rb);
  }
}

int um_rb(const FwdConfig& cfg) { return cfg.rows_per_chunk == 16 ? 16 : 32; }

}  // namespace

size_t umma_forward_smem_bytes(const FwdConfig& cfg, int rmax, int C) {
  return um_layout(um_rb(cfg), rmax, C).total;
}

int umma_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int C) {
  if (rmax > kUmmaMaxRadius) return 0;
  const size_t smem = umma_forward_smem_bytes(cfg, rmax, C);
  void* k = pick_um(um_rb(cfg), C);
  if (set_smem_attrs(reinterpret_cast<const void*>(k), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // CTAs per SM from shared memory and registers. (The occupancy calculator
  // answers 1 for a kernel that allocates tensor memory; each CTA here takes
  // kTmemCols of the SM's 512 columns, so tensor memory is not the limit.)
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
  const int regs = ((fa.numRegs + 7) & ~7) * kThreads;
  const int by_regs = regs > 0 ? 65536 / regs : 0;
  const int by_tmem = 512 / kTmemCols;
  return std::min(std::min(by_smem, by_regs), std::min(by_tmem, 2));
}

cudaError_t launch_umma_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int C,
                                int grid, cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one) {
  const size_t smem = umma_forward_smem_bytes(cfg, rmax, C);
  void* k = pick_um(um_rb(cfg), C);
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (tmap_one) std::memcpy(&map, tmap_one, sizeof(map));
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &b, &map};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(kThreads);
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
