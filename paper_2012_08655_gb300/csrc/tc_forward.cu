// Tensor-core forward kernel for uint8 HWC frames.
//
// The same block-wise separable blur as forward.cu (paper Section 2,
// Algorithm 1; taps of Eq. 1 truncated at r = ceil(3 sigma)), with both
// passes written as the banded Toeplitz contractions they are:
//   pass 1 (vertical):   V[yo][e] = sum_v Wv[yo][v] T[v][e],  Wv[yo][v] = u(v - yo + D0)
//   pass 2 (horizontal): O[(c,yo)][x] = sum_p V[(c,yo)][p] Wh[p][x],  Wh[p][x] = u(offx + p - x)
// and run on the tensor cores with mma.sync.m16n8k16 (fp16 operands, fp32
// accumulation). To keep fp32-level accuracy the taps (scaled by 2^12, clear
// of fp16 subnormals) are split into hi + lo fp16 parts, and so is the
// intermediate V:
//   pass 1: Whi T + Wlo T;   pass 2: Vhi Whi + Vhi Wlo + Vlo Whi.
// Toeplitz structure means an operand fragment of Wv or Wh is a pair of
// consecutive taps per register: the fragments come straight from 1D
// tap-pair tables, no 2D weight matrix is built. Pass 1 reads its data
// operand straight from the staged uint8 rows: a byte b placed in the low
// bits of an fp16 is the subnormal b * 2^-24, exactly, so two byte permutes
// turn two staged rows into the fragment registers of four n-tiles and no
// converted copy of the tile is ever written. The taps of the folded edge
// rows / columns (clamp-to-edge, see forward.cu) are added as fp32 rank-one
// corrections. Slabs, row staging and the work list are shared with the fp32
// kernel (fwd_common.cuh).
#include <cuda_fp16.h>

#include "fwd_common.cuh"

namespace fovea {

namespace {

using namespace fwd;

constexpr float kWScale = 4096.0f;          // taps scaled by 2^12
constexpr float kWInv = 1.0f / 4096.0f;
constexpr float kDScale = 1.0f / 16777216.0f;  // a staged byte b enters pass 1 as b * 2^-24
constexpr float kVScale = 4096.0f;          // V = pass-1 accumulator * 2^12 (= 2^24 / 2^12)
constexpr int kRingPitch = 272;             // bytes per staged row: 68 words, rows 2 apart 8 banks apart
constexpr int kPairPad = 32;                // tap index -kPairPad is pair entry 0
constexpr int kVHalves = 128 * 72;     // halves of one V array (max over C of 32C rows x VP)

__host__ __device__ inline int npair(int rmax) { return rmax + 56; }

// Raw uint8 chunks staged or in flight: one load in flight while a chunk is
// converted and another multiplied, two for the short 16-row chunks.
__host__ __device__ constexpr int tc_stages(int rb) { return rb >= 32 ? 3 : 4; }

struct TcLayout {
  size_t ring, vh, vl, taps, cum, pairs, red, total;
};

// The normalised taps are needed only while the cumulative and tap-pair
// tables are built, before the first V is written: they live in the V arrays.
__host__ __device__ inline TcLayout tc_layout(int rb, int rmax) {
  TcLayout L;
  L.ring = 0;                                                  // u8 [stages][rb][kRingPitch]
  L.vh = L.ring + (size_t)tc_stages(rb) * rb * kRingPitch;     // half [kVHalves]
  L.vl = L.vh + (size_t)kVHalves * 2;                          // half [kVHalves]
  size_t end = L.vl + (size_t)kVHalves * 2;
  if ((size_t)tap_len(rmax) * sizeof(float2) <= (size_t)2 * kVHalves * 2) {
    L.taps = L.vh;                                             // float2 [tap_len], aliases V
  } else {
    L.taps = end;
    end += (size_t)tap_len(rmax) * sizeof(float2);
  }
  L.cum = end;                                                 // float [cum_len]
  L.pairs = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;    // uint32 [4][npair]
  L.red = L.pairs + (size_t)4 * npair(rmax) * 4;               // float [32]
  L.total = L.red + 32 * sizeof(float);
  return L;
}

__device__ __forceinline__ unsigned int pack_half2(__half a, __half b) {
  return (unsigned int)__half_as_ushort(a) | ((unsigned int)__half_as_ushort(b) << 16);
}

// Per channel count: pitch (halves) of the pass-2 operand rows V[(c, yo)][p]
// (an odd multiple of 16 bytes, at least the slab's pixels rounded up to 16).
template <int C> struct TcGeo;
template <> struct TcGeo<1> { static constexpr int VP = 264; };
template <> struct TcGeo<2> { static constexpr int VP = 136; };
template <> struct TcGeo<3> { static constexpr int VP = 88; };
template <> struct TcGeo<4> { static constexpr int VP = 72; };

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

// Tap-pair tables: entry j of the even table holds (w(m), w(m+1)) with
// m = 2j - kPairPad, the odd table the pair starting one tap later; hi and lo
// parts of the scaled taps. w is zero outside [0, 2r].
__device__ __forceinline__ void make_pairs(const float2* U, unsigned int* P, int r, int np) {
  unsigned int* PEh = P;
  unsigned int* POh = P + np;
  unsigned int* PEl = P + 2 * np;
  unsigned int* POl = P + 3 * np;
  for (int j = threadIdx.x; j < np; j += kThreads) {
    __half h[3], l[3];
    #pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int m = 2 * j - kPairPad + q;
      const float w = (m >= 0 && m <= 2 * r) ? U[kTapPad + m].x * kWScale : 0.0f;
      h[q] = __float2half_rn(w);
      l[q] = __float2half_rn(w - __half2float(h[q]));
    }
    PEh[j] = pack_half2(h[0], h[1]);
    POh[j] = pack_half2(h[1], h[2]);
    PEl[j] = pack_half2(l[0], l[1]);
    POl[j] = pack_half2(l[1], l[2]);
  }
}


// Everything the tensor-core kernel does for one item with C channels.
template <int RB, int C>
__device__ __forceinline__ void tc_item(const Item& it, float c_tap, unsigned char* ring, __half* Vh, __half* Vl,
                                        float2* U, float* CU, unsigned int* P, float* red, int np) {
  constexpr int VP = TcGeo<C>::VP;
  constexpr size_t stage_bytes = (size_t)RB * kRingPitch;
  constexpr int kStagesTc = tc_stages(RB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r = it.r;
  const int Q = it.nsl * it.nchunks;
  const size_t frame_bytes = (size_t)it.H * it.pitch;

  // Raw uint8 chunks (slab s, rows k*RB ..) stream through the ring stages.
  #pragma unroll
  for (int q = 0; q < kStagesTc - 1; ++q) {
    if (q < Q) stage_rows<true, RB, kRingPitch>(it, slab_of<true>(it, q / it.nchunks), q % it.nchunks,
                                                ring + (size_t)q * stage_bytes, frame_bytes);
    cp_async_commit();
  }
  make_taps(U, tap_len(r), r, c_tap, red);
  make_cumulative(U, CU, r);
  make_pairs(U, P, r, np);

  // Pass 1: each lane reads the tap-pair table of its parity (the tap index
  // of every A register of this lane has the parity of g, D0 being even).
  const unsigned int* Ph = P + ((g & 1) ? np : 0);
  const unsigned int* Pl = P + 2 * np + ((g & 1) ? np : 0);
  const int D0 = it.offy - it.ph;  // tap(v, yo) = v + D0 - yo
  // This warp's pass-1 columns are ring bytes 32w .. 32w+31. Lane (g, t)
  // feeds bytes 32w + 4g + j to n-tile j (column g) and accumulates, for
  // n-tile j, the ring bytes 32w + 8t + j (column 2t) and 32w + 8t + 4 + j
  // (column 2t + 1).
  const int colw = 32 * warp;

  float acc1[2][4][4];
  float acc2[C][4];
  #pragma unroll
  for (int i = 0; i < C; ++i)
    #pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = 0.f;

  for (int q = 0; q < Q; ++q) {
    cp_async_wait<kStagesTc - 2>();
    __syncthreads();  // chunk q landed for every thread; iteration q-1 finished everywhere
    {
      const int qn = q + kStagesTc - 1;
      if (qn < Q) stage_rows<true, RB, kRingPitch>(it, slab_of<true>(it, qn / it.nchunks), qn % it.nchunks,
                                                   ring + (size_t)(qn % kStagesTc) * stage_bytes, frame_bytes);
      cp_async_commit();
    }
    const int s = q / it.nchunks, k = q - s * it.nchunks;
    const Slab sl = slab_of<true>(it, s);
    const int R0 = k * RB;
    const unsigned char* st = ring + (size_t)(q % kStagesTc) * stage_bytes;
    const bool wact = colw < sl.ph + sl.sws && colw + 32 > sl.ph;  // warp holds slab bytes
    if (k == 0) {
      #pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          #pragma unroll
          for (int i = 0; i < 4; ++i) acc1[mt][nt][i] = 0.f;
      if (it.foldT && wact) {  // folded top row first: fixed summation order
        const uint2 wd = *reinterpret_cast<const uint2*>(st + (size_t)it.ph * kRingPitch + colw + 8 * t);
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const float c0 = cum_at(CU, it.offy - (16 * mt + g), r) * (kWScale * kDScale);
          const float c1 = cum_at(CU, it.offy - (16 * mt + g + 8), r) * (kWScale * kDScale);
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float d0 = (float)((wd.x >> (8 * j)) & 0xFFu), d1 = (float)((wd.y >> (8 * j)) & 0xFFu);
            acc1[mt][j][0] = fmaf(c0, d0, acc1[mt][j][0]);
            acc1[mt][j][1] = fmaf(c0, d1, acc1[mt][j][1]);
            acc1[mt][j][2] = fmaf(c1, d0, acc1[mt][j][2]);
            acc1[mt][j][3] = fmaf(c1, d1, acc1[mt][j][3]);
          }
        }
      }
    }
    // ---- pass 1 on the chunk: 16 virtual rows per k-step
    if (wact) {
      for (int ks = 0; ks < RB / 16; ++ks) {
        const int k0 = R0 + 16 * ks;
        if (k0 >= it.vrows) break;
        const bool on0 = k0 + 15 >= -D0 && k0 <= 15 - D0 + 2 * r;
        const bool on1 = k0 + 15 >= 16 - D0 && k0 <= 31 - D0 + 2 * r;
        if (!on0 && !on1) continue;
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
        // (byte of row v, byte of row v+1) -> two fp16 subnormals.
        unsigned int b[4][2];
        {
          const unsigned char* sb = st + (size_t)(k0 - R0 + 2 * t) * kRingPitch + colw + 4 * g;
          const unsigned int w0 = *reinterpret_cast<const unsigned int*>(sb);
          const unsigned int w1 = *reinterpret_cast<const unsigned int*>(sb + kRingPitch);
          const unsigned int w8 = *reinterpret_cast<const unsigned int*>(sb + 8 * kRingPitch);
          const unsigned int w9 = *reinterpret_cast<const unsigned int*>(sb + 9 * kRingPitch);
          const unsigned int lo01 = __byte_perm(w0, w1, 0x5140), lo23 = __byte_perm(w0, w1, 0x7362);
          const unsigned int hi01 = __byte_perm(w8, w9, 0x5140), hi23 = __byte_perm(w8, w9, 0x7362);
          b[0][0] = __byte_perm(lo01, 0u, 0x4140); b[1][0] = __byte_perm(lo01, 0u, 0x4342);
          b[2][0] = __byte_perm(lo23, 0u, 0x4140); b[3][0] = __byte_perm(lo23, 0u, 0x4342);
          b[0][1] = __byte_perm(hi01, 0u, 0x4140); b[1][1] = __byte_perm(hi01, 0u, 0x4342);
          b[2][1] = __byte_perm(hi23, 0u, 0x4140); b[3][1] = __byte_perm(hi23, 0u, 0x4342);
        }
        // all hi products, then all lo products: the two products into one
        // accumulator are 8 independent MMAs apart
        #pragma unroll
        for (int part = 0; part < 2; ++part) {
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (on0) mma16816(acc1[0][j], part ? al[0] : ah[0], b[j][0], b[j][1]);
            if (on1) mma16816(acc1[1][j], part ? al[1] : ah[1], b[j][0], b[j][1]);
          }
        }
      }
    }
    if (k != it.nchunks - 1) continue;

    // ---- slab complete: folded bottom row, then V -> hi/lo fp16 for pass 2
    const int npx = sl.sws / C;                 // pixels of the slab
    const int npx16 = (npx + 15) & ~15;
    {
      const int vb = it.ph + it.EH - 1;
      if (it.foldB && vb >= R0 && vb < R0 + RB && wact) {
        const uint2 wd = *reinterpret_cast<const uint2*>(st + (size_t)(vb - R0) * kRingPitch + colw + 8 * t);
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const float c0 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g)), r) * (kWScale * kDScale);
          const float c1 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g + 8)), r) * (kWScale * kDScale);
          #pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float d0 = (float)((wd.x >> (8 * j)) & 0xFFu), d1 = (float)((wd.y >> (8 * j)) & 0xFFu);
            acc1[mt][j][0] = fmaf(c0, d0, acc1[mt][j][0]);
            acc1[mt][j][1] = fmaf(c0, d1, acc1[mt][j][1]);
            acc1[mt][j][2] = fmaf(c1, d0, acc1[mt][j][2]);
            acc1[mt][j][3] = fmaf(c1, d1, acc1[mt][j][3]);
          }
        }
      }
      // V[(c, yo)][px] = acc * 2^12 as hi + lo fp16, de-interleaving the
      // channels: ring byte 32w + 8t + e8 is slab element e = byte - ph.
      if (wact) {
        #pragma unroll
        for (int e8 = 0; e8 < 8; ++e8) {
          const int e = colw + 8 * t + e8 - sl.ph;
          if (e < 0 || e >= sl.sws) continue;
          const int px = e / C, c = e - px * C;
          #pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            #pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const float v = acc1[mt][e8 & 3][2 * hh + (e8 >> 2)] * kVScale;
              const __half h = __float2half_rn(v);
              const __half l = __float2half_rn(v - __half2float(h));
              const size_t o = (size_t)(c * 32 + 16 * mt + g + 8 * hh) * VP + px;
              Vh[o] = h;
              Vl[o] = l;
            }
          }
        }
      }
      // zero the columns px in [npx, npx16) that pass 2 reads
      const int zc = npx16 - npx;
      for (int idx = tid; idx < C * 32 * zc; idx += kThreads) {
        const int row = idx / zc, px = npx + (idx - row * zc);
        Vh[(size_t)row * VP + px] = __ushort_as_half(0);
        Vl[(size_t)row * VP + px] = __ushort_as_half(0);
      }
    }
    __syncthreads();

    // ---- pass 2 over the slab's pixels: units (row tile, column tile)
    const int P0 = sl.e0 / C;  // first folded pixel of the slab
    // tap index of this lane's B registers has the parity of offx + P0 - g
    const int par2 = (it.offx + P0 + g) & 1;
    const unsigned int* Qh = P + (par2 ? np : 0);
    const unsigned int* Ql = P + 2 * np + (par2 ? np : 0);
    if (it.foldL && P0 == 0) {  // folded left column first: fixed summation order
      #pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = warp + 8 * i;
        const int mt2 = u >> 2, nt2 = u & 3;
        #pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = 16 * mt2 + g + 8 * h;
          const float v = __half2float(Vh[(size_t)row * VP]) + __half2float(Vl[(size_t)row * VP]);
          #pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int x = 8 * nt2 + 2 * t + cc;
            acc2[i][2 * h + cc] = fmaf(cum_at(CU, it.offx - x, r) * kWScale, v, acc2[i][2 * h + cc]);
          }
        }
      }
    }
    for (int kk = 0; kk < npx16; kk += 16) {
      unsigned int a_h[C][4], a_l[C][4], bh[C][2], bl[C][2];
      #pragma unroll
      for (int i = 0; i < C; ++i) {
        const int u = warp + 8 * i;
        const int mt2 = u >> 2, nt2 = u & 3;
        const int arow = 16 * mt2 + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int acol = kk + ((lane >> 4) & 1) * 8;
        ldsm_x4(a_h[i], Vh + (size_t)arow * VP + acol);
        ldsm_x4(a_l[i], Vl + (size_t)arow * VP + acol);
        const int jb = (it.offx + P0 + kk + 2 * t - 8 * nt2 - g + kPairPad) >> 1;
        bh[i][0] = Qh[jb]; bh[i][1] = Qh[jb + 4];
        bl[i][0] = Ql[jb]; bl[i][1] = Ql[jb + 4];
      }
      #pragma unroll
      for (int i = 0; i < C; ++i) mma16816(acc2[i], a_h[i], bh[i][0], bh[i][1]);
      #pragma unroll
      for (int i = 0; i < C; ++i) mma16816(acc2[i], a_h[i], bl[i][0], bl[i][1]);
      #pragma unroll
      for (int i = 0; i < C; ++i) mma16816(acc2[i], a_l[i], bh[i][0], bh[i][1]);
    }
    {
      const int pr = it.EW - 1 - P0;  // folded right column after the last slab's products
      if (it.foldR && pr >= 0 && pr < npx) {
        #pragma unroll
        for (int i = 0; i < C; ++i) {
          const int u = warp + 8 * i;
          const int mt2 = u >> 2, nt2 = u & 3;
          #pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 16 * mt2 + g + 8 * h;
            const float v = __half2float(Vh[(size_t)row * VP + pr]) + __half2float(Vl[(size_t)row * VP + pr]);
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
  cp_async_wait<0>();
  __syncthreads();  // the ring is no longer read: it becomes the output stage

  unsigned char* ost = ring;
  constexpr int opitch = 32 * C;
  #pragma unroll
  for (int i = 0; i < C; ++i) {
    const int u = warp + 8 * i;
    const int mt2 = u >> 2, nt2 = u & 3;
    #pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = 16 * mt2 + g + ((e >> 1) << 3);
      const int c = row >> 5, yo = row & 31;
      const int x = 8 * nt2 + 2 * t + (e & 1);
      ost[yo * opitch + x * C + c] = quant_u8(acc2[i][e] * kWInv);
    }
  }
  __syncthreads();
  const int rowBytes = it.bw * C;
  unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * C;
  if (((((size_t)out) | it.pitch | (size_t)rowBytes) & 15) == 0) {
    const int nv = rowBytes >> 4;  // 16-byte pieces per row
    for (int idx = tid; idx < it.bh * nv; idx += kThreads) {
      const int yo = idx / nv, v = idx - yo * nv;
      *reinterpret_cast<uint4*>(out + (size_t)yo * it.pitch + 16 * v) =
          *reinterpret_cast<const uint4*>(ost + yo * opitch + 16 * v);
    }
  } else {
    for (int idx = tid; idx < it.bh * rowBytes; idx += kThreads) {
      const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
      out[(size_t)yo * it.pitch + rem] = ost[yo * opitch + rem];
    }
  }
}

template <int RB, int C>
__global__ void __launch_bounds__(kThreads, 2)
tc_forward_kernel(FrameSource src, Workspace ws, int rmax, BucketList bl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TcLayout L = tc_layout(RB, rmax);
  unsigned char* ring = smem + L.ring;
  __half* Vh = reinterpret_cast<__half*>(smem + L.vh);
  __half* Vl = reinterpret_cast<__half*>(smem + L.vl);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  unsigned int* P = reinterpret_cast<unsigned int*>(smem + L.pairs);
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_state;
  __shared__ Item s_it;
  __shared__ float s_c;
  __shared__ int s_start[kBuckets];
  __shared__ int s_wsum[kThreads / 32];

  const int tid = threadIdx.x;
  const int np = npair(rmax);

  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool own_order = bl.list != nullptr;
  const int n_items = own_order ? (int)src.one_total : (int)ws.counters[CNT_NITEMS];
  if (own_order) bucket_starts(ws.counters + CNT_HIST, bl.nb, s_start, s_wsum);

  // Thread 0 holds the ticket of the item after the current one, so the
  // ticket counter's round trip overlaps the current item.
  int next_tk = 0;
  if (tid == 0) next_tk = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (tid == 0) {
      const int tk = next_tk;
      if (tk < n_items) next_tk = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
      int state = 0;
      if (tk >= n_items) {
        state = 2;
      } else {
        int item;
        if (own_order) {
          int lo = 0, hi = bl.nb - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_start[mid] <= tk) hi = mid; else lo = mid + 1;
          }
          item = bl.list[(size_t)lo * bl.cap + (tk - s_start[lo])];
        } else {
          item = ws.order[tk];
        }
        if ((unsigned)item >= (unsigned)n_items) {
          atomicOr(&ws.counters[CNT_ERROR], 16u);
          state = 1;
        } else {
          const ItemInfo inf = ws.items[item];
          const FrameDesc fd = load_frame(src, inf.frame);
          if (inf.r > rmax || fd.fmt != FOVEA_U8_HWC || fd.C != C) {
            atomicOr(&ws.counters[CNT_ERROR], 2u);
            state = 1;
          } else {
            item_geometry(s_it, inf, fd, RB);
            s_c = inf.neg_half_inv_s2;
          }
        }
      }
      s_state = state;
    }
    __syncthreads();
    if (s_state == 2) break;
    if (s_state == 1) continue;
    tc_item<RB, C>(s_it, s_c, ring, Vh, Vl, U, CU, P, red, np);
  }
  cp_async_wait<0>();
  if (own_order) {
    __threadfence();
    __syncthreads();
    if (tid == 0) s_state = atomicAdd(&ws.counters[CNT_DONE_SIGMA], 1u) == gridDim.x - 1 ? 3 : 0;
    __syncthreads();
    if (s_state == 3) {
      for (int j = tid; j < kBuckets; j += kThreads) ws.counters[CNT_HIST + j] = 0u;
      if (tid == 0) {
        ws.counters[CNT_TICKET] = 0u;
        ws.counters[CNT_DONE_SIGMA] = 0u;
      }
    }
  }
}

template <int RB, int C>
void* tc_kernel_ptr() { return reinterpret_cast<void*>(&tc_forward_kernel<RB, C>); }

template <int C>
void* pick_tc_rb(int rb) {
  switch (rb) {
    case 16: return tc_kernel_ptr<16, C>();
    case 64: return tc_kernel_ptr<64, C>();
    default: return tc_kernel_ptr<32, C>();
  }
}

void* pick_tc(int rb, int C) {
  switch (C) {
    case 1: return pick_tc_rb<1>(rb);
    case 2: return pick_tc_rb<2>(rb);
    case 3: return pick_tc_rb<3>(rb);
    default: return pick_tc_rb<4>(rb);
  }
}

}  // namespace

size_t tc_forward_smem_bytes(const FwdConfig& cfg, int rmax) { return tc_layout(cfg.rows_per_chunk, rmax).total; }

int tc_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int C) {
  const size_t smem = tc_forward_smem_bytes(cfg, rmax);
  void* k = pick_tc(cfg.rows_per_chunk, C);
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

cudaError_t launch_tc_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int C,
                              int grid, cudaStream_t s, const BucketList& bl, bool pdl) {
  const size_t smem = tc_forward_smem_bytes(cfg, rmax);
  void* k = pick_tc(cfg.rows_per_chunk, C);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &b};
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
