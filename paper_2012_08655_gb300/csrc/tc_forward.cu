// Tensor-core forward kernel for uint8 HWC frames.
//
// The same block-wise separable blur as forward.cu (paper Section 2,
// Algorithm 1; taps of Eq. 1 truncated at r = ceil(3 sigma)), with both
// passes written as the banded Toeplitz contractions they are:
//   pass 1 (vertical):   V[yo][e] = sum_v Wv[yo][v] T[v][e],  Wv[yo][v] = u(v - yo + D0)
//   pass 2 (horizontal): O[(c,yo)][x] = sum_p V[(c,yo)][p] Wh[p][x],  Wh[p][x] = u(offx + p - x)
// and run on the tensor cores with mma.sync.m16n8k16 (fp16 operands, fp32
// accumulation). uint8 values are exact in fp16. To keep fp32-level accuracy
// the taps (scaled by 2^12, clear of fp16 subnormals) are split into
// hi + lo fp16 parts, and so is the intermediate V:
//   pass 1: Whi T + Wlo T;   pass 2: Vhi Whi + Vhi Wlo + Vlo Whi.
// Toeplitz structure means an operand fragment of Wv or Wh is a pair of
// consecutive taps per register: the fragments come straight from 1D
// tap-pair tables, no 2D weight matrix is built. The taps of the folded edge
// rows / columns (clamp-to-edge, see forward.cu) are added as fp32 rank-one
// corrections. Tile staging, slabs and the work list are shared with the
// fp32 kernel (fwd_common.cuh).
#include <cuda_fp16.h>

#include "fwd_common.cuh"

namespace fovea {

namespace {

using namespace fwd;

constexpr float kWScale = 4096.0f;
constexpr float kWInv = 1.0f / 4096.0f;
constexpr int kThPitch = 264;          // halves per staged fp16 row: 528 B (odd multiple of 16 B)
constexpr int kPairPad = 32;           // tap index -kPairPad is pair entry 0
constexpr int kVHalves = 128 * 72;     // halves of one V array (max over C of 32C rows x VP)

__host__ __device__ inline int npair(int rmax) { return rmax + 56; }

// Raw uint8 chunks staged or in flight: one load in flight while a chunk is
// converted and another multiplied, two for the short 16-row chunks.
__host__ __device__ constexpr int tc_stages(int rb) { return rb >= 32 ? 3 : 4; }

struct TcLayout {
  size_t ring, th, vh, vl, taps, cum, pairs, red, total;
};

// The normalised taps are needed only while the cumulative and tap-pair
// tables are built, before the first V is written: they live in the V arrays.
__host__ __device__ inline TcLayout tc_layout(int rb, int rmax) {
  TcLayout L;
  L.ring = 0;                                                  // u8 [stages][rb][256]
  L.th = L.ring + (size_t)tc_stages(rb) * rb * kRowBytesU8;    // half [2][rb][kThPitch]
  L.vh = L.th + (size_t)2 * rb * kThPitch * 2;                 // half [kVHalves]
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

// Two bytes (low half of x) -> two fp16, exactly: 0x64XX is 1024 + XX.
__device__ __forceinline__ unsigned int u8x2_to_h2(unsigned int x) {
  const unsigned int b = __byte_perm(x, 0x64646464u, 0x5140);
  const __half2 bias = __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400));
  __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&b), bias);
  return *reinterpret_cast<unsigned int*>(&h);
}

__device__ __forceinline__ void stsm_x4(void* p, unsigned int r0, unsigned int r1, unsigned int r2, unsigned int r3) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(p);
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};\n" ::"r"(s), "r"(r0), "r"(r1), "r"(r2),
               "r"(r3) : "memory");
}

__device__ __forceinline__ unsigned int pack_f2h2(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<unsigned int*>(&h);
}

// Per channel count: fp16 columns reserved per channel in a staged row, and
// the pitch (halves) of the pass-2 operand rows (odd multiple of 16 bytes).
template <int C> struct TcGeo;
template <> struct TcGeo<1> { static constexpr int PXP = 256, VP = 264; };
template <> struct TcGeo<2> { static constexpr int PXP = 128, VP = 136; };
template <> struct TcGeo<3> { static constexpr int PXP = 80, VP = 88; };
template <> struct TcGeo<4> { static constexpr int PXP = 64, VP = 72; };

// One staged uint8 row -> fp16, de-interleaving the channels: pixels 8q..8q+7
// of every channel c go to Th[c*PXP + 8q ...]; pixels >= npx become 0.
// PH3 is the slab's byte phase modulo 4 (ring byte of pixel p, channel c is
// ph + C*p + c), so every byte position below is a compile-time constant.
template <int C, int PH3>
__device__ __forceinline__ void convert_group(const unsigned char* rowp, int ph, int q, int npx, __half* throw_) {
  constexpr int NW = 2 * C + 1;
  const int w0 = (ph + 8 * C * q) >> 2;
  const unsigned int* wp = reinterpret_cast<const unsigned int*>(rowp);
  unsigned int wd[NW];
  #pragma unroll
  for (int k = 0; k < NW; ++k) wd[k] = (w0 + k < kRowBytesU8 / 4) ? wp[w0 + k] : 0u;
  #pragma unroll
  for (int c = 0; c < C; ++c) {
    unsigned int h[4];
    #pragma unroll
    for (int i2 = 0; i2 < 4; ++i2) {
      const int b0 = PH3 + C * (2 * i2) + c, b1 = b0 + C;
      const unsigned int x = __byte_perm(wd[b0 >> 2], wd[b1 >> 2], (b0 & 3) | (((b1 & 3) + 4) << 4));
      h[i2] = u8x2_to_h2(x);
    }
    if (8 * q + 8 > npx) {
      #pragma unroll
      for (int i2 = 0; i2 < 4; ++i2) {
        if (8 * q + 2 * i2 >= npx) h[i2] = 0u;
        else if (8 * q + 2 * i2 + 1 >= npx) h[i2] &= 0xFFFFu;
      }
    }
    *reinterpret_cast<uint4*>(throw_ + c * TcGeo<C>::PXP + 8 * q) = make_uint4(h[0], h[1], h[2], h[3]);
  }
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

__device__ __forceinline__ void ldsm_x4_t(unsigned int (&r)[4], const void* p) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
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
__device__ __forceinline__ void tc_item(const Item& it, float c_tap, unsigned char* ring, __half* Th, __half* Vh,
                                        __half* Vl, float2* U, float* CU, unsigned int* P, float* red, int np) {
  constexpr int PXP = TcGeo<C>::PXP, VP = TcGeo<C>::VP;
  constexpr size_t stage_bytes = (size_t)RB * kRowBytesU8;
  constexpr int kStagesTc = tc_stages(RB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r = it.r;
  const int Q = it.nsl * it.nchunks;
  const size_t frame_bytes = (size_t)it.H * it.pitch;

  // Raw uint8 chunks stream through the ring stages (cp.async); chunk q+1 is
  // converted to fp16 while chunk q feeds the tensor cores, so the two fp16
  // buffers alternate and one barrier per chunk suffices.
  #pragma unroll
  for (int q = 0; q < kStagesTc - 1; ++q) {
    if (q < Q) stage_rows<true, RB>(it, slab_of<true>(it, q / it.nchunks), q % it.nchunks,
                                    ring + (size_t)q * stage_bytes, frame_bytes);
    cp_async_commit();
  }
  make_taps(U, tap_len(r), r, c_tap, red);
  make_cumulative(U, CU, r);
  make_pairs(U, P, r, np);

  // uint8 chunk qc -> channel-planar fp16 rows in Th buffer qc % 2
  auto convert_chunk = [&](int qc) {
    const Slab cs = slab_of<true>(it, qc / it.nchunks);
    const int cnpx = cs.sws / C;
    const int cngrp = ((cnpx + 15) & ~15) >> 3;  // 8-pixel groups per channel
    const unsigned char* st = ring + (size_t)(qc % kStagesTc) * stage_bytes;
    __half* dst = Th + (size_t)(qc & 1) * RB * kThPitch;
    const int ph3 = cs.ph & 3;
    for (int idx = threadIdx.x; idx < RB * cngrp; idx += kThreads) {
      const int row = idx / cngrp, gq = idx - row * cngrp;
      const unsigned char* rowp = st + (size_t)row * kRowBytesU8;
      __half* throw_ = dst + (size_t)row * kThPitch;
      switch (ph3) {
        case 0: convert_group<C, 0>(rowp, cs.ph, gq, cnpx, throw_); break;
        case 1: convert_group<C, 1>(rowp, cs.ph, gq, cnpx, throw_); break;
        case 2: convert_group<C, 2>(rowp, cs.ph, gq, cnpx, throw_); break;
        default: convert_group<C, 3>(rowp, cs.ph, gq, cnpx, throw_); break;
      }
    }
  };
  cp_async_wait<kStagesTc - 2>();
  __syncthreads();  // chunk 0 landed for every thread; tables ready, taps dead
  convert_chunk(0);

  // Pass 1: each lane reads the tap-pair table of its parity (the tap index
  // of every A register of this lane has the parity of g, D0 being even).
  const unsigned int* Ph = P + ((g & 1) ? np : 0);
  const unsigned int* Pl = P + 2 * np + ((g & 1) ? np : 0);
  const int D0 = it.offy - it.ph;  // tap(v, yo) = v + D0 - yo

  float acc1[2][4][4];
  float acc2[C][4];
  #pragma unroll
  for (int i = 0; i < C; ++i)
    #pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = 0.f;

  for (int q = 0; q < Q; ++q) {
    cp_async_wait<kStagesTc - 3>();
    __syncthreads();  // chunk q converted and q+1 landed; iteration q-1 finished everywhere
    {
      const int qn = q + kStagesTc - 1;
      if (qn < Q) stage_rows<true, RB>(it, slab_of<true>(it, qn / it.nchunks), qn % it.nchunks,
                                       ring + (size_t)(qn % kStagesTc) * stage_bytes, frame_bytes);
      cp_async_commit();
    }
    if (q + 1 < Q) convert_chunk(q + 1);
    const int s = q / it.nchunks, k = q - s * it.nchunks;
    const Slab sl = slab_of<true>(it, s);
    const int R0 = k * RB;
    const int npx = sl.sws / C;                 // pixels of the slab
    const int npx16 = (npx + 15) & ~15;
    const __half* thc = Th + (size_t)(q & 1) * RB * kThPitch;
    // This warp's 32 columns: channel c0 = 32w / PXP, pixel offset inside it.
    const int colw = 32 * warp;
    if (k == 0) {
      #pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          #pragma unroll
          for (int i = 0; i < 4; ++i) acc1[mt][nt][i] = 0.f;
      if (it.foldT && colw < C * PXP) {  // folded top row first: fixed summation order
        const __half* row = thc + (size_t)it.ph * kThPitch;
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float2 df = __half22float2(*reinterpret_cast<const __half2*>(row + colw + 8 * nt + 2 * t));
          #pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const float c0 = cum_at(CU, it.offy - (16 * mt + g), r) * kWScale;
            const float c1 = cum_at(CU, it.offy - (16 * mt + g + 8), r) * kWScale;
            acc1[mt][nt][0] = fmaf(c0, df.x, acc1[mt][nt][0]);
            acc1[mt][nt][1] = fmaf(c0, df.y, acc1[mt][nt][1]);
            acc1[mt][nt][2] = fmaf(c1, df.x, acc1[mt][nt][2]);
            acc1[mt][nt][3] = fmaf(c1, df.y, acc1[mt][nt][3]);
          }
        }
      }
    }
    // n-tile pairs of this warp that hold slab pixels
    bool pon[2];
    #pragma unroll
    for (int np2 = 0; np2 < 2; ++np2) {
      const int j0 = colw + 16 * np2;
      pon[np2] = j0 < C * PXP && (j0 % PXP) < npx16;
    }
    // ---- pass 1 on the chunk: 16 virtual rows per k-step
    if (pon[0] || pon[1]) {
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
        const __half* tb = thc + (size_t)(k0 - R0) * kThPitch + colw;
        unsigned int b[2][4];
        #pragma unroll
        for (int np2 = 0; np2 < 2; ++np2) {
          if (!pon[np2]) continue;
          const int rrow = (lane & 7) + ((lane >> 3) & 1) * 8;
          const int rcol = 16 * np2 + ((lane >> 4) & 1) * 8;
          ldsm_x4_t(b[np2], tb + (size_t)rrow * kThPitch + rcol);
        }
        // all hi products, then all lo products: the two products into one
        // accumulator are 8 independent MMAs apart
        #pragma unroll
        for (int part = 0; part < 2; ++part) {
          #pragma unroll
          for (int np2 = 0; np2 < 2; ++np2) {
            if (!pon[np2]) continue;
            #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int nt = 2 * np2 + h;
              const unsigned int b0 = b[np2][2 * h], b1 = b[np2][2 * h + 1];
              if (on0) mma16816(acc1[0][nt], part ? al[0] : ah[0], b0, b1);
              if (on1) mma16816(acc1[1][nt], part ? al[1] : ah[1], b0, b1);
            }
          }
        }
      }
    }
    if (k != it.nchunks - 1) continue;

    // ---- slab complete: folded bottom row, then V -> hi/lo fp16 for pass 2
    {
      const int vb = it.ph + it.EH - 1;
      if (it.foldB && vb >= R0 && vb < R0 + RB && colw < C * PXP) {
        const __half* row = thc + (size_t)(vb - R0) * kThPitch;
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float2 df = __half22float2(*reinterpret_cast<const __half2*>(row + colw + 8 * nt + 2 * t));
          #pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const float c0 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g)), r) * kWScale;
            const float c1 = cum_at(CU, 2 * r + 1 - (it.offy + it.EH - (16 * mt + g + 8)), r) * kWScale;
            acc1[mt][nt][0] = fmaf(c0, df.x, acc1[mt][nt][0]);
            acc1[mt][nt][1] = fmaf(c0, df.y, acc1[mt][nt][1]);
            acc1[mt][nt][2] = fmaf(c1, df.x, acc1[mt][nt][2]);
            acc1[mt][nt][3] = fmaf(c1, df.y, acc1[mt][nt][3]);
          }
        }
      }
      // V[(c, yo)][px] = acc / 2^12 as hi + lo fp16, written with stmatrix:
      // the accumulator fragment layout is the 8x8-tile register layout.
      #pragma unroll
      for (int np2 = 0; np2 < 2; ++np2) {
        if (!pon[np2]) continue;
        const int j0 = colw + 16 * np2;
        const int c = j0 / PXP, px0 = j0 - c * PXP;
        #pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          unsigned int hr[4], lr[4];
          #pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const int nt = 2 * np2 + (q4 >> 1), ii = (q4 & 1) * 2;
            const float v0 = acc1[mt][nt][ii] * kWInv, v1 = acc1[mt][nt][ii + 1] * kWInv;
            hr[q4] = pack_f2h2(v0, v1);
            const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hr[q4]));
            lr[q4] = pack_f2h2(v0 - hf.x, v1 - hf.y);
          }
          const int vrow = c * 32 + 16 * mt + (lane & 7) + ((lane >> 3) & 1) * 8;
          const int vcol = px0 + ((lane >> 4) & 1) * 8;
          stsm_x4(Vh + (size_t)vrow * VP + vcol, hr[0], hr[1], hr[2], hr[3]);
          stsm_x4(Vl + (size_t)vrow * VP + vcol, lr[0], lr[1], lr[2], lr[3]);
        }
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
  __syncthreads();  // ring and Th no longer read; Th becomes the output stage

  unsigned char* ost = reinterpret_cast<unsigned char*>(Th);
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
  for (int idx = tid; idx < it.bh * rowBytes; idx += kThreads) {
    const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
    out[(size_t)yo * it.pitch + rem] = ost[yo * opitch + rem];
  }
}

template <int RB, int C>
__global__ void __launch_bounds__(kThreads, 2)
tc_forward_kernel(FrameSource src, Workspace ws, int rmax, BucketList bl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TcLayout L = tc_layout(RB, rmax);
  unsigned char* ring = smem + L.ring;
  __half* Th = reinterpret_cast<__half*>(smem + L.th);
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

  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (tid == 0) {
      const int tk = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
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
    tc_item<RB, C>(s_it, s_c, ring, Th, Vh, Vl, U, CU, P, red, np);
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
