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
// corrections. The staged rows arrive by TMA: one thread issues, per row
// chunk, two 128-byte-wide tensor-map boxes (128-byte swizzle, so the
// fragment loads are free of bank conflicts) that complete on the stage's
// mbarrier. Slabs, item geometry and the work list are shared with the fp32
// kernel (fwd_common.cuh).
#include <cstring>

#include "tc_common.cuh"

namespace fovea {

namespace {

using namespace fwd;
using namespace tcc;

struct TcLayout {
  size_t ring, vh, vl, cum, pairs, starts, total;
};

// Offsets from the 1024-byte aligned start of the dynamic shared memory (the
// 128-byte swizzle pattern repeats every 1024 bytes), for nw warps.
__host__ __device__ inline TcLayout tc_layout(int rb, int rmax, int nw) {
  TcLayout L;
  const size_t vh = (size_t)tc_vhalves(nw);
  L.ring = 0;                                                  // u8 [stages][nw/4][rb][128] (swizzled)
  L.vh = L.ring + (size_t)tc_stages(rb) * rb * (32 * nw);      // half [vh]
  L.vl = L.vh + vh * 2;                                        // half [vh]
  L.cum = L.vl + vh * 2;                                       // float [cum_len]
  L.pairs = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;    // uint32 [4][npair]
  L.starts = L.pairs + (size_t)4 * npair(rmax) * 4;           // int [rmax + 1] bucket starts
  L.total = L.starts + (size_t)(rmax + 1) * 4 + 1024;          // + alignment slack
  return L;
}

// Returns false if a staged chunk never arrived (the item is abandoned and
// an error flag set; the caller stops). lookahead(step) is called by thread
// 0 at two points of the item (step 0 once the tables are built, step 1 once
// the first chunk has arrived) to fetch the next item's record in the
// background.
template <int RB, int C, int NW, typename LookAhead>
__device__ __forceinline__ bool tc_item(const Item& it, float c_tap, unsigned char* ring, __half* Vh, __half* Vl,
                                        float* CU, unsigned int* P, int np,
                                        unsigned long long* bars, const void* map, bool map_in_global,
                                        int& gq0, unsigned int* err, LookAhead&& lookahead) {
  using D = TcDims<NW>;
  constexpr int VP = tc_vp(C, NW);
  constexpr int NT = D::NT;
  constexpr size_t stage_bytes = (size_t)RB * D::ROW;
  constexpr int kStagesTc = tc_stages(RB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r = it.r;
  const int Q = it.nsl * it.nchunks;

  // Raw uint8 chunks (slab s, rows k*RB ..) stream through the ring stages:
  // global chunk number gq0 + q uses stage (gq0 + q) % stages, and its
  // mbarrier completes for the ((gq0 + q) / stages)-th time. gq0 counts the
  // chunks loaded by TMA only: chunks of an item staged with plain loads
  // (a frame whose rows TMA cannot address) complete no barrier phase, so
  // they must not advance it, or a later item of the same launch would wait
  // for the wrong phase parity.
  auto issue = [&](int qq) {  // one thread: the chunk's NW / 4 TMA boxes
    const Slab cs = slab_of<true>(it, qq / it.nchunks);
    const int gq = gq0 + qq, stg = gq % kStagesTc;
    unsigned char* dst = ring + (size_t)stg * stage_bytes;
    const int x = (int)cs.src - cs.ph;  // 16-byte aligned byte column
    const int y = it.gy0 - it.ph + (qq % it.nchunks) * RB;
    mbar_expect_tx(bars + stg, (unsigned int)D::BOXES * 128u * RB);
    #pragma unroll
    for (int bx = 0; bx < D::BOXES; ++bx) tma_load_2d(dst + 128 * RB * bx, map, x + 128 * bx, y, bars + stg);
  };
  auto load_plain = [&](int qq) {  // all threads: rows that TMA cannot load
    const Slab cs = slab_of<true>(it, qq / it.nchunks);
    unsigned char* dst = ring + (size_t)((gq0 + qq) % kStagesTc) * stage_bytes;
    const long long x0 = (long long)cs.src - cs.ph;
    const int nb = min(D::ROW, (cs.ph + cs.sws + 31) & ~31);
    const int y0 = it.gy0 - it.ph + (qq % it.nchunks) * RB;
    for (int idx = threadIdx.x; idx < RB * nb; idx += NT) {
      const int rho = idx / nb, b = idx - rho * nb;
      const int y = y0 + rho;
      const long long xb = x0 + b;
      unsigned char v = 0;
      if (y >= 0 && y < it.H && xb < (long long)it.pitch) v = it.in[(size_t)y * it.pitch + (size_t)xb];
      unsigned char* o = dst + ring_off<RB>(rho, b);
      if (smem_in_bounds(o, 1, err)) *o = v;
    }
  };
  if (map && tid == 0) {
    if (map_in_global) fence_tensormap_acquire(map);
    fence_proxy_async();
    for (int q = 0; q < kStagesTc - 1 && q < Q; ++q) issue(q);
  }
  // Tables of the item (no block barrier: the first chunk's barrier below
  // publishes them).
  {
    const float S = warp_tap_sum(r, c_tap);
    make_pairs<NT>(P, r, c_tap, S, np);
    if ((it.foldT || it.foldB || it.foldL || it.foldR) && warp == NW - 1)
      make_cumulative_tc(CU, r, c_tap, S);
  }
  if (tid == 0) lookahead(0);

  // Pass 1: each lane reads the tap-pair table of its parity (the tap index
  // of every A register of this lane has the parity of g, D0 being even).
  const unsigned int* Ph = P + ((g & 1) ? np : 0);
  const unsigned int* Pl = P + 2 * np + ((g & 1) ? np : 0);
  const int D0 = it.offy - it.ph;  // tap(v, yo) = v + D0 - yo
  // This warp's pass-1 columns are ring bytes 32w .. 32w+31. Lane (g, t)
  // feeds bytes 32w + 4g + j to n-tile j (column g) and accumulates, for
  // n-tile j, the ring bytes 32w + 8t + j (column 2t) and 32w + 8t + 4 + j
  // (column 2t + 1). (Giving two warps one 32-byte unit, one m-tile each,
  // when a slab has at most four units measured slower: the warps' loads and
  // fragment work do not shrink with their MMAs.)
  const int colw = 32 * warp;

  float acc1[2][4][4];
  float acc2[tc_units(C, NW)][4];
  #pragma unroll
  for (int i = 0; i < tc_units(C, NW); ++i)
    #pragma unroll
    for (int k = 0; k < 4; ++k) acc2[i][k] = 0.f;

  // this lane's pass-1 data word: byte colw + 4g of rows 2t, 2t+1 (+8) of a
  // k-step (row mod 8 is 2t or 2t+1, so the swizzled column is fixed)
  const int bcol = colw + 4 * g;
  const int dbox = (bcol >> 7) * RB;
  const int doffA = ((((bcol >> 4) & 7) ^ (2 * t)) << 4) + (bcol & 15);
  const int doffB = ((((bcol >> 4) & 7) ^ (2 * t + 1)) << 4) + (bcol & 15);

  int q = 0;
  bool ok = true;
  for (; q < Q; ++q) {
    if (map) {
      const int gq = gq0 + q;
      bool got = mbar_wait(bars + gq % kStagesTc, (unsigned int)(gq / kStagesTc) & 1u);
      // chunk q visible to every thread; iteration q-1 finished everywhere
      got = __syncthreads_and(got) != 0;
      if (!got) {
        ok = false;
        break;
      }
      if (tid == 0 && q + kStagesTc - 1 < Q) issue(q + kStagesTc - 1);
    } else {
      __syncthreads();  // iteration q-1 finished everywhere
      load_plain(q);
      __syncthreads();
    }
    if (q == 0 && tid == 0) lookahead(1);
    const int s = q / it.nchunks, k = q - s * it.nchunks;
    const Slab sl = slab_of<true>(it, s);
    const int R0 = k * RB;
    const unsigned char* st = ring + (size_t)((gq0 + q) % kStagesTc) * stage_bytes;
    const bool wact = colw < sl.ph + sl.sws && colw + 32 > sl.ph;  // warp holds slab bytes
    if (k == 0) {
      #pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        #pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          #pragma unroll
          for (int i = 0; i < 4; ++i) acc1[mt][nt][i] = 0.f;
      if (it.foldT && wact) {  // folded top row first: fixed summation order
        const uint2 wd = *reinterpret_cast<const uint2*>(st + ring_off<RB>(it.ph, colw + 8 * t));
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
          const unsigned char* sb = st + ((dbox + k0 - R0 + 2 * t) << 7);
          const unsigned int w0 = *reinterpret_cast<const unsigned int*>(sb + doffA);
          const unsigned int w1 = *reinterpret_cast<const unsigned int*>(sb + 128 + doffB);
          const unsigned int w8 = *reinterpret_cast<const unsigned int*>(sb + 8 * 128 + doffA);
          const unsigned int w9 = *reinterpret_cast<const unsigned int*>(sb + 9 * 128 + doffB);
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
        const uint2 wd = *reinterpret_cast<const uint2*>(st + ring_off<RB>(vb - R0, colw + 8 * t));
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
      for (int idx = tid; idx < C * 32 * zc; idx += NT) {
        const int row = idx / zc, px = npx + (idx - row * zc);
        const size_t o = (size_t)row * VP + px;
        if (smem_in_bounds(Vh + o, 2, err) && smem_in_bounds(Vl + o, 2, err)) {
          Vh[o] = __ushort_as_half(0);
          Vl[o] = __ushort_as_half(0);
        }
      }
    }
    __syncthreads();

    tc_pass2_slab<C, false, NW>(it, sl, Vh, Vl, CU, P, np, acc2);
  }
  if (!ok) {
    // a chunk never arrived: flag it, let the chunks still in flight land
    // (bounded) and give up on the item
    if (tid == 0) {
      atomicOr(err, kFaultWait);
      for (int qq = q; qq < Q && qq < q + kStagesTc - 1; ++qq) {
        const int gq = gq0 + qq;
        mbar_wait(bars + gq % kStagesTc, (unsigned int)(gq / kStagesTc) & 1u);
      }
    }
    __syncthreads();
    return false;
  }
  if (map) gq0 += Q;
  __syncthreads();  // the ring is no longer read: it becomes the output stage

  tc_write_output<C, NW>(it, ring, acc2, err);
  fence_proxy_async();  // the next item's TMA boxes overwrite the output stage
  return true;
}

// Resident CTAs the register budget is set for: 4 warps x 4, 8 x 2, 16 x 1.
__host__ __device__ constexpr int tc_min_blocks(int nw) { return nw == 4 ? 4 : (nw == 8 ? 2 : 1); }

template <int RB, int C, int NW>
__global__ void __launch_bounds__(32 * NW, tc_min_blocks(NW))
tc_forward_kernel(const __grid_constant__ FrameSource src, Workspace ws, int rmax, BucketList bl,
                  const __grid_constant__ CUtensorMap tmap1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const TcLayout L = tc_layout(RB, rmax, NW);
  unsigned char* ring = smem + L.ring;
  __half* Vh = reinterpret_cast<__half*>(smem + L.vh);
  __half* Vl = reinterpret_cast<__half*>(smem + L.vl);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  unsigned int* P = reinterpret_cast<unsigned int*>(smem + L.pairs);
  __shared__ __align__(8) unsigned long long s_bar[kMaxTcStages];
  const int np = npair(rmax);
  if (threadIdx.x == 0) {
    for (int i = 0; i < kMaxTcStages; ++i) mbar_init(&s_bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_proxy_async();
  }
  int gq0 = 0;  // chunks this CTA has loaded by TMA so far (identical in every thread)
  tc_item_loop<RB, C, true, NW>(src, tmap1, ws, rmax, bl, reinterpret_cast<int*>(smem + L.starts),
                      [&](const Item& it, float c, const void* map, bool map_global, auto& lookahead) {
                        return tc_item<RB, C, NW>(it, c, ring, Vh, Vl, CU, P, np, s_bar, map, map_global, gq0,
                                                  ws.counters + CNT_ERROR, lookahead);
                      });
}

template <int RB, int C, int NW>
void* tc_kernel_ptr() { return reinterpret_cast<void*>(&tc_forward_kernel<RB, C, NW>); }

template <int C, int NW>
void* pick_tc_rb(int rb) {
  switch (rb) {
    case 16: return tc_kernel_ptr<16, C, NW>();
    case 64: return tc_kernel_ptr<64, C, NW>();
    default: return tc_kernel_ptr<32, C, NW>();
  }
}

template <int NW>
void* pick_tc_c(int rb, int C) {
  switch (C) {
    case 1: return pick_tc_rb<1, NW>(rb);
    case 2: return pick_tc_rb<2, NW>(rb);
    case 3: return pick_tc_rb<3, NW>(rb);
    default: return pick_tc_rb<4, NW>(rb);
  }
}

// Warps of the kernel a configuration runs: threads / 32 (128, 256 or 512
// threads; anything else runs 256).
int tc_warps(const FwdConfig& cfg) { return cfg.threads == 128 ? 4 : (cfg.threads == 512 ? 16 : 8); }

void* pick_tc(const FwdConfig& cfg, int C) {
  switch (tc_warps(cfg)) {
    case 4: return pick_tc_c<4>(cfg.rows_per_chunk, C);
    case 16: return pick_tc_c<16>(cfg.rows_per_chunk, C);
    default: return pick_tc_c<8>(cfg.rows_per_chunk, C);
  }
}

}  // namespace

size_t tc_forward_smem_bytes(const FwdConfig& cfg, int rmax) {
  return tc_layout(cfg.rows_per_chunk, rmax, tc_warps(cfg)).total;
}

int tc_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int C) {
  const size_t smem = tc_forward_smem_bytes(cfg, rmax);
  void* k = pick_tc(cfg, C);
  if (set_smem_attrs(reinterpret_cast<const void*>(k), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 32 * tc_warps(cfg), smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_tc_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int C,
                              int grid, cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one) {
  const size_t smem = tc_forward_smem_bytes(cfg, rmax);
  void* k = pick_tc(cfg, C);
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (tmap_one) std::memcpy(&map, tmap_one, sizeof(map));
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &b, &map};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(32 * tc_warps(cfg));
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
