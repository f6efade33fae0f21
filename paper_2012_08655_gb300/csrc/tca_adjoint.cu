// Adjoint (transpose) of the foveation map for float32 CHW frames on the
// tensor cores (tensor_cores = 2; every other setting runs the fp32 kernel
// in adjoint.cu, which measured faster: 0.170 against 0.186 ms for the
// 32 x 3 x 224 x 224 training batch. Both issue the same ~29 M reductions
// into grad_in and neither is bound by its arithmetic.)
//
// The forward map of block b (Section 2, Algorithm 1, taps of Eq. 1) is
// out_b = Uv T_b Uh^T on the block's folded halo tile T_b; its transpose
// spreads the block's output gradient g back over the tile (as adjoint.cu):
//   pass A: Z[yo][ex] = sum_xo u(offx + ex - xo) g[yo][xo]
//   pass B: G[ey][ex] = sum_yo u(offy + ey - yo) Z[yo][ex]
//   g_in[gy0 + ey][gx0 + ex] += G[ey][ex]   (one fp32 atomic add per pixel)
// plus the clamped taps folded onto the tile's edge columns (pass A) and edge
// rows (pass B) through the prefix sums CU. The taps are symmetric (u(m) =
// u(2r - m), bit for bit), so pass A is the Toeplitz product
// B[k][n] = u(Dx + k - n) with Dx = 2r - offx and pass B the product
// A[m][k] = u(Dy + k - m) with Dy = 2r - offy: the forward kernel's
// fragment forms, read from the same tap-pair tables.
//
// Gradients have no fixed range, so each block plane is first scaled by a
// power of two (exact) that brings its largest |g| into [2^8, 2^9), then
// split into fp16 hi + lo like float32 frames in the forward kernel. (A
// folded edge column of Z collects the clamped weight of up to 32 output
// columns on each side, so |Z| stays below 65 x 2^9, inside fp16.) Pass A
// issues g_hi U_hi + g_lo U_hi + g_hi U_lo, Z is split again for pass B,
// and the result is scaled back. The error is about 2^-21 of the block's
// largest |g| (not of each element): an element below that scale carries
// an absolute, not a relative, error. A block plane of zeros is skipped; a
// non-finite gradient propagates (no scaling). Each unit has a K of 32 (two
// k-steps, six MMAs), so the tensor cores' truncating adds cost at most a
// few ulps.
//
// Work: persistent CTAs of 8 warps take items from the work list; per plane
// and 256-column slab of the tile, warp w takes the 8-column n-tiles w,
// w + 8, ... of both passes (pass A: its two 16-row m-tiles; pass B: the
// ceil(EH / 16) m-tiles two at a time, its Z fragments read once), every
// product group in its own accumulator so that independent MMA chains
// overlap; Z sits in shared memory transposed ([column][row], hi and lo
// fp16) so that pass B reads its B fragments as 32-bit words.
#include "tc_common.cuh"

namespace fovea {

namespace {

using namespace tcc;

constexpr int kNWA = 8;                 // warps
constexpr int kNTA = 32 * kNWA;
constexpr int kSlabA = 256;             // tile columns per slab
constexpr int kZP = 40;                 // Z^T row pitch (halves): 32 rows + 8; row starts 20 words apart
constexpr int kGP = 40;                 // g row pitch (halves): ldmatrix rows 20 words apart
constexpr float kInvW = 1.0f / 4096.0f; // taps are scaled by 2^12 in the pair tables

// Z^T capacity (halves per hi or lo array): the item's C planes share it,
// C slabs of (256 / C) columns (a multiple of 8) side by side.
constexpr int kZCols = kSlabA;
__host__ __device__ constexpr int tca_slab(int C) { return (kZCols / C) & ~7; }

struct TcaLayout {
  size_t zh, zl, gh, gl, gf, zf, pairs, cum, red, scale, total;
};

__host__ __device__ inline TcaLayout tca_layout(int rmax) {
  TcaLayout L;
  L.zh = 0;                                                   // half [C][slab][kZP]
  L.zl = L.zh + (size_t)kZCols * kZP * 2;                     // half [C][slab][kZP]
  L.gh = L.zl + (size_t)kZCols * kZP * 2;                     // half [4][32][kGP]
  L.gl = L.gh + (size_t)4 * 32 * kGP * 2;                     // half [4][32][kGP]
  L.gf = L.gl + (size_t)4 * 32 * kGP * 2;                     // float [4][32][33], unscaled g
  L.zf = L.gf + (size_t)4 * 32 * 33 * 4;                      // float [4][2][32], folded edge columns
  L.pairs = L.zf + (size_t)4 * 2 * 32 * 4;                    // uint32 [4][npair]
  L.cum = L.pairs + (size_t)4 * npair(rmax) * 4;              // float [cum_len]
  L.red = L.cum + (size_t)((cum_len(rmax) + 3) & ~3) * 4;     // float [kNWA][4]
  L.scale = L.red + (size_t)kNWA * 4 * 4;                     // float [4] scale, [4] inverse
  L.total = L.scale + (size_t)8 * 4;
  return L;
}

__global__ void __launch_bounds__(kNTA, 2)
tca_adjoint_kernel(FrameSource src, Workspace ws, int rmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TcaLayout L = tca_layout(rmax);
  __half* Zh = reinterpret_cast<__half*>(smem + L.zh);
  __half* Zl = reinterpret_cast<__half*>(smem + L.zl);
  __half* Gh = reinterpret_cast<__half*>(smem + L.gh);
  __half* Gl = reinterpret_cast<__half*>(smem + L.gl);
  float* GF = reinterpret_cast<float*>(smem + L.gf);
  float* ZF = reinterpret_cast<float*>(smem + L.zf);
  unsigned int* P = reinterpret_cast<unsigned int*>(smem + L.pairs);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  float* red = reinterpret_cast<float*>(smem + L.red);
  float* SC = reinterpret_cast<float*>(smem + L.scale);  // [4] scale 2^e per plane (0: a plane of zeros), [4] 2^-e
  __shared__ int s_ticket;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n_items = (int)ws.counters[CNT_NITEMS];
  const int np = npair(rmax);
  unsigned int* err = ws.counters + CNT_ERROR;

  for (;;) {
    if (tid == 0) s_ticket = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
    __syncthreads();  // also: the previous item is finished by every thread
    const int tk = s_ticket;
    __syncthreads();
    if (tk >= n_items) break;
    const int item = ws.order[tk];
    if ((unsigned)item >= (unsigned)n_items) {  // work list out of step: skip, flag
      if (tid == 0) atomicOr(err, kFaultWorklist);
      continue;
    }
    const ItemInfo inf = ws.items[item];
    const FrameDesc fd = load_frame(src, inf.frame);
    const int r = inf.r;
    if (r > rmax || fd.fmt != FOVEA_F32_CHW || fd.C > 4) {
      if (tid == 0) atomicOr(err, kFaultAdjBound);
      continue;
    }
    const int W = fd.W, H = fd.H, C = fd.C, T = fd.T;
    const int tx = inf.block % fd.nbx, ty = inf.block / fd.nbx;
    const int xs = tx * T - fd.ox, ys = ty * T - fd.oy;
    const int x0 = max(0, xs), y0 = max(0, ys);
    const int bw = min(xs + T, W) - x0, bh = min(ys + T, H) - y0;
    const int gx0 = max(0, x0 - r), EW = min(W - 1, x0 + bw - 1 + r) - gx0 + 1, offx = gx0 - (x0 - r);
    const int gy0 = max(0, y0 - r), EH = min(H - 1, y0 + bh - 1 + r) - gy0 + 1, offy = gy0 - (y0 - r);
    const bool foldL = x0 - r < 0, foldR = x0 + bw - 1 + r > W - 1;
    const bool foldT = y0 - r < 0, foldB = y0 + bh - 1 + r > H - 1;
    const int Dx = 2 * r - offx, Dy = 2 * r - offy;
    const size_t plane = (size_t)W * H;
    const float* gout = static_cast<const float*>(fd.in);
    float* gin = static_cast<float*>(fd.out);
    const size_t gin_bytes = plane * C * 4;

    {
      const float c_tap = inf.neg_half_inv_s2;
      const float S = warp_tap_sum(r, c_tap);
      make_pairs<kNTA>(P, r, c_tap, S, np);
      if ((foldL || foldR || foldT || foldB) && warp == kNWA - 1) make_cumulative_tc(CU, r, c_tap, S);
    }

    // ---- the block's gradient planes: unscaled copy, largest |g| per plane
    // (infinite where a plane holds a non-finite value)
    float mloc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 4 * C; ++k) {
      const int idx = tid + kNTA * k, c = idx >> 10, yo = (idx >> 5) & 31, xo = idx & 31;
      float v = 0.0f;
      if (yo < bh && xo < bw) v = __ldg(gout + (size_t)c * plane + (size_t)(y0 + yo) * W + x0 + xo);
      GF[(c * 32 + yo) * 33 + xo] = v;
      const float a = fabsf(v) <= 3.0e38f ? fabsf(v) : __int_as_float(0x7f800000);
      #pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q == c) mloc[q] = fmaxf(mloc[q], a);
    }
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
      #pragma unroll
      for (int o = 16; o > 0; o >>= 1) mloc[q] = fmaxf(mloc[q], __shfl_xor_sync(0xffffffffu, mloc[q], o));
      if (lane == 0) red[warp * 4 + q] = mloc[q];
    }
    __syncthreads();  // tables, GF and the warps' maxima are written
    if (tid < C) {
      // 2^e with M 2^e in [2^8, 2^9): exact power-of-two scaling (a folded
      // edge column of Z collects up to 64 clamped weights, so |Z| < 65 x
      // 2^9 stays inside fp16); no scaling for a non-finite plane
      float M = 0.0f;
      for (int w = 0; w < kNWA; ++w) M = fmaxf(M, red[w * 4 + tid]);
      int ex = 0;
      if (M <= 3.0e38f) {
        frexpf(M, &ex);  // M = f 2^ex, f in [0.5, 1)
        ex = 9 - ex;
        ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
      }
      SC[tid] = M == 0.0f ? 0.0f : ldexpf(1.0f, ex);  // 0: a plane of zeros adds nothing
      SC[4 + tid] = ldexpf(1.0f, -ex);
    }
    // folded edge columns of pass A, unscaled: (plane, side, row) per thread
    if (tid < C * 64) {
      const int c = tid >> 6, side = (tid >> 5) & 1, yo = tid & 31;
      if (side == 0 ? foldL : foldR) {
        float s = 0.0f;
        for (int xo = 0; xo < bw; ++xo) {
          const float cw = side == 0 ? cum_at(CU, offx - xo, r) : cum_at(CU, 2 * r + 1 - (offx + EW - xo), r);
          s = fmaf(cw, GF[(c * 32 + yo) * 33 + xo], s);
        }
        ZF[(c * 2 + side) * 32 + yo] = s;
      }
    }
    __syncthreads();  // scales and folded columns ready
    for (int k = 0; k < 4 * C; ++k) {
      const int idx = tid + kNTA * k, c = idx >> 10, yo = (idx >> 5) & 31, xo = idx & 31;
      const float v = GF[(c * 32 + yo) * 33 + xo] * SC[c];
      const __half h = __float2half_rn(v);
      Gh[(c * 32 + yo) * kGP + xo] = h;
      Gl[(c * 32 + yo) * kGP + xo] = __float2half_rn(v - __half2float(h));
    }
    __syncthreads();  // scaled hi / lo parts ready

    const int slab = tca_slab(C);  // tile columns per slab and plane
    for (int X0 = 0; X0 < EW; X0 += slab) {
      const int SW = min(slab, EW - X0);
      const int ntn = (SW + 7) >> 3;
      // ---- pass A: Z[c][yo][ex] for ex in [X0, X0 + 8 ntn), as Z^T hi / lo.
      // Warp w takes the (plane, n-tile) units w, w + 8, ...; both m-tiles of
      // each, the products of each m-tile in two accumulators (hi-B and
      // lo-B), so four independent MMA chains share the unit's tap fragments.
      {
        const int par = (Dx + g) & 1;
        const unsigned int* Qh = P + (par ? np : 0);
        const unsigned int* Ql = P + 2 * np + (par ? np : 0);
        for (int u = warp; u < C * ntn; u += kNWA) {
          const int c = u / ntn, nt = u - c * ntn;
          const float sc = SC[c];
          if (sc == 0.0f) continue;
          const int n0 = X0 + 8 * nt;  // tile column of the unit's first output
          float acc[2][2][4];
          #pragma unroll
          for (int mt = 0; mt < 2; ++mt)
            #pragma unroll
            for (int q = 0; q < 2; ++q)
              #pragma unroll
              for (int e = 0; e < 4; ++e) acc[mt][q][e] = 0.f;
          #pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const int i0 = Dx + 16 * ks - n0;  // tap index at k = 16 ks, n = n0
            if (i0 + 15 < 0 || i0 - 7 > 2 * r) continue;  // the band misses this k-step
            const int jb = (i0 + 2 * t - g + kPairPad) >> 1;
            const unsigned int bh0 = Qh[jb], bh1 = Qh[jb + 4], bl0 = Ql[jb], bl1 = Ql[jb + 4];
            const int acol = 16 * ks + ((lane >> 4) & 1) * 8;
            #pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              const int arow = c * 32 + 16 * mt + (lane & 7) + ((lane >> 3) & 1) * 8;
              unsigned int a_h[4], a_l[4];
              ldsm_x4(a_h, Gh + arow * kGP + acol);
              ldsm_x4(a_l, Gl + arow * kGP + acol);
              mma16816(acc[mt][0], a_h, bh0, bh1);
              mma16816(acc[mt][1], a_h, bl0, bl1);
              mma16816(acc[mt][0], a_l, bh0, bh1);
            }
          }
          #pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            #pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int yo = 16 * mt + g + ((e >> 1) << 3), exl = 8 * nt + 2 * t + (e & 1);
              const int ext = X0 + exl;  // tile column
              float v = acc[mt][0][e] + acc[mt][1][e];
              if (foldL && ext == 0) v = fmaf(ZF[(c * 2) * 32 + yo] * sc, kWScale, v);
              if (foldR && ext == EW - 1) v = fmaf(ZF[(c * 2 + 1) * 32 + yo] * sc, kWScale, v);
              v *= kInvW;
              const __half h = __float2half_rn(v);
              const size_t o = (size_t)(c * slab + exl) * kZP + yo;
              if (smem_in_bounds(Zh + o, 2, err) && smem_in_bounds(Zl + o, 2, err)) {
                Zh[o] = h;
                Zl[o] = __float2half_rn(v - __half2float(h));
              }
            }
          }
        }
      }
      __syncthreads();  // Z complete
      // ---- pass B: G[c][ey][ex] = sum_yo u(Dy + yo - ey) Z[c][yo][ex], then
      // the reductions into g_in. Warp w takes the (plane, n-tile) units w,
      // w + 8, ...: the unit's Z fragments (both k-steps) are read once, then
      // its m-tiles go two at a time, each in two accumulators.
      {
        const int ntm = (EH + 15) >> 4;
        const int par = (Dy + g) & 1;
        const unsigned int* Ph = P + (par ? np : 0);
        const unsigned int* Pl = P + 2 * np + (par ? np : 0);
        for (int u = warp; u < C * ntn; u += kNWA) {
          const int c = u / ntn, nt = u - c * ntn;
          if (SC[c] == 0.0f) continue;
          const float isc = SC[4 + c];
          const int n0 = 8 * nt;  // slab column
          unsigned int zf[2][4];  // [ks]: hi b0, hi b1, lo b0, lo b1
          #pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const size_t zb = (size_t)(c * slab + n0 + g) * kZP + 16 * ks + 2 * t;
            zf[ks][0] = *reinterpret_cast<const unsigned int*>(Zh + zb);
            zf[ks][1] = *reinterpret_cast<const unsigned int*>(Zh + zb + 8);
            zf[ks][2] = *reinterpret_cast<const unsigned int*>(Zl + zb);
            zf[ks][3] = *reinterpret_cast<const unsigned int*>(Zl + zb + 8);
          }
          float* gplane = gin + (size_t)c * plane;
          for (int mp = 0; mp < ntm; mp += 2) {
            float acc[2][2][4];
            #pragma unroll
            for (int h = 0; h < 2; ++h)
              #pragma unroll
              for (int q = 0; q < 2; ++q)
                #pragma unroll
                for (int e = 0; e < 4; ++e) acc[h][q][e] = 0.f;
            #pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int m0 = 16 * (mp + h);
              if (mp + h >= ntm) continue;
              #pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const int i0 = Dy + 16 * ks - m0;  // tap index at k = 16 ks, m = m0
                if (i0 + 15 < 0 || i0 - 15 > 2 * r) continue;
                const int j0 = (i0 + 2 * t - g + kPairPad) >> 1;
                const unsigned int ah[4] = {Ph[j0], Ph[j0 - 4], Ph[j0 + 4], Ph[j0]};
                const unsigned int al[4] = {Pl[j0], Pl[j0 - 4], Pl[j0 + 4], Pl[j0]};
                mma16816(acc[h][0], ah, zf[ks][0], zf[ks][1]);
                mma16816(acc[h][1], ah, zf[ks][2], zf[ks][3]);
                mma16816(acc[h][0], al, zf[ks][0], zf[ks][1]);
              }
            }
            #pragma unroll
            for (int h = 0; h < 2; ++h) {
              #pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int ey = 16 * (mp + h) + g + ((e >> 1) << 3), exl = n0 + 2 * t + (e & 1);
                if (ey >= EH || exl >= SW) continue;
                float v = acc[h][0][e] + acc[h][1][e];
                const bool ft = foldT && ey == 0, fb = foldB && ey == EH - 1;
                if (ft || fb) {  // folded edge rows: the clamped taps' weight on Z's column
                  float s = 0.0f;
                  for (int yo = 0; yo < bh; ++yo) {
                    float cw = 0.0f;
                    if (ft) cw += cum_at(CU, offy - yo, r);
                    if (fb) cw += cum_at(CU, 2 * r + 1 - (offy + EH - yo), r);
                    const size_t o = (size_t)(c * slab + exl) * kZP + yo;
                    s = fmaf(cw, __half2float(Zh[o]) + __half2float(Zl[o]), s);
                  }
                  v = fmaf(s, kWScale, v);
                }
                v *= kInvW * isc;
                if (v != 0.0f) {
                  float* p = gplane + (size_t)(gy0 + ey) * W + gx0 + X0 + exl;
                  if (in_bounds(p, 4, gin, gin_bytes, err)) red_add_f32(p, v);
                }
              }
            }
          }
        }
      }
      __syncthreads();  // Z is rewritten by the next slab
    }
  }
}

}  // namespace

size_t tca_adjoint_smem_bytes(int rmax) { return tca_layout(rmax).total; }

int tca_adjoint_max_ctas_per_sm(int rmax) {
  const size_t smem = tca_adjoint_smem_bytes(rmax);
  const void* k = reinterpret_cast<const void*>(&tca_adjoint_kernel);
  if (set_smem_attrs(k, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kNTA, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_tca_adjoint(const FrameSource& src, const Workspace& ws, int rmax, int grid, cudaStream_t s) {
  const size_t smem = tca_adjoint_smem_bytes(rmax);
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(&tca_adjoint_kernel), smem);
  if (e != cudaSuccess) return e;
  tca_adjoint_kernel<<<grid, kNTA, smem, s>>>(src, ws, rmax);
  return cudaGetLastError();
}

}  // namespace fovea
