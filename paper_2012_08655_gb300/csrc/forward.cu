// Forward foveation kernel: one persistent CTA loop over (frame, block) items.
//
// For one block (paper Section 2 and Algorithm 1: "place padded fragment into
// shared memory", "horizontal convolution", "place result into shared
// memory", "vertical convolution", "write result"):
//   * taps: the block's normalised 1D Gaussian (Eq. 1, truncated at
//     r = ceil(3 sigma)), generated in the CTA and summed with warp shuffles,
//     plus their exclusive prefix sums;
//   * folded halo tile: only the in-frame rows y0-r .. y0+bh-1+r and columns
//     x0-r .. x0+bw-1+r are staged; the taps that clamp-to-edge sends to a
//     position outside the frame are folded onto the edge row / column with
//     one prefix-summed weight (exact in real arithmetic);
//   * staging: rows stream through a 3-stage shared-memory ring filled with
//     16-byte cp.async copies, so the loads of later rows overlap the
//     arithmetic on earlier ones; uint8 is unpacked exactly in registers;
//   * pass 1 (vertical, halo rows): V[yo][e] = sum_y u[y - yo] T[y][e] for the
//     32 output rows and every tile element column e (pixel x channel);
//   * pass 2 (horizontal): O[yo][x][c] = sum_x' u[x' - x] V[yo][x'][c];
//   * round/pack and store.
// The vertical pass runs first so the tile can stream by rows: shared memory
// does not grow with the radius. Wide tiles are cut into column slabs and
// pass 2 accumulates across slabs. All products are fp32 FMAs, two lanes per
// instruction (fma.rn.f32x2). In pass 1 a thread owns 2 element columns x 16
// output rows and keeps a sliding window of 16 taps in registers, so each
// value it loads feeds 16 packed FMAs; in pass 2 a thread owns 8 output
// columns x 2 rows (the register data reuse of the paper's "Data Reuse"
// subsection, generalised).
#include "fwd_common.cuh"

namespace fovea {

namespace {

using namespace fwd;

struct SmemLayout {
  size_t ring, vv, taps, cum, red, total;
};

// Ring stages of a kernel mode: float32-only launches (1024-byte rows) keep
// two stages, so that 32-row chunks still leave room for two CTAs per SM.
__host__ __device__ constexpr int mode_stages(int mode) { return mode == 1 ? 2 : kStages; }

__host__ __device__ inline SmemLayout smem_layout(int rb, int row_bytes, int rmax, int stages) {
  SmemLayout L;
  L.ring = 0;
  L.vv = L.ring + (size_t)stages * rb * row_bytes;
  L.taps = L.vv + (size_t)16 * kVVPitch * sizeof(float2);
  L.cum = L.taps + (size_t)tap_len(rmax) * sizeof(float2);
  L.red = L.cum + (size_t)cum_len(rmax) * sizeof(float);
  L.total = L.red + 32 * sizeof(float);
  return L;
}

// Element pair of one staged row as floats.
template <bool U8>
__device__ __forceinline__ float2 load_pair(const unsigned char* row, int pi) {
  if (U8) {
    return u8x2_to_f32(*reinterpret_cast<const unsigned short*>(row + 2 * pi));
  } else {
    return *reinterpret_cast<const float2*>(row + 8 * pi);
  }
}

struct Smem {
  unsigned char* ring;
  float2* VV;
  const float2* U;
  const float* CU;
};

// All slabs of one item; returns with acc2 holding the block's outputs.
template <bool U8, int RB, int ST>
__device__ __forceinline__ void process_item(const Item& it, const Smem& sm, float2 (&acc2)[8]) {
  constexpr int row_bytes = U8 ? kRowBytesU8 : kRowBytesF32;
  constexpr size_t stage_bytes = (size_t)RB * row_bytes;
  const int tid = threadIdx.x;
  const int r = it.r;
  const int nslabs = U8 ? it.nsl : it.nsl * it.C;
  const int Q = nslabs * it.nchunks;
  const size_t frame_bytes = (size_t)it.H * it.pitch * (U8 ? 1 : it.C);
  // pass-1 identity: element pair pi, row group G1 of kN1 output rows
  const int pi = tid & 127, G1 = tid >> 7;
  // pass-2 identity: row pair p2, channel c2, group g2 of 8 output columns
  const int g2 = tid >> 6, c2 = (tid >> 4) & 3, p2 = tid & 15;

  const int groups1 = (it.bh + kN1 - 1) / kN1, groups2 = (it.bw + 7) >> 3;
  const int steps1 = 1 + (2 * r + kN1 - 1) / kN1;  // kN1-row steps covering 2r + kN1 taps
  const int steps2 = 1 + ((2 * r + 7) >> 3);       // 8-column steps covering 2r + 8 taps
  const int vs1 = kN1 * G1 - it.offy + it.ph;      // virtual row where acc[0] sees tap 0
  const int v1lo = max(0, vs1), v1hi = min(it.vrows, vs1 + kN1 * steps1);
  const bool grp1 = G1 < groups1;
  const int xg = 8 * g2;
  const bool act2base = g2 < groups2 && c2 < it.C && 2 * p2 < it.bh;
  float2 a1[kN1];
  float2 wv[kN1];

  for (int q = 0; q < Q; ++q) {
    cp_async_wait<ST - 2>();
    __syncthreads();  // chunk q landed for every thread; chunk q-1 fully consumed
    {
      const int qn = q + ST - 1;
      if (qn < Q) stage_rows<U8, RB>(it, slab_of<U8>(it, qn / it.nchunks), qn % it.nchunks,
                                     sm.ring + (size_t)(qn % ST) * stage_bytes, frame_bytes);
      cp_async_commit();
    }
    const int s = q / it.nchunks, k = q - s * it.nchunks;
    const Slab sl = slab_of<U8>(it, s);
    const unsigned char* st = sm.ring + (size_t)(q % ST) * stage_bytes;
    const int R0 = k * RB;
    // ring pair pi holds slab elements 2*pi - ph and 2*pi - ph + 1
    const int e_first = 2 * pi - sl.ph;
    const bool act1 = grp1 && e_first + 1 >= 0 && e_first < sl.sws;
    if (k == 0) {
      #pragma unroll
      for (int j = 0; j < kN1; ++j) a1[j] = make_float2(0.f, 0.f);
      // Folded top row: taps clamped onto the first frame row (applied first,
      // so the summation order does not depend on the chunk size).
      if (act1 && it.foldT) {
        const float2 d = load_pair<U8>(st + (size_t)it.ph * row_bytes, pi);
        #pragma unroll
        for (int j = 0; j < kN1; ++j) {
          const float cw = cum_at(sm.CU, it.offy - (kN1 * G1 + j), r);
          a1[j] = ffma2(make_float2(cw, cw), d, a1[j]);
        }
      }
    }
    if (act1) {
      const int lo = max(R0, v1lo), hi = min(R0 + RB, v1hi);
      if (lo < hi && lo == v1lo) {  // first row of the group: preload the tap window
        #pragma unroll
        for (int u = 1; u < kN1; ++u) wv[u] = sm.U[kTapPad + (lo - vs1) - kN1 + u];
      }
      const unsigned char* rowp = st + (size_t)(lo - R0) * row_bytes;
      const float2* up = sm.U + kTapPad + (lo - vs1);
      for (int v0 = lo; v0 < hi; v0 += kN1) {
        #pragma unroll
        for (int u = 0; u < kN1; ++u) {
          wv[u] = up[u];
          const float2 d = load_pair<U8>(rowp + (size_t)u * row_bytes, pi);
          #pragma unroll
          for (int j = 0; j < kN1; ++j) a1[j] = ffma2(wv[(u - j) & (kN1 - 1)], d, a1[j]);
        }
        rowp += (size_t)kN1 * row_bytes;
        up += kN1;
      }
      // Folded bottom row: taps clamped onto the last frame row.
      const int vb = it.ph + it.EH - 1;
      if (it.foldB && vb >= R0 && vb < R0 + RB) {
        const float2 d = load_pair<U8>(st + (size_t)(vb - R0) * row_bytes, pi);
        #pragma unroll
        for (int j = 0; j < kN1; ++j) {
          const float cw = cum_at(sm.CU, 2 * r + 1 - (it.offy + it.EH - (kN1 * G1 + j)), r);
          a1[j] = ffma2(make_float2(cw, cw), d, a1[j]);
        }
      }
    }
    if (k != it.nchunks - 1) continue;

    // ---- slab complete: V rows -> row-pair buffer, then pass 2 over the slab
    if (act1) {
      #pragma unroll
      for (int pp = 0; pp < kN1 / 2; ++pp) {
        float2* dst = sm.VV + (kN1 / 2 * G1 + pp) * kVVPitch + kVVPad;
        if (e_first >= 0) dst[e_first] = make_float2(a1[2 * pp].x, a1[2 * pp + 1].x);
        if (e_first + 1 < sl.sws) dst[e_first + 1] = make_float2(a1[2 * pp].y, a1[2 * pp + 1].y);
      }
    }
    // zero the columns right of the slab (pass 2 reads up to 7 pixels past it)
    for (int idx = tid; idx < 16 * kVVPad; idx += kThreads) {
      const int row = idx / kVVPad, col = idx - row * kVVPad;
      sm.VV[row * kVVPitch + kVVPad + sl.sws + col] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const bool act2 = act2base && (U8 || c2 == sl.c);
    if (act2) {
      const int Cs = U8 ? it.C : 1;
      const int P0 = sl.e0 / Cs, P1 = P0 + sl.sws / Cs;  // folded columns of the slab
      const int xs = xg - it.offx;                         // column whose tap index is 0 for x = xg
      const int lo = max(P0, xs), hi = min(P1, xs + 8 * steps2);
      const float2* vrow = sm.VV + p2 * kVVPitch + kVVPad + (U8 ? c2 : 0);
      if (lo < hi) {
        const int la = lo - ((lo - xs) & 7);
        float2 w2[8];
        #pragma unroll
        for (int u = 1; u < 8; ++u) w2[u] = sm.U[kTapPad + (la - xs) - 8 + u];
        const float2* up = sm.U + kTapPad + (la - xs);
        const float2* vp = vrow + (la - P0) * Cs;
        for (int x0c = la; x0c < hi; x0c += 8) {
          #pragma unroll
          for (int u = 0; u < 8; ++u) {
            w2[u] = up[u];
            const float2 d = vp[u * Cs];
            #pragma unroll
            for (int j = 0; j < 8; ++j) acc2[j] = ffma2(w2[(u - j) & 7], d, acc2[j]);
          }
          up += 8;
          vp += 8 * Cs;
        }
      }
      // Folded edge columns.
      #pragma unroll
      for (int f = 0; f < 2; ++f) {
        const bool on = f == 0 ? it.foldL : it.foldR;
        const int ex = f == 0 ? 0 : it.EW - 1;
        if (on && ex >= P0 && ex < P1) {
          const float2 d = vrow[(ex - P0) * Cs];
          #pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int x = xg + j;
            const float cw = f == 0 ? cum_at(sm.CU, it.offx - x, r) : cum_at(sm.CU, 2 * r + 1 - (it.offx + it.EW - x), r);
            acc2[j] = ffma2(make_float2(cw, cw), d, acc2[j]);
          }
        }
      }
    }
  }
}

// One item (one block of one frame), start to finish: stage its folded halo
// tile, build its taps, run both passes and store the block. Every thread of
// the CTA calls it; `c` is -1 / (2 sigma^2). taps_ready: U and CU already
// hold the item's taps and their prefix sums.
template <int RB, int MODE>
__device__ __forceinline__ void run_item(const Item& it, float c, const Smem& sm, float2* U, float* CU, float* red,
                                         unsigned int* err, bool taps_ready = false) {
  const int tid = threadIdx.x;
  const int g2 = tid >> 6, c2 = (tid >> 4) & 3, p2 = tid & 15;
  const bool u8 = MODE == 0 ? true : (MODE == 1 ? false : it.isu8);
  const int r = it.r;

  // Start staging before the taps are ready: the copies do not need them.
  {
    constexpr int rbu = kRowBytesU8, rbf = kRowBytesF32;
    #pragma unroll
    for (int q = 0; q < mode_stages(MODE) - 1; ++q) {
      const int Q = (u8 ? it.nsl : it.nsl * it.C) * it.nchunks;
      if (q < Q) {
        if (MODE != 1 && u8) stage_rows<true, RB>(it, slab_of<true>(it, q / it.nchunks), q % it.nchunks,
                                                  sm.ring + (size_t)q * RB * rbu, (size_t)it.H * it.pitch);
        if (MODE != 0 && !u8) stage_rows<false, RB>(it, slab_of<false>(it, q / it.nchunks), q % it.nchunks,
                                                    sm.ring + (size_t)q * RB * rbf, (size_t)it.H * it.pitch * it.C);
      }
      cp_async_commit();
    }
  }
  if (!taps_ready) {
    make_taps(U, tap_len(r), r, c, red);
    make_cumulative(U, CU, r);
  }
  __syncthreads();

  float2 acc2[8];
  #pragma unroll
  for (int j = 0; j < 8; ++j) acc2[j] = make_float2(0.f, 0.f);
  if (MODE != 1 && u8) process_item<true, RB, mode_stages(MODE)>(it, sm, acc2);
  if (MODE != 0 && !u8) process_item<false, RB, mode_stages(MODE)>(it, sm, acc2);

  cp_async_wait<0>();
  __syncthreads();  // ring no longer read; it becomes the output stage

  const int groups2 = (it.bw + 7) >> 3, xg = 8 * g2;
  const bool act2base = g2 < groups2 && c2 < it.C && 2 * p2 < it.bh;
  if (!u8) {
    if (act2base) {
      float* out = reinterpret_cast<float*>(it.out) + (size_t)c2 * it.W * it.H +
                   (size_t)(it.y0 + 2 * p2) * it.W + it.x0;
      const bool second = 2 * p2 + 1 < it.bh;
      #pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int x = xg + j;
        if (x < it.bw) {
          const size_t plane_bytes = (size_t)it.W * it.H * it.C * 4;
          if (in_bounds(out + x, 4, it.out, plane_bytes, err)) out[x] = acc2[j].x;
          if (second && in_bounds(out + it.W + x, 4, it.out, plane_bytes, err))
            out[it.W + x] = acc2[j].y;
        }
      }
    }
  } else {
    unsigned char* ost = sm.ring;
    const int opitch = 32 * it.C;
    if (act2base) {
      #pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int x = xg + j;
        ost[(2 * p2) * opitch + x * it.C + c2] = quant_u8(acc2[j].x);
        ost[(2 * p2 + 1) * opitch + x * it.C + c2] = quant_u8(acc2[j].y);
      }
    }
    __syncthreads();
    const int rowBytes = it.bw * it.C;
    unsigned char* out = it.out + (size_t)it.y0 * it.pitch + (size_t)it.x0 * it.C;
    for (int idx = tid; idx < it.bh * rowBytes; idx += kThreads) {
      const int yo = idx / rowBytes, rem = idx - yo * rowBytes;
      unsigned char* o = out + (size_t)yo * it.pitch + rem;
      if (in_bounds(o, 1, it.out, (size_t)it.H * it.pitch, err)) *o = ost[yo * opitch + rem];
    }
  }
}

// MODE 0: uint8 frames only; 1: float32 frames only; 2: both (batches).
template <int RB, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
forward_kernel(FrameSource src, Workspace ws, int rmax, int row_bytes, BucketList bl) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(RB, row_bytes, rmax, mode_stages(MODE));
  Smem sm;
  sm.ring = smem + L.ring;
  sm.VV = reinterpret_cast<float2*>(smem + L.vv);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  sm.U = U;
  sm.CU = CU;
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_state;  // 0 run, 1 skip item, 2 stop
  __shared__ Item s_it;
  __shared__ float s_c;
  __shared__ int s_start[kBuckets];
  __shared__ int s_wsum[kThreads / 32];

  const int tid = threadIdx.x;
  // The VV pads must read as zeros: clear the whole buffer once.
  for (int i = tid; i < 16 * kVVPitch; i += kThreads) sm.VV[i] = make_float2(0.f, 0.f);
  // Launched as a programmatic dependent of the sigma kernel: wait for its
  // results (no-op otherwise).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const bool own_order = bl.list != nullptr;
  const int n_items = own_order ? (int)src.one_total : (int)ws.counters[CNT_NITEMS];
  if (own_order) bucket_starts(ws.counters + CNT_HIST, bl.nb, s_start, s_wsum);

  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (tid == 0) {
      const int t = (int)atomicAdd(&ws.counters[CNT_TICKET], 1u);
      int state = 0;
      if (t >= n_items) {
        state = 2;
      } else {
        int item;
        if (own_order) {  // smallest radius bucket whose first ticket is <= t
          int lo = 0, hi = bl.nb - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_start[mid] <= t) hi = mid; else lo = mid + 1;
          }
          item = bl.list[(size_t)lo * bl.cap + (t - s_start[lo])];
        } else {
          item = ws.order[t];
        }
        if ((unsigned)item >= (unsigned)n_items) {  // work list out of step: skip, flag
          atomicOr(&ws.counters[CNT_ERROR], kFaultWorklist);
          state = 1;
        } else {
          const ItemInfo inf = ws.items[item];
          const FrameDesc fd = load_frame(src, inf.frame);
          const bool u8f = fd.fmt == FOVEA_U8_HWC;
          const bool fmt_ok = MODE == 2 ? (u8f || row_bytes >= kRowBytesF32) : (MODE == 0 ? u8f : !u8f);
          if (inf.r > rmax || !fmt_ok) {
            atomicOr(&ws.counters[CNT_ERROR], kFaultRadiusBound);
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
    run_item<RB, MODE>(s_it, s_c, sm, U, CU, red, ws.counters + CNT_ERROR);
  }
  cp_async_wait<0>();
  if (own_order) {
    // The last CTA out clears the histogram and re-arms the ticket counter
    // for the next launch (every CTA read the histogram before it got here).
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

// Single-launch form for frames with no more blocks than one wave of CTAs:
// CTA b serves tile b alone. It evaluates the block's sigma itself (the
// sigma kernel's item_record, so the radius and taps are the same bit for
// bit) and runs the same item body, so no sigma kernel, work list or ticket
// precedes it: a small frame costs one launch and one CTA's latency. As a
// programmatic dependent launch it builds the block's sigma and taps (kernel
// arguments only) before it waits for the previous grid, and lets the next
// launch start as soon as every CTA got that far; a sigma map, the frame and
// the output are touched only after the wait.
template <int RB, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
direct_kernel(const __grid_constant__ FrameDesc fd, Workspace ws, int rmax, int row_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout L = smem_layout(RB, row_bytes, rmax, mode_stages(MODE));
  Smem sm;
  sm.ring = smem + L.ring;
  sm.VV = reinterpret_cast<float2*>(smem + L.vv);
  float2* U = reinterpret_cast<float2*>(smem + L.taps);
  float* CU = reinterpret_cast<float*>(smem + L.cum);
  sm.U = U;
  sm.CU = CU;
  float* red = reinterpret_cast<float*>(smem + L.red);
  __shared__ int s_state;
  __shared__ Item s_it;
  __shared__ float s_c;
  const int tid = threadIdx.x;
  unsigned int* err = ws.counters + CNT_ERROR;
  auto record = [&]() {  // thread 0: the block's item and geometry
    const ItemInfo inf = item_record(fd, 0, (int)blockIdx.x, err);
    const bool u8f = fd.fmt == FOVEA_U8_HWC;
    if (inf.r > rmax || (MODE == 0 ? !u8f : u8f)) {
      atomicOr(err, kFaultRadiusBound);
      s_state = 1;
    } else {
      item_geometry(s_it, inf, fd, RB);
      s_c = inf.neg_half_inv_s2;
      s_state = 0;
    }
  };
  for (int i = tid; i < 16 * kVVPitch; i += kThreads) sm.VV[i] = make_float2(0.f, 0.f);
  const bool early = fd.smap == nullptr;  // the law reads no device memory
  if (early) {
    if (tid == 0) record();
    __syncthreads();
    if (s_state == 0) {
      make_taps(U, tap_len(s_it.r), s_it.r, s_c, red);
      make_cumulative(U, CU, s_it.r);
    }
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (!early) {
    if (tid == 0) record();
    __syncthreads();
  }
  if (s_state == 0) run_item<RB, MODE>(s_it, s_c, sm, U, CU, red, err, early);
  cp_async_wait<0>();
}

template <int RB, int MODE>
void* direct_ptr() { return reinterpret_cast<void*>(&direct_kernel<RB, MODE>); }

void* pick_direct(int rb, int mode) {
  if (mode == 0) return rb == 16 ? direct_ptr<16, 0>() : (rb == 64 ? direct_ptr<64, 0>() : direct_ptr<32, 0>());
  return rb == 16 ? direct_ptr<16, 1>() : (rb == 64 ? direct_ptr<64, 1>() : direct_ptr<32, 1>());
}

template <int RB, int MODE>
void* kernel_ptr() { return reinterpret_cast<void*>(&forward_kernel<RB, MODE>); }

template <int MODE>
void* pick_rb(int rb) {
  switch (rb) {
    case 16: return kernel_ptr<16, MODE>();
    case 64: return kernel_ptr<64, MODE>();
    default: return kernel_ptr<32, MODE>();
  }
}

void* pick_kernel(int rb, int mode) {
  return mode == 0 ? pick_rb<0>(rb) : (mode == 1 ? pick_rb<1>(rb) : pick_rb<2>(rb));
}

int mode_of(int fmt_mask) { return fmt_mask == 1 ? 0 : (fmt_mask == 2 ? 1 : 2); }

}  // namespace

namespace {

// Row chunk the launch uses: the configured one, halved (down to 16 rows)
// while a float32 launch's ring of 1024-byte rows would leave room for only
// one CTA per SM (measured on 224 x 224 float32 batches: two CTAs per SM beat
// one with longer chunks).
int effective_rb(const FwdConfig& cfg, int rmax, int fmt_mask) {
  int rb = cfg.rows_per_chunk;
  if (fmt_mask & 2) {
    constexpr size_t kTwoPerSm = 110 * 1024;
    const int st = mode_stages(mode_of(fmt_mask));
    while (rb > 16 && smem_layout(rb, kRowBytesF32, rmax, st).total > kTwoPerSm) rb /= 2;
  }
  return rb;
}

}  // namespace

size_t forward_smem_bytes(const FwdConfig& cfg, int rmax, int fmt_mask) {
  return smem_layout(effective_rb(cfg, rmax, fmt_mask), (fmt_mask & 2) ? kRowBytesF32 : kRowBytesU8, rmax,
                     mode_stages(mode_of(fmt_mask))).total;
}

int forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int fmt_mask) {
  const size_t smem = forward_smem_bytes(cfg, rmax, fmt_mask);
  void* k = pick_kernel(effective_rb(cfg, rmax, fmt_mask), mode_of(fmt_mask));
  if (set_smem_attrs(reinterpret_cast<const void*>(k), smem) != cudaSuccess) {
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

cudaError_t launch_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg,
                           int rmax, int fmt_mask, int grid, cudaStream_t s, const BucketList& bl, bool pdl) {
  const size_t smem = forward_smem_bytes(cfg, rmax, fmt_mask);
  int row_bytes = (fmt_mask & 2) ? kRowBytesF32 : kRowBytesU8;
  void* k = pick_kernel(effective_rb(cfg, rmax, fmt_mask), mode_of(fmt_mask));
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  BucketList b = bl;
  void* args[] = {const_cast<FrameSource*>(&src), const_cast<Workspace*>(&ws), &rmax, &row_bytes, &b};
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

cudaError_t launch_forward_direct(const FrameDesc& fd, long long items, const Workspace& ws, const FwdConfig& cfg,
                                  int rmax, int fmt_mask, cudaStream_t s, bool pdl) {
  if (fmt_mask != 1 && fmt_mask != 2) return cudaErrorInvalidValue;
  int row_bytes = fmt_mask == 2 ? kRowBytesF32 : kRowBytesU8;
  // 64-row chunks where they fit: a halo of up to 64 rows is then staged in
  // one chunk, one global-memory round trip (a single wave needs no second
  // CTA per SM); the chunk size does not change the result
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return cudaGetLastError();
  const int st = mode_stages(mode_of(fmt_mask));
  int rb = smem_layout(64, row_bytes, rmax, st).total + 2048 <= (size_t)optin ? 64 : effective_rb(cfg, rmax, fmt_mask);
  (void)cfg;
  const size_t smem = smem_layout(rb, row_bytes, rmax, st).total;
  void* k = pick_direct(rb, mode_of(fmt_mask));
  cudaError_t e = set_smem_attrs(reinterpret_cast<const void*>(k), smem);
  if (e != cudaSuccess) return e;
  FrameDesc d = fd;
  Workspace w = ws;
  void* args[] = {&d, &w, &rmax, &row_bytes};
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned int)items);
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
