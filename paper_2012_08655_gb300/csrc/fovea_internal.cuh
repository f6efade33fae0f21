// Internal declarations shared by the libfovea translation units.
//
// Work decomposition: one work ITEM is one (frame, block) pair with all of
// its channels. A sigma-table kernel computes every item's sigma and radius,
// a second small kernel sorts the items by radius (largest first, the
// longest-processing-time order), and persistent kernels pull items from
// that list through an atomic ticket counter.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fovea.h"

namespace fovea {

constexpr int kMaxBlock = FOVEA_MAX_BLOCK;   // block side: <= 32, or a multiple of 32 up to this
constexpr int kMaxRadius = FOVEA_MAX_RADIUS; // r <= 1023
constexpr int kBuckets = 1024;               // radius buckets of the work-list sort
constexpr int kTapPad = 16;                  // zero taps stored before offset 0

// One frame as the kernels see it (host fills it in; 112 bytes). Work items
// are tiles of side T = min(B, 32); a block of side B > 32 (a multiple of 32)
// is (B / T)^2 tiles that share its sigma.
struct FrameDesc {
  const void* in;
  void* out;
  int W, H, C, fmt;        // fmt: FOVEA_U8_HWC or FOVEA_F32_CHW
  int nbx, nby, B, tma;    // block grid and block side; tma: a tensor map of the frame's rows is provided
  float fx, fy;            // fixation (pixels)
  double sigma0, k;        // sigma law
  long long item0;         // index of the frame's first item in a batch
  int ox, oy;              // grid origin: block (bx, by) starts at (B bx - ox, B by - oy)
  const float* smap;       // per-block sigma [blocks along y][nbxb] replacing the law, or null
  int T, nbxb;             // tile side; blocks along x (nbx, nby count tiles)
  double smap_max;         // declared bound of the map's values (map values above it are clamped)
};

// Device-resident batch: header followed by the frame descriptors, then
// (at maps_offset bytes from the header, 64-byte aligned) one 128-byte
// tensor map per frame, valid for the frames whose tma flag is set.
struct BatchHeader {
  int nframes;
  int maps_offset;
  long long total_items;
};

// Per-item record written by the sigma kernel.
struct ItemInfo {
  float sigma;             // sigma_b rounded to float
  float neg_half_inv_s2;   // -1 / (2 sigma_b^2), rounded from binary64
  int r;                   // ceil(3 sigma_b), clamped to kMaxRadius
  int frame;               // frame index in the batch
  int block;               // row-major block index within the frame
  int pad;
};

enum {
  CNT_TICKET = 0,     // next ticket of the persistent kernels
  CNT_DONE_SIGMA = 1, // finished CTAs of the sigma kernel
  CNT_DONE_ORDER = 2, // finished CTAs of the order kernel
  CNT_NITEMS = 3,     // items of the current launch
  CNT_ERROR = 4,      // device fault word (FOVEA_FAULT_* bits, read by fovea_check)
  CNT_HIST = 8,       // kBuckets radius histogram
  CNT_TOTAL = CNT_HIST + kBuckets
};

struct Workspace {
  ItemInfo* items;         // [capacity]
  int* rank;               // [capacity] rank of the item inside its radius bucket
  int* order;              // [capacity] ticket -> item (radius descending)
  unsigned int* counters;  // [CNT_TOTAL]
  long long capacity;
};

// Per-radius item lists of a single-frame launch: list[r * cap + k] is the
// k-th item with radius r (k below the histogram count of r).
struct BucketList {
  int* list;
  int cap;  // items per bucket row (the frame's item count)
  int nb;   // buckets (radius bound + 1)
};

// Where the kernels read frame descriptors from: a device-resident batch
// (hdr != nullptr) or a single frame passed by value in the launch.
struct FrameSource {
  const BatchHeader* hdr;
  const FrameDesc* frames;
  FrameDesc one;
  long long one_total;
};

__device__ __forceinline__ FrameDesc load_frame(const FrameSource& s, int f) {
  return s.hdr ? s.frames[f] : s.one;
}

__device__ __forceinline__ long long source_total(const FrameSource& s) {
  return s.hdr ? s.hdr->total_items : s.one_total;
}

// Sigma law of one block in IEEE binary64 with every operation rounded on
// its own (no fused multiply-add), so the radius ceil(3 sigma) is reproduced
// bit for bit by any implementation that follows the same order:
//   centre = B*b + B/2;  e = sqrt(dx*dx + dy*dy);  sigma = sigma0 + k*e.
__device__ __forceinline__ void block_sigma(int bx, int by, int B, int ox, int oy, double fx, double fy,
                                            double sigma0, double k, double& sigma, int& r) {
  double half = __dmul_rn(0.5, (double)B);
  double cx = __dsub_rn(__dadd_rn(__dmul_rn((double)B, (double)bx), half), (double)ox);
  double cy = __dsub_rn(__dadd_rn(__dmul_rn((double)B, (double)by), half), (double)oy);
  double dx = __dsub_rn(cx, fx);
  double dy = __dsub_rn(cy, fy);
  double e = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  sigma = __dadd_rn(sigma0, __dmul_rn(k, e));
  r = (int)ceil(__dmul_rn(3.0, sigma));
}

// Device fault bits (the public FOVEA_FAULT_* values).
constexpr unsigned int kFaultSigmaRange = FOVEA_FAULT_SIGMA_RANGE;
constexpr unsigned int kFaultRadiusBound = FOVEA_FAULT_RADIUS_BOUND;
constexpr unsigned int kFaultAdjBound = FOVEA_FAULT_ADJ_BOUND;
constexpr unsigned int kFaultOrder = FOVEA_FAULT_ORDER;
constexpr unsigned int kFaultWorklist = FOVEA_FAULT_WORKLIST;
constexpr unsigned int kFaultBuckets = FOVEA_FAULT_BUCKETS;
constexpr unsigned int kFaultWait = FOVEA_FAULT_WAIT;
constexpr unsigned int kFaultPixelRadius = FOVEA_FAULT_PIXEL_RADIUS;
constexpr unsigned int kFaultBounds = FOVEA_FAULT_BOUNDS;
constexpr unsigned int kFaultValueRange = FOVEA_FAULT_VALUE_RANGE;

// Bounds-checked builds (-DFOVEA_BOUNDS): stores check their address first.
#if defined(FOVEA_BOUNDS)
constexpr bool kBoundsChecks = true;
#else
constexpr bool kBoundsChecks = false;
#endif

// True when [p, p + n) lies inside [base, base + bytes). Otherwise (bounds-
// checked builds only) records kFaultBounds in *fault (if not null) and
// returns false, and the caller skips the access. Always true, and free, in
// ordinary builds.
__device__ __forceinline__ bool in_bounds(const void* p, size_t n, const void* base, size_t bytes,
                                          unsigned int* fault) {
  if (!kBoundsChecks) return true;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(base);
  if (a >= b && a - b <= bytes && n <= bytes - (a - b)) return true;
  if (fault) atomicOr(fault, kFaultBounds);
  return false;
}

// The same for shared memory, against the CTA's dynamic shared memory.
extern __shared__ __align__(16) unsigned char fovea_dyn_smem[];
__device__ __forceinline__ bool smem_in_bounds(const void* p, size_t n, unsigned int* fault) {
  if (!kBoundsChecks) return true;
  unsigned int dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  return in_bounds(p, n, fovea_dyn_smem, dyn, fault);
}

// Sigma and radius of block (bx, by) of a frame: the sigma law at the
// block's nominal centre, or the frame's per-block map (r = ceil(3 sigma) of
// the map value in binary64). A map value above the frame's declared bound
// is clamped to the bound, and a negative or non-finite one to 0; both
// return true (the caller records FOVEA_FAULT_SIGMA_RANGE).
__device__ __forceinline__ bool item_sigma(const FrameDesc& fd, int bx, int by, double& sigma, int& r) {
  bool clamped = false;
  if (fd.smap) {
    sigma = (double)fd.smap[(size_t)by * fd.nbxb + bx];
    if (!(sigma >= 0.0)) {  // negative or NaN
      sigma = 0.0;
      clamped = true;
    } else if (sigma > fd.smap_max) {  // above the bound (or +inf)
      sigma = fd.smap_max;
      clamped = true;
    }
    r = (int)ceil(__dmul_rn(3.0, sigma));
  } else {
    block_sigma(bx, by, fd.B, fd.ox, fd.oy, (double)fd.fx, (double)fd.fy, fd.sigma0, fd.k, sigma, r);
  }
  return clamped;
}

// The work record of tile b of frame f (frame descriptor fd): sigma from the
// frame's law in binary64, its radius, and -1 / (2 sigma^2). Out-of-range
// sigma-map values and radii are clamped and flagged in *err (the sigma
// kernel and the single-launch small-frame kernel both build items here, so
// they agree bit for bit).
__device__ __forceinline__ ItemInfo item_record(const FrameDesc& fd, int f, int b, unsigned int* err) {
  const int tpb = fd.B / fd.T;  // tiles per block side
  const int bx = (b % fd.nbx) / tpb, by = (b / fd.nbx) / tpb;
  double sigma;
  int r;
  if (item_sigma(fd, bx, by, sigma, r)) atomicOr(err, kFaultSigmaRange);
  if (r > kMaxRadius || r < 0) {  // the host refuses such laws and map bounds: never expected
    r = r < 0 ? 0 : kMaxRadius;
    if (!(sigma >= 0.0)) sigma = 0.0;
    atomicOr(err, kFaultSigmaRange);
  }
  ItemInfo inf;
  inf.sigma = (float)sigma;
  inf.neg_half_inv_s2 = sigma > 0.0 ? (float)__ddiv_rn(-0.5, __dmul_rn(sigma, sigma)) : -INFINITY;
  inf.r = r;
  inf.frame = f;
  inf.block = b;
  inf.pad = 0;
  return inf;
}

// Packed two-lane FMA: d = a * b + c on both float lanes (one f32x2
// instruction on sm_100-family GPUs).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
#if defined(FOVEA_SCALAR_FMA)
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#else
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
#endif
}

// Exact uint8 -> float: 2^23 + b has b in its low mantissa bits.
__device__ __forceinline__ float u8_to_f32(unsigned int b) {
  return __int_as_float(0x4B000000u | b) - 8388608.0f;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Block-wide sum with warp shuffles; `red` holds >= 32 floats of shared memory.
__device__ __forceinline__ float block_sum(float v, float* red) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  float s = lane < nw ? red[lane] : 0.0f;
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Normalised taps of one item as (w, w) pairs: U[kTapPad + m] holds the tap
// of offset m - r for m in [0, 2r]; every other entry of [0, len) is zero.
// Eq. 1 sampled at integer offsets, truncated at r = ceil(3 sigma) and
// normalised to unit sum. Sums with warp shuffles.
__device__ __forceinline__ void make_taps(float2* U, int len, int r, float c, float* red) {
  float part = 0.0f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    int d = i - kTapPad - r;
    float w = 0.0f;
    if (d >= -r && d <= r) w = (d == 0) ? 1.0f : expf(c * (float)(d * d));
    U[i].x = w;
    part += w;
  }
  float S = block_sum(part, red);
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    float w = U[i].x / S;
    U[i] = make_float2(w, w);
  }
  __syncthreads();
}

// Number of tap entries a launch needs for radius bound rmax.
__host__ __device__ __forceinline__ int tap_len(int rmax) { return kTapPad + 2 * rmax + 40; }
// Entries of the cumulative-tap table for radius bound rmax.
__host__ __device__ __forceinline__ int cum_len(int rmax) { return 2 * rmax + 4; }

// Exclusive prefix sums of the normalised taps: CU[m] = sum_{m' < m} u[m']
// for m in [0, 2r+1] (u[m] is the tap of offset m - r). Used to fold the
// taps that clamp-to-edge sends onto an edge row or column: the clamped taps
// below tap index M weigh CU[M], and (taps being symmetric) those at or above
// M weigh CU[2r + 1 - M]. One warp scans; the caller synchronises after.
__device__ __forceinline__ void make_cumulative(const float2* U, float* CU, int r) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int n = 2 * r + 1;
  const int seg = (n + 31) >> 5;
  const int b = lane * seg, e = min(n, b + seg);
  float s = 0.0f;
  for (int m = b; m < e; ++m) s += U[kTapPad + m].x;
  float incl = s;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  float run = incl - s;
  for (int m = b; m < e; ++m) {
    CU[m] = run;
    run += U[kTapPad + m].x;
  }
  if (lane == 31) CU[n] = incl;
}

// CU at tap index m, clamped to the table ([0, 2r+1]).
__device__ __forceinline__ float cum_at(const float* CU, int m, int r) {
  return CU[m < 0 ? 0 : (m > 2 * r + 1 ? 2 * r + 1 : m)];
}

// Fire-and-forget fp32 add into global memory (red.global: no value comes
// back, the issuing warp does not wait). atomicAdd through a generic pointer
// with its result unused compiled to a generic atomic that returns the old
// value (one read-back sector per update and a scoreboard wait).
__device__ __forceinline__ void red_add_f32(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;\n" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}

// Four consecutive floats at a 16-byte aligned address, one vector reduction
// (sm_90 and later).
__device__ __forceinline__ void red_add_f32x4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(__cvta_generic_to_global(p)), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

// Packed two-lane add.
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
#if defined(FOVEA_SCALAR_FMA)
  return make_float2(a.x + b.x, a.y + b.y);
#else
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
#endif
}

// Two packed bytes (low half of w) -> one float pair, exactly.
__device__ __forceinline__ float2 u8x2_to_f32(unsigned int w) {
  const unsigned int k = 0x4B000000u;
  return fadd2(make_float2(__uint_as_float(__byte_perm(w, k, 0x7650)), __uint_as_float(__byte_perm(w, k, 0x7651))),
               make_float2(-8388608.0f, -8388608.0f));
}

// Four packed bytes -> two float pairs, exactly (2^23 + b - 2^23).
__device__ __forceinline__ void u8x4_to_f32(unsigned int w, float2& lo, float2& hi) {
  const float2 bias = make_float2(-8388608.0f, -8388608.0f);
  const unsigned int k = 0x4B000000u;
  lo = fadd2(make_float2(__uint_as_float(__byte_perm(w, k, 0x7650)), __uint_as_float(__byte_perm(w, k, 0x7651))), bias);
  hi = fadd2(make_float2(__uint_as_float(__byte_perm(w, k, 0x7652)), __uint_as_float(__byte_perm(w, k, 0x7653))), bias);
}

// 16-byte asynchronous global->shared copy; bytes past `src_bytes` are zero
// filled (src_bytes = 0 writes zeros and reads nothing).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned int s = (unsigned int)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Lets kernel k use `smem` bytes of dynamic shared memory and asks for the
// largest shared-memory carveout, so that as many CTAs fit per SM as the
// shared memory allows (the occupancy calculator and the launch both follow
// the carveout preference).
inline cudaError_t set_smem_attrs(const void* k, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// ------------------------------------------------------------------ launchers
// (defined in sigma.cu, forward.cu, adjoint.cu)

struct FwdConfig {
  int threads;        // threads per CTA of the mma.sync tensor-core kernel: 128, 256 or 512 (others: 256)
  int ctas_per_sm;
  int rows_per_chunk; // RB, multiple of 16
  int tc;             // uint8 frames on the tensor-core kernel
};

cudaError_t launch_sigma_order(const FrameSource& src, const Workspace& ws, int grid_ctas,
                               float* sigma_out, int* radius_out, cudaStream_t s);
// Sigma kernel only, filling per-radius item lists (single-frame blur path).
cudaError_t launch_sigma_buckets(const FrameSource& src, const Workspace& ws, int grid_ctas,
                                 const BucketList& bl, cudaStream_t s);
int sigma_threads();
// fmt_mask: bit 0 = some frame is uint8 HWC, bit 1 = some frame is float32 CHW.
size_t forward_smem_bytes(const FwdConfig& cfg, int rmax, int fmt_mask);
// With bl.list set, the kernel orders its own work from the radius histogram
// and bucket lists (single frame), and it may be launched as a programmatic
// dependent of the sigma kernel (pdl).
// One frame whose blocks all fit in one wave: one CTA per block, sigma
// evaluated in the CTA (no sigma kernel before it). fmt_mask 1 or 2; pdl:
// launch as a programmatic dependent of the stream's previous kernel.
cudaError_t launch_forward_direct(const FrameDesc& fd, long long items, const Workspace& ws, const FwdConfig& cfg,
                                  int rmax, int fmt_mask, cudaStream_t s, bool pdl);
cudaError_t launch_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg,
                           int rmax, int fmt_mask, int grid, cudaStream_t s,
                           const BucketList& bl = BucketList{nullptr, 0, 0}, bool pdl = false);
int forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int fmt_mask);
// Tensor-core variant (uint8 HWC frames, all with C channels).
size_t tc_forward_smem_bytes(const FwdConfig& cfg, int rmax);
int tc_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int C);
// tmap_one: tensor map (128-byte CUtensorMap) of a single frame, read when
// src.one.tma is set; a batch's maps sit in its device buffer (see
// BatchHeader::maps_offset).
cudaError_t launch_tc_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int C,
                              int grid, cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one);
// Pass 1 on tcgen05 (umma_forward.cu): radius bound up to kUmmaMaxRadius
// (its tap strips grow with r), row chunks of 16 or 32 rows.
constexpr int kUmmaMaxRadius = 255;
size_t umma_forward_smem_bytes(const FwdConfig& cfg, int rmax, int C);
int umma_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax, int C);
cudaError_t launch_umma_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int C,
                                int grid, cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one);
// Both passes on tcgen05 (tc05_forward.cu): uint8 RGB frames (C = 3) whose
// rows TMA can load, radius bound up to 192, 16-row chunks.
bool tc05_supports(int rmax, int C);
size_t tc05_forward_smem_bytes(const FwdConfig& cfg, int rmax);
int tc05_forward_max_ctas_per_sm(const FwdConfig& cfg, int rmax);
cudaError_t launch_tc05_forward(const FrameSource& src, const Workspace& ws, const FwdConfig& cfg, int rmax, int grid,
                                cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one);
// Float32 CHW frames on mma.sync (tcf_forward.cu): every frame's rows
// TMA-loadable (W a multiple of 4, 16-byte aligned base), 16-row chunks.
// channels: the launch's common channel count (0: mixed); 2 to 4 with a
// radius bound up to 128 process all planes of a tile in one pass, else
// one plane at a time.
bool tcf_supports(int rmax);
size_t tcf_forward_smem_bytes(int rmax, int channels);
int tcf_forward_max_ctas_per_sm(int rmax, int channels);
cudaError_t launch_tcf_forward(const FrameSource& src, const Workspace& ws, int rmax, int channels, int grid,
                               cudaStream_t s, const BucketList& bl, bool pdl, const void* tmap_one);
size_t adjoint_smem_bytes(int rmax);
cudaError_t launch_adjoint(const FrameSource& src, const Workspace& ws, int rmax, int grid,
                           cudaStream_t s);
// The adjoint on mma.sync (tca_adjoint.cu): per block plane a power-of-two
// scale, fp16 hi + lo splits of the gradient and of Z, the forward kernel's
// tap-pair tables; any radius bound.
size_t tca_adjoint_smem_bytes(int rmax);
int tca_adjoint_max_ctas_per_sm(int rmax);
cudaError_t launch_tca_adjoint(const FrameSource& src, const Workspace& ws, int rmax, int grid, cudaStream_t s);
int adjoint_max_ctas_per_sm(int rmax);

// ------------------------------------------------------------------ per-pixel foveation
// (pixel_forward.cu): every pixel blurred with the sigma of its own centre.

struct PixelParams {
  const void* in;
  void* out;
  int W, H, C, isu8;       // uint8 HWC or float32 CHW
  double fx, fy, sigma0, k;
  int rmax;                // bound on every pixel's radius (the frame's corner pixels)
  int words;               // uint8 rows may be read as aligned 32-bit words
  unsigned int* err;       // fault word: kFaultPixelRadius when a pixel's radius exceeded rmax (never expected)
};

constexpr size_t kPixelSmemBudget = 220 * 1024;
constexpr int kPixelMaxRadius = 255;

// Shared memory of the tensor-core per-pixel kernel (uint8 HWC, 16 x 16
// output tiles): per channel a plane of `pr` pair rows of `pp` bytes, where a
// pair row interleaves two staged rows byte by byte in 8-byte words of 4
// pixels (pp = 32 or 96 mod 128: conflict-free 8-byte fragment loads); then
// the per-pixel tap tables (tp 4-byte entries for each of the 256 pixels)
// and small per-pixel arrays.
struct PixelTcLayout {
  int tp, pp, pr, sw;
  size_t plane_bytes, tile_bytes, tap_bytes, total;
};
__host__ __device__ inline PixelTcLayout pixel_tc_layout(int rmax, int C) {
  PixelTcLayout L;
  // Table of a pixel: offsets 0 .. rmax, then zero entries; the stride is
  // 9 or 23 mod 32 words, which spreads the fragment gathers over the banks.
  L.tp = rmax + 2;
  while (L.tp % 32 != 9 && L.tp % 32 != 23) ++L.tp;
  L.sw = (16 + 2 * rmax + 31) / 32 * 32;           // staged pixels per row (whole 32-pixel groups)
  int pp = 2 * L.sw;
  while (pp % 128 != 32 && pp % 128 != 96) pp += 32;
  L.pp = pp;
  L.pr = (16 + 2 * rmax + 15) / 16 * 8;            // pair rows: whole 16-row k-steps
  L.plane_bytes = (size_t)L.pr * L.pp;
  L.tile_bytes = L.plane_bytes * C;
  L.tap_bytes = (size_t)256 * L.tp * 4;
  L.total = L.tile_bytes + L.tap_bytes + 2 * 256 * 4 + 16;
  return L;
}
bool pixel_tc_fits(int rmax, int C);
// Rows of input the fp32 per-pixel kernel stages at a time (0: rmax too
// large), and its shared memory for that chunk.
int pixel_fp32_rows(int rmax, int C);
size_t pixel_fp32_smem(int rmax, int C, int rb);
cudaError_t launch_pixel_forward(const PixelParams& pp, bool tensor_cores, cudaStream_t s);

// ------------------------------------------------------------------ pyramid (pyramid.cu)
// Levels 1 .. top of a Gaussian pyramid (float32 planes, channel-major);
// level 0 is the frame.
constexpr int kMaxPyramidLevels = 32;
struct PyramidLevels {
  float* ptr[kMaxPyramidLevels];
  int w[kMaxPyramidLevels], h[kMaxPyramidLevels];
  int top;
};
cudaError_t launch_pyramid(const void* in, void* out, int W, int H, int C, int isu8, float fx, float fy,
                           float sigma0, float k, const PyramidLevels& lv, cudaStream_t s);

// ------------------------------------------------------------------ SSIM (ssim.cu)
cudaError_t launch_ssim(const void* a, const void* b, int W, int H, int C, int isu8, float data_range,
                        float* map, double* sum, cudaStream_t s);

}  // namespace fovea
