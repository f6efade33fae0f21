// Sigma-table kernel and work-list ordering.
//
// The paper's host computes a "blur grid" of per-fragment filter indices and
// offsets it to the fixation every frame (Algorithm 1, setup and per-frame
// CPU steps). Here that table is computed on the device every launch: one
// thread per (frame, block) evaluates the sigma law in binary64 (so the radius
// ceil(3 sigma) is reproducible bit for bit), and the items are then ordered
// by radius, largest first, so the persistent blur kernels start the most
// expensive blocks first and finish on the cheap ones.
#include "fovea_internal.cuh"

namespace fovea {

namespace {

constexpr int kSigmaThreads = 128;
constexpr int kOrderThreads = 256;

__device__ __forceinline__ int frame_of_item(const FrameSource& src, long long i) {
  if (!src.hdr) return 0;
  int lo = 0, hi = src.hdr->nframes - 1;
  while (lo < hi) {  // last frame with item0 <= i
    int mid = (lo + hi + 1) >> 1;
    if (src.frames[mid].item0 <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kSigmaThreads) sigma_kernel(FrameSource src, Workspace ws,
                                                              float* sigma_out, int* radius_out, BucketList bl) {
  const long long total = source_total(src);
  unsigned int* hist = ws.counters + CNT_HIST;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = frame_of_item(src, i);
    const FrameDesc fd = load_frame(src, f);
    const int b = (int)(i - fd.item0);        // tile index
    const ItemInfo inf = item_record(fd, f, b, &ws.counters[CNT_ERROR]);
    const int r = inf.r;
    ws.items[i] = inf;
    const int bucket = r < kBuckets ? r : kBuckets - 1;
    const int rank = (int)atomicAdd(&hist[bucket], 1u);
    ws.rank[i] = rank;
    if (bl.list) {  // per-radius item lists for the single-frame blur kernel
      if (bucket < bl.nb && rank < bl.cap) bl.list[(size_t)bucket * bl.cap + rank] = (int)i;
      else atomicOr(&ws.counters[CNT_ERROR], kFaultBuckets);
    }
    if (sigma_out) sigma_out[i] = inf.sigma;
    if (radius_out) radius_out[i] = r;
  }
  // Let a dependent launch (the blur kernel) start its prologue; it waits for
  // this grid's results with griddepcontrol.wait before reading them.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Every CTA rebuilds the bucket start offsets (radius descending) from the
// histogram, then places its items; the last CTA to finish clears the
// histogram and arms the ticket counter for the blur kernel that follows.
__global__ void __launch_bounds__(kOrderThreads) order_kernel(FrameSource src, Workspace ws) {
  __shared__ unsigned int start[kBuckets];
  __shared__ unsigned int wsum[kOrderThreads / 32];
  __shared__ bool last;
  const long long total = source_total(src);
  unsigned int* hist = ws.counters + CNT_HIST;
  constexpr int per = kBuckets / kOrderThreads;  // 4 buckets per thread
  // Thread t owns descending positions [t*per, t*per+per): bucket kBuckets-1-pos.
  unsigned int v[per], run = 0;
  #pragma unroll
  for (int j = 0; j < per; ++j) {
    v[j] = hist[kBuckets - 1 - (threadIdx.x * per + j)];
    run += v[j];
  }
  // exclusive scan of `run` across the CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int incl = run;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned int base = 0;
  for (int w = 0; w < warp; ++w) base += wsum[w];
  unsigned int acc = base + incl - run;
  #pragma unroll
  for (int j = 0; j < per; ++j) {
    start[kBuckets - 1 - (threadIdx.x * per + j)] = acc;
    acc += v[j];
  }
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = ws.items[i].r;
    const int bucket = r < kBuckets ? r : kBuckets - 1;
    const unsigned int pos = start[bucket] + (unsigned int)ws.rank[i];
    if (pos < (unsigned long long)total) ws.order[pos] = (int)i;
    else atomicOr(&ws.counters[CNT_ERROR], kFaultOrder);  // histogram out of step: never write out of range
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&ws.counters[CNT_DONE_ORDER], 1u) == gridDim.x - 1);
  __syncthreads();
  if (last) {
    for (int j = threadIdx.x; j < kBuckets; j += blockDim.x) hist[j] = 0u;
    if (threadIdx.x == 0) {
      ws.counters[CNT_DONE_ORDER] = 0u;
      ws.counters[CNT_TICKET] = 0u;
      ws.counters[CNT_NITEMS] = (unsigned int)total;
    }
  }
}

}  // namespace

cudaError_t launch_sigma_order(const FrameSource& src, const Workspace& ws, int grid_ctas,
                               float* sigma_out, int* radius_out, cudaStream_t s) {
  BucketList none{nullptr, 0, 0};
  sigma_kernel<<<grid_ctas, kSigmaThreads, 0, s>>>(src, ws, sigma_out, radius_out, none);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  order_kernel<<<grid_ctas, kOrderThreads, 0, s>>>(src, ws);
  return cudaGetLastError();
}

cudaError_t launch_sigma_buckets(const FrameSource& src, const Workspace& ws, int grid_ctas,
                                 const BucketList& bl, cudaStream_t s) {
  sigma_kernel<<<grid_ctas, kSigmaThreads, 0, s>>>(src, ws, nullptr, nullptr, bl);
  return cudaGetLastError();
}

int sigma_threads() { return kSigmaThreads; }

}  // namespace fovea
