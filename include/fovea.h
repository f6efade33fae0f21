/*
 * fovea.h -- C ABI of libfovea, a GB300 (sm_103a) implementation of
 * block-wise foveated Gaussian blur ("CUDA-Optimized real-time rendering of a
 * Foveated Visual System", arXiv 2012.08655).
 *
 * The operation (paper Section 2 and Algorithm 1; filter of Eq. 1 and the
 * truncation/normalisation paragraph after it):
 *   - the image is split into square blocks of side B ("fragments");
 *   - block b gets sigma_b = sigma0 + k * e_b, with e_b the Euclidean distance
 *     in pixels from the block centre (B*bx + B/2, B*by + B/2) to the fixation
 *     (fix_x, fix_y); pixel (x, y) covers [x, x+1) x [y, y+1), so the centre
 *     of a W x H frame is (W/2, H/2). The law is evaluated in IEEE binary64
 *     without fused multiply-add; r_b = ceil(3 * sigma_b);
 *   - every output pixel of block b is the normalised Gaussian-weighted sum of
 *     its (2 r_b + 1)^2 clamp-to-edge neighbourhood at sigma_b:
 *        out(x,y,c) = sum_{|i|,|j| <= r_b} w_i w_j / S^2 * in(clamp(x+i), clamp(y+j), c)
 *        w_i = exp(-i^2 / (2 sigma_b^2)),  S = sum_{|i| <= r_b} w_i.
 *     Because all outputs of a block share one sigma, the library computes it
 *     as an in-tile separable pass (vertical, then horizontal) over the halo
 *     tile of the block, which is exact in real arithmetic.
 *   - uint8 data is converted to float on load and coded back as
 *     min(255, max(0, floor(v + 0.5))).
 *
 * Conventions for every entry point below:
 *   - Device pointers are CUDA global-memory pointers on the current device;
 *     host pointers are ordinary (preferably pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls enqueue work on it and return without synchronising;
 *     errors raised while kernels run surface on the next synchronising CUDA
 *     call of the caller, as usual for CUDA.
 *   - A context is not thread-safe and its workspace is reused by every call:
 *     calls on one context must be ordered on one stream (or otherwise
 *     serialised by the caller). Use one context per concurrent stream.
 *   - The caller owns all image and gradient buffers; the library owns its
 *     workspace (per-block sigma/radius tables, work lists, descriptors,
 *     graphs) and never frees the caller's memory.
 *   - Every function returns FOVEA_OK (0) or a negative fovea_status; nothing
 *     throws across the ABI.
 *   - Layouts: FOVEA_U8_HWC is a row-major H x W x C array of bytes (channels
 *     interleaved, the usual frame layout); FOVEA_F32_CHW is a C x H x W
 *     float32 array (the torch layout of one image). Input and output of a
 *     call must not overlap.
 */
#ifndef FOVEA_H_
#define FOVEA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fovea_ctx fovea_ctx;
typedef struct fovea_server fovea_server;

typedef enum {
  FOVEA_OK = 0,
  FOVEA_EINVAL = -1,        /* bad argument (null pointer, aliasing, bad size, non-finite fixation, ...) */
  FOVEA_ENOMEM = -2,        /* device or pinned-host allocation failed */
  FOVEA_ECUDA = -3,         /* a CUDA runtime call failed (see fovea_last_cuda_error) */
  FOVEA_EBUSY = -4,         /* no free slot / memory for the request right now (serving) */
  FOVEA_ETIMEOUT = -5,      /* a bounded wait ran out */
  FOVEA_EUNSUPPORTED = -6   /* valid request outside what this build supports */
} fovea_status;

typedef enum { FOVEA_U8_HWC = 0, FOVEA_F32_CHW = 1 } fovea_format;

typedef enum {
  FOVEA_LAW_LINEAR = 0,         /* sigma_b = sigma0 + k * e_b (pixels) */
  FOVEA_LAW_GEISLER_PERRY = 1,  /* Eqs. 2-6 with the frame corner at e_corner_deg */
  FOVEA_LAW_MAP = 2             /* caller-supplied sigma per block */
} fovea_law_kind;

typedef enum {
  FOVEA_GRID_ANCHORED = 0,  /* block (bx, by) starts at pixel (B bx, B by) */
  FOVEA_GRID_CENTRED = 1    /* the grid is shifted so that a block is centred on the
                               fixation (Algorithm 1), to the nearest pixel */
} fovea_grid_mode;

/* Sigma law of a context (Section 2; Appendix "Choosing the Standard
 * Deviation", Eqs. 2-6). e_b is the distance in pixels from block b's
 * nominal centre to the fixation.
 *  - LINEAR: sigma0 and k finite and >= 0.
 *  - GEISLER_PERRY: the cut-off law with alpha = 0.106, e2 = 2.3, CT0 = 1/64
 *    and eccentricity proportional to pixel distance (Eq. 5), the frame
 *    corner at e_corner_deg degrees (finite, >= 0). It is linear in e_b,
 *    sigma = 1/pi + e_corner / (pi e2 d_corner) e_b (see fovea_gp_law).
 *  - MAP: sigma_map is a device array of nby x nbx floats (row-major, the
 *    grid in force for the frame: see fovea_grid) owned by the caller and
 *    read by every render; sigma_map_max is an upper bound of its values
 *    (it sizes the kernels). A value above sigma_map_max is clamped to it,
 *    and a negative or non-finite value to 0, on the device; the block is
 *    then blurred with the clamped sigma and FOVEA_FAULT_SIGMA_RANGE is
 *    recorded, which the next fovea_check on the context reports as
 *    FOVEA_EINVAL (the render call itself has already returned, as it only
 *    enqueues work). The fixation only places the grid.
 * grid: a fovea_grid_mode. */
typedef struct {
  int kind;                /* fovea_law_kind */
  double sigma0;           /* LINEAR */
  double k;                /* LINEAR */
  double e_corner_deg;     /* GEISLER_PERRY */
  const float* sigma_map;  /* MAP: device pointer */
  double sigma_map_max;    /* MAP */
  int grid;                /* fovea_grid_mode */
} fovea_sigma_law;

/* The Geisler-Perry law of a width x height frame whose corner lies at
 * e_corner_deg degrees, as the linear law's coefficients: *sigma0 = 1/pi,
 * *k = e_corner_deg / ((pi * 2.3) * d_corner), d_corner = half the frame
 * diagonal (binary64, in that order). FOVEA_EINVAL for a bad argument. */
int fovea_gp_law(int width, int height, double e_corner_deg, double* sigma0, double* k);

/* Largest radius r = ceil(3 sigma) a block may reach; larger requests are
 * refused with FOVEA_EUNSUPPORTED before any work is enqueued. */
#define FOVEA_MAX_RADIUS 1023
/* Block side B: 1 <= B <= 32, or a multiple of 32 up to FOVEA_MAX_BLOCK (a
 * block larger than 32 is processed as 32 x 32 tiles sharing its sigma). */
#define FOVEA_MAX_BLOCK 256

/* Create a context for frames of width x height x channels (channels in
 * {1, 2, 3, 4}) in `format`, split into block x block blocks, with sigma law
 * `law`. width = height = 0 creates a batch-only context whose workspace is
 * sized on first use (fovea_render_batch / fovea_backward_batch).
 * Allocates device workspace on the current device (Algorithm 1, the
 * once-per-setup CPU steps: fragment size and blur-grid parameters). */
int fovea_create(int width, int height, int channels, int block, const fovea_sigma_law* law,
                 int format, fovea_ctx** out);

/* Foveate one frame that is resident on the device (Algorithm 1, the
 * per-frame GPU steps: padded tile, horizontal and vertical convolution,
 * write-out). `in_dev` and `out_dev` hold one frame in the context's format
 * and shape; the fixation (fix_x, fix_y) is in pixel coordinates and may lie
 * anywhere, inside or outside the frame (Section 2). The call may be
 * captured into a CUDA graph once an earlier call on this context had a
 * radius bound at least as large (the same fixation, for instance): a call
 * whose bound exceeds every earlier one grows a work-list buffer, which
 * synchronises the device and would end the capture with an error. */
int fovea_render(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                 void* stream);

/* One frame of a batch. Frames of one batch may differ in size, channels,
 * format, fixation, sigma law and grid mode; the block side is the
 * context's. The law is linear (sigma0, k; fovea_gp_law converts the
 * Geisler-Perry law) unless sigma_map is set (a device array of per-block
 * sigma for this frame's grid, bounded by sigma_map_max, as in
 * fovea_sigma_law). */
typedef struct {
  int width, height, channels, format;
  const void* in;     /* device pointer */
  void* out;          /* device pointer */
  float fix_x, fix_y;
  double sigma0, k;
  int grid;                /* fovea_grid_mode */
  const float* sigma_map;  /* or NULL */
  double sigma_map_max;
} fovea_frame;

/* Block grid of a frame of the context's shape for a fixation: *nbx x *nby
 * blocks, block (bx, by) starting at pixel (B bx - *ox, B by - *oy) (clipped
 * to the frame); sigma tables and sigma maps are laid out on this grid. */
int fovea_grid(const fovea_ctx* ctx, float fix_x, float fix_y, int* nbx, int* nby, int* ox, int* oy);

/* Foveate n frames in one launch sequence: a sigma-table kernel over every
 * (frame, block), a cost-ordered work list, and one persistent kernel that
 * pulls (frame, block) items from it, replayed from a CUDA graph. The
 * `frames` array is read before the call returns. */
int fovea_render_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, void* stream);

/* Pre-size the context's batch buffers for batches of up to `max_frames`
 * frames holding up to `max_items` (frame, block) items in all (an item is
 * one block of one frame; a W x H frame has about ceil(W/B) * ceil(H/B)).
 * Without it the buffers grow on demand, at least twofold each time, and a
 * growth recaptures the batch graphs on the calling thread (hundreds of
 * microseconds), which a latency-bound caller such as a serving loop wants to
 * pay up front. Zero leaves that part as it is. Memory: 32 device bytes per
 * item, and per frame 240 bytes of device table plus as much in each of four
 * pinned host staging slots; replaced buffers stay allocated until
 * fovea_destroy. Returns FOVEA_EINVAL for a null context, negative sizes,
 * max_frames above 2^24 or max_items above 2^31 - 1, FOVEA_ECUDA when an
 * allocation fails. Not in the paper: buffer management of the batch path. */
int fovea_reserve(fovea_ctx* ctx, int max_frames, long long max_items);

/* Foveate one frame held in HOST memory (Algorithm 1's transfers of the
 * input from and the output to pinned host memory around the render). The
 * context owns two device staging slots and three internal streams (copy in,
 * kernels, copy out); consecutive calls alternate slots, so the input copy of
 * call i+1 and the output copy of call i-1 overlap the kernels of call i.
 * Ordering: the kernels run after this context's earlier calls on `stream`;
 * `stream` is made to wait for this call's output copy, so synchronising it
 * (or any later work on it) sees out_host complete. The input copy starts as
 * soon as the call is made: in_host must already hold the frame (it is not
 * ordered after other work on `stream`) and must stay unchanged, like
 * out_host, until `stream` is synchronised. Host buffers should be pinned
 * (cudaHostAlloc) for the copies to be asynchronous. Not capturable into a
 * CUDA graph (the internal streams are not part of the capture). */
int fovea_render_host(fovea_ctx* ctx, const void* in_host, void* out_host, float fix_x,
                      float fix_y, void* stream);

/* Adjoint of fovea_render (the transpose of the linear map in -> out) for an
 * FOVEA_F32_CHW context: grad_in = A^T grad_out, with the same fixation.
 * grad_in is overwritten. Not in the paper; it lets the blur sit inside
 * network training. */
int fovea_backward(fovea_ctx* ctx, const float* grad_out_dev, float* grad_in_dev, float fix_x,
                   float fix_y, void* stream);

/* Adjoint of fovea_render_batch for FOVEA_F32_CHW frames: for each frame,
 * `in` is grad_out and `out` (overwritten) is grad_in. */
int fovea_backward_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, void* stream);

/* Per-pixel ("perfect") foveation: the reference the paper scores its
 * block-wise output against (Section 3.1, Fig. 3). Every pixel is blurred
 * with the Gaussian of its own eccentricity: sigma_p = sigma0 + k * |c_p - f|
 * for the pixel centre c_p = (x + 1/2, y + 1/2) (binary64, the block law's
 * operations in the same order), r_p = ceil(3 sigma_p), taps of Eq. 1
 * truncated at r_p and normalised, clamp-to-edge border; this equals the
 * block-wise map with 1 x 1 blocks. Uses the context's frame shape, format
 * and law (linear or Geisler-Perry; a context with a per-block sigma map is
 * refused with FOVEA_EINVAL); its block size and grid mode play no part.
 * uint8 frames run on the tensor cores (unless the context's configuration
 * has tensor_cores = 0) while the shared memory they need fits, else, like
 * float32 frames, on the fp32 kernel. Radii above 255 anywhere in the frame
 * are refused with FOVEA_EUNSUPPORTED. in_dev and out_dev must not overlap. */
int fovea_render_pixelwise(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                           void* stream);

/* Gaussian-pyramid (mipmap) foveation, the earlier approach the paper
 * compares its block-wise blur against (Section 3.2, Fig. 4; appendix on
 * previous foveated rendering), in CUDA: a Burt-Adelson pyramid (5-tap
 * (1,4,6,4,1)/16 kernel, clamp-to-edge, subsampling at the even indices) is
 * built on the device, and every pixel is read at the fractional level
 * L = log4(3 sigma_p^2 + 1) (level l carries a blur of variance
 * (4^l - 1)/3) by bilinear interpolation in levels floor(L) and floor(L)+1,
 * blended by the fraction; sigma_p is the per-pixel law at the pixel centre
 * (computed in fp32 here: L is continuous in sigma). Levels are built up to
 * the largest L the frame needs, in a device workspace the context owns.
 * Same context rules as fovea_render_pixelwise (a per-block map is refused). */
int fovea_render_pyramid(fovea_ctx* ctx, const void* in_dev, void* out_dev, float fix_x, float fix_y,
                         void* stream);

/* SSIM map of two device images of the same shape and format (the quality
 * measure of Section 3.1; Wang, Bovik, Sheikh and Simoncelli 2004): 11 x 11
 * Gaussian window of standard deviation 1.5 normalised to unit sum,
 * clamp-to-edge border, C1 = (0.01 L)^2, C2 = (0.03 L)^2 with L = data_range
 * (<= 0 selects 255 for uint8 and 1 for float32); the value of a pixel is the
 * mean over its channels. Writes the height x width float map to map_dev
 * and/or the sum of the map (one double, zeroed by the call) to sum_dev;
 * either may be NULL, not both. Computed in fp32 (values taken relative to
 * L/2), within about 1e-4 of the binary64 definition. */
int fovea_ssim(int width, int height, int channels, int format, const void* a_dev, const void* b_dev,
               double data_range, float* map_dev, double* sum_dev, void* stream);

/* Per-block sigma (float32, rounded from the binary64 value) and radius for
 * the context's frame at the given fixation, row-major over the block grid
 * (nby x nbx of fovea_grid), written to device arrays. This is the table the
 * render path computes internally (Algorithm 1, "blur grid" with its per-frame
 * offset to the fixation). */
int fovea_sigma_table(fovea_ctx* ctx, float fix_x, float fix_y, float* sigma_dev, int* radius_dev,
                      void* stream);

/* Kernel configuration of the forward path. Chosen by the built-in
 * autotuner (fovea_autotune) or set explicitly (fovea_set_config). */
typedef struct {
  int threads;        /* threads per CTA of the mma.sync tensor-core kernel: 128,
                         256 or 512 (4, 8 or 16 warps; a staged row, and so a
                         column slab of the halo tile, is 32 bytes per warp:
                         112, 240 or 496 bytes of data). The fp32 and tcgen05
                         kernels always run 256. */
  int ctas_per_sm;    /* persistent CTAs per SM (0 = as many as fit) */
  int rows_per_chunk; /* tile rows staged per chunk: 16, 32 or 64 (float32
                         launches of the fp32 kernel keep a two-stage ring and
                         halve it, down to 16, while the ring would fit only
                         one CTA per SM) */
  int tensor_cores;   /* uint8 frames on the tensor cores (fp16 hi/lo split operands,
                         fp32 accumulation): 1 both passes on mma.sync; 2 the
                         vertical pass on tcgen05 with its accumulator in tensor
                         memory (radius bound <= 255 and 16 or 32 rows per chunk,
                         else as 1); 3 both passes on tcgen05, accumulators in
                         tensor memory, one CTA per SM (RGB frames whose rows
                         TMA can load, radius bound <= 192, 16 rows per
                         chunk, else as 1); 0: fp32 FMA kernel.
                         Any non-zero value also runs launches whose frames are
                         all float32 on mma.sync (data and taps split into fp16
                         hi + lo parts, about 2^-21 relative error) when every
                         frame's rows TMA can load (16-byte aligned base, width
                         a multiple of 4), except a single frame whose blocks
                         fit one wave of the fp32 kernel; staged values must
                         satisfy |x| < 32760 = 2^15 - 8, below what fp16
                         rounds to 2^15 (else FOVEA_FAULT_VALUE_RANGE).
                         The adjoint (fovea_backward*) runs on the fp32 kernel,
                         except with 2: on mma.sync with a power-of-two scale
                         per block plane (measured slower; error about 2^-21
                         of the block's largest |gradient|) */
} fovea_config;

/* Copy the context's current configuration into *cfg. FOVEA_EINVAL for a
 * null argument. */
int fovea_get_config(const fovea_ctx* ctx, fovea_config* cfg);

/* Use *cfg for later launches on this context (not in the paper: the paper
 * fixes one CUDA block per fragment). FOVEA_EUNSUPPORTED for threads other
 * than 128, 256 or 512 or rows_per_chunk other than 16, 32 or 64;
 * FOVEA_EINVAL for a null argument, ctas_per_sm outside 0..8 or tensor_cores
 * outside 0..3. A CTA count above what fits is reduced to what fits at
 * launch. Output does not depend on ctas_per_sm or rows_per_chunk, only on
 * the kernel (tensor_cores and, for the mma.sync kernel, threads, which sets
 * where a wide halo tile is cut into column slabs and so the fp32 summation
 * order). After this call the context's batches also run *cfg, instead of a
 * configuration fovea_autotune_batch chose for them. */
int fovea_set_config(fovea_ctx* ctx, const fovea_config* cfg);

/* Time every built-in configuration on the context's own frame shape (a
 * synthetic frame, fixation at the centre, `iters` timed launches each):
 * the kernel (fp32; mma.sync tensor cores with 128, 256 or 512 threads per
 * CTA, i.e. staged tiles of rows_per_chunk rows x 112, 240 or 496 bytes;
 * tcgen05 vertical pass) and rows per chunk, then CTAs per SM for the
 * fastest. Keeps the fastest, and caches it under the device
 * name, SM count, shape, format, block side and radius bucket. Synchronises
 * the device. If `cache_path` is not NULL the cache is read from and written
 * to that JSON file. */
int fovea_autotune(fovea_ctx* ctx, int iters, const char* cache_path);

/* The same search on the caller's own batch: every candidate renders
 * `frames` (their outputs are overwritten with the usual results) with
 * `iters` timed launches after one untimed one, and the fastest is cached
 * under the batch's key: device, SM count, block side, the formats and
 * channel count of the frames, their largest block radius (rounded up to a
 * multiple of 64) and the numbers of blocks and frames (rounded down to
 * powers of two). Later fovea_render_batch calls on any context of the
 * process run batches with the same key with that configuration, unless
 * fovea_set_config fixed the context's own. An existing entry for the key is
 * kept (no timing). Synchronises the device first. *chosen (if not NULL)
 * receives the configuration. FOVEA_EINVAL for a null or empty batch or
 * iters <= 0; the statuses of fovea_render_batch for a bad frame. Not in the
 * paper, which fixes one CUDA block per fragment. */
int fovea_autotune_batch(fovea_ctx* ctx, const fovea_frame* frames, int n, int iters, const char* cache_path,
                         fovea_config* chosen);

/* Measurement hook: when both are non-NULL, every later render call on this
 * context records `ev_start` (a cudaEvent_t) immediately before launching its
 * persistent blur kernel and `ev_stop` immediately after, on the call's
 * stream, so a caller can time that kernel alone. NULL, NULL turns it off. */
int fovea_set_kernel_events(fovea_ctx* ctx, void* ev_start, void* ev_stop);

/* Synchronise the device, then free everything the context owns (workspace,
 * graphs, staging buffers, internal streams). The caller's buffers are not
 * touched. NULL is a no-op. */
void fovea_destroy(fovea_ctx* ctx);

/* Most blocks a frame may have for fovea_render_noalloc (e.g. 3840x2160 at
 * B = 32 is 8160 blocks). */
#define FOVEA_NOALLOC_MAX_BLOCKS 16384

/* Foveate one device-resident frame without allocating any memory. The paper
 * has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc -- code whose device memory is owned by a host framework or a
 * server that has reserved it up front, or that must not allocate while it
 * drives the GPU -- and for whom fovea_create's workspace is not an option.
 * Arguments are those of fovea_create and fovea_render combined, with the
 * linear sigma law on the anchored grid and a block side of 1 to 32 (one work
 * item per block; larger blocks are refused with FOVEA_EUNSUPPORTED); the
 * caller still owns and passes the input and output buffers. All working
 * memory (per-block sigma/radius records, the radius-ordered work list,
 * counters; about 0.5 MB) is one fixed-size array inside the library image,
 * held by every GPU that loads the library until the process exits. No
 * cudaMalloc, cudaFree or allocating library routine is called. Blocks are
 * rendered by the fp32 CUDA-core kernel (the same outputs as a context
 * configured with tensor_cores = 0).
 *   - Frames with more than FOVEA_NOALLOC_MAX_BLOCKS blocks are refused with
 *     FOVEA_EUNSUPPORTED before any work is enqueued.
 *   - The first call on a device looks up the array's device address (a
 *     one-time set-up per device, with that device current; repeated only
 *     if the device's CUDA context was replaced, e.g. by cudaDeviceReset);
 *     make that first call before any stream capture.
 *   - Every call uses the same array, which keeps the last call's contents;
 *     each call clears the counters that must start at zero, its fault word
 *     included, on its stream. Calls whose GPU work overlaps (other streams,
 *     other host threads) race and must be serialised by the caller. */
int fovea_render_noalloc(const void* in_dev, void* out_dev, int width, int height, int channels,
                         int format, int block, double sigma0, double k, float fix_x, float fix_y,
                         void* stream);

/* ------------------------------------------------------------ device faults
 * Conditions the kernels detect while they run. A render or adjoint call only
 * enqueues work, so it cannot return them; each kernel ORs a bit into a fault
 * word of the context instead, and fovea_check turns that word into a
 * negative status like every other failure, and clears it. Unless
 * stated otherwise the item concerned (one block of one frame) is skipped and
 * its output pixels are left as they were.
 */
#define FOVEA_FAULT_SIGMA_RANGE  0x01u /* a per-block sigma map value was above sigma_map_max, negative or
                                          not finite: clamped (to sigma_map_max, or 0) and blurred with that */
#define FOVEA_FAULT_RADIUS_BOUND 0x02u /* forward: a block's radius exceeded the bound its launch was sized
                                          for (internal: the host bound covers every clamped sigma) */
#define FOVEA_FAULT_ADJ_BOUND    0x04u /* adjoint: the same */
#define FOVEA_FAULT_ORDER        0x08u /* internal: the radius histogram and the work list were out of step */
#define FOVEA_FAULT_WORKLIST     0x10u /* internal: a work ticket named no item */
#define FOVEA_FAULT_BUCKETS      0x20u /* internal: a per-radius item list overflowed */
#define FOVEA_FAULT_WAIT         0x40u /* a bounded wait on the device (a TMA row chunk, a tensor-core
                                          commit) ran out: the item was abandoned */
#define FOVEA_FAULT_PIXEL_RADIUS 0x80u /* per-pixel path: a pixel's radius exceeded the launch's bound
                                          (internal); the pixel is written unblurred */
#define FOVEA_FAULT_BOUNDS      0x100u /* bounds-checked builds (-DFOVEA_BOUNDS) only: a store fell outside
                                          the buffer it belongs to and was skipped (internal) */
#define FOVEA_FAULT_VALUE_RANGE 0x200u /* float32 frames on the tensor cores: a staged value was not finite
                                          or |x| >= 32760 (fp16 rounds it to 2^15 or more),
                                          beyond the fp16 hi + lo split; the
                                          blocks it fed are not trustworthy (caller's data) */

/* Waits for `stream` (a cudaStream_t; the stream the context's calls were
 * ordered on), then reads and clears the context's device fault word. Stores
 * the word in *faults when faults is not NULL. Returns FOVEA_OK when no bit
 * was set; otherwise FOVEA_ETIMEOUT if FOVEA_FAULT_WAIT is set, else
 * FOVEA_ECUDA if an internal bit (ORDER, WORKLIST, BUCKETS, PIXEL_RADIUS,
 * RADIUS_BOUND, ADJ_BOUND, BOUNDS) is set, else FOVEA_EINVAL (the caller's sigma map
 * was out of its declared range). FOVEA_ECUDA also when the stream or the
 * copy fails. The word accumulates over every call made since the last
 * check, so one check after a sequence of calls covers all of them. Not in
 * the paper: the error contract of the library. */
int fovea_check(fovea_ctx* ctx, void* stream, unsigned int* faults);

/* Non-blocking form of fovea_check for callers that must not wait (a
 * training step, a render loop). Enqueues on `stream` a copy of the
 * context's fault word into pinned host memory the context owns and returns
 * FOVEA_OK without waiting; a later call looks at that copy once it has
 * landed, and if it holds a fault, finishes like fovea_check (waits for
 * `stream`, reads and clears the word) and returns its status. The fault word
 * is only cleared by fovea_check, so a fault is reported at the latest by the
 * second fovea_check_async after the faulting work and the copy behind it
 * have completed, or by the next fovea_check. */
int fovea_check_async(fovea_ctx* ctx, void* stream, unsigned int* faults);

/* fovea_check for fovea_render_noalloc: waits for `stream`, then reads the
 * device fault word of the latest fovea_render_noalloc call on the current
 * device (each call clears it) into *faults (if not NULL) and returns the
 * status fovea_check would. Allocates nothing. The paper has no
 * counterpart. */
int fovea_noalloc_check(void* stream, unsigned int* faults);

/* A static, human-readable description of a fovea_status value ("unknown
 * status" for any other value); never NULL. */
const char* fovea_strerror(int status);

/* The cudaError_t of the last failed CUDA call in this thread (0 if none). */
int fovea_last_cuda_error(void);

#define FOVEA_BUILD_BOUNDS 1
/* Build flags of the loaded library: FOVEA_BUILD_BOUNDS when it is the
 * bounds-checked build (compiled with FOVEA_BOUNDS: every kernel store checks
 * its address, skips one outside its buffer and records FOVEA_FAULT_BOUNDS in
 * the context's fault word), 0 for the regular build. */
int fovea_build_flags(void);

/* Diagnostic (no counterpart in the paper): measures the current GPU's FP32
 * FMA throughput, the roof of the blur kernels' arithmetic. Runs a kernel of
 * independent packed two-lane FMA chains (fma.rn.f32x2) on every SM of the
 * current device, on the given stream, for a fraction of a second, timed with
 * CUDA events, and synchronises that stream. On success stores the measured
 * rate in FMA lane-operations per second (one f32x2 FMA counts 2) in
 * *fma_per_s. The kernel writes one float per thread into a device buffer it
 * allocates and frees itself. FOVEA_EINVAL for a null pointer, FOVEA_ECUDA /
 * FOVEA_ENOMEM on failure. */
int fovea_measure_fma_rate(double* fma_per_s, void* stream);

/* ------------------------------------------------------------------ serving
 * Continuous-batching request loop (not in the paper; it serves frames of
 * different resolutions and fixations as they arrive). Frames start and end
 * in host memory. Requests are admitted while device memory for their input
 * and output is available within `device_budget_bytes`, and their inputs
 * copy in on a copy stream at once. Whenever no batch is rendering, the
 * worker renders up to max_batch admitted requests, one batch per (format,
 * channel count) (same kernels as fovea_render_batch), on a compute stream
 * that waits on the device for their input copies; requests admitted while a
 * batch renders gather into the next one. Results are copied back to the
 * caller's host buffer.
 */
typedef struct {
  size_t device_budget_bytes;  /* cap on device memory used for request buffers */
  int max_batch;               /* most frames rendered in one batch */
  int block;                   /* block side B */
  int max_inflight;            /* most admitted-but-unfinished requests */
} fovea_server_config;

typedef struct {
  double arrival_us;   /* caller-supplied arrival time (steady clock, microseconds) */
  double admit_us;     /* admission (device memory reserved) */
  double start_us;     /* host time its batch was launched */
  double done_us;      /* host time its output copy was seen complete */
  int batch_size;      /* frames in the batch it was rendered in */
  int status;          /* FOVEA_OK or an error */
} fovea_request_times;

/* Start a serving loop on the current device: allocates the device arena
 * (device_budget_bytes), three streams and a batch context whose buffers are
 * reserved for the largest batch the arena holds, and starts the worker
 * thread. *out is set on success (NULL otherwise). FOVEA_EINVAL for a null
 * argument, a budget below 512 bytes, or max_batch, max_inflight or block
 * <= 0; FOVEA_ENOMEM when the arena or a stream cannot be created; the
 * status of fovea_create or fovea_reserve otherwise. Free with
 * fovea_server_destroy. */
int fovea_server_create(const fovea_server_config* cfg, fovea_server** out);

/* Submit one frame. `in_host` / `out_host` stay owned by the caller and must
 * stay valid until the request completes. Returns a request id >= 0, or a
 * negative status (FOVEA_EBUSY when the request can never fit the budget).
 * Admission waits, inside the worker, for memory to free up. */
long long fovea_server_submit(fovea_server* srv, const fovea_frame* frame_host,
                              double arrival_us);

/* Wait up to timeout_ms for request `id` to finish (0 = poll). Returns
 * FOVEA_OK when done (times filled in), FOVEA_ETIMEOUT otherwise. */
int fovea_server_wait(fovea_server* srv, long long id, int timeout_ms, fovea_request_times* times);

/* Microseconds on the steady clock the server uses for its timestamps. */
double fovea_server_now_us(void);

/* Drain all requests and stop the worker. */
void fovea_server_destroy(fovea_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* FOVEA_H_ */
