// Host-side helpers shared by the libfovea translation units (not exported).
#pragma once

#include <stddef.h>

#include <nvtx3/nvToolsExt.h>

#include "fovea.h"

namespace fovea {

// One NVTX range over a scope (the library's host phases as named ranges on
// a profiler's timeline; a push and a pop of a few nanoseconds when no tool
// is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Sigma law and block grid of one frame as the host sees it: the linear law
// (sigma0, k), or a per-block device map with an upper bound of its values;
// and a fovea_grid_mode.
struct FrameLaw {
  double sigma0 = 0.0, k = 0.0;
  const float* smap = nullptr;
  double smap_max = 0.0;
  int grid = FOVEA_GRID_ANCHORED;
};
// Grid origin offset along one axis (0, or the offset that centres a block
// on fixation coordinate f: (floor(B/2) - floor(f + 1/2)) mod B).
int grid_origin(float f, int B, int grid);
// Blocks along each axis for origin offsets (ox, oy).
void grid_dims(int W, int H, int B, int ox, int oy, int* nbx, int* nby);
// Largest radius ceil(3 sigma) over the block grid of a W x H frame
// (computed exactly as the device does for the farthest block; for a map,
// ceil(3 smap_max)).
int radius_bound(int W, int H, int B, float fx, float fy, const FrameLaw& law);
// FOVEA_OK or the status a frame with these parameters is refused with.
int check_frame(int W, int H, int C, int fmt, int B, const FrameLaw& law, float fx, float fy);
size_t frame_bytes(int W, int H, int C, int fmt);
int ctx_shape(const fovea_ctx* ctx, int* W, int* H, int* C, int* fmt, int* B);
int ctx_device_info(const fovea_ctx* ctx, int* device, int* num_sms);
// A configuration's validity (the fovea_set_config statuses), and setting it
// on a context without marking it as the caller's choice (the autotuner).
int check_config(const fovea_config* cfg);
int apply_config(fovea_ctx* ctx, const fovea_config* cfg);
// What the batch autotuner keys its choice on: the formats and channel
// counts of the frames (fmt_mask bit 0 uint8, bit 1 float32; channels 0 when
// mixed), the largest block radius, the number of blocks and of frames.
struct BatchSummary {
  int fmt_mask, channels, rmax;
  long long blocks;
  int frames;
};
int summarize_batch(const fovea_ctx* ctx, const fovea_frame* frames, int n, BatchSummary* out);
// The configuration fovea_autotune_batch chose for batches like bs on this
// context's device (false if none); defined with the autotuner.
bool lookup_batch_config(const fovea_ctx* ctx, const BatchSummary& bs, fovea_config* cfg);
// fovea_render_batch with a given configuration (the autotuner's timing runs).
int render_batch_with(fovea_ctx* ctx, const fovea_frame* frames, int n, const fovea_config* cfg, void* stream);
// Device address of the context's fault word (FOVEA_FAULT_* bits).
int ctx_fault_word(const fovea_ctx* ctx, unsigned int** word);
// Radius bound of a sized context with the fixation at the frame centre (the
// autotuner's timing frame); 0 for a batch-only context.
int ctx_centre_radius_bound(const fovea_ctx* ctx);
// Bytes of one tensor map (CUtensorMap) and the alignment it needs.
constexpr size_t kTensorMapBytes = 128;
constexpr size_t kTensorMapAlign = 64;
// Encodes the tensor map the tensor-core kernel loads a uint8 HWC frame's
// rows with (2D: W*C bytes x H rows, boxes of 128 bytes x `rows`, 128-byte
// swizzle, zero fill outside the frame) into map (kTensorMapBytes, aligned to
// kTensorMapAlign). Returns false, leaving map zeroed, when the frame's base
// address or row pitch is not a multiple of 16 bytes or the driver refuses.
bool make_u8_tensor_map(void* map, const void* base, int W, int H, int C, int rows);
// The same for a float32 CHW frame: a 3D map (x, y, plane), boxes of 32
// elements x `rows` rows of one plane (16-byte aligned base, W a multiple of 4).
bool make_f32_tensor_map(void* map, const void* base, int W, int H, int C, int rows);
// Status a device fault word maps to (see fovea_check): FOVEA_OK for 0,
// FOVEA_ETIMEOUT when a wait ran out, FOVEA_ECUDA for an internal fault,
// FOVEA_EINVAL when only a sigma-map value was out of range.
int fault_status(unsigned int word);
// Records a failed cudaError_t for fovea_last_cuda_error and returns the
// status it maps to (FOVEA_ENOMEM for an allocation failure, else FOVEA_ECUDA).
int record_cuda_failure(int cuda_error);

}  // namespace fovea

// Applies a configuration the autotuner has already chosen for this
// context's device and shape, if any (defined in tune.cpp).
void fovea_apply_cached_config(fovea_ctx* ctx);
