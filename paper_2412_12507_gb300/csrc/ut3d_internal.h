// ut3d_internal.h — host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ut3d.h"

namespace ut3d {

struct DevOpts;
struct DevCam;
struct BatchDesc;

// Unscented-Transform spread and weights (eq. weights_1/2), computed on the host in FP64.
struct UTWeights {
  float gamma;  // sqrt(3 + lambda)
  float wm0;    // lambda / (3 + lambda)
  float wi;     // 1 / (2 (3 + lambda))
  float wc0;    // lambda / (3 + lambda) + (1 - alpha^2 + beta)
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Debug-build records of the translation units with checks (ut3d_debug.cuh); all zero in a
// release build.
ut_status dbg_read_binsort(uint32_t out[4], bool reset);
ut_status dbg_read_project(uint32_t out[4], bool reset);
ut_status dbg_read_fwd(uint32_t out[4], bool reset);
ut_status dbg_read_bwd(uint32_t out[4], bool reset);
ut_status dbg_read_kbuffer(uint32_t out[4], bool reset);
// Debug build: checks the guard bytes of a binning workspace (records UT_DBG_CANARY).
ut_status dbg_check_bin_guards(const void *ws, int n, int64_t cap, int tiles, int cols, int max_rows,
                               cudaStream_t stream);

// Process-wide count of kernel launches (ut_kernel_launch_count); every launch site adds to it.
void count_launches(int k);

// SM count of the current device (cached per device).
int device_sm_count();

// Projection of every flattened (view, particle) entry of the batch.
// g of n world points (one view's camera), with the rolling-shutter fixed point.
ut_status launch_project_points(const DevCam &cam, const DevOpts &op, const float *points, int n, float *uv,
                                int32_t *valid, cudaStream_t stream);
ut_status launch_project(const BatchDesc &bd, const DevOpts &op, const UTWeights &w, float *mean2d, float *cov2d,
                         float *depth, int16_t *rect, uint32_t *ntiles, cudaStream_t stream);

// Duplicate + sort + ranges over the batch's flattened entries and global tiles.
size_t bin_workspace_bytes(int n, int64_t cap, int tiles, int cols, int max_rows);
// bin_and_sort's argument checks other than the workspace's; *need = the workspace size.
ut_status bin_check_args(int32_t n, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                         const ut_camera *cam, const ut_options *opt, int64_t key_capacity, const uint32_t *vals,
                         const uint32_t *tile_ranges, const int64_t *k_out, DevCam &dc, DevOpts &dop, size_t *need);
// short_sort: a depth sort of at most 128 radix tiles skips its spine scans (fewer launches for
// small scenes); batches pass false so that one launch sequence serves every scene size and the
// serving loop's captured graphs stay updatable.
ut_status launch_bin(const BatchDesc &bd, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                     const DevOpts &op, void *ws, int64_t cap, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                     int64_t *k_out, cudaStream_t stream, bool short_sort);

// Compositing of every global tile of the batch into the views' outputs; sched: scratch of
// tile_sched_bytes(total tiles) for the tile order.
ut_status launch_composite_fwd(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                               const uint32_t *ranges, unsigned long long *stats, void *sched, cudaStream_t stream);

// Backward of the batch into the scenes' gradient outputs (accumulators cleared here).
size_t backward_workspace_bytes(int n, bool kbuffer);  // accumulators, and the k-buffer record table
// Scratch of a tile schedule (forward or backward) for `tiles` tiles.
size_t tile_sched_bytes(int tiles);
ut_status launch_composite_bwd(const BatchDesc &bd, const DevOpts &op, const int16_t *rect, const uint32_t *vals,
                               const uint32_t *ranges, void *sched, cudaStream_t stream);
// The backward of the per-ray k-buffer compositing (accumulators cleared by the caller).
ut_status launch_composite_bwd_kbuffer(const BatchDesc &bd, const DevOpts &op, const int16_t *rect,
                                       const uint32_t *vals, const uint32_t *ranges, cudaStream_t stream);

}  // namespace ut3d
