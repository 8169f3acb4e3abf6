// ut3d_internal.h — host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ut3d.h"

namespace ut3d {

struct DevCam;
struct DevOpts;

// Unscented-Transform spread and weights (eq. weights_1/2), computed on the host in FP64.
struct UTWeights {
  float gamma;  // sqrt(3 + lambda)
  float wm0;    // lambda / (3 + lambda)
  float wi;     // 1 / (2 (3 + lambda))
  float wc0;    // lambda / (3 + lambda) + (1 - alpha^2 + beta)
};

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Process-wide count of kernel launches (ut_kernel_launch_count); every launch site adds to it.
void count_launches(int k);
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// SM count of the current device (cached per device).
int device_sm_count();

ut_status launch_project(int n, const ut_scene &sc, const DevCam &cam, const DevOpts &op, const UTWeights &w,
                         float *mean2d, float *cov2d, float *depth, int16_t *rect, uint32_t *ntiles,
                         cudaStream_t stream);

size_t bin_workspace_bytes(int n, int64_t cap, int tiles);
ut_status launch_bin(int n, const float *depth, const int16_t *rect, const uint32_t *ntiles, const DevOpts &op,
                     int tiles, void *ws, int64_t cap, uint64_t *keys, uint32_t *vals, uint32_t *ranges,
                     int64_t *k_out, cudaStream_t stream);

ut_status launch_composite_fwd(const ut_scene &sc, const DevCam &cam, const DevOpts &op, const int16_t *rect,
                               const uint32_t *vals, const uint32_t *ranges, float *rgb, float *alpha,
                               float *t_final, uint32_t *n_used, unsigned long long *stats, cudaStream_t stream);

size_t backward_workspace_bytes(int n);
ut_status launch_composite_bwd(const ut_scene &sc, const DevCam &cam, const DevOpts &op, const int16_t *rect,
                               const uint32_t *vals, const uint32_t *ranges, const float *rgb, const float *t_final,
                               const uint32_t *n_used, const float *d_rgb, const float *d_alpha, void *ws,
                               float *d_means, float *d_log_scales, float *d_quats, float *d_logits, float *d_sh,
                               cudaStream_t stream);

}  // namespace ut3d
