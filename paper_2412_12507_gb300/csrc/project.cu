// project.cu — Unscented-Transform projection of every particle (Sec. 4.1; Algorithms 1-2).
//
// One thread per particle, one warp per 32 consecutive particles.  The warp loads its
// 32 twelve-byte records (means, log-scales) as 24 aligned float4 through shared
// memory and writes the twelve-byte covariance records back the same way, so every
// global access of the kernel is a coalesced vector access.  The 7 sigma points are
// projected through the camera (with the rolling-shutter time fixed point), and the
// weighted mean / covariance, depth, opacity-tightened rectangle and tile count are
// written out.
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {

namespace {

constexpr int kWarps = 8;

__global__ void __launch_bounds__(kWarps * 32) k_project(int n, const float *__restrict__ means,
                                                         const float *__restrict__ log_scales,
                                                         const float4 *__restrict__ quats,
                                                         const float *__restrict__ logits, DevCam cam, DevOpts op,
                                                         UTWeights w, int vec_ok, float2 *__restrict__ mean2d,
                                                         float *__restrict__ cov2d, float *__restrict__ depth,
                                                         short4 *__restrict__ rect, uint32_t *__restrict__ ntiles) {
  __shared__ float4 s_stage[kWarps][24];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = (blockIdx.x * kWarps + warp) * 32;
  if (base >= n) return;  // warp-uniform
  const int i = base + lane;
  const bool full = vec_ok && (base + 32 <= n);
  const bool live = i < n;
  float *st = reinterpret_cast<float *>(s_stage[warp]);

  float3 mu = make_float3(0.f, 0.f, 0.f), ls = make_float3(0.f, 0.f, 0.f);
  if (full) {
    if (lane < 24) s_stage[warp][lane] = reinterpret_cast<const float4 *>(means + 3 * (size_t)base)[lane];
    __syncwarp();
    mu = make_float3(st[3 * lane], st[3 * lane + 1], st[3 * lane + 2]);
    __syncwarp();
    if (lane < 24) s_stage[warp][lane] = reinterpret_cast<const float4 *>(log_scales + 3 * (size_t)base)[lane];
    __syncwarp();
    ls = make_float3(st[3 * lane], st[3 * lane + 1], st[3 * lane + 2]);
    __syncwarp();
  } else if (live) {
    mu = make_float3(means[3 * i], means[3 * i + 1], means[3 * i + 2]);
    ls = make_float3(log_scales[3 * i], log_scales[3 * i + 1], log_scales[3 * i + 2]);
  }
  float4 q4 = live ? quats[i] : make_float4(1.f, 0.f, 0.f, 0.f);
  float logit = live ? logits[i] : 0.f;

  Particle p;
  bool ok = live && activate(mu, ls, q4, logit, p);
  ok = ok && (p.sigma >= op.alpha_min);

  // sigma points in start-pose camera rotation: y_0 = R0 mu, y_(1+k) / y_(4+k) = y_0 +- gamma s_k R0 R[:,k]
  float2 v[7];
  float t_mu = 0.f;
  float3 y0 = mat3_mul(cam.R0, mu);
  ok = ok & project_world(cam, op.rs_iters, y0, v[0], t_mu);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float g = w.gamma * p.s[k];
    float3 col = make_float3(g * p.R[k], g * p.R[3 + k], g * p.R[6 + k]);
    float3 dy = mat3_mul(cam.R0, col);
    float tt;
    ok = ok & project_world(cam, op.rs_iters, make_float3(y0.x + dy.x, y0.y + dy.y, y0.z + dy.z), v[1 + k], tt);
    ok = ok & project_world(cam, op.rs_iters, make_float3(y0.x - dy.x, y0.y - dy.y, y0.z - dy.z), v[4 + k], tt);
  }
  // eq. 2d_conic_1 / 2d_conic_2
  float2 vm = make_float2(w.wm0 * v[0].x, w.wm0 * v[0].y);
#pragma unroll
  for (int j = 1; j < 7; ++j) {
    vm.x = fmaf(w.wi, v[j].x, vm.x);
    vm.y = fmaf(w.wi, v[j].y, vm.y);
  }
  float cxx = 0.f, cxy = 0.f, cyy = 0.f;
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    float ww = j == 0 ? w.wc0 : w.wi;
    float dx = v[j].x - vm.x, dy = v[j].y - vm.y;
    cxx = fmaf(ww * dx, dx, cxx);
    cxy = fmaf(ww * dx, dy, cxy);
    cyy = fmaf(ww * dy, dy, cyy);
  }
  float3 xc = cam_point_at(cam, y0, t_mu);
  float dep = sqrtf(fmaf(xc.x, xc.x, fmaf(xc.y, xc.y, xc.z * xc.z)));

  // opacity-tightened extent (Algorithm 1) and pixel rectangle
  float kx = fminf(op.extent_sigma, sqrtf(2.f * logf(p.sigma / op.alpha_min)));
  float hx = kx * sqrtf(cxx), hy = kx * sqrtf(cyy);
  ok = ok && isfinite(vm.x) && isfinite(vm.y) && isfinite(hx) && isfinite(hy);
  float fx0 = fmaxf(ceilf(vm.x - hx - 0.5f), 0.f), fx1 = fminf(floorf(vm.x + hx - 0.5f), (float)(cam.W - 1));
  float fy0 = fmaxf(ceilf(vm.y - hy - 0.5f), 0.f), fy1 = fminf(floorf(vm.y + hy - 0.5f), (float)(cam.H - 1));
  ok = ok && (fx0 <= fx1) && (fy0 <= fy1);

  short4 r = make_short4(0, 0, -1, -1);
  uint32_t nt = 0;
  if (ok) {
    int x0 = (int)fx0, x1 = (int)fx1, y0i = (int)fy0, y1 = (int)fy1;
    r = make_short4((short)x0, (short)y0i, (short)x1, (short)y1);
    nt = (uint32_t)((x1 / op.tile_w - x0 / op.tile_w + 1) * (y1 / op.tile_h - y0i / op.tile_h + 1));
  } else {
    vm = make_float2(0.f, 0.f);
    cxx = cxy = cyy = 0.f;
    dep = 0.f;
  }
  if (full) {
    st[3 * lane] = cxx;
    st[3 * lane + 1] = cxy;
    st[3 * lane + 2] = cyy;
    __syncwarp();
    if (lane < 24) reinterpret_cast<float4 *>(cov2d + 3 * (size_t)base)[lane] = s_stage[warp][lane];
  } else if (live) {
    cov2d[3 * i] = cxx;
    cov2d[3 * i + 1] = cxy;
    cov2d[3 * i + 2] = cyy;
  }
  if (live) {
    mean2d[i] = vm;
    depth[i] = dep;
    rect[i] = r;
    ntiles[i] = nt;
  }
}

}  // namespace

ut_status launch_project(int n, const ut_scene &sc, const DevCam &cam, const DevOpts &op, const UTWeights &w,
                         float *mean2d, float *cov2d, float *depth, int16_t *rect, uint32_t *ntiles,
                         cudaStream_t stream) {
  if (n == 0) return UT_OK;
  int vec_ok = aligned16(sc.means) && aligned16(sc.log_scales) && aligned16(cov2d);
  int blocks = (n + kWarps * 32 - 1) / (kWarps * 32);
  k_project<<<blocks, kWarps * 32, 0, stream>>>(n, sc.means, sc.log_scales, reinterpret_cast<const float4 *>(sc.quats),
                                                sc.opacity_logits, cam, op, w, vec_ok,
                                                reinterpret_cast<float2 *>(mean2d), cov2d, depth,
                                                reinterpret_cast<short4 *>(rect), ntiles);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

}  // namespace ut3d
