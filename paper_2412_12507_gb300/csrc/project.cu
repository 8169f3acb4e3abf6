// project.cu — Unscented-Transform projection of every particle (Sec. 4.1; Algorithms 1-2),
// or, as an A/B baseline, the first-order EWA projection of 3DGS (eq. ewa_splatting).
//
// One thread per (view, particle) entry of the flattened batch, one warp per 32
// consecutive entries.  When a warp's 32 entries belong to one view, the warp loads its 32
// twelve-byte records (means, log-scales) as 24 aligned float4 through shared memory and
// writes the twelve-byte covariance records back the same way, so the global accesses are
// coalesced vector accesses.  The 7 sigma points are projected through the view's camera
// (with the rolling-shutter time fixed point), and the weighted mean / covariance, depth,
// opacity-tightened rectangle and tile count are written out.
#include "ut3d_debug.cuh"
#include "ut3d_device.cuh"
#include "ut3d_internal.h"

namespace ut3d {

namespace {

constexpr int kWarps = 8;

// The camera map of the kernel: CAM = 2 model + rolling shutter when every view of the launch
// shares them (a specialised kernel with no camera branches), or -1 for a batch that mixes them
// (the runtime dispatch of project_world / cam_point_at).
template <int CAM>
__device__ __forceinline__ bool proj_world(const DevCam &c, int rs_iters, float3 y, float2 &uv, float &t) {
  if constexpr (CAM < 0) return project_world(c, rs_iters, y, uv, t);
  else return project_world_t<CAM / 2, (CAM & 1) != 0>(c, rs_iters, y, uv, t);
}

template <int CAM>
__device__ __forceinline__ float3 point_at(const DevCam &c, float3 y, float t) {
  if constexpr (CAM < 0) return cam_point_at(c, y, t);
  else return cam_point_at_t<(CAM & 1) != 0>(c, y, t);
}

// EWA: the first-order projection of 3DGS (eq. ewa_splatting) instead of the UT, as an A/B
// baseline: the mean projects through g and the covariance through the Jacobian of g at the
// camera-space mean (under a rolling shutter, at the pose of the mean's own shutter time).
template <bool EWA, int CAM>
__global__ void __launch_bounds__(kWarps * 32, 4) k_project(const __grid_constant__ BatchDesc bd, DevOpts op, UTWeights w,
                                                         float2 *__restrict__ mean2d, float *__restrict__ cov2d,
                                                         float *__restrict__ depth, short4 *__restrict__ rect,
                                                         uint32_t *__restrict__ ntiles) {
  __shared__ float4 s_stage[kWarps][24];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = bd.total_particles;
  const int base = (blockIdx.x * kWarps + warp) * 32;
  if (base >= n) return;  // warp-uniform
  const int g = base + lane;
  const bool live = g < n;
  const int vi = view_of_particle(bd, live ? g : n - 1);
  const DevView &view = bd.v[vi];
  const DevScene &sc = bd.s[view.scene];
  const int i = (live ? g : n - 1) - view.part_off;
  // vector path: all 32 entries in this view, 16-byte aligned records
  const int v_last = __shfl_sync(0xffffffffu, vi, 31);
  const int v_first = __shfl_sync(0xffffffffu, vi, 0);
  const int i0 = __shfl_sync(0xffffffffu, i, 0);
  const bool full = (base + 32 <= n) && v_first == v_last && ((i0 & 3) == 0) &&
                    ((reinterpret_cast<uintptr_t>(sc.means) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(sc.log_scales) & 15) == 0) &&
                    ((reinterpret_cast<uintptr_t>(cov2d) & 15) == 0);
  float *st = reinterpret_cast<float *>(s_stage[warp]);

  float3 mu, ls;
  if (full) {
    if (lane < 24) s_stage[warp][lane] = reinterpret_cast<const float4 *>(sc.means + 3 * (size_t)i0)[lane];
    __syncwarp();
    mu = make_float3(st[3 * lane], st[3 * lane + 1], st[3 * lane + 2]);
    __syncwarp();
    if (lane < 24) s_stage[warp][lane] = reinterpret_cast<const float4 *>(sc.log_scales + 3 * (size_t)i0)[lane];
    __syncwarp();
    ls = make_float3(st[3 * lane], st[3 * lane + 1], st[3 * lane + 2]);
    __syncwarp();
  } else {
    mu = make_float3(sc.means[3 * i], sc.means[3 * i + 1], sc.means[3 * i + 2]);
    ls = make_float3(sc.log_scales[3 * i], sc.log_scales[3 * i + 1], sc.log_scales[3 * i + 2]);
  }
  const float4 q4 = sc.quats[i];
  const float logit = sc.logits[i];
  const DevCam &cam = view.cam;  // read from the kernel parameter (no register copy)

  Particle p;
  bool ok = live && activate(mu, ls, q4, logit, p);
  ok = ok && (p.sigma >= op.alpha_min);

  float2 vm;
  float t_mu = 0.f;
  float3 y0 = mat3_mul(cam.R0, mu);
  float cxx = 0.f, cxy = 0.f, cyy = 0.f;
  if (EWA) {
    ok = ok & project_world(cam, op.rs_iters, y0, vm, t_mu);
    float3 ju, jv;
    cam_jacobian(cam, cam_point_at(cam, y0, t_mu), ju, jv);
    // Sigma' = A A^T with column k of A = J W (s_k R[:,k]), W the pose at t_mu
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float3 col = mat3_mul(cam.R0, make_float3(p.s[k] * p.R[k], p.s[k] * p.R[3 + k], p.s[k] * p.R[6 + k]));
      if (cam.rs) col = rotate_axis(cam.ax, col, t_mu * cam.phi);
      const float au = dot3(ju, col), av = dot3(jv, col);
      cxx = fmaf(au, au, cxx);
      cxy = fmaf(au, av, cxy);
      cyy = fmaf(av, av, cyy);
    }
  } else {
    // sigma points in start-pose camera rotation: y_0 = R0 mu, y = y_0 +- gamma s_k R0 R[:,k].
    // The six off-centre points go through one (not unrolled) loop, each projection taken
    // relative to the centre's v_0 (d_j = v_j - v_0), which keeps the moments free of
    // cancellation: eq. 2d_conic_1 gives v_mu = v_0 + wi sum d_j (the mean weights sum to one)
    // and eq. 2d_conic_2 gives Sigma' = wi sum d_j d_j^T + (W - 2) dm dm^T with dm = wi sum d_j
    // and W = wc0 + 6 wi the sum of the covariance weights.
    float2 v0;
    ok = ok & proj_world<CAM>(cam, op.rs_iters, y0, v0, t_mu);
    float3 col[3];  // gamma s_k R0 R[:,k]
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float gs = w.gamma * p.s[k];
      col[k] = mat3_mul(cam.R0, make_float3(gs * p.R[k], gs * p.R[3 + k], gs * p.R[6 + k]));
    }
    float sx = 0.f, sy = 0.f, pxx = 0.f, pxy = 0.f, pyy = 0.f;
#pragma unroll 1
    for (int j = 0; j < 6; ++j) {
      const int k = j < 3 ? j : j - 3;
      const float3 c3 = k == 0 ? col[0] : (k == 1 ? col[1] : col[2]);  // selects, no local memory
      const float3 dy = j < 3 ? c3 : make_float3(-c3.x, -c3.y, -c3.z);
      float2 v;
      float tt;
      ok = ok & proj_world<CAM>(cam, op.rs_iters, make_float3(y0.x + dy.x, y0.y + dy.y, y0.z + dy.z), v, tt);
      const float dx = v.x - v0.x, dz = v.y - v0.y;
      sx += dx;
      sy += dz;
      pxx = fmaf(dx, dx, pxx);
      pxy = fmaf(dx, dz, pxy);
      pyy = fmaf(dz, dz, pyy);
    }
    const float dmx = w.wi * sx, dmy = w.wi * sy;
    const float c = w.wc0 + 6.f * w.wi - 2.f;
    vm = make_float2(v0.x + dmx, v0.y + dmy);
    cxx = fmaf(w.wi, pxx, c * dmx * dmx);
    cxy = fmaf(w.wi, pxy, c * dmx * dmy);
    cyy = fmaf(w.wi, pyy, c * dmy * dmy);
  }
  float3 xc = point_at<CAM>(cam, y0, t_mu);
  float dep = sqrtf(fmaf(xc.x, xc.x, fmaf(xc.y, xc.y, xc.z * xc.z)));

  // opacity-tightened extent (Algorithm 1) and pixel rectangle
  // Mahalanobis distance where sigma rho falls to alpha_min: sqrt(2 ln(sigma / alpha_min)) for the
  // Gaussian, (ln(sigma / alpha_min) / lambda)^(1/n) for the degree-n kernel exp(-lambda d^n)
  const float lnr = logf(p.sigma / op.alpha_min);
  float kx = fminf(op.extent_sigma, op.kernel_degree == 2 ? sqrtf(2.f * lnr)
                                                          : powf(lnr / op.kernel_lambda, 1.f / op.kernel_degree));
  float hx = kx * sqrtf(cxx), hy = kx * sqrtf(cyy);
  ok = ok && isfinite(vm.x) && isfinite(vm.y) && isfinite(hx) && isfinite(hy);
  float fx0 = fmaxf(ceilf(vm.x - hx - 0.5f), 0.f), fx1 = fminf(floorf(vm.x + hx - 0.5f), (float)(cam.W - 1));
  float fy0 = fmaxf(ceilf(vm.y - hy - 0.5f), 0.f), fy1 = fminf(floorf(vm.y + hy - 0.5f), (float)(cam.H - 1));
  ok = ok && (fx0 <= fx1) && (fy0 <= fy1);

  short4 r = make_short4(0, 0, -1, -1);
  uint32_t nt = 0;
  if (ok) {
    int x0 = (int)fx0, x1 = (int)fx1, y0i = (int)fy0, y1 = (int)fy1;
    UT_DBG_CHECK(x0 >= 0 && y0i >= 0 && x0 <= x1 && y0i <= y1 && x1 < cam.W && y1 < cam.H, UT_DBG_RECT,
                 blockIdx.x * blockDim.x + threadIdx.x, x0 | (y0i << 16), x1 | (y1 << 16));
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
    cov2d[3 * (size_t)g] = cxx;
    cov2d[3 * (size_t)g + 1] = cxy;
    cov2d[3 * (size_t)g + 2] = cyy;
  }
  if (live) {
    mean2d[g] = vm;
    depth[g] = dep;
    rect[g] = r;
    ntiles[g] = nt;
  }
}

__global__ void k_project_points(DevCam cam, DevOpts op, const float *__restrict__ pts, int n,
                                 float2 *__restrict__ uv, int32_t *__restrict__ valid) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float3 x = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    float2 v;
    float t;
    const bool ok = project_world(cam, op.rs_iters, mat3_mul(cam.R0, x), v, t);
    uv[i] = v;
    valid[i] = ok ? 1 : 0;
  }
}

template <bool EWA, int CAM>
void project_launch(int blocks, const BatchDesc &bd, const DevOpts &op, const UTWeights &w, float *mean2d,
                    float *cov2d, float *depth, int16_t *rect, uint32_t *ntiles, cudaStream_t stream) {
  k_project<EWA, CAM><<<blocks, kWarps * 32, 0, stream>>>(bd, op, w, reinterpret_cast<float2 *>(mean2d), cov2d,
                                                         depth, reinterpret_cast<short4 *>(rect), ntiles);
}

}  // namespace

ut_status launch_project_points(const DevCam &cam, const DevOpts &op, const float *points, int n, float *uv,
                                int32_t *valid, cudaStream_t stream) {
  if (n == 0) return UT_OK;
  const int cap = device_sm_count() * 8, g = (n + 255) / 256;
  k_project_points<<<g < cap ? g : cap, 256, 0, stream>>>(cam, op, points, n, reinterpret_cast<float2 *>(uv),
                                                          valid);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

ut_status launch_project(const BatchDesc &bd, const DevOpts &op, const UTWeights &w, float *mean2d, float *cov2d,
                         float *depth, int16_t *rect, uint32_t *ntiles, cudaStream_t stream) {
  const int n = bd.total_particles;
  if (n == 0) return UT_OK;
  int blocks = (n + kWarps * 32 - 1) / (kWarps * 32);
  // one camera map for every view: the specialised UT kernel
  int cam = 2 * bd.v[0].cam.model + (bd.v[0].cam.rs ? 1 : 0);
  for (int v = 1; v < bd.nv; ++v)
    if (2 * bd.v[v].cam.model + (bd.v[v].cam.rs ? 1 : 0) != cam) cam = -1;
  if (op.projection == UT_PROJECTION_EWA) {
    project_launch<true, -1>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream);
  } else {
    switch (cam) {
      case 2 * UT_CAM_PINHOLE: project_launch<false, 2 * UT_CAM_PINHOLE>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      case 2 * UT_CAM_PINHOLE + 1: project_launch<false, 2 * UT_CAM_PINHOLE + 1>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      case 2 * UT_CAM_FISHEYE: project_launch<false, 2 * UT_CAM_FISHEYE>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      case 2 * UT_CAM_FISHEYE + 1: project_launch<false, 2 * UT_CAM_FISHEYE + 1>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      case 2 * UT_CAM_PINHOLE_RADIAL: project_launch<false, 2 * UT_CAM_PINHOLE_RADIAL>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      case 2 * UT_CAM_PINHOLE_RADIAL + 1: project_launch<false, 2 * UT_CAM_PINHOLE_RADIAL + 1>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
      default: project_launch<false, -1>(blocks, bd, op, w, mean2d, cov2d, depth, rect, ntiles, stream); break;
    }
  }
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? UT_OK : UT_ERR_CUDA;
}

UT_DBG_READER(dbg_read_project)

}  // namespace ut3d
