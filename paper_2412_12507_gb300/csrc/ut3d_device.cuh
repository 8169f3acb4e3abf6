// ut3d_device.cuh — device-side building blocks of the 3DGUT hot path (internal).
//
// Camera model g(x), pixel rays, particle activation and the real SH basis, all FP32.
// Shared by the projection, compositing and backward kernels so that every kernel
// takes the same decisions from the same arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ut3d.h"

namespace ut3d {

// Camera as the kernels see it: the host converts ut_camera once per call
// (rotation matrices, rolling-shutter relative rotation, fisheye limits) in FP64.
struct DevCam {
  int model, W, H, rs;
  float fx, fy, cx, cy, ifx, ify;
  float k1, k2, k3, k4;
  float R0[9];    // world->camera rotation at t = 0 (row-major)
  float T0[3];    // translation at t = 0
  float dT[3];    // t_end - t_start
  float ax[3];    // axis of the rotation taking the start pose to the end pose
  float phi;      // its angle (0 for a global shutter)
  float near_plane;
  float theta_max;  // fisheye: largest imaged angle
  float rd_max;     // fisheye: theta_d(theta_max), the imaged radius in normalised units
  float inv_hm1;    // 1 / (H - 1) (rolling shutter row -> time)
  float cen[3];     // camera centre -R0^T T0 at t = 0 (the ray origin of a global shutter)
};

struct DevOpts {
  int tile_w, tile_h, tiles_x, tiles_y;
  float t_min, alpha_min, alpha_max, extent_sigma;
  int rs_iters, newton_iters;
  int projection;   // UT_PROJECTION_UT / UT_PROJECTION_EWA
  int colour_mode;  // UT_COLOUR_PER_PIXEL / UT_COLOUR_PER_PARTICLE
  int kernel_degree;   // n of the generalised Gaussian (2 = Gaussian)
  float kernel_lambda; // 1/2 3^(2-n): rho = exp(-kernel_lambda d^n)
  int kbuffer;         // 0: blend in tile order; k: per-ray k-buffer of k entries
};

// ---------------------------------------------------------------- batches of views
//
// Every kernel works on a batch of V views (a camera looking at one of S scenes).  The
// particles of all views are flattened (view v owns entries [part_off, part_off + n) of the
// projection arrays) and so are the tiles (view v owns global tiles [tile_off, tile_off +
// tiles_x * tiles_y)).  The descriptor travels as a __grid_constant__ kernel parameter, so a
// batch needs no host-to-device copy.  A single-view call is the batch V = S = 1.
constexpr int kMaxViews = 32;
constexpr int kMaxScenes = 8;

struct DevView {
  DevCam cam;
  int scene;
  int part_off, n;             // flattened particle range of this view
  int tile_off, tiles_x, tiles_y;
  int col_off, row_off;         // global tile-column / tile-row offsets of this view (binning)
  float *rgb, *alpha, *tfinal;  // outputs ([3][H][W], [H][W], [H][W]); tfinal may be null
  uint32_t *n_used;             // [H][W], may be null
  const float *d_rgb, *d_alpha; // backward inputs
};

struct DevScene {
  const float *means, *log_scales;
  const float4 *quats;
  const float *logits, *sh;
  int n, deg;
  float *gacc;                  // backward accumulators [n][16]
  float4 *kbrec;                // k-buffer backward: per-particle record [n][4] (M, M mu, mu, sigma), else null
  float *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh;
  int grad_off;                 // flattened offset of this scene in finalize's range
  int sh_vec;                   // sh is 16-byte aligned and (deg+1)^2 * 3 is a multiple of 4
};

struct BatchDesc {
  int nv, ns;
  int total_particles, total_tiles;
  int total_cols, total_rows;   // tile columns / rows summed over the views
  int col_bits;                 // bits of the largest per-view tile-column index
  DevView v[kMaxViews];
  DevScene s[kMaxScenes];
};

// View owning global tile column c (views are sorted by col_off).
__device__ __forceinline__ int view_of_col(const BatchDesc &b, int c) {
  int lo = 0, hi = b.nv - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.v[mid].col_off <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// View owning global tile row r (views are sorted by row_off).
__device__ __forceinline__ int view_of_row(const BatchDesc &b, int r) {
  int lo = 0, hi = b.nv - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.v[mid].row_off <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// View owning flattened particle g (views are sorted by part_off).
__device__ __forceinline__ int view_of_particle(const BatchDesc &b, int g) {
  int lo = 0, hi = b.nv - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.v[mid].part_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// View owning global tile t.
__device__ __forceinline__ int view_of_tile(const BatchDesc &b, int t) {
  int lo = 0, hi = b.nv - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.v[mid].tile_off <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Scene owning flattened gradient index g (scenes are sorted by grad_off).
__device__ __forceinline__ int scene_of_grad(const BatchDesc &b, int g) {
  int lo = 0, hi = b.ns - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.s[mid].grad_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float3 mat3_mul(const float *R, float3 v) {
  return make_float3(fmaf(R[0], v.x, fmaf(R[1], v.y, R[2] * v.z)), fmaf(R[3], v.x, fmaf(R[4], v.y, R[5] * v.z)),
                     fmaf(R[6], v.x, fmaf(R[7], v.y, R[8] * v.z)));
}

__device__ __forceinline__ float3 mat3_tmul(const float *R, float3 v) {  // R^T v
  return make_float3(fmaf(R[0], v.x, fmaf(R[3], v.y, R[6] * v.z)), fmaf(R[1], v.x, fmaf(R[4], v.y, R[7] * v.z)),
                     fmaf(R[2], v.x, fmaf(R[5], v.y, R[8] * v.z)));
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// sin and cos of th for |th| <= pi (rotation angles between two poses): Cody-Waite reduction by
// pi/2 (k = rint(2 th / pi) in -2..2, r = th - k pi/2 with pi/2 split into two floats, so r is
// exact to about 1e-15), then odd / even polynomials on [-pi/4, pi/4] -- sin r = r + r^3 P(r^2),
// cos r = 1 - r^2 / 2 + r^4 Q(r^2), coefficients fitted to sin and cos by least squares with
// minimax reweighting (absolute error <= 2e-9 before rounding) -- and the quadrant by selects.
// Within about an ulp, like sincosf, without its path for huge arguments.
__device__ __forceinline__ void sincos_pi(float th, float &s, float &c) {
  const float k = rintf(th * 0.63661977236758134f);
  float r = fmaf(-k, 1.5707963705062866f, th);
  r = fmaf(-k, -4.371139000186243e-08f, r);
  const float r2 = r * r;
  const float sr = fmaf(r * r2, fmaf(r2, fmaf(r2, -1.9496e-4f, 8.33198e-3f), -0.16666651f), r);
  const float cr = fmaf(r2 * r2, fmaf(r2, fmaf(r2, 2.44385385e-05f, -1.38873683e-03f), 4.16666469e-02f),
                        fmaf(-0.5f, r2, 1.f));
  const int q = ((int)k) & 3;
  const float ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
  s = (q & 2) ? -ss : ss;
  c = (q == 1 || q == 2) ? -cc : cc;
}

// Rodrigues rotation of y by angle th (|th| <= pi) about the unit axis a.
__device__ __forceinline__ float3 rotate_axis(const float *a, float3 y, float th) {
  float s, c;
  sincos_pi(th, s, c);
  float ad = a[0] * y.x + a[1] * y.y + a[2] * y.z;
  float3 axy = make_float3(a[1] * y.z - a[2] * y.y, a[2] * y.x - a[0] * y.z, a[0] * y.y - a[1] * y.x);
  float oc = (1.f - c) * ad;
  return make_float3(fmaf(y.x, c, fmaf(axy.x, s, a[0] * oc)), fmaf(y.y, c, fmaf(axy.y, s, a[1] * oc)),
                     fmaf(y.z, c, fmaf(axy.z, s, a[2] * oc)));
}

// Rodrigues rotation with the fast hardware sine / cosine (absolute error about 4e-7 for
// |th| <= pi): used only inside the rolling-shutter time fixed point, whose iterates feed nothing
// but the next time estimate (see project_world_t).
__device__ __forceinline__ float3 rotate_axis_fast(const float *a, float3 y, float th) {
  float s, c;
  __sincosf(th, &s, &c);
  float ad = a[0] * y.x + a[1] * y.y + a[2] * y.z;
  float3 axy = make_float3(a[1] * y.z - a[2] * y.y, a[2] * y.x - a[0] * y.z, a[0] * y.y - a[1] * y.x);
  float oc = (1.f - c) * ad;
  return make_float3(fmaf(y.x, c, fmaf(axy.x, s, a[0] * oc)), fmaf(y.y, c, fmaf(axy.y, s, a[1] * oc)),
                     fmaf(y.z, c, fmaf(axy.z, s, a[2] * oc)));
}

// atan2(y, x) for y >= 0, in [0, pi]: atan of a = min(y, |x|) / max(y, |x|) in [0, 1] by an odd
// polynomial a P(a^2) of degree 15 (coefficients fitted to atan on [0, 1] by least squares with
// minimax reweighting; |error| <= 1.2e-7 in FP32), then the octant by selects.  For the
// rolling-shutter fixed point's iterates (see project_world_t).
__device__ __forceinline__ float atan2_pos_fast(float y, float x) {
  const float ax = fabsf(x);
  const float mx = fmaxf(y, ax), mn = fminf(y, ax);
  const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  const float a2 = a * a;
  float p = -0.004054596647620201f;
  p = fmaf(p, a2, 0.021863065659999847f);
  p = fmaf(p, a2, -0.05591248348355293f);
  p = fmaf(p, a2, 0.09642209112644196f);
  p = fmaf(p, a2, -0.13908633589744568f);
  p = fmaf(p, a2, 0.19946566224098206f);
  p = fmaf(p, a2, -0.33329862356185913f);
  p = fmaf(p, a2, 0.9999993443489075f);
  float r = p * a;
  r = y > ax ? 1.5707963267948966f - r : r;
  return x < 0.f ? 3.141592653589793f - r : r;
}

// x_c(t) for a point whose start-pose camera coordinates rotated part is y = R0 x.  RS: the
// camera has a rolling shutter (c.rs != 0); the runtime form below tests c.rs itself.
template <bool RS>
__device__ __forceinline__ float3 cam_point_at_t(const DevCam &c, float3 y, float t) {
  float3 r = RS ? rotate_axis(c.ax, y, t * c.phi) : y;
  return make_float3(r.x + fmaf(t, c.dT[0], c.T0[0]), r.y + fmaf(t, c.dT[1], c.T0[1]),
                     r.z + fmaf(t, c.dT[2], c.T0[2]));
}

__device__ __forceinline__ float3 cam_point_at(const DevCam &c, float3 y, float t) {
  return c.rs ? cam_point_at_t<true>(c, y, t) : cam_point_at_t<false>(c, y, t);
}

__device__ __forceinline__ float theta_d_poly(const DevCam &c, float th) {
  float t2 = th * th;
  return th * fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, c.k4, c.k3), c.k2), c.k1), 1.f);
}

__device__ __forceinline__ float theta_d_prime(const DevCam &c, float th) {
  float t2 = th * th;
  return fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 9.f * c.k4, 7.f * c.k3), 5.f * c.k2), 3.f * c.k1), 1.f);
}

// Radial pinhole: r_d(r) = r (1 + k1 r^2 + k2 r^4 + k3 r^6) and its derivative.
__device__ __forceinline__ float radial_scale(const DevCam &c, float r2) {
  return fmaf(r2, fmaf(r2, fmaf(r2, c.k3, c.k2), c.k1), 1.f);
}

__device__ __forceinline__ float radial_prime(const DevCam &c, float r2) {
  return fmaf(r2, fmaf(r2, fmaf(r2, 7.f * c.k3, 5.f * c.k2), 3.f * c.k1), 1.f);
}

// g(x_c): camera-space point to pixel coordinates; returns false when not imaged.  MODEL is the
// camera model (ut_cam_model); cam_project dispatches on c.model at run time.
template <int MODEL>
__device__ __forceinline__ bool cam_project_t(const DevCam &c, float3 p, float2 &uv) {
  if constexpr (MODEL == UT_CAM_PINHOLE) {
    float iz = 1.f / p.z;
    uv.x = fmaf(c.fx * p.x, iz, c.cx);
    uv.y = fmaf(c.fy * p.y, iz, c.cy);
    return p.z > c.near_plane;
  } else if constexpr (MODEL == UT_CAM_PINHOLE_RADIAL) {
    // theta_max holds the largest imaged normalised radius r_max
    float iz = 1.f / p.z;
    float xn = p.x * iz, yn = p.y * iz;
    float r2 = fmaf(xn, xn, yn * yn);
    float sd = radial_scale(c, r2);
    uv.x = fmaf(c.fx * xn, sd, c.cx);
    uv.y = fmaf(c.fy * yn, sd, c.cy);
    return p.z > c.near_plane && sqrtf(r2) <= c.theta_max;
  } else {
    // 1 / rho by the reciprocal square root and one Newton step (within about an ulp, like the
    // IEEE square root and division it replaces); the near-plane test on squares
    const float r2 = fmaf(p.x, p.x, p.y * p.y);
    float rq = rsqrtf(r2);
    rq = rq * fmaf(-0.5f * r2, rq * rq, 1.5f);
    const bool axis = !(r2 > 0.f);
    const float th = atan2f(axis ? 0.f : r2 * rq, p.z);
    const float s = axis ? 1.f / p.z : theta_d_poly(c, th) * rq;
    uv.x = fmaf(c.fx * s, p.x, c.cx);
    uv.y = fmaf(c.fy * s, p.y, c.cy);
    return (fmaf(p.z, p.z, r2) > c.near_plane * c.near_plane) && (th <= c.theta_max);
  }
}

// g(x_c) with fast reciprocal square root / division and atan2_pos_fast: for the rolling-shutter
// fixed point's iterates only (see project_world_t).  Same validity tests as cam_project_t.
template <int MODEL>
__device__ __forceinline__ bool cam_project_fast_t(const DevCam &c, float3 p, float2 &uv) {
  if constexpr (MODEL == UT_CAM_FISHEYE) {
    const float r2 = fmaf(p.x, p.x, p.y * p.y);
    const float rq = rsqrtf(r2);
    const bool axis = !(r2 > 0.f);
    const float th = atan2_pos_fast(axis ? 0.f : r2 * rq, p.z);
    const float s = axis ? __fdividef(1.f, p.z) : theta_d_poly(c, th) * rq;
    uv.x = fmaf(c.fx * s, p.x, c.cx);
    uv.y = fmaf(c.fy * s, p.y, c.cy);
    return (fmaf(p.z, p.z, r2) > c.near_plane * c.near_plane) && (th <= c.theta_max);
  } else if constexpr (MODEL == UT_CAM_PINHOLE_RADIAL) {
    const float iz = __fdividef(1.f, p.z);
    const float xn = p.x * iz, yn = p.y * iz;
    const float r2 = fmaf(xn, xn, yn * yn);
    const float sd = radial_scale(c, r2);
    uv.x = fmaf(c.fx * xn, sd, c.cx);
    uv.y = fmaf(c.fy * yn, sd, c.cy);
    return p.z > c.near_plane && r2 <= c.theta_max * c.theta_max;
  } else {
    const float iz = __fdividef(1.f, p.z);
    uv.x = fmaf(c.fx * p.x, iz, c.cx);
    uv.y = fmaf(c.fy * p.y, iz, c.cy);
    return p.z > c.near_plane;
  }
}

__device__ __forceinline__ bool cam_project(const DevCam &c, float3 p, float2 &uv) {
  if (c.model == UT_CAM_PINHOLE) return cam_project_t<UT_CAM_PINHOLE>(c, p, uv);
  if (c.model == UT_CAM_PINHOLE_RADIAL) return cam_project_t<UT_CAM_PINHOLE_RADIAL>(c, p, uv);
  return cam_project_t<UT_CAM_FISHEYE>(c, p, uv);
}

// Jacobian d g / d x_c (rows u, v) of the camera map at a camera-space point.  Fisheye:
// u = fx s X + cx with s = theta_d(theta) / rho, theta = atan2(rho, Z), hence
// d s = (theta_d'(theta) d theta - s d rho) / rho, d theta = (X Z, Y Z, -rho^2) / (rho r^2),
// d rho = (X, Y, 0) / rho; on the optical axis the map is the pinhole one.
__device__ __forceinline__ void cam_jacobian(const DevCam &c, float3 p, float3 &ju, float3 &jv) {
  if (c.model == UT_CAM_PINHOLE || c.model == UT_CAM_PINHOLE_RADIAL) {  // radial: 3DGS's undistorted one
    const float iz = 1.f / p.z;
    ju = make_float3(c.fx * iz, 0.f, -c.fx * p.x * iz * iz);
    jv = make_float3(0.f, c.fy * iz, -c.fy * p.y * iz * iz);
    return;
  }
  const float rho2 = fmaf(p.x, p.x, p.y * p.y), rho = sqrtf(rho2);
  if (!(rho > 0.f)) {
    ju = make_float3(c.fx / p.z, 0.f, 0.f);
    jv = make_float3(0.f, c.fy / p.z, 0.f);
    return;
  }
  const float r2 = fmaf(p.z, p.z, rho2);
  const float th = atan2f(rho, p.z);
  const float irho = 1.f / rho;
  const float s = theta_d_poly(c, th) * irho, tdp = theta_d_prime(c, th);
  const float a = p.z / (rho * r2);
  const float3 ds = make_float3((tdp * p.x * a - s * p.x * irho) * irho, (tdp * p.y * a - s * p.y * irho) * irho,
                                (-tdp * rho / r2) * irho);
  ju = make_float3(c.fx * fmaf(p.x, ds.x, s), c.fx * p.x * ds.y, c.fx * p.x * ds.z);
  jv = make_float3(c.fy * p.y * ds.x, c.fy * fmaf(p.y, ds.y, s), c.fy * p.y * ds.z);
}

// Projection of a world point with the rolling-shutter time fixed point
// (t = 1/2, rs_iters updates t <- clamp((v - 1/2)/(H-1)), final projection).
// y = R0 x.  Returns validity of every projection taken; t_out = the final time.
// The iterates only produce the next time estimate: an error dv in their row moves t by
// dv / (H - 1) and the final projection by (dv / dt) dv / (H - 1), five orders of magnitude less
// for any camera that moves less than a frame height over the exposure, so they take the fast
// camera map (rotation with the hardware sine / cosine, fast reciprocal square root and atan2;
// a few 1e-4 px each); the final projection, which alone sets the result, takes the IEEE one.
template <int MODEL, bool RS>
__device__ __forceinline__ bool project_world_t(const DevCam &c, int rs_iters, float3 y, float2 &uv, float &t_out) {
  bool ok = true;
  float t = 0.f;
  if (RS) {
    t = 0.5f;
    for (int it = 0; it < rs_iters; ++it) {
      const float3 r = rotate_axis_fast(c.ax, y, t * c.phi);
      const float3 p = make_float3(r.x + fmaf(t, c.dT[0], c.T0[0]), r.y + fmaf(t, c.dT[1], c.T0[1]),
                                   r.z + fmaf(t, c.dT[2], c.T0[2]));
      ok &= cam_project_fast_t<MODEL>(c, p, uv);
      t = fminf(fmaxf((uv.y - 0.5f) * c.inv_hm1, 0.f), 1.f);
    }
  }
  ok &= cam_project_t<MODEL>(c, cam_point_at_t<RS>(c, y, t), uv);
  t_out = t;
  return ok;
}

__device__ __forceinline__ bool project_world(const DevCam &c, int rs_iters, float3 y, float2 &uv, float &t_out) {
  if (c.model == UT_CAM_PINHOLE)
    return c.rs ? project_world_t<UT_CAM_PINHOLE, true>(c, rs_iters, y, uv, t_out)
                : project_world_t<UT_CAM_PINHOLE, false>(c, rs_iters, y, uv, t_out);
  if (c.model == UT_CAM_PINHOLE_RADIAL)
    return c.rs ? project_world_t<UT_CAM_PINHOLE_RADIAL, true>(c, rs_iters, y, uv, t_out)
                : project_world_t<UT_CAM_PINHOLE_RADIAL, false>(c, rs_iters, y, uv, t_out);
  return c.rs ? project_world_t<UT_CAM_FISHEYE, true>(c, rs_iters, y, uv, t_out)
              : project_world_t<UT_CAM_FISHEYE, false>(c, rs_iters, y, uv, t_out);
}

// World ray of pixel (px, py) (integer indices; the ray goes through the pixel centre).
// Returns false for a fisheye pixel outside the imaged disc.
__device__ __forceinline__ bool pixel_ray(const DevCam &c, int px, int py, int newton_iters, float3 &o, float3 &d) {
  float mx = (px + 0.5f - c.cx) * c.ifx;
  float my = (py + 0.5f - c.cy) * c.ify;
  float3 dc;
  if (c.model == UT_CAM_PINHOLE) {
    dc = make_float3(mx, my, 1.f);
  } else if (c.model == UT_CAM_PINHOLE_RADIAL) {
    float rd = sqrtf(fmaf(mx, mx, my * my));
    if (!(rd <= c.rd_max)) return false;
    // safeguarded Newton for r_d(r) = rd on the increasing branch [0, r_max]
    float lo = 0.f, hi = fminf(c.theta_max, fmaxf(2.f * rd, 1.f));
    for (int it = 0; it < 40 && isinf(c.theta_max) && rd > hi * radial_scale(c, hi * hi); ++it) hi *= 2.f;
    float r = fminf(rd, hi);
    for (int it = 0; it < newton_iters; ++it) {
      float f = fmaf(r, radial_scale(c, r * r), -rd);
      if (f == 0.f) break;
      if (f > 0.f) hi = r; else lo = r;
      float nr = r - f / radial_prime(c, r * r);
      if (!(nr >= lo && nr <= hi)) nr = 0.5f * (lo + hi);  // Newton left the bracket: bisect
      if (nr == r) break;
      r = nr;
    }
    dc = rd > 0.f ? make_float3(mx * (r / rd), my * (r / rd), 1.f) : make_float3(0.f, 0.f, 1.f);
  } else {
    float rd = sqrtf(fmaf(mx, mx, my * my));
    if (!(rd <= c.rd_max)) return false;
    // safeguarded Newton for theta_d(theta) = rd on the increasing branch [0, theta_max]
    float lo = 0.f, hi = c.theta_max;
    float th = fminf(rd, c.theta_max);
    for (int it = 0; it < newton_iters; ++it) {
      float f = theta_d_poly(c, th) - rd;
      if (f == 0.f) break;
      if (f > 0.f) hi = th; else lo = th;
      float fp = theta_d_prime(c, th);
      float nt = th - f / fp;
      if (!(nt >= lo && nt <= hi)) nt = 0.5f * (lo + hi);  // Newton left the bracket: bisect
      if (nt == th) break;
      th = nt;
    }
    float s, co;
    sincosf(th, &s, &co);
    if (rd > 0.f) {
      float k = s / rd;
      dc = make_float3(k * mx, k * my, co);
    } else {
      dc = make_float3(0.f, 0.f, 1.f);
    }
  }
  float t = c.rs ? py * c.inv_hm1 : 0.f;
  // pose at the row time: R(t) = Rot(ax, t phi) R0, T(t) = T0 + t dT; camera centre o = -R^T T
  float3 Tt = make_float3(fmaf(t, c.dT[0], c.T0[0]), fmaf(t, c.dT[1], c.T0[1]), fmaf(t, c.dT[2], c.T0[2]));
  if (c.rs) {
    // R(t)^T v = R0^T Rot(ax, -t phi) v
    float3 mT = rotate_axis(c.ax, make_float3(-Tt.x, -Tt.y, -Tt.z), -t * c.phi);
    float3 dr = rotate_axis(c.ax, dc, -t * c.phi);
    o = mat3_tmul(c.R0, mT);
    d = mat3_tmul(c.R0, dr);
  } else {
    o = mat3_tmul(c.R0, make_float3(-Tt.x, -Tt.y, -Tt.z));
    d = mat3_tmul(c.R0, dc);
  }
  return true;
}

// Real spherical harmonics with the Condon-Shortley phase, orthonormal, degrees 0..DEG,
// index l*l + l + m, at the unit direction (x, y, z).  The constants are
// sqrt(2) K_l^|m| times the constant factor of P_l^|m| / (1 - z^2)^{|m|/2}, with
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
  Y[0] = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
  if (DEG >= 1) {
    const float c1 = 0.4886025119029199f;  // sqrt(3 / (4 pi))
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;                 // 3 sqrt(5 / (12 pi)) xy
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);  // sqrt(5 / (16 pi)) (3z^2 - 1)
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);             // 3 sqrt(5 / (48 pi))
    if (DEG >= 3) {
      Y[9] = -0.5900435899266435f * y * (3.f * xx - yy);   // 15 sqrt(7 / (1440 pi))
      Y[10] = 2.890611442640554f * x * y * z;              // 30 sqrt(7 / (240 pi))
      Y[11] = -0.4570457994644658f * y * (4.f * zz - xx - yy);  // 1.5 sqrt(7 / (24 pi))
      Y[12] = 0.3731763325901154f * z * (2.f * zz - 3.f * xx - 3.f * yy);  // sqrt(7 / (16 pi))
      Y[13] = -0.4570457994644658f * x * (4.f * zz - xx - yy);
      Y[14] = 1.445305721320277f * z * (xx - yy);           // 15 sqrt(7 / (240 pi))
      Y[15] = -0.5900435899266435f * x * (xx - 3.f * yy);
    }
  }
}

// Activated particle parameters: s = exp(log_s), sigma = sigmoid(logit), unit quaternion,
// R(q), M = S^-1 R^T.  Returns false for non-finite parameters or a zero quaternion.
struct Particle {
  float3 mu;
  float s[3];
  float q[4];   // normalised
  float qn;     // |q| before normalisation
  float R[9];
  float M[9];
  float sigma;
};

__device__ __forceinline__ void quat_to_rot(const float *q, float *R) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ bool activate(float3 mu, float3 ls, float4 q4, float logit, Particle &p) {
  p.mu = mu;
  p.s[0] = expf(ls.x); p.s[1] = expf(ls.y); p.s[2] = expf(ls.z);
  float qq = fmaf(q4.x, q4.x, fmaf(q4.y, q4.y, fmaf(q4.z, q4.z, q4.w * q4.w)));
  p.qn = sqrtf(qq);
  float iq = 1.f / p.qn;
  p.q[0] = q4.x * iq; p.q[1] = q4.y * iq; p.q[2] = q4.z * iq; p.q[3] = q4.w * iq;
  quat_to_rot(p.q, p.R);
  for (int k = 0; k < 3; ++k) {
    float is = 1.f / p.s[k];
    p.M[3 * k + 0] = p.R[0 + k] * is;
    p.M[3 * k + 1] = p.R[3 + k] * is;
    p.M[3 * k + 2] = p.R[6 + k] * is;
  }
  p.sigma = 1.f / (1.f + expf(-logit));
  bool ok = isfinite(mu.x) && isfinite(mu.y) && isfinite(mu.z) && isfinite(logit) && qq > 0.f && isfinite(qq);
  ok = ok && p.s[0] > 0.f && p.s[1] > 0.f && p.s[2] > 0.f && isfinite(p.s[0]) && isfinite(p.s[1]) &&
       isfinite(p.s[2]);
  return ok;
}

}  // namespace ut3d
