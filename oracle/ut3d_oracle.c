/*
 * ut3d_oracle.c — plain, slow FP64 CPU oracle of the 3DGUT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is loaded by the tests, by __graft_entry__.smoke() and by the CPU
 * baseline leg of bench.py, and by nothing else.  It shares no code, header,
 * constant table or helper with the CUDA library.
 *
 * What it computes (each function cites the passage it restates):
 *   - 3D Gaussian particles: response rho(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)),
 *     Sigma = R S S^T R^T (Sec. 3, eq. gaussian_kernel, eq. gaussian_covariance).
 *   - The Unscented Transform projection of every particle (Sec. 4.1,
 *     eq. sigma_points, eq. weights_1/2, eq. 2d_conic_1/2; Algorithms 1 and 2
 *     of the supplementary), through a pinhole, a polynomial (Kannala-Brandt)
 *     fisheye or a test-only orthographic camera, with an optional rolling
 *     shutter ("a different extrinsic matrix" per sigma point, Sec. 1).
 *   - Duplicate keys (tile | depth) and their global stable sort per tile
 *     (Sec. 4.3, Table 2 phases Duplicate and Sort).
 *   - The first-order (EWA) projection Sigma' = J W Sigma W^T J^T of 3DGS (eq. ewa_splatting),
 *     with J the Jacobian of the camera map at the mean, as the A/B baseline of the UT.
 *   - Front-to-back volumetric compositing (eq. QuadratureVolumeRendering) with
 *     each particle evaluated in 3D at its maximum response along the pixel ray
 *     (Sec. 4.2, eq. GaussianMaxResponse), brute force over ALL particles in
 *     global depth order with no tiling.
 *   - The reverse-mode gradient of the composited colour and opacity with
 *     respect to every particle parameter (supplementary Sec. B, extended to
 *     S, R, opacity and SH as the paper says "follow analogously").
 *
 * Readings where the paper is silent (listed with reasons in the design notes):
 *   pinhole / fisheye formulas, rolling-shutter time rule (fixed point on the
 *   projected row), depth = Euclidean distance, extent = min(cap, sqrt(2 ln(sigma/alpha_min)))
 *   standard deviations, pixel-centre-in-rect membership, alpha = min(alpha_max, sigma rho),
 *   skip below alpha_min, stop before blending when T(1-alpha) < t_min, SH colour
 *   max(sum beta Y + 0.5, 0) at the pixel's ray direction.
 *
 * Everything is computed in double precision from FP32 inputs promoted to FP64.
 * The only decisions taken in FP32 are the ones the key format fixes: the
 * depth that enters the sort key is the FP64 depth rounded to FP32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
  int32_t model;           /* 0 pinhole, 1 fisheye (polynomial), 2 orthographic (test-only affine),
                              3 pinhole with radial distortion k1..k3 */
  int32_t width, height;
  int32_t rolling_shutter; /* 0 global shutter (start pose), 1 rows exposed top to bottom */
  double fx, fy, cx, cy;
  double k[4];
  double q_start[4], t_start[3]; /* world->camera rotation (w,x,y,z) and translation at row 0 */
  double q_end[4], t_end[3];     /* same at row H-1 */
  double near_plane;
} orc_camera;

typedef struct {
  const float *means, *log_scales, *quats, *opacity_logits, *sh;
  int32_t n, sh_degree;
} orc_scene;

typedef struct {
  int32_t tile_w, tile_h;
  double t_min, alpha_min, alpha_max;
  int32_t rs_iters;
  double ut_alpha, ut_beta, ut_kappa;
  double extent_sigma;
  int32_t projection;  /* 0: Unscented Transform (Sec. 4.1); 1: first-order EWA (eq. ewa_splatting) */
  int32_t colour_mode; /* 0: SH at each pixel's ray direction; 1: SH once per particle at the
                          direction from the camera centre (at the mean's shutter time) to the mean */
  int32_t kernel_degree; /* n of the generalised Gaussian (supplementary Sec. A); 2 = Gaussian */
  int32_t kbuffer;       /* 0: blend in tile (global depth) order; k > 0: per-ray k-buffer (Sec. 4.4, MLAB) */
  double eps_tau;        /* k-buffer near-tie tolerance on tau (relative), for flags only */
} orc_options;

/* near-tie tolerances used only to flag pixels whose FP32 result may legitimately differ */
typedef struct {
  double eps_px;   /* rect edge distance in pixels */
  double eps_rel;  /* relative distance of alpha / transmittance / culling to a threshold */
  int32_t depth_ulps; /* depth keys closer than this many FP32 ulps may swap */
  double cond_min; /* fisheye: pixels where d theta_d / d theta is below this are ill-conditioned */
  double eps_t;    /* relative distance of T (1 - alpha) to t_min */
} orc_tol;

/* pixel flag bits */
enum {
  ORC_F_RECT_EDGE = 1, ORC_F_ALPHA_MIN = 2, ORC_F_TSTOP = 4, ORC_F_DEPTH_TIE = 8,
  ORC_F_CULL_TIE = 16, ORC_F_PIXEL_EDGE = 32, ORC_F_ILL_COND = 64, ORC_F_ALPHA_MAX = 128,
  ORC_F_INVALID_PIXEL = 256, ORC_F_CLAMP = 512
};

/* A blended particle's colour channel sum_k beta_k Y_k + 1/2 within eps_rel of 0, relative to
 * the size of its terms: the clamp max(., 0) may go either way in FP32.  The colour itself is
 * continuous there (it is ~0 on both sides), but its derivative is not, so a gradient through
 * such a pixel may legitimately differ: ORC_F_CLAMP (it does not concern the forward). */
static int orc_clamp_tie(const float *beta, const double *Yc, int nsh, const double raw[3], double eps) {
  for (int ch = 0; ch < 3; ++ch) {
    double scale = 0.5;
    for (int kk = 0; kk < nsh; ++kk) scale += fabs(beta[3 * kk + ch] * Yc[kk]);
    if (fabs(raw[ch]) < eps * scale) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------ rotations */

/* Rotation matrix of a unit quaternion (w,x,y,z), row-major. */
static void orc_quat_to_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void orc_normalize4(const double *q, double out[4]) {
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) out[i] = q[i] / n;
}

/* Spherical linear interpolation between unit quaternions along the shorter arc. */
static void orc_slerp(const double a[4], const double b_in[4], double t, double out[4]) {
  double b[4];
  double dot = a[0] * b_in[0] + a[1] * b_in[1] + a[2] * b_in[2] + a[3] * b_in[3];
  double sgn = dot < 0 ? -1.0 : 1.0;
  for (int i = 0; i < 4; ++i) b[i] = sgn * b_in[i];
  dot = fabs(dot);
  if (dot > 1.0) dot = 1.0;
  double th = acos(dot);
  double wa, wb;
  if (th < 1e-12) { wa = 1.0 - t; wb = t; }
  else { wa = sin((1.0 - t) * th) / sin(th); wb = sin(t * th) / sin(th); }
  double q[4];
  for (int i = 0; i < 4; ++i) q[i] = wa * a[i] + wb * b[i];
  orc_normalize4(q, out);
}

/* World->camera pose at shutter time t in [0,1]: rotation slerped, translation lerped. */
static void orc_pose_at(const orc_camera *c, double t, double R[9], double T[3]) {
  double qa[4], qb[4], q[4];
  orc_normalize4(c->q_start, qa);
  if (!c->rolling_shutter) {
    orc_quat_to_rot(qa, R);
    for (int i = 0; i < 3; ++i) T[i] = c->t_start[i];
    return;
  }
  orc_normalize4(c->q_end, qb);
  orc_slerp(qa, qb, t, q);
  orc_quat_to_rot(q, R);
  for (int i = 0; i < 3; ++i) T[i] = (1.0 - t) * c->t_start[i] + t * c->t_end[i];
}

/* The pose at shutter time t as the tests see it (same function, exported). */
void orc_pose(const orc_camera *c, double t, double R[9], double T[3]) { orc_pose_at(c, t, R, T); }

/* ------------------------------------------------------------------ fisheye polynomial */

static double orc_theta_d(const double k[4], double th) {
  double t2 = th * th;
  return th * (1.0 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
}

static double orc_theta_d_prime(const double k[4], double th) {
  double t2 = th * th;
  return 1.0 + t2 * (3 * k[0] + t2 * (5 * k[1] + t2 * (7 * k[2] + t2 * 9 * k[3])));
}

/* Largest angle the polynomial fisheye can image: pi/2, or the first zero of
 * d theta_d / d theta on (0, pi/2] when the distortion polynomial turns over. */
double orc_theta_max(const double k[4]) {
  const int steps = 1 << 14;
  double lo = 0.0, prev = orc_theta_d_prime(k, 0.0);
  for (int i = 1; i <= steps; ++i) {
    double th = 0.5 * ORC_PI * (double)i / steps;
    double v = orc_theta_d_prime(k, th);
    if (v <= 0.0 && prev > 0.0) {
      double a = lo, b = th;
      for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b);
        if (orc_theta_d_prime(k, m) > 0.0) a = m; else b = m;
      }
      return a;
    }
    lo = th; prev = v;
  }
  return 0.5 * ORC_PI;
}

/* theta in [0, theta_max] with theta_d(theta) = rd (theta_d is increasing there) */
static double orc_theta_inverse(const double k[4], double theta_max, double rd) {
  double a = 0.0, b = theta_max;
  double th = rd < theta_max ? rd : theta_max;
  for (int it = 0; it < 200; ++it) {
    double f = orc_theta_d(k, th) - rd;
    if (f == 0.0) break; /* exact root */
    if (f > 0) b = th; else a = th;
    double fp = orc_theta_d_prime(k, th);
    double nt = fp > 0 ? th - f / fp : 0.5 * (a + b);
    if (!(nt >= a && nt <= b)) nt = 0.5 * (a + b); /* Newton left the bracket: bisect */
    if (fabs(nt - th) < 1e-16 * (1.0 + th)) { th = nt; break; }
    th = nt;
    if (b - a < 1e-17) break;
  }
  return th;
}

/* ------------------------------------------------------------------ radial pinhole */

/* r_d(r) = r (1 + k1 r^2 + k2 r^4 + k3 r^6) on the normalised image plane, and its derivative. */
static double orc_radial_rd(const double k[4], double r) {
  double q = r * r;
  return r * (1.0 + q * (k[0] + q * (k[1] + q * k[2])));
}

static double orc_radial_rd_prime(const double k[4], double r) {
  double q = r * r;
  return 1.0 + q * (3 * k[0] + q * (5 * k[1] + q * 7 * k[2]));
}

/* Largest normalised radius the radial model images: the first zero of d r_d / d r on
 * (0, 10] (the distortion polynomial turns over there), else unbounded. */
static double orc_radial_rmax(const double k[4]) {
  const int steps = 1 << 14;
  double lo = 0.0, prev = orc_radial_rd_prime(k, 0.0);
  for (int i = 1; i <= steps; ++i) {
    double r = 10.0 * (double)i / steps;
    double v = orc_radial_rd_prime(k, r);
    if (v <= 0.0 && prev > 0.0) {
      double a = lo, b = r;
      for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b);
        if (orc_radial_rd_prime(k, m) > 0.0) a = m; else b = m;
      }
      return a;
    }
    lo = r; prev = v;
  }
  return INFINITY;
}

/* r >= 0 with r_d(r) = rd on the increasing branch [0, rmax]: bisection on a bracket. */
static double orc_radial_inverse(const double k[4], double rmax, double rd) {
  double a = 0.0, b = rmax;
  if (!isfinite(b)) {
    b = rd > 1.0 ? rd : 1.0;
    while (orc_radial_rd(k, b) < rd) b *= 2.0;
  }
  for (int it = 0; it < 300 && b - a > 1e-16 * (1.0 + b); ++it) {
    double m = 0.5 * (a + b);
    if (orc_radial_rd(k, m) < rd) a = m; else b = m;
  }
  return 0.5 * (a + b);
}

/* The model's field limit passed to the projection / ray functions: theta_max for the
 * fisheye, the largest normalised radius for the radial pinhole, pi/2 otherwise (unused). */
double orc_cam_limit(const orc_camera *c) {
  if (c->model == 1) return orc_theta_max(c->k);
  if (c->model == 3) return orc_radial_rmax(c->k);
  return 0.5 * ORC_PI;
}

/* ------------------------------------------------------------------ camera model g(x) */

/* Projects a camera-space point; returns 1 if it is imaged.  *margin receives the
 * signed relative distance to the validity boundary (positive = valid). */
static int orc_project_cam(const orc_camera *c, double theta_max, const double xc[3], double uv[2],
                           double *margin) {
  double X = xc[0], Y = xc[1], Z = xc[2];
  if (c->model == 0) {
    *margin = (Z - c->near_plane) / c->near_plane;
    if (!(Z > c->near_plane)) return 0;
    uv[0] = c->fx * X / Z + c->cx;
    uv[1] = c->fy * Y / Z + c->cy;
    return 1;
  } else if (c->model == 1) {
    double rho = sqrt(X * X + Y * Y);
    double r3 = sqrt(X * X + Y * Y + Z * Z);
    double th = atan2(rho, Z);
    double m1 = (r3 - c->near_plane) / c->near_plane;
    double m2 = (theta_max - th) / theta_max;
    *margin = m1 < m2 ? m1 : m2;
    if (!(r3 > c->near_plane) || !(th <= theta_max)) return 0;
    if (rho > 0.0) {
      double s = orc_theta_d(c->k, th) / rho;
      uv[0] = c->fx * s * X + c->cx;
      uv[1] = c->fy * s * Y + c->cy;
    } else {
      uv[0] = c->cx;
      uv[1] = c->cy;
    }
    return 1;
  } else if (c->model == 3) {
    /* theta_max carries the largest normalised radius of the radial model */
    double m1 = (Z - c->near_plane) / c->near_plane;
    if (!(Z > c->near_plane)) { *margin = m1; return 0; }
    double xn = X / Z, yn = Y / Z, r = sqrt(xn * xn + yn * yn);
    double m2 = isfinite(theta_max) ? (theta_max - r) / theta_max : INFINITY;
    *margin = m1 < m2 ? m1 : m2;
    if (!(r <= theta_max)) return 0;
    double q = r * r, sd = 1.0 + q * (c->k[0] + q * (c->k[1] + q * c->k[2]));
    uv[0] = c->fx * xn * sd + c->cx;
    uv[1] = c->fy * yn * sd + c->cy;
    return 1;
  } else {
    *margin = INFINITY;
    uv[0] = c->fx * X + c->cx;
    uv[1] = c->fy * Y + c->cy;
    return 1;
  }
}

/* g(x) for a world point, with the rolling-shutter time found as a fixed point on
 * the projected row: t <- clamp((v - 1/2)/(H-1), 0, 1), rs_iters updates from t = 1/2,
 * then the final projection at the last t.  Every projection must be valid. */
int orc_project_world(const orc_camera *c, double theta_max, int rs_iters, const double x[3],
                      double uv[2], double *t_out, double *margin_out) {
  double R[9], T[3], xc[3], m, margin = INFINITY;
  int valid = 1;
  double t = 0.0;
  if (c->rolling_shutter) {
    t = 0.5;
    for (int it = 0; it < rs_iters; ++it) {
      orc_pose_at(c, t, R, T);
      for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + T[r];
      valid &= orc_project_cam(c, theta_max, xc, uv, &m);
      if (m < margin) margin = m;
      if (!valid) break;
      t = (uv[1] - 0.5) / (double)(c->height - 1);
      if (t < 0.0) t = 0.0;
      if (t > 1.0) t = 1.0;
    }
  }
  if (valid) {
    orc_pose_at(c, t, R, T);
    for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + T[r];
    valid &= orc_project_cam(c, theta_max, xc, uv, &m);
    if (m < margin) margin = m;
  }
  if (t_out) *t_out = t;
  if (margin_out) *margin_out = margin;
  return valid;
}

/* Camera ray of the pixel-plane point (px, py) (pixel centres at integer + 1/2), in world
 * space; rolling shutter uses the row time (py - 1/2)/(H-1).  Returns 1 if the point is
 * inside the imaged region.  *dprime receives d theta_d / d theta at the ray (fisheye) or 1. */
int orc_pixel_ray(const orc_camera *c, double theta_max, double px, double py, double o[3], double d[3],
                  double *edge_margin, double *dprime) {
  double t = 0.0;
  if (c->rolling_shutter) {
    t = (py - 0.5) / (double)(c->height - 1);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
  }
  double R[9], T[3];
  orc_pose_at(c, t, R, T);
  double oc[3] = {0, 0, 0}, dc[3];
  double mx = (px - c->cx) / c->fx, my = (py - c->cy) / c->fy;
  *edge_margin = INFINITY;
  *dprime = 1.0;
  if (c->model == 0) {
    dc[0] = mx; dc[1] = my; dc[2] = 1.0;
  } else if (c->model == 1) {
    double rd = sqrt(mx * mx + my * my);
    double rmax = orc_theta_d(c->k, theta_max);
    *edge_margin = (rmax - rd) / rmax;
    if (!(rd <= rmax)) return 0;
    double th = orc_theta_inverse(c->k, theta_max, rd);
    *dprime = orc_theta_d_prime(c->k, th);
    if (rd > 0) {
      double s = sin(th) / rd;
      dc[0] = s * mx; dc[1] = s * my; dc[2] = cos(th);
    } else {
      dc[0] = 0; dc[1] = 0; dc[2] = 1;
    }
  } else if (c->model == 3) {
    /* theta_max carries the largest normalised radius r_max of the radial model */
    double rd = sqrt(mx * mx + my * my);
    double rdmax = isfinite(theta_max) ? orc_radial_rd(c->k, theta_max) : INFINITY;
    *edge_margin = isfinite(rdmax) ? (rdmax - rd) / rdmax : INFINITY;
    if (!(rd <= rdmax)) return 0;
    double r = orc_radial_inverse(c->k, theta_max, rd);
    *dprime = orc_radial_rd_prime(c->k, r);
    if (rd > 0) {
      dc[0] = mx * r / rd; dc[1] = my * r / rd; dc[2] = 1.0;
    } else {
      dc[0] = 0; dc[1] = 0; dc[2] = 1;
    }
  } else {
    oc[0] = mx; oc[1] = my;
    dc[0] = 0; dc[1] = 0; dc[2] = 1;
  }
  /* camera -> world: x = R^T (x_c - T) */
  for (int j = 0; j < 3; ++j) {
    o[j] = R[j] * (oc[0] - T[0]) + R[3 + j] * (oc[1] - T[1]) + R[6 + j] * (oc[2] - T[2]);
    d[j] = R[j] * dc[0] + R[3 + j] * dc[1] + R[6 + j] * dc[2];
  }
  return 1;
}

/* ------------------------------------------------------------------ spherical harmonics */

/* Real spherical harmonics with the Condon-Shortley phase, orthonormal on the sphere,
 * for the unit direction d, degrees 0..deg, index l*l + l + m (m = -l..l).
 * Built from associated Legendre functions P_l^m (three-term recurrence) divided by
 * (1 - z^2)^{m/2}, times Re / Im of (x + i y)^m.  (Radiance phi_beta(d), Sec. 3.) */
void orc_sh_basis(int deg, const double dir[3], double *Y) {
  double x = dir[0], y = dir[1], z = dir[2];
  double cm = 1.0, sm = 0.0; /* Re, Im of (x + i y)^m */
  double pmm = 1.0;          /* (-1)^m (2m-1)!! */
  for (int m = 0; m <= deg; ++m) {
    if (m > 0) {
      double ncm = cm * x - sm * y, nsm = cm * y + sm * x;
      cm = ncm; sm = nsm;
      pmm *= -(2.0 * m - 1.0);
    }
    double p_lm2 = 0.0, p_lm1 = 0.0;
    for (int l = m; l <= deg; ++l) {
      double p;
      if (l == m) p = pmm;
      else if (l == m + 1) p = z * (2.0 * m + 1.0) * pmm;
      else p = ((2.0 * l - 1.0) * z * p_lm1 - (l + m - 1.0) * p_lm2) / (double)(l - m);
      p_lm2 = p_lm1; p_lm1 = p;
      double ratio = 1.0; /* (l-m)!/(l+m)! */
      for (int f = l - m + 1; f <= l + m; ++f) ratio /= (double)f;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * ratio);
      if (m == 0) Y[l * l + l] = K * p;
      else {
        Y[l * l + l + m] = sqrt(2.0) * K * cm * p;
        Y[l * l + l - m] = sqrt(2.0) * K * sm * p;
      }
    }
  }
}

/* Gradient of the basis polynomials of orc_sh_basis with respect to (x, y, z), carried through
 * the same recurrences (forward-mode): d/dx (x + i y)^m = m (x + i y)^(m-1) and
 * d/dy (x + i y)^m = i m (x + i y)^(m-1) via the product rule on cm, sm; the Legendre part
 * depends on z alone.  G[16 j + k] = dY_k / d(dir_j) for j = x, y, z (the polynomial's
 * gradient; the derivative along the unit sphere is its tangential part). */
void orc_sh_basis_grad(int deg, const double dir[3], double *Y, double *G) {
  double x = dir[0], y = dir[1], z = dir[2];
  double cm = 1.0, sm = 0.0, cmx = 0.0, cmy = 0.0, smx = 0.0, smy = 0.0;
  double pmm = 1.0;
  for (int k = 0; k < 48; ++k) G[k] = 0.0;
  for (int m = 0; m <= deg; ++m) {
    if (m > 0) {
      double ncm = cm * x - sm * y, nsm = cm * y + sm * x;
      double ncmx = cmx * x + cm - smx * y, ncmy = cmy * x - smy * y - sm;
      double nsmx = cmx * y + smx * x + sm, nsmy = cmy * y + cm + smy * x;
      cm = ncm; sm = nsm; cmx = ncmx; cmy = ncmy; smx = nsmx; smy = nsmy;
      pmm *= -(2.0 * m - 1.0);
    }
    double p_lm2 = 0.0, p_lm1 = 0.0, d_lm2 = 0.0, d_lm1 = 0.0;
    for (int l = m; l <= deg; ++l) {
      double p, dp;
      if (l == m) { p = pmm; dp = 0.0; }
      else if (l == m + 1) { p = z * (2.0 * m + 1.0) * pmm; dp = (2.0 * m + 1.0) * pmm; }
      else {
        p = ((2.0 * l - 1.0) * z * p_lm1 - (l + m - 1.0) * p_lm2) / (double)(l - m);
        dp = ((2.0 * l - 1.0) * (p_lm1 + z * d_lm1) - (l + m - 1.0) * d_lm2) / (double)(l - m);
      }
      p_lm2 = p_lm1; p_lm1 = p; d_lm2 = d_lm1; d_lm1 = dp;
      double ratio = 1.0;
      for (int f = l - m + 1; f <= l + m; ++f) ratio /= (double)f;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * ratio);
      if (m == 0) {
        int k = l * l + l;
        Y[k] = K * p;
        G[32 + k] = K * dp;
      } else {
        double s2 = sqrt(2.0) * K;
        int kc = l * l + l + m, ks = l * l + l - m;
        Y[kc] = s2 * cm * p;
        Y[ks] = s2 * sm * p;
        G[kc] = s2 * cmx * p; G[16 + kc] = s2 * cmy * p; G[32 + kc] = s2 * cm * dp;
        G[ks] = s2 * smx * p; G[16 + ks] = s2 * smy * p; G[32 + ks] = s2 * sm * dp;
      }
    }
  }
}

/* ------------------------------------------------------------------ particles */

typedef struct {
  double mu[3], s[3], qn[4], qnorm, R[9], M[9], sigma;
  int ok; /* finite parameters and a normalisable quaternion */
} orc_particle;

static void orc_load_particle(const orc_scene *sc, int i, orc_particle *p) {
  double q[4];
  p->ok = 1;
  for (int j = 0; j < 3; ++j) {
    p->mu[j] = sc->means[3 * i + j];
    p->s[j] = exp((double)sc->log_scales[3 * i + j]);
    if (!isfinite(p->mu[j]) || !isfinite(p->s[j]) || !(p->s[j] > 0)) p->ok = 0;
  }
  for (int j = 0; j < 4; ++j) q[j] = sc->quats[4 * i + j];
  p->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(p->qnorm > 0) || !isfinite(p->qnorm)) { p->ok = 0; p->qnorm = 1; q[0] = 1; q[1] = q[2] = q[3] = 0; }
  for (int j = 0; j < 4; ++j) p->qn[j] = q[j] / p->qnorm;
  double lg = sc->opacity_logits[i];
  p->sigma = 1.0 / (1.0 + exp(-lg));
  if (!isfinite(lg)) p->ok = 0;
  orc_quat_to_rot(p->qn, p->R);
  /* M = S^-1 R^T : row k is column k of R divided by s_k */
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) p->M[3 * k + j] = p->R[3 * j + k] / p->s[k];
}

/* Unscented-Transform estimate of the 2D mean and covariance of a particle
 * (Algorithm 2; eq. sigma_points, weights_1, weights_2, 2d_conic_1, 2d_conic_2).
 * Sigma points use the square root R S of Sigma = R S S^T R^T: column k is s_k R[:,k]. */
int orc_ut_estimate(const orc_camera *c, double theta_max, int rs_iters, double a, double b, double kappa,
                    const double mu[3], const double R[9], const double s[3], double vmu[2], double cov[3],
                    double *t_mean, double *margin) {
  double lam = a * a * (3.0 + kappa) - 3.0;
  double gam = sqrt(3.0 + lam);
  double wm0 = lam / (3.0 + lam), wi = 1.0 / (2.0 * (3.0 + lam));
  double wc0 = wm0 + (1.0 - a * a + b);
  double X[7][3], V[7][2];
  for (int j = 0; j < 3; ++j) X[0][j] = mu[j];
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) {
      double col = gam * s[k] * R[3 * j + k];
      X[1 + k][j] = mu[j] + col;
      X[4 + k][j] = mu[j] - col;
    }
  int valid = 1;
  double mg = INFINITY;
  for (int i = 0; i < 7; ++i) {
    double m, t;
    int v = orc_project_world(c, theta_max, rs_iters, X[i], V[i], &t, &m);
    if (i == 0 && t_mean) *t_mean = t;
    if (m < mg) mg = m;
    valid &= v;
  }
  if (margin) *margin = mg;
  if (!valid) return 0;
  vmu[0] = wm0 * V[0][0]; vmu[1] = wm0 * V[0][1];
  for (int i = 1; i < 7; ++i) { vmu[0] += wi * V[i][0]; vmu[1] += wi * V[i][1]; }
  cov[0] = cov[1] = cov[2] = 0.0;
  for (int i = 0; i < 7; ++i) {
    double w = i == 0 ? wc0 : wi;
    double dx = V[i][0] - vmu[0], dy = V[i][1] - vmu[1];
    cov[0] += w * dx * dx; cov[1] += w * dx * dy; cov[2] += w * dy * dy;
  }
  return 1;
}

/* Jacobian d g / d x_c (2x3, row-major) of the camera map at a camera-space point.
 * Pinhole: u = fx X/Z + cx.  Fisheye: u = fx s X + cx with s = theta_d(theta)/rho,
 * theta = atan2(rho, Z), so d s = (theta_d' d theta - s d rho) / rho with
 * d theta = (X Z, Y Z, -rho^2) / (rho r^2) and d rho = (X, Y, 0) / rho; on the axis (rho = 0)
 * theta_d ~ rho / Z and the map is the pinhole one.  Orthographic: u = fx X + cx.  Radial
 * pinhole: the undistorted pinhole Jacobian, as 3DGS's EWA uses (it ignores the distortion). */
static void orc_cam_jacobian(const orc_camera *c, const double xc[3], double J[6]) {
  double X = xc[0], Y = xc[1], Z = xc[2];
  if (c->model == 0 || c->model == 3) { /* radial pinhole: the undistorted Jacobian of 3DGS */
    J[0] = c->fx / Z; J[1] = 0.0; J[2] = -c->fx * X / (Z * Z);
    J[3] = 0.0; J[4] = c->fy / Z; J[5] = -c->fy * Y / (Z * Z);
  } else if (c->model == 1) {
    double rho2 = X * X + Y * Y, rho = sqrt(rho2), r2 = rho2 + Z * Z;
    if (rho > 0.0) {
      double th = atan2(rho, Z);
      double s = orc_theta_d(c->k, th) / rho, tdp = orc_theta_d_prime(c->k, th);
      double dth[3] = {X * Z / (rho * r2), Y * Z / (rho * r2), -rho / r2};
      double drho[3] = {X / rho, Y / rho, 0.0};
      double ds[3];
      for (int j = 0; j < 3; ++j) ds[j] = (tdp * dth[j] - s * drho[j]) / rho;
      J[0] = c->fx * (s + X * ds[0]); J[1] = c->fx * X * ds[1]; J[2] = c->fx * X * ds[2];
      J[3] = c->fy * Y * ds[0]; J[4] = c->fy * (s + Y * ds[1]); J[5] = c->fy * Y * ds[2];
    } else {
      J[0] = c->fx / Z; J[1] = 0.0; J[2] = 0.0;
      J[3] = 0.0; J[4] = c->fy / Z; J[5] = 0.0;
    }
  } else {
    J[0] = c->fx; J[1] = 0.0; J[2] = 0.0;
    J[3] = 0.0; J[4] = c->fy; J[5] = 0.0;
  }
}

/* First-order (EWA) estimate of the 2D mean and covariance (eq. ewa_splatting, the 3DGS
 * baseline the UT replaces): v_mu = g(W mu) and Sigma' = J W Sigma W^T J^T, J the Jacobian of g
 * at the camera-space mean.  Under a rolling shutter W is the pose at the mean's own shutter
 * time (the fixed point of orc_project_world); the dependence of the pose on the projected row
 * is not linearised.  Only the mean must project validly. */
int orc_ewa_estimate(const orc_camera *c, double theta_max, int rs_iters, const double mu[3], const double R[9],
                     const double s[3], double vmu[2], double cov[3], double *t_mean, double *margin) {
  double t = 0.0, m = INFINITY;
  int valid = orc_project_world(c, theta_max, rs_iters, mu, vmu, &t, &m);
  if (t_mean) *t_mean = t;
  if (margin) *margin = m;
  if (!valid) return 0;
  double Rc[9], Tc[3], xc[3], J[6], A[6];
  orc_pose_at(c, t, Rc, Tc);
  for (int r = 0; r < 3; ++r) xc[r] = Rc[3 * r] * mu[0] + Rc[3 * r + 1] * mu[1] + Rc[3 * r + 2] * mu[2] + Tc[r];
  orc_cam_jacobian(c, xc, J);
  /* A = J W (R S): column k is J W (s_k R[:,k]); Sigma' = A A^T */
  for (int k = 0; k < 3; ++k) {
    double col[3] = {s[k] * R[k], s[k] * R[3 + k], s[k] * R[6 + k]}, w[3];
    for (int r = 0; r < 3; ++r) w[r] = Rc[3 * r] * col[0] + Rc[3 * r + 1] * col[1] + Rc[3 * r + 2] * col[2];
    A[k] = J[0] * w[0] + J[1] * w[1] + J[2] * w[2];
    A[3 + k] = J[3] * w[0] + J[4] * w[1] + J[5] * w[2];
  }
  cov[0] = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
  cov[1] = A[0] * A[3] + A[1] * A[4] + A[2] * A[5];
  cov[2] = A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
  return 1;
}

/* The projection the options select: UT (Algorithm 2) or EWA. */
static int orc_estimate(const orc_camera *c, double theta_max, const orc_options *op, const double mu[3],
                        const double R[9], const double s[3], double vmu[2], double cov[3], double *t_mean,
                        double *margin) {
  if (op->projection == 1) return orc_ewa_estimate(c, theta_max, op->rs_iters, mu, R, s, vmu, cov, t_mean, margin);
  return orc_ut_estimate(c, theta_max, op->rs_iters, op->ut_alpha, op->ut_beta, op->ut_kappa, mu, R, s, vmu, cov,
                         t_mean, margin);
}

/* Per-particle projection (Algorithm 1): UT (or EWA) estimate, opacity-tightened extent,
 * pixel rectangle, depth, tile count.
 * Outputs (arrays of n): mean2d[2], cov2d[3], depth (FP64), depth32 (the FP64 depth rounded
 * to FP32, which enters the sort key), rect[4] = (x0,y0,x1,y1) inclusive pixel indices
 * (culled: 0,0,-1,-1), ntiles, edges[4] = unrounded (x0,x1,y0,y1) edge values before
 * clipping (NaN when unavailable), tie[n] = 1 when a culling decision is within eps_rel
 * of its threshold. */
void orc_project(const orc_scene *sc, const orc_camera *c, const orc_options *op, const orc_tol *tol,
                 double *mean2d, double *cov2d, double *depth, float *depth32, int32_t *rect,
                 int32_t *ntiles, double *edges, int32_t *tie) {
  double theta_max = orc_cam_limit(c);
  int W = c->width, H = c->height;
#pragma omp parallel for schedule(dynamic, 256)
  for (int i = 0; i < sc->n; ++i) {
    orc_particle p;
    orc_load_particle(sc, i, &p);
    int32_t *r = rect + 4 * i;
    r[0] = 0; r[1] = 0; r[2] = -1; r[3] = -1;
    ntiles[i] = 0;
    depth[i] = 0.0; depth32[i] = 0.0f;
    mean2d[2 * i] = mean2d[2 * i + 1] = NAN;
    cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = NAN;
    for (int j = 0; j < 4; ++j) edges[4 * i + j] = NAN;
    tie[i] = 0;
    if (!p.ok) continue;
    double sig_margin = (p.sigma - op->alpha_min) / op->alpha_min;
    if (fabs(sig_margin) < tol->eps_rel) tie[i] = 1;
    double vmu[2], cov[3], tmu = 0.0, vm;
    int valid = orc_estimate(c, theta_max, op, p.mu, p.R, p.s, vmu, cov, &tmu, &vm);
    if (fabs(vm) < tol->eps_rel) tie[i] = 1;
    if (!valid) {
      if (tie[i]) {
        /* a near-valid particle: estimate its footprint anyway so that pixels under it get flagged */
        orc_camera c2 = *c;
        c2.near_plane = 1e-9;
        /* the polynomial fisheye extends to the whole sphere but the pole behind the camera */
        double th2 = c->model == 1 ? ORC_PI : theta_max;
        if (orc_estimate(&c2, th2, op, p.mu, p.R, p.s, vmu, cov, NULL, NULL)) {
          double k = op->extent_sigma;
          double hx = k * sqrt(cov[0]), hy = k * sqrt(cov[2]);
          edges[4 * i + 0] = vmu[0] - hx - 0.5; edges[4 * i + 1] = vmu[0] + hx - 0.5;
          edges[4 * i + 2] = vmu[1] - hy - 0.5; edges[4 * i + 3] = vmu[1] + hy - 0.5;
        }
      }
      continue;
    }
    mean2d[2 * i] = vmu[0]; mean2d[2 * i + 1] = vmu[1];
    cov2d[3 * i] = cov[0]; cov2d[3 * i + 1] = cov[1]; cov2d[3 * i + 2] = cov[2];
    /* depth: distance from the camera centre to the mean at the mean's shutter time */
    double Rm[9], Tm[3], xc[3];
    orc_pose_at(c, tmu, Rm, Tm);
    for (int rr = 0; rr < 3; ++rr)
      xc[rr] = Rm[3 * rr] * p.mu[0] + Rm[3 * rr + 1] * p.mu[1] + Rm[3 * rr + 2] * p.mu[2] + Tm[rr];
    double dep = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
    depth[i] = dep;
    depth32[i] = (float)dep;
    if (!(p.sigma >= op->alpha_min)) continue;
    /* opacity-tightened extent: the Mahalanobis distance where sigma rho falls to alpha_min
     * (Gaussian: sqrt(2 ln(sigma / alpha_min)); degree n: (2 ln(sigma / alpha_min) 3^(n-2))^(1/n)), capped */
    int kn = op->kernel_degree > 0 ? op->kernel_degree : 2;
    double k = kn == 2 ? sqrt(2.0 * log(p.sigma / op->alpha_min))
                       : pow(2.0 * log(p.sigma / op->alpha_min) * pow(3.0, kn - 2.0), 1.0 / kn);
    if (k > op->extent_sigma) k = op->extent_sigma;
    double hx = k * sqrt(cov[0]), hy = k * sqrt(cov[2]);
    double e0 = vmu[0] - hx - 0.5, e1 = vmu[0] + hx - 0.5, e2 = vmu[1] - hy - 0.5, e3 = vmu[1] + hy - 0.5;
    edges[4 * i + 0] = e0; edges[4 * i + 1] = e1; edges[4 * i + 2] = e2; edges[4 * i + 3] = e3;
    if (!isfinite(e0) || !isfinite(e1) || !isfinite(e2) || !isfinite(e3)) continue;
    double x0 = ceil(e0), x1 = floor(e1), y0 = ceil(e2), y1 = floor(e3);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    if (x0 > x1 || y0 > y1) continue;
    r[0] = (int32_t)x0; r[1] = (int32_t)y0; r[2] = (int32_t)x1; r[3] = (int32_t)y1;
    int tx0 = r[0] / op->tile_w, tx1 = r[2] / op->tile_w, ty0 = r[1] / op->tile_h, ty1 = r[3] / op->tile_h;
    ntiles[i] = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
  }
}

/* ------------------------------------------------------------------ duplicate + sort */

typedef struct { uint64_t key; uint64_t seq; uint32_t val; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b) {
  const orc_kv *x = (const orc_kv *)a, *y = (const orc_kv *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->seq != y->seq) return x->seq < y->seq ? -1 : 1;
  return 0;
}

static uint32_t orc_f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Number of duplicated keys for the given rects. */
int64_t orc_count_keys(int n, const int32_t *rect, int tile_w, int tile_h) {
  int64_t K = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t *r = rect + 4 * i;
    if (r[0] > r[2] || r[1] > r[3]) continue;
    K += (int64_t)(r[2] / tile_w - r[0] / tile_w + 1) * (r[3] / tile_h - r[1] / tile_h + 1);
  }
  return K;
}

/* Duplicate (Table 2, "Duplicate"): one key (tile << 32 | bits(depth32)) per tile a particle's
 * rect overlaps, particles in index order, tiles row-major; then a stable sort ("Sort"), and
 * per-tile ranges [start, end) into the sorted list (empty tiles: [0, 0)).
 * keys/vals must hold orc_count_keys() entries; ranges holds 2 * tiles_x * tiles_y. */
void orc_bin(int n, const float *depth32, const int32_t *rect, int W, int H, int tile_w, int tile_h,
             uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
  int tx = (W + tile_w - 1) / tile_w, ty = (H + tile_h - 1) / tile_h;
  int64_t K = orc_count_keys(n, rect, tile_w, tile_h);
  orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (size_t)(K > 0 ? K : 1));
  int64_t e = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t *r = rect + 4 * i;
    if (r[0] > r[2] || r[1] > r[3]) continue;
    for (int y = r[1] / tile_h; y <= r[3] / tile_h; ++y)
      for (int x = r[0] / tile_w; x <= r[2] / tile_w; ++x) {
        uint64_t tile = (uint64_t)y * tx + x;
        kv[e].key = (tile << 32) | orc_f32_bits(depth32[i]);
        kv[e].seq = (uint64_t)e;
        kv[e].val = (uint32_t)i;
        ++e;
      }
  }
  qsort(kv, (size_t)K, sizeof(orc_kv), orc_kv_cmp);
  for (int t = 0; t < tx * ty; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
  for (int64_t j = 0; j < K; ++j) {
    keys[j] = kv[j].key;
    vals[j] = kv[j].val;
    uint32_t t = (uint32_t)(kv[j].key >> 32);
    if (j == 0 || (uint32_t)(kv[j - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)j;
    if (j == K - 1 || (uint32_t)(kv[j + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
  }
  free(kv);
}

/* ------------------------------------------------------------------ compositing */

typedef struct {
  int n, deg, nsh;
  orc_particle *P;
  const int32_t *rect;
  const float *depth32;
  const double *edges;
  const int32_t *tie;
  int32_t *order; /* valid particles sorted by (bits(depth32), index) */
  int norder;
  int32_t *tie_list;
  int ntie;
  double *Yp;    /* colour_mode 1: SH basis at each particle's direction [n][16] */
  double *dYdmu; /* colour_mode 1: its derivative with respect to the mean [n][3][16] */
} orc_ctx;

static const float *orc_depth_sort_key;
static int orc_order_cmp(const void *a, const void *b) {
  int i = *(const int32_t *)a, j = *(const int32_t *)b;
  uint32_t ki = orc_f32_bits(orc_depth_sort_key[i]), kj = orc_f32_bits(orc_depth_sort_key[j]);
  if (ki != kj) return ki < kj ? -1 : 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

static void orc_ctx_init(orc_ctx *x, const orc_scene *sc, const int32_t *rect, const float *depth32,
                         const double *edges, const int32_t *tie) {
  x->n = sc->n;
  x->deg = sc->sh_degree;
  x->nsh = (sc->sh_degree + 1) * (sc->sh_degree + 1);
  x->P = (orc_particle *)malloc(sizeof(orc_particle) * (size_t)(sc->n > 0 ? sc->n : 1));
  x->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sc->n > 0 ? sc->n : 1));
  x->tie_list = (int32_t *)malloc(sizeof(int32_t) * (size_t)(sc->n > 0 ? sc->n : 1));
  x->rect = rect; x->depth32 = depth32; x->edges = edges; x->tie = tie;
  x->norder = 0; x->ntie = 0;
  x->Yp = NULL; x->dYdmu = NULL;
  for (int i = 0; i < sc->n; ++i) {
    orc_load_particle(sc, i, &x->P[i]);
    const int32_t *r = rect + 4 * i;
    if (x->P[i].ok && r[0] <= r[2] && r[1] <= r[3]) x->order[x->norder++] = i;
    if (tie && tie[i]) x->tie_list[x->ntie++] = i;
  }
  orc_depth_sort_key = depth32;
  qsort(x->order, (size_t)x->norder, sizeof(int32_t), orc_order_cmp);
}

static void orc_ctx_free(orc_ctx *x) { free(x->P); free(x->order); free(x->tie_list); free(x->Yp); free(x->dYdmu); }

/* Colour direction of a particle in colour_mode 1: the unit vector from the camera centre
 * -R(t)^T T(t), at the mean's shutter time t (the fixed point of orc_project_world), to mu. */
static void orc_particle_dir(const orc_camera *c, double theta_max, int rs_iters, const double mu[3],
                             double dir[3]) {
  double uv[2], t = 0.0, m, R[9], T[3], v[3];
  orc_project_world(c, theta_max, rs_iters, mu, uv, &t, &m);
  orc_pose_at(c, t, R, T);
  for (int j = 0; j < 3; ++j) v[j] = mu[j] + (R[j] * T[0] + R[3 + j] * T[1] + R[6 + j] * T[2]);
  double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int j = 0; j < 3; ++j) dir[j] = v[j] / nv;
}

/* colour_mode 1: the SH basis at every particle's direction, and its derivative with respect
 * to the mean, analytic (orc_sh_basis_grad; the shutter time, like the whole projection, is a
 * discrete selection and carries no gradient: it is held fixed). */
static void orc_ctx_colour(orc_ctx *x, const orc_camera *c, double theta_max, const orc_options *op) {
  size_t n = (size_t)(x->n > 0 ? x->n : 1);
  x->Yp = (double *)calloc(n * 16, sizeof(double));
  x->dYdmu = (double *)calloc(n * 48, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
  for (int q = 0; q < x->norder; ++q) {
    int i = x->order[q];
    const orc_particle *p = &x->P[i];
    double dir[3], uv[2], t = 0.0, m, R[9], T[3], C[3];
    orc_particle_dir(c, theta_max, op->rs_iters, p->mu, dir);
    orc_sh_basis(x->deg, dir, x->Yp + 16 * (size_t)i);
    orc_project_world(c, theta_max, op->rs_iters, p->mu, uv, &t, &m);
    orc_pose_at(c, t, R, T);
    for (int j = 0; j < 3; ++j) C[j] = -(R[j] * T[0] + R[3 + j] * T[1] + R[6 + j] * T[2]);
    double v[3] = {p->mu[0] - C[0], p->mu[1] - C[1], p->mu[2] - C[2]};
    /* dY/dmu = (I - dir dir^T) grad Y(dir) / |mu - C|, the camera centre C held at the mean's
     * shutter time; the basis polynomials' gradient analytically */
    double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]), Yd[16], G[48];
    orc_sh_basis_grad(x->deg, dir, Yd, G);
    for (int k = 0; k < x->nsh; ++k) {
      double gd = G[k] * dir[0] + G[16 + k] * dir[1] + G[32 + k] * dir[2];
      for (int j = 0; j < 3; ++j) x->dYdmu[48 * (size_t)i + 16 * j + k] = (G[16 * j + k] - gd * dir[j]) / len;
    }
  }
}

/* Maximum response of particle p along the ray o + tau d (eq. GaussianMaxResponse):
 * o_g = S^-1 R^T (o - mu), d_g = S^-1 R^T d, tau_max = -o_g.d_g / d_g.d_g, and the squared
 * canonical distance omega^2 = |o_g + tau_max d_g|^2 = |o_g x d_g|^2 / |d_g|^2. */
static double orc_omega2(const orc_particle *p, const double o[3], const double d[3], double og[3], double dg[3],
                         double *tau) {
  double om[3] = {o[0] - p->mu[0], o[1] - p->mu[1], o[2] - p->mu[2]};
  for (int k = 0; k < 3; ++k) {
    og[k] = p->M[3 * k] * om[0] + p->M[3 * k + 1] * om[1] + p->M[3 * k + 2] * om[2];
    dg[k] = p->M[3 * k] * d[0] + p->M[3 * k + 1] * d[1] + p->M[3 * k + 2] * d[2];
  }
  double dd = dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2];
  double od = og[0] * dg[0] + og[1] * dg[1] + og[2] * dg[2];
  double cx = og[1] * dg[2] - og[2] * dg[1], cy = og[2] * dg[0] - og[0] * dg[2], cz = og[0] * dg[1] - og[1] * dg[0];
  *tau = -od / dd;
  return (cx * cx + cy * cy + cz * cz) / dd;
}

/* Maximum response along the ray for the kernel of degree n (supplementary Sec. A): the
 * generalised Gaussian exp(-lambda d^n) of the Mahalanobis distance d, with lambda chosen so
 * that the response at d = r = 3 equals the Gaussian's exp(-r^2/2), i.e.
 * rho = exp(-1/2 3^(2-n) (omega^2)^(n/2)); it peaks at the same tau_max as the Gaussian
 * (it is decreasing in d).  n = 2 is eq. gaussian_kernel. */
static double orc_response(const orc_options *op, double w2) {
  int n = op->kernel_degree > 0 ? op->kernel_degree : 2;
  if (n == 2) return exp(-0.5 * w2);
  return exp(-0.5 * pow(3.0, 2.0 - n) * pow(w2, 0.5 * n));
}

/* d rho / d omega^2 */
static double orc_dresponse(const orc_options *op, double w2, double rho) {
  int n = op->kernel_degree > 0 ? op->kernel_degree : 2;
  if (n == 2) return -0.5 * rho;
  return -0.5 * pow(3.0, 2.0 - n) * 0.5 * n * pow(w2, 0.5 * n - 1.0) * rho;
}

typedef struct {
  int i;
  double alpha, a, T, rho, tau, w2, og[3], dg[3], raw[3], col[3];
} orc_contrib;

/* Bounds a pixel's FP32 result may legitimately differ by from this FP64 one (all >= 0):
 * slack / aslack for reorderings of depth-tied pairs and stop-threshold ties (exact effects),
 * fslack / faslack for the other flagged decisions (a bound on what flipping them can do). */
typedef struct {
  double slack, aslack, fslack, faslack, rslack, raslack;
} orc_slack;

/* Bound on the FP32 rounding of a blended particle's alpha.  The response is evaluated from the
 * canonical-frame ray o_g = M (o - mu), d_g = M d: o - mu (and the ray) are known to about
 * u (|o| + |mu|) in FP32 (u = 2^-24), so the ray's Mahalanobis distance omega carries an
 * absolute error of about u |M|_F (|o| + |mu|), which the response's slope turns into
 * |d alpha| = |d alpha / d omega^2| 2 omega |d omega|.  For a particle much smaller than its
 * distance (|M| large) this dominates every other rounding.  The factor 2 covers the two
 * roundings on the way (o - mu, then M times it); |M|_F >= |M|_2 and |o| + |mu| >= |o - mu|
 * already make the estimate an upper one. */
static double orc_alpha_rounding(const orc_options *op, const orc_particle *p, const double o[3], double w2,
                                 double rho) {
  double mf = 0.0, on = 0.0, mn = 0.0;
  for (int j = 0; j < 9; ++j) mf += p->M[j] * p->M[j];
  for (int j = 0; j < 3; ++j) {
    on += o[j] * o[j];
    mn += p->mu[j] * p->mu[j];
  }
  const double u = ldexp(1.0, -24);
  const double dw = 2.0 * u * sqrt(mf) * (sqrt(on) + sqrt(mn));
  return fabs(p->sigma * orc_dresponse(op, w2, rho)) * 2.0 * sqrt(w2) * dw;
}

/* Composites one pixel ray over the particles in `order` (eq. QuadratureVolumeRendering with
 * alpha_i = sigma_i rho_i at tau_max).  Returns the number of blended particles; fills rgb, T.
 * When `rec` is given, records every blended particle (up to cap).
 * Depth near-ties: two consecutive blended particles whose FP32 depth keys are within
 * depth_ulps may legitimately come in either order from an FP32 depth; swapping them changes
 * the colour by exactly T_i alpha_i alpha_j (c_j - c_i), which is added to sl->slack.  Three or
 * more in a row set ORC_F_DEPTH_TIE instead.  A transmittance T (1 - alpha) within eps_t of t_min
 * may stop one particle earlier or later: its T alpha c is added to sl->slack and T alpha to
 * sl->aslack.
 * Flip bounds: a flagged decision about one particle (membership at a rect edge, alpha_min,
 * the alpha_max clamp, the order inside a run of three or more depth ties) changes what that
 * particle adds, T alpha c, by at most T dalpha c (dalpha = its alpha, or the clamp's change),
 * and scales what comes after it, T (1 - alpha) S with S <= the largest colour c_max among the
 * particles this ray evaluates, by at most T dalpha c_max; so sl->fslack = sum over flagged
 * decisions of T dalpha (c + c_max) (+ t_min c_max for a stop that moves), and sl->faslack =
 * sum of T dalpha (+ t_min).  The same two terms with dalpha = the FP32 rounding bound of each
 * blended particle's alpha (orc_alpha_rounding) give sl->rslack / sl->raslack. */
static int orc_composite_ray(const orc_ctx *x, const orc_scene *sc, const orc_options *op, const orc_tol *tol,
                             int px, int py, const double o[3], const double d[3], const double *Y, double rgb[3],
                             double *Tout, int32_t *flags, orc_contrib *rec, int cap, int no_rect, orc_slack *sl) {
  double T = 1.0;
  int nb = 0;
  uint32_t last_bits = 0;
  int have_last = 0, last_tie = 0;
  double last_alpha = 0.0, last_T = 1.0, last_col[3] = {0, 0, 0}, last_cmax = 0.0;
  double fb_c = 0.0, fb_a = 0.0, cmax_seen = 0.0, rb_c = 0.0, rb_a = 0.0;
  int n_events = 0;
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  if (sl) sl->slack = sl->aslack = sl->fslack = sl->faslack = sl->rslack = sl->raslack = 0.0;
  for (int j = 0; j < x->norder; ++j) {
    int i = x->order[j];
    const orc_particle *p = &x->P[i];
    const int32_t *r = x->rect + 4 * i;
    int inside = px >= r[0] && px <= r[2] && py >= r[1] && py <= r[3];
    double og[3], dg[3], tau;
    const float *beta = sc->sh + (size_t)i * x->nsh * 3;
    const double *Yc = op->colour_mode == 1 ? x->Yp + 16 * (size_t)i : Y;
    if (!inside && !no_rect) {
      /* only a rect edge within eps of this pixel could flip membership */
      if (x->edges && flags) {
        const double *e = x->edges + 4 * i;
        double ex = fmin(fabs(px - e[0]), fabs(px - e[1])), ey = fmin(fabs(py - e[2]), fabs(py - e[3]));
        int nx = px >= e[0] - tol->eps_px && px <= e[1] + tol->eps_px;
        int ny = py >= e[2] - tol->eps_px && py <= e[3] + tol->eps_px;
        if (nx && ny && (ex < tol->eps_px || ey < tol->eps_px) && px >= 0 && py >= 0) {
          double w2 = orc_omega2(p, o, d, og, dg, &tau);
          double ao = p->sigma * orc_response(op, w2);
          if (ao >= op->alpha_min * (1.0 - tol->eps_rel)) {
            *flags |= ORC_F_RECT_EDGE;
            double co = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
              double v = 0.5;
              for (int kk = 0; kk < x->nsh; ++kk) v += beta[3 * kk + ch] * Yc[kk];
              co = fmax(co, v);
            }
            double al = ao < op->alpha_max ? ao : op->alpha_max;
            fb_c += T * al * co;
            fb_a += T * al;
            cmax_seen = fmax(cmax_seen, co);
            ++n_events;
          }
        }
      }
      continue;
    }
    double w2 = orc_omega2(p, o, d, og, dg, &tau);
    double rho = orc_response(op, w2);
    double a = p->sigma * rho;
    double raw[3], col[3], cmax = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      double v = 0.5;
      for (int kk = 0; kk < x->nsh; ++kk) v += beta[3 * kk + ch] * Yc[kk];
      raw[ch] = v;
      col[ch] = v > 0.0 ? v : 0.0;
      cmax = fmax(cmax, col[ch]);
    }
    double alpha = a < op->alpha_max ? a : op->alpha_max;
    int event = 0;
    if (flags && x->edges && !no_rect) {
      const double *e = x->edges + 4 * i;
      double ex = fmin(fabs(px - e[0]), fabs(px - e[1])), ey = fmin(fabs(py - e[2]), fabs(py - e[3]));
      if ((ex < tol->eps_px || ey < tol->eps_px) && a >= op->alpha_min * (1.0 - tol->eps_rel)) {
        *flags |= ORC_F_RECT_EDGE;
        event = 1;
      }
    }
    if (flags && fabs(a - op->alpha_min) < tol->eps_rel * op->alpha_min) {
      *flags |= ORC_F_ALPHA_MIN;
      event = 1;
    }
    if (a >= op->alpha_min * (1.0 - tol->eps_rel)) cmax_seen = fmax(cmax_seen, cmax);
    if (event) {
      fb_c += T * alpha * cmax;
      fb_a += T * alpha;
      ++n_events;
    }
    if (a < op->alpha_min) continue;
    if (flags && fabs(a - op->alpha_max) < tol->eps_rel * op->alpha_max) {
      *flags |= ORC_F_ALPHA_MAX;
      double da = fabs(a - op->alpha_max);
      fb_c += T * da * cmax;
      fb_a += T * da;
      ++n_events;
    }
    double Tn = T * (1.0 - alpha);
    if (fabs(Tn - op->t_min) < tol->eps_t * op->t_min) {
      /* the stop decision may flip: this one particle is blended or not (and at most one more
       * after it, whose T is already below t_min) */
      if (flags) *flags |= ORC_F_TSTOP;
      if (sl) {
        sl->slack += T * alpha * cmax;
        sl->aslack += T * alpha;
      }
    }
    if (Tn < op->t_min) break;
    if (flags && orc_clamp_tie(beta, Yc, x->nsh, raw, tol->eps_rel)) *flags |= ORC_F_CLAMP;
    uint32_t bits = orc_f32_bits(x->depth32[i]);
    for (int ch = 0; ch < 3; ++ch) rgb[ch] += col[ch] * alpha * T;
    if (sl && a <= op->alpha_max) {
      const double dr = orc_alpha_rounding(op, p, o, w2, rho);
      rb_c += T * dr * cmax;
      rb_a += T * dr;
    }
    if (have_last && (int64_t)bits - (int64_t)last_bits <= tol->depth_ulps) {
      if (flags && last_tie) {
        /* a run of three or more: the order inside it is bounded, not tracked */
        *flags |= ORC_F_DEPTH_TIE;
        fb_c += T * alpha * cmax + last_T * last_alpha * last_cmax;
        fb_a += T * alpha + last_T * last_alpha;
        ++n_events;
      }
      double dc = 0.0;
      for (int ch = 0; ch < 3; ++ch) dc = fmax(dc, fabs(col[ch] - last_col[ch]));
      if (sl) sl->slack += last_T * last_alpha * alpha * dc;
      last_tie = 1;
    } else {
      last_tie = 0;
    }
    last_bits = bits; have_last = 1;
    last_alpha = alpha; last_T = T; last_cmax = cmax;
    for (int ch = 0; ch < 3; ++ch) last_col[ch] = col[ch];
    if (rec && nb < cap) {
      orc_contrib *c = &rec[nb];
      c->i = i; c->alpha = alpha; c->a = a; c->T = T; c->rho = rho; c->tau = tau; c->w2 = w2;
      for (int k = 0; k < 3; ++k) { c->og[k] = og[k]; c->dg[k] = dg[k]; c->raw[k] = raw[k]; c->col[k] = col[k]; }
    }
    ++nb;
    T = Tn;
  }
  if (sl && n_events) {
    sl->fslack = fb_c + fb_a * cmax_seen + op->t_min * cmax_seen;
    sl->faslack = fb_a + op->t_min;
  }
  if (sl) {
    sl->rslack = rb_c + rb_a * cmax_seen;
    sl->raslack = rb_a;
  }
  *Tout = T;
  return nb;
}

/* "Ours (sorted)" (Sec. 4.4): the per-ray k-buffer of the multi-layer alpha blending
 * approximation.  Hits (particles with sigma rho >= alpha_min, met in the global depth order)
 * enter a buffer of at most k entries; when a hit arrives at a full buffer, the closest of the
 * buffered hits and the new one -- smallest tau_max, earlier arrival on equal tau -- is blended
 * (front to back, with the same stop rule) and leaves; the new hit takes its place unless it
 * was itself the closest.  At the end of the list the remaining entries are blended in
 * ascending tau.  Returns the number of blended particles.  A selection whose runner-up tau is
 * within eps_tau (relative) of the chosen one may go the other way in FP32: ORC_F_DEPTH_TIE.
 * Bound on what any flagged decision can change (slack, aslack, when given): the decisions
 * before the first flagged one are the same on both sides, so the colour composited up to it
 * is the same, and what follows adds at most T_f c_max per channel to either side's colour
 * (T_f the transmittance at the first flagged decision, c_max the largest clamped colour
 * channel of any particle that could be a hit at this pixel) and moves T_final within [0, T_f];
 * a pixel flagged by the ray setup takes T_f = 1. */
typedef struct {
  double tau, alpha, col[3];
  int seq;
  orc_contrib c; /* everything the backward needs of this (pixel, particle) pair */
} orc_kb_entry;

static int orc_kb_pick(const orc_kb_entry *e, int n, double eps, int *tie) {
  int best = 0;
  for (int j = 1; j < n; ++j)
    if (e[j].tau < e[best].tau || (e[j].tau == e[best].tau && e[j].seq < e[best].seq)) best = j;
  for (int j = 0; j < n; ++j)
    if (j != best && fabs(e[j].tau - e[best].tau) <= eps * fabs(e[best].tau)) *tie = 1;
  return best;
}

static int orc_composite_ray_kbuffer(const orc_ctx *x, const orc_scene *sc, const orc_options *op,
                                     const orc_tol *tol, int px, int py, const double o[3], const double d[3],
                                     const double *Y, double rgb[3], double *Tout, int32_t *flags,
                                     int *stopped_out, orc_contrib *rec, int cap, double *slack, double *aslack) {
  orc_kb_entry buf[65];
  int k = op->kbuffer < 64 ? op->kbuffer : 64, nbuf = 0, nb = 0, seq = 0, stopped = 0, tie = 0;
  double T = 1.0;
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  /* transmittance at the first flagged decision (-1: none yet), largest possible hit colour */
  double Tf = flags && (*flags & (ORC_F_PIXEL_EDGE | ORC_F_ILL_COND)) ? 1.0 : -1.0, cmax = 0.0;
#define ORC_KB_NOTE() do { if (Tf < 0.0) Tf = T; } while (0)
  for (int j = 0; j < x->norder && !stopped; ++j) {
    int i = x->order[j];
    const orc_particle *p = &x->P[i];
    const int32_t *r = x->rect + 4 * i;
    const int inside = px >= r[0] && px <= r[2] && py >= r[1] && py <= r[3];
    double og[3], dg[3], tau;
    double w2 = orc_omega2(p, o, d, og, dg, &tau);
    double rho = orc_response(op, w2);
    double a = p->sigma * rho;
    if (flags && x->edges) {  /* membership may flip where a rect edge is within eps_px of the pixel */
      const double *e = x->edges + 4 * i;
      double ex = fmin(fabs(px - e[0]), fabs(px - e[1])), ey = fmin(fabs(py - e[2]), fabs(py - e[3]));
      int nx = px >= e[0] - tol->eps_px && px <= e[1] + tol->eps_px;
      int ny = py >= e[2] - tol->eps_px && py <= e[3] + tol->eps_px;
      if (nx && ny && (ex < tol->eps_px || ey < tol->eps_px) && a >= op->alpha_min * (1.0 - tol->eps_rel)) {
        *flags |= ORC_F_RECT_EDGE;
        ORC_KB_NOTE();
        if (slack) {  /* a hit on the other side: its colour counts for c_max */
          const float *bt = sc->sh + (size_t)i * x->nsh * 3;
          const double *Yc = op->colour_mode == 1 ? x->Yp + 16 * (size_t)i : Y;
          for (int ch = 0; ch < 3; ++ch) {
            double s = 0.5;
            for (int kk = 0; kk < x->nsh; ++kk) s += bt[3 * kk + ch] * Yc[kk];
            if (s > cmax) cmax = s;
          }
        }
      }
    }
    if (!inside) continue;
    if (flags && fabs(a - op->alpha_min) < tol->eps_rel * op->alpha_min) { *flags |= ORC_F_ALPHA_MIN; ORC_KB_NOTE(); }
    if (a < op->alpha_min) {
      if (slack && flags && a >= op->alpha_min * (1.0 - tol->eps_rel)) {  /* a near-threshold miss: c_max */
        const float *bt = sc->sh + (size_t)i * x->nsh * 3;
        const double *Yc = op->colour_mode == 1 ? x->Yp + 16 * (size_t)i : Y;
        for (int ch = 0; ch < 3; ++ch) {
          double s = 0.5;
          for (int kk = 0; kk < x->nsh; ++kk) s += bt[3 * kk + ch] * Yc[kk];
          if (s > cmax) cmax = s;
        }
      }
      continue;
    }
    if (flags && fabs(a - op->alpha_max) < tol->eps_rel * op->alpha_max) { *flags |= ORC_F_ALPHA_MAX; ORC_KB_NOTE(); }
    orc_kb_entry h;
    h.tau = tau;
    h.alpha = a < op->alpha_max ? a : op->alpha_max;
    h.seq = seq++;
    const float *beta = sc->sh + (size_t)i * x->nsh * 3;
    const double *Yc = op->colour_mode == 1 ? x->Yp + 16 * (size_t)i : Y;
    for (int ch = 0; ch < 3; ++ch) {
      double s = 0.5;
      for (int kk = 0; kk < x->nsh; ++kk) s += beta[3 * kk + ch] * Yc[kk];
      h.col[ch] = s > 0.0 ? s : 0.0;
      h.c.raw[ch] = s;
      h.c.col[ch] = h.col[ch];
      if (h.col[ch] > cmax) cmax = h.col[ch];
    }
    if (flags && orc_clamp_tie(beta, Yc, x->nsh, h.c.raw, tol->eps_rel)) { *flags |= ORC_F_CLAMP; ORC_KB_NOTE(); }
    h.c.i = i; h.c.alpha = h.alpha; h.c.a = a; h.c.rho = rho; h.c.tau = tau; h.c.w2 = w2;
    for (int kk = 0; kk < 3; ++kk) { h.c.og[kk] = og[kk]; h.c.dg[kk] = dg[kk]; }
    if (nbuf < k) { buf[nbuf++] = h; continue; }
    buf[nbuf] = h;  /* the closest of the k buffered hits and the new one is blended */
    int b = orc_kb_pick(buf, nbuf + 1, op->eps_tau, &tie);
    if (tie) ORC_KB_NOTE();
    double Tn = T * (1.0 - buf[b].alpha);
    if (flags && fabs(Tn - op->t_min) < tol->eps_t * op->t_min) { *flags |= ORC_F_TSTOP; ORC_KB_NOTE(); }
    if (Tn < op->t_min) { stopped = 1; break; }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] += buf[b].col[ch] * buf[b].alpha * T;
    if (rec && nb < cap) { rec[nb] = buf[b].c; rec[nb].T = T; }
    T = Tn;
    ++nb;
    buf[b] = buf[nbuf];
  }
  while (!stopped && nbuf > 0) {  /* end of the list: the rest in ascending tau */
    int b = orc_kb_pick(buf, nbuf, op->eps_tau, &tie);
    if (tie) ORC_KB_NOTE();
    double Tn = T * (1.0 - buf[b].alpha);
    if (flags && fabs(Tn - op->t_min) < tol->eps_t * op->t_min) { *flags |= ORC_F_TSTOP; ORC_KB_NOTE(); }
    if (Tn < op->t_min) { stopped = 1; break; }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] += buf[b].col[ch] * buf[b].alpha * T;
    if (rec && nb < cap) { rec[nb] = buf[b].c; rec[nb].T = T; }
    T = Tn;
    ++nb;
    buf[b] = buf[--nbuf];
  }
#undef ORC_KB_NOTE
  if (flags && tie) *flags |= ORC_F_DEPTH_TIE;
  if (slack) *slack = Tf > 0.0 ? Tf * cmax : 0.0;
  if (aslack) *aslack = Tf > 0.0 ? Tf : 0.0;
  *Tout = T;
  if (stopped_out) *stopped_out = stopped;
  return nb;
}

static void orc_pixel_setup(const orc_camera *c, double theta_max, int deg, int px, int py, const orc_tol *tol,
                            double o[3], double d[3], double *Y, int *valid, int32_t *flags) {
  double em, dp;
  *valid = orc_pixel_ray(c, theta_max, px + 0.5, py + 0.5, o, d, &em, &dp);
  if (flags && (c->model == 1 || c->model == 3) && fabs(em) < tol->eps_rel) *flags |= ORC_F_PIXEL_EDGE;
  if (!*valid) { if (flags) *flags |= ORC_F_INVALID_PIXEL; return; }
  if (flags && dp < tol->cond_min) *flags |= ORC_F_ILL_COND;
  double nd = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double dh[3] = {d[0] / nd, d[1] / nd, d[2] / nd};
  orc_sh_basis(deg, dh, Y);
}

/* Renders the listed pixels by brute force over all particles in global depth order.
 * rect / depth32 / valid come from orc_project or are given directly (synthetic).
 * edges / tie may be NULL (then no near-tie flags of those kinds).  no_rect != 0 evaluates
 * every particle at every pixel (culling disabled).
 * Outputs per listed pixel: rgb[3], alpha = 1 - T_final, tfinal, nblend, flags, slack / aslack =
 * the largest colour / opacity change that FP32 depth ties and stop-threshold ties can cause, and
 * fslack / faslack (nullable) = a bound on what the other flagged decisions can change, and
 * rslack / raslack (nullable) = the FP32 rounding bound of the blended particles' alphas (see
 * orc_composite_ray; the k-buffer path leaves these at 0). */
void orc_render(const orc_scene *sc, const orc_camera *c, const orc_options *op, const orc_tol *tol,
                const int32_t *rect, const float *depth32, const double *edges, const int32_t *tie, int npix,
                const int32_t *pix_x, const int32_t *pix_y, int no_rect, double *rgb, double *alpha,
                double *tfinal, int32_t *nblend, int32_t *flags, double *slack, double *aslack, double *fslack,
                double *faslack, double *rslack, double *raslack) {
  orc_ctx x;
  orc_ctx_init(&x, sc, rect, depth32, edges, tie);
  double theta_max = orc_cam_limit(c);
  if (op->colour_mode == 1) orc_ctx_colour(&x, c, theta_max, op);
#pragma omp parallel for schedule(dynamic, 4)
  for (int q = 0; q < npix; ++q) {
    int px = pix_x[q], py = pix_y[q];
    double o[3], d[3], Y[16];
    int valid;
    int32_t fl = 0;
    orc_pixel_setup(c, theta_max, x.deg, px, py, tol, o, d, Y, &valid, &fl);
    if (!valid) {
      rgb[3 * q] = rgb[3 * q + 1] = rgb[3 * q + 2] = 0.0;
      alpha[q] = 0.0; tfinal[q] = 1.0; nblend[q] = 0; flags[q] = fl; slack[q] = 0.0; aslack[q] = 0.0;
      if (fslack) fslack[q] = 0.0;
      if (faslack) faslack[q] = 0.0;
      if (rslack) rslack[q] = 0.0;
      if (raslack) raslack[q] = 0.0;
      continue;
    }
    for (int t = 0; t < x.ntie; ++t) {
      const double *e = edges ? edges + 4 * x.tie_list[t] : NULL;
      /* a near-tie particle without a footprint estimate flags every pixel */
      if (!e || isnan(e[0]) || (px >= e[0] - 1 && px <= e[1] + 1 && py >= e[2] - 1 && py <= e[3] + 1))
        fl |= ORC_F_CULL_TIE;
    }
    double T;
    slack[q] = 0.0;
    aslack[q] = 0.0;
    if (fslack) fslack[q] = 0.0;
    if (faslack) faslack[q] = 0.0;
    if (rslack) rslack[q] = 0.0;
    if (raslack) raslack[q] = 0.0;
    if (op->kbuffer > 0) {
      nblend[q] = orc_composite_ray_kbuffer(&x, sc, op, tol, px, py, o, d, Y, rgb + 3 * q, &T, &fl, NULL, NULL, 0,
                                            slack + q, aslack + q);
    } else {
      orc_slack sl;
      nblend[q] = orc_composite_ray(&x, sc, op, tol, px, py, o, d, Y, rgb + 3 * q, &T, &fl, NULL, 0, no_rect, &sl);
      slack[q] = sl.slack;
      aslack[q] = sl.aslack;
      if (fslack) fslack[q] = sl.fslack;
      if (faslack) faslack[q] = sl.faslack;
      if (rslack) rslack[q] = sl.rslack;
      if (raslack) raslack[q] = sl.raslack;
    }
    alpha[q] = 1.0 - T;
    tfinal[q] = T;
    flags[q] = fl;
  }
  orc_ctx_free(&x);
}

/* Composites an explicitly given ordered particle list for one pixel (used to check that
 * per-tile lists reproduce the brute-force order). */
void orc_render_list(const orc_scene *sc, const orc_camera *c, const orc_options *op, const int32_t *rect,
                     const float *depth32, int px, int py, int nlist, const uint32_t *list, double rgb[3],
                     double *tfinal) {
  orc_ctx x;
  orc_ctx_init(&x, sc, rect, depth32, NULL, NULL);
  for (int j = 0; j < nlist; ++j) x.order[j] = (int32_t)list[j];
  x.norder = nlist;
  double theta_max = orc_cam_limit(c);
  if (op->colour_mode == 1) orc_ctx_colour(&x, c, theta_max, op);
  orc_tol tol = {0, 0, 0, 0, 0};
  double o[3], d[3], Y[16];
  int valid;
  orc_pixel_setup(c, theta_max, x.deg, px, py, &tol, o, d, Y, &valid, NULL);
  if (!valid) { rgb[0] = rgb[1] = rgb[2] = 0; *tfinal = 1.0; }
  else orc_composite_ray(&x, sc, op, &tol, px, py, o, d, Y, rgb, tfinal, NULL, NULL, 0, 0, NULL);
  orc_ctx_free(&x);
}

/* ------------------------------------------------------------------ gradients */

/* d rotation / d unit quaternion, contracted with G = dL/dR (row-major). */
static void orc_rot_grad(const double q[4], const double G[9], double gq[4]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  gq[0] = 2 * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  gq[1] = 2 * (y * G[1] + z * G[2] + y * G[3] - 2 * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2 * x * G[8]);
  gq[2] = 2 * (-2 * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2 * y * G[8]);
  gq[3] = 2 * (-2 * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2 * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

/* Reverse-mode gradient of L with respect to every particle parameter, given dL/drgb and
 * dL/dalpha at the listed pixels, over each pixel's blended pairs in the order they were
 * blended (tile order, or the k-buffer's order with op->kbuffer > 0, whose selection decisions
 * are piecewise constant and carry no gradient) (supplementary Sec. B: d alpha / d omega^2 = -1/2 sigma
 * exp(-omega^2/2); d omega^2 / d o_g = 2 (o_g + tau d_g); d o_g / d mu = -S^-1 R^T; the S, R
 * terms follow from d omega^2 / d d_g = 2 tau (o_g + tau d_g) and M = S^-1 R^T).  The 2D
 * projection contributes no gradient: it only selects particles (Sec. 4.1).
 * Outputs are overwritten: d_means[n][3], d_log_scales[n][3], d_quats[n][4],
 * d_logits[n], d_sh[n][nsh][3]. */
void orc_backward(const orc_scene *sc, const orc_camera *c, const orc_options *op, const int32_t *rect,
                  const float *depth32, int npix, const int32_t *pix_x, const int32_t *pix_y, const double *g_rgb,
                  const double *g_alpha, double *d_means, double *d_log_scales, double *d_quats,
                  double *d_logits, double *d_sh, double *m_means, double *m_log_scales, double *m_quats,
                  double *m_logits, double *m_sh) {
  orc_ctx x;
  orc_ctx_init(&x, sc, rect, depth32, NULL, NULL);
  int n = sc->n, nsh = x.nsh;
  double theta_max = orc_cam_limit(c);
  if (op->colour_mode == 1) orc_ctx_colour(&x, c, theta_max, op);
  /* accumulators: dM (9), dmu (3), dsigma (1), dL/d colour (3, colour_mode 1) */
  double *acc = (double *)calloc((size_t)(n > 0 ? n : 1) * 16, sizeof(double));
  memset(d_sh, 0, sizeof(double) * (size_t)n * nsh * 3);
  /* Optional magnitudes (m_* non-NULL): the whole computation evaluated on absolute values --
   * every sum (and difference) of the per-pair chain, the sums over pairs and the final linear
   * maps taken over the absolute values of their operands.  A floating-point evaluation with
   * unit roundoff u deviates from the exact value by at most about (number of rounding steps)
   * u times this magnitude (the running error bound of forward error analysis; Higham,
   * "Accuracy and Stability of Numerical Algorithms", Sec. 3.1 and 4.2), whatever the order of
   * the sums, so it gives the scale of an FP32 result's error.  The suffix colour of a pair is
   * bounded by twice the pixel's final colour, which covers an evaluation that forms it as the
   * final colour minus a running prefix. */
  const int want_mag = m_means && m_log_scales && m_quats && m_logits && m_sh;
  double *macc = want_mag ? (double *)calloc((size_t)(n > 0 ? n : 1) * 16, sizeof(double)) : NULL;
  if (want_mag) memset(m_sh, 0, sizeof(double) * (size_t)n * nsh * 3);
  orc_tol tol = {0, 0, 0, 0, 0};
#pragma omp parallel
  {
    orc_contrib *rec = (orc_contrib *)malloc(sizeof(orc_contrib) * (size_t)(x.norder > 0 ? x.norder : 1));
#pragma omp for schedule(dynamic, 4)
    for (int q = 0; q < npix; ++q) {
      int px = pix_x[q], py = pix_y[q];
      double o[3], d[3], Y[16];
      int valid;
      orc_pixel_setup(c, theta_max, x.deg, px, py, &tol, o, d, Y, &valid, NULL);
      if (!valid) continue;
      double rgb[3], Tf;
      /* the blended pairs in blending order: the tile (depth) order, or the k-buffer's order */
      int nb = op->kbuffer > 0
                   ? orc_composite_ray_kbuffer(&x, sc, op, &tol, px, py, o, d, Y, rgb, &Tf, NULL, NULL, rec, x.norder,
                                               NULL, NULL)
                   : orc_composite_ray(&x, sc, op, &tol, px, py, o, d, Y, rgb, &Tf, NULL, rec, x.norder, 0, NULL);
      const double *g = g_rgb + 3 * q;
      double gA = g_alpha[q];
      double S[3] = {0, 0, 0}; /* sum over later blended particles of c alpha T */
      for (int b = nb - 1; b >= 0; --b) {
        orc_contrib *k = &rec[b];
        const orc_particle *p = &x.P[k->i];
        double om1 = 1.0 - k->alpha;
        double dalpha = gA * Tf / om1;
        for (int ch = 0; ch < 3; ++ch) dalpha += g[ch] * (k->col[ch] * k->T - S[ch] / om1);
        for (int ch = 0; ch < 3; ++ch) S[ch] += k->col[ch] * k->alpha * k->T;
        /* colour: d c / d beta = Y where the clamp is inactive (colour_mode 1: the particle's
         * basis, and the colour gradient is kept to be mapped onto beta and mu below) */
        for (int ch = 0; ch < 3; ++ch) {
          if (!(k->raw[ch] > 0.0)) continue;
          double gc = g[ch] * k->alpha * k->T;
          if (op->colour_mode == 1) {
#pragma omp atomic
            acc[16 * (size_t)k->i + 13 + ch] += gc;
            if (want_mag) {
#pragma omp atomic
              macc[16 * (size_t)k->i + 13 + ch] += fabs(gc);
            }
            continue;
          }
          for (int kk = 0; kk < nsh; ++kk) {
#pragma omp atomic
            d_sh[((size_t)k->i * nsh + kk) * 3 + ch] += gc * Y[kk];
            if (want_mag) {
#pragma omp atomic
              m_sh[((size_t)k->i * nsh + kk) * 3 + ch] += fabs(gc * Y[kk]);
            }
          }
        }
        double da = k->a > op->alpha_max ? 0.0 : dalpha;
        double dsig = da * k->rho;
        double dw2 = da * p->sigma * orc_dresponse(op, k->w2, k->rho);
        double pv[3], xw[3];
        for (int j = 0; j < 3; ++j) {
          pv[j] = 2.0 * dw2 * (k->og[j] + k->tau * k->dg[j]); /* dL/d o_g */
          xw[j] = o[j] - p->mu[j] + k->tau * d[j];             /* o - mu + tau d */
        }
        double *A = acc + 16 * (size_t)k->i;
        for (int r = 0; r < 3; ++r)
          for (int j = 0; j < 3; ++j) {
#pragma omp atomic
            A[3 * r + j] += pv[r] * xw[j];
          }
        for (int j = 0; j < 3; ++j) {
          double dm = -(p->M[j] * pv[0] + p->M[3 + j] * pv[1] + p->M[6 + j] * pv[2]);
#pragma omp atomic
          A[9 + j] += dm;
        }
#pragma omp atomic
        A[12] += dsig;
        if (want_mag) {
          /* the per-pair chain on absolute values */
          double dal_a = fabs(gA) * Tf / om1;
          for (int ch = 0; ch < 3; ++ch) dal_a += fabs(g[ch]) * (k->col[ch] * k->T + 2.0 * rgb[ch] / om1);
          const double da_a = k->a > op->alpha_max ? 0.0 : dal_a;
          const double dw2_a = da_a * p->sigma * fabs(orc_dresponse(op, k->w2, k->rho));
          double og_a[3], dg_a[3], dd = 0.0, num = 0.0;
          for (int r = 0; r < 3; ++r) {
            og_a[r] = dg_a[r] = 0.0;
            for (int j = 0; j < 3; ++j) {
              og_a[r] += fabs(p->M[3 * r + j]) * (fabs(o[j]) + fabs(p->mu[j]));
              dg_a[r] += fabs(p->M[3 * r + j]) * fabs(d[j]);
            }
            dd += k->dg[r] * k->dg[r];
            num += og_a[r] * dg_a[r];
          }
          const double tau_a = num / dd;
          double pv_a[3], xw_a[3];
          for (int j = 0; j < 3; ++j) {
            pv_a[j] = 2.0 * dw2_a * (og_a[j] + tau_a * dg_a[j]);
            xw_a[j] = fabs(o[j]) + fabs(p->mu[j]) + tau_a * fabs(d[j]);
          }
          double *MA = macc + 16 * (size_t)k->i;
          for (int r = 0; r < 3; ++r)
            for (int j = 0; j < 3; ++j) {
#pragma omp atomic
              MA[3 * r + j] += pv_a[r] * xw_a[j];
            }
          for (int j = 0; j < 3; ++j) {
            double dm = fabs(p->M[j]) * pv_a[0] + fabs(p->M[3 + j]) * pv_a[1] + fabs(p->M[6 + j]) * pv_a[2];
#pragma omp atomic
            MA[9 + j] += dm;
          }
#pragma omp atomic
          MA[12] += da_a * k->rho;
        }
      }
    }
    free(rec);
  }
  for (int i = 0; i < n; ++i) {
    const orc_particle *p = &x.P[i];
    const double *A = acc + 16 * (size_t)i;
    for (int j = 0; j < 3; ++j) d_means[3 * i + j] = A[9 + j];
    if (op->colour_mode == 1) {
      /* c_ch = sum_k beta_k,ch Y_k(dir(mu)) + 1/2: dL/dbeta_k,ch = gc_ch Y_k and
       * dL/dmu_j += sum_ch gc_ch sum_k beta_k,ch dY_k/dmu_j */
      const float *beta = sc->sh + (size_t)i * nsh * 3;
      for (int ch = 0; ch < 3; ++ch) {
        double gc = A[13 + ch];
        if (gc == 0.0) continue;
        for (int kk = 0; kk < nsh; ++kk) {
          d_sh[((size_t)i * nsh + kk) * 3 + ch] += gc * x.Yp[16 * (size_t)i + kk];
          for (int j = 0; j < 3; ++j) d_means[3 * i + j] += gc * beta[3 * kk + ch] * x.dYdmu[48 * (size_t)i + 16 * j + kk];
        }
      }
    }
    /* M_kj = R_jk / s_k, s_k = exp(l_k): dL/dl_k = -sum_j dM_kj M_kj; dL/dR_jk = dM_kj / s_k */
    double G[9];
    for (int k = 0; k < 3; ++k) {
      double acc_l = 0;
      for (int j = 0; j < 3; ++j) {
        acc_l += A[3 * k + j] * p->M[3 * k + j];
        G[3 * j + k] = A[3 * k + j] / p->s[k];
      }
      d_log_scales[3 * i + k] = -acc_l;
    }
    double gq[4];
    orc_rot_grad(p->qn, G, gq);
    double dot = gq[0] * p->qn[0] + gq[1] * p->qn[1] + gq[2] * p->qn[2] + gq[3] * p->qn[3];
    for (int j = 0; j < 4; ++j) d_quats[4 * i + j] = (gq[j] - p->qn[j] * dot) / p->qnorm;
    d_logits[i] = A[12] * p->sigma * (1.0 - p->sigma);
    if (want_mag) {
      /* the same maps, entry-wise absolute, applied to the absolute sums */
      const double *MA = macc + 16 * (size_t)i;
      for (int j = 0; j < 3; ++j) m_means[3 * i + j] = MA[9 + j];
      if (op->colour_mode == 1) {
        const float *beta = sc->sh + (size_t)i * nsh * 3;
        for (int ch = 0; ch < 3; ++ch) {
          double gc = MA[13 + ch];
          for (int kk = 0; kk < nsh; ++kk) {
            m_sh[((size_t)i * nsh + kk) * 3 + ch] += gc * fabs(x.Yp[16 * (size_t)i + kk]);
            for (int j = 0; j < 3; ++j)
              m_means[3 * i + j] += gc * fabs(beta[3 * kk + ch] * x.dYdmu[48 * (size_t)i + 16 * j + kk]);
          }
        }
      }
      double Ga[9];
      for (int k = 0; k < 3; ++k) {
        double acc_l = 0;
        for (int j = 0; j < 3; ++j) {
          acc_l += MA[3 * k + j] * fabs(p->M[3 * k + j]);
          Ga[3 * j + k] = MA[3 * k + j] / p->s[k];
        }
        m_log_scales[3 * i + k] = acc_l;
      }
      /* quaternion map L = (I - q q^T) J / |q| with J = d gq / d G, column by column */
      double L[4][9];
      for (int m = 0; m < 9; ++m) {
        double e[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gj[4];
        e[m] = 1.0;
        orc_rot_grad(p->qn, e, gj);
        double dj = gj[0] * p->qn[0] + gj[1] * p->qn[1] + gj[2] * p->qn[2] + gj[3] * p->qn[3];
        for (int j = 0; j < 4; ++j) L[j][m] = (gj[j] - p->qn[j] * dj) / p->qnorm;
      }
      for (int j = 0; j < 4; ++j) {
        double mq = 0.0;
        for (int m = 0; m < 9; ++m) mq += fabs(L[j][m]) * Ga[m];
        m_quats[4 * i + j] = mq;
      }
      m_logits[i] = MA[12] * p->sigma * (1.0 - p->sigma);
    }
  }
  free(acc);
  free(macc);
  orc_ctx_free(&x);
}

/* ------------------------------------------------------------------ misc */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
