// abi.cu — the extern "C" entry points declared in include/ut3d.h: host-side validation,
// camera / UT-weight preparation in FP64, and kernel launches.
#include <cmath>
#include <cstring>

#include "ut3d_device.cuh"
#include "ut3d_internal.h"

#include <atomic>

namespace ut3d {

static std::atomic<unsigned long long> g_launches{0};

void count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

namespace {

bool finite_all(const float *v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

double poly_theta_d(const double k[4], double th) {
  double t2 = th * th;
  return th * (1.0 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
}

// d theta_d / d theta as a polynomial in u = theta^2: 1 + 3 k1 u + 5 k2 u^2 + 7 k3 u^3 + 9 k4 u^4.
double dpoly_u(const double k[4], double u) { return 1.0 + u * (3 * k[0] + u * (5 * k[1] + u * (7 * k[2] + u * 9 * k[3]))); }

// Largest imaged angle of the polynomial fisheye: the first sign change of d theta_d / d theta
// on (0, pi/2], located on a uniform grid in u = theta^2 and refined by bisection; pi/2 if none.
double fisheye_theta_max(const double k[4]) {
  const double umax = 0.25 * M_PI * M_PI;
  const int steps = 4096;
  double prev_u = 0.0;
  for (int i = 1; i <= steps; ++i) {
    double u = umax * i / steps;
    if (dpoly_u(k, u) <= 0.0) {
      double lo = prev_u, hi = u;
      for (int it = 0; it < 100; ++it) {
        double m = 0.5 * (lo + hi);
        (dpoly_u(k, m) > 0.0 ? lo : hi) = m;
      }
      return std::sqrt(lo);
    }
    prev_u = u;
  }
  return 0.5 * M_PI;
}

// Radial pinhole: first zero of d r_d / d r = 1 + 3 k1 r^2 + 5 k2 r^4 + 7 k3 r^6 on (0, 10]
// (scanned in u = r^2, refined by bisection), or infinity when the model is monotone there.
double radial_rmax(const double k[3]) {
  auto dr = [&](double u) { return 1.0 + u * (3.0 * k[0] + u * (5.0 * k[1] + u * 7.0 * k[2])); };
  const int steps = 16384;
  double prev_u = 0.0;
  for (int i = 1; i <= steps; ++i) {
    double u = 100.0 * i / steps;
    if (dr(u) <= 0.0) {
      double lo = prev_u, hi = u;
      for (int it = 0; it < 100; ++it) {
        double m = 0.5 * (lo + hi);
        (dr(m) > 0.0 ? lo : hi) = m;
      }
      return std::sqrt(lo);
    }
    prev_u = u;
  }
  return INFINITY;
}

void quat_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

ut_status make_cam(const ut_camera *c, DevCam &d) {
  if (!c) return UT_ERR_INVALID_ARG;
  if (c->model != UT_CAM_PINHOLE && c->model != UT_CAM_FISHEYE && c->model != UT_CAM_PINHOLE_RADIAL)
    return UT_ERR_INVALID_ARG;
  if (c->width < 1 || c->height < 1 || c->width > 32767 || c->height > 32767) return UT_ERR_INVALID_ARG;
  if (c->rolling_shutter != 0 && c->rolling_shutter != 1) return UT_ERR_INVALID_ARG;
  if (c->rolling_shutter && c->height < 2) return UT_ERR_INVALID_ARG;
  const float sc[5] = {c->fx, c->fy, c->cx, c->cy, c->near_plane};
  if (!finite_all(sc, 5) || !finite_all(c->k, 4) || !finite_all(c->q_start, 4) || !finite_all(c->t_start, 3) ||
      !finite_all(c->q_end, 4) || !finite_all(c->t_end, 3))
    return UT_ERR_INVALID_ARG;
  if (!(c->fx > 0) || !(c->fy > 0) || !(c->near_plane > 0)) return UT_ERR_INVALID_ARG;
  double q0[4], q1[4], n0 = 0, n1 = 0;
  for (int i = 0; i < 4; ++i) {
    q0[i] = c->q_start[i];
    q1[i] = c->q_end[i];
    n0 += q0[i] * q0[i];
    n1 += q1[i] * q1[i];
  }
  if (!(n0 > 0) || (c->rolling_shutter && !(n1 > 0))) return UT_ERR_INVALID_ARG;
  n0 = std::sqrt(n0);
  for (int i = 0; i < 4; ++i) q0[i] /= n0;
  std::memset(&d, 0, sizeof(d));
  d.model = c->model;
  d.W = c->width;
  d.H = c->height;
  d.rs = c->rolling_shutter;
  d.fx = c->fx; d.fy = c->fy; d.cx = c->cx; d.cy = c->cy;
  d.ifx = (float)(1.0 / c->fx);
  d.ify = (float)(1.0 / c->fy);
  d.k1 = c->k[0]; d.k2 = c->k[1]; d.k3 = c->k[2]; d.k4 = c->k[3];
  double R0[9];
  quat_rot(q0, R0);
  for (int i = 0; i < 9; ++i) d.R0[i] = (float)R0[i];
  for (int i = 0; i < 3; ++i) d.T0[i] = c->t_start[i];
  for (int j = 0; j < 3; ++j) d.cen[j] = (float)-(R0[j] * c->t_start[0] + R0[3 + j] * c->t_start[1] + R0[6 + j] * c->t_start[2]);
  d.ax[0] = 1.f;
  if (c->rolling_shutter) {
    n1 = std::sqrt(n1);
    for (int i = 0; i < 4; ++i) q1[i] /= n1;
    double dot = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2] + q0[3] * q1[3];
    if (dot < 0)
      for (int i = 0; i < 4; ++i) q1[i] = -q1[i];
    // relative rotation q1 * conj(q0): R(t) = Rot(axis, t phi) R0 is the slerp of the two poses
    double a1 = q1[0], b1 = q1[1], c1 = q1[2], d1 = q1[3];
    double a2 = q0[0], b2 = -q0[1], c2 = -q0[2], d2 = -q0[3];
    double rw = a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2;
    double rx = a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2;
    double ry = a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2;
    double rz = a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2;
    double s = std::sqrt(rx * rx + ry * ry + rz * rz);
    if (s > 1e-15) {
      d.phi = (float)(2.0 * std::atan2(s, rw));
      d.ax[0] = (float)(rx / s);
      d.ax[1] = (float)(ry / s);
      d.ax[2] = (float)(rz / s);
    }
    for (int i = 0; i < 3; ++i) d.dT[i] = (float)((double)c->t_end[i] - (double)c->t_start[i]);
    d.inv_hm1 = (float)(1.0 / (c->height - 1));
  }
  d.near_plane = c->near_plane;
  if (c->model == UT_CAM_FISHEYE) {
    double k[4] = {c->k[0], c->k[1], c->k[2], c->k[3]};
    double tm = fisheye_theta_max(k);
    d.theta_max = (float)tm;
    d.rd_max = (float)poly_theta_d(k, tm);
  } else if (c->model == UT_CAM_PINHOLE_RADIAL) {
    // theta_max carries the largest imaged normalised radius r_max, rd_max = r_d(r_max)
    double k[3] = {c->k[0], c->k[1], c->k[2]};
    double rm = radial_rmax(k);
    d.theta_max = std::isfinite(rm) ? (float)rm : INFINITY;
    d.rd_max = std::isfinite(rm) ? (float)(rm * (1.0 + rm * rm * (k[0] + rm * rm * (k[1] + rm * rm * k[2]))))
                                 : INFINITY;
  } else {
    d.theta_max = (float)(0.5 * M_PI);
    d.rd_max = INFINITY;
  }
  return UT_OK;
}

ut_status make_opts(const ut_options *o, const ut_camera *c, DevOpts &d) {
  if (!o) return UT_ERR_INVALID_ARG;
  int area = o->tile_w * o->tile_h;
  if (o->tile_w < 1 || o->tile_h < 1 || o->tile_w > 512 || o->tile_h > 512 || area < 64 || area > 512 ||
      area % 32 != 0)
    return UT_ERR_INVALID_ARG;
  const float f[4] = {o->t_min, o->alpha_min, o->alpha_max, o->extent_sigma};
  if (!finite_all(f, 4)) return UT_ERR_INVALID_ARG;
  if (!(o->t_min >= 0) || !(o->t_min < 1) || !(o->alpha_min > 0) || !(o->alpha_min < 1) || !(o->alpha_max > 0) ||
      !(o->alpha_max < 1) || !(o->extent_sigma > 0))
    return UT_ERR_INVALID_ARG;
  if (o->rs_iters < 0 || o->rs_iters > 64 || o->newton_iters < 1 || o->newton_iters > 64) return UT_ERR_INVALID_ARG;
  if ((o->projection != UT_PROJECTION_UT && o->projection != UT_PROJECTION_EWA) ||
      (o->colour_mode != UT_COLOUR_PER_PIXEL && o->colour_mode != UT_COLOUR_PER_PARTICLE) ||
      o->kernel_degree < 2 || o->kernel_degree > 8)
    return UT_ERR_INVALID_ARG;
  if (o->kbuffer < 0 || o->kbuffer > 16) return UT_ERR_INVALID_ARG;
  if (o->kernel_degree != 2 && o->colour_mode == UT_COLOUR_PER_PARTICLE) return UT_ERR_UNSUPPORTED;
  if (o->kbuffer > 0 && (o->kernel_degree != 2 || o->colour_mode == UT_COLOUR_PER_PARTICLE)) return UT_ERR_UNSUPPORTED;
  d.tile_w = o->tile_w;
  d.tile_h = o->tile_h;
  d.tiles_x = (c->width + o->tile_w - 1) / o->tile_w;
  d.tiles_y = (c->height + o->tile_h - 1) / o->tile_h;
  d.t_min = o->t_min;
  d.alpha_min = o->alpha_min;
  d.alpha_max = o->alpha_max;
  d.extent_sigma = o->extent_sigma;
  d.rs_iters = o->rs_iters;
  d.newton_iters = o->newton_iters;
  d.projection = o->projection;
  d.colour_mode = o->colour_mode;
  d.kernel_degree = o->kernel_degree;
  d.kernel_lambda = (float)(0.5 * std::pow(3.0, 2.0 - o->kernel_degree));
  d.kbuffer = o->kbuffer;
  return UT_OK;
}

ut_status check_scene(const ut_scene *s, bool need_sh) {
  if (!s || s->n < 0 || s->sh_degree < 0 || s->sh_degree > 3) return UT_ERR_INVALID_ARG;
  if (s->n == 0) return UT_OK;
  if (!s->means || !s->log_scales || !s->quats || !s->opacity_logits || (need_sh && !s->sh)) return UT_ERR_INVALID_ARG;
  if (!aligned16(s->quats) || (reinterpret_cast<uintptr_t>(s->means) & 3) ||
      (reinterpret_cast<uintptr_t>(s->log_scales) & 3))
    return UT_ERR_INVALID_ARG;
  return UT_OK;
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

DevScene scene_desc(const ut_scene &s) {
  DevScene d;
  std::memset(&d, 0, sizeof(d));
  d.means = s.means;
  d.log_scales = s.log_scales;
  d.quats = reinterpret_cast<const float4 *>(s.quats);
  d.logits = s.opacity_logits;
  d.sh = s.sh;
  d.n = s.n;
  d.deg = s.sh_degree;
  const int nc = 3 * (s.sh_degree + 1) * (s.sh_degree + 1);
  d.sh_vec = (nc % 4 == 0) && aligned16(s.sh);
  return d;
}

// Bits needed to hold the indices 0 .. count - 1.
int bits_for_count(long long count) {
  int b = 0;
  while ((1ll << b) < count) ++b;
  return b;
}

// A batch of one view of one scene (the single-view entry points).
void single_view(BatchDesc &bd, const DevCam &cam, const DevOpts &op, const ut_scene *scene, int n) {
  std::memset(&bd, 0, sizeof(bd));
  bd.nv = 1;
  bd.ns = 1;
  bd.total_particles = n;
  bd.total_tiles = op.tiles_x * op.tiles_y;
  bd.v[0].cam = cam;
  bd.v[0].n = n;
  bd.v[0].tiles_x = op.tiles_x;
  bd.v[0].tiles_y = op.tiles_y;
  bd.total_cols = op.tiles_x;
  bd.total_rows = op.tiles_y;
  bd.col_bits = bits_for_count(op.tiles_x);
  if (scene) bd.s[0] = scene_desc(*scene);
  bd.s[0].n = n;
}

ut_status make_weights(const ut_params *ut, UTWeights &w) {
  if (!ut || !std::isfinite(ut->alpha) || !std::isfinite(ut->beta) || !std::isfinite(ut->kappa))
    return UT_ERR_INVALID_ARG;
  double a = ut->alpha, b = ut->beta, k = ut->kappa;
  double lam = a * a * (3.0 + k) - 3.0;
  if (!(3.0 + lam > 0)) return UT_ERR_INVALID_ARG;
  w.gamma = (float)std::sqrt(3.0 + lam);
  w.wm0 = (float)(lam / (3.0 + lam));
  w.wi = (float)(1.0 / (2.0 * (3.0 + lam)));
  w.wc0 = (float)(lam / (3.0 + lam) + (1.0 - a * a + b));
  return UT_OK;
}

// ---------------------------------------------------------------- batches

// Validates a batch and fills its descriptor (flattened particle / tile offsets).
ut_status make_batch(const ut_scene *scenes, int ns, const ut_view *views, int nv, const ut_options *opt,
                     BatchDesc &bd, DevOpts &dop) {
  if (!scenes || !views || ns < 1 || ns > kMaxScenes || nv < 1 || nv > kMaxViews || !opt) return UT_ERR_INVALID_ARG;
  std::memset(&bd, 0, sizeof(bd));
  for (int s = 0; s < ns; ++s) {
    ut_status st = check_scene(&scenes[s], true);
    if (st != UT_OK) return st;
    if (scenes[s].sh_degree != scenes[0].sh_degree) return UT_ERR_INVALID_ARG;
    bd.s[s] = scene_desc(scenes[s]);
  }
  bd.ns = ns;
  bd.nv = nv;
  long long part = 0, tiles = 0, cols = 0, rows = 0, max_tx = 1;
  for (int v = 0; v < nv; ++v) {
    const ut_view &vw = views[v];
    if (vw.scene < 0 || vw.scene >= ns || !vw.rgb || !vw.alpha) return UT_ERR_INVALID_ARG;
    DevView &d = bd.v[v];
    ut_status st = make_cam(&vw.camera, d.cam);
    if (st != UT_OK) return st;
    DevOpts o;
    if ((st = make_opts(opt, &vw.camera, o)) != UT_OK) return st;
    if (v == 0) dop = o;
    d.scene = vw.scene;
    d.n = scenes[vw.scene].n;
    d.part_off = (int)part;
    d.tile_off = (int)tiles;
    d.tiles_x = o.tiles_x;
    d.tiles_y = o.tiles_y;
    d.col_off = (int)cols;
    d.row_off = (int)rows;
    d.rgb = vw.rgb;
    d.alpha = vw.alpha;
    d.tfinal = vw.t_final;
    d.n_used = vw.n_used;
    d.d_rgb = vw.d_rgb;
    d.d_alpha = vw.d_alpha;
    part += d.n;
    tiles += (long long)o.tiles_x * o.tiles_y;
    cols += o.tiles_x;
    rows += o.tiles_y;
    max_tx = o.tiles_x > max_tx ? o.tiles_x : max_tx;
  }
  if (part >= (1ll << 31) || tiles >= (1ll << 31)) return UT_ERR_INVALID_ARG;
  bd.total_particles = (int)part;
  bd.total_tiles = (int)tiles;
  bd.total_cols = (int)cols;
  bd.total_rows = (int)rows;
  bd.col_bits = bits_for_count(max_tx);
  // binning packs a global tile column and a particle's tile-row count into 16 bits each
  if (cols > 0xffff || rows > 0xffff || bd.col_bits + bits_for_count(rows) > 32) return UT_ERR_INVALID_ARG;
  return UT_OK;
}

// Layout of the render_batch workspace: projection of every flattened entry, ranges of every
// global tile, the sorted values, then bin_and_sort's own scratch.
struct BatchLayout {
  size_t mean2d, cov2d, depth, rect, ntiles, ranges, vals, sched, bin, total;
};

int max_tiles_y(const BatchDesc &bd) {
  int m = 0;
  for (int v = 0; v < bd.nv; ++v) m = bd.v[v].tiles_y > m ? bd.v[v].tiles_y : m;
  return m;
}

BatchLayout batch_layout(long long part, long long tiles, long long cols, int max_rows, long long cap) {
  BatchLayout L;
  size_t off = 0;
  size_t p = (size_t)(part > 0 ? part : 1), t = (size_t)(tiles > 0 ? tiles : 1), c = (size_t)(cap > 0 ? cap : 1);
  L.mean2d = off; off += align256(p * 8);
  L.cov2d = off; off += align256(p * 12);
  L.depth = off; off += align256(p * 4);
  L.rect = off; off += align256(p * 8);
  L.ntiles = off; off += align256(p * 4);
  L.ranges = off; off += align256(t * 8);
  L.vals = off; off += align256(c * 4);
  L.sched = off; off += tile_sched_bytes((int)t);
  L.bin = off; off += bin_workspace_bytes((int)p, (int64_t)c, (int)t, (int)cols, max_rows);
  L.total = off;
  return L;
}

}  // namespace
}  // namespace ut3d

using namespace ut3d;

extern "C" {

void ut_default_options(ut_options *o) {
  if (!o) return;
  o->tile_w = 16;
  o->tile_h = 16;
  o->t_min = 1e-4f;
  o->alpha_min = 1.f / 255.f;
  o->alpha_max = 0.99f;
  o->rs_iters = 3;
  o->newton_iters = 12;
  o->extent_sigma = 3.f;
  o->projection = UT_PROJECTION_UT;
  o->colour_mode = UT_COLOUR_PER_PIXEL;
  o->kernel_degree = 2;
  o->kbuffer = 0;
}

uint64_t ut_kernel_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

int32_t ut_debug_enabled(void) {
#ifdef UT_DEBUG
  return 1;
#else
  return 0;
#endif
}

ut_status ut_debug_read(uint32_t record[4], int32_t reset) {
#ifdef UT_DEBUG
  if (!record) return UT_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return UT_ERR_CUDA;
  ut_status (*readers[])(uint32_t *, bool) = {dbg_read_binsort, dbg_read_project, dbg_read_fwd, dbg_read_bwd,
                                              dbg_read_kbuffer};
  record[0] = record[1] = record[2] = record[3] = 0u;
  for (auto rd : readers) {  // the first unit with a record reports; every record is read (and reset)
    uint32_t r[4];
    const ut_status st = rd(r, reset != 0);
    if (st != UT_OK) return st;
    if (record[0] == 0u && r[0] != 0u)
      for (int i = 0; i < 4; ++i) record[i] = r[i];
  }
  return UT_OK;
#else
  (void)record;
  (void)reset;
  return UT_ERR_UNSUPPORTED;
#endif
}

ut_status ut_debug_check_bin_workspace(const void *workspace, int32_t n, int64_t key_capacity, const ut_camera *cam,
                                       const ut_options *opt, ut_stream stream) {
  DevCam dc;
  ut_status st = make_cam(cam, dc);
  if (st != UT_OK) return st;
  DevOpts dop;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  if (!workspace || n < 0 || key_capacity < 0) return UT_ERR_INVALID_ARG;
  return dbg_check_bin_guards(workspace, n, key_capacity, dop.tiles_x * dop.tiles_y, dop.tiles_x, dop.tiles_y,
                              reinterpret_cast<cudaStream_t>(stream));
}

const char *ut_status_string(ut_status s) {
  switch (s) {
    case UT_OK: return "ok";
    case UT_ERR_INVALID_ARG: return "invalid argument";
    case UT_ERR_CAPACITY: return "capacity exceeded";
    case UT_ERR_CUDA: return "CUDA error";
    case UT_ERR_TIMEOUT: return "device wait timed out";
    case UT_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

ut_status ut_project(const ut_scene *scene, const ut_camera *cam, const ut_params *ut, const ut_options *opt,
                     float *mean2d, float *cov2d, float *depth, int16_t *rect, uint32_t *ntiles,
                     ut_stream stream) {
  ut_status st = check_scene(scene, false);
  if (st != UT_OK) return st;
  DevCam dc;
  if ((st = make_cam(cam, dc)) != UT_OK) return st;
  DevOpts dop;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  UTWeights w;
  if ((st = make_weights(ut, w)) != UT_OK) return st;
  if (scene->n > 0 && (!mean2d || !cov2d || !depth || !rect || !ntiles || !aligned8(mean2d) || !aligned8(rect)))
    return UT_ERR_INVALID_ARG;
  BatchDesc bd;
  single_view(bd, dc, dop, scene, scene->n);
  return launch_project(bd, dop, w, mean2d, cov2d, depth, rect, ntiles, reinterpret_cast<cudaStream_t>(stream));
}

ut_status ut_project_points(const float *points, int32_t n, const ut_camera *cam, const ut_options *opt, float *uv,
                            int32_t *valid, ut_stream stream) {
  DevCam dc;
  ut_status st = make_cam(cam, dc);
  if (st != UT_OK) return st;
  DevOpts dop;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  if (n < 0 || (n > 0 && (!points || !uv || !valid || !aligned8(uv)))) return UT_ERR_INVALID_ARG;
  return launch_project_points(dc, dop, points, n, uv, valid, reinterpret_cast<cudaStream_t>(stream));
}

size_t ut_bin_workspace_size(int32_t n, int64_t key_capacity, const ut_camera *cam, const ut_options *opt) {
  if (n < 0 || key_capacity < 0 || !cam || !opt || opt->tile_w < 1 || opt->tile_h < 1) return 0;
  const int cols = (cam->width + opt->tile_w - 1) / opt->tile_w, rows = (cam->height + opt->tile_h - 1) / opt->tile_h;
  return bin_workspace_bytes(n, key_capacity, cols * rows, cols, rows);
}

}  // extern "C"

namespace ut3d {
// Every check bin_and_sort makes on its arguments except the workspace's; on success *need is
// the workspace size.  bin_and_sort_static shares it, so both give the same status.
ut_status bin_check_args(int32_t n, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                         const ut_camera *cam, const ut_options *opt, int64_t key_capacity, const uint32_t *vals,
                         const uint32_t *tile_ranges, const int64_t *k_out, DevCam &dc, DevOpts &dop, size_t *need) {
  ut_status st = make_cam(cam, dc);
  if (st != UT_OK) return st;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  if (n < 0 || key_capacity < 0 || key_capacity >= (int64_t(1) << 32)) return UT_ERR_INVALID_ARG;
  if (n > 0 && (!depth || !rect || !ntiles || !aligned8(rect))) return UT_ERR_INVALID_ARG;
  if (!tile_ranges || !k_out || (key_capacity > 0 && !vals) || !aligned8(tile_ranges)) return UT_ERR_INVALID_ARG;
  *need = bin_workspace_bytes(n, key_capacity, dop.tiles_x * dop.tiles_y, dop.tiles_x, dop.tiles_y);
  return UT_OK;
}
}  // namespace ut3d

extern "C" {

ut_status bin_and_sort(int32_t n, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                       const ut_camera *cam, const ut_options *opt, void *workspace, size_t workspace_bytes,
                       int64_t key_capacity, uint64_t *keys, uint32_t *vals, uint32_t *tile_ranges,
                       int64_t *k_out, ut_stream stream) {
  DevCam dc;
  DevOpts dop;
  size_t need = 0;
  ut_status st = bin_check_args(n, depth, rect, ntiles, cam, opt, key_capacity, vals, tile_ranges, k_out, dc, dop,
                                &need);
  if (st != UT_OK) return st;
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return UT_ERR_INVALID_ARG;
  BatchDesc bd;
  single_view(bd, dc, dop, nullptr, n);
  return launch_bin(bd, depth, rect, ntiles, dop, workspace, key_capacity, keys, vals, tile_ranges, k_out,
                    reinterpret_cast<cudaStream_t>(stream), true);
}

size_t ut_forward_workspace_size(const ut_camera *cam, const ut_options *opt) {
  if (!cam || !opt || opt->tile_w < 1 || opt->tile_h < 1 || cam->width < 1 || cam->height < 1) return 0;
  int tiles = ((cam->width + opt->tile_w - 1) / opt->tile_w) * ((cam->height + opt->tile_h - 1) / opt->tile_h);
  return tile_sched_bytes(tiles);
}

ut_status composite_forward(const ut_scene *scene, const ut_camera *cam, const ut_options *opt,
                            const int16_t *rect, const uint32_t *vals, const uint32_t *tile_ranges, float *rgb,
                            float *alpha, float *t_final, uint32_t *n_used, void *workspace,
                            size_t workspace_bytes, unsigned long long *stats, ut_stream stream) {
  ut_status st = check_scene(scene, true);
  if (st != UT_OK) return st;
  DevCam dc;
  if ((st = make_cam(cam, dc)) != UT_OK) return st;
  DevOpts dop;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  if (!tile_ranges || !rgb || !alpha || !t_final || !n_used || !aligned8(tile_ranges)) return UT_ERR_INVALID_ARG;
  if (scene->n > 0 && (!rect || !aligned8(rect))) return UT_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < tile_sched_bytes(dop.tiles_x * dop.tiles_y) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return UT_ERR_INVALID_ARG;
  BatchDesc bd;
  single_view(bd, dc, dop, scene, scene->n);
  bd.v[0].rgb = rgb;
  bd.v[0].alpha = alpha;
  bd.v[0].tfinal = t_final;
  bd.v[0].n_used = n_used;
  return launch_composite_fwd(bd, dop, rect, vals, tile_ranges, stats, workspace,
                              reinterpret_cast<cudaStream_t>(stream));
}

size_t ut_backward_workspace_size(int32_t n, const ut_camera *cam, const ut_options *opt) {
  if (n < 0 || !cam || !opt || opt->tile_w < 1 || opt->tile_h < 1 || cam->width < 1 || cam->height < 1) return 0;
  int tiles = ((cam->width + opt->tile_w - 1) / opt->tile_w) * ((cam->height + opt->tile_h - 1) / opt->tile_h);
  return backward_workspace_bytes(n, opt->kbuffer > 0) + tile_sched_bytes(tiles);
}

ut_status composite_backward(const ut_scene *scene, const ut_camera *cam, const ut_options *opt,
                             const int16_t *rect, const uint32_t *vals, const uint32_t *tile_ranges,
                             const float *rgb, const float *t_final, const uint32_t *n_used, const float *d_rgb,
                             const float *d_alpha, void *workspace, size_t workspace_bytes, float *d_means,
                             float *d_log_scales, float *d_quats, float *d_opacity_logits, float *d_sh,
                             ut_stream stream) {
  ut_status st = check_scene(scene, true);
  if (st != UT_OK) return st;
  DevCam dc;
  if ((st = make_cam(cam, dc)) != UT_OK) return st;
  DevOpts dop;
  if ((st = make_opts(opt, cam, dop)) != UT_OK) return st;
  if (!tile_ranges || !rgb || !t_final || !n_used || !d_rgb || !d_alpha || !aligned8(tile_ranges))
    return UT_ERR_INVALID_ARG;
  if (scene->n > 0 && (!rect || !aligned8(rect) || !d_means || !d_log_scales || !d_quats || !d_opacity_logits ||
                       !d_sh))
    return UT_ERR_INVALID_ARG;
  const size_t acc_bytes = backward_workspace_bytes(scene->n, dop.kbuffer > 0);
  if (!workspace || workspace_bytes < acc_bytes + tile_sched_bytes(dop.tiles_x * dop.tiles_y) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return UT_ERR_INVALID_ARG;
  BatchDesc bd;
  single_view(bd, dc, dop, scene, scene->n);
  DevView &v = bd.v[0];
  v.rgb = const_cast<float *>(rgb);
  v.tfinal = const_cast<float *>(t_final);
  v.n_used = const_cast<uint32_t *>(n_used);
  v.d_rgb = d_rgb;
  v.d_alpha = d_alpha;
  DevScene &s = bd.s[0];
  s.gacc = static_cast<float *>(workspace);
  s.kbrec = dop.kbuffer > 0 ? reinterpret_cast<float4 *>(static_cast<char *>(workspace) + acc_bytes / 2) : nullptr;
  s.d_means = d_means;
  s.d_log_scales = d_log_scales;
  s.d_quats = d_quats;
  s.d_logits = d_opacity_logits;
  s.d_sh = d_sh;
  s.grad_off = 0;
  return launch_composite_bwd(bd, dop, rect, vals, tile_ranges, static_cast<char *>(workspace) + acc_bytes,
                              reinterpret_cast<cudaStream_t>(stream));
}

size_t ut_batch_workspace_size(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                               const ut_options *opt, int64_t key_capacity) {
  BatchDesc bd;
  DevOpts dop;
  if (key_capacity < 0 || make_batch(scenes, n_scenes, views, n_views, opt, bd, dop) != UT_OK) return 0;
  return batch_layout(bd.total_particles, bd.total_tiles, bd.total_cols, max_tiles_y(bd), key_capacity).total;
}

ut_status render_batch(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                       const ut_params *ut, const ut_options *opt, void *workspace, size_t workspace_bytes,
                       int64_t key_capacity, int64_t *k_out, ut_stream stream) {
  BatchDesc bd;
  DevOpts dop;
  ut_status st = make_batch(scenes, n_scenes, views, n_views, opt, bd, dop);
  if (st != UT_OK) return st;
  UTWeights w;
  if ((st = make_weights(ut, w)) != UT_OK) return st;
  if (key_capacity < 0 || key_capacity >= (int64_t(1) << 32) || !k_out) return UT_ERR_INVALID_ARG;
  BatchLayout L = batch_layout(bd.total_particles, bd.total_tiles, bd.total_cols, max_tiles_y(bd), key_capacity);
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return UT_ERR_INVALID_ARG;
  char *ws = static_cast<char *>(workspace);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float *depth = reinterpret_cast<float *>(ws + L.depth);
  int16_t *rect = reinterpret_cast<int16_t *>(ws + L.rect);
  uint32_t *ntiles = reinterpret_cast<uint32_t *>(ws + L.ntiles);
  uint32_t *ranges = reinterpret_cast<uint32_t *>(ws + L.ranges);
  uint32_t *vals = reinterpret_cast<uint32_t *>(ws + L.vals);
  if ((st = launch_project(bd, dop, w, reinterpret_cast<float *>(ws + L.mean2d), reinterpret_cast<float *>(ws + L.cov2d),
                           depth, rect, ntiles, s)) != UT_OK)
    return st;
  if ((st = launch_bin(bd, depth, rect, ntiles, dop, ws + L.bin, key_capacity, nullptr, vals, ranges, k_out, s,
                       false)) != UT_OK)
    return st;
  return launch_composite_fwd(bd, dop, rect, vals, ranges, nullptr, ws + L.sched, s);
}

size_t ut_batch_backward_workspace_size(const ut_scene *scenes, int32_t n_scenes, const ut_view *views,
                                        int32_t n_views, const ut_options *opt) {
  BatchDesc bd;
  DevOpts dop;
  if (make_batch(scenes, n_scenes, views, n_views, opt, bd, dop) != UT_OK) return 0;
  size_t total = 0;
  for (int k = 0; k < n_scenes; ++k) total += backward_workspace_bytes(scenes[k].n, dop.kbuffer > 0);
  return total + tile_sched_bytes(bd.total_tiles);
}

ut_status render_batch_backward(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                                const ut_options *opt, const void *workspace, size_t workspace_bytes,
                                int64_t key_capacity, void *grad_workspace, size_t grad_workspace_bytes,
                                const ut_scene_grads *grads, ut_stream stream) {
  BatchDesc bd;
  DevOpts dop;
  ut_status st = make_batch(scenes, n_scenes, views, n_views, opt, bd, dop);
  if (st != UT_OK) return st;
  for (int v = 0; v < n_views; ++v)
    if (!views[v].t_final || !views[v].n_used || !views[v].d_rgb || !views[v].d_alpha) return UT_ERR_INVALID_ARG;
  if (key_capacity < 0 || key_capacity >= (int64_t(1) << 32) || !grads) return UT_ERR_INVALID_ARG;
  BatchLayout L = batch_layout(bd.total_particles, bd.total_tiles, bd.total_cols, max_tiles_y(bd), key_capacity);
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return UT_ERR_INVALID_ARG;
  if (!grad_workspace || grad_workspace_bytes < ut_batch_backward_workspace_size(scenes, n_scenes, views, n_views, opt) ||
      (reinterpret_cast<uintptr_t>(grad_workspace) & 255))
    return UT_ERR_INVALID_ARG;
  char *gw = static_cast<char *>(grad_workspace);
  int goff = 0;
  for (int k = 0; k < n_scenes; ++k) {
    const ut_scene_grads &g = grads[k];
    if (scenes[k].n > 0 && (!g.d_means || !g.d_log_scales || !g.d_quats || !g.d_opacity_logits || !g.d_sh))
      return UT_ERR_INVALID_ARG;
    DevScene &s = bd.s[k];
    s.gacc = reinterpret_cast<float *>(gw);
    const size_t acc_bytes = backward_workspace_bytes(scenes[k].n, dop.kbuffer > 0);
    s.kbrec = dop.kbuffer > 0 ? reinterpret_cast<float4 *>(gw + acc_bytes / 2) : nullptr;
    gw += acc_bytes;
    s.d_means = g.d_means;
    s.d_log_scales = g.d_log_scales;
    s.d_quats = g.d_quats;
    s.d_logits = g.d_opacity_logits;
    s.d_sh = g.d_sh;
    s.grad_off = goff;
    goff += scenes[k].n;
  }
  const char *ws = static_cast<const char *>(workspace);
  return launch_composite_bwd(bd, dop, reinterpret_cast<const int16_t *>(ws + L.rect),
                              reinterpret_cast<const uint32_t *>(ws + L.vals),
                              reinterpret_cast<const uint32_t *>(ws + L.ranges), gw,
                              reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
