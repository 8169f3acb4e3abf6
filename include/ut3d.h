/*
 * ut3d.h — C ABI of the GB300-native 3DGUT hot path (one GPU, sm_103a).
 *
 * 3DGUT renders a set of 3D Gaussian particles by (1) estimating every particle's
 * 2D footprint with the Unscented Transform through an arbitrary camera model
 * (Sec. 4.1, Algorithms 1-2 of the supplementary), (2) duplicating and sorting
 * (tile | depth) keys (Sec. 4.3; the Duplicate and Sort phases of Table 2), and
 * (3) compositing each pixel front to back, evaluating every particle in 3D at the
 * point of maximum response along the pixel ray (Sec. 4.2, eq. GaussianMaxResponse,
 * eq. QuadratureVolumeRendering).  A hand-written backward (supplementary Sec. B)
 * differentiates (3) with respect to all particle parameters.
 *
 * Conventions shared by every entry point
 *   - Every pointer to array data is a DEVICE pointer unless stated otherwise; the
 *     caller owns all memory.  Structs (ut_scene, ut_camera, ...) are host structs
 *     passed by host pointer and only read during the call.
 *   - Calls are asynchronous on `stream` (NULL = the legacy default stream) and
 *     return a ut_status.  Host-side validation failures return without launching
 *     anything.  UT_ERR_CUDA reports a launch error seen by cudaGetLastError().
 *     Nothing aborts and no C++ exception crosses the ABI.
 *   - Nothing allocates device memory: scratch memory is passed in by the caller,
 *     sized with the *_workspace_size() queries.
 *   - Arrays are structure-of-arrays, FP32, row-major, with no padding:
 *       means[n][3], log_scales[n][3] (s = exp), quats[n][4] (w,x,y,z; need not be
 *       normalised), opacity_logits[n] (sigma = sigmoid), sh[n][(deg+1)^2][3]
 *       (real spherical harmonics with the Condon-Shortley phase, index l*l+l+m,
 *       colour = max(sum beta Y(d) + 1/2, 0) at the unit pixel-ray direction d).
 *   - Cameras map world to camera as x_c = R x + t, +z forward, +y down; pixel
 *     centres are at integer + 1/2.  Images are H rows of W pixels.
 */
#ifndef UT3D_H
#define UT3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ut_stream; /* identical to cudaStream_t */

typedef enum {
  UT_OK = 0,
  UT_ERR_INVALID_ARG = 1, /* a size, enum, pointer or camera field failed validation */
  UT_ERR_CAPACITY = 2,    /* a caller buffer is too small (see bin_and_sort) */
  UT_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
  UT_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  UT_ERR_UNSUPPORTED = 5  /* a valid request the library does not implement */
} ut_status;

/* UT_CAM_PINHOLE_RADIAL: u = fx x_n (1 + k1 r^2 + k2 r^4 + k3 r^6) + cx (likewise v) with
 * (x_n, y_n) = (X, Y) / Z and r = |(x_n, y_n)| (k[3] unused); points beyond the first turning
 * point of r_d(r) = r (1 + ...) are not imaged, nor pixels beyond r_d there. */
typedef enum { UT_CAM_PINHOLE = 0, UT_CAM_FISHEYE = 1, UT_CAM_PINHOLE_RADIAL = 2 } ut_cam_model;

/* Camera (the extrinsic W and intrinsic D of Algorithm 1).
 *   pinhole: valid iff z > near_plane; (u,v) = (fx x/z + cx, fy y/z + cy).
 *   fisheye (polynomial, Kannala-Brandt): theta = atan2(sqrt(x^2+y^2), z),
 *     theta_d = theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8),
 *     (u,v) = (fx theta_d x/r + cx, fy theta_d y/r + cy), r = sqrt(x^2+y^2);
 *     valid iff |x_c| > near_plane and theta <= theta_max, where theta_max is pi/2 or
 *     the first zero of d theta_d / d theta on (0, pi/2].
 *   rolling_shutter = 1: row v is exposed at time t = v / (H-1); the pose at t has the
 *     translation lerped and the rotation slerped between (q_start, t_start) and
 *     (q_end, t_end).  A projected point takes its time from a fixed point on its
 *     own projected row (see ut_project).  rolling_shutter = 0 uses the start pose.
 *   Limits: 1 <= width, height <= 32767 (rectangles are int16); rolling shutter needs
 *   height >= 2; fx, fy > 0; near_plane > 0; quaternions non-zero; all finite. */
typedef struct {
  int32_t model;
  int32_t width, height;
  int32_t rolling_shutter;
  float fx, fy, cx, cy;
  float k[4];
  float q_start[4], t_start[3];
  float q_end[4], t_end[3];
  float near_plane;
} ut_camera;

/* Unscented-Transform hyperparameters (eq. weights_1/2): lambda = alpha^2 (3 + kappa) - 3;
 * the paper uses (alpha, beta, kappa) = (1, 2, 0).  Requires 3 + lambda > 0. */
typedef struct {
  float alpha, beta, kappa;
} ut_params;

/* The particles (Sec. 3): device pointers, n >= 0, 0 <= sh_degree <= 3. */
typedef struct {
  const float *means;
  const float *log_scales;
  const float *quats;
  const float *opacity_logits;
  const float *sh;
  int32_t n, sh_degree;
} ut_scene;

/* Renderer knobs.  Defaults (ut_default_options): 16x16 tiles, t_min = 1e-4,
 * alpha_min = 1/255, alpha_max = 0.99, rs_iters = 3, newton_iters = 12, extent_sigma = 3.
 *   alpha = min(alpha_max, sigma rho); a particle with sigma rho < alpha_min is skipped;
 *   compositing stops BEFORE blending a particle that would take T below t_min.
 *   extent: half-widths k sqrt(Sigma'_xx), k sqrt(Sigma'_yy) with
 *   k = min(extent_sigma, sqrt(2 ln(sigma / alpha_min))) ("use opacity to compute a
 *   tighter 2D extent", Algorithm 1).  tile_w * tile_h must be 64..512 and a multiple of 32.
 *   newton_iters bounds the fisheye ray inversion (safeguarded Newton).
 *   projection: UT_PROJECTION_UT (default; Sec. 4.1) or UT_PROJECTION_EWA, the first-order
 *   estimate of 3DGS (eq. ewa_splatting) kept as an A/B baseline: v = g(W mu),
 *   Sigma' = J W Sigma W^T J^T with J the Jacobian of g at the camera-space mean (under a
 *   rolling shutter, W is the pose at the mean's own shutter time).  It changes only the 2D
 *   extent and the culling (compositing is in 3D either way).
 *   colour_mode: UT_COLOUR_PER_PIXEL (default; SH at each pixel's ray direction, Sec. 3) or
 *   UT_COLOUR_PER_PARTICLE, a faster mode that evaluates the SH once per particle at the
 *   direction from the camera centre (at the mean's shutter time) to the mean; its gradient
 *   also reaches the mean through that direction.  Under UT_PROJECTION_EWA the radial pinhole
 *   uses the undistorted pinhole Jacobian (as 3DGS's EWA does). */
/*   kernel_degree: n = 2 (default) is the Gaussian (eq. gaussian_kernel); n in 3..8 the
 *   generalised Gaussian of supplementary Sec. A, rho = exp(-1/2 3^(2-n) d^n) of the Mahalanobis
 *   distance d (the same response as the Gaussian at d = 3), evaluated at the same tau_max;
 *   combined with UT_COLOUR_PER_PARTICLE it is rejected with UT_ERR_UNSUPPORTED.
 *   kbuffer: 0 (default) blends in the tile's depth order; k in 1..16 selects "Ours (sorted)"
 *   (Sec. 4.4), a per-ray k-buffer: hits enter a buffer of k entries, a full buffer blends the
 *   closest (by tau_max; the earlier arrival on equal tau_max) of its hits and the arriving one,
 *   and the rest are blended in that order at the end of the list (the paper uses k = 16).  composite_backward and
 *   render_batch_backward differentiate through the same blending order (the selections carry
 *   no gradient; every allowed tile size and k fits one block's shared memory).
 *   composite_forward rejects statistics
 *   with a k-buffer; combined with per-particle colours or kernel_degree != 2 it is unsupported. */
#define UT_PROJECTION_UT 0
#define UT_PROJECTION_EWA 1
#define UT_COLOUR_PER_PIXEL 0
#define UT_COLOUR_PER_PARTICLE 1
typedef struct {
  int32_t tile_w, tile_h;
  float t_min, alpha_min, alpha_max;
  int32_t rs_iters, newton_iters;
  float extent_sigma;
  int32_t projection;
  int32_t colour_mode;
  int32_t kernel_degree;
  int32_t kbuffer;
} ut_options;

void ut_default_options(ut_options *opt);
const char *ut_status_string(ut_status s);

/* Number of CUDA kernels this library has launched in the calling process (all devices,
 * all threads).  A measurement aid with no counterpart in the paper: benchmarks read it
 * before and after a step to report how many of the library's kernels the step ran. */
uint64_t ut_kernel_launch_count(void);

/* Peak-throughput probes (a measurement aid with no counterpart in the paper: the compositing
 * kernels' roofline fractions divide by peaks measured on the same GPU).  Launches blocks x
 * threads threads (threads a multiple of 32, at most 256), each running `iters` iterations of 8
 * independent dependency chains of one operation:
 *   UT_PROBE_FMA: fma.rn.f32 (2 FP32 flop each),
 *   UT_PROBE_EX2: ex2.approx.ftz.f32 (the special-function unit's base-2 exponential).
 * Operations launched = blocks * threads * iters * 8; time the launch with events on `stream`.
 * out[blocks * threads] (device, caller-owned) receives each thread's chain sum.
 * Errors: UT_ERR_INVALID_ARG for an unknown kind, bad sizes or a NULL out. */
#define UT_PROBE_FMA 0
#define UT_PROBE_EX2 1
ut_status ut_peak_probe(int32_t kind, int32_t blocks, int32_t threads, int32_t iters, float *out, ut_stream stream);

/* Debug builds (a testing aid with no counterpart in the paper).  A library compiled with
 * UT_DEBUG checks, where a wrong index would write outside a buffer, that key and value positions
 * are below the key capacity, tile ids below the number of tiles, particle indices below the
 * scene's count and rectangles inside the image, and records the first violation instead of
 * faulting; its binning workspace carries guard bytes after every sub-buffer (so its
 * ut_bin_workspace_size is larger), filled at the start of each bin_and_sort and checked at its
 * end.  A release build compiles all of this away.
 *   ut_debug_enabled: 1 in a debug build, else 0.
 *   ut_debug_read: record[4] = {code, a, b, c} of the first violation since the last reset
 *     (code UT_DBG_NONE = 0 when there is none); reset != 0 clears it.  Synchronises with the
 *     device.  UT_ERR_UNSUPPORTED in a release build.
 *   ut_debug_check_bin_workspace: checks the guard bytes of a binning workspace that bin_and_sort
 *     used with the same n, key_capacity, camera and options (recording UT_DBG_CANARY with a =
 *     the sub-buffer, b = the byte offset in its guard, c = the byte found).  UT_ERR_UNSUPPORTED
 *     in a release build. */
#define UT_DBG_NONE 0
#define UT_DBG_KEY_INDEX 1 /* a = position, b = capacity */
#define UT_DBG_TILE_ID 2   /* a = tile, b = number of tiles */
#define UT_DBG_RECT 3      /* a = particle, b = x0 | y0 << 16, c = x1 | y1 << 16 */
#define UT_DBG_PARTICLE 4  /* a = particle index, b = the scene's count */
#define UT_DBG_CANARY 5
int32_t ut_debug_enabled(void);
ut_status ut_debug_read(uint32_t record[4], int32_t reset);
ut_status ut_debug_check_bin_workspace(const void *workspace, int32_t n, int64_t key_capacity, const ut_camera *cam,
                                       const ut_options *opt, ut_stream stream);

/* UT projection of every particle (Algorithm 1 and Algorithm 2; eq. sigma_points,
 * weights_1, weights_2, 2d_conic_1, 2d_conic_2).
 *   Sigma points: mu, mu +- sqrt(3+lambda) s_k R[:,k] (the square root R S of
 *   Sigma = R S S^T R^T).  Each is projected by the camera; under a rolling shutter
 *   its time starts at 1/2 and is updated rs_iters times by
 *   t <- clamp((v - 1/2)/(H-1), 0, 1), then projected once more at that time.
 *   A particle is culled if any projection is invalid, if sigma < alpha_min, if a
 *   parameter is not finite, or if its pixel rectangle is empty.
 * Outputs (device, n entries each; written for every particle):
 *   mean2d[n][2] = v_mu; cov2d[n][3] = (xx, xy, yy) of Sigma';
 *   depth[n] = |x_c(mu)| at the mean's shutter time (0 when culled);
 *   rect[n][4] int16 = (x0, y0, x1, y1) inclusive pixel indices whose centres lie in
 *   [v - h, v + h], clipped to the image; culled => (0, 0, -1, -1);
 *   ntiles[n] = number of tiles the rect overlaps (0 when culled).
 * Errors: UT_ERR_INVALID_ARG for a bad scene / camera / params / options or a NULL
 * output with n > 0. */
ut_status ut_project(const ut_scene *scene, const ut_camera *cam, const ut_params *ut, const ut_options *opt,
                     float *mean2d, float *cov2d, float *depth, int16_t *rect, uint32_t *ntiles,
                     ut_stream stream);

/* The camera map g of a batch of world points (no counterpart in the paper's pipeline; the
 * reference projection of Monte Carlo samples in the UT / EWA accuracy study, and a utility):
 * uv[i] = g(points[i]) with the model and the rolling-shutter time fixed point of ut_project
 * (rs_iters from opt); valid[i] = 1 when every projection taken was valid (imaged), else 0 and
 * uv[i] holds what the last projection gave.  points[n][3], uv[n][2] (float), valid[n] (int32),
 * all device.  Errors: UT_ERR_INVALID_ARG for a bad camera / options or NULL buffers with n > 0. */
ut_status ut_project_points(const float *points, int32_t n, const ut_camera *cam, const ut_options *opt, float *uv,
                            int32_t *valid, ut_stream stream);

/* Bytes of scratch memory bin_and_sort needs for n particles and a key capacity. */
size_t ut_bin_workspace_size(int32_t n, int64_t key_capacity, const ut_camera *cam, const ut_options *opt);

/* Duplicate and sort (Sec. 4.3; Table 2 "Duplicate" and "Sort").
 *   For every particle with ntiles > 0, in increasing index order, and every tile its
 *   rect overlaps in row-major order, one entry key = (tile << 32) | bits(depth),
 *   val = particle index, where tile = ty * ceil(W / tile_w) + tx and bits() is the IEEE
 *   bit pattern of the positive FP32 depth.  Entries are sorted stably by key, so equal
 *   keys keep increasing particle index.  tile_ranges[t] = {start, end} of tile t's run
 *   in the sorted list, {0, 0} for an empty tile.
 * Inputs: depth, rect, ntiles as written by ut_project (n entries, device).
 * Outputs (device): keys[key_capacity] (may be NULL: the keys are then not written),
 *   vals[key_capacity], tile_ranges[2 * T], T = ceil(W/tile_w) * ceil(H/tile_h),
 *   k_out = one device int64 receiving the number of entries K.
 * Capacity: the call is asynchronous and cannot know K in advance.  If K > key_capacity
 *   the kernels write K to *k_out, leave keys / vals untouched and set every range to
 *   {0, 0}; the caller must check *k_out after the stream completes and retry with a
 *   larger capacity.  key_capacity must be < 2^32.
 * Workspace: workspace_bytes >= ut_bin_workspace_size(n, key_capacity, cam, opt),
 *   256-byte aligned, contents need not be initialised. */
ut_status bin_and_sort(int32_t n, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                       const ut_camera *cam, const ut_options *opt, void *workspace, size_t workspace_bytes,
                       int64_t key_capacity, uint64_t *keys, uint32_t *vals, uint32_t *tile_ranges,
                       int64_t *k_out, ut_stream stream);

/* bin_and_sort without caller scratch memory (the paper has no counterpart: this is a
 * deployment convenience).  For callers that cannot allocate device memory or hand the
 * library a workspace, e.g. a plugin inside a host application that owns all device memory
 * through its own pool, or a real-time frame loop that must never enter the CUDA allocator.
 * Same inputs, outputs, asynchrony and capacity contract as bin_and_sort; the scratch comes
 * from a fixed array of UT_BIN_STATIC_SCRATCH_BYTES (32 MiB) compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   - Arguments bin_and_sort rejects are rejected with the same status.  Then, launching
 *     nothing, UT_ERR_CAPACITY when
 *     ut_bin_workspace_size(n, key_capacity, cam, opt) > UT_BIN_STATIC_SCRATCH_BYTES.
 *     The scratch takes about 16 B per particle plus 22 B per unit of key capacity, so the
 *     largest key_capacity that fits is 1,446,400 for n = 100k particles on a 1920x1080
 *     camera with 16x16 tiles (562,816 for n = 1M; 1,524,480 for n = 0).
 *   - Every call looks up the array's device address with the calling thread's device
 *     current; the first call on a device also loads the library's device code there, so
 *     make that first call before capturing any stream.
 *   - Allocates nothing.  All calls share the one array and it keeps the last call's
 *     contents; calls whose work overlaps on the GPU race on it: order them (one stream). */
#define UT_BIN_STATIC_SCRATCH_BYTES (32u << 20)
ut_status bin_and_sort_static(int32_t n, const float *depth, const int16_t *rect, const uint32_t *ntiles,
                              const ut_camera *cam, const ut_options *opt, int64_t key_capacity, uint64_t *keys,
                              uint32_t *vals, uint32_t *tile_ranges, int64_t *k_out, ut_stream stream);

/* Bytes of scratch memory composite_forward needs for this camera and these options; 0 for
 * invalid arguments. */
size_t ut_forward_workspace_size(const ut_camera *cam, const ut_options *opt);

/* Front-to-back compositing (eq. QuadratureVolumeRendering) with the particle response
 * evaluated in 3D at its maximum along the pixel ray (eq. GaussianMaxResponse):
 *   o_g = S^-1 R^T (o - mu), d_g = S^-1 R^T d, omega^2 = |o_g x d_g|^2 / |d_g|^2,
 *   alpha = min(alpha_max, sigma exp(-omega^2 / 2)).
 * Pixel (x, y) considers, in tile order, only particles whose rect contains (x, y);
 * rays: pinhole d_c = ((x+1/2-cx)/fx, (y+1/2-cy)/fy, 1); fisheye inverts theta_d by a
 * safeguarded Newton iteration; pixels beyond theta_d(theta_max) are not imaged
 * (rgb = 0, alpha = 0, t_final = 1).  Rolling shutter: row y uses the pose at y/(H-1).
 * Inputs: scene, camera, options as for ut_project; rect from ut_project; vals and
 *   tile_ranges from bin_and_sort (same camera and options).
 * Outputs (device): rgb[3][H][W] (planar), alpha[H][W] = 1 - T_final,
 *   t_final[H][W] = T_final, n_used[H][W] = one past the position in vals of the last
 *   blended particle (0 if none; consumed by composite_backward).
 * Workspace: >= ut_forward_workspace_size(cam, opt) bytes, 256-byte aligned (the tile
 *   schedule: tiles are composited longest predicted walk first; the order changes no result).
 * stats (device, nullable): if given, stats[0] += number of (pixel, particle) response
 *   evaluations (pixel inside the rect, before the pixel stopped) and stats[1] += number
 *   of blended particles; a measurement aid, NULL in normal use. */
ut_status composite_forward(const ut_scene *scene, const ut_camera *cam, const ut_options *opt,
                            const int16_t *rect, const uint32_t *vals, const uint32_t *tile_ranges, float *rgb,
                            float *alpha, float *t_final, uint32_t *n_used, void *workspace,
                            size_t workspace_bytes, unsigned long long *stats, ut_stream stream);

/* Bytes of scratch memory composite_backward needs for n particles rendered with this camera
 * and these options (per-particle accumulators, with opt->kbuffer > 0 a per-particle record
 * table of the same size, and a per-tile schedule); 0 for invalid arguments. */
size_t ut_backward_workspace_size(int32_t n, const ut_camera *cam, const ut_options *opt);

/* Gradient of a scalar loss L through composite_forward (supplementary Sec. B):
 *   given dL/drgb[3][H][W] and dL/dalpha[H][W], writes dL/d(parameter) for every
 *   particle: d_means[n][3], d_log_scales[n][3], d_quats[n][4], d_opacity_logits[n],
 *   d_sh[n][(deg+1)^2][3] (overwritten, not accumulated).  The projection contributes no
 *   gradient: rect, depth order and tile membership are piecewise constant (Sec. 4.1).
 * Inputs: everything composite_forward was given plus its outputs rgb, t_final, n_used.
 * Workspace: >= ut_backward_workspace_size(n, cam, opt) bytes, 256-byte aligned. */
ut_status composite_backward(const ut_scene *scene, const ut_camera *cam, const ut_options *opt,
                             const int16_t *rect, const uint32_t *vals, const uint32_t *tile_ranges,
                             const float *rgb, const float *t_final, const uint32_t *n_used, const float *d_rgb,
                             const float *d_alpha, void *workspace, size_t workspace_bytes, float *d_means,
                             float *d_log_scales, float *d_quats, float *d_opacity_logits, float *d_sh,
                             ut_stream stream);

/* ------------------------------------------------------------------------------------------
 * Batches of views: one launch sequence renders several (scene, camera) views at once — the
 * multi-view training step and the unit of work of the serving loop.  The method per view is
 * exactly that of ut_project + bin_and_sort + composite_forward (the single-view calls are
 * the batch of one view); particles of all views are projected in one kernel, all their
 * (tile, particle) entries are sorted together (tile ids are global over the batch), and
 * one compositing kernel covers every tile of every view.
 * ------------------------------------------------------------------------------------------ */
#define UT_MAX_BATCH_VIEWS 32
#define UT_MAX_BATCH_SCENES 8

/* One view of a batch.  rgb[3][H][W] and alpha[H][W] (device) are written by render_batch;
 * t_final[H][W] and n_used[H][W] are written when non-NULL and are required by
 * render_batch_backward, which also reads d_rgb[3][H][W] and d_alpha[H][W]. */
typedef struct {
  int32_t scene; /* index into the scenes array */
  ut_camera camera;
  float *rgb, *alpha, *t_final;
  uint32_t *n_used;
  const float *d_rgb, *d_alpha;
} ut_view;

/* Bytes of scratch render_batch needs; the same buffer, untouched, feeds render_batch_backward.
 * Returns 0 for invalid arguments. */
size_t ut_batch_workspace_size(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                               const ut_options *opt, int64_t key_capacity);

/* Forward render of n_views (1..UT_MAX_BATCH_VIEWS) views of n_scenes (1..UT_MAX_BATCH_SCENES)
 * scenes (all with the same sh_degree), with the UT projection, binning and compositing defined
 * by ut_project, bin_and_sort and composite_forward.  key_capacity bounds the total number of
 * (tile, particle) entries of the batch; *k_out (device int64) receives that total, and if it
 * exceeds key_capacity every view's image is left black (all ranges empty): check *k_out after
 * the stream completes and retry with a larger capacity (and workspace).  Asynchronous on
 * `stream`; allocates nothing. */
ut_status render_batch(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                       const ut_params *ut, const ut_options *opt, void *workspace, size_t workspace_bytes,
                       int64_t key_capacity, int64_t *k_out, ut_stream stream);

/* Per-scene gradient outputs of render_batch_backward (device, layouts as composite_backward). */
typedef struct {
  float *d_means, *d_log_scales, *d_quats, *d_opacity_logits, *d_sh;
} ut_scene_grads;

/* Bytes of scratch render_batch_backward needs for these scenes and views (per-particle
 * accumulators of every scene, with opt->kbuffer > 0 a per-particle record table of the same
 * size, and a per-tile schedule over all views); 0 for invalid arguments. */
size_t ut_batch_backward_workspace_size(const ut_scene *scenes, int32_t n_scenes, const ut_view *views,
                                        int32_t n_views, const ut_options *opt);

/* Gradient of a loss through render_batch (supplementary Sec. B): every view's d_rgb / d_alpha
 * is propagated into its scene's parameters; gradients of views sharing a scene add up.
 * workspace / key_capacity must be the buffer and capacity render_batch used, unchanged since;
 * views must carry the t_final and n_used render_batch wrote.  grads[n_scenes] are overwritten. */
ut_status render_batch_backward(const ut_scene *scenes, int32_t n_scenes, const ut_view *views, int32_t n_views,
                                const ut_options *opt, const void *workspace, size_t workspace_bytes,
                                int64_t key_capacity, void *grad_workspace, size_t grad_workspace_bytes,
                                const ut_scene_grads *grads, ut_stream stream);

/* ------------------------------------------------------------------------------------------
 * Serving: a device-resident request loop (no counterpart in the paper; the paper renders one
 * image at a time).  Scenes stay resident (caller-owned device memory).  Requests (scene,
 * camera) are submitted from any host thread and return immediately; a worker thread admits
 * pending requests as memory in the caller's device arena frees up (each request needs its
 * output image; each batch its render_batch workspace), groups up to max_batch_views of them
 * into one render_batch launch sequence (optionally captured and replayed as a CUDA graph),
 * and keeps up to max_in_flight batches on the GPU at once on separate streams, so requests
 * that arrive while others render overlap with them on the device.  Completion is detected
 * with CUDA events polled on the host; no kernel waits on anything.  A batch whose key count
 * overflowed its capacity is re-run with a larger capacity before its requests complete; a
 * request whose batch overflowed six times fails with UT_ERR_CAPACITY (reported by
 * ut_server_wait).  Outputs are carved from the top of the arena and workspaces from the
 * bottom, so that outputs waiting for their reader do not fragment the workspaces' space.
 * ------------------------------------------------------------------------------------------ */
typedef struct ut_server ut_server;

typedef struct {
  int32_t max_batch_views; /* 1..UT_MAX_BATCH_VIEWS views per launch sequence */
  int32_t max_in_flight;   /* 1..8 batches concurrently on the GPU (one stream each) */
  int32_t use_graphs;      /* 1: capture each batch's launches and replay them as a CUDA graph */
  float key_headroom;      /* key capacity = headroom x (estimated keys); >= 1, e.g. 1.3 */
  ut_options options;      /* renderer knobs shared by all requests */
  ut_params ut;            /* UT parameters shared by all requests */
} ut_server_config;

/* Creates a server over n_scenes resident scenes (1..UT_MAX_BATCH_SCENES, same sh_degree; the
 * arrays must stay valid until ut_server_destroy) and a caller-owned device arena of
 * arena_bytes (256-byte aligned) from which it carves outputs and workspaces.  Starts the
 * worker thread.  The calling thread's current device is the server's device. */
ut_status ut_server_create(const ut_server_config *cfg, const ut_scene *scenes, int32_t n_scenes, void *arena,
                           size_t arena_bytes, ut_server **out);

/* Queues a request; *id identifies it.  UT_ERR_CAPACITY if the request alone can never fit
 * the arena. */
ut_status ut_server_submit(ut_server *s, int32_t scene, const ut_camera *cam, uint64_t *id);

/* Waits up to timeout_ms (0 = just poll) for request id.  On completion sets *done = 1 and
 * returns device pointers to its rgb[3][H][W] and alpha[H][W] (valid until released) and its
 * latency in ms from submission to completion; otherwise *done = 0 (UT_ERR_TIMEOUT only if
 * timeout_ms > 0 elapsed).  Errors of the request's batch are reported here. */
ut_status ut_server_wait(ut_server *s, uint64_t id, int32_t timeout_ms, int32_t *done, const float **rgb,
                         const float **alpha, double *latency_ms);

/* Releases a completed request's output memory back to the arena. */
ut_status ut_server_release(ut_server *s, uint64_t id);

/* Counters since creation: completed requests, batches launched, key-capacity retries, graph
 * replays, graph (re)instantiations, retries whose batch went back to the queue (no memory for
 * the larger workspace yet), and failed requests. */
typedef struct {
  uint64_t completed, batches, retries, graph_launches, graph_instantiations, requeued, failed;
} ut_server_stats;
ut_status ut_server_get_stats(ut_server *s, ut_server_stats *stats);

/* Stops the worker after the batches in flight complete (bounded wait) and frees host state.
 * Pending requests are dropped.  The arena is the caller's to free. */
ut_status ut_server_destroy(ut_server *s);

#ifdef __cplusplus
}
#endif

#endif /* UT3D_H */
