"""Seeded synthetic inputs for the 3DGUT hot path.

This module only draws inputs (scenes, cameras, options, targets) with numpy's
``default_rng``; it holds none of the method's arithmetic and imports neither the
CUDA library nor the oracle, so both sides can be fed the identical FP32 arrays.

The recipes mirror the workloads the paper measures on (MipNeRF360-like dense
object scenes, a Scannet++-like 180-degree fisheye, Waymo-like rolling-shutter
motion), which are not available here; synthetic scenes of the stated shapes,
sizes and distributions stand in for them.

Conventions: quaternions are (w, x, y, z); camera poses are world->camera
(x_c = R x + t) with +z forward and +y down; pixel centres sit at integer + 1/2.
"""
from __future__ import annotations

import math

import numpy as np

# The degree-0 SH basis value is the constant 1/(2 sqrt(pi)); a DC colour u in
# [0,1] is stored as the coefficient (u - 1/2) * 2 sqrt(pi) so that the colour the
# renderer reconstructs at any direction is u.
_DC_SCALE = 2.0 * math.sqrt(math.pi)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n, deg, higher_std=0.1):
    K = (deg + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (rng.uniform(0.0, 1.0, (n, 3)) - 0.5) * _DC_SCALE
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_std, (n, K - 1, 3))
    return sh


def _pack(means, log_scales, quats, logits, sh, deg):
    return dict(means=np.ascontiguousarray(means, np.float32),
                log_scales=np.ascontiguousarray(log_scales, np.float32),
                quats=np.ascontiguousarray(quats, np.float32),
                opacity_logits=np.ascontiguousarray(logits, np.float32),
                sh=np.ascontiguousarray(sh, np.float32), sh_degree=int(deg))


def scene_cube(n, seed, log_s=(-3.0, 0.5), logit_std=1.0, deg=0, lo=(-1, -1, 2), hi=(1, 1, 4), higher_std=0.1):
    """Means uniform in the box [lo, hi]; log-scales N(mean, std); random unit quaternions;
    opacity logits N(0, logit_std); SH of degree `deg` with DC colour U(0,1), higher bands
    N(0, higher_std)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(lo, hi, (n, 3))
    ls = rng.normal(log_s[0], log_s[1], (n, 3))
    q = _unit_quats(rng, n)
    lg = rng.normal(0.0, logit_std, n)
    sh = _sh(rng, n, deg, higher_std)
    return _pack(means, ls, q, lg, sh, deg)


def scene_shell(n, seed, radius=5.0, radial_std=0.3, log_s=(-4.0, 0.7), logit_std=1.5, deg=3, higher_std=0.1,
                volume_frac=0.0, volume_half=1.0):
    """Means on a noisy spherical shell around the origin (direction uniform on S^2,
    radius + N(0, radial_std)); a fraction `volume_frac` uniform in the cube
    [-volume_half, volume_half]^3 instead."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = radius + rng.normal(0.0, radial_std, n)
    means = u * r[:, None]
    nv = int(round(volume_frac * n))
    if nv:
        idx = rng.permutation(n)[:nv]
        means[idx] = rng.uniform(-volume_half, volume_half, (nv, 3))
    ls = rng.normal(log_s[0], log_s[1], (n, 3))
    q = _unit_quats(rng, n)
    lg = rng.normal(0.0, logit_std, n)
    sh = _sh(rng, n, deg, higher_std)
    return _pack(means, ls, q, lg, sh, deg)


def _rot_to_quat(R):
    """Unit quaternion (w,x,y,z) of a rotation matrix (input construction only)."""
    R = np.asarray(R, dtype=np.float64)
    tr = np.trace(R)
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    else:
        i = int(np.argmax(np.diag(R)))
        if i == 0:
            s = math.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
            q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
        elif i == 1:
            s = math.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
            q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
        else:
            s = math.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
            q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    return q / np.linalg.norm(q)


def look_at_pose(position, target=(0.0, 0.0, 0.0)):
    """World->camera (q, t) of a camera at `position` looking at `target`, +y down."""
    c = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    r = np.cross(down, f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R_cw = np.stack([r, d, f], axis=1)
    R_wc = R_cw.T
    return _rot_to_quat(R_wc), -R_wc @ c


def camera(model, width, height, fx=None, fy=None, cx=None, cy=None, k=(0, 0, 0, 0), q=(1, 0, 0, 0),
           t=(0, 0, 0), q_end=None, t_end=None, rolling_shutter=0, near_plane=0.2):
    """Plain camera description shared by both sides (a dict of numbers)."""
    if fx is None:
        fx = width / math.pi if model == "fisheye" else float(width)
    if fy is None:
        fy = fx
    f = lambda v: float(np.float32(v))  # noqa: E731  (FP32 values: both sides see identical numbers)
    return dict(model=model, width=int(width), height=int(height), fx=f(fx), fy=f(fy),
                cx=f(width / 2 if cx is None else cx), cy=f(height / 2 if cy is None else cy),
                k=[f(v) for v in k], q_start=[f(v) for v in q], t_start=[f(v) for v in t],
                q_end=[f(v) for v in (q if q_end is None else q_end)],
                t_end=[f(v) for v in (t if t_end is None else t_end)],
                rolling_shutter=int(rolling_shutter), near_plane=f(near_plane))


def options(**kw):
    o = dict(tile_w=16, tile_h=16, t_min=1e-4, alpha_min=1.0 / 255.0, alpha_max=0.99, rs_iters=3,
             newton_iters=12, ut_alpha=1.0, ut_beta=2.0, ut_kappa=0.0, extent_sigma=3.0,
             projection=0, colour_mode=0, kernel_degree=2, kbuffer=0)
    o.update(kw)
    # FP32 values: both sides see identical thresholds
    for k in ("t_min", "alpha_min", "alpha_max", "ut_alpha", "ut_beta", "ut_kappa", "extent_sigma"):
        o[k] = float(np.float32(o[k]))
    return o


def rs_end_pose(shift=0.05, yaw_deg=2.0):
    """End-of-frame world->camera pose for a camera starting at the identity that moved
    `shift` along its x axis and yawed `yaw_deg` about its y axis."""
    a = math.radians(yaw_deg)
    R_cw = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    c = np.array([shift, 0.0, 0.0])
    R_wc = R_cw.T
    return _rot_to_quat(R_wc), -R_wc @ c


def fisheye_k(rng):
    return rng.uniform(-0.05, 0.05, 4)


# ---------------------------------------------------------------- named workloads

def small_pinhole(seed=0, n=1000):
    """1,000 Gaussians in the box [-1,1]^2 x [2,4] in front of a 64x64 pinhole (f = 64)."""
    scene = scene_cube(n, seed, log_s=(-3.0, 0.5), logit_std=1.0, deg=0)
    cam = camera("pinhole", 64, 64, fx=64.0, fy=64.0)
    return dict(name="pinhole64_n1k", scene=scene, camera=cam, options=options())


def fisheye_shell(seed=1, n=100_000, width=1280, height=720):
    """100k Gaussians on a shell of radius 5 around a 180-degree polynomial fisheye at the origin."""
    scene = scene_shell(n, seed, radius=5.0, radial_std=0.3, log_s=(-4.0, 0.7), logit_std=1.5, deg=3)
    rng = np.random.default_rng(seed + 1000)
    cam = camera("fisheye", width, height, k=fisheye_k(rng))
    return dict(name=f"fisheye{width}x{height}_shell_n{n}", scene=scene, camera=cam, options=options())


def rs_fisheye(seed=2, n=1_000_000, width=1920, height=1080, deg=3):
    """1M Gaussians as in the small case (box in front), SH degree 3; 1920x1080 polynomial
    fisheye with a rolling shutter moving 0.05 along x and yawing 2 degrees over the frame."""
    scene = scene_cube(n, seed, log_s=(-3.0, 0.5), logit_std=1.0, deg=deg)
    rng = np.random.default_rng(seed + 1000)
    qe, te = rs_end_pose(0.05, 2.0)
    cam = camera("fisheye", width, height, k=fisheye_k(rng), q_end=qe, t_end=te, rolling_shutter=1)
    return dict(name=f"rsfisheye{width}x{height}_n{n}", scene=scene, camera=cam, options=options())


def target_image(seed, width, height):
    rng = np.random.default_rng(seed + 5000)
    return rng.uniform(0.0, 1.0, (3, height, width)).astype(np.float32)


def orbit_cameras(seed, specs, radius=4.0):
    """Cameras on a radius-`radius` orbit looking at the origin, seeded azimuth U(0, 2 pi)
    and elevation U(-30, 30) degrees. specs: list of (model, width, height, rolling_shutter)."""
    rng = np.random.default_rng(seed + 2000)
    cams = []
    for model, w, h, rs in specs:
        az = rng.uniform(0, 2 * math.pi)
        el = math.radians(rng.uniform(-30, 30))
        pos = radius * np.array([math.cos(el) * math.cos(az), -math.sin(el), math.cos(el) * math.sin(az)])
        q, t = look_at_pose(pos)
        if model == "pinhole":
            cams.append(camera("pinhole", w, h, fx=0.6 * w, fy=0.6 * w, q=q, t=t))
            continue
        k = fisheye_k(rng)
        if rs:
            # the camera moves 0.05 along its own x axis and yaws 2 degrees during the frame
            R_wc = _quat_to_rot_np(q)
            a = math.radians(2.0)
            R_yaw = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
            R_cw_end = R_wc.T @ R_yaw
            c_end = pos + R_wc.T @ np.array([0.05, 0.0, 0.0])
            qe = _rot_to_quat(R_cw_end.T)
            te = -R_cw_end.T @ c_end
            cams.append(camera("fisheye", w, h, k=k, q=q, t=t, q_end=qe, t_end=te, rolling_shutter=1))
        else:
            cams.append(camera("fisheye", w, h, k=k, q=q, t=t))
    return cams


def _quat_to_rot_np(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def multiview(seed=3, n=3_000_000):
    """3M Gaussians (70% shell of radius 5, 30% uniform in [-1,1]^3), SH degree 3, and 8 orbit
    views: 4 pinhole 1920x1080, 2 fisheye 1600x1600, 2 rolling-shutter fisheye 2048x1536."""
    scene = scene_shell(n, seed, radius=5.0, radial_std=0.3, log_s=(-4.5, 0.8), logit_std=1.0, deg=3,
                        volume_frac=0.3)
    specs = [("pinhole", 1920, 1080, 0)] * 4 + [("fisheye", 1600, 1600, 0)] * 2 + [("fisheye", 2048, 1536, 1)] * 2
    return dict(name=f"multiview8_n{n}", scene=scene, cameras=orbit_cameras(seed, specs), options=options())


def random_rects(seed, n, width, height, max_w=40, max_h=40, cull_frac=0.1):
    """Synthetic integer pixel rectangles and positive depths for exercising the integer
    stage on its own (no projection involved)."""
    rng = np.random.default_rng(seed)
    x0 = rng.integers(0, width, n)
    y0 = rng.integers(0, height, n)
    x1 = np.minimum(x0 + rng.integers(0, max_w, n), width - 1)
    y1 = np.minimum(y0 + rng.integers(0, max_h, n), height - 1)
    rect = np.stack([x0, y0, x1, y1], axis=1).astype(np.int32)
    cull = rng.uniform(size=n) < cull_frac
    rect[cull] = (0, 0, -1, -1)
    depth = rng.uniform(0.5, 20.0, n).astype(np.float32)
    # a few exact depth ties so that stability is exercised
    if n >= 8:
        depth[1::7] = depth[0]
    return rect, depth
