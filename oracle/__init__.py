"""FP64 CPU oracle of the 3DGUT hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It wraps ``ut3d_oracle.c`` (plain C, FP64, OpenMP over
pixels and particles) through ctypes and shares no code with the CUDA library.

Everything here is marshalling: numpy arrays in, numpy arrays out.  The arithmetic
lives in ``ut3d_oracle.c``, where each function cites the paper passage it restates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ut3d_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

# pixel flag bits (mirror the enum in ut3d_oracle.c)
F_RECT_EDGE, F_ALPHA_MIN, F_TSTOP, F_DEPTH_TIE = 1, 2, 4, 8
F_CULL_TIE, F_PIXEL_EDGE, F_ILL_COND, F_ALPHA_MAX, F_INVALID_PIXEL, F_CLAMP = 16, 32, 64, 128, 256, 512
# flags that can change the forward result between an FP32 and an FP64 evaluation
# (depth-tied pairs and stop-threshold ties are not in this set: their effect is bounded by the
# per-pixel slack / aslack that render() returns)
F_FORWARD_TIES = (F_RECT_EDGE | F_ALPHA_MIN | F_DEPTH_TIE | F_CULL_TIE | F_PIXEL_EDGE | F_ILL_COND)
# flags whose decisions can change a gradient between an FP32 and an FP64 evaluation: the
# forward's, the alpha_max clamp and the stop (both change which terms are differentiated),
# and a colour channel at its clamp at 0 (the colour is continuous there, its derivative not)
F_BACKWARD_TIES = F_FORWARD_TIES | F_ALPHA_MAX | F_TSTOP | F_CLAMP


def build(force: bool = False) -> str:
    """Compiles ut3d_oracle.c into liboracle.so beside it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(C.Structure):
    _fields_ = [("model", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("rolling_shutter", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("k", C.c_double * 4),
                ("q_start", C.c_double * 4), ("t_start", C.c_double * 3),
                ("q_end", C.c_double * 4), ("t_end", C.c_double * 3), ("near_plane", C.c_double)]


class Scene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int32),
                ("sh_degree", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("t_min", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("rs_iters", C.c_int32),
                ("ut_alpha", C.c_double), ("ut_beta", C.c_double), ("ut_kappa", C.c_double),
                ("extent_sigma", C.c_double), ("projection", C.c_int32), ("colour_mode", C.c_int32),
                ("kernel_degree", C.c_int32), ("kbuffer", C.c_int32), ("eps_tau", C.c_double)]


class Tol(C.Structure):
    _fields_ = [("eps_px", C.c_double), ("eps_rel", C.c_double), ("depth_ulps", C.c_int32),
                ("cond_min", C.c_double), ("eps_t", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.orc_theta_max.restype = C.c_double
        L.orc_theta_max.argtypes = [P]
        L.orc_project_world.restype = C.c_int
        L.orc_project_world.argtypes = [C.POINTER(Camera), C.c_double, C.c_int, P, P, P, P]
        L.orc_pixel_ray.restype = C.c_int
        L.orc_pixel_ray.argtypes = [C.POINTER(Camera), C.c_double, C.c_double, C.c_double, P, P, P, P]
        L.orc_sh_basis.argtypes = [C.c_int, P, P]
        L.orc_sh_basis_grad.argtypes = [C.c_int, P, P, P]
        L.orc_ut_estimate.restype = C.c_int
        L.orc_ut_estimate.argtypes = [C.POINTER(Camera), C.c_double, C.c_int, C.c_double, C.c_double,
                                      C.c_double, P, P, P, P, P, P, P]
        L.orc_pose.argtypes = [C.POINTER(Camera), C.c_double, P, P]
        L.orc_cam_limit.restype = C.c_double
        L.orc_cam_limit.argtypes = [C.POINTER(Camera)]
        L.orc_ewa_estimate.restype = C.c_int
        L.orc_ewa_estimate.argtypes = [C.POINTER(Camera), C.c_double, C.c_int, P, P, P, P, P, P, P]
        L.orc_project.argtypes = [C.POINTER(Scene), C.POINTER(Camera), C.POINTER(Options), C.POINTER(Tol),
                                  P, P, P, P, P, P, P, P]
        L.orc_count_keys.restype = C.c_int64
        L.orc_count_keys.argtypes = [C.c_int, P, C.c_int, C.c_int]
        L.orc_bin.argtypes = [C.c_int, P, P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]
        L.orc_render.argtypes = [C.POINTER(Scene), C.POINTER(Camera), C.POINTER(Options), C.POINTER(Tol),
                                 P, P, P, P, C.c_int, P, P, C.c_int, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_render_list.argtypes = [C.POINTER(Scene), C.POINTER(Camera), C.POINTER(Options), P, P,
                                      C.c_int, C.c_int, C.c_int, P, P, P]
        L.orc_backward.argtypes = [C.POINTER(Scene), C.POINTER(Camera), C.POINTER(Options), P, P, C.c_int,
                                   P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- structs from plain dicts

def make_camera(cam: dict) -> Camera:
    """cam: dict with model ('pinhole'|'fisheye'|'ortho' or 0/1/2), width, height, fx, fy, cx, cy,
    k (4), q_start (w,x,y,z), t_start, q_end, t_end, rolling_shutter, near_plane."""
    models = {"pinhole": 0, "fisheye": 1, "ortho": 2, "pinhole_radial": 3}
    m = cam["model"]
    c = Camera()
    c.model = models[m] if isinstance(m, str) else int(m)
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.rolling_shutter = int(cam.get("rolling_shutter", 0))
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    c.k[:] = [float(v) for v in cam.get("k", (0, 0, 0, 0))]
    c.q_start[:] = [float(v) for v in cam.get("q_start", (1, 0, 0, 0))]
    c.t_start[:] = [float(v) for v in cam.get("t_start", (0, 0, 0))]
    c.q_end[:] = [float(v) for v in cam.get("q_end", cam.get("q_start", (1, 0, 0, 0)))]
    c.t_end[:] = [float(v) for v in cam.get("t_end", cam.get("t_start", (0, 0, 0)))]
    c.near_plane = float(cam.get("near_plane", 0.2))
    return c


def make_options(opts: dict | None = None) -> Options:
    o = opts or {}
    r = Options()
    r.tile_w, r.tile_h = int(o.get("tile_w", 16)), int(o.get("tile_h", 16))
    r.t_min = float(o.get("t_min", 1e-4))
    r.alpha_min = float(o.get("alpha_min", 1.0 / 255.0))
    r.alpha_max = float(o.get("alpha_max", 0.99))
    r.rs_iters = int(o.get("rs_iters", 3))
    r.ut_alpha, r.ut_beta, r.ut_kappa = (float(o.get(k, d)) for k, d in
                                         (("ut_alpha", 1.0), ("ut_beta", 2.0), ("ut_kappa", 0.0)))
    r.extent_sigma = float(o.get("extent_sigma", 3.0))
    r.projection = int(o.get("projection", 0))    # 0 UT, 1 EWA
    r.colour_mode = int(o.get("colour_mode", 0))  # 0 per pixel, 1 per particle
    r.kernel_degree = int(o.get("kernel_degree", 2))  # generalised Gaussian degree n
    r.kbuffer = int(o.get("kbuffer", 0))              # 0: tile order; k > 0: per-ray k-buffer
    r.eps_tau = float(o.get("eps_tau", 1e-5))          # k-buffer near-tie tolerance (flags only)
    return r


def make_tol(tol: dict | None = None) -> Tol:
    t = tol or {}
    r = Tol()
    r.eps_px = float(t.get("eps_px", 2e-3))
    r.eps_rel = float(t.get("eps_rel", 1e-4))
    r.depth_ulps = int(t.get("depth_ulps", 4))
    r.cond_min = float(t.get("cond_min", 0.05))
    r.eps_t = float(t.get("eps_t", 1e-3))
    return r


class _SceneArrays:
    def __init__(self, scene: dict):
        self.means = _f32(scene["means"]).reshape(-1, 3)
        self.log_scales = _f32(scene["log_scales"]).reshape(-1, 3)
        self.quats = _f32(scene["quats"]).reshape(-1, 4)
        self.logits = _f32(scene["opacity_logits"]).reshape(-1)
        self.sh = _f32(scene["sh"])
        self.deg = int(scene["sh_degree"])
        n = self.means.shape[0]
        self.sh = self.sh.reshape(n, (self.deg + 1) ** 2, 3)
        self.s = Scene(_p(self.means), _p(self.log_scales), _p(self.quats), _p(self.logits), _p(self.sh),
                       n, self.deg)
        self.n = n


# ---------------------------------------------------------------- public functions

def theta_max(k) -> float:
    return lib().orc_theta_max(_p(_f64(k)))


def sh_basis(deg: int, d) -> np.ndarray:
    d = _f64(d)
    Y = np.zeros((deg + 1) ** 2)
    lib().orc_sh_basis(deg, _p(d), _p(Y))
    return Y


def sh_basis_grad(deg: int, d):
    """(Y, G): the basis at d and the gradient of its polynomials, G[j][k] = dY_k / d(d_j)."""
    d = _f64(d)
    Y = np.zeros(16)
    G = np.zeros(48)
    lib().orc_sh_basis_grad(deg, _p(d), _p(Y), _p(G))
    n = (deg + 1) ** 2
    return Y[:n], G.reshape(3, 16)[:, :n]


def project_point(cam: dict, x, rs_iters: int = 3):
    """g(x) for a world point (rolling-shutter fixed point included). Returns (valid, uv, t)."""
    c = make_camera(cam)
    tm = lib().orc_cam_limit(C.byref(c))
    uv = np.zeros(2)
    t = np.zeros(1)
    m = np.zeros(1)
    v = lib().orc_project_world(C.byref(c), tm, rs_iters, _p(_f64(x)), _p(uv), _p(t), _p(m))
    return bool(v), uv, float(t[0])


def pose_at(cam: dict, t: float):
    """World->camera rotation (3x3) and translation of the camera at shutter time t."""
    c = make_camera(cam)
    R = np.zeros(9)
    T = np.zeros(3)
    lib().orc_pose(C.byref(c), float(t), _p(R), _p(T))
    return R.reshape(3, 3), T


def pixel_ray(cam: dict, px: float, py: float):
    """World ray (o, d) through the pixel-plane point (px, py). Returns (valid, o, d)."""
    c = make_camera(cam)
    tm = lib().orc_cam_limit(C.byref(c))
    o, d, em, dp = np.zeros(3), np.zeros(3), np.zeros(1), np.zeros(1)
    v = lib().orc_pixel_ray(C.byref(c), tm, float(px), float(py), _p(o), _p(d), _p(em), _p(dp))
    return bool(v), o, d


def ut_estimate(cam: dict, mu, R, s, ut=(1.0, 2.0, 0.0), rs_iters: int = 3):
    """Unscented-Transform 2D mean and covariance (xx, xy, yy) of one Gaussian."""
    c = make_camera(cam)
    tm = lib().orc_cam_limit(C.byref(c))
    vmu, cov, t, m = np.zeros(2), np.zeros(3), np.zeros(1), np.zeros(1)
    v = lib().orc_ut_estimate(C.byref(c), tm, rs_iters, float(ut[0]), float(ut[1]), float(ut[2]),
                              _p(_f64(mu)), _p(_f64(np.asarray(R).reshape(9))), _p(_f64(s)), _p(vmu), _p(cov),
                              _p(t), _p(m))
    return bool(v), vmu, cov


def ewa_estimate(cam: dict, mu, R, s, rs_iters: int = 3):
    """First-order (EWA) 2D mean and covariance (xx, xy, yy) of one Gaussian (eq. ewa_splatting)."""
    c = make_camera(cam)
    tm = lib().orc_cam_limit(C.byref(c))
    vmu, cov, t, m = np.zeros(2), np.zeros(3), np.zeros(1), np.zeros(1)
    v = lib().orc_ewa_estimate(C.byref(c), tm, rs_iters, _p(_f64(mu)), _p(_f64(np.asarray(R).reshape(9))),
                               _p(_f64(s)), _p(vmu), _p(cov), _p(t), _p(m))
    return bool(v), vmu, cov


def project(scene: dict, cam: dict, opts: dict | None = None, tol: dict | None = None) -> dict:
    """Per-particle projection (Algorithm 1; UT, or EWA when opts["projection"] == 1) of the scene."""
    S = _SceneArrays(scene)
    n = S.n
    out = dict(mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), depth=np.zeros(n),
               depth32=np.zeros(n, np.float32), rect=np.zeros((n, 4), np.int32), ntiles=np.zeros(n, np.int32),
               edges=np.zeros((n, 4)), tie=np.zeros(n, np.int32))
    c, o, t = make_camera(cam), make_options(opts), make_tol(tol)
    lib().orc_project(C.byref(S.s), C.byref(c), C.byref(o), C.byref(t), *(_p(out[k]) for k in
                      ("mean2d", "cov2d", "depth", "depth32", "rect", "ntiles", "edges", "tie")))
    return out


def bin_keys(depth32, rect, width: int, height: int, tile_w: int = 16, tile_h: int = 16):
    """Duplicate + stable sort + per-tile ranges. Returns (keys u64, vals u32, ranges u32[T,2])."""
    depth32 = _f32(depth32)
    rect = _i32(rect).reshape(-1, 4)
    n = rect.shape[0]
    L = lib()
    K = L.orc_count_keys(n, _p(rect), tile_w, tile_h)
    T = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    keys = np.zeros(max(K, 1), np.uint64)
    vals = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros((T, 2), np.uint32)
    L.orc_bin(n, _p(depth32), _p(rect), width, height, tile_w, tile_h, _p(keys), _p(vals), _p(ranges))
    return keys[:K], vals[:K], ranges


def render(scene: dict, cam: dict, opts: dict | None = None, proj: dict | None = None,
           pixels=None, tol: dict | None = None, no_rect: bool = False) -> dict:
    """Brute-force FP64 render of the listed pixels (all pixels by default).

    proj: output of project() (or a dict with rect / depth32 and optionally edges / tie,
    e.g. synthetic arrays).  Returns rgb[P,3], alpha[P], tfinal[P], nblend[P], flags[P],
    slack / aslack (the colour / opacity change depth-tied pairs and stop ties can cause),
    fslack / faslack (a bound on what flipping the other flagged decisions can change),
    rslack / raslack (the FP32 rounding bound of the blended particles' alphas), and px, py."""
    S = _SceneArrays(scene)
    if proj is None:
        proj = project(scene, cam, opts, tol)
    W, H = int(cam["width"]), int(cam["height"])
    if pixels is None:
        yy, xx = np.mgrid[0:H, 0:W]
        px, py = xx.reshape(-1), yy.reshape(-1)
    else:
        px, py = pixels
    px, py = _i32(px), _i32(py)
    P = px.shape[0]
    rect = _i32(proj["rect"]).reshape(-1, 4)
    depth32 = _f32(proj["depth32"])
    edges = _f64(proj["edges"]).reshape(-1, 4) if proj.get("edges") is not None else None
    tie = _i32(proj["tie"]) if proj.get("tie") is not None else None
    out = dict(rgb=np.zeros((P, 3)), alpha=np.zeros(P), tfinal=np.zeros(P), nblend=np.zeros(P, np.int32),
               flags=np.zeros(P, np.int32), slack=np.zeros(P), aslack=np.zeros(P), fslack=np.zeros(P),
               faslack=np.zeros(P), rslack=np.zeros(P), raslack=np.zeros(P), px=px, py=py)
    c, o, t = make_camera(cam), make_options(opts), make_tol(tol)
    lib().orc_render(C.byref(S.s), C.byref(c), C.byref(o), C.byref(t), _p(rect), _p(depth32), _p(edges),
                     _p(tie), P, _p(px), _p(py), int(no_rect), _p(out["rgb"]), _p(out["alpha"]),
                     _p(out["tfinal"]), _p(out["nblend"]), _p(out["flags"]), _p(out["slack"]),
                     _p(out["aslack"]), _p(out["fslack"]), _p(out["faslack"]), _p(out["rslack"]),
                     _p(out["raslack"]))
    return out


def render_list(scene: dict, cam: dict, opts: dict | None, rect, depth32, px: int, py: int, lst):
    """Composites an explicit ordered particle list at one pixel. Returns (rgb[3], tfinal)."""
    S = _SceneArrays(scene)
    lst = np.ascontiguousarray(lst, dtype=np.uint32)
    rgb, tf = np.zeros(3), np.zeros(1)
    c, o = make_camera(cam), make_options(opts)
    lib().orc_render_list(C.byref(S.s), C.byref(c), C.byref(o), _p(_i32(rect)), _p(_f32(depth32)), int(px),
                          int(py), lst.shape[0], _p(lst), _p(rgb), _p(tf))
    return rgb, float(tf[0])


def backward(scene: dict, cam: dict, opts: dict | None, proj: dict, pixels, g_rgb, g_alpha,
             magnitudes: bool = False) -> dict:
    """FP64 reverse-mode gradients of sum(g_rgb * rgb) + sum(g_alpha * alpha) over the listed pixels.

    magnitudes=True also returns, under "mag", the same sums taken over the absolute values of
    every pair's term (with the linear maps made entry-wise absolute): the scale of the rounding
    error of a floating-point evaluation of each gradient element."""
    S = _SceneArrays(scene)
    px, py = _i32(pixels[0]), _i32(pixels[1])
    P = px.shape[0]
    n, nsh = S.n, (S.deg + 1) ** 2

    def zeros():
        return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                    opacity_logits=np.zeros(n), sh=np.zeros((n, nsh, 3)))
    out = zeros()
    mag = zeros() if magnitudes else None
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    c, o = make_camera(cam), make_options(opts)
    lib().orc_backward(C.byref(S.s), C.byref(c), C.byref(o), _p(_i32(proj["rect"])), _p(_f32(proj["depth32"])),
                       P, _p(px), _p(py), _p(_f64(g_rgb).reshape(-1)), _p(_f64(g_alpha).reshape(-1)),
                       *(_p(out[k]) for k in keys), *((_p(mag[k]) for k in keys) if mag else (None,) * 5))
    if mag is not None:
        out["mag"] = mag
    return out


def num_threads() -> int:
    return lib().orc_num_threads()
