"""ctypes binding of the C ABI in include/ut3d.h (argument marshalling only).

Every function here forwards device pointers and plain structs to libut3d.so; all
arithmetic of the hot path runs in the library's CUDA kernels.  Loading fails loudly
when the library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libut3d.so")

UT_OK, UT_ERR_INVALID_ARG, UT_ERR_CAPACITY, UT_ERR_CUDA, UT_ERR_TIMEOUT, UT_ERR_UNSUPPORTED = range(6)
CAM_MODELS = {"pinhole": 0, "fisheye": 1, "pinhole_radial": 2}
UT_PROBE_FMA, UT_PROBE_EX2 = 0, 1  # ut_peak_probe kinds


class UtError(RuntimeError):
    def __init__(self, fn: str, status: int, text: str):
        super().__init__(f"{fn} failed: {text} (status {status})")
        self.status = status


class UtCamera(C.Structure):
    _fields_ = [("model", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("rolling_shutter", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("k", C.c_float * 4), ("q_start", C.c_float * 4), ("t_start", C.c_float * 3),
                ("q_end", C.c_float * 4), ("t_end", C.c_float * 3), ("near_plane", C.c_float)]


class UtParams(C.Structure):
    _fields_ = [("alpha", C.c_float), ("beta", C.c_float), ("kappa", C.c_float)]


class UtScene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int32), ("sh_degree", C.c_int32)]


class UtOptions(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("t_min", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("rs_iters", C.c_int32), ("newton_iters", C.c_int32),
                ("extent_sigma", C.c_float), ("projection", C.c_int32), ("colour_mode", C.c_int32),
                ("kernel_degree", C.c_int32), ("kbuffer", C.c_int32)]


class UtView(C.Structure):
    _fields_ = [("scene", C.c_int32), ("camera", UtCamera), ("rgb", C.c_void_p), ("alpha", C.c_void_p),
                ("t_final", C.c_void_p), ("n_used", C.c_void_p), ("d_rgb", C.c_void_p), ("d_alpha", C.c_void_p)]


class UtSceneGrads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p)]


class UtServerConfig(C.Structure):
    _fields_ = [("max_batch_views", C.c_int32), ("max_in_flight", C.c_int32), ("use_graphs", C.c_int32),
                ("key_headroom", C.c_float), ("options", UtOptions), ("ut", UtParams)]


class UtServerStats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("batches", C.c_uint64), ("retries", C.c_uint64),
                ("graph_launches", C.c_uint64), ("graph_instantiations", C.c_uint64), ("requeued", C.c_uint64),
                ("failed", C.c_uint64)]


MAX_BATCH_VIEWS = 32
MAX_BATCH_SCENES = 8

# every exported symbol of include/ut3d.h, with its ctypes signature
_P = C.c_void_p
_SC, _VW = C.POINTER(UtScene), C.POINTER(UtView)
SIGNATURES = {
    "ut_default_options": (None, [C.POINTER(UtOptions)]),
    "ut_status_string": (C.c_char_p, [C.c_int]),
    "ut_kernel_launch_count": (C.c_uint64, []),
    "ut_peak_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P]),
    "ut_debug_enabled": (C.c_int32, []),
    "ut_debug_read": (C.c_int, [C.POINTER(C.c_uint32), C.c_int32]),
    "ut_debug_check_bin_workspace": (C.c_int, [_P, C.c_int32, C.c_int64, C.POINTER(UtCamera), C.POINTER(UtOptions),
                                               _P]),
    "ut_project": (C.c_int, [C.POINTER(UtScene), C.POINTER(UtCamera), C.POINTER(UtParams), C.POINTER(UtOptions),
                             _P, _P, _P, _P, _P, _P]),
    "ut_bin_workspace_size": (C.c_size_t, [C.c_int32, C.c_int64, C.POINTER(UtCamera), C.POINTER(UtOptions)]),
    "bin_and_sort": (C.c_int, [C.c_int32, _P, _P, _P, C.POINTER(UtCamera), C.POINTER(UtOptions), _P, C.c_size_t,
                               C.c_int64, _P, _P, _P, _P, _P]),
    "bin_and_sort_static": (C.c_int, [C.c_int32, _P, _P, _P, C.POINTER(UtCamera), C.POINTER(UtOptions), C.c_int64,
                                      _P, _P, _P, _P, _P]),
    "ut_project_points": (C.c_int, [_P, C.c_int32, C.POINTER(UtCamera), C.POINTER(UtOptions), _P, _P, _P]),
    "ut_forward_workspace_size": (C.c_size_t, [C.POINTER(UtCamera), C.POINTER(UtOptions)]),
    "composite_forward": (C.c_int, [C.POINTER(UtScene), C.POINTER(UtCamera), C.POINTER(UtOptions), _P, _P, _P, _P,
                                    _P, _P, _P, _P, C.c_size_t, _P, _P]),
    "ut_backward_workspace_size": (C.c_size_t, [C.c_int32, C.POINTER(UtCamera), C.POINTER(UtOptions)]),
    "ut_batch_workspace_size": (C.c_size_t, [_SC, C.c_int32, _VW, C.c_int32, C.POINTER(UtOptions), C.c_int64]),
    "render_batch": (C.c_int, [_SC, C.c_int32, _VW, C.c_int32, C.POINTER(UtParams), C.POINTER(UtOptions), _P,
                               C.c_size_t, C.c_int64, _P, _P]),
    "ut_batch_backward_workspace_size": (C.c_size_t, [_SC, C.c_int32, _VW, C.c_int32, C.POINTER(UtOptions)]),
    "ut_server_create": (C.c_int, [C.POINTER(UtServerConfig), _SC, C.c_int32, _P, C.c_size_t,
                                   C.POINTER(C.c_void_p)]),
    "ut_server_submit": (C.c_int, [_P, C.c_int32, C.POINTER(UtCamera), C.POINTER(C.c_uint64)]),
    "ut_server_wait": (C.c_int, [_P, C.c_uint64, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_void_p), C.POINTER(C.c_double)]),
    "ut_server_release": (C.c_int, [_P, C.c_uint64]),
    "ut_server_get_stats": (C.c_int, [_P, C.POINTER(UtServerStats)]),
    "ut_server_destroy": (C.c_int, [_P]),
    "render_batch_backward": (C.c_int, [_SC, C.c_int32, _VW, C.c_int32, C.POINTER(UtOptions), _P, C.c_size_t,
                                        C.c_int64, _P, C.c_size_t, C.POINTER(UtSceneGrads), _P]),
    "composite_backward": (C.c_int, [C.POINTER(UtScene), C.POINTER(UtCamera), C.POINTER(UtOptions), _P, _P, _P, _P,
                                     _P, _P, _P, _P, _P, C.c_size_t, _P, _P, _P, _P, _P, _P]),
}

_lib = None


def lib(path: str | None = None):
    """Loads libut3d.so (built by paper_2412_12507_gb300.build) and declares its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libut3d.so not found at {p}: build it with paper_2412_12507_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def check(fn: str, status: int):
    if status != UT_OK:
        raise UtError(fn, status, lib().ut_status_string(status).decode())


def default_options() -> UtOptions:
    o = UtOptions()
    lib().ut_default_options(C.byref(o))
    return o


def make_camera(cam: dict) -> UtCamera:
    c = UtCamera()
    m = cam["model"]
    c.model = CAM_MODELS[m] if isinstance(m, str) else int(m)
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


def make_options(opts: dict | None = None) -> UtOptions:
    o = default_options()
    for k, v in (opts or {}).items():
        if k in ("tile_w", "tile_h", "rs_iters", "newton_iters", "projection", "colour_mode", "kernel_degree",
                 "kbuffer"):
            setattr(o, k, int(v))
        elif k in ("t_min", "alpha_min", "alpha_max", "extent_sigma"):
            setattr(o, k, float(v))
    return o


def make_params(opts: dict | None = None) -> UtParams:
    o = opts or {}
    return UtParams(float(o.get("ut_alpha", 1.0)), float(o.get("ut_beta", 2.0)), float(o.get("ut_kappa", 0.0)))


def make_scene(means, log_scales, quats, logits, sh, sh_degree: int) -> UtScene:
    """Scene struct from device tensors (anything with data_ptr()); the caller keeps them alive."""
    n = int(means.shape[0])
    ptr = lambda t: t.data_ptr() if t is not None and n > 0 else None  # noqa: E731
    return UtScene(ptr(means), ptr(log_scales), ptr(quats), ptr(logits), ptr(sh), n, int(sh_degree))
