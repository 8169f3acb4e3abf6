"""The C-ABI library loads and exports every entry point include/ut3d.h declares; its
host-side validation rejects bad arguments without touching a GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_2412_12507_gb300 import abi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2412_12507_gb300 import build
    build.build()
    return abi.lib()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ut3d.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", txt, re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return")))


def test_every_declared_symbol_is_exported(L):
    names = header_functions()
    assert {"ut_project", "bin_and_sort", "composite_forward", "composite_backward"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
        assert n in abi.SIGNATURES, f"binding lacks {n}"


def test_defaults_and_strings(L):
    o = abi.default_options()
    assert (o.tile_w, o.tile_h, o.rs_iters, o.newton_iters) == (16, 16, 3, 12)
    assert abs(o.t_min - 1e-4) < 1e-9 and abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    assert L.ut_status_string(abi.UT_ERR_CAPACITY) == b"capacity exceeded"
    assert L.ut_status_string(99) == b"unknown status"


def test_workspace_sizes(L):
    cam = abi.make_camera(synth.camera("fisheye", 1920, 1080))
    o = abi.default_options()
    a = L.ut_bin_workspace_size(1000, 10000, C.byref(cam), C.byref(o))
    b = L.ut_bin_workspace_size(1000, 20000, C.byref(cam), C.byref(o))
    assert 0 < a < b
    assert L.ut_bin_workspace_size(-1, 10, C.byref(cam), C.byref(o)) == 0
    w = L.ut_backward_workspace_size(1000, C.byref(cam), C.byref(o))
    tiles = 120 * 68  # 1920x1080 in 16x16 tiles
    assert w >= 1000 * 16 * 4 + 2 * 4 * tiles and w % 256 == 0
    ok = abi.default_options()
    ok.kbuffer = 16  # the k-buffer backward adds a 64-byte record per particle
    assert L.ut_backward_workspace_size(1000, C.byref(cam), C.byref(ok)) >= w + 1000 * 16 * 4
    assert L.ut_backward_workspace_size(-1, C.byref(cam), C.byref(o)) == 0
    assert L.ut_backward_workspace_size(1000, None, C.byref(o)) == 0
    f = L.ut_forward_workspace_size(C.byref(cam), C.byref(o))
    assert f >= 2 * 4 * tiles and f % 256 == 0
    assert L.ut_forward_workspace_size(None, C.byref(o)) == 0


def test_workspace_sizes_never_shrink_as_the_key_capacity_grows(L):
    """The serving loop searches for the largest key capacity whose scratch fits its arena,
    which relies on the workspace size being non-decreasing in the capacity."""
    o = abi.default_options()
    caps = (0, 1, 1023, 1024, 4096, 1 << 16, 1 << 20, 12_345_678, 1 << 31)
    cams = (synth.camera("fisheye", 1920, 1080), synth.camera("pinhole", 64, 48, fx=60.0),
            synth.camera("pinhole", 3840, 2160, fx=2000.0))
    for cam in cams:
        c = abi.make_camera(cam)
        sizes = [L.ut_bin_workspace_size(5000, k, C.byref(c), C.byref(o)) for k in caps]
        assert sizes[0] > 0 and all(a <= b for a, b in zip(sizes, sizes[1:])), sizes
    dummy = 256  # a 256-byte aligned stand-in address: the size query never dereferences it
    sc = abi.UtScene(dummy, dummy, dummy, dummy, dummy, 5000, 3)
    views = (abi.UtView * len(cams))()
    for v, cam in zip(views, cams):
        v.scene, v.camera, v.rgb, v.alpha = 0, abi.make_camera(cam), dummy, dummy
    sizes = [L.ut_batch_workspace_size(C.byref(sc), 1, views, len(cams), C.byref(o), k) for k in caps]
    assert sizes[0] > 0 and all(a <= b for a, b in zip(sizes, sizes[1:])), sizes


def _project(L, cam, opts=None, n=0, params=None):
    sc = abi.UtScene(None, None, None, None, None, n, 0)
    c = abi.make_camera(cam)
    o = abi.make_options(opts)
    u = params or abi.make_params(None)
    return L.ut_project(C.byref(sc), C.byref(c), C.byref(u), C.byref(o), None, None, None, None, None, None)


def test_validation_rejects_bad_arguments(L):
    good = synth.camera("pinhole", 64, 64, fx=64.0)
    assert _project(L, good) == abi.UT_OK  # n = 0: nothing to launch
    bad_cams = [dict(good, model=7), dict(good, width=0), dict(good, height=40000), dict(good, fx=-1.0),
                dict(good, near_plane=0.0), dict(good, fx=float("nan")), dict(good, q_start=[0, 0, 0, 0]),
                dict(good, rolling_shutter=1, height=1), dict(good, rolling_shutter=2)]
    for c in bad_cams:
        assert _project(L, c) == abi.UT_ERR_INVALID_ARG, c
    for o in (dict(tile_w=4, tile_h=4), dict(tile_w=33, tile_h=2), dict(tile_w=32, tile_h=32),
              dict(t_min=-1.0), dict(alpha_min=0.0), dict(alpha_max=1.0), dict(extent_sigma=0.0),
              dict(newton_iters=0), dict(rs_iters=100)):
        assert _project(L, good, o) == abi.UT_ERR_INVALID_ARG, o
    # 3 + lambda must be positive
    assert _project(L, good, params=abi.UtParams(0.1, 2.0, -3.0)) == abi.UT_ERR_INVALID_ARG
    # a scene with particles but NULL arrays
    sc = abi.UtScene(None, None, None, None, None, 5, 0)
    c, o, u = abi.make_camera(good), abi.default_options(), abi.make_params(None)
    assert L.ut_project(C.byref(sc), C.byref(c), C.byref(u), C.byref(o), None, None, None, None, None,
                        None) == abi.UT_ERR_INVALID_ARG
    # sh degree out of range
    sc = abi.UtScene(None, None, None, None, None, 0, 4)
    assert L.ut_project(C.byref(sc), C.byref(c), C.byref(u), C.byref(o), None, None, None, None, None,
                        None) == abi.UT_ERR_INVALID_ARG


def test_bin_and_sort_validation(L):
    cam = abi.make_camera(synth.camera("pinhole", 64, 64, fx=64.0))
    o = abi.default_options()
    # capacity must fit 32 bits; workspace must be present and large enough
    assert L.bin_and_sort(0, None, None, None, C.byref(cam), C.byref(o), None, 0, 1 << 32, None, None, None, None,
                          None) == abi.UT_ERR_INVALID_ARG
    fake = C.c_void_p(256)
    assert L.bin_and_sort(0, None, None, None, C.byref(cam), C.byref(o), fake, 16, 100, None, fake, fake, fake,
                          None) == abi.UT_ERR_INVALID_ARG


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        abi.lib(str(tmp_path / "nope.so"))


def test_peak_probe_validates_arguments(L):
    """The throughput probe rejects bad arguments on the host, before any launch."""
    for args in ((7, 1, 256, 10), (0, 0, 256, 10), (0, 1, 48, 10), (0, 1, 512, 10), (1, 1, 256, 0)):
        assert L.ut_peak_probe(*args, C.c_void_p(16), None) == abi.UT_ERR_INVALID_ARG
    assert L.ut_peak_probe(0, 1, 256, 10, None, None) == abi.UT_ERR_INVALID_ARG


def test_release_build_has_no_debug_checks(L):
    """The release library reports no debug build and refuses the debug entry points."""
    assert L.ut_debug_enabled() == 0
    rec = (C.c_uint32 * 4)()
    assert L.ut_debug_read(rec, 1) == abi.UT_ERR_UNSUPPORTED
    cam = abi.make_camera(synth.camera("pinhole", 32, 32, fx=32.0))
    o = abi.default_options()
    st = L.ut_debug_check_bin_workspace(C.c_void_p(256), 10, 100, C.byref(cam), C.byref(o), None)
    assert st == abi.UT_ERR_UNSUPPORTED
