"""The debug build of the library (-DUT_DEBUG) on small cases.

Its index range checks (key and value positions below the key capacity, tile ids below the
number of tiles, listed particles inside the scene, rectangles inside the image) must stay silent
on the parity workloads, and the guard bytes after every sub-buffer of the binning workspace must
survive every call; a guard overwritten from the host (the only fault injected: bytes of our own
allocation) must be reported.  No GPU fault is provoked.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2412_12507_gb300 import abi, build, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbg():
    """Routes the module's calls through the debug library; the release one is restored after."""
    L = abi.lib(build.build(debug=True))
    assert L.ut_debug_enabled() == 1
    saved = abi.lib()
    abi._lib = L
    _read(L)  # clear
    yield L
    abi._lib = saved


def _read(L, reset=True):
    rec = (C.c_uint32 * 4)()
    assert L.ut_debug_read(rec, int(reset)) == abi.UT_OK
    return list(rec)


def _tiny(n, W, H, seed, model="pinhole", rs=0):
    sc = synth.scene_cube(n, seed, log_s=(-1.8, 0.3), deg=1, lo=(-0.3, -0.3, 1.5), hi=(0.3, 0.3, 2.5))
    qe, te = synth.rs_end_pose(0.05, 2.0)
    cam = synth.camera(model, W, H, fx=float(W) if model != "fisheye" else None, q_end=qe, t_end=te,
                       rolling_shutter=rs)
    return sc, cam


CASES = {
    "pinhole64_n1k": lambda: (synth.small_pinhole()["scene"], synth.small_pinhole()["camera"]),
    **{f"8x8_n{n}": (lambda n=n: _tiny(n, 8, 8, 70 + n)) for n in (1, 2, 3, 5)},
    "fisheye_rs_40x30": lambda: _tiny(200, 40, 30, 80, "fisheye", 1),
    "ragged_37x29": lambda: _tiny(300, 37, 29, 81),
}


@pytest.mark.parametrize("name", list(CASES))
def test_debug_checks_stay_silent(dbg, name):
    sc, cam = CASES[name]()
    op = synth.options()
    scene = render.Scene.from_arrays(sc)
    r = render.Renderer(cam, op, capacity=1 << 12)
    f = r.forward(scene)
    g = r.backward(scene, torch.ones_like(f.rgb), torch.ones_like(f.alpha))
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in g.values())
    assert _read(dbg) == [0, 0, 0, 0], name
    # the binning workspace's guards are intact after the call
    n = scene.n
    p = r.ws.buf.data_ptr()
    assert dbg.ut_debug_check_bin_workspace(p + (-p) % 256, n, r.capacity, C.byref(abi.make_camera(cam)),
                                            C.byref(abi.make_options(op)), None) == abi.UT_OK
    assert _read(dbg) == [0, 0, 0, 0], name


def test_debug_k_buffer_and_batch_stay_silent(dbg):
    sc, cam = _tiny(400, 48, 32, 90, "fisheye", 1)
    scene = render.Scene.from_arrays(sc)
    for op in (synth.options(kbuffer=4), synth.options(tile_w=8, tile_h=8)):
        r = render.Renderer(cam, op, capacity=1 << 12)
        f = r.forward(scene)
        r.backward(scene, torch.ones_like(f.rgb), torch.ones_like(f.alpha))
    views = [(0, cam), (0, synth.camera("pinhole", 33, 21, fx=30.0))]
    br = render.BatchRenderer([scene], synth.options(), capacity=1 << 12)
    frames = br.forward(views, grad=True)
    br.backward([torch.ones_like(fr.rgb) for fr in frames], [torch.ones_like(fr.alpha) for fr in frames])
    torch.cuda.synchronize()
    assert _read(dbg) == [0, 0, 0, 0]


def test_overwritten_guard_is_reported(dbg):
    """Bytes written over the binning workspace from the host (its guards included) are found by
    the guard check, which names the first damaged guard."""
    sc, cam = _tiny(50, 32, 32, 91)
    op = synth.options()
    scene = render.Scene.from_arrays(sc)
    proj = render.project(scene, cam, op)
    c, o = abi.make_camera(cam), abi.make_options(op)
    cap = 4096
    nbytes = dbg.ut_bin_workspace_size(scene.n, cap, C.byref(c), C.byref(o))
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) & ~255
    T = render.tile_count(cam, op)
    vals = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = torch.empty((T, 2), dtype=torch.int32, device="cuda")
    k_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = dbg.bin_and_sort(scene.n, proj.depth.data_ptr(), proj.rect.data_ptr(), proj.ntiles.data_ptr(), C.byref(c),
                          C.byref(o), base, nbytes, cap, None, vals.data_ptr(), ranges.data_ptr(), k_out.data_ptr(),
                          None)
    assert st == abi.UT_OK
    assert dbg.ut_debug_check_bin_workspace(base, scene.n, cap, C.byref(c), C.byref(o), None) == abi.UT_OK
    assert _read(dbg) == [0, 0, 0, 0]
    ws.fill_(0)  # the host overwrites everything, guards included
    assert dbg.ut_debug_check_bin_workspace(base, scene.n, cap, C.byref(c), C.byref(o), None) == abi.UT_OK
    rec = _read(dbg)
    assert rec[0] == 5 and rec[1] == 0 and rec[3] == 0, rec  # UT_DBG_CANARY in the first guard, byte 0
    assert _read(dbg) == [0, 0, 0, 0]  # reset
