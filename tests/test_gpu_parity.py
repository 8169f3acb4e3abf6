"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on identical seeded inputs.

Integer outputs (sort keys, per-tile lists, ranges) must be bit-exact; RGB and alpha within
1e-4 absolute; gradients within 1e-3 relative.  Where FP32 and FP64 can legitimately take
a different discrete decision (the oracle flags those near-ties), the oracle also returns a
bound on what the decision can change, and the pixel is held to 1e-4 beyond that bound.  Two
modes: independent (the oracle projects and decides on its own) and decision-injected (the
oracle composites with the GPU's rects and depth bits, so only alpha / stop thresholds remain
as near-ties).
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from gpu_helpers import (RGB_TOL, TOL, TOL_INJECTED, compare_frame, gpu_decisions, grad_compare,  # noqa: E402
                         run_gpu, sample_pixels, to_np)
from paper_2412_12507_gb300 import abi, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_12507_gb300 import build
    build.build()
    abi.lib()


def small_cases():
    return {
        "pinhole64": synth.small_pinhole(),
        "fisheye_shell": synth.fisheye_shell(n=20_000, width=640, height=360),
        "rs_fisheye": synth.rs_fisheye(n=20_000, width=480, height=270),
        "rs_fisheye_deg1": synth.rs_fisheye(n=5_000, width=200, height=120, deg=1),
        "pinhole_deg2_ragged": dict(scene=synth.scene_cube(3000, 9, deg=2, log_s=(-3.2, 0.4)),
                                    camera=synth.camera("pinhole", 150, 97, fx=120.0, fy=110.0, cx=70.3, cy=50.1),
                                    options=synth.options()),
    }


CASES = small_cases()


# ------------------------------------------------------------------ projection

@pytest.mark.parametrize("name", list(CASES))
def test_projection_matches_oracle(name):
    case = CASES[name]
    sc, cam, op = case["scene"], case["camera"], case["options"]
    g = run_gpu(sc, cam, op)
    ref = oracle.project(sc, cam, op, TOL)
    p = g["proj"]
    rect = to_np(p.rect).astype(np.int64)
    nt = to_np(p.ntiles)
    valid_g = nt > 0
    valid_o = ref["ntiles"] > 0
    # culling decisions agree except at oracle-flagged near-ties (or rect edges at an integer)
    e = ref["edges"]
    edge_tie = np.any(np.abs(e - np.round(e)) < TOL["eps_px"], axis=1) & np.isfinite(e).all(axis=1)
    tie = (ref["tie"] != 0) | edge_tie
    mism = valid_g != valid_o
    assert not np.any(mism & ~tie), np.nonzero(mism & ~tie)[0][:10]
    both = valid_g & valid_o
    assert both.sum() > 0.2 * len(valid_o)
    m2 = to_np(p.mean2d)[both]
    assert np.max(np.abs(m2 - ref["mean2d"][both])) < 5e-3
    c2 = to_np(p.cov2d)[both]
    scale = ref["cov2d"][both][:, [0, 2]].sum(1)
    assert np.max(np.abs(c2 - ref["cov2d"][both]).max(1) / (scale + 1e-6)) < 2e-4
    dep = to_np(p.depth)[both]
    assert np.max(np.abs(dep - ref["depth"][both]) / ref["depth"][both]) < 2e-6
    print(name, "mean2d err", np.max(np.abs(m2 - ref["mean2d"][both])), "cov rel err",
          np.max(np.abs(c2 - ref["cov2d"][both]).max(1) / (scale + 1e-6)),
          "depth ulps", np.max(np.abs(dep.view(np.int32).astype(np.int64) -
                                      ref["depth32"][both].view(np.int32).astype(np.int64))),
          "cull mismatches", int(mism.sum()))
    # rects: identical except edges the oracle places within eps of an integer
    diff = rect[both] != ref["rect"][both]
    eb = e[both][:, [0, 2, 1, 3]]  # x0, y0, x1, y1 order of rect
    near = np.abs(eb - np.round(eb)) < TOL["eps_px"]
    assert not np.any(diff & ~near)
    assert np.array_equal(nt[valid_g & ~valid_o] > 0, np.ones((valid_g & ~valid_o).sum(), bool))
    assert np.all(rect[~valid_g] == [0, 0, -1, -1])


# ------------------------------------------------------------------ binning / sorting (bit-exact)

BIN_CASES = [
    (64, 48, 16, 16, 200, 30, 20),
    (70, 33, 16, 16, 500, 40, 20),
    (37, 29, 8, 8, 300, 12, 12),
    (1000, 600, 16, 16, 20_000, 80, 80),        # > one radix tile of keys, 2 tile passes
    (4096, 4096, 8, 8, 30_000, 60, 60),         # 262144 tiles; 512 tile rows, the most the row scatter takes
    (3840, 2160, 32, 8, 10_000, 200, 40),
    (64, 64, 16, 16, 1, 10, 10),
    (256, 2048, 16, 4, 3_000, 40, 400),         # tall rects (up to 100 tile rows): scatter groups past the window
    (512, 512, 32, 8, 20_000, 20, 6),           # one or two tile rows per entry: windows of many groups
    (128, 1200, 64, 1, 3_000, 60, 40),          # 1200 tile rows: rows emitted and radix-sorted (2 passes)
    (17_000, 64, 1, 64, 2_000, 40, 40),         # 17000 tile columns: rows emitted and radix-sorted
]


@pytest.mark.parametrize("W,H,tw,th,n,mw,mh", BIN_CASES)
def test_bin_and_sort_bit_exact(W, H, tw, th, n, mw, mh):
    rect, depth = synth.random_rects(W + n, n, W, H, max_w=mw, max_h=mh)
    cam = synth.camera("pinhole", W, H, fx=float(W))
    op = synth.options(tile_w=tw, tile_h=th)
    sc = synth.scene_cube(n, 1)
    g = run_gpu(sc, cam, op, want_keys=True, rect=rect, depth=depth)
    k_ref, v_ref, r_ref = oracle.bin_keys(depth, rect, W, H, tw, th)
    K = g["K"]
    assert K == len(k_ref) == g["K_sum"]
    b = g["binning"]
    assert np.array_equal(to_np(b.keys)[:K].view(np.uint64), k_ref)
    assert np.array_equal(to_np(b.vals)[:K].view(np.uint32), v_ref)
    assert np.array_equal(to_np(b.ranges).view(np.uint32), r_ref)


def test_bin_empty_and_all_culled():
    cam = synth.camera("pinhole", 64, 64, fx=64.0)
    op = synth.options()
    for n in (0, 17):
        rect = np.tile(np.array([[0, 0, -1, -1]], np.int16), (n, 1))
        g = run_gpu(synth.scene_cube(n, 2), cam, op, rect=rect, depth=np.ones(n, np.float32), capacity=64)
        assert g["K"] == 0
        assert not to_np(g["binning"].ranges).any()
        f = g["frame"]
        assert not to_np(f.rgb).any() and not to_np(f.alpha).any()
        assert np.all(to_np(f.t_final) == 1.0)


@pytest.mark.parametrize("k", [0, 4])
def test_backward_of_empty_and_all_culled_scenes_is_zero(k):
    """The backward (tile order and k-buffer) of a scene with no particle, and of one whose
    every particle is culled, succeeds and writes zero gradients."""
    cam = synth.camera("pinhole", 64, 64, fx=64.0)
    op = synth.options(kbuffer=k)
    for n in (0, 17):
        rect = np.tile(np.array([[0, 0, -1, -1]], np.int16), (n, 1))
        g = run_gpu(synth.scene_cube(n, 2, deg=3), cam, op, rect=rect, depth=np.ones(n, np.float32), capacity=64)
        d_rgb = torch.ones((3, 64, 64), device="cuda")
        d_a = torch.ones((64, 64), device="cuda")
        grads = render.composite_backward(g["scene"], cam, op, g["proj"], g["binning"], g["frame"], d_rgb, d_a)
        torch.cuda.synchronize()
        for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            assert grads[key].shape[0] == n
            assert not to_np(grads[key]).any(), (k, n, key)


def test_bin_capacity_overflow_reports_k_and_writes_nothing():
    W, H = 200, 120
    rect, depth = synth.random_rects(5, 400, W, H, max_w=50, max_h=50)
    cam = synth.camera("pinhole", W, H, fx=200.0)
    op = synth.options()
    k_ref, _, _ = oracle.bin_keys(depth, rect, W, H)
    cap = len(k_ref) - 1
    sc = synth.scene_cube(400, 3)
    scene = render.Scene.from_arrays(sc)
    proj = render.project(scene, cam, op)
    proj.rect = torch.as_tensor(rect.astype(np.int16)).cuda()
    proj.depth = torch.as_tensor(depth).cuda()
    r = rect.astype(np.int64)
    nt = np.where(r[:, 0] <= r[:, 2], (r[:, 2] // 16 - r[:, 0] // 16 + 1) * (r[:, 3] // 16 - r[:, 1] // 16 + 1), 0)
    proj.ntiles = torch.as_tensor(nt.astype(np.int32)).cuda()
    b = render.Binning(torch.full((cap,), -7, dtype=torch.int32, device="cuda"),
                       torch.full((render.tile_count(cam, op), 2), -7, dtype=torch.int32, device="cuda"),
                       torch.zeros(1, dtype=torch.int64, device="cuda"), None, cap)
    b = render.bin_and_sort(proj, cam, op, cap, out=b)
    torch.cuda.synchronize()
    assert b.count() == len(k_ref)
    assert not to_np(b.ranges).any()
    assert np.all(to_np(b.vals) == -7)


# ------------------------------------------------------------------ compositing on its own

def test_composite_with_shared_synthetic_rects():
    """Both sides get the same synthetic rects and depths (no projection involved), so only
    the compositing arithmetic is compared."""
    W, H = 96, 72
    n = 1500
    sc = synth.scene_cube(n, 21, deg=3, log_s=(-2.8, 0.4))
    rect, depth = synth.random_rects(22, n, W, H, max_w=40, max_h=40, cull_frac=0.05)
    cam = synth.camera("pinhole", W, H, fx=80.0, fy=80.0)
    op = synth.options()
    g = run_gpu(sc, cam, op, rect=rect, depth=depth)
    ref = oracle.render(sc, cam, op, proj=dict(rect=rect.astype(np.int32), depth32=depth), tol=TOL)
    r = compare_frame(g["frame"], ref)
    assert r["n_bad"] == 0, r
    assert r["max_err"] < RGB_TOL
    assert r["n_flagged"] <= 0.02 * r["n"], r


# ------------------------------------------------------------------ full renders

@pytest.mark.parametrize("name", list(CASES))
def test_render_matches_oracle(name):
    case = CASES[name]
    sc, cam, op = case["scene"], case["camera"], case["options"]
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    pix = None if W * H <= 70_000 else sample_pixels(W, H, 20_000, 7)
    ref = oracle.render(sc, cam, op, proj=oracle.project(sc, cam, op, TOL), pixels=pix, tol=TOL)
    r = compare_frame(g["frame"], ref)
    print(name, r)
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.03 * r["n"], r
    # invalid (not imaged) fisheye pixels are exactly zero
    inval = (ref["flags"] & oracle.F_INVALID_PIXEL) != 0
    if inval.any():
        rgb = to_np(g["frame"].rgb)[:, ref["py"][inval], ref["px"][inval]]
        assert not rgb.any()


@pytest.mark.parametrize("name", list(CASES))
def test_render_decision_injected(name):
    """The oracle composites with the GPU's own rects and depth bits: the per-pixel lists are then
    identical, and every pixel must be within 1e-4 (plus the exact slack of stop-threshold ties
    and the bound of alpha_min / alpha_max ties, the only decisions left to each side)."""
    case = CASES[name]
    sc, cam, op = case["scene"], case["camera"], case["options"]
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    pix = None if W * H <= 70_000 else sample_pixels(W, H, 20_000, 7)
    ref = oracle.render(sc, cam, op, proj=gpu_decisions(g), pixels=pix, tol=TOL_INJECTED)
    r = compare_frame(g["frame"], ref)
    print(name, r)
    assert r["n_unbounded"] == 0 and r["n_bad"] == 0, r
    assert r["max_err"] < RGB_TOL


def test_render_independent_of_tile_shape():
    """The pixel predicate (centre in rect) does not depend on the tiling, so every tile
    shape gives bit-identical images."""
    case = CASES["pinhole_deg2_ragged"]
    sc, cam = case["scene"], case["camera"]
    imgs = []
    for tw, th in ((16, 16), (8, 8), (32, 8), (16, 32), (64, 2)):
        g = run_gpu(sc, cam, synth.options(tile_w=tw, tile_h=th))
        imgs.append((to_np(g["frame"].rgb), to_np(g["frame"].alpha)))
    for rgb, a in imgs[1:]:
        assert np.array_equal(rgb, imgs[0][0]) and np.array_equal(a, imgs[0][1])


def test_degenerate_particles_are_culled():
    sc = synth.scene_cube(64, 4)
    sc["quats"][3] = 0.0                       # zero quaternion
    sc["means"][5] = [0.0, 0.0, -3.0]          # behind the camera
    sc["opacity_logits"][7] = -20.0            # sigma < alpha_min
    sc["log_scales"][9] = np.inf               # non-finite scale
    cam = synth.camera("pinhole", 64, 64, fx=64.0)
    op = synth.options()
    g = run_gpu(sc, cam, op)
    nt = to_np(g["proj"].ntiles)
    ref = oracle.project(sc, cam, op)
    for i in (3, 5, 7, 9):
        assert nt[i] == 0 and ref["ntiles"][i] == 0
    r = compare_frame(g["frame"], oracle.render(sc, cam, op, tol=TOL))
    assert r["n_bad"] == 0


# ------------------------------------------------------------------ full-size workload, sampled

@pytest.mark.slow
def test_full_size_rs_fisheye_sampled():
    """The 1M-particle rolling-shutter fisheye 1920x1080 workload in the launch configuration
    the benchmark times: sampled pixels against the oracle, and properties of the sorted
    lists that hold at any size."""
    case = synth.rs_fisheye()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    # pixels sampled where the scene is, plus a few anywhere
    px, py = sample_pixels(W, H, 400, 11)
    yy, xx = np.mgrid[H // 2 - 300:H // 2 + 300:7, W // 2 - 300:W // 2 + 300:7]
    px = np.concatenate([px, xx.ravel()[::4]]).astype(np.int32)
    py = np.concatenate([py, yy.ravel()[::4]]).astype(np.int32)
    ref = oracle.render(sc, cam, op, proj=proj_ref, pixels=(px, py), tol=TOL)
    r = compare_frame(g["frame"], ref)
    print("full size", r, "K", g["K"])
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.1 * r["n"], r
    # decision-injected: the same pixels composited by the oracle from the GPU's rects and depths
    ri = compare_frame(g["frame"], oracle.render(sc, cam, op, proj=gpu_decisions(g), pixels=(px, py),
                                                 tol=TOL_INJECTED))
    print("full size, decision-injected", ri)
    assert ri["n_unbounded"] == 0 and ri["n_bad"] == 0, ri
    # key count equals the oracle's up to rect near-ties
    K_ref = int(proj_ref["ntiles"].astype(np.int64).sum())
    assert abs(g["K"] - K_ref) <= 1e-3 * K_ref
    # properties of the sorted lists: every entry's tile lies in its particle's rect, each tile's
    # run is sorted by (depth bits, index), and every particle appears ntiles times
    b = g["binning"]
    K = g["K"]
    vals = to_np(b.vals)[:K].astype(np.int64)
    ranges = to_np(b.ranges).astype(np.int64)
    rect = to_np(g["proj"].rect).astype(np.int64)
    dbits = to_np(g["proj"].depth).view(np.uint32).astype(np.int64)
    tx = (W + 15) // 16
    tile_of = np.repeat(np.arange(len(ranges)), ranges[:, 1] - ranges[:, 0])
    assert len(tile_of) == K
    order = np.concatenate([np.arange(s, e) for s, e in ranges if e > s])
    v = vals[order]
    t = tile_of
    r_ = rect[v]
    assert np.all((t % tx >= r_[:, 0] // 16) & (t % tx <= r_[:, 2] // 16) &
                  (t // tx >= r_[:, 1] // 16) & (t // tx <= r_[:, 3] // 16))
    key = dbits[v] * (1 << 24) + v
    same = t[1:] == t[:-1]
    assert np.all(key[1:][same] > key[:-1][same])
    assert np.array_equal(np.bincount(v, minlength=len(rect)), to_np(g["proj"].ntiles).astype(np.int64))


@pytest.mark.slow
def test_full_size_fisheye_shell_sampled():
    """The forward-only fisheye-shell workload at full size (100k Gaussians on a radius-5 shell,
    1280x720 180-degree polynomial fisheye, SH degree 3) in the benchmark's configuration: seeded
    pixel samples against the oracle in both modes, and the key count."""
    case = synth.fisheye_shell()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    px, py = sample_pixels(W, H, 3000, 13)
    ref = oracle.render(sc, cam, op, proj=proj_ref, pixels=(px, py), tol=TOL)
    r = compare_frame(g["frame"], ref)
    print("fisheye shell", r, "K", g["K"])
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.05 * r["n"], r
    ri = compare_frame(g["frame"], oracle.render(sc, cam, op, proj=gpu_decisions(g), pixels=(px, py),
                                                 tol=TOL_INJECTED))
    assert ri["n_unbounded"] == 0 and ri["n_bad"] == 0, ri
    K_ref = int(proj_ref["ntiles"].astype(np.int64).sum())
    assert abs(g["K"] - K_ref) <= 1e-3 * K_ref


# ------------------------------------------------------------------ gradients

GRAD_CASES = {
    "rs_fisheye_crop": lambda: synth.rs_fisheye(n=2000, width=320, height=180),
    # the headline camera (1920x1080 rolling-shutter fisheye) with 2000 Gaussians of its scene
    "rs_fisheye_1080p_2k": lambda: synth.rs_fisheye(n=2000),
    "pinhole_deg2": lambda: dict(scene=synth.scene_cube(1500, 13, deg=2, log_s=(-2.8, 0.4)),
                                 camera=synth.camera("pinhole", 96, 80, fx=90.0, fy=90.0),
                                 options=synth.options()),
    "fisheye_deg0": lambda: dict(scene=synth.scene_cube(1500, 14, deg=0, log_s=(-2.8, 0.4)),
                                 camera=synth.camera("fisheye", 160, 120), options=synth.options()),
}


@pytest.mark.parametrize("name", list(GRAD_CASES))
def test_backward_matches_oracle(name):
    """A linear loss sum(w_rgb * rgb) + sum(w_a * alpha) with fixed seeded weights (zero at
    near-tie pixels, where the decisions may differ) gives both sides the identical dL/drgb."""
    case = GRAD_CASES[name]()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    ref_f = oracle.render(sc, cam, op, proj=proj_ref, tol=TOL)
    flagged = (ref_f["flags"] & oracle.F_BACKWARD_TIES) != 0
    rng = np.random.default_rng(123)
    w_rgb = rng.standard_normal((H * W, 3)) * ~flagged[:, None]
    w_a = rng.standard_normal(H * W) * ~flagged
    ref = oracle.backward(sc, cam, op, proj_ref, (ref_f["px"], ref_f["py"]), w_rgb, w_a, magnitudes=True)
    g = run_gpu(sc, cam, op)
    d_rgb = torch.as_tensor(w_rgb.T.reshape(3, H, W).astype(np.float32)).cuda()
    d_a = torch.as_tensor(w_a.reshape(H, W).astype(np.float32)).cuda()
    grads = render.composite_backward(g["scene"], cam, op, g["proj"], g["binning"], g["frame"], d_rgb, d_a)
    torch.cuda.synchronize()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        e = grad_compare(to_np(grads[k]), ref[k], ref["mag"][k], k)
        print(name, k, f"rel err {e:.2e}")


def test_autograd_l2_training_step():
    """The torch.autograd.Function path: L2 loss against a seeded target, gradients of every
    parameter against the oracle's (each side uses its own rendered image for dL/drgb)."""
    case = synth.rs_fisheye(n=2000, width=256, height=144)
    sc, cam, op = case["scene"], case["camera"], case["options"]
    W, H = cam["width"], cam["height"]
    target = synth.target_image(2, W, H)
    proj_ref = oracle.project(sc, cam, op, TOL)
    ref_f = oracle.render(sc, cam, op, proj=proj_ref, tol=TOL)
    flagged = (ref_f["flags"] & oracle.F_BACKWARD_TIES) != 0
    mask = (~flagged).reshape(H, W)
    tgt = target.reshape(3, -1).T
    g_ref = 2.0 * (ref_f["rgb"] - tgt) * (~flagged)[:, None] / (3 * H * W)
    ref = oracle.backward(sc, cam, op, proj_ref, (ref_f["px"], ref_f["py"]), g_ref, np.zeros(H * W),
                          magnitudes=True)
    scene = render.Scene.from_arrays(sc)
    leaves = [t.clone().requires_grad_(True) for t in (scene.means, scene.log_scales, scene.quats,
                                                        scene.opacity_logits, scene.sh)]
    r = render.Renderer(cam, op, capacity=1 << 14)
    rgb, alpha = render.render(*leaves, scene.sh_degree, r)
    m = torch.as_tensor(mask).cuda()
    loss = (((rgb - torch.as_tensor(target).cuda()) ** 2) * m).sum() / (3 * H * W)
    loss.backward()
    torch.cuda.synchronize()
    for leaf, k in zip(leaves, ("means", "log_scales", "quats", "opacity_logits", "sh")):
        grad_compare(to_np(leaf.grad), ref[k], ref["mag"][k], k)
