"""Parity of the optional modes with the FP64 oracle, through the C ABI:

- projection = EWA: the first-order projection of 3DGS (eq. ewa_splatting), the A/B
  baseline of the UT — 2D moments, depth, culling and rects, then full renders;
- colour_mode = per particle: SH evaluated once per particle at its view direction —
  renders and gradients (including the mean's gradient through the direction).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from gpu_helpers import TOL, compare_frame, gpu_decisions, grad_compare, run_gpu, sample_pixels, to_np  # noqa: E402,E501
from paper_2412_12507_gb300 import abi, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_12507_gb300 import build
    build.build()
    abi.lib()


def _cases():
    return {
        "fisheye_shell": synth.fisheye_shell(n=20_000, width=640, height=360),
        "rs_fisheye": synth.rs_fisheye(n=20_000, width=480, height=270),
        "pinhole_deg2_ragged": dict(scene=synth.scene_cube(3000, 9, deg=2, log_s=(-3.2, 0.4)),
                                    camera=synth.camera("pinhole", 150, 97, fx=120.0, fy=110.0, cx=70.3, cy=50.1),
                                    options=synth.options()),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_ewa_projection_matches_oracle(name):
    case = CASES[name]
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], projection=1)
    g = run_gpu(sc, cam, op)
    ref = oracle.project(sc, cam, op, TOL)
    p = g["proj"]
    rect = to_np(p.rect).astype(np.int64)
    nt = to_np(p.ntiles)
    valid_g, valid_o = nt > 0, ref["ntiles"] > 0
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
    cov_err = np.max(np.abs(c2 - ref["cov2d"][both]).max(1) / (scale + 1e-6))
    assert cov_err < 2e-4, cov_err
    dep = to_np(p.depth)[both]
    assert np.max(np.abs(dep - ref["depth"][both]) / ref["depth"][both]) < 2e-6
    diff = rect[both] != ref["rect"][both]
    eb = e[both][:, [0, 2, 1, 3]]
    assert not np.any(diff & ~(np.abs(eb - np.round(eb)) < TOL["eps_px"]))
    # the EWA moments are not the UT ones (a fisheye bends the footprint)
    if name != "pinhole_deg2_ragged":
        ut = oracle.project(sc, cam, case["options"], TOL)
        assert np.abs(ut["cov2d"][both] - ref["cov2d"][both]).max() > 1e-3 * np.abs(ref["cov2d"][both]).max()


@pytest.mark.parametrize("name,mode", [("rs_fisheye", dict(projection=1)),
                                       ("rs_fisheye", dict(colour_mode=1)),
                                       ("fisheye_shell", dict(colour_mode=1)),
                                       ("pinhole_deg2_ragged", dict(colour_mode=1, projection=1))])
def test_mode_render_matches_oracle(name, mode):
    case = CASES[name]
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], **mode)
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    pix = None if W * H <= 70_000 else sample_pixels(W, H, 20_000, 7)
    ref = oracle.render(sc, cam, op, proj=oracle.project(sc, cam, op, TOL), pixels=pix, tol=TOL)
    r = compare_frame(g["frame"], ref)
    print(name, mode, r)
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.03 * r["n"], r


def test_per_particle_colour_degree_zero_is_the_per_pixel_image():
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    a = run_gpu(sc, cam, op)["frame"]
    b = run_gpu(sc, cam, dict(op, colour_mode=1))["frame"]
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.alpha, b.alpha)


GRAD_CASES = {
    "rs_fisheye_crop": lambda: synth.rs_fisheye(n=2000, width=320, height=180),
    "pinhole_deg2": lambda: dict(scene=synth.scene_cube(1500, 13, deg=2, log_s=(-2.8, 0.4)),
                                 camera=synth.camera("pinhole", 96, 80, fx=90.0, fy=90.0),
                                 options=synth.options()),
}


@pytest.mark.parametrize("name", list(GRAD_CASES))
def test_per_particle_colour_backward_matches_oracle(name):
    """Gradients of all five parameter tensors in the per-particle colour mode, including the
    means' gradient through the view direction, against the FP64 oracle's."""
    case = GRAD_CASES[name]()
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], colour_mode=1)
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    ref_f = oracle.render(sc, cam, op, proj=proj_ref, tol=TOL)
    flagged = (ref_f["flags"] & oracle.F_BACKWARD_TIES) != 0
    rng = np.random.default_rng(321)
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
    # the two colour modes give different gradients (the mode is not silently ignored)
    op0 = dict(op, colour_mode=0)
    ref0 = oracle.backward(sc, cam, op0, oracle.project(sc, cam, op0, TOL), (ref_f["px"], ref_f["py"]), w_rgb, w_a)
    assert np.linalg.norm(ref0["sh"] - ref["sh"]) > 1e-3 * np.linalg.norm(ref["sh"])


# ------------------------------------------------------------------ radial pinhole, degree-n kernels

def _radial(rs=0):
    qe, te = synth.rs_end_pose(0.05, 2.0)
    return dict(scene=synth.scene_cube(6000, 19, deg=3, log_s=(-3.2, 0.4)),
                camera=synth.camera("pinhole_radial", 320, 240, fx=200.0, fy=200.0, k=[-0.12, 0.03, -0.002, 0.0],
                                    q_end=qe, t_end=te, rolling_shutter=rs),
                options=synth.options())


@pytest.mark.parametrize("rs,mode", [(0, {}), (1, {}), (0, dict(projection=1)), (0, dict(kernel_degree=4)),
                                     (1, dict(kernel_degree=3))])
def test_radial_and_kernel_degree_render_matches_oracle(rs, mode):
    case = _radial(rs)
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], **mode)
    g = run_gpu(sc, cam, op)
    ref_p = oracle.project(sc, cam, op, TOL)
    assert (to_np(g["proj"].ntiles) > 0).sum() > 0.5 * len(ref_p["ntiles"])
    ref = oracle.render(sc, cam, op, proj=ref_p, tol=TOL)
    r = compare_frame(g["frame"], ref)
    print("radial rs", rs, mode, r)
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.05 * r["n"], r


@pytest.mark.parametrize("kdeg,cam_model", [(4, "pinhole"), (3, "pinhole_radial"), (8, "pinhole")])
def test_kernel_degree_backward_matches_oracle(kdeg, cam_model):
    sc = synth.scene_cube(1500, 23, deg=1, log_s=(-2.8, 0.4))
    cam = synth.camera(cam_model, 96, 80, fx=90.0, fy=90.0,
                       k=[-0.1, 0.02, 0.0, 0.0] if cam_model == "pinhole_radial" else [0, 0, 0, 0])
    op = synth.options(kernel_degree=kdeg)
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    ref_f = oracle.render(sc, cam, op, proj=proj_ref, tol=TOL)
    flagged = (ref_f["flags"] & oracle.F_BACKWARD_TIES) != 0
    rng = np.random.default_rng(77)
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
        print(kdeg, cam_model, k, f"rel err {e:.2e}")


# ------------------------------------------------------------------ "Ours (sorted)": per-ray k-buffer

@pytest.mark.parametrize("name,k", [("rs_fisheye", 16), ("fisheye_shell", 16), ("pinhole_deg2_ragged", 4),
                                    ("pinhole_deg2_ragged", 1)])
def test_kbuffer_render_matches_oracle(name, k):
    case = CASES[name]
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], kbuffer=k)
    g = run_gpu(sc, cam, op)
    W, H = cam["width"], cam["height"]
    pix = None if W * H <= 70_000 else sample_pixels(W, H, 20_000, 7)
    ref = oracle.render(sc, cam, op, proj=oracle.project(sc, cam, op, TOL), pixels=pix, tol=TOL)
    # every pixel but a culling near-tie, flagged ones against the oracle's k-buffer bound (what
    # any decision after the first flagged one can change)
    r = compare_frame(g["frame"], ref)
    print(name, "k", k, r)
    assert r["n_bad"] == 0, r
    assert r["n_flagged"] <= 0.1 * r["n"], r
    # the k-buffer changes the image (the tau order differs from the tile order somewhere)
    base = run_gpu(sc, cam, case["options"])["frame"]
    assert torch.max(torch.abs(base.rgb - g["frame"].rgb)).item() > 1e-4


@pytest.mark.parametrize("name", list(GRAD_CASES))
@pytest.mark.parametrize("k", [4, 16])
def test_kbuffer_backward_matches_oracle(name, k):
    """The "Ours (sorted)" backward: gradients of all five parameter tensors over each pixel's
    k-buffer blending order against the FP64 oracle's (pixels whose selection, stop or culling is
    within the near-tie tolerances carry no weight), and different from the tile-order ones."""
    case = GRAD_CASES[name]()
    sc, cam = case["scene"], case["camera"]
    op = dict(case["options"], kbuffer=k)
    W, H = cam["width"], cam["height"]
    proj_ref = oracle.project(sc, cam, op, TOL)
    ref_f = oracle.render(sc, cam, dict(op, eps_tau=1e-4), proj=proj_ref, tol=TOL)
    flagged = (ref_f["flags"] & oracle.F_BACKWARD_TIES) != 0
    assert flagged.mean() < 0.2
    rng = np.random.default_rng(432)
    w_rgb = rng.standard_normal((H * W, 3)) * ~flagged[:, None]
    w_a = rng.standard_normal(H * W) * ~flagged
    ref = oracle.backward(sc, cam, op, proj_ref, (ref_f["px"], ref_f["py"]), w_rgb, w_a, magnitudes=True)
    g = run_gpu(sc, cam, op)
    d_rgb = torch.as_tensor(w_rgb.T.reshape(3, H, W).astype(np.float32)).cuda()
    d_a = torch.as_tensor(w_a.reshape(H, W).astype(np.float32)).cuda()
    grads = render.composite_backward(g["scene"], cam, op, g["proj"], g["binning"], g["frame"], d_rgb, d_a)
    torch.cuda.synchronize()
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        e = grad_compare(to_np(grads[key]), ref[key], ref["mag"][key], key)
        print(name, "k", k, key, f"rel err {e:.2e}")
    # the blending order matters: the tile-order gradients are different
    op0 = dict(op, kbuffer=0)
    ref0 = oracle.backward(sc, cam, op0, proj_ref, (ref_f["px"], ref_f["py"]), w_rgb, w_a)
    assert np.linalg.norm(ref0["means"] - ref["means"]) > 1e-3 * np.linalg.norm(ref["means"])


def _tied_pairs_scene(n_pairs, seed):
    """Particles 2i and 2i+1 share mean, scales and rotation (so their tau_max is bit-identical at
    every pixel and so is their depth) but have different opacities and colours: the order in
    which a tied pair is blended changes the image."""
    a = synth.scene_cube(n_pairs, seed, deg=1, log_s=(-2.6, 0.3))
    b = synth.scene_cube(n_pairs, seed + 1, deg=1, log_s=(-2.6, 0.3))
    sc = {}
    for key in ("means", "log_scales", "quats"):
        sc[key] = np.repeat(a[key], 2, axis=0)
    for key in ("opacity_logits", "sh"):
        sc[key] = np.stack([a[key], b[key]], axis=1).reshape((2 * n_pairs,) + a[key].shape[1:])
    sc["opacity_logits"] = sc["opacity_logits"] + 1.0
    sc["sh_degree"] = 1
    return sc


@pytest.mark.parametrize("k", [1, 4])
def test_kbuffer_exact_tau_ties_break_by_arrival(k):
    """Equal tau_max: the earlier arrival (the lower index of an equal-depth pair) blends first, in
    the kernels as in the oracle.  Every pixel is compared, including those the oracle flags as tau
    ties; the projection's decisions are the GPU's own (rect and depth fed to the oracle), so only
    alpha_min / alpha_max / stop-threshold ties are left out."""
    sc = _tied_pairs_scene(150, 61)
    cam = synth.camera("pinhole", 96, 72, fx=80.0, fy=80.0)
    op = dict(synth.options(), kbuffer=k)
    W, H = cam["width"], cam["height"]
    g = run_gpu(sc, cam, op)
    proj = dict(rect=to_np(g["proj"].rect).astype(np.int32), depth32=to_np(g["proj"].depth))
    ref = oracle.render(sc, cam, op, proj=proj, tol=dict(TOL, depth_ulps=-1))
    fl = ref["flags"]
    keep = (fl & (oracle.F_ALPHA_MIN | oracle.F_ALPHA_MAX | oracle.F_TSTOP)) == 0
    keep_b = keep & ((fl & oracle.F_CLAMP) == 0)
    ties = (fl & oracle.F_DEPTH_TIE) != 0
    assert ties.sum() > 50, ties.sum()
    got = to_np(g["frame"].rgb).reshape(3, -1).T
    err = np.maximum(np.abs(got - ref["rgb"]).max(axis=1), np.abs(to_np(g["frame"].alpha).ravel() - ref["alpha"]))
    assert err[keep].max() < 1e-4, (err[keep].max(), int((err[keep] >= 1e-4).sum()))
    # the order of a tied pair is visible: blending the later arrival first gives another image
    swapped = {key: (v.reshape((-1, 2) + v.shape[1:])[:, ::-1].reshape(v.shape) if key != "sh_degree" else v)
               for key, v in sc.items()}
    ref_sw = oracle.render(swapped, cam, op, proj=proj, tol=dict(TOL, depth_ulps=-1))
    assert np.abs(ref_sw["rgb"] - ref["rgb"])[ties & keep].max() > 1e-3
    # and the backward follows the same order
    rng = np.random.default_rng(5)
    w_rgb = rng.standard_normal((H * W, 3)) * keep_b[:, None]
    w_a = rng.standard_normal(H * W) * keep_b
    gref = oracle.backward(sc, cam, op, proj, (ref["px"], ref["py"]), w_rgb, w_a, magnitudes=True)
    d_rgb = torch.as_tensor(w_rgb.T.reshape(3, H, W).astype(np.float32)).cuda()
    d_a = torch.as_tensor(w_a.reshape(H, W).astype(np.float32)).cuda()
    grads = render.composite_backward(g["scene"], cam, op, g["proj"], g["binning"], g["frame"], d_rgb, d_a)
    torch.cuda.synchronize()
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        grad_compare(to_np(grads[key]), gref[key], gref["mag"][key], key)


def test_kbuffer_rejects_per_particle_colour():
    case = GRAD_CASES["pinhole_deg2"]()
    sc, cam = case["scene"], case["camera"]
    with pytest.raises(abi.UtError):
        run_gpu(sc, cam, dict(case["options"], kbuffer=16, colour_mode=1))
