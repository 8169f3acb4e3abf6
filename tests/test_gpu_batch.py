"""Batches of views (render_batch / render_batch_backward) through the C ABI.

A batch must render every view exactly as the single-view path does (the single-view calls
are the batch of one view), match the FP64 oracle view by view, and propagate the gradients
of all views into their scenes (views sharing a scene add up).
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from gpu_helpers import (TOL, TOL_INJECTED, compare_frame, gpu_decisions, grad_compare, run_gpu,  # noqa: E402
                         sample_pixels, to_np)
from paper_2412_12507_gb300 import abi, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_12507_gb300 import build
    build.build()
    abi.lib()


def _scenes():
    a = synth.scene_shell(6000, 41, radius=3.0, radial_std=0.2, log_s=(-3.5, 0.5), logit_std=1.0, deg=3)
    b = synth.scene_cube(4000, 42, log_s=(-3.0, 0.4), deg=3)
    return [a, b]


def _cams():
    qe, te = synth.rs_end_pose(0.05, 2.0)
    q1, t1 = synth.look_at_pose([0.5, -0.3, -2.5])
    return [
        (1, synth.camera("pinhole", 160, 96, fx=140.0, fy=140.0)),
        (0, synth.camera("fisheye", 200, 150, k=[0.01, -0.02, 0.005, 0.0])),
        (1, synth.camera("fisheye", 176, 99, k=[0.02, 0.01, -0.004, 0.001], q_end=qe, t_end=te, rolling_shutter=1)),
        (0, synth.camera("pinhole", 128, 128, fx=100.0, fy=100.0, q=q1, t=t1)),
        (1, synth.camera("pinhole", 64, 48, fx=60.0, fy=60.0)),
    ]


def _single(scene_np, cam, op):
    scene = render.Scene.from_arrays(scene_np)
    r = render.Renderer(cam, op, capacity=1 << 12)
    f = r.forward(scene)
    torch.cuda.synchronize()
    return f


def test_global_shutter_batch_is_bit_identical_to_single_views():
    """All-global-shutter batch: same kernels, same per-pixel particle sequence -> identical bits."""
    scenes_np = _scenes()
    op = synth.options()
    views = [v for v in _cams() if not v[1]["rolling_shutter"]]
    br = render.BatchRenderer([render.Scene.from_arrays(s) for s in scenes_np], op, capacity=1 << 12)
    frames = br.forward(views)
    torch.cuda.synchronize()
    for (si, cam), f in zip(views, frames):
        g = _single(scenes_np[si], cam, op)
        assert torch.equal(f.rgb, g.rgb) and torch.equal(f.alpha, g.alpha)


def test_mixed_batch_matches_single_views_and_oracle():
    scenes_np = _scenes()
    op = synth.options()
    views = _cams()
    br = render.BatchRenderer([render.Scene.from_arrays(s) for s in scenes_np], op, capacity=1 << 12)
    frames = br.forward(views)
    torch.cuda.synchronize()
    assert br.capacity >= int(br.k_dev.item())
    for (si, cam), f in zip(views, frames):
        g = _single(scenes_np[si], cam, op)
        # views of a batch with a rolling-shutter member take the general ray-origin path
        assert torch.max(torch.abs(f.rgb - g.rgb)).item() < 2e-5
        ref = oracle.render(scenes_np[si], cam, op, proj=oracle.project(scenes_np[si], cam, op, TOL), tol=TOL)
        r = compare_frame(f, ref)
        assert r["n_bad"] == 0, (cam["model"], r)
        assert r["n_flagged"] <= 0.1 * r["n"], r  # small views of dense scenes: near-ties are common
        # decision-injected: the oracle composites with the single-view call's rects and depths
        # (the batch's are the same arithmetic)
        ri = compare_frame(f, oracle.render(scenes_np[si], cam, op, proj=_decisions(scenes_np[si], cam, op),
                                            tol=TOL_INJECTED))
        assert ri["n_unbounded"] == 0 and ri["n_bad"] == 0, (cam["model"], ri)


def _decisions(sc, cam, op):
    """Rects and depth bits of the single-view projection call (the batch's projection runs the
    same kernel arithmetic per view)."""
    g = run_gpu(sc, cam, op)
    return gpu_decisions(g)


@pytest.mark.slow
def test_full_multiview_batch_sampled_pixels():
    """The full 8-view batch (3M particles; 4 pinhole 1920x1080, 2 fisheye 1600x1600, 2 rolling-
    shutter fisheye 2048x1536) rendered as one batch in the benchmark's configuration (16x16
    tiles): seeded pixel samples of every view against the oracle, independently and with the
    view's own decisions injected."""
    case = synth.multiview()
    sc, op = case["scene"], case["options"]
    views = [(0, c) for c in case["cameras"]]
    br = render.BatchRenderer([render.Scene.from_arrays(sc)], op, capacity=1 << 20)
    frames = br.forward(views)
    torch.cuda.synchronize()
    for j, ((_, cam), f) in enumerate(zip(views, frames)):
        W, H = cam["width"], cam["height"]
        px, py = sample_pixels(W, H, 300, 100 + j)
        yy, xx = np.mgrid[H // 2 - 200:H // 2 + 200:20, W // 2 - 200:W // 2 + 200:20]
        px = np.concatenate([px, xx.ravel()]).astype(np.int32)
        py = np.concatenate([py, yy.ravel()]).astype(np.int32)
        ref = oracle.render(sc, cam, op, proj=oracle.project(sc, cam, op, TOL), pixels=(px, py), tol=TOL)
        r = compare_frame(f, ref)
        ri = compare_frame(f, oracle.render(sc, cam, op, proj=_decisions(sc, cam, op), pixels=(px, py),
                                            tol=TOL_INJECTED))
        print(j, cam["model"], cam["rolling_shutter"], r, ri)
        assert ri["n_unbounded"] == 0 and ri["n_bad"] == 0, (j, ri)
        assert r["n_bad"] == 0, (j, r)
        assert r["n_flagged"] <= 0.1 * r["n"], (j, r)


def test_batch_capacity_overflow_is_reported_and_retried():
    scenes_np = _scenes()
    op = synth.options()
    views = _cams()[:2]
    br = render.BatchRenderer([render.Scene.from_arrays(s) for s in scenes_np], op, capacity=16)
    frames = br.forward(views, sync_check=False)
    torch.cuda.synchronize()
    K = int(br.k_dev.item())
    assert K > 16
    assert not any(to_np(f.rgb).any() for f in frames)  # overflowing batch renders nothing
    frames = br.forward(views)  # grows the capacity and retries
    torch.cuda.synchronize()
    assert br.capacity >= K and any(to_np(f.rgb).any() for f in frames)


def test_batch_validation():
    scenes_np = _scenes()
    op = synth.options()
    sc = [render.Scene.from_arrays(s) for s in scenes_np]
    br = render.BatchRenderer(sc, op)
    views = [(0, synth.camera("pinhole", 32, 32, fx=30.0))] * (abi.MAX_BATCH_VIEWS + 1)
    with pytest.raises(abi.UtError):
        br.forward(views)
    with pytest.raises(abi.UtError):
        br.forward([(5, synth.camera("pinhole", 32, 32, fx=30.0))])
    mixed = [sc[0], render.Scene.from_arrays(synth.scene_cube(100, 1, deg=1))]
    with pytest.raises(abi.UtError):
        render.BatchRenderer(mixed, op).forward([(0, synth.camera("pinhole", 32, 32, fx=30.0))])


@pytest.mark.parametrize("k", [0, 8])
def test_batch_backward_sums_views_of_a_scene(k):
    """Three views of one scene plus one of another: each scene's gradient equals the sum of
    its views' single-view gradients and the FP64 oracle's, in tile order and through the
    per-ray k-buffer (k = 8: one record table per scene in the batch's gradient workspace)."""
    scenes_np = _scenes()
    op = synth.options(kbuffer=k)
    views = [_cams()[k] for k in (0, 2, 4, 1)]  # scene 1 three times, scene 0 once
    br = render.BatchRenderer([render.Scene.from_arrays(s) for s in scenes_np], op, capacity=1 << 12)
    frames = br.forward(views, grad=True)
    rng = np.random.default_rng(5)
    d_rgb, d_a, refs = [], [], [dict(), dict()]
    for (si, cam), f in zip(views, frames):
        H, W = cam["height"], cam["width"]
        pr = oracle.project(scenes_np[si], cam, op, TOL)
        rf = oracle.render(scenes_np[si], cam, dict(op, eps_tau=1e-4) if k else op, proj=pr, tol=TOL)
        keep = (rf["flags"] & oracle.F_BACKWARD_TIES) == 0
        w_rgb = rng.standard_normal((H * W, 3)) * keep[:, None]
        w_a = rng.standard_normal(H * W) * keep
        d_rgb.append(torch.as_tensor(w_rgb.T.reshape(3, H, W).astype(np.float32)).cuda())
        d_a.append(torch.as_tensor(w_a.reshape(H, W).astype(np.float32)).cuda())
        g = oracle.backward(scenes_np[si], cam, op, pr, (rf["px"], rf["py"]), w_rgb, w_a, magnitudes=True)
        for k, v in g["mag"].items():
            refs[si]["mag_" + k] = refs[si].get("mag_" + k, 0) + v
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            refs[si][k] = refs[si].get(k, 0) + g[k]
    grads = br.backward(d_rgb, d_a)
    torch.cuda.synchronize()
    for si in (0, 1):
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            grad_compare(to_np(grads[si][k]), refs[si][k], refs[si]["mag_" + k], (si, k))


def test_multiview_autograd_matches_batch_backward():
    scene_np = _scenes()[1]
    op = synth.options()
    cams = [c for s, c in _cams() if s == 1]
    scene = render.Scene.from_arrays(scene_np)
    leaves = [t.clone().requires_grad_(True) for t in (scene.means, scene.log_scales, scene.quats,
                                                        scene.opacity_logits, scene.sh)]
    br = render.BatchRenderer([scene], op, capacity=1 << 12)
    outs = render.render_views(*leaves, scene.sh_degree, cams, br)
    loss = sum((rgb ** 2).sum() + alpha.sum() for rgb, alpha in outs)
    loss.backward()
    torch.cuda.synchronize()
    # same gradient via single-view autograd calls, summed
    tot = [torch.zeros_like(t) for t in leaves]
    for cam in cams:
        ls = [t.detach().clone().requires_grad_(True) for t in leaves]
        rgb, alpha = render.render(*ls, scene.sh_degree, render.Renderer(cam, op, capacity=1 << 12))
        ((rgb ** 2).sum() + alpha.sum()).backward()
        for a, b in zip(tot, ls):
            a += b.grad
    for a, b in zip(leaves, tot):
        e = (torch.linalg.norm(a.grad - b) / torch.linalg.norm(b)).item()
        assert e < 1e-4, e


def test_batch_images_do_not_depend_on_tile_shape():
    """The pixel predicate (pixel centre inside the particle's rect) makes every image of a
    batch bit-identical for every tile shape the autotuner may pick."""
    scenes_np = _scenes()
    scenes = [render.Scene.from_arrays(s) for s in scenes_np]
    views = _cams()
    ref = None
    for tw, th in render.TILE_CANDIDATES:
        br = render.BatchRenderer(scenes, synth.options(tile_w=tw, tile_h=th), capacity=1 << 12)
        frames = br.forward(views)
        torch.cuda.synchronize()
        if ref is None:
            ref = frames
            continue
        for f, g in zip(frames, ref):
            assert torch.equal(f.rgb, g.rgb) and torch.equal(f.alpha, g.alpha), (tw, th)


def test_autotune_tiles_returns_a_candidate_and_timings():
    scenes = [render.Scene.from_arrays(s) for s in _scenes()]
    views = _cams()[:3]
    d_rgb = [torch.ones((3, c["height"], c["width"]), device="cuda") for _, c in views]
    d_a = [torch.ones((c["height"], c["width"]), device="cuda") for _, c in views]
    best, res = render.autotune_tiles(scenes, views, synth.options(), d_rgb, d_a, steps=1, warmup=1)
    assert (best["tile_w"], best["tile_h"]) in render.TILE_CANDIDATES
    assert set(res) == {f"{w}x{h}" for w, h in render.TILE_CANDIDATES}
    assert all(r["ms"] > 0 and r["keys"] > 0 for r in res.values())


def test_captured_step_replays_bit_identically_and_follows_new_inputs():
    """Renderer.capture: the forward (+ backward) step recorded as a CUDA graph gives, on replay,
    the eager step's image bit for bit and its gradients up to the rounding order of the
    backward's atomic accumulation, and a replay after the scene's tensors
    were overwritten in place renders the new values (the graph reads the same buffers)."""
    sc_np = _scenes()[0]
    cam = _cams()[2][1]
    op = synth.options()
    scene = render.Scene.from_arrays(sc_np)
    r = render.Renderer(cam, op, capacity=1 << 12)
    r.forward(scene)
    torch.cuda.synchronize()
    H, W = cam["height"], cam["width"]
    g = torch.Generator().manual_seed(7)
    d_rgb = torch.randn((3, H, W), generator=g).cuda()
    d_alpha = torch.randn((H, W), generator=g).cuda()
    eager_f = {k: getattr(r.forward(scene), k).clone() for k in ("rgb", "alpha", "t_final", "n_used")}
    eager_g = {k: v.clone() for k, v in r.backward(scene, d_rgb, d_alpha).items()}
    torch.cuda.synchronize()
    graph, frame, grads = r.capture(scene, d_rgb, d_alpha)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for k, v in eager_f.items():
        assert torch.equal(getattr(frame, k), v), k
    for k, v in eager_g.items():  # the backward accumulates with float atomics: order-dependent rounding
        torch.testing.assert_close(grads[k], v, rtol=1e-4, atol=1e-5 * float(v.abs().max()), msg=k)
    # new opacities in place: the replay must follow them
    with torch.no_grad():
        scene.opacity_logits.sub_(1.0)
    graph.replay()
    torch.cuda.synchronize()
    moved = frame.alpha.clone()
    ref = render.Renderer(cam, op, capacity=1 << 12).forward(scene)
    torch.cuda.synchronize()
    assert torch.equal(moved, ref.alpha)
    assert not torch.equal(moved, eager_f["alpha"])


def test_frame_pipeline_matches_plain_renders_of_each_frame():
    """render.FramePipeline: frames whose parameters arrive from pinned host memory, rendered
    with overlapped copies, give exactly the images of plain renders of the same parameters."""
    sc_np = dict(_scenes()[1])
    cam = _cams()[1][1]
    op = synth.options()
    fields = ("means", "log_scales", "quats", "opacity_logits", "sh")
    frames = []
    for f in range(4):
        d = {k: np.array(sc_np[k], np.float32, copy=True) for k in fields}
        d["opacity_logits"] = d["opacity_logits"] - 0.3 * f
        d["means"] = d["means"] + np.float32(0.01 * f)
        frames.append({k: torch.as_tensor(v).pin_memory() for k, v in d.items()})
    got = []
    for depth in (2, 3):
        pipe = render.FramePipeline(cam, op, frames[0], sc_np["sh_degree"], depth=depth)
        outs = [pipe.submit(fr) for fr in frames[:depth]]  # `depth` frames in flight at once
        for out in outs:
            pipe.done(out).synchronize()
            got.append(out.clone())
        for fr in frames[depth:]:
            out = pipe.submit(fr)
            pipe.done(out).synchronize()
            got.append(out.clone())
    frames = frames + frames
    for fr, img in zip(frames, got):
        scene = render.Scene.from_arrays(dict({k: v.numpy() for k, v in fr.items()}, sh_degree=sc_np["sh_degree"]))
        f = render.Renderer(cam, op, capacity=1 << 12).forward(scene)
        torch.cuda.synchronize()
        assert torch.equal(img[:3], f.rgb.cpu())
        assert torch.equal(img[3], f.alpha.cpu())
