"""The serving loop (ut_server_*): requests of mixed scenes, camera models and resolutions,
submitted together so that they batch and overlap, must give the same images as the same
request served alone, and as a plain single-view render, within the stated tolerance."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from gpu_helpers import TOL, compare_frame, sample_pixels  # noqa: E402
from paper_2412_12507_gb300 import abi, render, synth  # noqa: E402

pytestmark = pytest.mark.gpu

RGB_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_12507_gb300 import build
    build.build()
    abi.lib()


def _scenes():
    return [synth.scene_cube(20_000, 51, log_s=(-3.2, 0.5), deg=3, lo=(-1, -1, -1), hi=(1, 1, 1)),
            synth.scene_cube(60_000, 52, log_s=(-3.5, 0.5), deg=3, lo=(-1, -1, -1), hi=(1, 1, 1))]


def _requests(seed=9, n=14):
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n):
        model = ["pinhole", "fisheye", "rs"][int(rng.integers(3))]
        W, H = [(160, 120), (320, 180), (480, 270), (64, 48)][int(rng.integers(4))]
        specs.append((int(rng.integers(2)), model if model != "rs" else "fisheye", W, H, int(model == "rs")))
    cams = synth.orbit_cameras(seed, [(m, W, H, rs) for _, m, W, H, rs in specs])
    return [(s[0], c) for s, c in zip(specs, cams)]


def _plain(scene, cam, op):
    r = render.Renderer(cam, op, capacity=1 << 12)
    f = r.forward(scene)
    torch.cuda.synchronize()
    return f.rgb.clone(), f.alpha.clone()


@pytest.mark.parametrize("use_graphs", [True, False])
def test_requests_in_the_mix_equal_alone_and_plain(use_graphs):
    op = synth.options()
    scenes = [render.Scene.from_arrays(s) for s in _scenes()]
    reqs = _requests()
    srv = render.Server(scenes, op, arena_bytes=1 << 30, max_batch_views=4, max_in_flight=3,
                        use_graphs=use_graphs)
    try:
        ids = [srv.submit(s, c) for s, c in reqs]          # all at once: they batch and overlap
        mixed = []
        for rid in ids:
            out = srv.wait(rid, 60_000)
            assert out is not None
            rgb, alpha, lat = out
            mixed.append((rgb.clone(), alpha.clone()))
            assert lat >= 0
            srv.release(rid)
        st = srv.stats()
        assert st["completed"] == len(reqs)
        assert st["batches"] < len(reqs) + st["retries"]   # several requests per launch
        if use_graphs:
            assert st["graph_launches"] == st["batches"]
        for (s, c), (rgb_m, a_m) in zip(reqs, mixed):
            rid = srv.submit(s, c)                            # the same request alone
            rgb_a, a_a, _ = srv.wait(rid, 60_000)
            assert torch.max(torch.abs(rgb_m - rgb_a)).item() <= RGB_TOL
            assert torch.max(torch.abs(a_m - a_a)).item() <= RGB_TOL
            srv.release(rid)
            rgb_p, a_p = _plain(scenes[s], c, op)             # one plain render call
            assert torch.max(torch.abs(rgb_m - rgb_p)).item() <= RGB_TOL
            assert torch.max(torch.abs(a_m - a_p)).item() <= RGB_TOL
    finally:
        srv.close()


def test_served_images_match_the_oracle_on_sampled_pixels():
    """Every request of the mix, served batched and overlapped, against the FP64 oracle on
    seeded pixel samples (the oracle's own projection; near-tie pixels against its bounds)."""
    from types import SimpleNamespace
    op = synth.options()
    scenes_np = _scenes()
    scenes = [render.Scene.from_arrays(s) for s in scenes_np]
    reqs = _requests(seed=13, n=10)
    srv = render.Server(scenes, op, arena_bytes=1 << 30, max_batch_views=4, max_in_flight=3)
    try:
        ids = [srv.submit(si, c) for si, c in reqs]
        for j, (rid, (si, cam)) in enumerate(zip(ids, reqs)):
            out = srv.wait(rid, 60_000)
            assert out is not None
            rgb, alpha, _ = out
            f = SimpleNamespace(rgb=rgb.clone(), alpha=alpha.clone(), t_final=None)
            srv.release(rid)
            W, H = cam["width"], cam["height"]
            px, py = sample_pixels(W, H, 400, 700 + j)
            sc = scenes_np[si]
            ref = oracle.render(sc, cam, op, proj=oracle.project(sc, cam, op, TOL), pixels=(px, py), tol=TOL)
            r = compare_frame(f, ref)
            assert r["n_bad"] == 0, (j, cam["model"], r)
            assert r["n_flagged"] <= 0.1 * r["n"], (j, r)
    finally:
        srv.close()


def test_first_request_of_a_class_may_overflow_and_is_retried():
    op = synth.options()
    scenes = [render.Scene.from_arrays(s) for s in _scenes()]
    # a small image of the larger scene: far more than 2 keys per pixel (the initial estimate)
    cam = synth.orbit_cameras(3, [("pinhole", 64, 48, 0)])[0]
    srv = render.Server(scenes, op, arena_bytes=1 << 30, key_headroom=1.0)
    try:
        rid = srv.submit(1, cam)
        rgb, alpha, _ = srv.wait(rid, 60_000)
        rgb_p, a_p = _plain(scenes[1], cam, op)
        assert torch.max(torch.abs(rgb - rgb_p)).item() <= RGB_TOL
        srv.release(rid)
        assert srv.stats()["retries"] >= 1  # the initial estimate of 2 keys / pixel is too low here
    finally:
        srv.close()


def test_overestimated_request_runs_with_the_capacity_the_arena_holds():
    """A request whose estimated key count needs more scratch than the arena holds still runs
    (with the largest capacity that fits; an overflow would re-run it with the observed count)."""
    op = synth.options()
    scenes = [render.Scene.from_arrays(synth.scene_cube(50, 53, log_s=(-3.0, 0.3), deg=3, lo=(-1, -1, -1),
                                                        hi=(1, 1, 1)))]
    cam = synth.orbit_cameras(5, [("pinhole", 256, 256, 0)])[0]
    # first estimate: 2 keys / pixel x 65536 pixels x headroom 8 = ~1M keys, ~25 MB of scratch
    srv = render.Server(scenes, op, arena_bytes=8 << 20, key_headroom=8.0)
    try:
        rid = srv.submit(0, cam)
        rgb, alpha, _ = srv.wait(rid, 60_000)
        rgb_p, a_p = _plain(scenes[0], cam, op)
        assert torch.max(torch.abs(rgb - rgb_p)).item() <= RGB_TOL
        assert torch.max(torch.abs(alpha - a_p)).item() <= RGB_TOL
        srv.release(rid)
    finally:
        srv.close()


def test_request_larger_than_the_arena_is_rejected():
    op = synth.options()
    scenes = [render.Scene.from_arrays(_scenes()[0])]
    srv = render.Server(scenes, op, arena_bytes=1 << 20)
    try:
        with pytest.raises(abi.UtError) as e:
            srv.submit(0, synth.camera("pinhole", 3840, 2160, fx=2000.0))
        assert e.value.status == abi.UT_ERR_CAPACITY
    finally:
        srv.close()


def test_wait_times_out_without_blocking_forever():
    op = synth.options()
    scenes = [render.Scene.from_arrays(_scenes()[1])]
    srv = render.Server(scenes, op, arena_bytes=1 << 30)
    try:
        cam = synth.orbit_cameras(4, [("fisheye", 480, 270, 1)])[0]
        rid = srv.submit(0, cam)
        t0 = time.time()
        srv.wait(rid, 0)  # poll: returns at once whether or not it is done
        assert time.time() - t0 < 1.0
        assert srv.wait(rid, 60_000) is not None
        srv.release(rid)
    finally:
        srv.close()


def test_burst_larger_than_the_arena_completes_in_order():
    """A burst of requests whose outputs together exceed the arena: admission stays at most one
    batch ahead of the GPU, so waiting outputs never crowd out the workspaces, and a client that
    waits for and releases the requests in arrival order sees every one of them complete."""
    op = synth.options()
    scenes = [render.Scene.from_arrays(_scenes()[1])]
    cams = synth.orbit_cameras(12, [("fisheye", 480, 270, j % 2) for j in range(60)])
    out_mb = 16 * 480 * 270 / 2**20
    arena = 80 << 20
    assert len(cams) * out_mb > arena / 2**20  # the outputs alone would not fit together
    srv = render.Server(scenes, op, arena_bytes=arena, max_batch_views=4, max_in_flight=3)
    try:
        ids = [srv.submit(0, c) for c in cams]
        for rid in ids:
            out = srv.wait(rid, 60_000)
            assert out is not None, "a request of the burst did not complete"
            srv.release(rid)
        assert srv.stats()["completed"] == len(ids)
    finally:
        srv.close()
