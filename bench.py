"""Benchmark of the 3DGUT hot path on GB300 (one JSON line on stdout).

Workload (default): 1,000,000 Gaussians (box in front of the camera, log-scales N(-3, 0.5),
SH degree 3), a 1920x1080 polynomial fisheye with a rolling shutter (0.05 units / 2 degrees
over the frame), 16x16 tiles.  A step is one pass of the whole path: UT projection,
binning + radix sort + ranges, compositing forward, and (fwd+bwd phase) the backward for a
fixed seeded upstream gradient dL/drgb, dL/dalpha resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

value = forward Mpix/s over all ranks (each rank renders its own replica of the workload:
weak scaling, no collective on the data path).  Extra keys: fwd_ms, fwd_bwd_ms_per_view,
per-call times, roofline of the dominant kernel, the oracle's CPU baseline, clocks, e2e.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rs_fisheye_1m_1080p")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle's CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="leave out the forward-only lines of the fisheye shell (100k Gaussians, 1280x720) and "
                         "the small pinhole case (1k Gaussians, 64x64)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="measured serving requests (0: skip)")
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests / s")
    ap.add_argument("--serve-arena-gb", type=float, default=64.0)
    ap.add_argument("--serve-saturated-requests", type=int, default=600,
                    help="measured requests of the saturated serving run (0: skip)")
    ap.add_argument("--serve-saturated-rate", type=float, default=2000.0,
                    help="arrival rate of the saturated serving run, requests / s (above capacity)")
    ap.add_argument("--multiview-steps", type=int, default=5,
                    help="timed steps of the 8-view 3M-particle fwd+bwd batch (0: skip)")
    return ap.parse_args()


def workload(name):
    from paper_2412_12507_gb300 import synth
    if name == "rs_fisheye_1m_1080p":
        return synth.rs_fisheye(seed=2, n=1_000_000, width=1920, height=1080, deg=3)
    if name == "rs_fisheye_300k_1080p":
        return synth.rs_fisheye(seed=2, n=300_000, width=1920, height=1080, deg=3)
    if name == "fisheye_shell_100k_720p":
        return synth.fisheye_shell(seed=1, n=100_000, width=1280, height=720)
    if name == "pinhole_1k_64":
        return synth.small_pinhole()
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    """(world size, rank, local rank) of this process; 1, 0, 0 without a launcher."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device) -> float:
    """The maximum of a per-rank number over all ranks (a job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mpix_s(pixels_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: every rank renders its own replica, so the job's pixels are
    world x pixels_per_rank in the slowest rank's time."""
    return world * pixels_per_rank / (ms / 1e3) / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def measured_traffic(kernel, workload_name):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu record
    `profiles/dram_traffic.json`, or None when there is none for this workload or the
    kernel's sources changed since the capture (their SHA-256 is stored with the bytes)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)[kernel]
        h = hashlib.sha256()
        for name in rec["sources"]:
            with open(os.path.join(ROOT, name), "rb") as f:
                h.update(f.read())
    except Exception:
        return None
    if h.hexdigest() != rec["sources_sha256"] or rec["workload"] != workload_name:
        return None
    return float(rec["bytes_per_launch"])


def measure_alu_peaks(L, dev, stream, sms):
    """FP32 FMA and special-function (ex2) throughput of this GPU, from the library's probe
    kernels (ut_peak_probe: 8 independent chains per thread, 8 blocks of 256 per SM, a few ms
    per launch); the median of 5 launches timed with events on the launching stream."""
    import torch

    from paper_2412_12507_gb300 import abi
    blocks, threads = sms * 8, 256
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    res = {}
    for kind, name, iters, flop_per_op in ((abi.UT_PROBE_FMA, "fp32", 40000, 2.0), (abi.UT_PROBE_EX2, "ex2", 5000, 1.0)):
        def launch():
            abi.check("ut_peak_probe", L.ut_peak_probe(kind, blocks, threads, iters, out.data_ptr(), stream.cuda_stream))
        launch()
        torch.cuda.synchronize()
        times = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        res[name] = (blocks * threads * iters * 8 * flop_per_op / (ms / 1e3), ms)
    return {"fp32_tflops": res["fp32"][0] / 1e12, "ex2_gops": res["ex2"][0] / 1e9,
            "fp32_ms": res["fp32"][1], "ex2_ms": res["ex2"][1],
            "how": f"ut_peak_probe: {blocks} x {threads} threads x 8 chains of fma.rn.f32 / ex2.approx.ftz.f32, "
                   "median of 5 launches"}


def queue_ahead(stream, us=300):
    """Holds `stream` with a device-side spin of a fixed cycle count (about `us` microseconds at
    2 GHz), so that the calls enqueued after it are queued before the GPU reaches them: a pair of
    events around one call then times its kernels, not the host's marshalling and launch."""
    import torch
    with torch.cuda.stream(stream):
        torch.cuda._sleep(int(us * 2000))


def projection_work(cam, rs_iters=3):
    """FP32 operations and transcendental calls (sqrt, atan2, sin / cos, exp, log, division:
    one each) of the UT projection of one particle, counted from the arithmetic the method
    needs (term by term in the design notes): 7 sigma points, each projected 1 + rs_iters
    times under a rolling shutter, plus activation, moments, depth, extent and rectangle."""
    rs = bool(cam.get("rolling_shutter", 0))
    if cam["model"] == "fisheye":
        cam_f, cam_s = 23, 4  # |x|, rho, theta = atan2, theta_d polynomial, scale and (u, v)
    elif cam["model"] == "pinhole_radial":
        cam_f, cam_s = 17, 2
    else:
        cam_f, cam_s = 6, 1
    # per projection: the pose at time t (rotation about the fixed axis 31 + sin / cos,
    # translation 9) and the time update 4 under a rolling shutter, else the translation 9
    per_f, per_s, per_pt = (cam_f + 44, cam_s + 2, 1 + rs_iters) if rs else (cam_f + 9, cam_s, 1)
    # per particle: activation 49, R0 mu 15, sigma-point columns 57 and points 18, moments 78,
    # depth (pose 9 / 40, norm 5), extent 5, rectangle 16, tile count 8
    base_f, base_s = 254 + (31 if rs else 0), 12 + (2 if rs else 0)
    return 7 * per_pt * per_f + base_f, 7 * per_pt * per_s + base_s


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0:  # first sample before the timed region
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nme, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nme)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference arm: the oracle on host cores

def oracle_frame_time(case, budget_s, seed=0):
    """The FP64 oracle as it stands, on a bounded sample of the workload: the projection of
    all particles, then brute-force compositing of a seeded pixel sample sized to the budget.
    Returns (seconds per full frame extrapolated from the sample, description, threads)."""
    import oracle
    sc, cam, op = case["scene"], case["camera"], case["options"]
    W, H = cam["width"], cam["height"]
    t0 = time.perf_counter()
    proj = oracle.project(sc, cam, op)
    t_proj = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    npx = 64
    t_pix = None
    while True:
        q = rng.choice(W * H, size=npx, replace=False)
        t0 = time.perf_counter()
        oracle.render(sc, cam, op, proj=proj, pixels=(q % W, q // W))
        dt = time.perf_counter() - t0
        t_pix = dt / npx
        spent = t_proj + dt
        if dt > 0.25 * budget_s or npx >= W * H or spent > budget_s:
            break
        npx = int(min(W * H, max(2 * npx, npx * 0.5 * budget_s / max(dt, 1e-3))))
    frame = t_proj + t_pix * W * H
    desc = (f"projection of all {len(sc['means'])} particles ({t_proj:.2f} s) + brute-force compositing of "
            f"{npx} seeded pixels ({dt:.2f} s), extrapolated to {W}x{H}")
    return frame, desc, oracle.num_threads()


def run_reference(args):
    _, rank, _ = dist_env()
    if rank != 0:  # under torchrun only rank 0 times the oracle; the others exit without work
        return
    case = workload(args.workload)
    W, H = case["camera"]["width"], case["camera"]["height"]
    frames, walls = [], []
    desc, thr = "", 1
    per = max(2.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        f, desc, thr = oracle_frame_time(case, per)
        walls.append(time.perf_counter() - t0)
        frames.append(f)
    frames, walls = frames[args.warmup:], walls[args.warmup:]
    frame_ms = 1e3 * statistics.median(frames)
    v = W * H / (frame_ms / 1e3) / 1e6
    # a step is one bounded sample (the projection of every particle and a seeded pixel sample):
    # ms_per_step is its measured wall time, so steps x ms_per_step is what ran; value is the
    # per-frame rate extrapolated from the sample
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case["name"]},
            "value_basis": "extrapolated: full-frame time estimated from each step's sample",
            "frame_ms_extrapolated": frame_ms,
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": thr, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "Mpix/s fwd & fwd+bwd ms/view, 1M Gaussians fisheye 1080p; serve p50/p99 ms"


# ---------------------------------------------------------------- serving workload

def serving_requests(n, rate, seed=4):
    """Poisson arrivals at `rate` req/s; each request picks a scene U{4}, a camera model
    U{pinhole, fisheye, rolling-shutter fisheye} and a resolution U{640x480, 1280x720,
    1920x1080, 3840x2160}, posed on a radius-4 orbit around the scenes."""
    from paper_2412_12507_gb300 import synth
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    res = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    specs, scenes = [], []
    for _ in range(n):
        m = int(rng.integers(3))
        W, H = res[int(rng.integers(4))]
        specs.append(("pinhole" if m == 0 else "fisheye", W, H, int(m == 2)))
        scenes.append(int(rng.integers(4)))
    cams = synth.orbit_cameras(seed, specs)
    return [(float(t[j]), scenes[j], cams[j]) for j in range(n)]


def serving_scenes(dev, sizes=(200_000, 1_000_000, 3_000_000, 6_000_000)):
    """Four resident scenes generated like the 1M workload (box of side 2 at the origin,
    log-scales N(-3, 0.5), SH degree 3)."""
    from paper_2412_12507_gb300 import render, synth
    return [render.Scene.from_arrays(synth.scene_cube(n, 10 + j, log_s=(-3.0, 0.5), deg=3, lo=(-1, -1, -1),
                                                      hi=(1, 1, 1)), dev) for j, n in enumerate(sizes)]


def run_serving(scenes, opts, reqs, n_warm, arena_bytes, max_batch_views=8, max_in_flight=3, use_graphs=True):
    """Replays the arrival trace against the library's server; returns latencies (ms) and the
    wall time of the measured part."""
    import torch

    from paper_2412_12507_gb300 import render
    srv = render.Server(scenes, opts, arena_bytes=arena_bytes, max_batch_views=max_batch_views,
                        max_in_flight=max_in_flight, use_graphs=use_graphs)
    ids = [None] * len(reqs)
    lag = [0.0] * len(reqs)
    lat = [0.0] * len(reqs)
    t_done = [0.0] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for j, (ta, s, cam) in enumerate(reqs):
            while True:
                now = time.perf_counter() - t0
                if now >= ta:
                    break
                time.sleep(min(0.0005, ta - now))
            ids[j] = srv.submit(s, cam)
            lag[j] = (time.perf_counter() - t0) - ta

    th = threading.Thread(target=submitter)
    th.start()
    for j in range(len(reqs)):
        while ids[j] is None:
            time.sleep(0.0001)
        out = srv.wait(ids[j], 120_000)
        if out is None:
            ta, s_, cam = reqs[j]
            raise SystemExit(f"serving: request {j} (scene {s_}, {cam['model']} {cam['width']}x{cam['height']}, "
                             f"rolling shutter {cam['rolling_shutter']}) did not complete in 120 s; server {srv.stats()}")
        lat[j] = out[2] + 1e3 * lag[j]
        t_done[j] = time.perf_counter() - t0
        srv.release(ids[j])
    th.join()
    stats = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    meas = slice(n_warm, len(reqs))
    wall = max(t_done[meas]) - reqs[n_warm][0]
    return np.array(lat[meas]), wall, stats


def latency_breakdown(lat, reqs, sizes):
    """p50 / p99 latency of the measured requests grouped by resolution and by scene."""
    out = {"by_resolution": {}, "by_scene": {}}
    res = [f"{c['width']}x{c['height']}" for _, _, c in reqs]
    sc = [f"{sizes[s] // 1000}k" for _, s, _ in reqs]
    for key, labels in (("by_resolution", res), ("by_scene", sc)):
        for lab in sorted(set(labels), key=lambda x: (len(x), x)):
            v = np.array([l for l, g in zip(lat, labels) if g == lab])
            out[key][lab] = {"n": int(v.size), "p50_ms": float(np.percentile(v, 50)),
                             "p99_ms": float(np.percentile(v, 99))}
    return out


def run_plain(scenes, opts, reqs, n_warm):
    """The same trace through one plain single-view render call per request, in arrival order."""
    import torch

    from paper_2412_12507_gb300 import render
    ws, caps = render.Workspace(), {}
    lat, t_done = [], []
    t0 = time.perf_counter()
    for j, (ta, s, cam) in enumerate(reqs):
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        key = (s, cam["model"], cam["width"], cam["height"])
        r = render.Renderer(cam, opts, capacity=caps.get(key, 1 << 20), ws=ws)
        r.forward(scenes[s])
        torch.cuda.synchronize()
        caps[key] = max(caps.get(key, 0), r.capacity)
        t = time.perf_counter() - t0
        lat.append(1e3 * (t - ta))
        t_done.append(t)
    meas = slice(n_warm, len(reqs))
    return np.array(lat[meas]), max(t_done[meas]) - reqs[n_warm][0]


# ---------------------------------------------------------------- our arm

def run_multiview(dev, steps, warmup, timed):
    """Eight views of one 3M-particle scene rendered and differentiated as one batch
    (render_batch + render_batch_backward): 4 pinhole 1920x1080, 2 fisheye 1600x1600,
    2 rolling-shutter fisheye 2048x1536 on a radius-4 orbit.  The tile shape is picked by the
    library's autotuner over 8x8, 16x16, 32x8, 16x32; the chosen shape is then timed over
    `steps` batch steps (forward alone, and forward + backward)."""
    import torch
    from paper_2412_12507_gb300 import render, synth
    case = synth.multiview()
    scene = render.Scene.from_arrays(case["scene"], dev)
    cams = case["cameras"]
    views = [(0, c) for c in cams]
    pix = sum(c["width"] * c["height"] for c in cams)
    rng = np.random.default_rng(78)
    d_rgb = [torch.as_tensor(rng.standard_normal((3, c["height"], c["width"])).astype(np.float32) / pix).to(dev)
             for c in cams]
    d_a = [torch.as_tensor(rng.standard_normal((c["height"], c["width"])).astype(np.float32) / pix).to(dev)
           for c in cams]
    best, tuned = render.autotune_tiles([scene], views, case["options"], d_rgb, d_a)
    br = render.BatchRenderer([scene], best, capacity=1 << 20)
    frames = br.forward(views, grad=True)
    K = int(br.k_dev.item())

    def fwd():
        br.forward(views, frames=frames, grad=True, sync_check=False)

    def fwd_bwd():
        fwd()
        br.backward(d_rgb, d_a)

    f_ms = timed(fwd, steps, warmup)
    fb_ms = timed(fwd_bwd, steps, warmup)
    if int(br.k_dev.item()) != K:
        raise SystemExit("multiview key count changed during the timed region")
    nv = len(views)
    # where the batch's time goes: every view rendered on its own through the single-view calls
    # (same tile shape), each ABI call timed with events on the stream
    stream = torch.cuda.current_stream()
    per_view = []
    for (si, cam), g_rgb, g_a in zip(views, d_rgb, d_a):
        r = render.Renderer(cam, best, capacity=1 << 20)
        r.forward(scene)
        torch.cuda.synchronize()
        calls = {"ut_project": [], "bin_and_sort": [], "composite_forward": [], "composite_backward": []}
        for _ in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            queue_ahead(stream)
            ev[0].record(stream)
            render.project(scene, cam, best, r.proj)
            ev[1].record(stream)
            render.bin_and_sort(r.proj, cam, best, r.capacity, ws=r.ws, out=r.binning)
            ev[2].record(stream)
            render.composite_forward(scene, cam, best, r.proj, r.binning, r.frame, ws=r.fws)
            ev[3].record(stream)
            r.backward(scene, g_rgb, g_a)
            ev[4].record(stream)
            torch.cuda.synchronize()
            for j, k in enumerate(calls):
                calls[k].append(ev[j].elapsed_time(ev[j + 1]))
        cm = {k: statistics.median(v) for k, v in calls.items()}
        stats = torch.zeros(2, dtype=torch.int64, device=dev)
        render.composite_forward(scene, cam, best, r.proj, r.binning, r.frame, stats=stats, ws=r.fws)
        torch.cuda.synchronize()
        per_view.append({"model": cam["model"] + ("+rs" if cam.get("rolling_shutter") else ""),
                         "width": cam["width"], "height": cam["height"], "keys": r.binning.count(),
                         "evaluations": int(stats[0]), "blended": int(stats[1]), "ms": cm})
        del r
    single_f = sum(v["ms"]["ut_project"] + v["ms"]["bin_and_sort"] + v["ms"]["composite_forward"] for v in per_view)
    single_b = sum(v["ms"]["composite_backward"] for v in per_view)
    out = {"workload": case["name"], "particles": scene.n, "views": nv, "pixels": pix, "keys": K,
           "tile": f"{best['tile_w']}x{best['tile_h']}", "autotune_ms_per_batch": tuned,
           "fwd_ms_per_view": f_ms / nv, "fwd_bwd_ms_per_view": fb_ms / nv,
           "fwd_mpix_s": pix / (f_ms / 1e3) / 1e6, "fwd_bwd_mpix_s": pix / (fb_ms / 1e3) / 1e6, "steps": steps,
           "single_view_calls": per_view, "single_view_sum_fwd_ms": single_f,
           "single_view_sum_bwd_ms": single_b}
    del br, frames, scene
    torch.cuda.empty_cache()
    return out


def run_variants(scene, cam, op, d_rgb, d_alpha, timed, steps, warmup):
    """A/B lines on the bench workload: the UT projection against the first-order EWA one
    (the paper's "Preprocess" comparison with 3DGS; per call, and the whole forward with each),
    the per-ray k-buffer of "Ours (sorted)" (the paper's "Render" comparison), the
    per-particle SH colour mode (forward and forward + backward) against the per-pixel one, and
    the same scene with SH degree 0 (forward and forward + backward)."""
    import torch
    from paper_2412_12507_gb300 import render
    P = cam["width"] * cam["height"]
    out = {}
    stream = torch.cuda.current_stream()

    def per_call(fn, n=max(5, steps)):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(stream)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for name, mode in (("ut", {}), ("ewa", {"projection": 1})):
        o = dict(op, **mode)
        pr = render.project(scene, cam, o)
        proj_ms = per_call(lambda: render.project(scene, cam, o, pr))
        r = render.Renderer(cam, o, capacity=1 << 20)
        r.forward(scene)
        torch.cuda.synchronize()
        K = r.binning.count()
        fwd_ms = timed(lambda: r.forward(scene, sync_check=False), steps, warmup)
        out[name] = {"project_ms": proj_ms, "fwd_ms": fwd_ms, "keys": K, "fwd_mpix_s": P / (fwd_ms / 1e3) / 1e6}
        del r
    out["ewa_over_ut_project"] = out["ewa"]["project_ms"] / out["ut"]["project_ms"]
    # "Ours (sorted)": the per-ray k-buffer (k = 16), forward and backward
    o = dict(op, kbuffer=16)
    r = render.Renderer(cam, o, capacity=1 << 20)
    r.forward(scene)
    torch.cuda.synchronize()
    k_ms = timed(lambda: r.forward(scene, sync_check=False), steps, warmup)
    calls = {}
    for k, fn in (("composite_forward", lambda: render.composite_forward(scene, cam, o, r.proj, r.binning, r.frame,
                                                                         ws=r.fws)),
                  ("composite_backward", lambda: r.backward(scene, d_rgb, d_alpha))):
        calls[k] = per_call(fn)
    out["kbuffer16"] = {"fwd_ms": k_ms, "composite_forward_ms": calls["composite_forward"],
                        "composite_backward_ms": calls["composite_backward"],
                        "fwd_mpix_s": P / (k_ms / 1e3) / 1e6}
    del r
    o = dict(op, colour_mode=1)
    r = render.Renderer(cam, o, capacity=1 << 20)
    r.forward(scene)
    torch.cuda.synchronize()
    f_ms = timed(lambda: r.forward(scene, sync_check=False), steps, warmup)

    def fb():
        r.forward(scene, sync_check=False)
        r.backward(scene, d_rgb, d_alpha)

    fb_ms = timed(fb, steps, warmup)
    out["per_particle_colour"] = {"fwd_ms": f_ms, "fwd_bwd_ms": fb_ms, "fwd_mpix_s": P / (f_ms / 1e3) / 1e6,
                                  "fwd_bwd_mpix_s": P / (fb_ms / 1e3) / 1e6}
    del r
    # the same scene with SH degree 0 (the DC colour alone), forward and forward + backward
    s0 = render.Scene(scene.means, scene.log_scales, scene.quats, scene.opacity_logits,
                      scene.sh[:, :1, :].contiguous(), 0)
    r = render.Renderer(cam, op, capacity=1 << 20)
    r.forward(s0)
    torch.cuda.synchronize()
    f_ms = timed(lambda: r.forward(s0, sync_check=False), steps, warmup)

    def fb0():
        r.forward(s0, sync_check=False)
        r.backward(s0, d_rgb, d_alpha)

    fb_ms = timed(fb0, steps, warmup)
    out["sh_degree_0"] = {"fwd_ms": f_ms, "fwd_bwd_ms": fb_ms, "fwd_mpix_s": P / (f_ms / 1e3) / 1e6,
                          "fwd_bwd_mpix_s": P / (fb_ms / 1e3) / 1e6}
    del r, s0
    torch.cuda.empty_cache()
    return out


def call_fractions(call_ms, n, K, M_cols, n_eval, n_blend, P, cam, op, hbm, alu):
    """Roofline fraction of each ABI call from its measured duration and its algorithmic work:
    bytes for the projection (HBM side) and the binning, FP32 operations for the compositing,
    plus the projection's arithmetic and the compositing's special-function side against the
    FP32 and ex2 peaks measured in the same run."""
    fp32_peak, ex2_peak = alu["fp32_tflops"], alu["ex2_gops"]
    # per-evaluation / per-blend FP32 operation counts of the compositing arithmetic, term by
    # term in the design notes; a rolling-shutter view adds the per-pixel origin's canonical
    # image M o - M mu to every evaluation (9 FMA + 3 subtractions)
    F_EVAL = 40 + (21 if cam.get("rolling_shutter", 0) else 0)
    F_BLEND_FWD, F_BLEND_BWD, F_PIX = 110, 275, 120
    work = {
        "ut_project": ("hbm", 80.0 * n / 1e9),
        # binning: the K values written once, 16 B of projection output read per particle, the
        # column list (8 B per column entry) written and read once
        "bin_and_sort": ("hbm", (4.0 * K + 16.0 * n + 16.0 * M_cols) / 1e9),
        "composite_forward": ("alu", (F_EVAL * n_eval + F_BLEND_FWD * n_blend + F_PIX * P) / 1e12),
        "composite_backward": ("alu", (F_EVAL * n_eval + F_BLEND_BWD * n_blend + F_PIX * P) / 1e12),
    }
    kernels = {}
    for k, (bound, amount) in work.items():
        if k not in call_ms:
            continue
        ach = amount / (call_ms[k] / 1e3)
        peak = hbm if bound == "hbm" else fp32_peak
        kernels[k] = {"ms": call_ms[k], "bound": bound, "achieved": ach, "peak": peak,
                      "unit": "GB/s" if bound == "hbm" else "TFLOP/s", "frac": ach / peak}
    # the binning also against the algorithmic model of a 64-bit key sort: every key (8 B key + 4 B value)
    # emitted, sorted (read + written) and scanned for ranges (44 B / key), 8 B per particle
    kernels["bin_and_sort"]["model_44B_per_key"] = {
        "achieved_gbs": (44.0 * K + 8.0 * n) / 1e9 / (call_ms["bin_and_sort"] / 1e3),
        "frac": (44.0 * K + 8.0 * n) / 1e9 / (call_ms["bin_and_sort"] / 1e3) / hbm}
    # the special-function side of the compositing (one ex2 and one reciprocal per evaluation)
    # and the arithmetic side of the projection
    for k in ("composite_forward", "composite_backward"):
        if k in kernels:
            g = 2.0 * n_eval / (call_ms[k] / 1e3) / 1e9
            kernels[k]["sfu"] = {"ops": 2 * n_eval, "achieved_gops": g, "peak_gops": ex2_peak, "frac": g / ex2_peak}
    pf, ps = projection_work(cam, op["rs_iters"])
    sec = call_ms["ut_project"] / 1e3
    kernels["ut_project"]["fp32"] = {"flop_per_particle": pf, "achieved_tflops": pf * n / sec / 1e12,
                                     "peak_tflops": fp32_peak, "frac": pf * n / sec / 1e12 / fp32_peak}
    kernels["ut_project"]["transcendental"] = {"per_particle": ps, "achieved_gops": ps * n / sec / 1e9,
                                               "ex2_peak_gops": ex2_peak, "frac": ps * n / sec / 1e9 / ex2_peak}
    return kernels


def run_forward_workload(name, dev, steps, warmup, timed, alu, hbm):
    """A forward-only workload (the fisheye shell: 100k Gaussians on a radius-5 shell around a
    1280x720 180-degree polynomial fisheye, SH degree 3; or the small pinhole case: 1k Gaussians,
    64x64): the captured forward step timed over `steps`, each ABI call timed with events, and the
    calls' roofline fractions."""
    import torch

    from paper_2412_12507_gb300 import render
    case = workload(name)
    sc_np, cam, op = case["scene"], case["camera"], case["options"]
    W, H = cam["width"], cam["height"]
    scene = render.Scene.from_arrays(sc_np, dev)
    r = render.Renderer(cam, op, capacity=1 << 20)
    r.forward(scene)
    torch.cuda.synchronize()
    K = r.binning.count()
    r.capacity = int(K * 1.05) + 1024
    r.binning = None
    r.forward(scene)
    g, _, _ = r.capture(scene)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # the scene fits in the 129 MB L2: every timed step starts from a flushed L2 (a 256 MB buffer
    # written between steps, outside the events around each step)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(warmup):
        g.replay()
    step_ms = []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    fwd_ms = statistics.median(step_ms)
    calls = {"ut_project": [], "bin_and_sort": [], "composite_forward": []}
    for _ in range(max(5, steps)):
        flush.fill_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        queue_ahead(stream)
        ev[0].record(stream)
        render.project(scene, cam, op, r.proj)
        ev[1].record(stream)
        render.bin_and_sort(r.proj, cam, op, r.capacity, ws=r.ws, out=r.binning)
        ev[2].record(stream)
        render.composite_forward(scene, cam, op, r.proj, r.binning, r.frame, ws=r.fws)
        ev[3].record(stream)
        torch.cuda.synchronize()
        for j, k in enumerate(calls):
            calls[k].append(ev[j].elapsed_time(ev[j + 1]))
    call_ms = {k: statistics.median(v) for k, v in calls.items()}
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    render.composite_forward(scene, cam, op, r.proj, r.binning, r.frame, stats=stats, ws=r.fws)
    torch.cuda.synchronize()
    n_eval, n_blend = (int(v) for v in stats.cpu())
    rc = r.proj.rect.long()
    M_cols = int(torch.where(r.proj.ntiles > 0, rc[:, 2] // op["tile_w"] - rc[:, 0] // op["tile_w"] + 1,
                             torch.zeros_like(rc[:, 0])).sum())
    kernels = call_fractions(call_ms, scene.n, K, M_cols, n_eval, n_blend, W * H, cam, op, hbm, alu)
    out = {"workload": case["name"], "particles": scene.n, "width": W, "height": H, "keys": K,
           "fwd_ms": fwd_ms, "fwd_mpix_s": W * H / (fwd_ms / 1e3) / 1e6, "evaluations": n_eval,
           "blended": n_blend, "kernels": kernels, "launch": "cuda_graph", "steps": steps,
           "l2": "flushed (256 MB written) before every timed step; median step"}
    del r, g, scene, flush
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2412_12507_gb300 import abi, build, render

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    build.build()
    L = abi.lib()

    case = workload(args.workload)
    sc_np, cam, op = case["scene"], case["camera"], case["options"]
    W, H = cam["width"], cam["height"]
    P = W * H
    scene = render.Scene.from_arrays(sc_np, dev)
    r = render.Renderer(cam, op, capacity=1 << 20)
    r.forward(scene)                       # sizes the key capacity (one sync, outside timing)
    torch.cuda.synchronize()
    K = r.binning.count()
    r.capacity = int(K * 1.05) + 1024
    r.binning = None
    frame0 = r.forward(scene)
    # upstream gradient of the training step's loss L = mean((rgb - target)^2) against a seeded
    # U(0, 1) target, taken at the rendered image (fixed over the timed steps; no alpha term)
    rng = np.random.default_rng(77)
    target = torch.as_tensor(rng.uniform(0.0, 1.0, (3, H, W)).astype(np.float32)).to(dev)
    d_rgb = (2.0 / (3 * P)) * (frame0.rgb - target)
    d_alpha = torch.zeros((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def fwd_eager():
        r.forward(scene, sync_check=False)

    def fwd_bwd_eager():
        r.forward(scene, sync_check=False)
        r.backward(scene, d_rgb, d_alpha)

    # the timed steps replay the library's own step captured as CUDA graphs (every kernel runs,
    # no host launch gaps); the eager steps are timed too
    g_fwd, g_frame, _ = r.capture(scene)
    g_fb, _, _ = r.capture(scene, d_rgb, d_alpha)
    torch.cuda.synchronize()

    def fwd():
        g_fwd.replay()

    def fwd_bwd():
        g_fb.replay()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), world, dev) / steps

    # launches per step (host-side counter of the library, counted on an eager step: a graph
    # replay runs the same kernels)
    c0 = L.ut_kernel_launch_count()
    fwd_eager()
    launches_fwd = L.ut_kernel_launch_count() - c0
    c0 = L.ut_kernel_launch_count()
    fwd_bwd_eager()
    launches_fb = L.ut_kernel_launch_count() - c0
    torch.cuda.synchronize()

    # clocks are sampled from here through the multi-view batch (every timed region; 200 ms period)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    fwd_ms = timed(fwd, args.steps, max(3, args.warmup))
    fb_ms = timed(fwd_bwd, args.steps, max(3, args.warmup))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu = measure_alu_peaks(L, dev, stream, sms)
    fwd_eager_ms = timed(fwd_eager, args.steps, max(3, args.warmup))
    fb_eager_ms = timed(fwd_bwd_eager, args.steps, max(3, args.warmup))
    if K > r.binning.capacity or r.binning.count() != K:
        raise SystemExit("key count changed during the timed region")

    # per-call durations (events on the launching stream around each ABI call, eager steps)
    calls = {"ut_project": [], "bin_and_sort": [], "composite_forward": [], "composite_backward": []}
    for _ in range(max(3, args.steps // 2)):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        queue_ahead(stream)
        ev[0].record(stream)
        render.project(scene, cam, op, r.proj)
        ev[1].record(stream)
        render.bin_and_sort(r.proj, cam, op, r.capacity, ws=r.ws, out=r.binning)
        ev[2].record(stream)
        render.composite_forward(scene, cam, op, r.proj, r.binning, r.frame, ws=r.fws)
        ev[3].record(stream)
        r.backward(scene, d_rgb, d_alpha)
        ev[4].record(stream)
        torch.cuda.synchronize()
        for j, k in enumerate(calls):
            calls[k].append(ev[j].elapsed_time(ev[j + 1]))
    call_ms = {k: statistics.median(v) for k, v in calls.items()}

    # algorithmic work: evaluations / blends counted by the forward kernel itself
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    render.composite_forward(scene, cam, op, r.proj, r.binning, r.frame, stats=stats, ws=r.fws)
    torch.cuda.synchronize()
    n_eval, n_blend = (int(v) for v in stats.cpu())
    n = scene.n
    rc = r.proj.rect.long()
    M_cols = int(torch.where(r.proj.ntiles > 0, rc[:, 2] // op["tile_w"] - rc[:, 0] // op["tile_w"] + 1,
                             torch.zeros_like(rc[:, 0])).sum())  # column entries of the binning
    hbm, sm_max, src = peaks()
    fp32_peak = alu["fp32_tflops"]  # measured in this run
    fp32_nominal = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
    kernels = call_fractions(call_ms, n, K, M_cols, n_eval, n_blend, P, cam, op, hbm, alu)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": measured_traffic(dom, case["name"]),
                "peak_source": (f"{src} HBM copy" if d["bound"] == "hbm" else
                                f"measured FP32 FMA-chain probe in this run ({alu['how']}; nominal "
                                f"{sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz = {fp32_nominal:.1f})")}

    # end to end through the public API with host buffers: every step copies the scene in from
    # pinned host memory and the image (rgb, alpha) back out; render.FramePipeline overlaps a
    # step's copies with the neighbouring steps' rendering (two device scene buffers, a copy
    # stream and a read-back stream)
    host = {k: torch.as_tensor(sc_np[k]).pin_memory() for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    pipe = render.FramePipeline(cam, op, host, int(sc_np["sh_degree"]))
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = pipe.host_out[0].numel() * pipe.host_out[0].element_size()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(3):
        pipe.submit(host)
    pipe.join(stream)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pipe.copy_stream.wait_stream(stream)  # the first copy starts after the start event
    for _ in range(e2e_steps):
        pipe.submit(host)
    pipe.join(stream)  # the end event follows the last image read-back
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / e2e_steps
    del pipe

    variants = run_variants(scene, cam, op, d_rgb, d_alpha, timed, args.steps, max(3, args.warmup))
    fisheye_shell = small = None
    if args.workload != "fisheye_shell_100k_720p" and not args.no_extra_workloads:
        fisheye_shell = run_forward_workload("fisheye_shell_100k_720p", dev, args.steps, max(3, args.warmup), timed,
                                             alu, peaks()[0])
    if args.workload != "pinhole_1k_64" and not args.no_extra_workloads:
        small = run_forward_workload("pinhole_1k_64", dev, args.steps, max(3, args.warmup), timed, alu, peaks()[0])

    multiview = None
    if args.multiview_steps > 0:
        multiview = run_multiview(dev, args.multiview_steps, max(3, args.warmup), timed)
    clk = clocks.stop()  # sampled over every timed region above

    serve = None
    if args.serve_requests > 0:
        sc_list = serving_scenes(dev)
        reqs = serving_requests(args.serve_warmup + args.serve_requests, args.serve_rate)
        pix = sum(c["width"] * c["height"] for _, _, c in reqs[args.serve_warmup:])
        lat_s, wall_s, st = run_serving(sc_list, op, reqs, args.serve_warmup, int(args.serve_arena_gb * (1 << 30)))
        lat_p, wall_p = run_plain(sc_list, op, reqs, args.serve_warmup)
        sizes = [s.n for s in sc_list]
        meas = reqs[args.serve_warmup:]
        serve = {"requests": args.serve_requests, "warmup_requests": args.serve_warmup, "rate_req_s": args.serve_rate,
                 "p50_ms": float(np.percentile(lat_s, 50)), "p99_ms": float(np.percentile(lat_s, 99)),
                 "mean_ms": float(lat_s.mean()), "mpix_s": pix / wall_s / 1e6,
                 "plain_p50_ms": float(np.percentile(lat_p, 50)), "plain_p99_ms": float(np.percentile(lat_p, 99)),
                 "plain_mpix_s": pix / wall_p / 1e6, "offered_mpix_s": pix / (reqs[-1][0] - reqs[args.serve_warmup][0]) / 1e6,
                 "server": st, "scenes": sizes, "server_latency": latency_breakdown(lat_s, meas, sizes),
                 "plain_latency": latency_breakdown(lat_p, meas, sizes)}
        if args.serve_saturated_requests > 0:
            # the same kind of trace offered far above capacity: the sustained throughput of each arm
            n_w = min(100, args.serve_saturated_requests // 4)
            sreqs = serving_requests(n_w + args.serve_saturated_requests, args.serve_saturated_rate, seed=5)
            spix = sum(c["width"] * c["height"] for _, _, c in sreqs[n_w:])
            lat_s2, wall_s2, st2 = run_serving(sc_list, op, sreqs, n_w, int(args.serve_arena_gb * (1 << 30)))
            lat_p2, wall_p2 = run_plain(sc_list, op, sreqs, n_w)
            serve["saturated"] = {
                "requests": args.serve_saturated_requests, "rate_req_s": args.serve_saturated_rate,
                "offered_mpix_s": spix / (sreqs[-1][0] - sreqs[n_w][0]) / 1e6,
                "mpix_s": spix / wall_s2 / 1e6, "plain_mpix_s": spix / wall_p2 / 1e6,
                "p50_ms": float(np.percentile(lat_s2, 50)), "p99_ms": float(np.percentile(lat_s2, 99)),
                "plain_p50_ms": float(np.percentile(lat_p2, 50)), "plain_p99_ms": float(np.percentile(lat_p2, 99)),
                "server": st2}
        del sc_list
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        f_s, desc, thr = oracle_frame_time(case, args.cpu_seconds)
        cpu = {"value": P / f_s / 1e6, "unit": "Mpix/s", "cores": thr, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": job_mpix_s(P, world, fwd_ms), "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": fwd_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": case["name"], "particles": n, "width": W, "height": H,
                       "camera": "fisheye+rolling_shutter", "sh_degree": int(sc_np["sh_degree"]),
                       "tile": f"{op['tile_w']}x{op['tile_h']}", "keys": K, "parallelism": f"replicas{world}",
                       "launch": "cuda_graph (the library step captured by Renderer.capture)",
                       "l2": "inputs larger than L2 (236 MB scene + 2 x keys), no flush"},
            "fwd_ms": fwd_ms, "fwd_bwd_ms_per_view": fb_ms, "fwd_bwd_mpix_s": job_mpix_s(P, world, fb_ms),
            "eager": {"fwd_ms": fwd_eager_ms, "fwd_bwd_ms": fb_eager_ms,
                      "fwd_mpix_s": job_mpix_s(P, world, fwd_eager_ms)},
            "kernels": kernels, "evaluations": n_eval, "blended": n_blend, "alu_peaks": alu,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "e2e": {"value": job_mpix_s(P, world, e2e_ms), "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "overlap": "render.FramePipeline: a step's copies overlap the neighbouring steps' rendering"},
            "gpu_launches": int(launches_fwd * args.steps + launches_fb * args.steps),
            "launches_per_step": {"fwd": int(launches_fwd), "fwd_bwd": int(launches_fb)},
            "variants": variants,
            "fisheye_shell_100k_720p": fisheye_shell,
            "pinhole_1k_64": small,
            "multiview": multiview,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
