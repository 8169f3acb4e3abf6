"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare
with the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_2412_12507_gb300 import render

# near-tie tolerances handed to the oracle: pixels whose FP64 decisions lie this close to
# a threshold may legitimately differ from the FP32 kernels and are reported separately
TOL = dict(eps_px=5e-3, eps_rel=2e-4, eps_t=2e-3, depth_ulps=4, cond_min=0.05)
RGB_TOL = 1e-4


def run_gpu(scene_np, cam, opts, capacity=None, want_keys=False, rect=None, depth=None):
    """Projection + binning + forward on cuda:0.  rect / depth override the projection's
    (synthetic inputs for exercising the later stages on their own)."""
    scene = render.Scene.from_arrays(scene_np, "cuda")
    proj = render.project(scene, cam, opts)
    if rect is not None:
        proj.rect = torch.as_tensor(np.asarray(rect, np.int16)).cuda()
        proj.depth = torch.as_tensor(np.asarray(depth, np.float32)).cuda()
        o = render.abi.make_options(opts)
        r = np.asarray(rect, np.int64)
        nt = np.where(r[:, 0] <= r[:, 2], (r[:, 2] // o.tile_w - r[:, 0] // o.tile_w + 1) *
                      (r[:, 3] // o.tile_h - r[:, 1] // o.tile_h + 1), 0)
        proj.ntiles = torch.as_tensor(nt.astype(np.int32)).cuda()
    K = int(proj.ntiles.to(torch.int64).sum().item())
    cap = capacity if capacity is not None else max(K, 1)
    b = render.bin_and_sort(proj, cam, opts, cap, want_keys=want_keys)
    frame = render.composite_forward(scene, cam, opts, proj, b)
    torch.cuda.synchronize()
    return dict(scene=scene, proj=proj, binning=b, frame=frame, K=b.count(), K_sum=K)


def to_np(t):
    return t.detach().cpu().numpy()


def frame_at(frame, px, py):
    rgb = to_np(frame.rgb)
    tf = to_np(frame.t_final)[py, px] if frame.t_final is not None else None
    return rgb[:, py, px].T, to_np(frame.alpha)[py, px], tf


# flags whose pixels carry no bound: a particle whose culling is a near tie may be present on one
# side only, and the oracle does not evaluate a culled particle
UNBOUNDED = oracle.F_CULL_TIE


def compare_frame(frame, ref, tol=RGB_TOL, unbounded=None):
    """Per-pixel error of the GPU frame beyond what the oracle bounds:
    err = max(|rgb - oracle| - slack - fslack - rslack, |alpha - oracle| - aslack - faslack - raslack),
    where slack covers depth-tied pairs and stop-threshold ties, fslack the other flagged decisions
    and rslack the FP32 rounding of the blended particles' alphas.  Every pixel without an
    `unbounded` flag (default: a culling near-tie) is compared against tol."""
    unb = UNBOUNDED if unbounded is None else unbounded
    got_rgb, got_a, _ = frame_at(frame, ref["px"], ref["py"])
    flags = ref["flags"]
    flagged = (flags & oracle.F_FORWARD_TIES) != 0
    bounded = (flags & unb) == 0
    raw = np.maximum(np.abs(got_rgb - ref["rgb"]).max(axis=1), np.abs(got_a - ref["alpha"]))
    err = np.maximum(np.abs(got_rgb - ref["rgb"]).max(axis=1) - ref["slack"] - ref["fslack"] - ref["rslack"],
                     np.abs(got_a - ref["alpha"]) - ref["aslack"] - ref["faslack"] - ref["raslack"])
    fb = flagged & bounded
    out = dict(max_err=float(err[bounded].max()) if bounded.any() else 0.0, n=int(err.size),
               n_flagged=int(flagged.sum()), n_unbounded=int((~bounded).sum()),
               n_slack=int((ref["slack"] > 0).sum()), n_bad=int((err[bounded] > tol).sum()),
               max_err_flagged=float(err[fb].max()) if fb.any() else 0.0, max_raw=float(raw.max()),
               max_rslack=float(ref["rslack"].max()))
    if bounded.any():
        q = int(np.argmax(np.where(bounded, err, -np.inf)))
        out["worst"] = dict(px=int(ref["px"][q]), py=int(ref["py"][q]), flags=int(flags[q]), raw=float(raw[q]),
                            slack=float(ref["slack"][q]), fslack=float(ref["fslack"][q]),
                            rslack=float(ref["rslack"][q]))
    return out


def gpu_decisions(g):
    """The GPU projection's discrete decisions (rects and FP32 depth bits) for the oracle: with
    them the oracle composites exactly the per-pixel lists the kernels composite."""
    return dict(rect=to_np(g["proj"].rect).astype(np.int32), depth32=to_np(g["proj"].depth))


# the oracle's tolerances in decision-injected mode: rects and depth order come from the GPU,
# so no rect-edge, culling or depth-order flags remain
TOL_INJECTED = dict(TOL, depth_ulps=-1)


def sample_pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    q = rng.choice(W * H, size=min(n, W * H), replace=False)
    return (q % W).astype(np.int32), (q // W).astype(np.int32)

# Element-wise gradient bar: |g - g_ref| <= 1e-3 |g_ref| + 1e-6 max |g_ref| + KAPPA mag, where mag
# is the oracle's magnitude of that element (its whole computation evaluated on absolute values).
# A floating-point evaluation errs by at most about (rounding steps) x u x mag (u = 2^-24, the
# running error bound).  The SH coefficients' gradients are contracted on the tensor cores with
# BF16 hi / lo operands, whose three-term products carry a relative error up to 2^-15 each;
# KAPPA = 2^-14 covers that and the sums' own rounding (1024 u).
KAPPA = 2.0 ** -14


def grad_compare(got, ref, mag, name, rel=1e-3):
    """Per tensor ||g - g_ref|| / ||g_ref|| <= rel, and every element within the bar above."""
    g = got.reshape(-1).astype(np.float64)
    r = ref.reshape(-1)
    m = mag.reshape(-1)
    nrm = np.linalg.norm(r)
    assert nrm > 0, name
    e = np.linalg.norm(g - r) / nrm
    assert e <= rel, (name, e)
    bound = rel * np.abs(r) + 1e-6 * np.max(np.abs(r)) + KAPPA * m
    bad = np.abs(g - r) > bound
    if bad.any():
        j = int(np.argmax(np.abs(g - r) / bound))
        raise AssertionError((name, int(bad.sum()), "worst", j, float(g[j]), float(r[j]), float(m[j])))
    return e
