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


def compare_frame(frame, ref, tol=RGB_TOL):
    """Max |rgb - oracle| and |alpha - oracle| over pixels without a forward near-tie flag."""
    got_rgb, got_a, _ = frame_at(frame, ref["px"], ref["py"])
    flagged = (ref["flags"] & oracle.F_FORWARD_TIES) != 0
    # reordering depth-tied pairs changes the colour by at most the oracle's slack
    err = np.maximum(np.abs(got_rgb - ref["rgb"]).max(axis=1) - ref["slack"],
                     np.abs(got_a - ref["alpha"]) - ref["aslack"])
    ok = ~flagged
    return dict(max_err=float(err[ok].max()) if ok.any() else 0.0, n=int(err.size), n_flagged=int(flagged.sum()),
                n_slack=int((ref["slack"] > 0).sum()),
                n_bad=int((err[ok] > tol).sum()), max_err_flagged=float(err[flagged].max()) if flagged.any() else 0.0)


def sample_pixels(W, H, n, seed):
    rng = np.random.default_rng(seed)
    q = rng.choice(W * H, size=min(n, W * H), replace=False)
    return (q % W).astype(np.int32), (q // W).astype(np.int32)
