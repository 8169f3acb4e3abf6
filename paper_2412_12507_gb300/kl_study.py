"""Accuracy of the projected 2D Gaussians: UT vs first-order EWA against a Monte Carlo reference.

The supplementary material's projection validation compares, per visible Gaussian, the 2D
Gaussian each method produces with a Monte Carlo reference (500 samples of the 3D Gaussian
pushed through the camera model, rolling shutter included) by the KL divergence of the two 2D
normals, over pinhole / fisheye cameras with and without rolling shutter, a fisheye field-of-
view sweep, a radial-distortion sweep (k2) and a rolling-shutter lateral-translation sweep.
This module reruns that study on synthetic Gaussians (the paper's trained scenes are not
available, so its printed medians are not a target; the qualitative claims are):

    python -m paper_2412_12507_gb300.kl_study [--gaussians 4000] [--samples 500] [--json out.json]

Everything runs through the library: ut_project (UT and EWA) and ut_project_points (the Monte
Carlo samples).  KL(reference || method) of the 2D normals.  With S samples per reference the
estimated moments alone give a KL of about 5 / (2 S) (five estimated parameters): 5e-3 at the
paper's 500 samples, which is the level of its printed UT medians; use more samples to resolve
smaller differences.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import synth


def gauss_kl(m0, C0, m1, C1):
    """KL(N(m0, C0) || N(m1, C1)) for batches of 2D normals: m [n, 2], C [n, 2, 2] (float64)."""
    m0, C0, m1, C1 = (np.asarray(a, np.float64) for a in (m0, C0, m1, C1))
    inv1 = np.linalg.inv(C1)
    dm = (m1 - m0)[..., None]
    tr = np.einsum("nij,nji->n", inv1, C0)
    quad = (np.swapaxes(dm, 1, 2) @ inv1 @ dm)[:, 0, 0]
    ld = np.linalg.slogdet(C1)[1] - np.linalg.slogdet(C0)[1]
    return 0.5 * (tr + quad - 2.0 + ld)


def _cov(c3):
    c3 = np.asarray(c3, np.float64)
    return np.stack([np.stack([c3[:, 0], c3[:, 1]], -1), np.stack([c3[:, 1], c3[:, 2]], -1)], -2)


def gaussians_in_view(cam: dict, n: int, seed: int, log_s=(-3.3, 0.4), depth=(2.0, 6.0), max_angle_deg=75.0):
    """n Gaussians whose means lie along random camera rays within max_angle of the optical axis
    (and inside a pinhole's frustum), at depths U(depth), with log-scales N(log_s), in the
    start pose's world frame."""
    rng = np.random.default_rng(seed)
    if cam["model"] == "fisheye":
        th = np.arccos(rng.uniform(math.cos(math.radians(max_angle_deg)), 1.0, n))
        ph = rng.uniform(0, 2 * math.pi, n)
        dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    else:
        W, H = cam["width"], cam["height"]
        u, v = rng.uniform(0, W, n), rng.uniform(0, H, n)
        dirs = np.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], np.ones(n)], 1)
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    xc = dirs * rng.uniform(depth[0], depth[1], n)[:, None]
    from .synth import _quat_to_rot_np
    R0 = _quat_to_rot_np(np.asarray(cam["q_start"], np.float64) / np.linalg.norm(cam["q_start"]))
    means = (xc - np.asarray(cam["t_start"], np.float64)) @ R0  # x = R0^T (x_c - t)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return dict(means=means.astype(np.float32), log_scales=rng.normal(log_s[0], log_s[1], (n, 3)).astype(np.float32),
                quats=q.astype(np.float32), opacity_logits=np.full(n, 4.0, np.float32),
                sh=np.zeros((n, 1, 3), np.float32), sh_degree=0)


def study(cam: dict, n: int = 4000, samples: int = 500, seed: int = 0, opts: dict | None = None, device="cuda"):
    """Median / 90th-percentile KL of the UT and EWA 2D Gaussians against the Monte Carlo
    reference for n Gaussians in view of `cam` (only Gaussians that every method keeps and
    whose samples all project validly are compared)."""
    import torch

    from . import render
    op = synth.options(**(opts or {}))
    sc = gaussians_in_view(cam, n, seed)
    scene = render.Scene.from_arrays(sc, device)
    res = {}
    for name, mode in (("ut", 0), ("ewa", 1)):
        p = render.project(scene, cam, dict(op, projection=mode))
        res[name] = (p.mean2d.double().cpu().numpy(), p.cov2d.double().cpu().numpy(),
                     (p.ntiles > 0).cpu().numpy())
    # Monte Carlo reference: x = mu + R S z, z ~ N(0, I)
    rng = np.random.default_rng(seed + 1)
    from .synth import _quat_to_rot_np
    R = np.stack([_quat_to_rot_np(q) for q in sc["quats"].astype(np.float64)])
    S = np.exp(sc["log_scales"].astype(np.float64))
    z = rng.standard_normal((n, samples, 3))
    x = sc["means"].astype(np.float64)[:, None, :] + np.einsum("nij,nsj->nsi", R, z * S[:, None, :])
    uv, ok = render.project_points(torch.as_tensor(x.reshape(-1, 3), dtype=torch.float32, device=device), cam, op)
    uv = uv.double().cpu().numpy().reshape(n, samples, 2)
    ok = ok.cpu().numpy().reshape(n, samples).all(1)
    mref = uv.mean(1)
    d = uv - mref[:, None, :]
    Cref = np.einsum("nsi,nsj->nij", d, d) / (samples - 1)
    keep = ok & res["ut"][2] & res["ewa"][2] & (np.linalg.det(Cref) > 0)
    out = {"gaussians": int(keep.sum()), "samples": samples}
    kl = {}
    for name in ("ut", "ewa"):
        m, c, _ = res[name]
        kl[name] = gauss_kl(mref[keep], Cref[keep], m[keep], _cov(c[keep]))
        out[name] = {"median": float(np.median(kl[name])), "p90": float(np.percentile(kl[name], 90))}
    out["ut_better_fraction"] = float(np.mean(kl["ut"] < kl["ewa"]))
    return out


def _rs_pose(shift, yaw_deg=0.0):
    return synth.rs_end_pose(shift, yaw_deg)


def configurations(width=1280, height=720, seed=5):
    """The study's camera set: the four static / rolling-shutter pinhole and fisheye cases, an
    equidistant-fisheye field-of-view sweep, a radial-distortion (k2) sweep and a rolling-
    shutter lateral-translation sweep."""
    rng = np.random.default_rng(seed)
    k_fish = rng.uniform(-0.05, 0.05, 4)
    qe, te = _rs_pose(0.35, 5.0)
    cfg = {
        "pinhole": synth.camera("pinhole", width, height, fx=0.6 * width),
        "pinhole_rs": synth.camera("pinhole", width, height, fx=0.6 * width, q_end=qe, t_end=te, rolling_shutter=1),
        "fisheye": synth.camera("fisheye", width, height, k=k_fish),
        "fisheye_rs": synth.camera("fisheye", width, height, k=k_fish, q_end=qe, t_end=te, rolling_shutter=1),
    }
    for fov in (90, 120, 150, 180):
        cfg[f"equidistant_fov{fov}"] = synth.camera("fisheye", width, height, fx=width / math.radians(fov))
    for k2 in (0.0, 0.1, 0.3, 0.5):
        cfg[f"radial_k2_{k2:.1f}"] = synth.camera("pinhole_radial", width, height, fx=0.6 * width, k=[0.0, k2, 0.0, 0.0])
    for shift in (0.0, 0.1, 0.2, 0.35):
        qe2, te2 = _rs_pose(shift, 0.0)
        cfg[f"rs_shift_{shift:.2f}"] = synth.camera("pinhole", width, height, fx=0.6 * width, q_end=qe2, t_end=te2,
                                                    rolling_shutter=1)
    return cfg


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gaussians", type=int, default=4000)
    ap.add_argument("--samples", type=int, default=500)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    rows = {}
    print("| camera | Gaussians | UT median KL | EWA median KL | UT p90 | EWA p90 | UT better |")
    print("|---|---|---|---|---|---|---|")
    for name, cam in configurations().items():
        r = study(cam, a.gaussians, a.samples)
        rows[name] = r
        print(f"| {name} | {r['gaussians']} | {r['ut']['median']:.2e} | {r['ewa']['median']:.2e} | "
              f"{r['ut']['p90']:.2e} | {r['ewa']['p90']:.2e} | {100 * r['ut_better_fraction']:.0f} % |", flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
