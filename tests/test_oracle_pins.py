"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these tests retypes the oracle's formulas: each compares it with a closed
form, an invariant, a library routine, brute force, or a hand-derived expansion,
chosen so that a dropped term, a wrong sign / index or a transposed operand in the
oracle fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest

from paper_2412_12507_gb300 import synth


def rot(q):
    q = np.asarray(q, float)
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def axis_angle_rot(axis, ang):
    """Rodrigues' formula (an independent route to a rotation matrix)."""
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def one_scene(mu, log_s, q, logit, sh, deg=0):
    return dict(means=np.array([mu], np.float32), log_scales=np.array([log_s], np.float32),
                quats=np.array([q], np.float32), opacity_logits=np.array([logit], np.float32),
                sh=np.array(sh, np.float32).reshape(1, (deg + 1) ** 2, 3), sh_degree=deg)


# ------------------------------------------------------------------ rotations

def test_quaternion_rotation_matches_rodrigues(orc):
    """R(q) of the oracle (through an orthographic UT of a needle Gaussian) equals the
    axis-angle rotation built by Rodrigues' formula."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        axis = rng.standard_normal(3)
        ang = rng.uniform(0, math.pi)
        a = axis / np.linalg.norm(axis)
        q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * a])
        R = axis_angle_rot(axis, ang)
        assert np.allclose(rot(q), R, atol=1e-12)
        # the oracle sees R through the 2D covariance of an orthographic camera: A R S^2 R^T A^T
        s = np.array([0.3, 0.1, 0.05])
        cam = synth.camera("ortho", 64, 64, fx=10.0, fy=10.0)
        ok, vmu, cov = orc.ut_estimate(cam, [0.1, 0.2, 3.0], R, s)
        Sig = (R * s**2) @ R.T
        assert ok
        assert np.allclose(cov, [100 * Sig[0, 0], 100 * Sig[0, 1], 100 * Sig[1, 1]], rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ Unscented Transform

@pytest.mark.parametrize("ut", [(1.0, 2.0, 0.0), (0.5, 2.0, 0.0), (1.0, 0.0, 1.0), (1.3, 2.0, -0.5)])
def test_ut_exact_for_affine_camera(orc, ut):
    """For an affine g the UT mean and covariance are A mu + b and A Sigma A^T exactly, for
    any (alpha, beta, kappa) with 3 + lambda > 0 (moment matching, Sec. 4.1)."""
    rng = np.random.default_rng(11)
    Rc = axis_angle_rot([0.3, -1.0, 0.2], 0.7)
    qc = synth._rot_to_quat(Rc)
    tc = np.array([0.2, -0.1, 1.5])
    cam = synth.camera("ortho", 100, 80, fx=37.0, fy=29.0, cx=41.0, cy=33.0, q=qc, t=tc)
    # the camera carries FP32-rounded pose numbers: use exactly those
    Rc, tc = rot(cam["q_start"]), np.array(cam["t_start"])
    for _ in range(10):
        mu = rng.uniform(-1, 1, 3)
        R = rot(rng.standard_normal(4))
        s = np.exp(rng.normal(-1.5, 0.5, 3))
        ok, vmu, cov = orc.ut_estimate(cam, mu, R, s, ut=ut)
        assert ok
        A = np.array([[37.0, 0, 0], [0, 29.0, 0]]) @ Rc
        b = np.array([37.0 * tc[0] + 41.0, 29.0 * tc[1] + 33.0])
        Sig = R @ np.diag(s**2) @ R.T
        C2 = A @ Sig @ A.T
        assert np.allclose(vmu, A @ mu + b, rtol=0, atol=1e-10)
        assert np.allclose(cov, [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-10, atol=1e-10)


def test_ut_pinhole_constant_depth_is_exact(orc):
    """A flat Gaussian parallel to the image plane of a pinhole camera sees an affine map on
    its support, so the UT recovers the projected moments exactly."""
    cam = synth.camera("pinhole", 640, 480, fx=500.0, fy=450.0, cx=320.0, cy=240.0)
    ang = 0.6
    R = axis_angle_rot([0, 0, 1], ang)
    s = np.array([0.05, 0.02, 1e-12])
    mu = np.array([0.3, -0.2, 2.5])
    ok, vmu, cov = orc.ut_estimate(cam, mu, R, s)
    assert ok
    assert np.allclose(vmu, [500 * 0.3 / 2.5 + 320, 450 * -0.2 / 2.5 + 240], atol=1e-9)
    J = np.diag([500 / 2.5, 450 / 2.5])
    C2 = J @ (R[:2, :2] @ np.diag(s[:2] ** 2) @ R[:2, :2].T) @ J
    assert np.allclose(cov, [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-9)


def test_ut_depth_expansion_pins_weights(orc):
    """Needle Gaussian along the optical axis, offset in x, pinhole camera: with
    eps = (s_z / Z0)^2 and a = f X / Z0, a hand expansion of eq. weights_1/2 and
    eq. 2d_conic_1/2 at (alpha, beta, kappa) = (1, 2, 0) gives
        mean / a = 1 + eps + 3 eps^2 + O(eps^3)
        var  / a^2 = eps + 10 eps^2 + O(eps^3)
    The true moments of f X / Z are 1 + eps + 3 eps^2 and eps + 8 eps^2; the extra 2 eps^2 is
    the (1 - alpha^2 + beta) covariance weight of the centre point, so dropping that term,
    or a wrong sqrt(3 + lambda) spread, fails here."""
    cam = synth.camera("pinhole", 64, 64, fx=100.0, fy=100.0, cx=0.0, cy=0.0)
    X, Z0 = 0.7, 3.0
    a = 100.0 * X / Z0
    E, C1, C2 = [], [], []
    for sz in (0.015, 0.03, 0.045, 0.06):
        eps = (sz / Z0) ** 2
        ok, vmu, cov = orc.ut_estimate(cam, [X, 0.0, Z0], np.eye(3), [1e-14, 1e-14, sz])
        assert ok
        E.append(eps)
        C1.append((vmu[0] / a - 1 - eps) / eps**2)
        C2.append((cov[0] / a**2 - eps) / eps**2)
    # the second-order coefficients, extrapolated to eps -> 0 by a linear fit in eps
    c1 = np.polyfit(E, C1, 1)[1]
    c2 = np.polyfit(E, C2, 1)[1]
    assert abs(c1 - 3.0) < 2e-3, c1
    assert abs(c2 - 10.0) < 2e-3, c2


@pytest.mark.parametrize("model", ["pinhole", "fisheye"])
def test_ut_close_to_monte_carlo(orc, model):
    """Sanity check of the UT against Monte Carlo moments (the supplementary's reference):
    for small Gaussians the UT mean / covariance agree with MC up to sampling error and
    higher-order terms."""
    rng = np.random.default_rng(3)
    if model == "pinhole":
        cam = synth.camera("pinhole", 640, 480, fx=400.0, fy=400.0)
    else:
        cam = synth.camera("fisheye", 640, 480, k=[0.03, -0.01, 0.004, -0.001])
    for _ in range(4):
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2.5, 4)])
        R = rot(rng.standard_normal(4))
        s = np.exp(rng.normal(-3.5, 0.3, 3))
        ok, vmu, cov = orc.ut_estimate(cam, mu, R, s)
        assert ok
        x = mu + (rng.standard_normal((200_000, 3)) * s) @ R.T
        uv = np.array([orc.project_point(cam, xi)[1] for xi in x[:20000]])
        m = uv.mean(0)
        C = np.cov(uv.T)
        se = np.sqrt(np.diag(C) / len(uv))
        assert np.all(np.abs(m - vmu) < 6 * se + 1e-3 * np.sqrt(np.diag(C)))
        assert np.allclose(cov, [C[0, 0], C[0, 1], C[1, 1]], rtol=0.08, atol=0.05 * np.sqrt(C[0, 0] * C[1, 1]))


# ------------------------------------------------------------------ cameras

def test_fisheye_equidistant_closed_form(orc):
    """k = 0: the polynomial fisheye is equidistant, radius = f * angle from the axis."""
    cam = synth.camera("fisheye", 800, 600, fx=300.0, fy=300.0)
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = rng.standard_normal(3)
        x[2] = abs(x[2]) + 0.1
        ok, uv, _ = orc.project_point(cam, x)
        assert ok
        ang = math.acos(x[2] / np.linalg.norm(x))
        r = math.hypot(uv[0] - 400, uv[1] - 300)
        assert abs(r - 300 * ang) < 1e-9
        # direction in the image plane is the direction of (X, Y)
        assert abs(math.atan2(uv[1] - 300, uv[0] - 400) - math.atan2(x[1], x[0])) < 1e-9


@pytest.mark.parametrize("k", [[0, 0, 0, 0], [0.03, -0.01, 0.004, -0.001], [-0.05, -0.04, 0.03, -0.05]])
def test_fisheye_ray_inverts_the_distortion(orc, k):
    """The pixel ray's angle theta from the optical axis solves theta_d(theta) = r_d; for k = 0
    (equidistant) theta = r_d exactly, which starts the root search on an exact root."""
    cam = synth.camera("fisheye", 640, 480, fx=200.0, fy=200.0, k=k)
    kk = np.array(cam["k"])
    tm = orc.theta_max(kk)
    rng = np.random.default_rng(3)
    for _ in range(200):
        px, py = rng.uniform(0, 640), rng.uniform(0, 480)
        rd = math.hypot((px - 320) / 200, (py - 240) / 200)
        ok, o, d = orc.pixel_ray(cam, px, py)
        th_lim = tm * (1 + kk[0] * tm**2 + kk[1] * tm**4 + kk[2] * tm**6 + kk[3] * tm**8)
        assert ok == (rd <= th_lim)
        if not ok:
            continue
        th = math.acos(d[2] / np.linalg.norm(d))
        td = th * (1 + kk[0] * th**2 + kk[1] * th**4 + kk[2] * th**6 + kk[3] * th**8)
        assert abs(td - rd) < 1e-12, (td, rd)
        if not any(k):
            assert abs(th - rd) < 1e-13


def test_theta_max_is_first_root_of_derivative(orc):
    assert abs(orc.theta_max([0, 0, 0, 0]) - math.pi / 2) < 1e-15
    # strongly negative distortion: d theta_d / d theta turns over before pi/2
    k = [-0.05, -0.04, 0.03, -0.05]
    tm = orc.theta_max(k)
    # roots of 1 + 3 k1 u + 5 k2 u^2 + 7 k3 u^3 + 9 k4 u^4 in u = theta^2 (numpy.roots)
    r = np.roots([9 * k[3], 7 * k[2], 5 * k[1], 3 * k[0], 1.0])
    u = min(v.real for v in r if abs(v.imag) < 1e-12 and v.real > 0)
    assert tm < math.pi / 2
    assert abs(tm - math.sqrt(u)) < 1e-12


@pytest.mark.parametrize("model,rs", [("pinhole", 0), ("fisheye", 0), ("pinhole", 1), ("fisheye", 1),
                                      ("pinhole_radial", 0), ("pinhole_radial", 1)])
def test_pixel_ray_passes_through_projected_point(orc, model, rs):
    """Inverse consistency of g: the pixel ray at g(x) passes through x, including under a
    rolling shutter once the row-time fixed point has converged."""
    rng = np.random.default_rng(7)
    qe, te = synth.rs_end_pose(0.05, 2.0)
    k = {"fisheye": [0.02, -0.01, 0.003, -0.0005], "pinhole_radial": [-0.12, 0.03, -0.002, 0.0]}.get(model, [0] * 4)
    cam = synth.camera(model, 640, 480, fx=300.0 if model != "fisheye" else None, k=k, q_end=qe, t_end=te,
                       rolling_shutter=rs)
    for _ in range(20):
        x = np.array([rng.uniform(-1, 1), rng.uniform(-0.7, 0.7), rng.uniform(2, 4)])
        ok, uv, t = orc.project_point(cam, x, rs_iters=80)
        assert ok
        ok2, o, d = orc.pixel_ray(cam, uv[0], uv[1])
        assert ok2
        dn = d / np.linalg.norm(d)
        v = x - o
        dist = np.linalg.norm(v - (v @ dn) * dn)
        assert dist < 1e-9, dist
        assert v @ dn > 0


def test_rolling_shutter_with_static_pose_equals_global(orc):
    cam = synth.camera("fisheye", 640, 480, k=[0.01, 0, 0, 0])
    cam_rs = dict(cam, rolling_shutter=1)
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2, 4)])
        a = orc.project_point(cam, x)
        b = orc.project_point(cam_rs, x)
        assert a[0] and b[0]
        assert np.array_equal(a[1], b[1])


def test_rolling_shutter_fixed_point_converges_to_row_time(orc):
    """With many updates the sigma-point time equals the time of the row it lands on."""
    qe, te = synth.rs_end_pose(0.05, 2.0)
    cam = synth.camera("fisheye", 1920, 1080, q_end=qe, t_end=te, rolling_shutter=1)
    rng = np.random.default_rng(4)
    for _ in range(10):
        x = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(2, 4)])
        ok, uv, t = orc.project_point(cam, x, rs_iters=60)
        assert ok
        assert abs(t - np.clip((uv[1] - 0.5) / 1079, 0, 1)) < 1e-12


def _geodesic_pose(Ra, Ta, Rb, Tb, t):
    """Pose at time t along the rotation geodesic from Ra to Rb, by axis-angle (scipy), and
    the straight segment from Ta to Tb: an independent route to the interpolated pose."""
    from scipy.spatial.transform import Rotation
    rv = Rotation.from_matrix(Ra.T @ Rb).as_rotvec()  # angle in [0, pi]: the shorter way round
    return Ra @ Rotation.from_rotvec(t * rv).as_matrix(), (1.0 - t) * np.asarray(Ta) + t * np.asarray(Tb)


def _big_rs_camera(model="pinhole", flip=False):
    """Rolling-shutter camera whose end pose is 120 degrees from its start pose (large enough
    that a normalised lerp of the quaternions, or t read backwards, is far off the geodesic)."""
    qa = np.array([0.9, 0.1, -0.3, 0.2])
    qa /= np.linalg.norm(qa)
    axis = np.array([0.3, -0.8, 0.5]) / np.linalg.norm([0.3, -0.8, 0.5])
    rel = np.concatenate([[math.cos(math.radians(60))], math.sin(math.radians(60)) * axis])
    w1, v1 = qa[0], qa[1:]
    w2, v2 = rel[0], rel[1:]
    qb = np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])  # qa (x) rel
    if flip:
        qb = -qb  # the same rotation on the other sheet of the double cover
    return synth.camera(model, 640, 480, fx=300.0, q=qa, t=(0.1, -0.2, 0.3), q_end=qb, t_end=(0.6, 0.1, -0.4),
                        rolling_shutter=1)


@pytest.mark.parametrize("flip", [False, True])
def test_rolling_shutter_pose_follows_the_geodesic(orc, flip):
    """The pose at shutter time t (Sec. 1: each sigma point seen through its own extrinsic
    matrix): t = 0 and t = 1 give the start and end poses exactly; in between the rotation lies
    on the shorter geodesic at the fraction t of its angle and the translation on the segment.
    Checked at t = 1/4 and 3/4, where a normalised lerp, a reversed time axis or swapped end
    poses are far off."""
    cam = _big_rs_camera(flip=flip)
    Ra, Rb = rot(cam["q_start"]), rot(cam["q_end"])
    Ta, Tb = cam["t_start"], cam["t_end"]
    R0, T0 = orc.pose_at(cam, 0.0)
    R1, T1 = orc.pose_at(cam, 1.0)
    assert np.allclose(R0, Ra, atol=1e-14) and np.allclose(T0, Ta, atol=1e-15)
    assert np.allclose(R1, Rb, atol=1e-14) and np.allclose(T1, Tb, atol=1e-15)
    for t in (0.25, 0.5, 0.75, 0.1, 0.9):
        R, T = orc.pose_at(cam, t)
        Rg, Tg = _geodesic_pose(Ra, Ta, Rb, Tb, t)
        assert np.allclose(R, Rg, atol=1e-12), t
        assert np.allclose(T, Tg, atol=1e-15), t
        # the rotation angle from the start grows linearly in t (120 degrees in all, up to the
        # FP32 rounding of the camera's quaternions)
        ang = math.degrees(math.acos(np.clip((np.trace(Ra.T @ R) - 1) / 2, -1, 1)))
        total = math.degrees(math.acos(np.clip((np.trace(Ra.T @ Rb) - 1) / 2, -1, 1)))
        assert abs(total - 120.0) < 1e-4
        assert abs(ang - total * t) < 1e-9, (t, ang)
    # a global-shutter camera ignores the end pose
    R, T = orc.pose_at(dict(cam, rolling_shutter=0), 0.7)
    assert np.allclose(R, Ra, atol=1e-14) and np.allclose(T, Ta, atol=1e-15)


def test_rolling_shutter_projection_and_rays_use_the_row_pose(orc):
    """g(x) under a rolling shutter equals the plain pinhole map through the geodesic pose at
    the point's shutter time, and a pixel's ray is the camera centre and direction of the pose
    at its row's time (t = (y - 1/2) / (H - 1))."""
    cam = _big_rs_camera()
    Ra, Rb = rot(cam["q_start"]), rot(cam["q_end"])
    Ta, Tb = cam["t_start"], cam["t_end"]
    H = cam["height"]
    rng = np.random.default_rng(17)
    n_ok = 0
    for _ in range(200):
        # points in front of the camera at a random shutter time
        t0 = rng.uniform(0, 1)
        R, T = _geodesic_pose(Ra, Ta, Rb, Tb, t0)
        xc = np.array([rng.uniform(-1, 1), rng.uniform(-0.7, 0.7), rng.uniform(2, 4)])
        x = R.T @ (xc - T)
        ok, uv, t = orc.project_point(cam, x, rs_iters=3)
        if not ok:
            continue
        n_ok += 1
        R, T = _geodesic_pose(Ra, Ta, Rb, Tb, t)
        y = R @ x + T
        assert np.allclose(uv, [cam["fx"] * y[0] / y[2] + cam["cx"], cam["fy"] * y[1] / y[2] + cam["cy"]],
                           atol=1e-9)
    assert n_ok > 50
    for py in (0.5, 120.5, 239.5, 400.0, 479.5):
        px = rng.uniform(0, 640)
        ok, o, d = orc.pixel_ray(cam, px, py)
        assert ok
        R, T = _geodesic_pose(Ra, Ta, Rb, Tb, min(max((py - 0.5) / (H - 1), 0.0), 1.0))
        assert np.allclose(o, -R.T @ T, atol=1e-12)
        dc = np.array([(px - cam["cx"]) / cam["fx"], (py - cam["cy"]) / cam["fy"], 1.0])
        dw = R.T @ dc
        assert np.allclose(d / np.linalg.norm(d), dw / np.linalg.norm(dw), atol=1e-12)


# ------------------------------------------------------------------ spherical harmonics

def test_sh_orthonormal(orc):
    """Orthonormality of the degree-3 real basis by Gauss-Legendre x uniform quadrature."""
    z, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for zi, wi in zip(z, wz):
        r = math.sqrt(1 - zi * zi)
        for p in phi:
            Y = orc.sh_basis(3, [r * math.cos(p), r * math.sin(p), zi])
            G += wi * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_gradient(orc):
    """The analytic gradient of the basis polynomials (the per-particle colour's dY/dmu) against
    central differences of the polynomials themselves, and its tangential part against central
    differences of scipy's spherical harmonics of the normalised direction."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(12)

    def real_sh(v):
        d = v / np.linalg.norm(v)
        theta, phi = math.acos(max(-1.0, min(1.0, d[2]))), math.atan2(d[1], d[0])
        out = np.zeros(16)
        for l in range(4):
            for m in range(0, l + 1):
                c = sp.sph_harm_y(l, m, theta, phi) if hasattr(sp, "sph_harm_y") else sp.sph_harm(m, l, phi, theta)
                if m == 0:
                    out[l * l + l] = c.real
                else:
                    out[l * l + l + m] = math.sqrt(2) * c.real
                    out[l * l + l - m] = math.sqrt(2) * c.imag
        return out

    for deg in (1, 2, 3):
        n = (deg + 1) ** 2
        for _ in range(10):
            v = rng.standard_normal(3) * rng.uniform(0.5, 3.0)
            d = v / np.linalg.norm(v)
            Y, G = orc.sh_basis_grad(deg, d)
            assert np.allclose(Y, orc.sh_basis(deg, d), atol=1e-15)
            h = 1e-6
            for j in range(3):
                e = np.zeros(3)
                e[j] = h
                fd = (orc.sh_basis(deg, d + e) - orc.sh_basis(deg, d - e)) / (2 * h)
                assert np.allclose(G[j], fd, atol=1e-8), (deg, j)
            # derivative of Y(v / |v|) with respect to v: (I - d d^T) grad / |v|
            T = (G - np.outer(d, d @ G)) / np.linalg.norm(v)
            hv = 1e-6 * np.linalg.norm(v)
            for j in range(3):
                e = np.zeros(3)
                e[j] = hv
                fd = (real_sh(v + e) - real_sh(v - e))[:n] / (2 * hv)
                assert np.allclose(T[j], fd, atol=1e-7), (deg, j)


def test_sh_matches_scipy(orc):
    """Real basis with the Condon-Shortley phase: Y_l0 = Re Y_l^0, Y_lm = sqrt2 Re Y_l^m and
    Y_l,-m = sqrt2 Im Y_l^m (m > 0), against scipy's complex spherical harmonics."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(9)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = orc.sh_basis(3, d)
        for l in range(4):
            for m in range(0, l + 1):
                if hasattr(sp, "sph_harm_y"):
                    c = sp.sph_harm_y(l, m, theta, phi)
                else:
                    c = sp.sph_harm(m, l, phi, theta)
                if m == 0:
                    assert abs(Y[l * l + l] - c.real) < 1e-12
                else:
                    assert abs(Y[l * l + l + m] - math.sqrt(2) * c.real) < 1e-12
                    assert abs(Y[l * l + l - m] - math.sqrt(2) * c.imag) < 1e-12


# ------------------------------------------------------------------ particle response

def _single_alpha(orc, mu, log_s, q, logit, cam, px, py, opts=None):
    sc = one_scene(mu, log_s, q, logit, [[0.5 * 2 * math.sqrt(math.pi)] * 3])
    proj = dict(rect=np.array([[0, 0, cam["width"] - 1, cam["height"] - 1]], np.int32),
                depth32=np.array([1.0], np.float32))
    out = orc.render(sc, cam, opts or synth.options(alpha_min=1e-300, t_min=0.0), proj=proj,
                     pixels=([px], [py]), no_rect=True)
    return out["alpha"][0]


def test_max_response_along_ray_matches_dense_scan(orc):
    """alpha / sigma equals max over tau of rho(o + tau d) (eq. GaussianMaxResponse), checked
    by a dense 1-D scan of eq. gaussian_kernel with Sigma^-1 built explicitly."""
    rng = np.random.default_rng(21)
    cam = synth.camera("pinhole", 32, 32, fx=30.0, fy=30.0)
    for _ in range(8):
        mu = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(2, 3)]).astype(np.float32)
        ls = rng.normal(-2.0, 0.3, 3).astype(np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        logit = np.float32(0.3)
        px, py = int(rng.integers(8, 24)), int(rng.integers(8, 24))
        a = _single_alpha(orc, mu, ls, q, logit, cam, px, py)
        sigma = 1 / (1 + math.exp(-float(logit)))
        R = rot(q.astype(float))
        Sinv = R @ np.diag(np.exp(-2 * ls.astype(float))) @ R.T
        d = np.array([(px + 0.5 - 16) / 30, (py + 0.5 - 16) / 30, 1.0])
        taus = np.linspace(0, 6, 200001)
        X = taus[:, None] * d[None, :] - mu.astype(float)[None, :]
        m2 = np.einsum("ni,ij,nj->n", X, Sinv, X)
        j = int(np.argmin(m2))
        # refine with the exact 1-D minimiser of the quadratic around the scan's best point
        tau_w = (mu.astype(float) @ Sinv @ d) / (d @ Sinv @ d)  # world-space form of eq. GaussianMaxResponse
        assert abs(tau_w - taus[j]) < 1e-4
        Xs = tau_w * d - mu.astype(float)
        rho = math.exp(-0.5 * Xs @ Sinv @ Xs)
        assert abs(a - sigma * rho) < 1e-12 * max(1.0, sigma * rho) + 1e-15
        assert sigma * math.exp(-0.5 * m2[j]) <= sigma * rho + 1e-15


def test_isotropic_response_closed_form(orc):
    """Isotropic Gaussian: omega = distance from mu to the ray / s."""
    cam = synth.camera("pinhole", 32, 32, fx=30.0, fy=30.0)
    mu = np.array([0.1, -0.05, 2.0], np.float32)
    s = 0.125
    ls = np.full(3, math.log(s), np.float32)
    for (px, py) in [(16, 16), (18, 15), (20, 11)]:
        a = _single_alpha(orc, mu, ls, [1, 0, 0, 0], 0.0, cam, px, py)
        d = np.array([(px + 0.5 - 16) / 30, (py + 0.5 - 16) / 30, 1.0])
        d /= np.linalg.norm(d)
        m = mu.astype(float)
        dist = np.linalg.norm(m - (m @ d) * d)
        s_true = math.exp(float(ls[0]))
        assert abs(a - 0.5 * math.exp(-0.5 * (dist / s_true) ** 2)) < 1e-12


# ------------------------------------------------------------------ compositing

def test_opaque_particle_gives_clamped_alpha(orc):
    cam = synth.camera("pinhole", 8, 8, fx=8.0, fy=8.0)
    c = np.array([0.2, 0.5, 0.9])
    beta = (c - 0.5) * 2 * math.sqrt(math.pi)
    sc = one_scene([0.0, 0.0, 2.0], [1.0, 1.0, 1.0], [1, 0, 0, 0], 12.0, [beta])
    proj = dict(rect=np.array([[0, 0, 7, 7]], np.int32), depth32=np.array([2.0], np.float32))
    op = synth.options()
    amax = op["alpha_max"]  # 0.99 as an FP32 number
    out = orc.render(sc, cam, op, proj=proj, pixels=([3, 4], [3, 4]))
    for q in range(2):
        assert np.allclose(out["rgb"][q], amax * np.float32(beta).astype(float) / (2 * math.sqrt(math.pi)) + amax * 0.5,
                           atol=1e-12)
        assert abs(out["alpha"][q] - amax) < 1e-15


def test_two_particles_quadrature_closed_form(orc):
    """c = c1 a1 + c2 a2 (1 - a1) (eq. QuadratureVolumeRendering) for two particles in depth order,
    with a1, a2 the single-particle alphas."""
    cam = synth.camera("pinhole", 16, 16, fx=16.0, fy=16.0)
    p1 = ([0.05, 0.0, 2.0], [-1.5, -1.8, -1.2], [0.9, 0.1, 0.2, -0.3], 0.4, [0.9, 0.1, 0.3])
    p2 = ([-0.05, 0.02, 2.6], [-1.3, -1.4, -1.6], [0.2, 0.8, -0.1, 0.4], -0.2, [0.2, 0.7, 0.5])
    cols = []
    alphas = []
    px, py = 8, 8
    for mu, ls, q, lg, col in (p1, p2):
        beta = (np.array(col) - 0.5) * 2 * math.sqrt(math.pi)
        sc = one_scene(mu, ls, q, lg, [beta])
        o = orc.render(sc, cam, synth.options(), pixels=([px], [py]), no_rect=True)
        alphas.append(o["alpha"][0])
        cols.append(np.float32(beta).astype(float) / (2 * math.sqrt(math.pi)) + 0.5)
    sc2 = {k: (np.concatenate([one_scene(*p1[:4], [(np.array(p1[4]) - .5) * 2 * math.sqrt(math.pi)])[k],
                               one_scene(*p2[:4], [(np.array(p2[4]) - .5) * 2 * math.sqrt(math.pi)])[k]])
               if k != "sh_degree" else 0) for k in ("means", "log_scales", "quats", "opacity_logits", "sh",
                                                      "sh_degree")}
    o = orc.render(sc2, cam, synth.options(), pixels=([px], [py]), no_rect=True)
    a1, a2 = alphas
    assert 1 / 255 < a1 < 0.99 and 1 / 255 < a2 < 0.99
    exp = cols[0] * a1 + cols[1] * a2 * (1 - a1)
    assert np.allclose(o["rgb"][0], exp, atol=1e-12)
    assert abs(o["alpha"][0] - (1 - (1 - a1) * (1 - a2))) < 1e-12


def test_transmittance_monotone_and_alpha_bounded(orc):
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    proj = orc.project(sc, cam, op)
    out = orc.render(sc, cam, op, proj=proj)
    assert np.all(out["alpha"] >= 0) and np.all(out["alpha"] <= 1)
    assert np.all(out["tfinal"] >= 0) and np.all(out["tfinal"] <= 1)
    assert np.all(out["tfinal"][out["nblend"] > 0] >= op["t_min"])
    # along one pixel's ordered list, the transmittance of every prefix is non-increasing
    keys, vals, ranges = orc.bin_keys(proj["depth32"], proj["rect"], 64, 64)
    t = 2 * 4 + 1
    lst = vals[ranges[t, 0]:ranges[t, 1]]
    px, py = 16 + 5, 32 + 7
    prev = 1.0
    for j in range(0, len(lst) + 1, max(1, len(lst) // 20)):
        _, tf = orc.render_list(sc, cam, op, proj["rect"], proj["depth32"], px, py, lst[:j])
        assert tf <= prev + 1e-15 and 0 <= tf <= 1
        prev = tf


# ------------------------------------------------------------------ tiling == brute force

def test_tile_lists_reproduce_brute_force(orc):
    """Compositing each pixel over its tile's sorted list gives bit-identical results to the
    brute-force render over all particles in global order (pixel predicate = centre in rect)."""
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    proj = orc.project(sc, cam, op)
    ref = orc.render(sc, cam, op, proj=proj)
    for tw, th in ((16, 16), (8, 8), (32, 8), (13, 7)):
        keys, vals, ranges = orc.bin_keys(proj["depth32"], proj["rect"], 64, 64, tw, th)
        txn = (64 + tw - 1) // tw
        for (px, py) in [(0, 0), (17, 33), (40, 12), (63, 63), (31, 31), (5, 60)]:
            t = (py // th) * txn + px // tw
            lst = vals[ranges[t, 0]:ranges[t, 1]]
            rgb, tf = orc.render_list(sc, cam, op, proj["rect"], proj["depth32"], px, py, lst)
            q = py * 64 + px
            assert np.array_equal(rgb, ref["rgb"][q]) and tf == ref["tfinal"][q]


def test_rect_culling_lossless_for_orthographic_camera(orc):
    """Orthographic camera: the UT is exact and the 2D Mahalanobis distance of a pixel equals the
    canonical distance omega along its ray, so with the extent cap lifted the opacity-tightened
    rectangle drops only particles with alpha < alpha_min: culled == unculled brute force."""
    sc = synth.scene_cube(300, 12, log_s=(-2.5, 0.4), deg=1, lo=(-1, -1, 1), hi=(1, 1, 3))
    cam = synth.camera("ortho", 48, 40, fx=20.0, fy=20.0, cx=24.0, cy=20.0)
    op = synth.options(extent_sigma=10.0, t_min=0.0)
    proj = orc.project(sc, cam, op)
    a = orc.render(sc, cam, op, proj=proj)
    b = orc.render(sc, cam, op, proj=proj, no_rect=True)
    assert np.max(np.abs(a["rgb"] - b["rgb"])) < 1e-12
    assert np.max(np.abs(a["alpha"] - b["alpha"])) < 1e-12
    # and with the default 3-sigma cap the loss is visible but small
    op3 = synth.options(t_min=0.0)
    c = orc.render(sc, cam, op3, proj=orc.project(sc, cam, op3))
    assert np.max(np.abs(c["rgb"] - b["rgb"])) < 0.05


# ------------------------------------------------------------------ integer stage

def _brute_bin(depth32, rect, W, H, tw, th):
    txn = (W + tw - 1) // tw
    items = []
    for i in range(len(rect)):
        x0, y0, x1, y1 = (int(v) for v in rect[i])
        if x0 > x1 or y0 > y1:
            continue
        for ty in range(y0 // th, y1 // th + 1):
            for tx in range(x0 // tw, x1 // tw + 1):
                key = ((ty * txn + tx) << 32) | int(np.float32(depth32[i]).view(np.uint32))
                items.append((key, len(items), i))
    items.sort()
    T = txn * ((H + th - 1) // th)
    ranges = np.zeros((T, 2), np.uint32)
    for j, (k, _, _) in enumerate(items):
        t = k >> 32
        if j == 0 or (items[j - 1][0] >> 32) != t:
            ranges[t, 0] = j
        ranges[t, 1] = j + 1
    return (np.array([k for k, _, _ in items], np.uint64), np.array([i for _, _, i in items], np.uint32), ranges)


@pytest.mark.parametrize("W,H,tw,th", [(64, 48, 16, 16), (70, 33, 16, 16), (37, 29, 8, 4), (100, 10, 32, 8)])
def test_bin_matches_brute_force(orc, W, H, tw, th):
    rect, depth = synth.random_rects(3, 200, W, H, max_w=30, max_h=20)
    k1, v1, r1 = orc.bin_keys(depth, rect, W, H, tw, th)
    k2, v2, r2 = _brute_bin(depth, rect, W, H, tw, th)
    assert np.array_equal(k1, k2) and np.array_equal(v1, v2) and np.array_equal(r1, r2)


def test_bin_edge_cases(orc):
    # empty input, all culled
    k, v, r = orc.bin_keys(np.zeros(0, np.float32), np.zeros((0, 4), np.int32), 32, 32)
    assert len(k) == 0 and not r.any()
    rect = np.array([[0, 0, -1, -1]] * 5, np.int32)
    k, v, r = orc.bin_keys(np.ones(5, np.float32), rect, 32, 32)
    assert len(k) == 0 and not r.any()


# ------------------------------------------------------------------ EWA projection (the A/B baseline)

def test_ewa_exact_for_affine_camera(orc):
    """For an affine camera the first-order (EWA) estimate is exact: A mu + b, A Sigma A^T."""
    rng = np.random.default_rng(12)
    Rc = axis_angle_rot([0.3, -1.0, 0.2], 0.7)
    cam = synth.camera("ortho", 100, 80, fx=37.0, fy=29.0, cx=41.0, cy=33.0, q=synth._rot_to_quat(Rc),
                       t=np.array([0.2, -0.1, 1.5]))
    Rc, tc = rot(cam["q_start"]), np.array(cam["t_start"])
    for _ in range(10):
        mu = rng.uniform(-1, 1, 3)
        R = rot(rng.standard_normal(4))
        s = np.exp(rng.normal(-1.5, 0.5, 3))
        ok, vmu, cov = orc.ewa_estimate(cam, mu, R, s)
        assert ok
        A = np.array([[37.0, 0, 0], [0, 29.0, 0]]) @ Rc
        C2 = A @ (R @ np.diag(s**2) @ R.T) @ A.T
        assert np.allclose(vmu, A @ mu + np.array([37.0 * tc[0] + 41.0, 29.0 * tc[1] + 33.0]), atol=1e-10)
        assert np.allclose(cov, [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("model,k", [("pinhole", (0, 0, 0, 0)), ("fisheye", (0, 0, 0, 0)),
                                     ("fisheye", (0.04, -0.03, 0.01, -0.005))])
def test_ewa_jacobian_matches_finite_differences(orc, model, k):
    """EWA covariance = J Sigma J^T with J = d g(W x) / d x at the mean, here taken by central
    differences of the oracle's own world-to-pixel map (an independent route to J), at points
    across the field of view including the optical axis."""
    rng = np.random.default_rng(13)
    q, t = synth.look_at_pose([0.3, -0.2, -3.0])
    cam = synth.camera(model, 640, 480, k=list(k), q=q, t=t) if model == "fisheye" else \
        synth.camera(model, 640, 480, fx=400.0, fy=380.0, q=q, t=t)
    Rc, tc = rot(cam["q_start"]), np.array(cam["t_start"])
    pts = [-Rc.T @ tc + Rc.T @ np.array([0.0, 0.0, 2.5])]  # on the optical axis
    while len(pts) < 12:
        d = Rc.T @ np.array([*rng.uniform(-0.9, 0.9, 2), 1.0])
        pts.append(-Rc.T @ tc + rng.uniform(1.5, 4.0) * d)
    for mu in pts:
        R = rot(rng.standard_normal(4))
        s = np.exp(rng.normal(-2.5, 0.4, 3))
        ok, vmu, cov = orc.ewa_estimate(cam, mu, R, s)
        assert ok
        h = 1e-6
        J = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            J[:, j] = (orc.project_point(cam, mu + e)[1] - orc.project_point(cam, mu - e)[1]) / (2 * h)
        C2 = J @ (R @ np.diag(s**2) @ R.T) @ J.T
        assert np.allclose(vmu, orc.project_point(cam, mu)[1], atol=1e-9)
        assert np.allclose(cov, [C2[0, 0], C2[0, 1], C2[1, 1]], rtol=1e-6, atol=1e-6 * np.abs(C2).max())


def test_ewa_and_ut_agree_to_first_order(orc):
    """Both estimates match the true moments to first order in the Gaussian's size, so their
    covariances agree as the scale shrinks: the relative gap falls like s^2 (halving s quarters it)."""
    cam = synth.camera("fisheye", 640, 480, k=[0.03, -0.02, 0.0, 0.0])
    mu = np.array([1.5, -0.8, 1.2])
    R = rot([0.9, 0.1, -0.3, 0.2])
    gaps = []
    for sc in (0.08, 0.04, 0.02):
        s = sc * np.array([1.0, 0.6, 0.3])
        _, _, cu = orc.ut_estimate(cam, mu, R, s)
        _, _, ce = orc.ewa_estimate(cam, mu, R, s)
        gaps.append(abs(cu[0] - ce[0]) / ce[0] + abs(cu[2] - ce[2]) / ce[2])
    assert gaps[0] > 1e-4
    assert 3.0 < gaps[0] / gaps[1] < 5.0 and 3.0 < gaps[1] / gaps[2] < 5.0, gaps


def test_ewa_projection_option(orc):
    """project() with projection = 1 reports the EWA moments."""
    sc = synth.scene_cube(50, 14, deg=0)
    cam = synth.camera("fisheye", 320, 240, k=[0.02, 0.0, 0.0, 0.0])
    pe = orc.project(sc, cam, synth.options(projection=1))
    i = int(np.argmax(pe["ntiles"]))
    ok, vmu, cov = orc.ewa_estimate(cam, sc["means"][i].astype(float), rot(sc["quats"][i].astype(float)),
                                    np.exp(sc["log_scales"][i].astype(float)))
    assert ok and np.allclose(pe["mean2d"][i], vmu) and np.allclose(pe["cov2d"][i], cov)


# ------------------------------------------------------------------ radial pinhole camera

def test_radial_pinhole_without_distortion_is_the_pinhole(orc):
    """k = 0: the radial model is the plain pinhole (projection, rays and the rendered image)."""
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    camr = dict(cam, model="pinhole_radial")
    a = orc.render(sc, cam, op, proj=orc.project(sc, cam, op))
    pr = orc.project(sc, camr, op)
    assert np.array_equal(pr["rect"], orc.project(sc, cam, op)["rect"])
    b = orc.render(sc, camr, op, proj=pr)
    assert np.max(np.abs(a["rgb"] - b["rgb"])) < 1e-12


def test_radial_field_limit_closed_form(orc):
    """With k2 = k3 = 0 and k1 < 0, r_d = r (1 + k1 r^2) turns over at r = 1 / sqrt(-3 k1): points
    beyond that radius are not imaged, points inside are, and the image edge is r_d(r_max)."""
    k1 = -0.2
    rmax = 1.0 / math.sqrt(-3.0 * k1)
    cam = synth.camera("pinhole_radial", 640, 480, fx=200.0, k=[k1, 0, 0, 0])
    for r, ok_expected in ((0.97 * rmax, True), (1.03 * rmax, False)):
        x = np.array([r * 3.0, 0.0, 3.0])
        assert orc.project_point(cam, x)[0] == ok_expected
    rd_max = rmax * (1 + k1 * rmax**2)
    cx = np.float32(320.0)
    assert orc.pixel_ray(cam, float(cx) + 200.0 * rd_max * 0.999, 240.0)[0]
    assert not orc.pixel_ray(cam, float(cx) + 200.0 * rd_max * 1.001, 240.0)[0]


# ------------------------------------------------------------------ generalised kernels (degree n)

@pytest.mark.parametrize("n", [3, 4, 5, 8])
def test_generalised_kernel_max_response_matches_dense_scan(orc, n):
    """Degree-n kernel rho = exp(-lambda d^n), lambda = 3^(2-n) / 2 (equal to the Gaussian's
    response at d = 3): the maximum along a pixel ray from a dense 1-D scan of rho(x) equals the
    oracle's alpha / sigma, and the response is monotone in d so the argmax is the Gaussian's."""
    rng = np.random.default_rng(22 + n)
    cam = synth.camera("pinhole", 32, 32, fx=30.0, fy=30.0)
    lam = 0.5 * 3.0 ** (2 - n)
    for _ in range(6):
        mu = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(2, 3)]).astype(np.float32)
        ls = rng.normal(-2.0, 0.3, 3).astype(np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        logit = np.float32(0.3)
        px, py = int(rng.integers(8, 24)), int(rng.integers(8, 24))
        sc = one_scene(mu, ls, q, logit, [[0.1, 0.2, 0.3]])
        out = orc.render(sc, cam, synth.options(t_min=0.0, alpha_min=1e-30, kernel_degree=n),
                         proj=dict(rect=np.array([[0, 0, 31, 31]], np.int32), depth32=np.array([2.0], np.float32)),
                         pixels=([px], [py]), no_rect=True)
        a = out["alpha"][0]
        sigma = 1 / (1 + math.exp(-float(logit)))
        R = rot(q.astype(float))
        Sinv = R @ np.diag(np.exp(-2 * ls.astype(float))) @ R.T
        d = np.array([(px + 0.5 - 16) / 30, (py + 0.5 - 16) / 30, 1.0])
        taus = np.linspace(0, 6, 200001)
        X = taus[:, None] * d[None, :] - mu.astype(float)[None, :]
        rho = np.exp(-lam * np.einsum("ni,ij,nj->n", X, Sinv, X) ** (n / 2))
        assert abs(a - sigma * rho.max()) < 1e-6 * max(sigma * rho.max(), 1e-12) + 1e-14
    # the response at Mahalanobis distance 3 is the Gaussian's
    assert abs(math.exp(-lam * 3.0**n) - math.exp(-0.5 * 9.0)) < 1e-15


def test_generalised_kernel_degree_two_is_the_gaussian(orc):
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    a = orc.render(sc, cam, op, proj=orc.project(sc, cam, op))
    op2 = dict(op, kernel_degree=2)
    b = orc.render(sc, cam, op2, proj=orc.project(sc, cam, op2))
    assert np.array_equal(a["rgb"], b["rgb"])
    op4 = dict(op, kernel_degree=4)
    c = orc.render(sc, cam, op4, proj=orc.project(sc, cam, op4))
    assert np.abs(c["rgb"] - a["rgb"]).max() > 1e-3


@pytest.mark.parametrize("n", [2, 4])
def test_rect_culling_lossless_for_generalised_kernels(orc, n):
    """Orthographic camera, cap lifted: the degree-n extent (2 ln(sigma/alpha_min) 3^(n-2))^(1/n)
    drops only particles below alpha_min, so culled == unculled brute force."""
    sc = synth.scene_cube(300, 12, log_s=(-2.5, 0.4), deg=1, lo=(-1, -1, 1), hi=(1, 1, 3))
    cam = synth.camera("ortho", 48, 40, fx=20.0, fy=20.0, cx=24.0, cy=20.0)
    op = synth.options(extent_sigma=10.0, t_min=0.0, kernel_degree=n)
    proj = orc.project(sc, cam, op)
    a = orc.render(sc, cam, op, proj=proj)
    b = orc.render(sc, cam, op, proj=proj, no_rect=True)
    assert np.max(np.abs(a["rgb"] - b["rgb"])) < 1e-12


# ------------------------------------------------------------------ "Ours (sorted)": per-ray k-buffer

@pytest.mark.parametrize("k", [1, 4, 16])
def test_kbuffer_bound_covers_the_other_order_of_exact_ties(orc, k):
    """Pairs of particles with identical geometry (their tau_max ties exactly at every pixel)
    and different opacities and colours: swapping each pair's indices swaps their arrival and so
    the order the tie-break blends them in.  Wherever the two images differ the pixel carries a
    tie flag, and the difference lies within the oracle's k-buffer bound (slack, aslack) of
    either render."""
    n_pairs = 60
    a = synth.scene_cube(n_pairs, 31, deg=1, log_s=(-2.6, 0.3))
    b = synth.scene_cube(n_pairs, 32, deg=1, log_s=(-2.6, 0.3))
    sc = {}
    for key in ("means", "log_scales", "quats"):
        sc[key] = np.repeat(a[key], 2, axis=0)
    for key in ("opacity_logits", "sh"):
        sc[key] = np.stack([a[key], b[key]], axis=1).reshape((2 * n_pairs,) + a[key].shape[1:])
    sc["opacity_logits"] = sc["opacity_logits"] + 1.0
    sc["sh_degree"] = 1
    sw = {key: (v.reshape((n_pairs, 2) + v.shape[1:])[:, ::-1].reshape(v.shape) if key != "sh_degree" else v)
          for key, v in sc.items()}
    cam = synth.camera("pinhole", 48, 40, fx=40.0)
    op = synth.options(kbuffer=k)
    tol = dict(eps_px=5e-3, eps_rel=2e-4, eps_t=2e-3, depth_ulps=4, cond_min=0.05)
    r1 = orc.render(sc, cam, op, proj=orc.project(sc, cam, op, tol), tol=tol)
    r2 = orc.render(sw, cam, op, proj=orc.project(sw, cam, op, tol), tol=tol)
    drgb = np.abs(r1["rgb"] - r2["rgb"]).max(axis=1)
    da = np.abs(r1["alpha"] - r2["alpha"])
    differ = (drgb > 1e-12) | (da > 1e-12)
    assert differ.sum() > 20  # the order matters at many pixels
    tied = (r1["flags"] & orc.F_DEPTH_TIE) != 0
    assert np.all(tied[differ])
    for r in (r1, r2):
        assert np.all(drgb <= r["slack"] * (1 + 1e-12) + 1e-12)
        assert np.all(da <= r["aslack"] * (1 + 1e-12) + 1e-12)
    # the bound is not vacuous: it is below the largest colour at most of the tied pixels
    assert np.median(r1["slack"][tied]) < 1.0


def _two_crossing():
    """Two isotropic Gaussians where the mean nearer the camera is reached later along one pixel's
    ray: A sits on the ray at tau = 3.0 (0.05 off it), B at tau = 2.6 but 1.6 off the ray, so
    |mu_B| > |mu_A| while B's maximum along the ray comes first."""
    # pinhole 32x32, f = 30: pixel (20, 16) has ray d = (4.5/30, 0.5/30, 1) from the origin
    d = np.array([4.5 / 30, 0.5 / 30, 1.0])
    u = np.cross(d, [1.0, 0.0, 0.0])
    u /= np.linalg.norm(u)
    mu_a = 3.0 * d + 0.05 * u
    mu_b = 2.6 * d - 1.6 * u
    sc = dict(means=np.array([mu_a, mu_b], np.float32),
              log_scales=np.array([[-0.5, -0.5, -0.5], [0.2, 0.2, 0.2]], np.float32),
              quats=np.array([[1, 0, 0, 0], [1, 0, 0, 0]], np.float32),
              opacity_logits=np.array([0.4, 1.5], np.float32),
              sh=np.array([[[0.8, -0.3, 0.1]], [[-0.4, 0.6, 0.2]]], np.float32), sh_degree=0)
    return sc


def test_kbuffer_composites_in_tau_order():
    """k >= the number of hits: the k-buffer blends in ascending tau_max, which here is the
    reverse of the global depth order; the result equals the two-particle quadrature
    c_1 a_1 + c_2 a_2 (1 - a_1) in tau order, with each a_i taken from a render of particle i
    alone (an independent route to alpha)."""
    import oracle as orc
    sc = _two_crossing()
    cam = synth.camera("pinhole", 32, 32, fx=30.0, fy=30.0)
    proj = dict(rect=np.array([[0, 0, 31, 31]] * 2, np.int32),
                depth32=np.linalg.norm(sc["means"].astype(np.float64), axis=1).astype(np.float32))
    assert proj["depth32"][0] < proj["depth32"][1]  # A first in depth order
    px, py = 20, 16
    op = synth.options(t_min=0.0, kbuffer=16)
    single = []
    for i in (0, 1):
        s1 = {k: (v[i:i + 1] if k != "sh_degree" else v) for k, v in sc.items()}
        p1 = dict(rect=proj["rect"][i:i + 1], depth32=proj["depth32"][i:i + 1])
        o = orc.render(s1, cam, synth.options(t_min=0.0), proj=p1, pixels=([px], [py]))
        single.append((o["alpha"][0], o["rgb"][0] / o["alpha"][0]))
    (a_a, c_a), (a_b, c_b) = single
    assert a_a > 0.05 and a_b > 0.05
    tau_first_is_b = c_b * a_b + c_a * a_a * (1 - a_b)
    depth_first_is_a = c_a * a_a + c_b * a_b * (1 - a_a)
    assert np.abs(tau_first_is_b - depth_first_is_a).max() > 1e-3  # the orders differ visibly
    kb = orc.render(sc, cam, op, proj=proj, pixels=([px], [py]))
    tile = orc.render(sc, cam, synth.options(t_min=0.0), proj=proj, pixels=([px], [py]))
    assert np.allclose(kb["rgb"][0], tau_first_is_b, atol=1e-12)
    assert np.allclose(tile["rgb"][0], depth_first_is_a, atol=1e-12)
    # k = 1: the two hits compete in the buffer and the closer in tau is blended first as well
    kb1 = orc.render(sc, cam, synth.options(t_min=0.0, kbuffer=1), proj=proj, pixels=([px], [py]))
    assert np.allclose(kb1["rgb"][0], tau_first_is_b, atol=1e-12)


def test_kbuffer_equals_tile_order_when_depth_and_tau_orders_agree():
    """Small, well separated particles along the rays: tau_max order = depth order, so the
    k-buffer image is the tile-order image (any k)."""
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    sc = dict(sc, log_scales=np.full_like(sc["log_scales"], -5.0))
    import oracle as orc
    proj = orc.project(sc, cam, op)
    a = orc.render(sc, cam, op, proj=proj)
    for k in (1, 4, 16):
        b = orc.render(sc, cam, dict(op, kbuffer=k), proj=proj)
        ok = (b["flags"] & orc.F_DEPTH_TIE) == 0
        assert np.max(np.abs(a["rgb"][ok] - b["rgb"][ok])) < 1e-12, k


def test_kbuffer_transmittance_and_alpha_bounds():
    import oracle as orc
    case = synth.fisheye_shell(n=3000, width=96, height=64)
    sc, cam, op = case["scene"], case["camera"], dict(case["options"], kbuffer=16)
    o = orc.render(sc, cam, op, proj=orc.project(sc, cam, op))
    assert np.all(o["alpha"] >= 0) and np.all(o["alpha"] <= 1) and np.all(o["tfinal"] >= 0)
    assert np.all(o["rgb"] >= 0)


# ------------------------------------------------------------------ per-particle colour (colour_mode 1)

def test_per_particle_colour_equals_per_pixel_for_degree_zero(orc):
    """Degree-0 SH does not depend on the direction: both colour modes render the same image."""
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    a = orc.render(sc, cam, op, proj=orc.project(sc, cam, op))
    op1 = dict(op, colour_mode=1)
    b = orc.render(sc, cam, op1, proj=orc.project(sc, cam, op1))
    assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["alpha"], b["alpha"])


def test_per_particle_colour_at_the_pixel_through_the_mean(orc):
    """A particle whose mean lies on a pixel's ray has, at that pixel, the same view direction
    in both colour modes, so the two renders agree there (degree 3)."""
    cam = synth.camera("pinhole", 32, 32, fx=40.0, fy=40.0)
    px, py = 20, 11
    _, o, d = orc.pixel_ray(cam, px + 0.5, py + 0.5)
    rng = np.random.default_rng(15)
    mu = np.asarray(o) + 2.5 * np.asarray(d) / np.linalg.norm(d)
    sh = rng.normal(0, 0.3, (16, 3))
    sc = one_scene(mu, [-2.0, -2.2, -1.8], [0.9, 0.1, 0.2, -0.3], 1.0, sh, deg=3)
    proj = dict(rect=np.array([[0, 0, 31, 31]], np.int32), depth32=np.array([2.5], np.float32))
    a = orc.render(sc, cam, synth.options(), proj=proj, pixels=([px], [py]))
    b = orc.render(sc, cam, synth.options(colour_mode=1), proj=proj, pixels=([px], [py]))
    assert a["alpha"][0] > 0.1
    assert np.allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-6)
    # elsewhere the modes differ (the direction changes across the footprint)
    a2 = orc.render(sc, cam, synth.options(), proj=proj, pixels=([px + 3], [py - 2]))
    b2 = orc.render(sc, cam, synth.options(colour_mode=1), proj=proj, pixels=([px + 3], [py - 2]))
    assert np.abs(a2["rgb"] - b2["rgb"]).max() > 1e-5


# ------------------------------------------------------------------ gradients

def _fd_scene(n=12, deg=1, seed=31):
    sc = synth.scene_cube(n, seed, log_s=(-2.2, 0.3), deg=deg, lo=(-0.4, -0.4, 2.0), hi=(0.4, 0.4, 3.0))
    # exact FP32 perturbations: every base value is a multiple of 2^-12 well inside float32 range
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        sc[k] = (np.round(sc[k].astype(np.float64) * 4096) / 4096).astype(np.float32)
    return sc


def _loss(orc, sc, cam, op, proj, pix, g_rgb, g_a):
    o = orc.render(sc, cam, op, proj=proj, pixels=pix)
    return float(np.sum(o["rgb"] * g_rgb) + np.sum(o["alpha"] * g_a))


@pytest.mark.parametrize("colour_mode,deg,kdeg", [(0, 1, 2), (1, 2, 2), (0, 1, 4), (0, 0, 4)])
def test_gradients_match_central_differences(orc, colour_mode, deg, kdeg):
    """FP64 analytic gradients vs Richardson-extrapolated central differences (steps 2^-9, 2^-10,
    exact in FP32) with the culling decisions held fixed (they carry no gradient, Sec. 4.1).
    colour_mode 1 includes the mean's gradient through the per-particle view direction."""
    sc = _fd_scene(deg=deg)
    cam = synth.camera("pinhole", 24, 20, fx=30.0, fy=30.0, cx=12.0, cy=10.0)
    op = synth.options(t_min=1e-4, colour_mode=colour_mode, kernel_degree=kdeg)
    proj = orc.project(sc, cam, op)
    yy, xx = np.mgrid[0:20, 0:24]
    px, py = xx.reshape(-1), yy.reshape(-1)
    fl = orc.render(sc, cam, op, proj=proj, tol=dict(eps_rel=0.1, eps_px=0.0), pixels=(px, py))["flags"]
    keep = (fl & (orc.F_ALPHA_MIN | orc.F_TSTOP | orc.F_ALPHA_MAX)) == 0
    rng = np.random.default_rng(0)
    g_rgb = rng.standard_normal((len(px), 3)) * keep[:, None]
    g_a = rng.standard_normal(len(px)) * keep
    pix = (px, py)
    gr = orc.backward(sc, cam, op, proj, pix, g_rgb, g_a)
    checked = 0
    for name, arr in (("means", "means"), ("log_scales", "log_scales"), ("quats", "quats"),
                      ("opacity_logits", "opacity_logits"), ("sh", "sh")):
        base = sc[arr]
        flat = base.reshape(-1)
        ga = gr[name].reshape(-1)
        for j in range(flat.size):
            def f(h):
                s2 = dict(sc)
                b2 = base.copy().reshape(-1)
                b2[j] = np.float32(float(flat[j]) + h)
                assert float(b2[j]) == float(flat[j]) + h
                s2[arr] = b2.reshape(base.shape)
                return _loss(orc, s2, cam, op, proj, pix, g_rgb, g_a)
            h = 2.0**-9
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            fd = (4 * d2 - d1) / 3
            assert abs(fd - ga[j]) <= 1e-6 * max(1.0, abs(ga[j])) + 1e-7, (name, j, fd, ga[j])
            checked += 1
    assert checked >= 12 * 14  # every parameter of the 12 particles (SH degree >= 0)


@pytest.mark.parametrize("k", [2, 16])
def test_kbuffer_gradients_match_central_differences(orc, k):
    """The k-buffer ("Ours (sorted)") backward: analytic gradients over each pixel's blended pairs
    in the buffer's blending order vs Richardson central differences (exact FP32 steps).  The
    selection by tau_max is piecewise constant; pixels where a selection is within 2 % of a tie
    (it could flip under the steps), near alpha_min / alpha_max or near the stop are left out."""
    sc = _fd_scene(deg=1)
    cam = synth.camera("pinhole", 24, 20, fx=30.0, fy=30.0, cx=12.0, cy=10.0)
    op = synth.options(t_min=1e-4, kbuffer=k)
    proj = orc.project(sc, cam, op)
    yy, xx = np.mgrid[0:20, 0:24]
    px, py = xx.reshape(-1), yy.reshape(-1)
    fl = orc.render(sc, cam, dict(op, eps_tau=0.02), proj=proj, tol=dict(eps_rel=0.1, eps_px=0.0),
                    pixels=(px, py))["flags"]
    keep = (fl & (orc.F_ALPHA_MIN | orc.F_TSTOP | orc.F_ALPHA_MAX | orc.F_DEPTH_TIE)) == 0
    assert keep.mean() > 0.5
    rng = np.random.default_rng(1)
    g_rgb = rng.standard_normal((len(px), 3)) * keep[:, None]
    g_a = rng.standard_normal(len(px)) * keep
    pix = (px, py)
    gr = orc.backward(sc, cam, op, proj, pix, g_rgb, g_a)
    checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        base = sc[name]
        flat = base.reshape(-1)
        ga = gr[name].reshape(-1)
        for j in range(flat.size):
            def f(h):
                b2 = base.copy().reshape(-1)
                b2[j] = np.float32(float(flat[j]) + h)
                assert float(b2[j]) == float(flat[j]) + h
                return _loss(orc, dict(sc, **{name: b2.reshape(base.shape)}), cam, op, proj, pix, g_rgb, g_a)
            h = 2.0**-9
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            fd = (4 * d2 - d1) / 3
            assert abs(fd - ga[j]) <= 1e-6 * max(1.0, abs(ga[j])) + 1e-7, (name, j, fd, ga[j])
            checked += 1
    assert checked >= 12 * 14


def test_kbuffer_gradients_equal_tile_order_when_the_orders_agree(orc):
    """Small, well separated particles along the rays: tau_max order = depth order, so the
    k-buffer blends the tile order and its gradients are the tile-order gradients (any k)."""
    case = synth.small_pinhole()
    sc, cam, op = case["scene"], case["camera"], case["options"]
    sc = dict(sc, log_scales=np.full_like(sc["log_scales"], -5.0))
    proj = orc.project(sc, cam, op)
    H, W = cam["height"], cam["width"]
    yy, xx = np.mgrid[0:H, 0:W]
    pix = (xx.reshape(-1), yy.reshape(-1))
    rng = np.random.default_rng(2)
    g_rgb, g_a = rng.standard_normal((H * W, 3)), rng.standard_normal(H * W)
    ref = orc.backward(sc, cam, op, proj, pix, g_rgb, g_a)
    for k in (1, 16):
        opk = dict(op, kbuffer=k)
        assert not np.any(orc.render(sc, cam, opk, proj=proj)["flags"] & orc.F_DEPTH_TIE)
        got = orc.backward(sc, cam, opk, proj, pix, g_rgb, g_a)
        for name in ref:
            assert np.allclose(got[name], ref[name], rtol=1e-12, atol=1e-12 * np.abs(ref[name]).max()), (k, name)


@pytest.mark.parametrize("n", [3, 5])
def test_odd_degree_kernel_gradient_single_particle(orc, n):
    """Odd degrees are not twice differentiable where a ray crosses a particle's centre, so the
    scene-wide difference check above uses even degrees; here one particle and a pixel whose
    ray passes well off its centre: analytic dL/dmu, dL/dlog_s, dL/dq vs Richardson central
    differences (exact FP32 steps)."""
    cam = synth.camera("pinhole", 16, 16, fx=16.0, fy=16.0)
    base = dict(means=np.array([[0.0625, -0.03125, 2.0]], np.float32),
                log_scales=np.array([[-1.625, -1.875, -1.25]], np.float32),
                quats=np.array([[0.8125, 0.1875, -0.3125, 0.40625]], np.float32),
                opacity_logits=np.array([0.75], np.float32),
                sh=np.array([[[0.125, 0.25, 0.375]]], np.float32), sh_degree=0)
    proj = dict(rect=np.array([[0, 0, 15, 15]], np.int32), depth32=np.array([2.0], np.float32))
    op = synth.options(t_min=0.0, kernel_degree=n)
    px, py = 10, 6
    gr = orc.backward(base, cam, op, proj, ([px], [py]), np.ones((1, 3)), np.ones(1))
    for key in ("means", "log_scales", "quats"):
        flat = base[key].reshape(-1)
        for j in range(flat.size):
            def f(h):
                s2 = dict(base)
                b2 = flat.copy()
                b2[j] = np.float32(float(flat[j]) + h)
                s2[key] = b2.reshape(base[key].shape)
                o = orc.render(s2, cam, op, proj=proj, pixels=([px], [py]))
                return float(o["rgb"].sum() + o["alpha"].sum())
            h = 2.0**-10
            d1 = (f(h) - f(-h)) / (2 * h)
            d2 = (f(h / 2) - f(-h / 2)) / h
            fd = (4 * d2 - d1) / 3
            ga = gr[key].reshape(-1)[j]
            assert abs(fd - ga) <= 1e-5 * max(1.0, abs(ga)), (key, j, fd, ga)


def test_dalpha_dmu_matches_printed_chain(orc):
    """d alpha / d mu = (-1/2 sigma e^{-omega^2/2}) (2 o_g + 2 tau d_g)^T (-S^-1 R^T), the chain the
    supplementary prints (Sec. B), for one particle and one pixel with loss = alpha."""
    cam = synth.camera("pinhole", 16, 16, fx=16.0, fy=16.0)
    mu = np.array([0.03, -0.02, 2.0], np.float32)
    ls = np.array([-1.6, -1.9, -1.3], np.float32)
    q = np.array([0.8, 0.2, -0.3, 0.4], np.float32)
    logit = np.float32(0.7)
    sc = one_scene(mu, ls, q, logit, [[0.1, 0.2, 0.3]])
    proj = dict(rect=np.array([[0, 0, 15, 15]], np.int32), depth32=np.array([2.0], np.float32))
    px, py = 9, 7
    gr = orc.backward(sc, cam, synth.options(t_min=0.0), proj, ([px], [py]), np.zeros((1, 3)), np.ones(1))
    R = rot(q.astype(float))
    S_inv = np.diag(np.exp(-ls.astype(float)))
    M = S_inv @ R.T
    o = np.zeros(3)
    d = np.array([(px + 0.5 - 8) / 16, (py + 0.5 - 8) / 16, 1.0])
    og = M @ (o - mu.astype(float))
    dg = M @ d
    dgn = dg / np.linalg.norm(dg)
    tau_g = -og @ dgn
    w2 = np.sum((og + tau_g * dgn) ** 2)
    sigma = 1 / (1 + math.exp(-float(logit)))
    dalpha_dw2 = -0.5 * sigma * math.exp(-0.5 * w2)
    dw2_dog = 2 * og + 2 * tau_g * dgn
    dog_dmu = -M
    expect = dalpha_dw2 * dw2_dog @ dog_dmu
    assert np.allclose(gr["means"][0], expect, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ error-scale outputs of the oracle

def test_gradient_magnitudes_bound_the_gradients(orc):
    """The backward's magnitudes (the computation evaluated on absolute values) bound every
    gradient element (triangle inequality), and where a single term remains -- one particle, one
    pixel, an opacity-only loss for the logit, a colour-only loss for the SH coefficients -- they
    equal the absolute gradients."""
    sc = _fd_scene(deg=1)
    cam = synth.camera("pinhole", 24, 20, fx=30.0, fy=30.0, cx=12.0, cy=10.0)
    op = synth.options()
    proj = orc.project(sc, cam, op)
    yy, xx = np.mgrid[0:20, 0:24]
    pix = (xx.reshape(-1), yy.reshape(-1))
    rng = np.random.default_rng(3)
    g_rgb = rng.standard_normal((pix[0].size, 3))
    g_a = rng.standard_normal(pix[0].size)
    gr = orc.backward(sc, cam, op, proj, pix, g_rgb, g_a, magnitudes=True)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert np.all(gr["mag"][k] >= np.abs(gr[k]) * (1 - 1e-12) - 1e-300), k
        assert np.any(gr["mag"][k] > 1.5 * np.abs(gr[k])), k  # cancellation happens somewhere
    one = one_scene([0.05, -0.02, 3.0], [-1.2, -1.5, -1.4], [0.9, 0.2, -0.3, 0.1], 0.3,
                    [[0.3, -0.2, 0.1], [0.1, 0.05, -0.1], [0.02, -0.03, 0.04], [-0.05, 0.01, 0.02]], deg=1)
    p1 = orc.project(one, cam, op)
    px, py = np.array([12]), np.array([10])
    g1 = orc.backward(one, cam, op, p1, (px, py), np.zeros((1, 3)), np.array([0.3]), magnitudes=True)
    assert g1["opacity_logits"][0] != 0
    assert abs(g1["mag"]["opacity_logits"][0] - abs(g1["opacity_logits"][0])) < 1e-15 * abs(g1["opacity_logits"][0])
    g2 = orc.backward(one, cam, op, p1, (px, py), np.array([[0.7, -0.4, 0.2]]), np.zeros(1), magnitudes=True)
    assert np.abs(g2["sh"]).max() > 0
    assert np.allclose(g2["mag"]["sh"], np.abs(g2["sh"]), rtol=1e-15, atol=0)
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        assert np.all(g2["mag"][k] >= np.abs(g2[k]) * (1 - 1e-12)), k


def test_flip_bound_covers_an_alpha_min_decision(orc):
    """Where a particle's sigma rho sits at alpha_min, rendering with alpha_min just above and just
    below it includes and excludes the particle: the colour and opacity change between the two
    must stay within the flip bounds (fslack / faslack) the oracle reports for that pixel."""
    sc = _fd_scene(deg=1)
    cam = synth.camera("pinhole", 24, 20, fx=30.0, fy=30.0, cx=12.0, cy=10.0)
    op = synth.options()
    proj = orc.project(sc, cam, op)
    yy, xx = np.mgrid[0:20, 0:24]
    px, py = xx.reshape(-1), yy.reshape(-1)
    checked = 0
    for j in range(sc["means"].shape[0]):
        single = {k: (v[j:j + 1] if k != "sh_degree" else v) for k, v in sc.items()}
        pj = dict(rect=proj["rect"][j:j + 1], depth32=proj["depth32"][j:j + 1])
        a1 = orc.render(single, cam, op, proj=pj, pixels=(px, py), tol=dict(eps_px=0.0))["alpha"]
        q = int(np.argmax(np.where(a1 < 0.5, a1, 0)))  # a pixel where it is partly transparent
        a = a1[q]
        if not (0.01 < a < 0.5):
            continue
        renders = []
        for amin in (a * (1 - 1e-6), a * (1 + 1e-6)):
            o2 = dict(op, alpha_min=float(amin))
            renders.append(orc.render(sc, cam, o2, proj=proj, pixels=(px[q:q + 1], py[q:q + 1]),
                                      tol=dict(eps_px=0.0, eps_rel=1e-4)))
        dc = np.abs(renders[0]["rgb"] - renders[1]["rgb"]).max()
        da = abs(renders[0]["alpha"][0] - renders[1]["alpha"][0])
        assert renders[0]["flags"][0] & orc.F_ALPHA_MIN and renders[1]["flags"][0] & orc.F_ALPHA_MIN
        assert dc > 1e-4  # the decision matters
        for r in renders:
            assert dc <= r["fslack"][0] + r["slack"][0] + 1e-12, (dc, r["fslack"][0])
            assert da <= r["faslack"][0] + r["aslack"][0] + 1e-12, (da, r["faslack"][0])
            assert r["fslack"][0] < 20 * dc + 4e-4  # and the bound is not vacuous
        checked += 1
    assert checked >= 4


def test_colour_clamp_flag(orc):
    """A colour channel whose SH sum sits at 0 (where the clamp max(., 0) switches) is flagged at
    every pixel that blends the particle; 0.1 away from it, it is not."""
    C0 = 0.28209479177387814
    for off, want in ((0.0, True), (0.1, False)):
        one = one_scene([0.0, 0.0, 3.0], [-1.0, -1.0, -1.0], [1.0, 0.0, 0.0, 0.0], 2.0,
                        [[(-0.5 + off) / C0, 0.3, 0.2]], deg=0)
        cam = synth.camera("pinhole", 16, 16, fx=20.0, fy=20.0)
        r = orc.render(one, cam, synth.options(), tol=dict(eps_rel=1e-4))
        hit = r["nblend"] > 0
        assert hit.sum() > 20
        got = (r["flags"] & orc.F_CLAMP) != 0
        assert np.all(got[hit] == want) and not got[~hit].any()


def test_alpha_rounding_bound_covers_an_fp32_evaluation(orc):
    """The oracle's FP32 rounding bound of a blended particle's alpha (raslack of a one-particle
    render) covers the alpha an FP32 evaluation of eq. GaussianMaxResponse gives (canonical ray
    o_g = M (o - mu), d_g = M d, omega^2 = |o_g x d_g|^2 / |d_g|^2, all in numpy float32) for tiny
    particles far from the camera, where the evaluation is worst conditioned -- and stays within a
    small factor of the largest deviation seen."""
    f32 = np.float32
    rng = np.random.default_rng(23)
    cam = synth.camera("pinhole", 64, 64, fx=3000.0, fy=3000.0, t=(0.3, -0.2, 0.5))
    op = synth.options()
    worst_ratio, worst_dev = 0.0, 0.0
    for _ in range(40):
        mu = np.array([-0.3 + rng.uniform(-0.004, 0.004), 0.2 + rng.uniform(-0.004, 0.004), rng.uniform(7.0, 9.0)])
        ls = rng.normal(-6.0, 0.3, 3)
        q = rng.standard_normal(4)
        sc = one_scene(mu, ls, q, 3.0, [[0.3, 0.3, 0.3]], deg=0)
        okp, uv, _ = orc.project_point(cam, sc["means"][0].astype(np.float64))
        px, py = int(uv[0]), int(uv[1])
        if not (okp and 0 <= px < 64 and 0 <= py < 64):
            continue
        r = orc.render(sc, cam, op, pixels=(np.array([px]), np.array([py])))
        if r["nblend"][0] != 1 or r["alpha"][0] > 0.98:
            continue
        ok, o, d = orc.pixel_ray(cam, px + 0.5, py + 0.5)
        m32 = sc["means"][0].astype(f32)
        s32 = np.exp(sc["log_scales"][0].astype(f32))
        qq = sc["quats"][0].astype(np.float64)
        R = rot(qq).astype(f32)
        M = (R.T / s32[:, None]).astype(f32)  # S^-1 R^T
        og = M @ (o.astype(f32) - m32)
        dg = M @ d.astype(f32)
        c = np.cross(og, dg).astype(f32)
        w2 = f32(np.dot(c, c) / np.dot(dg, dg))
        sig = f32(1.0 / (1.0 + np.exp(-f32(3.0))))
        a32 = float(sig * np.exp(-f32(0.5) * w2))
        dev = abs(a32 - r["alpha"][0])
        bound = r["raslack"][0]
        assert dev <= bound, (dev, bound)
        worst_dev = max(worst_dev, dev)
        worst_ratio = max(worst_ratio, dev / bound)
    assert worst_dev > 1e-6          # the case is ill-conditioned enough to matter
    assert worst_ratio > 0.05        # and the bound is within 20x of the worst deviation
