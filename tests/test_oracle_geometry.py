"""Pins of the oracle's forward geometry and of its optimiser steps against
sources that share nothing with it:

* Eq. 1 (Sigma = R(q) S S^T R(q)^T): the quaternion's rotation is scipy's
  ``Rotation.from_quat`` (scalar-last order), the covariance is built here
  from that matrix;
* Eq. 2 (Sigma_hat = [J W Sigma W^T J^T]_2x2 + 0.3 I): J is the complex-step
  derivative of the pinhole map pi(x, y, z) = (fx x/z + cx, fy y/z + cy)
  at off-axis camera-space means (exact to rounding, no formula for J is
  typed in);
* the 3-sigma screen bound and the tile rectangle: radii and tile sets worked
  out by hand for Gaussians on the optical axis, with the rectangle's ends on
  tile boundaries and at the grid's edges;
* the SH view direction d = (mu - o_c) / |mu - o_c|: colours of a degree-1
  Gaussian seen from two opposite sides;
* Adam (Sec. 3.2 pose step, Sec. 3.3 Gaussian step) over several steps:
  with a constant gradient the bias-corrected moments equal the gradient at
  every step, and with varying gradients the moments equal their sum forms
  m_t = (1 - b1) sum_k b1^(t-k) g_k, v_t = (1 - b2) sum_k b2^(t-k) g_k^2.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle
from paper_2410_08743_gb300 import synth

C0 = 1.0 / (2.0 * math.sqrt(math.pi))
C1 = math.sqrt(3.0 / (4.0 * math.pi))
EPS2D = float(np.float32(0.3))


def _cam(W=64, H=48, f=60.0, cx=None, cy=None):
    return dict(fx=f, fy=f, cx=W / 2.0 if cx is None else cx, cy=H / 2.0 if cy is None else cy,
                width=W, height=H)


def _scene(mu, s, q, o, sh=None, deg=0):
    n = len(o)
    if sh is None:
        sh = np.zeros((n, 16, 3), np.float32)
    return dict(means=np.asarray(mu, np.float32).reshape(n, 3), scales=np.asarray(s, np.float32).reshape(n, 3),
                quats=np.asarray(q, np.float32).reshape(n, 4), opac=np.asarray(o, np.float32),
                sh=np.asarray(sh, np.float32), sh_degree=deg)


def _pi(mc, cam):
    x, y, z = mc
    return np.array([cam["fx"] * x / z + cam["cx"], cam["fy"] * y / z + cam["cy"]])


def _jacobian_complex_step(mc, cam, h=1e-30):
    J = np.zeros((2, 3))
    for k in range(3):
        p = np.array(mc, np.complex128)
        p[k] += 1j * h
        J[:, k] = _pi(p, cam).imag / h
    return J


def _look_at_pose(center, target, up=(0.0, 1.0, 0.0)):
    """World->camera pose [12] of a camera at `center` whose +z axis points at
    `target` (rows of R are the camera axes in world coordinates)."""
    z = np.asarray(target, float) - np.asarray(center, float)
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, float), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return np.concatenate([R.reshape(9), -R @ np.asarray(center, float)])


# ------------------------------------------------------------------ Eq. 1-2
def test_rotation_of_the_quaternion_matches_scipy_on_axis():
    """Identity camera, Gaussian on the optical axis: J = diag(f/z, f/z) on the
    x, y block and zero in the z column, so Sigma_hat = (f/z)^2 Sigma[:2,:2] +
    0.3 I exposes the top-left block of R(q) diag(s^2) R(q)^T directly."""
    rng = np.random.default_rng(40)
    z, f = 4.0, 60.0
    for _ in range(8):
        q = rng.standard_normal(4).astype(np.float32)            # (w, x, y, z), not normalised
        s = rng.uniform(0.02, 0.2, 3).astype(np.float32)
        sc = _scene([[0, 0, z]], [s], [q], [0.8])
        vals = oracle.project_values(sc, [_cam(f=f)], synth.pose_from_center(np.eye(3), np.zeros(3))[None])[0]
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar last, normalises
        Sig = R @ np.diag(s.astype(np.float64) ** 2) @ R.T
        Sh = (f / z) ** 2 * Sig[:2, :2] + EPS2D * np.eye(2)
        Q = np.linalg.inv(Sh)
        np.testing.assert_allclose(vals[2:5], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(vals[:2], [32.0, 24.0], atol=1e-12)


def test_projected_covariance_off_axis_matches_complex_step_jacobian():
    """Rotated, anisotropic Gaussians at off-axis camera-space positions under
    rotated, translated cameras: mu_hat = pi(mu_c) and Sigma_hat = J_cs Sigma_c
    J_cs^T + 0.3 I, with R(q) from scipy and J_cs the complex-step Jacobian of
    pi.  A transposed R(q), a wrong sign of an off-axis entry of J (Eq. 2) or a
    transposed camera rotation each moves the conic far outside the
    tolerance."""
    rng = np.random.default_rng(41)
    checked = 0
    for trial in range(40):
        cam = _cam(W=96 + 8 * (trial % 5), H=72, f=70.0 + trial)
        center = rng.uniform(-0.5, 0.5, 3)
        pose = _look_at_pose(center, center + np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 1.0]))
        Rc, tc = pose[:9].reshape(3, 3), pose[9:]
        # an off-axis point well inside the frustum clamp (|x/z| < 0.8 tan)
        zc = rng.uniform(2.0, 6.0)
        ux = rng.uniform(-0.8, 0.8) * cam["width"] / (2 * cam["fx"])
        uy = rng.uniform(-0.8, 0.8) * cam["height"] / (2 * cam["fy"])
        mc_target = np.array([ux * zc, uy * zc, zc])
        mu = (Rc.T @ (mc_target - tc)).astype(np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        s = np.array([rng.uniform(0.02, 0.1), rng.uniform(0.1, 0.3), rng.uniform(0.01, 0.05)], np.float32)
        sc = _scene([mu], [s], [q], [0.8])
        vals = oracle.project_values(sc, [cam], pose[None])[0]
        mc = Rc @ mu.astype(np.float64) + tc
        assert abs(mc[0] / mc[2]) > 1e-3 or abs(mc[1] / mc[2]) > 1e-3
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(s.astype(np.float64) ** 2) @ R.T
        Sc = Rc @ Sig @ Rc.T
        J = _jacobian_complex_step(mc, cam)
        Sh = J @ Sc @ J.T + EPS2D * np.eye(2)
        Q = np.linalg.inv(Sh)
        np.testing.assert_allclose(vals[:2], _pi(mc, cam), rtol=1e-12, atol=1e-10)
        scale = np.abs(Q).max()
        np.testing.assert_allclose(vals[2:5], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-10, atol=1e-12 * scale)
        checked += 1
    assert checked == 40


def test_key_path_radius_of_a_rotated_anisotropic_gaussian():
    """The FP32 key path's radius follows the same rotated covariance:
    r = ceil(3 sqrt(lambda_max)) of the independently built Sigma_hat, for
    cases whose 3 sqrt(lambda_max) is not within 1e-3 of an integer."""
    rng = np.random.default_rng(42)
    n_checked = 0
    for _ in range(60):
        cam = _cam(W=128, H=96, f=90.0)
        q = rng.standard_normal(4).astype(np.float32)
        s = np.array([rng.uniform(0.02, 0.08), rng.uniform(0.1, 0.4), rng.uniform(0.01, 0.05)], np.float32)
        zc = rng.uniform(2.5, 5.0)
        mu = np.array([rng.uniform(-0.3, 0.3) * zc, rng.uniform(-0.2, 0.2) * zc, zc], np.float32)
        sc = _scene([mu], [s], [q], [0.8])
        k = oracle.keys(sc, [cam], synth.pose_from_center(np.eye(3), np.zeros(3))[None])
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(s.astype(np.float64) ** 2) @ R.T
        J = _jacobian_complex_step(mu.astype(np.float64), cam)
        Sh = J @ Sig @ J.T + EPS2D * np.eye(2)
        mid = 0.5 * (Sh[0, 0] + Sh[1, 1])
        lam = mid + math.sqrt(max(0.1, mid * mid - np.linalg.det(Sh)))
        r = 3.0 * math.sqrt(lam)
        if abs(r - round(r)) < 1e-3:
            continue
        assert k["valid"][0] == 1
        assert k["radius"][0] == math.ceil(r), (k["radius"][0], r)
        n_checked += 1
    assert n_checked >= 50


# ------------------------------------------------------- screen bound, tiles
# Gaussians on the optical axis of an identity camera (f = 60, z = 4) with
# isotropic scale sigma, so Sigma_hat = s2 I with s2 = (60 sigma / 4)^2 + 0.3;
# then mid^2 - det = 0 is raised to 0.1 and lambda_max = s2 + sqrt(0.1).
#   sigma = 0.05: s2 = 0.8625, lambda_max = 1.17873, 3 sqrt = 3.2571 -> r = 4
#   sigma = 0.2:  s2 = 9.3,    lambda_max = 9.61623, 3 sqrt = 9.3030 -> r = 10
# The principal point (cx, cy) places mu_hat; a 64 x 48 image has 4 x 3 tiles
# of 16 px, tile id = ty * 4 + tx, and the rectangle holds the tiles whose
# 16 px span meets [mu_hat - r, mu_hat + r - 1] on each axis, clamped to the
# grid: x0 = floor((mu - r) / 16), x1 = floor((mu + r + 15) / 16), tiles
# [x0, x1).
HAND_CASES = [
    # sigma, cx, cy, radius, rect (x0, y0, x1, y1), tile ids
    (0.05, 32.0, 24.0, 4, (1, 1, 3, 2), [5, 6]),             # 28..35 -> tiles 1, 2; 20..27 -> tile 1
    (0.05, 28.0, 12.0, 4, (1, 0, 2, 1), [1]),                # mu + r = 32 and 16 fall on tile edges
    (0.05, 20.0, 20.0, 4, (1, 1, 2, 2), [5]),                # mu - r = 16 and 16 fall on tile edges
    (0.05, 62.0, 46.0, 4, (3, 2, 4, 3), [11]),               # spills past the right / bottom edge
    (0.05, 1.0, 2.0, 4, (0, 0, 1, 1), [0]),                  # spills past the left / top edge
    (0.2, 32.0, 24.0, 10, (1, 0, 3, 3), [1, 2, 5, 6, 9, 10]),  # 22..42 -> 1, 2; 14..34 -> 0, 1, 2
]


@pytest.mark.parametrize("sigma,cx,cy,radius,rect,tiles", HAND_CASES)
def test_radius_and_tile_rectangle_worked_by_hand(sigma, cx, cy, radius, rect, tiles):
    cam = _cam(cx=cx, cy=cy)
    sc = _scene([[0, 0, 4.0]], [[sigma] * 3], [[1, 0, 0, 0]], [0.9])
    k = oracle.keys(sc, [cam], synth.pose_from_center(np.eye(3), np.zeros(3))[None])
    assert k["valid"][0] == 1
    assert int(k["radius"][0]) == radius
    assert tuple(int(x) for x in k["rect"][0]) == rect
    got = [t for t in range(12) if k["ranges"][t, 1] > k["ranges"][t, 0]]
    assert got == tiles
    assert k["n_keys"] == len(tiles)


def test_rectangle_grows_exactly_at_a_tile_edge():
    """The next column of tiles joins once mu_hat + r - 1 reaches its first
    pixel, and not before: with r = 4, cx = 28.75 gives mu_hat + r - 1 = 31.75
    (tile 1 only) and cx = 29.25 gives 32.25 (tiles 1 and 2)."""
    for cx, want in ((28.75, [5]), (29.25, [5, 6])):
        sc = _scene([[0, 0, 4.0]], [[0.05] * 3], [[1, 0, 0, 0]], [0.9])
        k = oracle.keys(sc, [_cam(cx=cx, cy=24.0)], synth.pose_from_center(np.eye(3), np.zeros(3))[None])
        got = [t for t in range(12) if k["ranges"][t, 1] > k["ranges"][t, 0]]
        assert got == want, (cx, got)


# ------------------------------------------------------------ SH direction
def test_sh_view_direction_points_from_the_camera_to_the_gaussian():
    """A Gaussian at the world origin with DC 0 and only the l = 1, m = 1
    coefficient k (basis -C1 d_x, Condon-Shortley): seen from (-3, 0, 0) the
    direction is d = +x and the colour 0.5 - C1 k; seen from (+3, 0, 0) it is
    d = -x and 0.5 + C1 k.  Likewise for m = -1 (basis -C1 d_y) from below and
    above, and m = 0 (basis +C1 d_z) from behind and in front."""
    k = 0.2
    cases = [
        (3, [-3.0, 0.0, 0.0], [0.0, 0.0, 1.0], 0.5 - C1 * k),
        (3, [3.0, 0.0, 0.0], [0.0, 0.0, 1.0], 0.5 + C1 * k),
        (1, [0.0, -3.0, 0.0], [0.0, 0.0, 1.0], 0.5 - C1 * k),
        (1, [0.0, 3.0, 0.0], [0.0, 0.0, 1.0], 0.5 + C1 * k),
        (2, [0.0, 0.0, -3.0], [0.0, 1.0, 0.0], 0.5 + C1 * k),
        (2, [0.0, 0.0, 3.0], [0.0, 1.0, 0.0], 0.5 - C1 * k),
    ]
    for coef, centre, up, want in cases:
        sh = np.zeros((1, 16, 3), np.float32)
        sh[0, coef, :] = k
        sc = _scene([[0, 0, 0]], [[0.05] * 3], [[1, 0, 0, 0]], [0.9], sh=sh, deg=1)
        pose = _look_at_pose(centre, [0.0, 0.0, 0.0], up=up)
        vals = oracle.project_values(sc, [_cam()], pose[None])[0]
        kk = float(np.float32(k))
        want32 = 0.5 + (want - 0.5) * kk / k
        np.testing.assert_allclose(vals[6:9], [want32] * 3, atol=1e-12, err_msg=str((coef, centre)))
        np.testing.assert_allclose(vals[:2], [32.0, 24.0], atol=1e-9)   # the Gaussian is on the axis


# ------------------------------------------------------------------- Adam
def _hat(tau):
    rho, phi = tau[:3], tau[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return M


def _mat(T):
    M = np.eye(4)
    M[:3, :3] = T[:9].reshape(3, 3)
    M[:3, 3] = T[9:]
    return M


def test_pose_adam_constant_gradient_moves_by_lr_every_step():
    """With the same gradient g at steps 1..3 the bias-corrected moments are
    m_hat = g and v_hat = g^2 at every step, so every step is
    delta = -lr g / (|g| + eps) and three steps compose to expm(3 delta^) T0.
    Bias correction with b^1 in place of b^t fails at step 2."""
    rng = np.random.default_rng(43)
    V, lr, eps = 2, 1e-2, 1e-8
    poses = np.stack([oracle.se3_exp(rng.standard_normal(6) * 0.3) for _ in range(V)])
    g = rng.standard_normal((V, 6))
    m = np.zeros((V, 6)); v = np.zeros((V, 6))
    out = poses.copy()
    for step in (1, 2, 3):
        oracle.pose_adam(out, m, v, g, lr, step, eps=eps)
    for i in range(V):
        delta = -lr * g[i] / (np.abs(g[i]) + eps)
        M3 = scipy.linalg.expm(_hat(3.0 * delta)) @ _mat(poses[i])
        np.testing.assert_allclose(_mat(out[i]), M3, atol=1e-12)


def test_pose_adam_three_steps_match_the_sum_form_of_the_moments():
    rng = np.random.default_rng(44)
    V, lr, eps, b1, b2 = 3, 5e-3, 1e-8, 0.9, 0.999
    poses = np.stack([oracle.se3_exp(rng.standard_normal(6) * 0.3) for _ in range(V)])
    gs = [rng.standard_normal((V, 6)) * (1 + 3 * k) for k in range(3)]
    m = np.zeros((V, 6)); v = np.zeros((V, 6))
    out = poses.copy()
    expect = np.stack([_mat(p) for p in poses])
    for t in (1, 2, 3):
        oracle.pose_adam(out, m, v, gs[t - 1], lr, t, b1=b1, b2=b2, eps=eps)
        mt = (1 - b1) * sum(b1 ** (t - k) * gs[k - 1] for k in range(1, t + 1))
        vt = (1 - b2) * sum(b2 ** (t - k) * gs[k - 1] ** 2 for k in range(1, t + 1))
        np.testing.assert_allclose(m, mt, rtol=1e-13)
        np.testing.assert_allclose(v, vt, rtol=1e-13)
        delta = -lr * (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
        for i in range(V):
            expect[i] = scipy.linalg.expm(_hat(delta[i])) @ expect[i]
            np.testing.assert_allclose(_mat(out[i]), expect[i], atol=1e-12)


def test_gaussian_adam_three_steps_constant_and_varying_gradients():
    """Constant activated gradients on the raw means and SH: each of three
    steps moves by -lr sign(g).  Varying gradients on every group: the raw
    parameters follow the sum-form moments, with the activation chain
    ds/dlog s = s and do/dlogit = o (1 - o) taken at each step's parameters."""
    rng = np.random.default_rng(45)
    n, b1, b2, eps = 5, 0.9, 0.999, 1e-15
    lrs = dict(means=1e-3, scales=5e-3, quats=1e-3, opac=5e-2, sh_dc=2.5e-3, sh_rest=1.25e-4)
    lr_of = dict(means=1e-3, log_scales=5e-3, quats=1e-3, logit_opac=5e-2)
    raw = {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
           "quats": rng.standard_normal((n, 4)), "logit_opac": rng.standard_normal((n, 1)),
           "sh": rng.standard_normal((n, 48))}
    r0 = {k: a.copy() for k, a in raw.items()}
    m = {k: np.zeros_like(a) for k, a in raw.items()}
    v = {k: np.zeros_like(a) for k, a in raw.items()}
    g_const = {"means": rng.standard_normal((n, 3)), "scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
               "opac": np.zeros((n, 1)), "sh": rng.standard_normal((n, 48))}
    for step in (1, 2, 3):
        oracle.gaussian_adam(raw, g_const, m, v, lrs, step, sh_degree=3)
    np.testing.assert_allclose(raw["means"], r0["means"] - 3 * 1e-3 * np.sign(g_const["means"]), atol=1e-14)
    np.testing.assert_allclose(raw["sh"][:, :3], r0["sh"][:, :3] - 3 * 2.5e-3 * np.sign(g_const["sh"][:, :3]),
                               atol=1e-14)
    np.testing.assert_allclose(raw["sh"][:, 3:], r0["sh"][:, 3:] - 3 * 1.25e-4 * np.sign(g_const["sh"][:, 3:]),
                               atol=1e-14)
    assert np.array_equal(raw["quats"], r0["quats"])          # zero gradient, zero moments: no move

    raw = {k: a.copy() for k, a in r0.items()}
    m = {k: np.zeros_like(a) for k, a in raw.items()}
    v = {k: np.zeros_like(a) for k, a in raw.items()}
    expect = {k: a.copy() for k, a in r0.items()}
    hist = {k: [] for k in r0}
    for t in (1, 2, 3):
        g = {"means": rng.standard_normal((n, 3)), "scales": rng.standard_normal((n, 3)),
             "quats": rng.standard_normal((n, 4)), "opac": rng.standard_normal((n, 1)),
             "sh": rng.standard_normal((n, 48))}
        # raw-space gradients at this step's parameters
        graw = {"means": g["means"], "log_scales": g["scales"] * np.exp(expect["log_scales"]),
                "quats": g["quats"],
                "logit_opac": g["opac"] * (o := 1 / (1 + np.exp(-expect["logit_opac"]))) * (1 - o),
                "sh": g["sh"]}
        oracle.gaussian_adam(raw, g, m, v, lrs, t, sh_degree=3)
        for key in r0:
            hist[key].append(graw[key])
            mt = (1 - b1) * sum(b1 ** (t - k) * hist[key][k - 1] for k in range(1, t + 1))
            vt = (1 - b2) * sum(b2 ** (t - k) * hist[key][k - 1] ** 2 for k in range(1, t + 1))
            step = (mt / (1 - b1 ** t)) / (np.sqrt(vt / (1 - b2 ** t)) + eps)
            if key == "sh":
                lr = np.full(48, 1.25e-4); lr[:3] = 2.5e-3
            else:
                lr = lr_of[key]
            expect[key] = expect[key] - lr * step
            np.testing.assert_allclose(raw[key], expect[key], rtol=1e-12, atol=1e-14, err_msg=f"{key} step {t}")
