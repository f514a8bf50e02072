"""Pins of the oracle's building blocks against library routines and closed
forms (no CUDA involved).

- SH basis (Sec. 3.1, colour c = SH(f, d)): against scipy's complex spherical
  harmonics with the Condon-Shortley phase, and orthonormality by quadrature.
- SE(3) Exp/Log (Sec. 3.2, T = Exp(tau)): against scipy.linalg.expm of the 4x4
  hat matrix, and Log(Exp(tau)) = tau.
- SSIM window and D-SSIM (Eq. 16's DSSIM term): window against
  scipy.ndimage.gaussian_filter, SSIM(I, I) = 1, constant-image closed form.
- Pose Adam step: the first step's closed form.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.ndimage
import scipy.special

import oracle


def _real_sh_scipy(l, m, theta, phi):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included):
    sqrt(2) Im(Y_l^|m|) for m < 0, Y_l^0, sqrt(2) Re(Y_l^m) for m > 0."""
    if hasattr(scipy.special, "sph_harm_y"):
        Y = scipy.special.sph_harm_y(l, abs(m), theta, phi)
    else:  # older scipy: sph_harm(m, n, azimuth, polar)
        Y = scipy.special.sph_harm(abs(m), l, phi, theta)
    if m < 0:
        return math.sqrt(2.0) * Y.imag
    if m == 0:
        return Y.real
    return math.sqrt(2.0) * Y.real


def _dirs(n, seed=0):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy_real_harmonics():
    d = _dirs(257)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.sh_eval(d, 3)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, k], ref, rtol=1e-12, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform in phi integrates the degree <= 6
    # products exactly.
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phis, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_eval(d, 3)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree_truncation():
    d = _dirs(10)
    Y1 = oracle.sh_eval(d, 1)
    assert np.all(Y1[:, 4:] == 0) and np.all(Y1[:, 1:4] != 0)
    Y0 = oracle.sh_eval(d, 0)
    assert np.all(Y0[:, 1:] == 0)


def _hat(tau):
    rho, phi = tau[:3], tau[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    M[:3, 3] = rho
    return M


@pytest.mark.parametrize("scale", [1.0, 1e-3, 1e-6, 0.0, 2.5])
def test_se3_exp_matches_expm(scale):
    rng = np.random.default_rng(7)
    for _ in range(20):
        tau = rng.standard_normal(6) * scale
        E = scipy.linalg.expm(_hat(tau))
        T = oracle.se3_exp(tau)
        np.testing.assert_allclose(T[:9].reshape(3, 3), E[:3, :3], atol=1e-13)
        np.testing.assert_allclose(T[9:], E[:3, 3], atol=1e-13)


def test_se3_log_inverts_exp():
    rng = np.random.default_rng(8)
    for scale in (1.0, 1e-3, 1e-7):
        for _ in range(20):
            tau = rng.standard_normal(6) * scale
            if np.linalg.norm(tau[3:]) > 3.0:
                continue
            np.testing.assert_allclose(oracle.se3_log(oracle.se3_exp(tau)), tau, atol=1e-10 * max(1, scale))


def test_se3_left_update_composes():
    rng = np.random.default_rng(9)
    tau = rng.standard_normal(6) * 0.3
    T0 = oracle.se3_exp(rng.standard_normal(6) * 0.5)
    T1 = oracle.se3_left_update(tau, T0)
    M0 = np.eye(4); M0[:3, :3] = T0[:9].reshape(3, 3); M0[:3, 3] = T0[9:]
    M1 = scipy.linalg.expm(_hat(tau)) @ M0
    np.testing.assert_allclose(T1[:9].reshape(3, 3), M1[:3, :3], atol=1e-13)
    np.testing.assert_allclose(T1[9:], M1[:3, 3], atol=1e-13)


def test_pose_adam_first_step_closed_form():
    rng = np.random.default_rng(10)
    V = 3
    poses = np.stack([oracle.se3_exp(rng.standard_normal(6) * 0.2) for _ in range(V)])
    g = rng.standard_normal((V, 6))
    m = np.zeros((V, 6)); v = np.zeros((V, 6))
    lr, eps = 1e-2, 1e-8
    out = poses.copy()
    oracle.pose_adam(out, m, v, g, lr, 1, eps=eps)
    for i in range(V):
        delta = -lr * g[i] / (np.abs(g[i]) + eps)    # m_hat = g, v_hat = g^2 on step 1
        M0 = np.eye(4); M0[:3, :3] = poses[i, :9].reshape(3, 3); M0[:3, 3] = poses[i, 9:]
        M1 = scipy.linalg.expm(_hat(delta)) @ M0
        np.testing.assert_allclose(out[i, :9].reshape(3, 3), M1[:3, :3], atol=1e-12)
        np.testing.assert_allclose(out[i, 9:], M1[:3, 3], atol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_ssim_window_matches_scipy_gaussian_filter():
    rng = np.random.default_rng(11)
    x = rng.uniform(size=(23, 31))
    ref = scipy.ndimage.gaussian_filter(x, sigma=1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)
    np.testing.assert_allclose(oracle.ssim_filter(x), ref, atol=1e-13)


def _views(W, H):
    return [dict(fx=1.0, fy=1.0, cx=0.0, cy=0.0, width=W, height=H)]


def test_dssim_identity_is_zero():
    rng = np.random.default_rng(12)
    W, H = 40, 30
    img = rng.uniform(size=3 * W * H)
    L, d, smap = oracle.loss_dssim(_views(W, H), img.astype(np.float32).astype(np.float64),
                                   img.astype(np.float32))
    assert abs(L) < 1e-12
    np.testing.assert_allclose(smap, 1.0, atol=1e-12)
    assert np.abs(d).max() < 1e-12


def test_ssim_constant_images_interior_closed_form():
    W, H = 32, 28
    a, b = 0.3, 0.7
    img = np.full(3 * W * H, a)
    tgt = np.full(3 * W * H, b, np.float32)
    _, _, smap = oracle.loss_dssim(_views(W, H), img, tgt)
    C1 = 0.01 ** 2
    b32 = float(np.float32(b))
    expect = (2 * a * b32 + C1) / (a * a + b32 * b32 + C1)   # sigma terms vanish inside
    inner = smap.reshape(3, H, W)[:, 5:-5, 5:-5]
    np.testing.assert_allclose(inner, expect, atol=1e-12)


def test_l1_loss_and_sign_gradient():
    rng = np.random.default_rng(13)
    views = [dict(fx=1, fy=1, cx=0, cy=0, width=5, height=4), dict(fx=1, fy=1, cx=0, cy=0, width=3, height=2)]
    n = 3 * (20 + 6)
    img = rng.uniform(size=n)
    tgt = rng.uniform(size=n).astype(np.float32)
    tgt[0] = np.float32(img[0]); img[0] = float(tgt[0])    # an exact tie -> zero gradient
    L, d, _ = oracle.loss_l1(views, img, tgt, weight=0.8)
    e0 = np.abs(img[:60] - tgt[:60]).mean(); e1 = np.abs(img[60:] - tgt[60:]).mean()
    assert abs(L - 0.8 * (e0 + e1)) < 1e-14
    assert d[0] == 0.0
    np.testing.assert_allclose(d[1:60], 0.8 * np.sign(img[1:60] - tgt[1:60]) / 60)
    np.testing.assert_allclose(d[60:], 0.8 * np.sign(img[60:] - tgt[60:]) / 18)


def test_dssim_gradient_finite_differences():
    rng = np.random.default_rng(14)
    W, H = 14, 12
    views = _views(W, H)
    img = rng.uniform(size=3 * W * H)
    tgt = rng.uniform(size=3 * W * H).astype(np.float32)
    L, d, _ = oracle.loss_dssim(views, img, tgt, weight=0.2)
    for k in rng.choice(img.size, 25, replace=False):
        h = 1e-6
        ip = img.copy(); ip[k] += h
        im = img.copy(); im[k] -= h
        fd = (oracle.loss_dssim(views, ip, tgt, 0.2)[0] - oracle.loss_dssim(views, im, tgt, 0.2)[0]) / (2 * h)
        assert abs(fd - d[k]) <= 1e-6 * max(1e-3, abs(d[k])) + 1e-10, (k, fd, d[k])


def test_gaussian_adam_first_step_closed_form_and_chain():
    """First Adam step: m_hat = g, v_hat = g^2, so each raw parameter moves by
    -lr g / (|g| + eps); log-scales and logit-opacities see the activated
    gradient times ds/dlog s = s and do/dlogit = o (1 - o)."""
    rng = np.random.default_rng(15)
    n = 7
    raw = {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
           "quats": rng.standard_normal((n, 4)), "logit_opac": rng.standard_normal((n, 1)),
           "sh": rng.standard_normal((n, 48))}
    grads = {"means": rng.standard_normal((n, 3)), "scales": rng.standard_normal((n, 3)),
             "quats": rng.standard_normal((n, 4)), "opac": rng.standard_normal((n, 1)),
             "sh": rng.standard_normal((n, 48))}
    m = {k: np.zeros_like(a) for k, a in raw.items()}
    v = {k: np.zeros_like(a) for k, a in raw.items()}
    lrs = dict(means=1e-3, scales=5e-3, quats=1e-3, opac=5e-2, sh_dc=2.5e-3, sh_rest=1.25e-4)
    r0 = {k: a.copy() for k, a in raw.items()}
    sc, op = oracle.gaussian_adam(raw, grads, m, v, lrs, 1, sh_degree=1)
    eps = 1e-15
    step = lambda g, lr: -lr * g / (np.abs(g) + eps)
    np.testing.assert_allclose(raw["means"], r0["means"] + step(grads["means"], 1e-3), atol=1e-15)
    gs = grads["scales"] * np.exp(r0["log_scales"])
    np.testing.assert_allclose(raw["log_scales"], r0["log_scales"] + step(gs, 5e-3), atol=1e-15)
    o = 1 / (1 + np.exp(-r0["logit_opac"]))
    np.testing.assert_allclose(raw["logit_opac"], r0["logit_opac"] + step(grads["opac"] * o * (1 - o), 5e-2), atol=1e-15)
    np.testing.assert_allclose(raw["sh"][:, :3], r0["sh"][:, :3] + step(grads["sh"][:, :3], 2.5e-3), atol=1e-15)
    np.testing.assert_allclose(raw["sh"][:, 3:12], r0["sh"][:, 3:12] + step(grads["sh"][:, 3:12], 1.25e-4), atol=1e-15)
    assert np.array_equal(raw["sh"][:, 12:], r0["sh"][:, 12:])      # above degree 1: untouched
    np.testing.assert_allclose(sc, np.exp(raw["log_scales"]), rtol=1e-15)
    np.testing.assert_allclose(op, 1 / (1 + np.exp(-raw["logit_opac"][:, 0])), rtol=1e-15)


def test_dssim_conditioning_bounds_the_gradient_and_closed_form():
    """The conditioning diagnostic is a sum of the magnitudes of the terms the
    D-SSIM gradient adds up, so it bounds |dL/dC| (triangle inequality).  For
    two equal constant images c inside the border band, SSIM's partials are
    dmu = 0, dvx = -1/C2, dcxy = 2/C2, so the terms 2c/C2 + 2c/C2 (from the
    folded mu term) + 2c/C2 + 2c/C2 cancel to a zero gradient while their
    magnitudes add to 8 c w / (3 H W C2)."""
    rng = np.random.default_rng(16)
    W, H = 24, 20
    views = _views(W, H)
    img = rng.uniform(size=3 * W * H)
    tgt = rng.uniform(size=3 * W * H).astype(np.float32)
    _, d, _ = oracle.loss_dssim(views, img, tgt, weight=0.2)
    cond = oracle.loss_dssim_cond(views, img, tgt, weight=0.2)
    assert np.all(cond >= np.abs(d) * (1 - 1e-12))
    assert np.median(cond / np.maximum(np.abs(d), 1e-300)) > 2.0      # it does cancel
    c, w = 0.625, 0.2
    W, H = 40, 36
    views = _views(W, H)
    flat = np.full(3 * W * H, c)
    _, d0, _ = oracle.loss_dssim(views, flat, flat.astype(np.float32), weight=w)
    cond0 = oracle.loss_dssim_cond(views, flat, flat.astype(np.float32), weight=w)
    inner = cond0.reshape(3, H, W)[:, 10:-10, 10:-10]     # windows of windows inside the image
    assert inner.size == 3 * 16 * 20
    np.testing.assert_allclose(inner, 8 * c * w / (3 * W * H * 0.03 ** 2), rtol=1e-12)
    assert np.abs(d0).max() < 1e-12
