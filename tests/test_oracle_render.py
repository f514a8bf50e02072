"""Pins of the oracle's forward pass (Sec. 3.1, Eq. 1-4) against closed forms,
brute force and an independent assembly of the tile lists."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_08743_gb300 import synth

ALPHA_MIN = float(np.float32(1.0 / 255.0))
C0 = 1.0 / (2.0 * math.sqrt(math.pi))  # the constant SH basis function


def _cam(W=64, H=48, f=60.0):
    return dict(fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, width=W, height=H)


def _identity():
    return synth.pose_from_center(np.eye(3), np.zeros(3))[None, :]


def _scene(mu, s, q, o, col, deg=0):
    n = len(o)
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = (np.asarray(col, np.float64) - 0.5) / C0
    return dict(means=np.asarray(mu, np.float32).reshape(n, 3), scales=np.asarray(s, np.float32).reshape(n, 3),
                quats=np.asarray(q, np.float32).reshape(n, 4), opac=np.asarray(o, np.float32),
                sh=sh, sh_degree=deg)


def test_single_isotropic_gaussian_closed_form():
    """Isotropic Gaussian on the optical axis: Sigma_hat = ((f s / z)^2 + eps) I,
    mu_hat = principal point, C = c min(0.99, o exp(-r^2 / 2 s_hat^2))."""
    z, sig, o = 4.0, 0.05, 0.8
    col = np.array([0.2, 0.5, 0.9])
    sc = _scene([[0, 0, z]], [[sig, sig, sig]], [[0.3, -1.2, 0.7, 2.0]], [o], [col])
    cam = _cam()
    r = oracle.render(sc, [cam], _identity())
    vals = oracle.project_values(sc, [cam], _identity())[0]
    s2 = (60.0 * float(np.float32(sig)) / z) ** 2 + float(np.float32(0.3))
    np.testing.assert_allclose(vals[:2], [32.0, 24.0], atol=1e-12)
    np.testing.assert_allclose(vals[2:5], [1 / s2, 0.0, 1 / s2], rtol=1e-12, atol=1e-14)
    c32 = np.float32((col - 0.5) / C0).astype(np.float64) * C0 + 0.5
    np.testing.assert_allclose(vals[6:9], c32, atol=1e-14)
    img = r["image"].reshape(3, 48, 64)
    py, px = np.mgrid[0:48, 0:64]
    a = float(np.float32(o)) * np.exp(-0.5 * ((px - 32.0) ** 2 + (py - 24.0) ** 2) / s2)
    a = np.minimum(a, float(np.float32(0.99)))
    a = np.where(a >= ALPHA_MIN, a, 0.0)
    for ch in range(3):
        np.testing.assert_allclose(img[ch], c32[ch] * a, atol=1e-12)
    np.testing.assert_allclose(r["T_final"].reshape(48, 64), 1.0 - a, atol=1e-12)


def test_zero_opacity_gives_background_and_zero_gradients():
    w = synth.tiny_workload(0)
    sc = dict(w["scene"]); sc["opac"] = np.zeros_like(sc["opac"])
    bg = (0.25, 0.5, 0.75)
    r = oracle.render(sc, w["views"], w["poses"], opts=dict(bg=bg))
    img = r["image"].reshape(3, -1)
    for ch in range(3):
        assert np.all(img[ch] == bg[ch])
    assert np.all(r["T_final"] == 1.0)
    rng = np.random.default_rng(0)
    g = oracle.backward(sc, w["views"], w["poses"], rng.standard_normal(img.size), opts=dict(bg=bg))
    for k in ("means", "scales", "quats", "opac", "sh", "pose"):
        assert np.all(g[k] == 0.0), k


def test_weights_and_transmittance_sum_to_one():
    """sum_i alpha_i prod_{j<i}(1 - alpha_j) + prod_j (1 - alpha_j) = 1: with every
    colour exactly 0.5 and a black background, 2 C + T_final = 1."""
    w = synth.tiny_workload(3)
    sc = dict(w["scene"]); sc["sh"] = np.zeros_like(sc["sh"])
    r = oracle.render(sc, w["views"], w["poses"])
    img = r["image"].reshape(3, -1)
    for ch in range(3):
        np.testing.assert_allclose(2 * img[ch] + r["T_final"], 1.0, atol=1e-13)
    assert r["T_final"].min() < 0.01   # the scene is dense enough to matter


@pytest.mark.parametrize("swap", [False, True])
def test_two_gaussians_depth_order(swap):
    """Eq. 4 front to back: at the principal point alpha_i = o_i, so
    C = c1 o1 + c2 o2 (1 - o1) with Gaussian 1 in front."""
    z1, z2 = (3.0, 5.0) if not swap else (5.0, 3.0)
    o = [0.6, 0.7]
    cols = [[1.0, 0.0, 0.25], [0.0, 1.0, 0.75]]
    sc = _scene([[0, 0, z1], [0, 0, z2]], [[0.05] * 3, [0.08] * 3], [[1, 0, 0, 0]] * 2, o, cols)
    r = oracle.render(sc, [_cam()], _identity())
    img = r["image"].reshape(3, 48, 64)
    o32 = [float(np.float32(x)) for x in o]
    c32 = [np.float32((np.array(c) - 0.5) / C0).astype(np.float64) * C0 + 0.5 for c in cols]
    front, back = (0, 1) if not swap else (1, 0)
    expect = c32[front] * o32[front] + c32[back] * o32[back] * (1 - o32[front])
    np.testing.assert_allclose(img[:, 24, 32], expect, atol=1e-12)
    np.testing.assert_allclose(r["T_final"][24 * 64 + 32], (1 - o32[0]) * (1 - o32[1]), atol=1e-12)


def test_brute_force_equals_tiled_multi_view():
    rng = np.random.default_rng(5)
    sc = synth.make_scene_box(5, 3000, sh_degree=3, lo=(-1, -1, 2.5), hi=(1, 1, 5))
    views = [_cam(64, 48), _cam(40, 33, 45.0), _cam(17, 70, 50.0)]
    poses = np.stack([synth.perturb_normal(rng, _identity()[0], 4.0, 0.1) for _ in views])
    t = oracle.render(sc, views, poses)
    b = oracle.render(sc, views, poses, brute=True)
    assert np.array_equal(t["image"], b["image"])
    assert np.array_equal(t["T_final"], b["T_final"])
    assert t["image"].max() > 0.1


def test_tile_lists_match_independent_assembly():
    """Each tile's list = the valid Gaussians whose rectangle holds the tile,
    ordered by (FP32 depth bits, index); rebuilt here with numpy."""
    rng = np.random.default_rng(6)
    sc = synth.make_scene_box(6, 1500, sh_degree=1, lo=(-1, -1, 2.5), hi=(1, 1, 5))
    views = [_cam(64, 48), _cam(50, 37, 40.0)]
    poses = np.stack([synth.perturb_normal(rng, _identity()[0], 3.0, 0.1) for _ in views])
    k = oracle.keys(sc, views, poses)
    n = len(sc["opac"])
    base = 0
    for v, cam in enumerate(views):
        gw, gh = (cam["width"] + 15) // 16, (cam["height"] + 15) // 16
        valid = k["valid"][v * n:(v + 1) * n].astype(bool)
        rect = k["rect"][v * n:(v + 1) * n]
        dbits = k["depth"][v * n:(v + 1) * n].view(np.uint32)
        for t in range(gw * gh):
            tx, ty = t % gw, t / gw
            ty = t // gw
            ids = np.nonzero(valid & (rect[:, 0] <= tx) & (tx < rect[:, 2]) & (rect[:, 1] <= ty) & (ty < rect[:, 3]))[0]
            order = ids[np.lexsort((ids, dbits[ids]))]
            s, e = k["ranges"][base + t]
            got = k["idx"][s:e] if e > s else np.zeros(0, np.uint32)
            assert np.array_equal(got, order), (v, t)
        base += gw * gh
    assert k["n_keys"] == int(sum((r[2] - r[0]) * (r[3] - r[1]) for r, ok in zip(k["rect"], k["valid"]) if ok))


def test_key_path_agrees_with_value_path():
    """The FP32 key path (depth, mu_hat, radius) agrees with the FP64 values."""
    w = synth.tiny_workload(0)
    k = oracle.keys(w["scene"], w["views"], w["poses"])
    vals = oracle.project_values(w["scene"], w["views"], w["poses"])
    ok = k["valid"].astype(bool)
    np.testing.assert_allclose(k["mu2f"][ok], vals[ok, :2], rtol=1e-5, atol=1e-4)
    a, b, c = vals[ok, 2], vals[ok, 3], vals[ok, 4]
    det = a * c - b * b
    A, B, Cc = c / det, -b / det, a / det       # Sigma_hat back from the conic
    mid = 0.5 * (A + Cc)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (A * Cc - B * B)))
    r64 = np.ceil(3 * np.sqrt(lam))
    assert np.mean(r64 == k["radius"][ok]) > 0.99
    m = w["scene"]["means"]
    np.testing.assert_allclose(k["depth"][ok], m[ok, 2], rtol=1e-6)


def test_culling_behind_near_plane():
    sc = _scene([[0, 0, 0.1], [0, 0, -2.0], [0, 0, 3.0]], [[0.05] * 3] * 3, [[1, 0, 0, 0]] * 3,
                [0.9, 0.9, 0.5], [[1, 1, 1]] * 3)
    k = oracle.keys(sc, [_cam()], _identity())
    assert list(k["valid"]) == [0, 0, 1]
    r = oracle.render(sc, [_cam()], _identity())
    assert abs(r["T_final"][24 * 64 + 32] - (1 - float(np.float32(0.5)))) < 1e-12


def test_frustum_clamp_only_changes_far_lateral_gaussians():
    """J's lateral clamp (x/z beyond 1.3 W/(2 fx)) leaves on-screen Gaussians
    untouched; an off-axis Gaussian beyond the limit gets a smaller footprint."""
    sc = _scene([[0.2, 0.1, 4.0], [2.2, 0.0, 1.5]], [[0.05] * 3, [0.3, 0.3, 0.3]], [[1, 0, 0, 0]] * 2,
                [0.9, 0.9], [[1, 1, 1]] * 2)
    cam = _cam()
    on = oracle.project_values(sc, [cam], _identity(), opts=dict(clamp_factor=1.3))
    off = oracle.project_values(sc, [cam], _identity(), opts=dict(clamp_factor=0.0))
    np.testing.assert_allclose(on[0], off[0], rtol=1e-14)
    assert not np.allclose(on[1, 2:5], off[1, 2:5])
