"""Pins of the oracle's confidence-masked L1 (Sec. 3.4, Eq. 20-21).

* A threshold below every accumulated alpha keeps every pixel: the masked loss
  is then the plain L1 (pinned on its own) exactly, value and gradient.
* A single Gaussian never accumulates more than its clamped alpha 0.99, so at
  the paper's threshold (accumulated alpha > 0.99) its mask is empty: loss and
  gradient exactly zero.
* Two co-located opaque Gaussians accumulate more than 0.99 around the
  centre, so the mask is non-empty there and only masked pixels carry
  gradient; at the centre itself the stop rule blends only the first.
* Raising the threshold can only drop pixels: the loss is monotone.
* The analytic gradient of the masked loss through the renderer matches
  central finite differences wherever the mask does not change."""
import numpy as np

import oracle
from paper_2410_08743_gb300 import synth

from .test_oracle_grads import _fd_param, _fd_scene


def _single(n=1, opac=0.9995):
    sc = dict(means=np.array([[0.0, 0.0, 4.0]] * n, np.float32), scales=np.full((n, 3), 0.3, np.float32),
              quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), opac=np.full(n, opac, np.float32),
              sh=np.zeros((n, 16, 3), np.float32), sh_degree=0)
    sc["sh"][:, 0, :] = 0.2
    views = [dict(fx=60.0, fy=60.0, cx=16.0, cy=12.0, width=32, height=24)]
    return sc, views, synth.pose_from_center(np.eye(3), np.zeros(3))[None]


def test_threshold_below_everything_is_plain_l1():
    w = synth.tiny_workload(0)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    r = oracle.render(sc, views, poses)
    tgt = oracle.render(sc, views, w["target_poses"])["image"].astype(np.float32)
    L1, d1, _ = oracle.loss_l1(views, r["image"], tgt, weight=0.7)
    Lm, dm, _ = oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], mask_alpha=-1.0, weight=0.7)
    assert Lm == L1
    assert np.array_equal(dm, d1)


def test_single_gaussian_mask_is_empty():
    sc, views, poses = _single(1)
    r = oracle.render(sc, views, poses)
    assert (1.0 - r["T_final"]).max() == float(np.float32(0.99))  # the clamp is reached at the centre
    tgt = np.zeros(r["image"].size, np.float32)
    Lm, dm, _ = oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], 0.99)
    assert Lm == 0.0 and not dm.any()


def test_two_opaque_gaussians_mask_where_both_clamp():
    sc, views, poses = _single(2)
    r = oracle.render(sc, views, poses)
    acc = 1.0 - r["T_final"]
    inside = acc > float(np.float32(0.99))
    assert inside.any() and not inside.all()
    # at the centre the second splat would take T to 1e-4 - 2e-10 < t_min, so
    # the stop rule leaves the first alone: accumulated alpha 0.99, not kept
    c = 12 * 32 + 16
    assert acc[c] == float(np.float32(0.99)) and not inside[c]
    tgt = np.zeros(r["image"].size, np.float32)
    Lm, dm, _ = oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], 0.99)
    npx = r["T_final"].size
    for ch in range(3):
        assert np.all(dm[ch * npx:(ch + 1) * npx][~inside] == 0.0)
        assert np.all(dm[ch * npx:(ch + 1) * npx][inside] > 0.0)
    assert Lm > 0.0


def test_masked_loss_monotone_in_threshold():
    w = synth.tiny_workload(1)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    r = oracle.render(sc, views, poses)
    tgt = np.random.default_rng(3).uniform(size=r["image"].size).astype(np.float32)
    vals = [oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], a)[0] for a in (-1.0, 0.3, 0.6, 0.9, 0.99)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
    assert vals[0] == oracle.loss_l1(views, r["image"], tgt)[0]


def _masked_loss(sc, views, poses, tgt, a):
    r = oracle.render(sc, views, poses)
    L, _, _ = oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], a)
    mask = (1.0 - r["T_final"]) > a
    sign = np.sign(r["image"] - tgt.astype(np.float64))
    return L, hash((r["hash"], mask.tobytes(), sign.tobytes()))


def test_masked_gradient_matches_finite_differences():
    sc, views, poses = _fd_scene(22, 260, 1)
    sc["opac"][:] = np.maximum(sc["opac"], 0.9).astype(np.float32)   # some pixels pass 0.99
    a = 0.99
    r = oracle.render(sc, views, poses)
    assert ((1.0 - r["T_final"]) > a).mean() > 0.05
    tgt = (r["image"] + np.random.default_rng(5).normal(0, 0.05, r["image"].size)).astype(np.float32)
    _, d, _ = oracle.loss_l1_masked(views, r["image"], tgt, r["T_final"], a)
    g = oracle.backward(sc, views, poses, d)
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(40):
        i = int(rng.integers(len(sc["opac"])))
        k = int(rng.integers(3))
        if abs(g["means"][i, k]) < 1e-7:
            continue
        h = 1e-4
        x0 = sc["means"][i, k]
        Ls = []
        hs = []
        for sgn in (1, -1):
            sp = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in sc.items()}
            sp["means"][i, k] = np.float32(x0 + sgn * h)
            L_, h_ = _masked_loss(sp, views, poses, tgt, a)
            Ls.append(L_); hs.append(h_)
        if hs[0] != hs[1]:
            continue
        dx = float(np.float32(x0 + h)) - float(np.float32(x0 - h))
        fd = (Ls[0] - Ls[1]) / dx
        assert abs(fd - g["means"][i, k]) <= 1e-3 * abs(g["means"][i, k]) + 1e-9, (i, k, fd, g["means"][i, k])
        checked += 1
    assert checked >= 5
