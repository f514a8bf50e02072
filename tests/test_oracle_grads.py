"""Pins of the oracle's analytic backward (Sec. 3.2, Eq. 5-13 and the prior
art's per-Gaussian gradients) against central finite differences of its own
FP64 forward, and against exact identities of rigid motion.

Pose finite differences perturb T <- expm(h e_k^) T with scipy's matrix
exponential, independent of the oracle's Exp.  Samples whose discrete state
(culling, rectangles, list order, blended sets, clamps) changes between +h and
-h are skipped: the loss is only piecewise smooth."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2410_08743_gb300 import synth


def _hat(tau):
    rho, phi = tau[:3], tau[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    M[:3, 3] = rho
    return M


def _left(pose, tau):
    M = np.eye(4); M[:3, :3] = pose[:9].reshape(3, 3); M[:3, 3] = pose[9:]
    M = scipy.linalg.expm(_hat(tau)) @ M
    return np.concatenate([M[:3, :3].reshape(9), M[:3, 3]])


def _fd_scene(seed=21, n=260, deg=3):
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=deg, lo=(-0.8, -0.6, 2.0), hi=(0.8, 0.6, 3.5))
    sc["scales"] = (sc["scales"] * 2.5).astype(np.float32)       # large, anisotropic footprints
    sc["quats"] = (sc["quats"] * rng.uniform(0.5, 2.0, (n, 1))).astype(np.float32)  # unnormalised
    sc["opac"][:8] = 0.9995                                      # some hit the 0.99 clamp
    # two big off-axis Gaussians beyond the frustum clamp but still on screen
    sc["means"][-2:] = np.array([[2.6, 0.1, 1.6], [-0.1, -2.1, 1.5]], np.float32)
    sc["scales"][-2:] = 0.35
    views = [dict(fx=40.0, fy=42.0, cx=23.5, cy=19.0, width=48, height=40)]
    pose = synth.perturb_normal(rng, synth.pose_from_center(np.eye(3), np.zeros(3)), 4.0, 0.05)
    return sc, views, pose[None, :]


def _loss_and_hash(sc, views, poses, wts):
    r = oracle.render(sc, views, poses)
    return float(np.dot(r["image"], wts)), r["hash"]



def _fd_param(sc, views, poses, wts, key, idx, h):
    x0 = sc[key][idx]
    xp = np.float32(x0 + h); xm = np.float32(x0 - h)
    sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sp[key][idx] = xp
    Lp, hp = _loss_and_hash(sp, views, poses, wts)
    sp[key][idx] = xm
    Lm, hm = _loss_and_hash(sp, views, poses, wts)
    return (Lp - Lm) / (float(xp) - float(xm)), hp, hm


def test_gradients_all_parameters_finite_differences():
    sc, views, poses = _fd_scene()
    rng = np.random.default_rng(3)
    r0 = oracle.render(sc, views, poses)
    wts = rng.standard_normal(r0["image"].size)
    g = oracle.backward(sc, views, poses, wts)
    base_hash = r0["hash"]
    n = len(sc["opac"])
    # Gaussians that actually contribute somewhere
    active = np.nonzero(np.abs(g["opac"]) > 1e-6)[0]
    assert len(active) > 50
    checks = 0
    skipped = 0
    plan = []
    for i in rng.choice(active, 14, replace=False):
        plan += [("means", (i, rng.integers(3)), "means"), ("scales", (i, rng.integers(3)), "scales"),
                 ("quats", (i, rng.integers(4)), "quats"), ("opac", (i,), "opac"),
                 ("sh", (i, rng.integers(16), rng.integers(3)), "sh")]
    plan += [("means", (n - 1, 0), "means"), ("means", (n - 2, 1), "means"), ("means", (n - 1, 2), "means")]
    plan += [("opac", (k,), "opac") for k in range(4)]
    for key, idx, gk in plan:
        x0 = float(sc[key][idx])
        h = 2e-4 * max(abs(x0), 0.05)
        fd, hp, hm = _fd_param(sc, views, poses, wts, key, idx, h)
        if hp != base_hash or hm != base_hash:
            skipped += 1
            continue
        an = g[gk][idx]
        scale = max(abs(an), 1e-3 * np.abs(g[gk]).max())
        assert abs(fd - an) <= 2e-4 * scale, (key, idx, fd, an)
        checks += 1
    assert checks >= 0.7 * len(plan), (checks, skipped)


def test_pose_gradient_finite_differences_all_six():
    sc, views, poses = _fd_scene(seed=22)
    rng = np.random.default_rng(4)
    r0 = oracle.render(sc, views, poses)
    wts = rng.standard_normal(r0["image"].size)
    g = oracle.backward(sc, views, poses, wts)
    for k in range(6):
        e = np.zeros(6)
        for h in (1e-6, 3e-7, 1e-5):
            e[:] = 0; e[k] = h
            Lp, hp = _loss_and_hash(sc, views, _left(poses[0], e)[None], wts)
            Lm, hm = _loss_and_hash(sc, views, _left(poses[0], -e)[None], wts)
            if hp == r0["hash"] and hm == r0["hash"]:
                break
        else:
            pytest.fail(f"pose component {k}: discrete state changes at every step size")
        fd = (Lp - Lm) / (2 * h)
        an = g["pose"][0, k]
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-2 * np.abs(g["pose"]).max()), (k, fd, an)


def test_pose_gradient_finite_differences_multi_view_sh3_tiny():
    """Two views of the tiny workload with SH degree 3 colours: each view's
    6-vector against finite differences of that view's pose."""
    w = synth.tiny_workload(0)
    sc = dict(w["scene"])
    rng = np.random.default_rng(5)
    sh = sc["sh"].copy(); sh[:, 1:, :] = rng.normal(0, 0.2, sh[:, 1:, :].shape)
    sc["sh"] = sh.astype(np.float32); sc["sh_degree"] = 3
    poses = np.stack([w["poses"][0], synth.perturb_normal(rng, w["poses"][0], 5.0, 0.1)])
    views = [w["views"][0], w["views"][0]]
    r0 = oracle.render(sc, views, poses)
    wts = rng.standard_normal(r0["image"].size)
    g = oracle.backward(sc, views, poses, wts)
    for v in range(2):
        for k in range(6):
            ok = False
            for h in (1e-7, 1e-8, 1e-9):
                e = np.zeros(6); e[k] = h
                pp = poses.copy(); pp[v] = _left(poses[v], e)
                pm = poses.copy(); pm[v] = _left(poses[v], -e)
                Lp, hp = _loss_and_hash(sc, views, pp, wts)
                Lm, hm = _loss_and_hash(sc, views, pm, wts)
                if hp == r0["hash"] and hm == r0["hash"]:
                    ok = True
                    break
            assert ok, (v, k)
            fd = (Lp - Lm) / (2 * h)
            an = g["pose"][v, k]
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-2 * np.abs(g["pose"][v]).max()), (v, k, fd, an)


def test_rigid_motion_identity_translation():
    """Moving the camera by rho equals moving every Gaussian by -R_c^T rho:
    g_rho = R_c sum_i g_mu_i, exactly, for any SH degree."""
    for seed, deg in ((31, 3), (32, 0)):
        sc, views, poses = _fd_scene(seed=seed, deg=deg)
        rng = np.random.default_rng(seed)
        r0 = oracle.render(sc, views, poses)
        g = oracle.backward(sc, views, poses, rng.standard_normal(r0["image"].size))
        Rc = poses[0, :9].reshape(3, 3)
        np.testing.assert_allclose(g["pose"][0, :3], Rc @ g["means"].sum(0), rtol=1e-10, atol=1e-12)


def test_rigid_motion_identity_rotation_isotropic_sh0():
    """For isotropic Gaussians with view-independent colour, rotating the
    camera by phi equals rotating the means: g_phi = sum_i mu_c,i x (R_c g_mu_i)."""
    sc, views, poses = _fd_scene(seed=33, deg=0)
    iso = sc["scales"][:, :1].repeat(3, 1)
    sc["scales"] = np.ascontiguousarray(iso)
    rng = np.random.default_rng(33)
    r0 = oracle.render(sc, views, poses)
    g = oracle.backward(sc, views, poses, rng.standard_normal(r0["image"].size))
    Rc = poses[0, :9].reshape(3, 3); t = poses[0, 9:]
    mc = sc["means"].astype(np.float64) @ Rc.T + t
    ref = np.cross(mc, g["means"] @ Rc.T).sum(0)
    np.testing.assert_allclose(g["pose"][0, 3:], ref, rtol=1e-9, atol=1e-12)


def test_on_axis_isotropic_gaussian_has_no_roll_gradient():
    """A single isotropic Gaussian on the optical axis is symmetric under roll
    about the axis, so the phi_z component vanishes."""
    C0 = 0.28209479177387814
    sc = dict(means=np.array([[0, 0, 3.0]], np.float32), scales=np.full((1, 3), 0.08, np.float32),
              quats=np.array([[1, 0, 0, 0]], np.float32), opac=np.array([0.7], np.float32),
              sh=np.zeros((1, 16, 3), np.float32), sh_degree=0)
    sc["sh"][0, 0] = (np.array([0.9, 0.4, 0.1]) - 0.5) / C0
    views = [dict(fx=60.0, fy=60.0, cx=32.0, cy=24.0, width=64, height=48)]
    poses = synth.pose_from_center(np.eye(3), np.zeros(3))[None]
    r0 = oracle.render(sc, views, poses)
    tgt = np.zeros(r0["image"].size, np.float32)
    L, d, _ = oracle.loss_l1(views, r0["image"], tgt)
    g = oracle.backward(sc, views, poses, d)
    assert abs(g["pose"][0, 5]) < 1e-14 * max(1.0, np.abs(g["pose"]).max())
    assert np.abs(g["pose"][0, 2]) > 1e-6          # but depth does matter


def test_l1_loss_gradient_finite_differences_pose():
    w = synth.tiny_workload(0)
    tgt = oracle.render(w["scene"], w["views"], w["target_poses"])["image"].astype(np.float32)
    r0 = oracle.render(w["scene"], w["views"], w["poses"])
    L0, d, _ = oracle.loss_l1(w["views"], r0["image"], tgt)
    g = oracle.backward(w["scene"], w["views"], w["poses"], d)

    def loss(poses):
        r = oracle.render(w["scene"], w["views"], poses)
        return oracle.loss_l1(w["views"], r["image"], tgt)[0], r["hash"], np.sign(r["image"] - tgt)

    s0 = np.sign(r0["image"] - tgt)
    for k in range(6):
        done = False
        for h in (1e-7, 1e-8, 1e-9):
            e = np.zeros(6); e[k] = h
            Lp, hp, sp = loss(_left(w["poses"][0], e)[None])
            Lm, hm, sm = loss(_left(w["poses"][0], -e)[None])
            if hp == r0["hash"] and hm == r0["hash"] and np.array_equal(sp, s0) and np.array_equal(sm, s0):
                done = True
                break
        assert done, k
        fd = (Lp - Lm) / (2 * h)
        an = g["pose"][0, k]
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-2 * np.abs(g["pose"]).max()), (k, fd, an)
