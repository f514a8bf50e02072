"""Pins of the oracle's T x SO(3) pose step (Sec. 4.2).

* Its translation gradient g_o = -R^T g_rho is the derivative of the loss with
  respect to the camera centre in world coordinates: central finite
  differences of the FP64 renderer with the centre moved along each world
  axis (rotation held) reproduce it.
* A pure rotation step leaves the camera centre where it was; a pure centre
  step leaves the rotation alone and moves the centre by exactly the step.
* The first Adam step moves each coordinate by -lr sign(g) (m_hat / sqrt(v_hat)
  = sign(g) at step 1)."""
import numpy as np

import oracle
from paper_2410_08743_gb300 import synth

from .test_oracle_grads import _fd_scene


def _centre(P):
    return -P[:9].reshape(3, 3).T @ P[9:]


def _with_centre(P, o):
    R = P[:9].reshape(3, 3)
    return np.concatenate([R.reshape(9), -R @ o])


def test_centre_gradient_matches_finite_differences():
    sc, views, poses = _fd_scene(23, 200, 2)
    rng = np.random.default_rng(2)
    wts = rng.standard_normal(3 * 48 * 40) * 1e-2
    g = oracle.backward(sc, views, poses, wts)["pose"][0]
    P = poses[0]
    R = P[:9].reshape(3, 3)
    g_o = -R.T @ g[:3]
    o = _centre(P)
    checked = 0
    for k in range(3):
        for h in (1e-6, 1e-7, 1e-5, 1e-8):
            e = np.zeros(3); e[k] = h
            rp = oracle.render(sc, views, _with_centre(P, o + e)[None])
            rm = oracle.render(sc, views, _with_centre(P, o - e)[None])
            if rp["hash"] != rm["hash"]:
                continue
            fd = (rp["image"] @ wts - rm["image"] @ wts) / (2 * h)
            assert abs(fd - g_o[k]) <= 1e-5 * max(1.0, abs(g_o[k])) + 1e-7, (k, fd, g_o[k])
            checked += 1
            break
    assert checked >= 2


def test_rotation_step_keeps_centre_and_centre_step_keeps_rotation():
    rng = np.random.default_rng(4)
    P0 = synth.perturb_normal(rng, synth.pose_from_center(np.eye(3), np.array([0.3, -0.2, 1.5])), 20.0, 0.5)
    # gradient with only rotation components (in the T x SO(3) frame g_o = -R^T g_rho = 0)
    P = P0.copy()[None]
    m = np.zeros((1, 6)); v = np.zeros((1, 6))
    oracle.pose_adam_txso3(P, m, v, np.array([[0, 0, 0, 0.3, -0.2, 0.1]]), 0.05, 1)
    assert np.abs(_centre(P[0]) - _centre(P0)).max() < 1e-14
    assert np.abs(P[0, :9] - P0[:9]).max() > 1e-3
    # gradient with only translation components: the centre moves by -lr sign(g_o)
    P = P0.copy()[None]
    m = np.zeros((1, 6)); v = np.zeros((1, 6))
    g_rho = np.array([0.2, -0.5, 0.7])
    oracle.pose_adam_txso3(P, m, v, np.concatenate([g_rho, np.zeros(3)])[None], 0.05, 1)
    R0 = P0[:9].reshape(3, 3)
    g_o = -R0.T @ g_rho
    assert np.array_equal(P[0, :9], P0[:9])
    # |step| = lr |g| / (|g| + eps) with eps = 1e-8
    np.testing.assert_allclose(_centre(P[0]) - _centre(P0), -0.05 * np.sign(g_o), rtol=1e-6, atol=1e-12)
