"""Relative pose between nearby frames (Sec. 3.4) on the GPU.

* gs_unproject, gs_knn_mean_dist and gs_init_from_points against the oracle
  and the closed forms of the initial Gaussians.
* End to end on the synthetic room: frame images rendered by the oracle, the
  first frame's depth by ray casting the room; Gaussians from the depth map,
  fitted to the first frame, then the second frame's pose relative to the
  first estimated with the confidence-masked L1.  The estimate must land much
  closer to the true relative pose than the identity it starts from."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import relpose, synth
from paper_2410_08743_gb300.render import Renderer

from .gpu_util import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


@pytest.fixture(scope="module")
def frames():
    w = synth.trajectory_workload(n=300_000, n_frames=200, width=160, height=120, focal=110.0, scale=0.02)
    # a pair two frames apart on a gentle stretch (1-4 degrees of turn)
    a = next(k for k in range(100, 196) if 1.0 < _err(w["poses"][k], w["poses"][k + 2])[0] < 4.0)
    b = a + 2
    views = [w["views"][a], w["views"][b]]
    poses = w["poses"][[a, b]]
    imgs = oracle.render(w["scene"], views, poses)["image"].astype(np.float32)
    n3 = 3 * 160 * 120
    depth = synth.room_depth(w["geometry"], views[0], poses[0])
    return w, views, poses, imgs[:n3], imgs[n3:], depth


def _rel(Pa, Pb):
    """Pose of frame b in frame a's camera coordinates: T_b T_a^-1."""
    Ra, ta = Pa[:9].reshape(3, 3), Pa[9:]
    Rb, tb = Pb[:9].reshape(3, 3), Pb[9:]
    R = Rb @ Ra.T
    return np.concatenate([R.reshape(9), tb - R @ ta])


def _err(P, Q):
    Ra, Rb = P[:9].reshape(3, 3), Q[:9].reshape(3, 3)
    rot = math.degrees(math.acos(min(1.0, max(-1.0, (np.trace(Ra @ Rb.T) - 1) / 2))))
    ca, cb = -Ra.T @ P[9:], -Rb.T @ Q[9:]
    return rot, float(np.linalg.norm(ca - cb))


def test_unproject_knn_init_match_oracle(R, frames):
    w, views, poses, img0, _, depth = frames
    view = views[0]
    d = torch.from_numpy(depth).to(DEV)
    im = torch.from_numpy(img0).to(DEV)
    cap = ((160 + 1) // 2) * ((120 + 1) // 2)
    pts = torch.empty(cap, 3, device=DEV); cols = torch.empty(cap, 3, device=DEV)
    n = L.gs_unproject(R.ctx, view, d, im, 2, pts, cols)
    p_ref, c_ref = oracle.unproject(view, depth, img0, 2)
    assert n == len(p_ref) > 1000
    np.testing.assert_allclose(pts[:n].cpu().numpy(), p_ref, rtol=2e-6, atol=1e-6)
    np.testing.assert_array_equal(cols[:n].cpu().numpy().astype(np.float64), c_ref)
    pn = pts[:n].contiguous()
    dist = torch.empty(n, device=DEV)
    L.gs_knn_mean_dist(R.ctx, pn, 3, dist)
    # the oracle on the GPU's own (float) points: the neighbour search alone
    d_ref = oracle.knn_mean_dist(pn.cpu().numpy().astype(np.float64), 3)
    np.testing.assert_allclose(dist.cpu().numpy(), d_ref, rtol=2e-4, atol=1e-6)
    raw = {"means": torch.empty(n, 3, device=DEV), "log_scales": torch.empty(n, 3, device=DEV),
           "quats": torch.empty(n, 4, device=DEV), "logit_opac": torch.empty(n, device=DEV),
           "sh": torch.empty(n, 16, 3, device=DEV)}
    L.gs_init_from_points(R.ctx, pn, cols[:n].contiguous(), dist, raw, min_scale=1e-4, opacity=0.1)
    torch.cuda.synchronize()
    dd = dist.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(raw["log_scales"].cpu().numpy(), np.repeat(np.log(np.maximum(dd, 1e-4))[:, None], 3, 1),
                               rtol=1e-6, atol=1e-6)
    assert torch.equal(raw["means"], pn)
    q = raw["quats"].cpu().numpy()
    assert np.all(q[:, 0] == 1) and not q[:, 1:].any()
    np.testing.assert_allclose(raw["logit_opac"].cpu().numpy(), math.log(0.1 / 0.9), rtol=1e-6)
    sh = raw["sh"].cpu().numpy()
    C0 = 0.28209479177387814
    np.testing.assert_allclose(sh[:, 0, :] * C0 + 0.5, c_ref, atol=1e-6)
    assert not sh[:, 1:, :].any()


def test_relative_pose_end_to_end(R, frames):
    w, views, poses, img0, img1, depth = frames
    d = torch.from_numpy(depth).to(DEV)
    i0 = torch.from_numpy(img0).to(DEV)
    i1 = torch.from_numpy(img1).to(DEV)
    raw = relpose.gaussians_from_depth(R, views[0], i0, d, stride=2, opacity=0.5)
    J = relpose.fit_frame(R, raw, views[0], i0, iterations=100)
    torch.cuda.synchronize()
    fit_loss = float(J.loss[0].item())
    est = relpose.estimate_relative_pose(R, J, views[1], i1, steps=300).cpu().numpy()
    gt = _rel(poses[0], poses[1])
    rot0, tr0 = _err(relpose.IDENTITY, gt)
    rot1, tr1 = _err(est, gt)
    print(f"fit L1+DSSIM {fit_loss:.4f}; relative pose error: rotation {rot0:.3f} -> {rot1:.3f} deg, "
          f"centre {tr0:.4f} -> {tr1:.4f}")
    assert rot0 > 0.3 or tr0 > 0.02                    # the frames really moved
    assert rot1 < 0.25 * rot0 and tr1 < 0.25 * tr0
