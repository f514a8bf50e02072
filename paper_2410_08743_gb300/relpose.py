"""Relative pose between nearby frames (Sec. 3.4), the initialisation of
reconstruction without pose information.

For frames I_t, I_{t+1} and a depth map of I_t (a monocular estimate in the
paper; any z-depth map here):
1. a subset of I_t's pixels is unprojected into camera points, each becoming
   an isotropic Gaussian with the pixel's colour and the mean distance to its
   three nearest neighbours as scale (gs_unproject, gs_knn_mean_dist,
   gs_init_from_points);
2. these Gaussians are fitted to I_t with the photometric loss for a few
   steps (the paper reports under 100), camera fixed at the identity
   (JointRefiner with refine_poses=False);
3. the pose of I_{t+1} relative to I_t is found by minimising the
   confidence-masked L1 (Eq. 20-21) between the fitted Gaussians rendered at
   the pose and I_{t+1}, by Adam on the pose alone (gs_step pose-only +
   gs_pose_step).

All arithmetic runs in the library's kernels; this module owns the buffers
and the loop."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L
from .joint import JointRefiner, cosine_lr
from .render import Renderer

IDENTITY = np.concatenate([np.eye(3).reshape(9), np.zeros(3)])


def gaussians_from_depth(r: Renderer, view: dict, image, depth, stride: int = 2, k: int = 3,
                         opacity: float = 0.5, min_scale: float = 1e-4) -> dict:
    """Raw parameters (device) of the isotropic Gaussians of step 1; the
    frame's camera frame is the world frame.  The paper gives no initial
    opacity: the masked loss of step 3 only counts pixels whose accumulated
    alpha exceeds 0.99, which a fit of about 100 steps reaches from 0.5 but
    hardly from the prior art's 0.1 (the mask stays almost empty)."""
    dev = depth.device
    gw = (view["width"] + stride - 1) // stride
    gh = (view["height"] + stride - 1) // stride
    pts = torch.empty(gw * gh, 3, device=dev)
    cols = torch.empty(gw * gh, 3, device=dev)
    n = L.gs_unproject(r.ctx, view, depth, image, stride, pts, cols)
    pts, cols = pts[:n].contiguous(), cols[:n].contiguous()
    dist = torch.empty(n, device=dev)
    L.gs_knn_mean_dist(r.ctx, pts, k, dist)
    raw = {"means": torch.empty(n, 3, device=dev), "log_scales": torch.empty(n, 3, device=dev),
           "quats": torch.empty(n, 4, device=dev), "logit_opac": torch.empty(n, device=dev),
           "sh": torch.empty(n, 16, 3, device=dev)}
    L.gs_init_from_points(r.ctx, pts, cols, dist, raw, min_scale=min_scale, opacity=opacity)
    return raw


def fit_frame(r: Renderer, raw: dict, view: dict, image, iterations: int = 100, lrs: dict | None = None,
              w_dssim: float = 0.2) -> JointRefiner:
    """Step 2: fits the Gaussians to their own frame (identity camera)."""
    dev = raw["means"].device
    P = torch.from_numpy(IDENTITY[None].copy()).to(dev)
    J = JointRefiner(r, raw, 0, [view], P, image, w_l1=1.0 - w_dssim, w_dssim=w_dssim, gaussian_lrs=lrs,
                     iterations=iterations, refine_poses=False)
    J.run()
    return J


def estimate_relative_pose(r: Renderer, J: JointRefiner, view: dict, next_image, steps: int = 200,
                           mask_alpha: float = 0.99, lr: tuple = (1e-2, 1e-4), init_pose=None,
                           param: int = L.GS_POSE_SE3) -> torch.Tensor:
    """Step 3: the world->camera pose [12] (float64, device) of the next frame
    in the fitted frame's camera coordinates."""
    dev = J.raw["means"].device
    pose = torch.from_numpy((IDENTITY if init_pose is None else np.asarray(init_pose, np.float64))[None].copy()).to(dev)
    m = torch.zeros(1, 6, dtype=torch.float64, device=dev)
    v = torch.zeros_like(m)
    g = torch.zeros_like(m)
    img = torch.empty(3 * view["width"] * view["height"], device=dev)
    desc = J._desc()
    loss = L.make_loss(L.GS_LOSS_L1_MASKED, target=next_image, w_l1=1.0, mask_alpha=mask_alpha)
    varr = L.views_array([view])
    for k in range(steps):
        L.gs_step(r.ctx, r.frames, desc, varr, 1, L._ptr(pose), r.opts, loss, L._ptr(img), None, L._ptr(g), None)
        L.gs_pose_step(r.ctx, pose, m, v, g, cosine_lr(k, steps, *lr), k + 1, param=param)
    return pose[0]
