"""Joint refinement of Gaussians and camera poses (Sec. 3.3, Sec. 4.1).

Each iteration renders a batch of views (one in the paper's setting), evaluates
the photometric loss (w_l1 L1 + w_dssim D-SSIM, Eq. 16), back-propagates to
every Gaussian parameter and to the views' poses in one fused library call
(gs_step), then takes an Adam step on the raw Gaussian parameters
(gs_gaussian_adam) and a tangent-space Adam step on the poses of the rendered
views (gs_pose_step, T <- Exp(delta) T).  The camera learning rate follows a
cosine schedule from lr_start to lr_end over the run (Sec. 4.1).

Everything stays on the device; this module only holds the buffers and passes
pointers (no CPU arithmetic on the path)."""
from __future__ import annotations

import math

import torch

from . import _lib as L
from . import dist as D
from .render import Renderer

DEFAULT_GAUSSIAN_LRS = dict(means=1.6e-4, scales=5e-3, quats=1e-3, opac=5e-2, sh_dc=2.5e-3, sh_rest=1.25e-4)


def cosine_lr(it: int, total: int, lr_start: float, lr_end: float) -> float:
    """Cosine decay from lr_start at it = 0 to lr_end at it = total - 1."""
    if total <= 1:
        return lr_start
    c = 0.5 * (1.0 + math.cos(math.pi * min(it, total - 1) / (total - 1)))
    return lr_end + (lr_start - lr_end) * c


class JointRefiner:
    """raw: device float32 tensors means [N,3], log_scales [N,3], quats [N,4],
    logit_opac [N], sh [N,16,3]; poses: device float64 [V,12] (world->camera,
    updated in place); targets: device float32, the views' planar images packed
    in view order (or a list of them, one per view).  An iteration takes a
    contiguous range of views (one view in the paper's setting; a batch of
    frames for a trajectory).  With a process group of several ranks each rank passes its own
    views (dist.shard_views) and the same Gaussians; the Gaussian gradient is
    summed over the ranks before the (identical) Adam step."""

    def __init__(self, renderer: Renderer, raw: dict, sh_degree: int, views: list, poses: torch.Tensor,
                 targets: list, w_l1: float = 0.8, w_dssim: float = 0.2, gaussian_lrs: dict | None = None,
                 pose_lr: tuple = (1e-2, 1e-4), iterations: int = 1000, refine_gaussians: bool = True,
                 group=None, aniso_r: float | None = None, lambda_aniso: float = 0.0, lambda_opacity: float = 0.0,
                 opacity_l1_iters: int = 10000, refine_poses: bool = True, spatial_order: bool = False):
        self.r = renderer
        self.perm = None
        if spatial_order:
            # Gaussians in Morton order of their means (a layout step: the same
            # scene, better locality in every per-(view, Gaussian) pass);
            # self.perm[j] is the caller's index of row j
            n0 = raw["means"].shape[0]
            self.perm = torch.empty(n0, dtype=torch.int32, device=raw["means"].device)
            L.gs_spatial_order(renderer.ctx, raw["means"], self.perm)
            names = [("means", 3), ("log_scales", 3), ("quats", 4), ("logit_opac", 1), ("sh", 48)]
            out = {k: torch.empty_like(raw[k]) for k, _ in names}
            L.gs_gather_rows(renderer.ctx, self.perm, [raw[k] for k, _ in names], [out[k] for k, _ in names],
                             [w for _, w in names])
            raw = out
        self.raw = raw
        self.deg = int(sh_degree)
        self.views = views
        self.poses = poses
        if isinstance(targets, (list, tuple)):
            targets = torch.cat([t.reshape(-1) for t in targets])
        self.targets = targets
        self.img_off = [0]
        for vw in views:
            self.img_off.append(self.img_off[-1] + 3 * vw["width"] * vw["height"])
        if targets.numel() != self.img_off[-1]:
            raise ValueError("targets do not match the views")
        self.w_l1, self.w_dssim = float(w_l1), float(w_dssim)
        self.lrs = dict(DEFAULT_GAUSSIAN_LRS if gaussian_lrs is None else gaussian_lrs)
        self.pose_lr = pose_lr
        self.iterations = int(iterations)
        self.refine_gaussians = refine_gaussians
        self.refine_poses = refine_poses
        # Sec. 3.3 regularisers: anisotropy hinge (Eq. 17) and, for the first
        # opacity_l1_iters iterations, an L1 term on the opacities
        self.aniso_r = aniso_r
        self.lambda_aniso = float(lambda_aniso) if aniso_r is not None else 0.0
        self.lambda_opacity = float(lambda_opacity)
        self.opacity_l1_iters = int(opacity_l1_iters)
        dev = raw["means"].device
        n = raw["means"].shape[0]
        self.n = n
        # gradients in one flat buffer: with several ranks (each rendering its
        # own views of the replicated Gaussians) it is summed in one all-reduce
        self.group = group
        self.flat = D.FlatGrads(n, dev)
        self.grads = self.flat.as_dict()
        self.gm = torch.zeros(59 * n, device=dev)
        self.gv = torch.zeros(59 * n, device=dev)
        # activated parameters the renderer reads, written by the Adam kernel:
        # a zero-learning-rate step with zero gradients only activates
        self.scales = torch.empty_like(raw["log_scales"])
        self.opac = torch.empty_like(raw["logit_opac"])
        L.gs_gaussian_adam(self.r.ctx, self.raw, self.scales, self.opac, self.grads, self.gm, self.gv,
                           {k: 0.0 for k in self.lrs}, 1, self.deg)
        V = len(views)
        self.pm = torch.zeros(V, 6, dtype=torch.float64, device=dev)
        self.pv = torch.zeros(V, 6, dtype=torch.float64, device=dev)
        self.pose_steps = [0] * V    # per view: Adam steps taken on its pose
        self.pose_grad = torch.zeros(V, 6, dtype=torch.float64, device=dev)
        self.loss = torch.zeros(V, dtype=torch.float64, device=dev)
        self.image = {}
        self.it = 0
        self.gstep = 0

    def _desc(self):
        return L.scene_desc(self.raw["means"], self.scales, self.raw["quats"], self.opac, self.raw["sh"], self.deg)

    def step(self, v0: int, v1: int | None = None) -> None:
        """One iteration on views [v0, v1) (default: the single view v0): fused
        forward + loss + backward, then the Gaussian and pose Adam steps.
        Asynchronous on the current stream."""
        v1 = v0 + 1 if v1 is None else v1
        views = self.views[v0:v1]
        nv = v1 - v0
        n_img = self.img_off[v1] - self.img_off[v0]
        img = self.image.get(n_img)
        if img is None:
            img = self.image[n_img] = torch.empty(n_img, device=self.raw["means"].device)
        kind = L.GS_LOSS_L1_DSSIM if self.w_dssim != 0.0 else L.GS_LOSS_L1
        loss = L.make_loss(kind, target=self.targets[self.img_off[v0]:self.img_off[v1]], w_l1=self.w_l1,
                           w_dssim=self.w_dssim)
        grads = L.make_grads(**self.grads) if self.refine_gaussians else None
        pose = self.poses[v0:v1]
        pg = self.pose_grad[v0:v1]
        L.gs_step(self.r.ctx, self.r.frames, self._desc(), L.views_array(views), nv, L._ptr(pose), self.r.opts,
                  loss, L._ptr(img), grads, L._ptr(pg), L._ptr(self.loss[v0:v1]))
        if self.refine_gaussians:
            D.allreduce_grads(self.flat, self.group)
            lam_op = self.lambda_opacity if self.it < self.opacity_l1_iters else 0.0
            if self.lambda_aniso != 0.0 or lam_op != 0.0:
                L.gs_regularize(self.r.ctx, self.scales, self.opac, self.aniso_r or 1.0, self.lambda_aniso, lam_op,
                                self.grads["scales"], self.grads["opac"])
            self.gstep += 1
            L.gs_gaussian_adam(self.r.ctx, self.raw, self.scales, self.opac, self.grads, self.gm, self.gv, self.lrs,
                               self.gstep, self.deg)
        if self.refine_poses:
            steps = self.pose_steps[v0:v1]
            if min(steps) != max(steps):
                raise ValueError("a batch's poses must have taken the same number of steps")
            for k in range(v0, v1):
                self.pose_steps[k] += 1
            lr = cosine_lr(self.it, self.iterations, *self.pose_lr)
            L.gs_pose_step(self.r.ctx, pose, self.pm[v0:v1], self.pv[v0:v1], pg, lr, self.pose_steps[v0])
        self.it += 1

    def autotune(self, v0: int = 0, v1: int | None = None, repeats: int = 1) -> dict:
        """Picks the renderer's result-neutral launch parameters for iterations
        over views [v0, v1) (tune.autotune, cached per workload class)."""
        from . import tune
        v1 = v0 + 1 if v1 is None else v1
        views = self.views[v0:v1]
        params = dict(means=self.raw["means"], scales=self.scales, quats=self.raw["quats"], opac=self.opac,
                      sh=self.raw["sh"], sh_degree=self.deg)
        n_img = self.img_off[v1] - self.img_off[v0]
        img = self.image.get(n_img)
        if img is None:
            img = self.image[n_img] = torch.empty(n_img, device=self.raw["means"].device)
        kind = L.GS_LOSS_L1_DSSIM if self.w_dssim != 0.0 else L.GS_LOSS_L1
        loss = L.make_loss(kind, target=self.targets[self.img_off[v0]:self.img_off[v1]], w_l1=self.w_l1,
                           w_dssim=self.w_dssim)
        # the tuner's trial steps accumulate into scratch gradients, not the refiner's
        scratch = D.FlatGrads(self.n, self.raw["means"].device)
        self.r.forward(params, views, self.poses[v0:v1], image=img)
        return tune.autotune(self.r, params, views, self.poses[v0:v1], img, loss, scratch.as_dict(),
                             self.pose_grad[v0:v1], repeats=repeats)

    def prune(self, n_target: int, min_opacity: float = 0.005) -> int:
        """Adaptive opacity pruning (Sec. 3.3): removes the Gaussians whose
        opacity is at or below the threshold that leaves at most n_target of
        them (and at least min_opacity), from the parameters, their activated
        copies and both Adam moments.  Returns the new count."""
        thr, keep = L.gs_prune_threshold(self.r.ctx, self.opac, n_target, min_opacity)
        if keep == self.n:
            return keep
        n, k = self.n, keep
        dev = self.raw["means"].device
        widths = [("means", 3), ("log_scales", 3), ("quats", 4), ("logit_opac", 1), ("sh", 48)]
        src, dst, w = [], [], []
        new_raw = {}
        for name, wd in widths:
            t = self.raw[name]
            new_raw[name] = torch.empty((k,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
            src.append(t); dst.append(new_raw[name]); w.append(wd)
        new_scales = torch.empty(k, 3, device=dev)
        new_opac = torch.empty(k, device=dev)
        src += [self.scales, self.opac]; dst += [new_scales, new_opac]; w += [3, 1]
        gm = torch.empty(59 * k, device=dev)
        gv = torch.empty(59 * k, device=dev)
        off = 0
        for _, wd in widths:       # the moments are group-major: [3n | 3n | 4n | n | 48n]
            src += [self.gm[off * n:(off + wd) * n], self.gv[off * n:(off + wd) * n]]
            dst += [gm[off * k:(off + wd) * k], gv[off * k:(off + wd) * k]]
            w += [wd, wd]
            off += wd
        got = L.gs_compact(self.r.ctx, self.opac, thr, src, dst, w)
        assert got == k
        self.raw, self.scales, self.opac, self.gm, self.gv, self.n = new_raw, new_scales, new_opac, gm, gv, k
        self.flat = D.FlatGrads(k, dev)
        self.grads = self.flat.as_dict()
        return k

    def run(self, order=None, batch: int = 1) -> None:
        """The remaining iterations, cycling through the views in batches of
        `batch` consecutive views (or through `order`, a list of view indices,
        one per iteration)."""
        V = len(self.views)
        nb = (V + batch - 1) // batch
        for k in range(self.iterations - self.it):
            if order is not None:
                self.step(order[k % len(order)])
            else:
                b = self.it % nb
                self.step(b * batch, min(V, (b + 1) * batch))
