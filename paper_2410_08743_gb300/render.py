"""PyTorch-facing wrapper of libgsplat: device memory, streams and autograd.

`Renderer` owns a library context and a forward-state object; `render`
is a torch.autograd.Function whose backward calls the library's backward and
returns the gradients of every Gaussian parameter and, through a zero tangent
tensor `tau` of shape [V, 6], the per-view se(3) pose gradient (left
perturbation, tau = (rho, phi); Sec. 3.2, Eq. 7-13).  The rendering is always
evaluated at tau = 0: the poses tensor carries the current pose and
`pose_step` applies updates T <- Exp(delta) T on the device.
"""
from __future__ import annotations

import torch

from . import _lib as L


def _f32(t):
    return t.detach().contiguous().float()


class Renderer:
    """One library context plus one forward state, on one CUDA device."""

    def __init__(self, device: int = 0, **opts):
        self.device = int(device)
        self.ctx = L.gs_ctx_create(self.device)
        self.frames = L.gs_frames_create(self.ctx)
        self.opts = L.gs_default_opts(**opts)
        self._views_key = None
        self._views_arr = None

    def close(self):
        if getattr(self, "frames", None):
            L.gs_frames_destroy(self.frames)
            self.frames = None
        if getattr(self, "ctx", None):
            L.gs_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def views(self, views):
        key = tuple((float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"]), int(v["width"]),
                     int(v["height"])) for v in views)
        if key != self._views_key:
            self._views_arr = L.views_array(views)
            self._views_key = key
        return self._views_arr

    @staticmethod
    def image_numel(views) -> int:
        return sum(3 * int(v["width"]) * int(v["height"]) for v in views)

    def set_flags(self, flags: int):
        self.opts.flags = int(flags)

    def forward(self, params: dict, views, poses, target=None, loss_out=None, image=None, stream=None):
        """Renders all views; params holds device tensors means, scales,
        quats, opac, sh and the int sh_degree.  Returns the packed image."""
        dev = params["means"].device
        if image is None:
            image = torch.empty(self.image_numel(views), device=dev, dtype=torch.float32)
        sc = L.gs_scene_borrow(params["means"], params["scales"], params["quats"], params["opac"], params["sh"],
                               params["sh_degree"])
        try:
            L.gs_render_forward(self.ctx, sc, self.views(views), len(views), poses, self.opts, self.frames, image,
                                target=target, loss_out=loss_out, stream=stream)
        finally:
            L.gs_scene_free(sc)
        return image

    def backward(self, params: dict, views, poses, image, loss, grads: dict | None = None, pose_grad=None,
                 stream=None):
        """Back-propagates `loss` (an L.gs_loss).  grads: dict of device
        tensors shaped like params (accumulated into); pose_grad: [V, 6] f64."""
        sc = L.gs_scene_borrow(params["means"], params["scales"], params["quats"], params["opac"], params["sh"],
                               params["sh_degree"])
        g = None
        if grads is not None:
            g = L.make_grads(grads.get("means"), grads.get("scales"), grads.get("quats"), grads.get("opac"),
                             grads.get("sh"))
        try:
            L.gs_render_backward(self.ctx, sc, self.views(views), len(views), poses, self.opts, self.frames, image,
                                 loss, g, pose_grad, stream=stream)
        finally:
            L.gs_scene_free(sc)

    def pose_step(self, poses, m, v, grad, lr, step, **kw):
        L.gs_pose_step(self.ctx, poses, m, v, grad, lr, step, **kw)

    def status(self):
        return L.gs_status(self.ctx)

    def query(self, what: int):
        return L.gs_frames_query(self.frames, what)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opac, sh, tau, renderer, views, poses, sh_degree):
        params = dict(means=_f32(means), scales=_f32(scales), quats=_f32(quats), opac=_f32(opac), sh=_f32(sh),
                      sh_degree=int(sh_degree))
        poses = poses.detach().contiguous().double()
        image = renderer.forward(params, views, poses)
        ctx.renderer = renderer
        ctx.views = views
        ctx.params = params
        ctx.poses = poses
        ctx.save_for_backward(image)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        (image,) = ctx.saved_tensors
        p = ctx.params
        r = ctx.renderer
        dldc = grad_image.contiguous().float()
        grads = {k: torch.zeros_like(p[k]) for k in ("means", "scales", "quats", "opac", "sh")}
        pose_grad = torch.zeros(len(ctx.views), 6, device=image.device, dtype=torch.float64)
        loss = L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc)
        r.backward(p, ctx.views, ctx.poses, image, loss, grads, pose_grad)
        return (grads["means"], grads["scales"], grads["quats"], grads["opac"], grads["sh"], pose_grad,
                None, None, None, None)


def render(renderer: Renderer, params: dict, views, poses, tau=None):
    """Differentiable render.  params: dict of tensors (means [N,3], scales
    [N,3], quats [N,4], opac [N], sh [N,16,3], sh_degree).  tau: optional zero
    tensor [V, 6] (float64) whose gradient is the per-view pose gradient."""
    V = len(views)
    if tau is None:
        tau = torch.zeros(V, 6, device=params["means"].device, dtype=torch.float64)
    return _RenderFn.apply(params["means"], params["scales"], params["quats"], params["opac"], params["sh"], tau,
                           renderer, views, poses, params["sh_degree"])
