"""Helpers shared by the GPU parity tests: move a synthetic scene to the
device, run the library's forward/backward, compare with tolerances."""
import numpy as np
import torch

from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300.render import Renderer

DEV = "cuda:0"


def to_dev(scene):
    p = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).to(DEV) for k in ("means", "scales", "quats", "opac", "sh")}
    p["sh_degree"] = int(scene["sh_degree"])
    return p


def zero_grads(p):
    return {k: torch.zeros_like(p[k]) for k in ("means", "scales", "quats", "opac", "sh")}


def poses_dev(poses):
    return torch.from_numpy(np.ascontiguousarray(poses, np.float64)).to(DEV)


def gpu_forward(r: Renderer, scene, views, poses, target=None):
    p = to_dev(scene)
    P = poses_dev(poses)
    tg = torch.from_numpy(np.ascontiguousarray(target, np.float32)).to(DEV) if target is not None else None
    loss = torch.zeros(len(views), dtype=torch.float64, device=DEV) if target is not None else None
    img = r.forward(p, views, P, target=tg, loss_out=loss)
    torch.cuda.synchronize()
    return p, P, img, tg, loss


def gpu_backward_dldc(r: Renderer, p, views, P, img, dldc):
    d = torch.from_numpy(np.ascontiguousarray(dldc, np.float32)).to(DEV)
    g = zero_grads(p)
    pg = torch.zeros(len(views), 6, dtype=torch.float64, device=DEV)
    r.backward(p, views, P, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=d), g, pg)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}, pg.cpu().numpy()


def assert_grad_close(got, ref, name, rel=1e-3, abs_floor=1e-6, frac=1.0, mask=None):
    """Per element |got - ref| <= max(rel |ref|, abs_floor) on at least `frac`
    of the elements (all by default); mask selects the compared elements."""
    got = np.asarray(got, np.float64).reshape(len(ref), -1) if np.ndim(ref) > 0 else np.asarray(got)
    ref = np.asarray(ref, np.float64).reshape(len(ref), -1)
    got = got.reshape(ref.shape)
    if mask is not None:
        got, ref = got[mask], ref[mask]
    err = np.abs(got - ref)
    tol = np.maximum(rel * np.abs(ref), abs_floor)
    ok = err <= tol
    worst = np.argsort(-(err / tol).ravel())[:5]
    msg = f"{name}: {np.mean(ok):.6f} within tol; worst (got, ref): " + ", ".join(
        f"({got.ravel()[w]:.4g}, {ref.ravel()[w]:.4g})" for w in worst)
    assert np.mean(ok) >= frac, msg
    return float(np.mean(ok))


def assert_pose_close(got, ref, name="pose", rel=1e-3, abs_floor=1e-6, slack=None):
    """The per-element rule on each of the 6 components of each view's pose
    gradient: |got - ref| <= max(rel |ref|, abs_floor) (+ slack, an upper
    bound on the share of pixels whose forward decision is near a threshold,
    where a test has such pixels)."""
    got = np.asarray(got, np.float64).reshape(-1, 6)
    ref = np.asarray(ref, np.float64).reshape(-1, 6)
    tol = np.maximum(rel * np.abs(ref), abs_floor)
    if slack is not None:
        tol = tol + np.asarray(slack, np.float64).reshape(-1, 6)
    err = np.abs(got - ref)
    ratio = err / tol
    assert np.all(err <= tol), f"{name}: worst error / tolerance {ratio.max():.3g}; got {got.tolist()}, ref {ref.tolist()}"
    return float(ratio.max())


# FP32 roundings each term of the D-SSIM gradient goes through on the GPU:
# the forward's two 11-tap filter passes (10 + 10 additions), the partials of
# SSIM (4), the backward's two filter passes (10 + 10) and the final sum (4).
DSSIM_FP32_ROUNDINGS = 48


def assert_dssim_grad_close(got, ref, cond, name):
    """The D-SSIM term's dL/dC per element:
    |got - ref| <= max(1e-3 |ref|, 1e-6 max|ref|) + 48 * 2^-24 * cond,
    cond = the oracle's sum of the magnitudes of the terms that make up the
    element (oracle.loss_dssim_cond).  The gradient at a pixel is a sum of
    terms of up to ~1/C2 that cancel to a far smaller value where the image is
    smooth, so FP32 evaluation is accurate relative to cond, not to |ref|."""
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    cond = np.asarray(cond, np.float64).ravel()
    assert got.shape == ref.shape == cond.shape
    tol = np.maximum(1e-3 * np.abs(ref), 1e-6 * np.abs(ref).max()) + DSSIM_FP32_ROUNDINGS * 2.0 ** -24 * cond
    err = np.abs(got - ref)
    r = err / tol
    k = int(np.argmax(r))
    assert np.all(err <= tol), (f"{name}: worst error / tolerance {r[k]:.3g} at {k}: {got[k]:.6g} vs {ref[k]:.6g} "
                                f"(max |ref| {np.abs(ref).max():.4g}, cond {cond[k]:.3g})")
    return float(r.max())
