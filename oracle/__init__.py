"""FP64 CPU oracle of the pose-differentiable Gaussian-splatting renderer.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by
the benchmark's CPU-baseline leg, never by the product path.  It is a ctypes
binding of gs_oracle.c (plain C, FP64), which follows the paper's Sec. 3.1
(Eq. 1-4: projection, EWA covariance, alpha, SH colour, compositing) and
Sec. 3.2 (Eq. 5-13: the tangent-space pose gradient of a left perturbation).

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, brute force, library routines or central finite differences.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

F32P = C.POINTER(C.c_float)
F64P = C.POINTER(C.c_double)
I32P = C.POINTER(C.c_int32)
U8P = C.POINTER(C.c_uint8)
U32P = C.POINTER(C.c_uint32)
U64P = C.POINTER(C.c_uint64)


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int), ("sh_degree", C.c_int), ("means", F32P), ("scales", F32P),
                ("quats", F32P), ("opac", F32P), ("sh", F32P)]


class _Cam(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int), ("pose", C.c_double * 12)]


class _Opts(C.Structure):
    _fields_ = [("bg", C.c_double * 3), ("z_near", C.c_float), ("eps2d", C.c_float),
                ("clamp_factor", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float)]


DEFAULT_OPTS = dict(bg=(0.0, 0.0, 0.0), z_near=0.2, eps2d=0.3, clamp_factor=1.3,
                    alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_render.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Cam), C.POINTER(_Opts), C.c_int,
                                F64P, F64P, I32P, U8P, U64P]
        L.or_render.restype = C.c_int
        L.or_keys.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Cam), C.POINTER(_Opts),
                              U8P, F32P, F32P, I32P, I32P, U32P, U32P, C.c_int64]
        L.or_keys.restype = C.c_int64
        L.or_project_values.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Cam), C.POINTER(_Opts), F64P]
        L.or_backward.argtypes = [C.POINTER(_Scene), C.c_int, C.POINTER(_Cam), C.POINTER(_Opts), F64P,
                                  F64P, F64P, F64P, F64P, F64P, F64P, F64P, U8P]
        L.or_backward.restype = C.c_int
        L.or_loss_l1.argtypes = [C.c_int, I32P, F64P, F32P, C.c_double, F64P, U8P]
        L.or_loss_l1.restype = C.c_double
        L.or_loss_l1_masked.argtypes = [C.c_int, I32P, F64P, F32P, F64P, C.c_double, C.c_double, F64P, U8P]
        L.or_loss_l1_masked.restype = C.c_double
        L.or_loss_dssim.argtypes = [C.c_int, I32P, F64P, F32P, C.c_double, F64P, F64P]
        L.or_loss_dssim.restype = C.c_double
        L.or_loss_dssim_cond.argtypes = [C.c_int, I32P, F64P, F32P, C.c_double, F64P]
        L.or_ssim_filter.argtypes = [F64P, C.c_int, C.c_int, F64P]
        L.or_sh_eval.argtypes = [F64P, C.c_int, C.c_int, F64P]
        L.or_se3_exp.argtypes = [F64P, F64P]
        L.or_se3_log.argtypes = [F64P, F64P]
        L.or_se3_left_update.argtypes = [F64P, F64P]
        L.or_pose_adam.argtypes = [C.c_int, F64P, F64P, F64P, F64P, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_int]
        L.or_pose_adam_txso3.argtypes = [C.c_int, F64P, F64P, F64P, F64P, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_int]
        L.or_unproject.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, F32P, F32P,
                                   C.c_int, F64P, F64P]
        L.or_unproject.restype = C.c_int
        L.or_knn_mean_dist.argtypes = [C.c_int, F64P, C.c_int, F64P]
        L.or_regularize.argtypes = [C.c_int, F32P, F32P, C.c_double, C.c_double, C.c_double, F64P, F64P]
        L.or_regularize.restype = C.c_double
        L.or_prune_threshold.argtypes = [C.c_int, F32P, C.c_longlong, C.c_float, C.POINTER(C.c_longlong)]
        L.or_prune_threshold.restype = C.c_float
        PP = C.POINTER(F64P)
        L.or_gaussian_adam.argtypes = [C.c_int, C.c_int, PP, PP, PP, PP, F64P, C.c_double, C.c_double, C.c_double,
                                       C.c_int, F64P, F64P]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


class _Prepared:
    """Keeps the arrays behind the ctypes structs alive."""

    def __init__(self, scene, views, poses, opts):
        self.arrs = dict(
            means=np.ascontiguousarray(scene["means"], np.float32),
            scales=np.ascontiguousarray(scene["scales"], np.float32),
            quats=np.ascontiguousarray(scene["quats"], np.float32),
            opac=np.ascontiguousarray(scene["opac"], np.float32),
            sh=np.ascontiguousarray(scene["sh"], np.float32))
        a = self.arrs
        self.scene = _Scene(len(a["opac"]), int(scene["sh_degree"]), _p(a["means"], F32P),
                            _p(a["scales"], F32P), _p(a["quats"], F32P), _p(a["opac"], F32P),
                            _p(a["sh"], F32P))
        poses = np.asarray(poses, np.float64).reshape(len(views), 12)
        self.V = len(views)
        self.cams = (_Cam * max(1, self.V))()
        for k, v in enumerate(views):
            c = self.cams[k]
            c.fx, c.fy, c.cx, c.cy = v["fx"], v["fy"], v["cx"], v["cy"]
            c.width, c.height = v["width"], v["height"]
            for j in range(12):
                c.pose[j] = float(poses[k, j])
        o = dict(DEFAULT_OPTS)
        o.update(opts or {})
        self.opts = _Opts((C.c_double * 3)(*o["bg"]), o["z_near"], o["eps2d"], o["clamp_factor"],
                          o["alpha_min"], o["alpha_max"], o["t_min"])
        self.n_img = sum(3 * v["width"] * v["height"] for v in views)
        self.n_pix = sum(v["width"] * v["height"] for v in views)
        self.wh = np.array([[v["width"], v["height"]] for v in views], np.int32).reshape(-1)
        self.n = len(a["opac"])


def render(scene, views, poses, opts=None, brute=False):
    """Forward render.  Returns dict(image f64 [sum 3HW], T_final f64 [sum HW],
    n_contrib i32 [sum HW], fragile u8 [sum HW], hash int)."""
    P = _Prepared(scene, views, poses, opts)
    img = np.zeros(P.n_img, np.float64)
    T = np.zeros(P.n_pix, np.float64)
    nc = np.zeros(P.n_pix, np.int32)
    fr = np.zeros(P.n_pix, np.uint8)
    h = C.c_uint64(0)
    rc = lib().or_render(C.byref(P.scene), P.V, P.cams, C.byref(P.opts), int(brute), _p(img, F64P),
                         _p(T, F64P), _p(nc, I32P), _p(fr, U8P), C.byref(h))
    if rc != 0:
        raise MemoryError("oracle render failed")
    return dict(image=img, T_final=T, n_contrib=nc, fragile=fr, hash=int(h.value))


def keys(scene, views, poses, opts=None):
    """Key path and tile lists.  Returns dict(valid, depth, mu2f, radius, rect,
    ranges [total_tiles,2], idx [K])."""
    P = _Prepared(scene, views, poses, opts)
    VN = P.V * P.n
    valid = np.zeros(VN, np.uint8); depth = np.zeros(VN, np.float32)
    mu2f = np.zeros(2 * VN, np.float32); radius = np.zeros(VN, np.int32); rect = np.zeros(4 * VN, np.int32)
    tiles = sum(((v["width"] + 15) // 16) * ((v["height"] + 15) // 16) for v in views)
    ranges = np.zeros(2 * tiles, np.uint32)
    K = lib().or_keys(C.byref(P.scene), P.V, P.cams, C.byref(P.opts), _p(valid, U8P), _p(depth, F32P),
                      _p(mu2f, F32P), _p(radius, I32P), _p(rect, I32P), _p(ranges, U32P), None, 0)
    idx = np.zeros(max(K, 1), np.uint32)
    K2 = lib().or_keys(C.byref(P.scene), P.V, P.cams, C.byref(P.opts), None, None, None, None, None,
                       None, _p(idx, U32P), K)
    assert K == K2
    return dict(valid=valid, depth=depth, mu2f=mu2f.reshape(-1, 2), radius=radius, rect=rect.reshape(-1, 4),
                ranges=ranges.reshape(-1, 2), idx=idx[:K], n_keys=int(K))


def project_values(scene, views, poses, opts=None):
    """FP64 [V*N, 9]: mu_hat(2), conic(3), opacity, colour(3)."""
    P = _Prepared(scene, views, poses, opts)
    out = np.zeros(P.V * P.n * 9, np.float64)
    lib().or_project_values(C.byref(P.scene), P.V, P.cams, C.byref(P.opts), _p(out, F64P))
    return out.reshape(-1, 9)


def backward(scene, views, poses, dldc, opts=None, want_g2d=False):
    """Analytic backward given dL/dC.  Returns dict(means, scales, quats, opac,
    sh, pose [V,6] (rho, phi), fragile_g [V*N], g2d [V*N, 9] optional)."""
    P = _Prepared(scene, views, poses, opts)
    n = P.n
    g = dict(means=np.zeros((n, 3)), scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opac=np.zeros(n), sh=np.zeros((n, 16, 3)), pose=np.zeros((P.V, 6)))
    fr = np.zeros(P.V * n, np.uint8)
    g2d = np.zeros((P.V * n, 9)) if want_g2d else None
    d = np.ascontiguousarray(dldc, np.float64)
    assert d.size == P.n_img
    rc = lib().or_backward(C.byref(P.scene), P.V, P.cams, C.byref(P.opts), _p(d, F64P),
                           _p(g["means"], F64P), _p(g["scales"], F64P), _p(g["quats"], F64P),
                           _p(g["opac"], F64P), _p(g["sh"], F64P), _p(g["pose"], F64P),
                           _p(g2d, F64P), _p(fr, U8P))
    if rc != 0:
        raise MemoryError("oracle backward failed")
    g["fragile_g"] = fr
    if want_g2d:
        g["g2d"] = g2d
    return g


def _wh(views):
    return np.array([[v["width"], v["height"]] for v in views], np.int32).reshape(-1)


def loss_l1(views, image, target, weight=1.0):
    """Returns (loss, dL/dC f64, fragile_px u8)."""
    img = np.ascontiguousarray(image, np.float64)
    tgt = np.ascontiguousarray(target, np.float32)
    d = np.zeros_like(img)
    fr = np.zeros(sum(v["width"] * v["height"] for v in views), np.uint8)
    wh = _wh(views)
    L = lib().or_loss_l1(len(views), _p(wh, I32P), _p(img, F64P), _p(tgt, F32P), float(weight),
                         _p(d, F64P), _p(fr, U8P))
    return L, d, fr


def loss_l1_masked(views, image, target, T_final, mask_alpha=0.99, weight=1.0):
    """Confidence-masked L1 (Sec. 3.4, Eq. 20-21).  mask_alpha is taken as an
    FP32 number, the type the library's loss descriptor holds it in.  Returns
    (loss, dL/dC f64, fragile_px u8)."""
    img = np.ascontiguousarray(image, np.float64)
    tgt = np.ascontiguousarray(target, np.float32)
    T = np.ascontiguousarray(T_final, np.float64)
    d = np.zeros_like(img)
    fr = np.zeros(sum(v["width"] * v["height"] for v in views), np.uint8)
    assert T.size == fr.size
    wh = _wh(views)
    L = lib().or_loss_l1_masked(len(views), _p(wh, I32P), _p(img, F64P), _p(tgt, F32P), _p(T, F64P),
                                float(np.float32(mask_alpha)), float(weight), _p(d, F64P), _p(fr, U8P))
    return L, d, fr


def loss_dssim(views, image, target, weight=1.0):
    """Returns (loss, dL/dC f64, ssim map f64)."""
    img = np.ascontiguousarray(image, np.float64)
    tgt = np.ascontiguousarray(target, np.float32)
    d = np.zeros_like(img)
    smap = np.zeros_like(img)
    wh = _wh(views)
    L = lib().or_loss_dssim(len(views), _p(wh, I32P), _p(img, F64P), _p(tgt, F32P), float(weight),
                            _p(d, F64P), _p(smap, F64P))
    return L, d, smap


def loss_dssim_cond(views, image, target, weight=1.0):
    """Per element, the sum of the magnitudes of the terms that loss_dssim's
    dL/dC adds up (a conditioning diagnostic for tolerances: a computation
    that rounds each term k times with unit roundoff u is off by about
    k u cond)."""
    img = np.ascontiguousarray(image, np.float64)
    tgt = np.ascontiguousarray(target, np.float32)
    out = np.zeros_like(img)
    wh = _wh(views)
    lib().or_loss_dssim_cond(len(views), _p(wh, I32P), _p(img, F64P), _p(tgt, F32P), float(weight), _p(out, F64P))
    return out


def ssim_filter(plane):
    x = np.ascontiguousarray(plane, np.float64)
    H, W = x.shape
    out = np.zeros_like(x)
    lib().or_ssim_filter(_p(x, F64P), W, H, _p(out, F64P))
    return out


def sh_eval(dirs, deg=3):
    d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((len(d), 16))
    lib().or_sh_eval(_p(d, F64P), len(d), int(deg), _p(out, F64P))
    return out


def se3_exp(tau):
    t = np.ascontiguousarray(tau, np.float64)
    T = np.zeros(12)
    lib().or_se3_exp(_p(t, F64P), _p(T, F64P))
    return T


def se3_log(T):
    x = np.ascontiguousarray(T, np.float64)
    tau = np.zeros(6)
    lib().or_se3_log(_p(x, F64P), _p(tau, F64P))
    return tau


def se3_left_update(tau, T):
    t = np.ascontiguousarray(tau, np.float64)
    x = np.array(T, np.float64)
    lib().or_se3_left_update(_p(t, F64P), _p(x, F64P))
    return x


def unproject(view, depth, image, stride):
    """Sec. 3.4 unprojection.  Returns (points [n,3] f64, colours [n,3] f64)."""
    W, H = view["width"], view["height"]
    dp = np.ascontiguousarray(depth, np.float32).reshape(-1)
    im = np.ascontiguousarray(image, np.float32).reshape(-1) if image is not None else None
    cap = ((W + stride - 1) // stride) * ((H + stride - 1) // stride)
    pts = np.zeros((cap, 3)); cols = np.zeros((cap, 3))
    n = lib().or_unproject(W, H, float(view["fx"]), float(view["fy"]), float(view["cx"]), float(view["cy"]),
                           _p(dp, F32P), _p(im, F32P), int(stride), _p(pts, F64P), _p(cols, F64P))
    return pts[:n], cols[:n]


def knn_mean_dist(points, k=3):
    p = np.ascontiguousarray(points, np.float64).reshape(-1, 3)
    out = np.zeros(len(p))
    lib().or_knn_mean_dist(len(p), _p(p, F64P), int(k), _p(out, F64P))
    return out


def regularize(scales, opac, r, lam_aniso, lam_opacity):
    """Eq. 17 anisotropy hinge + opacity L1.  Returns (value, g_scales [n,3],
    g_opac [n])."""
    sc = np.ascontiguousarray(scales, np.float32).reshape(-1, 3)
    op = np.ascontiguousarray(opac, np.float32).reshape(-1)
    gs_ = np.zeros((len(sc), 3)); go = np.zeros(len(op))
    val = lib().or_regularize(len(sc), _p(sc, F32P), _p(op, F32P), float(r), float(lam_aniso), float(lam_opacity),
                              _p(gs_, F64P), _p(go, F64P))
    return val, gs_, go


def prune_threshold(opac, n_target, min_opacity):
    """Returns (threshold, n_keep) of the adaptive pruning rule."""
    op = np.ascontiguousarray(opac, np.float32).reshape(-1)
    nk = C.c_longlong(0)
    t = lib().or_prune_threshold(len(op), _p(op, F32P), int(n_target), float(min_opacity), C.byref(nk))
    return float(t), int(nk.value)


def pose_adam_txso3(poses, m, v, grad, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """T x SO(3) step (Sec. 4.2) in place on poses [V,12], m, v [V,6]; grad is
    the left-SE(3) gradient [V,6]."""
    V = len(poses)
    g = np.ascontiguousarray(grad, np.float64)
    lib().or_pose_adam_txso3(V, _p(poses, F64P), _p(m, F64P), _p(v, F64P), _p(g, F64P), float(lr), float(b1),
                             float(b2), float(eps), int(step))


def pose_adam(poses, m, v, grad, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """In place on poses [V,12], m, v [V,6]."""
    V = len(poses)
    g = np.ascontiguousarray(grad, np.float64)
    lib().or_pose_adam(V, _p(poses, F64P), _p(m, F64P), _p(v, F64P), _p(g, F64P), float(lr), float(b1),
                       float(b2), float(eps), int(step))


ADAM_GROUPS = ("means", "log_scales", "quats", "logit_opac", "sh")
GRAD_GROUPS = ("means", "scales", "quats", "opac", "sh")


def gaussian_adam(raw, grads, m, v, lrs, step, sh_degree, b1=0.9, b2=0.999, eps=1e-15):
    """In place on the float64 dicts raw, m, v (keys ADAM_GROUPS, arrays
    [n, width]); grads keyed by GRAD_GROUPS.  Returns (scales, opacities)."""
    n = len(raw["means"])
    arrs = {}
    def ptrs(d, keys):
        out = (F64P * 5)()
        for j, k in enumerate(keys):
            a = np.ascontiguousarray(d[k], np.float64)
            assert a.flags.c_contiguous
            d[k] = a
            out[j] = _p(a, F64P)
        return out
    g = {k: np.ascontiguousarray(grads[k], np.float64) for k in GRAD_GROUPS}
    pr, pg, pm, pv = ptrs(raw, ADAM_GROUPS), ptrs(g, GRAD_GROUPS), ptrs(m, ADAM_GROUPS), ptrs(v, ADAM_GROUPS)
    lr = np.array([lrs["means"], lrs["scales"], lrs["quats"], lrs["opac"], lrs["sh_dc"], lrs["sh_rest"]], np.float64)
    sc = np.zeros((n, 3)); op = np.zeros(n)
    lib().or_gaussian_adam(n, int(sh_degree), pr, pg, pm, pv, _p(lr, F64P), b1, b2, eps, int(step), _p(sc, F64P),
                           _p(op, F64P))
    return sc, op


def image_to_hwc(image, views, v):
    """View v's planar image as [H, W, 3] (test helper)."""
    off = sum(3 * u["width"] * u["height"] for u in views[:v])
    W, H = views[v]["width"], views[v]["height"]
    return image[off:off + 3 * W * H].reshape(3, H, W).transpose(1, 2, 0)
