"""ctypes binding of libgsplat (include/gsplat.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
tensor data pointers, sizes and the current CUDA stream straight through.  All
arithmetic happens in the library's CUDA kernels.  Importing this module does
not need a GPU; calling into the library needs the built libgsplat.so and
fails loudly (ImportError / GsError) when it is missing or a call fails.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgsplat.so")

GS_OK, GS_PENDING = 0, 1
GS_EINVAL, GS_ENOMEM, GS_ETIMEOUT, GS_EBUSY, GS_ECUDA, GS_EOVERFLOW = -1, -2, -3, -4, -5, -6
GS_F_NO_SYNC, GS_F_HOST_IO, GS_F_FULL_SORT, GS_F_RECOMPUTE, GS_F_COUNT = 1, 2, 4, 8, 16
GS_LOSS_DLDC, GS_LOSS_L1, GS_LOSS_L1_DSSIM, GS_LOSS_L1_MASKED = 0, 1, 2, 3
(GS_Q_NUM_KEYS, GS_Q_DEPTH, GS_Q_RECT, GS_Q_RADIUS, GS_Q_TILE_RANGES, GS_Q_SORTED_IDX, GS_Q_T_FINAL,
 GS_Q_N_CONTRIB, GS_Q_MEAN2D, GS_Q_SPLAT, GS_Q_SORTED_COUNT, GS_Q_DSSIM_GRAD) = range(12)

# names declared in include/gsplat.h (checked by the CPU test suite)
EXPORTED = (
    "gs_default_opts", "gs_ctx_create", "gs_ctx_destroy", "gs_scene_load", "gs_scene_borrow", "gs_scene_free",
    "gs_frames_create", "gs_frames_destroy", "gs_frames_reserve", "gs_render_forward", "gs_render_backward",
    "gs_pose_step", "gs_status", "gs_frames_query", "gs_last_error", "gs_version", "gs_ctx_set_profiling",
    "gs_ctx_profile", "gs_frames_counters", "gs_ctx_launch_count", "gs_step", "gs_loss_dssim_static",
    "gs_gaussian_adam", "gs_server_create", "gs_solve_submit", "gs_solve_poll", "gs_solve_wait", "gs_solve_cancel",
    "gs_server_stats_get", "gs_server_destroy", "gs_ctx_set_tuning", "gs_ctx_get_tuning", "gs_autotune",
    "gs_pose_step_txso3", "gs_regularize", "gs_prune_threshold", "gs_compact", "gs_unproject", "gs_knn_mean_dist",
    "gs_init_from_points", "gs_spatial_order", "gs_gather_rows", "gs_measure_alu_peaks", "gs_server_inject_enomem",
)
GS_POSE_SE3, GS_POSE_TXSO3 = 0, 1


class GsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gsplat error {code}: {msg}")
        self.code = code


class gs_scene_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacities", C.c_void_p), ("sh", C.c_void_p)]


class gs_view(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class gs_render_opts(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("z_near", C.c_float), ("eps2d", C.c_float), ("clamp_factor", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float), ("flags", C.c_uint32)]


class gs_loss(C.Structure):
    _fields_ = [("kind", C.c_int32), ("w_l1", C.c_float), ("w_dssim", C.c_float), ("target", C.c_void_p),
                ("dl_dimage", C.c_void_p), ("loss", C.c_void_p), ("mask_alpha", C.c_float)]


class gs_grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacities", C.c_void_p),
                ("sh", C.c_void_p)]


class gs_tuning(C.Structure):
    _fields_ = [("scatter_chunk", C.c_int32), ("sort_chunk", C.c_int32), ("preprocess_threads", C.c_int32),
                ("bwd_pixels_per_thread", C.c_int32), ("fwd_pixels_per_thread", C.c_int32)]


class gs_raw_params(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logit_opacities", C.c_void_p), ("sh", C.c_void_p)]


class gs_gaussian_lrs(C.Structure):
    _fields_ = [("means", C.c_float), ("scales", C.c_float), ("quats", C.c_float), ("opacities", C.c_float),
                ("sh_dc", C.c_float), ("sh_rest", C.c_float)]


class gs_server_config(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_width", C.c_int32), ("max_height", C.c_int32),
                ("mem_budget", C.c_int64), ("queue_capacity", C.c_int32), ("mask_alpha", C.c_float),
                ("pose_param", C.c_int32), ("tuning", gs_tuning)]


class gs_solve_request(C.Structure):
    _fields_ = [("view", gs_view), ("image", C.c_void_p), ("init_pose", C.c_double * 12), ("steps", C.c_int32),
                ("lr_start", C.c_double), ("lr_end", C.c_double)]


class gs_solve_result(C.Structure):
    _fields_ = [("pose", C.c_double * 12), ("loss", C.c_double), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("steps_done", C.c_int32), ("status", C.c_int32)]


class gs_alu_peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int), ("probe_sm_mhz", C.c_double), ("fp32_fma_per_sm_clk", C.c_double),
                ("fp32x2_fma_per_sm_clk", C.c_double), ("ex2_per_sm_clk", C.c_double),
                ("fp32_fma_per_s", C.c_double), ("fp32x2_fma_per_s", C.c_double), ("ex2_per_s", C.c_double),
                ("fp64_fma_per_sm_clk", C.c_double), ("fp64_fma_per_s", C.c_double),
                ("red_f32_per_s", C.c_double), ("red_f32x4_per_s", C.c_double)]


class gs_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("iterations", C.c_int64), ("active", C.c_int64), ("queued", C.c_int64), ("busy_ms", C.c_double),
                ("views_per_iteration", C.c_double), ("max_active", C.c_int64), ("budget_bytes", C.c_int64),
                ("requeued", C.c_int64)]


_lib = None


def load(path: str | None = None):
    """Loads libgsplat.so (built by paper_2410_08743_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libgsplat.so not built ({p}); run paper_2410_08743_gb300.build.build()")
    L = C.CDLL(p)
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.gs_default_opts.argtypes = [C.POINTER(gs_render_opts)]
    L.gs_default_opts.restype = None
    L.gs_ctx_create.argtypes = [i32, C.POINTER(vp)]
    L.gs_ctx_destroy.argtypes = [vp]
    L.gs_ctx_destroy.restype = None
    L.gs_scene_load.argtypes = [vp, C.POINTER(gs_scene_desc), i32, C.POINTER(vp)]
    L.gs_scene_borrow.argtypes = [C.POINTER(gs_scene_desc), C.POINTER(vp)]
    L.gs_scene_free.argtypes = [vp]
    L.gs_scene_free.restype = None
    L.gs_frames_create.argtypes = [vp, C.POINTER(vp)]
    L.gs_frames_destroy.argtypes = [vp]
    L.gs_frames_destroy.restype = None
    L.gs_frames_reserve.argtypes = [vp, i64, i64, i64, i64]
    L.gs_render_forward.argtypes = [vp, vp, i32, C.POINTER(gs_view), vp, C.POINTER(gs_render_opts), vp, vp, vp, vp, vp]
    L.gs_render_backward.argtypes = [vp, vp, i32, C.POINTER(gs_view), vp, C.POINTER(gs_render_opts), vp, vp,
                                     C.POINTER(gs_loss), C.POINTER(gs_grads), vp, vp]
    L.gs_step.argtypes = [vp, vp, C.POINTER(gs_scene_desc), i32, C.POINTER(gs_view), vp, C.POINTER(gs_render_opts),
                          C.POINTER(gs_loss), vp, C.POINTER(gs_grads), vp, vp, vp]
    L.gs_step.restype = C.c_int
    L.gs_loss_dssim_static.argtypes = [vp, vp, i32, i32, C.c_float, vp, vp, vp]
    L.gs_loss_dssim_static.restype = C.c_int
    L.gs_ctx_set_tuning.argtypes = [vp, C.POINTER(gs_tuning)]
    L.gs_ctx_get_tuning.argtypes = [vp, C.POINTER(gs_tuning)]
    L.gs_autotune.argtypes = [vp, vp, vp, i32, C.POINTER(gs_view), vp, C.POINTER(gs_render_opts), vp,
                              C.POINTER(gs_loss), C.POINTER(gs_grads), vp, i32, C.POINTER(gs_tuning),
                              C.POINTER(C.c_double), vp]
    for name in ("gs_ctx_set_tuning", "gs_ctx_get_tuning", "gs_autotune"):
        getattr(L, name).restype = C.c_int
    L.gs_gaussian_adam.argtypes = [vp, i64, i32, C.POINTER(gs_raw_params), vp, vp, C.POINTER(gs_grads), vp, vp,
                                   C.POINTER(gs_gaussian_lrs), C.c_float, C.c_float, C.c_float, i32, vp]
    L.gs_gaussian_adam.restype = C.c_int
    L.gs_server_create.argtypes = [i32, vp, C.POINTER(gs_render_opts), C.POINTER(gs_server_config), C.POINTER(vp)]
    L.gs_solve_submit.argtypes = [vp, C.POINTER(gs_solve_request), C.POINTER(C.c_uint64)]
    L.gs_solve_poll.argtypes = [vp, C.c_uint64, C.POINTER(gs_solve_result)]
    L.gs_solve_wait.argtypes = [vp, C.c_uint64, i32, C.POINTER(gs_solve_result)]
    L.gs_solve_cancel.argtypes = [vp, C.c_uint64]
    L.gs_server_stats_get.argtypes = [vp, C.POINTER(gs_server_stats)]
    L.gs_server_destroy.argtypes = [vp]
    L.gs_server_destroy.restype = None
    for name in ("gs_server_create", "gs_solve_submit", "gs_solve_poll", "gs_solve_wait", "gs_solve_cancel",
                 "gs_server_stats_get"):
        getattr(L, name).restype = C.c_int
    L.gs_pose_step.argtypes = [vp, i32, vp, vp, vp, vp, f64, f64, f64, f64, i32, vp]
    L.gs_pose_step_txso3.argtypes = [vp, i32, vp, vp, vp, vp, f64, f64, f64, f64, i32, vp]
    L.gs_pose_step_txso3.restype = C.c_int
    L.gs_regularize.argtypes = [vp, C.c_int64, vp, vp, C.c_float, C.c_float, C.c_float, vp, vp, vp, vp]
    L.gs_regularize.restype = C.c_int
    L.gs_prune_threshold.argtypes = [vp, C.c_int64, vp, C.c_int64, C.c_float, C.POINTER(C.c_float),
                                     C.POINTER(C.c_int64), vp]
    L.gs_prune_threshold.restype = C.c_int
    L.gs_compact.argtypes = [vp, C.c_int64, vp, C.c_float, C.c_int, vp, vp, vp, C.POINTER(C.c_int64), vp]
    L.gs_compact.restype = C.c_int
    L.gs_unproject.argtypes = [vp, C.POINTER(gs_view), vp, vp, C.c_int, vp, vp, C.c_int64, C.POINTER(C.c_int64), vp]
    L.gs_unproject.restype = C.c_int
    L.gs_knn_mean_dist.argtypes = [vp, C.c_int64, vp, C.c_int, vp, vp]
    L.gs_knn_mean_dist.restype = C.c_int
    L.gs_init_from_points.argtypes = [vp, C.c_int64, vp, vp, vp, C.c_float, C.c_float, C.POINTER(gs_raw_params), vp]
    L.gs_init_from_points.restype = C.c_int
    L.gs_spatial_order.argtypes = [vp, C.c_int64, vp, vp, vp]
    L.gs_spatial_order.restype = C.c_int
    L.gs_gather_rows.argtypes = [vp, C.c_int64, vp, C.c_int, vp, vp, vp, vp]
    L.gs_gather_rows.restype = C.c_int
    L.gs_status.argtypes = [vp, vp]
    L.gs_frames_query.argtypes = [vp, i32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
    L.gs_ctx_set_profiling.argtypes = [vp, i32]
    L.gs_ctx_profile.argtypes = [vp, i32, vp, vp, vp, C.POINTER(C.c_int)]
    L.gs_frames_counters.argtypes = [vp, C.POINTER(C.c_int64)]
    L.gs_measure_alu_peaks.argtypes = [i32, C.POINTER(gs_alu_peaks)]
    L.gs_measure_alu_peaks.restype = C.c_int
    L.gs_ctx_launch_count.argtypes = [vp]
    L.gs_ctx_launch_count.restype = C.c_int64
    L.gs_last_error.restype = C.c_char_p
    L.gs_version.restype = C.c_char_p
    for name in ("gs_ctx_create", "gs_scene_load", "gs_scene_borrow", "gs_frames_create", "gs_frames_reserve",
                 "gs_render_forward", "gs_render_backward", "gs_pose_step", "gs_status", "gs_frames_query",
                 "gs_ctx_set_profiling", "gs_ctx_profile", "gs_frames_counters"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ck(rc: int) -> int:
    if rc < 0:
        raise GsError(rc, load().gs_last_error().decode(errors="replace"))
    return rc


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor arguments must be contiguous")
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------- objects

def gs_default_opts(**over) -> gs_render_opts:
    o = gs_render_opts()
    load().gs_default_opts(C.byref(o))
    for k, v in over.items():
        if k == "bg":
            for j in range(3):
                o.bg[j] = float(v[j])
        else:
            setattr(o, k, v)
    return o


def gs_ctx_create(device: int = 0) -> int:
    h = C.c_void_p()
    _ck(load().gs_ctx_create(int(device), C.byref(h)))
    return h.value


def gs_ctx_destroy(ctx: int) -> None:
    load().gs_ctx_destroy(C.c_void_p(ctx))


def scene_desc(means, scales, quats, opac, sh, sh_degree: int) -> gs_scene_desc:
    return gs_scene_desc(int(means.shape[0]), int(sh_degree), _ptr(means), _ptr(scales), _ptr(quats), _ptr(opac),
                         _ptr(sh))


def gs_scene_borrow(means, scales, quats, opac, sh, sh_degree: int) -> int:
    d = scene_desc(means, scales, quats, opac, sh, sh_degree)
    h = C.c_void_p()
    _ck(load().gs_scene_borrow(C.byref(d), C.byref(h)))
    return h.value


def gs_scene_load(ctx: int, means, scales, quats, opac, sh, sh_degree: int) -> int:
    d = scene_desc(means, scales, quats, opac, sh, sh_degree)
    h = C.c_void_p()
    _ck(load().gs_scene_load(C.c_void_p(ctx), C.byref(d), int(means.is_cuda), C.byref(h)))
    return h.value


def gs_scene_free(scene: int) -> None:
    load().gs_scene_free(C.c_void_p(scene))


def gs_frames_create(ctx: int) -> int:
    h = C.c_void_p()
    _ck(load().gs_frames_create(C.c_void_p(ctx), C.byref(h)))
    return h.value


def gs_frames_destroy(fr: int) -> None:
    load().gs_frames_destroy(C.c_void_p(fr))


def gs_frames_reserve(fr: int, keys: int, pairs: int, pixels: int, tiles: int) -> None:
    _ck(load().gs_frames_reserve(C.c_void_p(fr), int(keys), int(pairs), int(pixels), int(tiles)))


def views_array(views) -> C.Array:
    arr = (gs_view * max(1, len(views)))()
    for k, v in enumerate(views):
        arr[k] = gs_view(float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"]), int(v["width"]),
                         int(v["height"]))
    return arr


def gs_render_forward(ctx: int, scene: int, views_arr, n_views: int, poses, opts: gs_render_opts, fr: int, image,
                      target=None, loss_out=None, stream=None) -> None:
    _ck(load().gs_render_forward(C.c_void_p(ctx), C.c_void_p(scene), int(n_views), views_arr, _ptr(poses),
                                 C.byref(opts), C.c_void_p(fr), _ptr(image), _ptr(target), _ptr(loss_out),
                                 _stream(stream)))


def gs_render_backward(ctx: int, scene: int, views_arr, n_views: int, poses, opts: gs_render_opts, fr: int, image,
                       loss: gs_loss, grads: gs_grads | None, pose_grad, stream=None) -> None:
    _ck(load().gs_render_backward(C.c_void_p(ctx), C.c_void_p(scene), int(n_views), views_arr, _ptr(poses),
                                  C.byref(opts), C.c_void_p(fr), _ptr(image), C.byref(loss),
                                  C.byref(grads) if grads is not None else None, _ptr(pose_grad), _stream(stream)))


def gs_step(ctx: int, fr: int, desc: gs_scene_desc, views_arr, n_views: int, poses_ptr, opts: gs_render_opts,
            loss: gs_loss, image_ptr, grads: gs_grads | None, pose_grad_ptr, loss_out_ptr, stream=None) -> None:
    """Raw pointers (ints) so that host (GS_F_HOST_IO) and device buffers pass alike."""
    _ck(load().gs_step(C.c_void_p(ctx), C.c_void_p(fr), C.byref(desc), int(n_views), views_arr,
                       C.c_void_p(poses_ptr), C.byref(opts), C.byref(loss), C.c_void_p(image_ptr),
                       C.byref(grads) if grads is not None else None, C.c_void_p(pose_grad_ptr),
                       C.c_void_p(loss_out_ptr), _stream(stream)))


def make_loss(kind: int, target=None, dl_dimage=None, w_l1: float = 1.0, w_dssim: float = 0.0, loss_out=None,
              mask_alpha: float = 0.0):
    return gs_loss(int(kind), float(w_l1), float(w_dssim), _ptr(target), _ptr(dl_dimage), _ptr(loss_out),
                   float(mask_alpha))


def make_grads(means=None, scales=None, quats=None, opac=None, sh=None) -> gs_grads:
    return gs_grads(_ptr(means), _ptr(scales), _ptr(quats), _ptr(opac), _ptr(sh))


def gs_pose_step(ctx: int, poses, m, v, grad, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8,
                 stream=None, param: int = GS_POSE_SE3) -> None:
    fn = load().gs_pose_step_txso3 if param == GS_POSE_TXSO3 else load().gs_pose_step
    _ck(fn(C.c_void_p(ctx), int(poses.shape[0]), _ptr(poses), _ptr(m), _ptr(v), _ptr(grad),
                            float(lr), float(beta1), float(beta2), float(eps), int(step), _stream(stream)))


def gs_regularize(ctx: int, scales, opac, aniso_r: float, lambda_aniso: float, lambda_opacity: float,
                  grad_scales=None, grad_opac=None, loss=None, stream=None) -> None:
    """Anisotropy hinge (Eq. 17) and opacity L1 on activated parameters;
    gradients are ADDED into grad_scales / grad_opac."""
    n = int(scales.shape[0]) if scales is not None else int(opac.shape[0])
    _ck(load().gs_regularize(C.c_void_p(ctx), n, _ptr(scales), _ptr(opac), float(aniso_r), float(lambda_aniso),
                             float(lambda_opacity), _ptr(grad_scales), _ptr(grad_opac), _ptr(loss), _stream(stream)))


def gs_prune_threshold(ctx: int, opac, n_target: int, min_opacity: float = 0.005, stream=None):
    """Returns (threshold, n_keep)."""
    thr = C.c_float(0.0)
    nk = C.c_int64(0)
    _ck(load().gs_prune_threshold(C.c_void_p(ctx), int(opac.shape[0]), _ptr(opac), int(n_target),
                                  float(min_opacity), C.byref(thr), C.byref(nk), _stream(stream)))
    return float(thr.value), int(nk.value)


def gs_compact(ctx: int, opac, threshold: float, src: list, dst: list, widths: list, stream=None) -> int:
    """Out-of-place stable compaction of row arrays; returns n_keep."""
    k = len(src)
    s_arr = (C.c_void_p * max(k, 1))(*[_ptr(a) for a in src])
    d_arr = (C.c_void_p * max(k, 1))(*[_ptr(a) for a in dst])
    w_arr = (C.c_int32 * max(k, 1))(*[int(w) for w in widths])
    nk = C.c_int64(0)
    _ck(load().gs_compact(C.c_void_p(ctx), int(opac.shape[0]), _ptr(opac), float(threshold), k,
                          C.cast(s_arr, C.c_void_p), C.cast(d_arr, C.c_void_p), C.cast(w_arr, C.c_void_p),
                          C.byref(nk), _stream(stream)))
    return int(nk.value)


def gs_unproject(ctx: int, view: dict, depth, image, stride: int, points, colours=None, stream=None) -> int:
    """Camera points of the stride grid's pixels with positive depth (Sec. 3.4);
    points / colours: device [capacity, 3].  Returns the count."""
    v = views_array([view])
    n = C.c_int64(0)
    _ck(load().gs_unproject(C.c_void_p(ctx), v, _ptr(depth), _ptr(image), int(stride), _ptr(points), _ptr(colours),
                            int(points.shape[0]), C.byref(n), _stream(stream)))
    return int(n.value)


def gs_knn_mean_dist(ctx: int, points, k: int, out, n: int | None = None, stream=None) -> None:
    n = int(points.shape[0]) if n is None else int(n)
    _ck(load().gs_knn_mean_dist(C.c_void_p(ctx), n, _ptr(points), int(k), _ptr(out), _stream(stream)))


def gs_init_from_points(ctx: int, points, colours, mean_dist, raw: dict, n: int | None = None, min_scale: float = 1e-4,
                        opacity: float = 0.1, stream=None) -> None:
    n = int(points.shape[0]) if n is None else int(n)
    rp = gs_raw_params(_ptr(raw["means"]), _ptr(raw["log_scales"]), _ptr(raw["quats"]), _ptr(raw["logit_opac"]),
                       _ptr(raw["sh"]))
    _ck(load().gs_init_from_points(C.c_void_p(ctx), n, _ptr(points), _ptr(colours), _ptr(mean_dist),
                                   float(min_scale), float(opacity), C.byref(rp), _stream(stream)))


def gs_spatial_order(ctx: int, means, perm, stream=None) -> None:
    """perm (device int32 [n], read as uint32): the Morton order of the means."""
    _ck(load().gs_spatial_order(C.c_void_p(ctx), int(means.shape[0]), _ptr(means), _ptr(perm), _stream(stream)))


def gs_gather_rows(ctx: int, perm, src: list, dst: list, widths: list, stream=None) -> None:
    k = len(src)
    s_arr = (C.c_void_p * max(k, 1))(*[_ptr(a) for a in src])
    d_arr = (C.c_void_p * max(k, 1))(*[_ptr(a) for a in dst])
    w_arr = (C.c_int32 * max(k, 1))(*[int(w) for w in widths])
    _ck(load().gs_gather_rows(C.c_void_p(ctx), int(perm.shape[0]), _ptr(perm), k, C.cast(s_arr, C.c_void_p),
                              C.cast(d_arr, C.c_void_p), C.cast(w_arr, C.c_void_p), _stream(stream)))


def spatially_ordered(ctx: int, params: dict, stream=None):
    """Returns (params in Morton order, perm) for a scene dict of device
    tensors (means, scales, quats, opac, sh, sh_degree)."""
    import torch
    n = int(params["means"].shape[0])
    perm = torch.empty(n, dtype=torch.int32, device=params["means"].device)
    gs_spatial_order(ctx, params["means"], perm, stream)
    names = [("means", 3), ("scales", 3), ("quats", 4), ("opac", 1), ("sh", 48)]
    out = {k: torch.empty_like(params[k]) for k, _ in names}
    gs_gather_rows(ctx, perm, [params[k] for k, _ in names], [out[k] for k, _ in names], [w for _, w in names],
                   stream)
    out["sh_degree"] = params["sh_degree"]
    return out, perm


def gs_loss_dssim_static(image, target, width: int, height: int, w_dssim: float, dl_dimage, loss=None,
                         stream=None) -> None:
    """D-SSIM term of one view with the library's static scratch (no allocation)."""
    _ck(load().gs_loss_dssim_static(_ptr(image), _ptr(target), int(width), int(height), float(w_dssim),
                                    _ptr(dl_dimage), _ptr(loss), _stream(stream)))


def gs_gaussian_adam(ctx: int, raw: dict, act_scales, act_opac, grads: dict, m, v, lrs: dict, step: int,
                     sh_degree: int, beta1=0.9, beta2=0.999, eps=1e-15, stream=None) -> None:
    """raw: means, log_scales, quats, logit_opac, sh (device tensors, updated in
    place); grads: renderer gradients (means, scales, quats, opac, sh)."""
    rp = gs_raw_params(_ptr(raw["means"]), _ptr(raw["log_scales"]), _ptr(raw["quats"]), _ptr(raw["logit_opac"]),
                       _ptr(raw["sh"]))
    g = make_grads(grads.get("means"), grads.get("scales"), grads.get("quats"), grads.get("opac"), grads.get("sh"))
    lr = gs_gaussian_lrs(lrs["means"], lrs["scales"], lrs["quats"], lrs["opac"], lrs["sh_dc"], lrs["sh_rest"])
    _ck(load().gs_gaussian_adam(C.c_void_p(ctx), int(raw["means"].shape[0]), int(sh_degree), C.byref(rp),
                                _ptr(act_scales), _ptr(act_opac), C.byref(g), _ptr(m), _ptr(v), C.byref(lr),
                                float(beta1), float(beta2), float(eps), int(step), _stream(stream)))


def gs_server_create(device: int, scene: int, opts: gs_render_opts, max_slots: int, max_width: int, max_height: int,
                     mem_budget: int = 0, queue_capacity: int = 65536, mask_alpha: float = 0.0,
                     pose_param: int = GS_POSE_SE3, tuning: dict | None = None) -> int:
    t = gs_tuning(*[int(tuning[k]) for k, _ in gs_tuning._fields_]) if tuning else gs_tuning()
    cfg = gs_server_config(int(max_slots), int(max_width), int(max_height), int(mem_budget), int(queue_capacity),
                           float(mask_alpha), int(pose_param), t)
    h = C.c_void_p()
    _ck(load().gs_server_create(int(device), C.c_void_p(scene), C.byref(opts), C.byref(cfg), C.byref(h)))
    return h.value


def gs_solve_submit(srv: int, view: dict, image, init_pose, steps: int, lr_start: float, lr_end: float) -> int:
    """image: host float32 array [3*H*W] (planar)."""
    import numpy as np
    img = np.ascontiguousarray(image, np.float32)
    req = gs_solve_request(views_array([view])[0], img.ctypes.data_as(C.c_void_p),
                           (C.c_double * 12)(*[float(x) for x in np.asarray(init_pose).reshape(12)]), int(steps),
                           float(lr_start), float(lr_end))
    t = C.c_uint64(0)
    _ck(load().gs_solve_submit(C.c_void_p(srv), C.byref(req), C.byref(t)))
    return int(t.value)


def _result_dict(r: gs_solve_result) -> dict:
    return dict(pose=list(r.pose), loss=r.loss, latency_ms=r.latency_ms, queue_ms=r.queue_ms, steps_done=r.steps_done,
                status=r.status)


def gs_solve_poll(srv: int, ticket: int):
    r = gs_solve_result()
    rc = _ck(load().gs_solve_poll(C.c_void_p(srv), C.c_uint64(ticket), C.byref(r)))
    return None if rc == GS_PENDING else _result_dict(r)


def gs_solve_wait(srv: int, ticket: int, timeout_ms: int):
    r = gs_solve_result()
    _ck(load().gs_solve_wait(C.c_void_p(srv), C.c_uint64(ticket), int(timeout_ms), C.byref(r)))
    return _result_dict(r)


def gs_solve_cancel(srv: int, ticket: int) -> None:
    _ck(load().gs_solve_cancel(C.c_void_p(srv), C.c_uint64(ticket)))


def gs_server_stats_get(srv: int) -> dict:
    st = gs_server_stats()
    _ck(load().gs_server_stats_get(C.c_void_p(srv), C.byref(st)))
    return {k: getattr(st, k) for k, _ in gs_server_stats._fields_}


def gs_server_destroy(srv: int) -> None:
    load().gs_server_destroy(C.c_void_p(srv))


def gs_server_inject_enomem(srv: int, iterations: int) -> None:
    """Test hook: the next `iterations` server iterations fail as a workspace
    growth would (GS_ENOMEM), made on the host."""
    L = load()
    L.gs_server_inject_enomem.argtypes = [C.c_void_p, C.c_int]
    L.gs_server_inject_enomem.restype = C.c_int
    _ck(L.gs_server_inject_enomem(C.c_void_p(srv), int(iterations)))


def gs_ctx_set_tuning(ctx: int, scatter_chunk: int, sort_chunk: int, preprocess_threads: int,
                      bwd_pixels_per_thread: int = 1, fwd_pixels_per_thread: int = 1) -> None:
    t = gs_tuning(int(scatter_chunk), int(sort_chunk), int(preprocess_threads), int(bwd_pixels_per_thread),
                  int(fwd_pixels_per_thread))
    _ck(load().gs_ctx_set_tuning(C.c_void_p(ctx), C.byref(t)))


def gs_ctx_get_tuning(ctx: int) -> dict:
    t = gs_tuning()
    _ck(load().gs_ctx_get_tuning(C.c_void_p(ctx), C.byref(t)))
    return {k: getattr(t, k) for k, _ in gs_tuning._fields_}


def gs_autotune(ctx: int, fr: int, scene: int, views_arr, n_views: int, poses, opts: gs_render_opts, image,
                loss: gs_loss, grads: gs_grads | None, pose_grad, repeats: int = 2, stream=None):
    best = gs_tuning()
    ms = C.c_double(0.0)
    _ck(load().gs_autotune(C.c_void_p(ctx), C.c_void_p(fr), C.c_void_p(scene), int(n_views), views_arr, _ptr(poses),
                           C.byref(opts), _ptr(image), C.byref(loss), C.byref(grads) if grads is not None else None,
                           _ptr(pose_grad), int(repeats), C.byref(best), C.byref(ms), _stream(stream)))
    return {k: getattr(best, k) for k, _ in gs_tuning._fields_}, ms.value


def gs_status(ctx: int, stream=None) -> int:
    return _ck(load().gs_status(C.c_void_p(ctx), _stream(stream)))


def gs_frames_query(fr: int, what: int):
    """Returns the queried internal array as a numpy array (synchronous)."""
    import numpy as np
    L = load()
    size = C.c_size_t(0)
    _ck(L.gs_frames_query(C.c_void_p(fr), int(what), None, 0, C.byref(size)))
    dtype = {GS_Q_NUM_KEYS: np.int64, GS_Q_DEPTH: np.float32, GS_Q_RECT: np.int32, GS_Q_RADIUS: np.int32,
             GS_Q_TILE_RANGES: np.uint32, GS_Q_SORTED_IDX: np.uint32, GS_Q_T_FINAL: np.float32,
             GS_Q_N_CONTRIB: np.uint32, GS_Q_MEAN2D: np.float32, GS_Q_SPLAT: np.float32,
             GS_Q_SORTED_COUNT: np.uint32, GS_Q_DSSIM_GRAD: np.float32}[what]
    out = np.zeros(max(1, size.value // np.dtype(dtype).itemsize), dtype)
    _ck(L.gs_frames_query(C.c_void_p(fr), int(what), out.ctypes.data_as(C.c_void_p), out.nbytes, None))
    return out[: size.value // np.dtype(dtype).itemsize]


def gs_ctx_set_profiling(ctx: int, enable: bool) -> None:
    _ck(load().gs_ctx_set_profiling(C.c_void_p(ctx), int(bool(enable))))


def gs_ctx_profile(ctx: int) -> dict:
    """{kernel kind: (total ms, launches)} since the last read (synchronous)."""
    K = 32
    names = (C.c_char * 32 * K)()
    ms = (C.c_double * K)()
    cnt = (C.c_int64 * K)()
    n = C.c_int(0)
    _ck(load().gs_ctx_profile(C.c_void_p(ctx), K, C.cast(names, C.c_void_p), C.cast(ms, C.c_void_p),
                              C.cast(cnt, C.c_void_p), C.byref(n)))
    return {names[i].value.decode(): (ms[i], int(cnt[i])) for i in range(n.value)}


def gs_ctx_launch_count(ctx: int) -> int:
    return int(load().gs_ctx_launch_count(C.c_void_p(ctx)))


def gs_measure_alu_peaks(device: int = 0) -> dict:
    """Measured FP32 / paired-FP32 FMA and MUFU ex2 rates of a device
    (per SM per cycle and per second) and its SM count."""
    out = gs_alu_peaks()
    _ck(load().gs_measure_alu_peaks(int(device), C.byref(out)))
    return {k: getattr(out, k) for k, _ in gs_alu_peaks._fields_}


GS_N_COUNTERS = 11


def gs_frames_counters(fr: int):
    out = (C.c_int64 * GS_N_COUNTERS)()
    _ck(load().gs_frames_counters(C.c_void_p(fr), out))
    return [int(x) for x in out]


def gs_last_error() -> str:
    return load().gs_last_error().decode(errors="replace")


def gs_version() -> str:
    return load().gs_version().decode()
