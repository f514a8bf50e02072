"""Autotuning of the renderer's result-neutral launch parameters.

`autotune` picks the tuning (Gaussians per count/scatter CTA, lazy-sort run
length, forward-preprocess block size, pixels per thread of the two blends)
with the library's gs_autotune for a
workload class and caches the choice in a JSON file keyed by GPU name,
resolution class and Gaussian-count class, so later runs of the same class
reuse it without timing again."""
from __future__ import annotations

import json
import math
import os

from . import _lib as L


def default_cache_path() -> str:
    return os.environ.get("GSPLAT_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gsplat_gb300", "tuning.json"))


def workload_key(gpu_name: str, views, n_gaussians: int) -> str:
    px = sum(int(v["width"]) * int(v["height"]) for v in views)
    res_class = f"views{len(views)}-px2^{int(round(math.log2(max(px, 1))))}"
    n_class = f"n2^{int(round(math.log2(max(n_gaussians, 1))))}"
    # the version prefix changes when the kernels' timing changes enough for a
    # cached choice to go stale (t4: paired-arithmetic and per-warp blends)
    return f"t4|{gpu_name}|{res_class}|{n_class}"


def autotune(renderer, params: dict, views, poses, image, loss, grads=None, pose_grad=None, repeats: int = 2,
             cache_path: str | None = None, force: bool = False) -> dict:
    """Sets renderer's tuning for this workload class (from the cache when
    present) and returns {'tuning': ..., 'ms': ..., 'cached': bool}."""
    import torch
    path = cache_path or default_cache_path()
    key = workload_key(torch.cuda.get_device_name(renderer.device), views, int(params["means"].shape[0]))
    cache = {}
    if os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and not force:
        t = cache[key]["tuning"]
        L.gs_ctx_set_tuning(renderer.ctx, t["scatter_chunk"], t["sort_chunk"], t["preprocess_threads"],
                            t.get("bwd_pixels_per_thread", 1), t.get("fwd_pixels_per_thread", 1))
        # one synchronising step with the new tuning grows the workspaces it
        # needs (a GS_F_NO_SYNC call cannot), as the tuner's own trials would;
        # like them it accumulates into grads / pose_grad
        flags = renderer.opts.flags
        renderer.set_flags(flags & ~L.GS_F_NO_SYNC)
        try:
            renderer.forward(params, views, poses, image=image)
            renderer.backward(params, views, poses, image, loss, grads, pose_grad)
        finally:
            renderer.set_flags(flags)
        return dict(tuning=t, ms=cache[key]["ms"], cached=True, key=key)
    sc = L.gs_scene_borrow(params["means"], params["scales"], params["quats"], params["opac"], params["sh"],
                           params["sh_degree"])
    g = None
    if grads is not None:
        g = L.make_grads(grads.get("means"), grads.get("scales"), grads.get("quats"), grads.get("opac"),
                         grads.get("sh"))
    try:
        t, ms = L.gs_autotune(renderer.ctx, renderer.frames, sc, renderer.views(views), len(views), poses,
                              renderer.opts, image, loss, g, pose_grad, repeats)
    finally:
        L.gs_scene_free(sc)
    cache[key] = dict(tuning=t, ms=ms)
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return dict(tuning=t, ms=ms, cached=False, key=key)
