"""GPU path vs the FP64 oracle at the full workload sizes, on sampled outputs.

* Batched fwd+bwd: 1M SH3 Gaussians, 64 views of mixed resolution, rendered in
  the single batched launch sequence the benchmark times.  The oracle renders a
  sample of views (one per resolution plus one more); the upstream image
  gradient is nonzero on those views only, so the oracle's backward over the
  sample is the exact reference for every per-Gaussian gradient of the whole
  launch and for the sampled views' pose gradients, and every other view's pose
  gradient must be exactly zero.
* Joint refinement: 300k SH3 Gaussians, one 504x378 view per launch, loss
  0.8 L1 + 0.2 D-SSIM against a target the oracle renders at the ground-truth
  pose.
* Trajectory: 3M SH3 Gaussians in a room, 8 frames of 1280x720 per launch,
  backward with the forward state recomputed (another batch was rendered in
  between).

Tolerances (large configurations, where FP32 atomics cancel): keys, tile
lists and key-path values bit-exact; images <= 1e-4 max-abs on pixels without
a near-threshold decision; per parameter group the norm-relative error
<= 1e-3 and the per-element rule |d| <= max(1e-3 |g_ref|, 1e-6 * max|g_ref|)
on >= 99.9% of the elements; each pose gradient component within
max(1e-3 |g_ref|, 1e-6).  The joint case also checks the GPU's own
L1 + D-SSIM backward: its D-SSIM dL/dC per element against the oracle's on the
GPU image, and its parameter and pose gradients against the oracle's backward
of the same dL/dC, with Gaussians reached by near-threshold pixels left out
and those pixels' share bounding the pose tolerance."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import synth
from paper_2410_08743_gb300.render import Renderer

from .gpu_util import DEV, assert_dssim_grad_close, assert_pose_close, gpu_forward, poses_dev, to_dev, zero_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def _oracle_threads(n_splats):
    """The oracle's backward keeps one [V*N, 9] FP64 buffer per thread; keep
    them within a quarter of the host's free memory."""
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 16 << 30
    t = int(max(1, min(oracle.max_threads(), (avail // 4) // max(1, n_splats * 72))))
    oracle.set_threads(t)
    return t


def _sub(views, poses, idx):
    return [views[k] for k in idx], np.ascontiguousarray(poses[idx])


def _view_slices(views, idx):
    img_off, pix_off = synth.image_offsets(views)
    return [(img_off[k], img_off[k + 1], pix_off[k], pix_off[k + 1]) for k in idx]


def _tile_bases(views):
    b = [0]
    for v in views:
        b.append(b[-1] + ((v["width"] + 15) // 16) * ((v["height"] + 15) // 16))
    return b


def _check_images(img, ref, views, idx):
    """img: the GPU's packed image of all views; ref: the oracle over views idx."""
    fr = ref["fragile"].astype(bool)
    assert fr.mean() < 0.01, fr.mean()
    ro = 0; rp = 0
    for (i0, i1, p0, p1) in _view_slices(views, idx):
        npx = p1 - p0
        ok = ~fr[rp:rp + npx]
        for ch in range(3):
            a = img[i0 + ch * npx:i0 + (ch + 1) * npx][ok]
            b = ref["image"][ro + ch * npx:ro + (ch + 1) * npx][ok]
            assert np.abs(a - b).max() <= 1e-4, (ch, np.abs(a - b).max())
        ro += 3 * npx; rp += npx


def _sample_dldc(rng, views, idx, ref):
    """Upstream gradient for the whole launch: random on the sampled views
    (zero on near-threshold pixels), zero elsewhere.  Returns (full f32, the
    sampled views' part as f64)."""
    img_off, _ = synth.image_offsets(views)
    full = np.zeros(img_off[-1], np.float32)
    parts = []
    rp = 0
    for k, (i0, i1, p0, p1) in zip(idx, _view_slices(views, idx)):
        npx = p1 - p0
        d = (rng.standard_normal(3 * npx) / (3 * npx)).astype(np.float32)
        fr = ref["fragile"][rp:rp + npx].astype(bool)
        for ch in range(3):
            d[ch * npx:(ch + 1) * npx][fr] = 0.0
        full[i0:i1] = d
        parts.append(d.astype(np.float64))
        rp += npx
    return full, np.concatenate(parts)


def _check_grads_large(g, go, n, sh_degree, keep=None):
    keep = ~go["fragile_g"].reshape(-1, n).any(0) & (True if keep is None else keep)
    nc = (sh_degree + 1) ** 2
    pairs = [("means", g["means"], go["means"]), ("scales", g["scales"], go["scales"]),
             ("quats", g["quats"], go["quats"]), ("opac", g["opac"].reshape(-1, 1), go["opac"].reshape(-1, 1)),
             ("sh", g["sh"][:, :nc].reshape(n, -1), go["sh"][:, :nc].reshape(n, -1))]
    for name, a, b in pairs:
        a = np.asarray(a, np.float64).reshape(n, -1)[keep]
        b = np.asarray(b, np.float64).reshape(n, -1)[keep]
        nb = np.linalg.norm(b)
        assert nb > 0, name
        assert np.linalg.norm(a - b) <= 1e-3 * nb, (name, np.linalg.norm(a - b) / nb)
        tol = np.maximum(1e-3 * np.abs(b), 1e-6 * np.abs(b).max())
        frac = float(np.mean(np.abs(a - b) <= tol))
        assert frac >= 0.999, (name, frac)
    assert np.all(np.asarray(g["sh"])[:, nc:] == 0)


def _bench_configuration(R, p, views, P):
    """The launch configuration bench.py times: the autotuner's choice for the
    workload class (a fresh cache, so it tunes as the bench does on a new box)."""
    import tempfile

    from paper_2410_08743_gb300 import tune
    image = torch.empty(Renderer.image_numel(views), device=DEV)
    tgt = torch.zeros_like(image)
    g = zero_grads(p)
    pg = torch.zeros(len(views), 6, dtype=torch.float64, device=DEV)
    l1 = L.make_loss(L.GS_LOSS_L1, target=tgt, w_l1=1.0)
    R.forward(p, views, P, image=image)
    with tempfile.TemporaryDirectory() as d:
        return tune.autotune(R, p, views, P, image, l1, g, pg, repeats=1, cache_path=os.path.join(d, "t.json"))


def test_batched_1M_64_views_sampled_parity(R):
    """In the bench's configuration: the scene loaded in Morton order of its
    means, the autotuned launch parameters (two pixels per thread in the
    blends where it picks them), one launch over all 64 views."""
    w = synth.batched_workload()
    sc0, views, poses = w["scene"], w["views"], w["poses"]
    n = len(sc0["opac"])
    res = [(v["width"], v["height"]) for v in views]
    idx = sorted({res.index(r) for r in set(res)} | {len(views) - 1})
    assert len(idx) >= 3
    p, perm = L.spatially_ordered(R.ctx, to_dev(sc0))
    perm = perm.cpu().numpy().astype(np.int64)
    sc = {k_: np.ascontiguousarray(sc0[k_][perm]) for k_ in ("means", "scales", "quats", "opac", "sh")}
    sc["sh_degree"] = sc0["sh_degree"]
    P = poses_dev(poses)
    tuned = _bench_configuration(R, p, views, P)
    try:
        _batched_sampled_parity(R, sc, p, views, poses, P, idx, n)
    finally:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1, 1)
    print("tuning", tuned["tuning"])


def _batched_sampled_parity(R, sc, p, views, poses, P, idx, n):
    img = R.forward(p, views, P)
    torch.cuda.synchronize()
    vs, ps = _sub(views, poses, idx)
    _oracle_threads(len(idx) * n)

    # keys: per-(view, Gaussian) key path and tile lists of the sampled views
    k = oracle.keys(sc, vs, ps)
    rect = R.query(L.GS_Q_RECT).reshape(-1, 4)
    radius = R.query(L.GS_Q_RADIUS)
    depth = R.query(L.GS_Q_DEPTH).view(np.uint32)
    m2 = R.query(L.GS_Q_MEAN2D).reshape(-1, 2).view(np.uint32)
    for j, v in enumerate(idx):
        sl, so = slice(v * n, (v + 1) * n), slice(j * n, (j + 1) * n)
        valid = k["valid"][so].astype(bool)
        assert np.array_equal(rect[sl], k["rect"][so]), v
        assert np.array_equal(radius[sl], k["radius"][so]), v
        assert np.array_equal(depth[sl][valid], k["depth"][so].view(np.uint32)[valid]), v
        assert np.array_equal(m2[sl][valid], k["mu2f"][so].view(np.uint32)[valid]), v
    del rect, radius, depth, m2
    ranges = R.query(L.GS_Q_TILE_RANGES).reshape(-1, 2).astype(np.int64)
    cnt = R.query(L.GS_Q_SORTED_COUNT)
    got = R.query(L.GS_Q_SORTED_IDX)
    gb, ob = _tile_bases(views), _tile_bases(vs)
    for j, v in enumerate(idx):
        nt = gb[v + 1] - gb[v]
        g_r = ranges[gb[v]:gb[v + 1]]
        o_r = k["ranges"][ob[j]:ob[j] + nt].astype(np.int64)
        assert np.array_equal(g_r[:, 1] - g_r[:, 0], o_r[:, 1] - o_r[:, 0]), v
        c = cnt[gb[v]:gb[v + 1]]
        assert np.all(c <= g_r[:, 1] - g_r[:, 0])
        for t in np.nonzero(c)[0]:
            assert np.array_equal(got[g_r[t, 0]:g_r[t, 0] + c[t]], k["idx"][o_r[t, 0]:o_r[t, 0] + c[t]]), (v, t)
    del got, k

    # image, T_final, n_contrib
    ref = oracle.render(sc, vs, ps)
    img_np = img.cpu().numpy()
    _check_images(img_np, ref, views, idx)
    T = R.query(L.GS_Q_T_FINAL); nc = R.query(L.GS_Q_N_CONTRIB)
    rp = 0
    fr = ref["fragile"].astype(bool)
    for (_, _, p0, p1) in _view_slices(views, idx):
        ok = ~fr[rp:rp + p1 - p0]
        assert np.abs(T[p0:p1][ok] - ref["T_final"][rp:rp + p1 - p0][ok]).max() <= 1e-4
        assert np.array_equal(nc[p0:p1][ok], ref["n_contrib"][rp:rp + p1 - p0][ok].astype(np.uint32))
        rp += p1 - p0

    # backward of the whole launch with the upstream gradient on the sample
    rng = np.random.default_rng(17)
    full, part = _sample_dldc(rng, views, idx, ref)
    g = zero_grads(p)
    pg = torch.zeros(len(views), 6, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=torch.from_numpy(full).to(DEV)), g, pg)
    torch.cuda.synchronize()
    go = oracle.backward(sc, vs, ps, part)
    _check_grads_large({k_: v_.cpu().numpy() for k_, v_ in g.items()}, go, n, sc["sh_degree"])
    pg = pg.cpu().numpy()
    assert_pose_close(pg[idx], go["pose"], "pose (1M x 64 sample)")
    others = np.setdiff1d(np.arange(len(views)), idx)
    assert np.all(pg[others] == 0)


def test_joint_300k_l1_dssim_one_view_parity(R):
    w = synth.joint_workload()
    sc, views, gt = w["scene"], w["views"], w["poses"]
    n = len(sc["opac"])
    v = [views[7]]
    init = w["init_poses"][7:8]
    _oracle_threads(n)
    target = oracle.render(sc, v, gt[7:8])["image"].astype(np.float32)
    p, P, img, tg, _ = gpu_forward(R, sc, v, init, target=target)
    ref = oracle.render(sc, v, init)
    _check_images(img.cpu().numpy(), ref, v, [0])
    L1, d1, fr1 = oracle.loss_l1(v, ref["image"], target, weight=0.8)
    Ld, dd, _ = oracle.loss_dssim(v, ref["image"], target, weight=0.2)
    lo = torch.zeros(1, dtype=torch.float64, device=DEV)
    g = zero_grads(p)
    pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    R.backward(p, v, P, img, L.make_loss(L.GS_LOSS_L1_DSSIM, target=tg, w_l1=0.8, w_dssim=0.2, loss_out=lo), g, pg)
    torch.cuda.synchronize()
    assert abs(lo.item() - (L1 + Ld)) <= 1e-5 * max(1.0, L1 + Ld), (lo.item(), L1 + Ld)
    # the GPU's own L1 + D-SSIM backward (g, pg): its D-SSIM dL/dC against the
    # oracle's on the same (GPU) image, then its gradients against the oracle's
    # backward of the dL/dC the GPU used (the L1 signs of the GPU image are the
    # signs its kernel took); Gaussians reached by near-threshold pixels are
    # left out and those pixels' share bounds the pose tolerance
    img64 = img.cpu().numpy().astype(np.float64)
    _, dd_g, _ = oracle.loss_dssim(v, img64, target, weight=0.2)
    ratio = assert_dssim_grad_close(R.query(L.GS_Q_DSSIM_GRAD), dd_g, oracle.loss_dssim_cond(v, img64, target, 0.2),
                                    "D-SSIM dL/dC (joint view)")
    print(f"D-SSIM dL/dC worst error / tolerance {ratio:.3g}")
    _, d1_g, _ = oracle.loss_l1(v, img64, target, weight=0.8)
    dl_gpu = d1_g + dd_g
    go_g = oracle.backward(sc, v, init, dl_gpu)
    frag_px = ref["fragile"].astype(bool)
    m = np.tile(frag_px, 3)
    gf = oracle.backward(sc, v, init, np.where(m, dl_gpu, 0.0), want_g2d=True)
    ind = oracle.backward(sc, v, init, np.where(m, 1.0, 0.0), want_g2d=True)
    keep = ~(go_g["fragile_g"].astype(bool) | (np.abs(ind["g2d"]).sum(1) > 0))
    assert keep.mean() > 0.9, keep.mean()
    gg = {k_: v_.cpu().numpy() for k_, v_ in g.items()}
    _check_grads_large(gg, go_g, n, sc["sh_degree"], keep=keep)
    assert_pose_close(pg.cpu().numpy(), go_g["pose"], "pose (GPU L1 + D-SSIM)", slack=2.0 * np.abs(gf["pose"]))
    # gradients through the oracle's combined dL/dC, pixels with a near-threshold
    # decision (blend or the sign of the L1 term) zeroed on both sides
    frag = ref["fragile"].astype(bool) | fr1.astype(bool)
    dldc = d1 + dd
    dldc[np.tile(frag, 3)] = 0.0
    d32 = dldc.astype(np.float32)
    g2 = zero_grads(p)
    pg2 = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    R.backward(p, v, P, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=torch.from_numpy(d32).to(DEV)), g2, pg2)
    torch.cuda.synchronize()
    go = oracle.backward(sc, v, init, d32.astype(np.float64))
    _check_grads_large({k_: v_.cpu().numpy() for k_, v_ in g2.items()}, go, n, sc["sh_degree"])
    assert_pose_close(pg2.cpu().numpy(), go["pose"], "pose (oracle dL/dC)")


def test_trajectory_3M_8_frames_recompute_sampled_parity(R):
    """With the launch parameters the trajectory leg's autotuner picks for an
    8-frame batch (a fresh cache)."""
    w = synth.trajectory_workload()
    sc, views, poses = w["scene"], w["views"], w["poses"]
    n = len(sc["opac"])
    p = to_dev(sc)
    A = list(range(40, 48)); B = list(range(48, 56))
    vA, pA = _sub(views, poses, A)
    vB, pB = _sub(views, poses, B)
    PA, PB = poses_dev(pA), poses_dev(pB)
    _bench_configuration(R, p, vA, PA)
    try:
        _trajectory_parity(R, sc, p, vA, pA, PA, vB, PB, n)
    finally:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1, 1)


def _trajectory_parity(R, sc, p, vA, pA, PA, vB, PB, n):
    img = R.forward(p, vA, PA).clone()
    torch.cuda.synchronize()
    idx = [1, 6]
    vs, ps = _sub(vA, pA, idx)
    _oracle_threads(len(idx) * n)
    ref = oracle.render(sc, vs, ps)
    _check_images(img.cpu().numpy(), ref, vA, idx)
    R.forward(p, vB, PB)                       # the frames now hold batch B
    rng = np.random.default_rng(23)
    full, part = _sample_dldc(rng, vA, idx, ref)
    g = zero_grads(p)
    pg = torch.zeros(len(vA), 6, dtype=torch.float64, device=DEV)
    R.set_flags(L.GS_F_RECOMPUTE)
    try:
        R.backward(p, vA, PA, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=torch.from_numpy(full).to(DEV)), g, pg)
    finally:
        R.set_flags(0)
    torch.cuda.synchronize()
    go = oracle.backward(sc, vs, ps, part)
    _check_grads_large({k_: v_.cpu().numpy() for k_, v_ in g.items()}, go, n, sc["sh_degree"])
    pg = pg.cpu().numpy()
    assert_pose_close(pg[idx], go["pose"], "pose (3M trajectory sample)")
    assert np.all(np.delete(pg, idx, axis=0) == 0)
