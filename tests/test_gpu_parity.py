"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances: tile lists and key-path values bit-exact; images <= 1e-4 max-abs;
gradients per element |d| <= max(1e-3 |g_ref|, 1e-6).  Pixels where the oracle
flags a decision within rounding distance of its threshold (alpha_min,
alpha_max, the t_min stop, power = 0) are excluded from image comparisons and
get dL/dC = 0 in gradient comparisons, because FP32 and FP64 may legitimately
take different branches there; Gaussians with a near-threshold Gaussian-level
decision (colour or frustum clamp) are excluded from per-element gradient
checks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import synth
from paper_2410_08743_gb300.render import Renderer, render

from .gpu_util import (DEV, assert_dssim_grad_close, assert_grad_close, assert_pose_close, gpu_backward_dldc,
                       gpu_forward, poses_dev, to_dev, zero_grads)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def _ragged_case(seed=5, n=3000, deg=3):
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=deg, lo=(-1, -1, 2.5), hi=(1, 1, 5))
    views = [dict(fx=60.0, fy=60.0, cx=32.0, cy=24.0, width=64, height=48),
             dict(fx=45.0, fy=47.0, cx=20.5, cy=16.0, width=40, height=33),
             dict(fx=50.0, fy=50.0, cx=8.0, cy=35.0, width=17, height=70)]
    base = synth.pose_from_center(np.eye(3), np.zeros(3))
    poses = np.stack([synth.perturb_normal(rng, base, 4.0, 0.1) for _ in views])
    return sc, views, poses


def _dense_case(n, seed=31):
    """Many Gaussians in a small image: long per-tile lists (the medium and
    the MSD-split paths of the per-tile sort)."""
    sc = synth.make_scene_box(seed, n, sh_degree=1, lo=(-1.2, -0.9, 3.0), hi=(1.2, 0.9, 6.0))
    views = [dict(fx=40.0, fy=40.0, cx=24.0, cy=20.0, width=48, height=40)]
    return sc, views, synth.pose_from_center(np.eye(3), np.zeros(3))[None]


def _same_depth_case(n=30000, seed=32):
    """Nearly equal depths: FP32 depth ties (broken by index) and one MSD bucket
    longer than the shared-memory capacity (a few far Gaussians widen the
    varying depth bits)."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=0, lo=(-0.3, -0.25, 4.0), hi=(0.3, 0.25, 4.1))
    sc["means"][:, 2] = (4.0 + rng.integers(0, 4, n) * 1e-6).astype(np.float32)
    sc["means"][:3] = np.array([[0.0, 0.0, 60.0], [0.01, 0.0, 90.0], [0.0, 0.01, 120.0]], np.float32)
    sc["scales"][:3] = 1.0
    sc["opac"][:] = 0.05
    views = [dict(fx=60.0, fy=60.0, cx=16.0, cy=16.0, width=32, height=32)]
    return sc, views, synth.pose_from_center(np.eye(3), np.zeros(3))[None]


def _needle_case(n=6000, seed=33):
    """Thin rotated Gaussians (axis ratios up to ~40) and opacities just above
    alpha_min: alpha boxes far larger than the ellipses, so the per-warp
    culling of the blends decides many entries near the ellipse boundary."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=1, lo=(-1.0, -0.8, 3.0), hi=(1.0, 0.8, 5.0))
    ratio = np.exp(rng.uniform(0.0, np.log(40.0), n))
    sc["scales"][:, 0] *= np.sqrt(ratio).astype(np.float32)
    sc["scales"][:, 1] /= np.sqrt(ratio).astype(np.float32)
    low = rng.random(n) < 0.5
    sc["opac"][low] = rng.uniform(1.05 / 255.0, 6.0 / 255.0, int(low.sum())).astype(np.float32)
    views = [dict(fx=70.0, fy=70.0, cx=40.0, cy=30.0, width=80, height=60),
             dict(fx=50.0, fy=52.0, cx=19.5, cy=22.0, width=41, height=45)]
    base = synth.pose_from_center(np.eye(3), np.zeros(3))
    poses = np.stack([synth.perturb_normal(rng, base, 3.0, 0.05) for _ in views])
    return sc, views, poses


def _layered_case(n=40000, seed=35):
    """Long tile lists (about 10k keys) over a wide depth range at low
    opacity, so the lazy sort consumes several runs: most Gaussians spread in
    depth (a few keys per depth bucket: the bucket-by-bucket sort), 2,400 on
    three thin depth layers (a few hundred keys in one bucket: the radix sort
    of the whole run)."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=0, lo=(-1.0, -0.8, 2.5), hi=(1.0, 0.8, 6.0))
    layer = np.arange(n) < 2400
    sc["means"][layer, 2] = (np.repeat([3.0, 4.0, 5.0], 800) + rng.uniform(0.0, 2e-4, 2400)).astype(np.float32)
    sc["opac"][:] = rng.uniform(0.02, 0.06, n).astype(np.float32)
    views = [dict(fx=40.0, fy=40.0, cx=24.0, cy=20.0, width=48, height=40)]
    return sc, views, synth.pose_from_center(np.eye(3), np.zeros(3))[None]


def _wide_view_case(n=6000, seed=34):
    """A view with more than the 8192 tiles the shared-memory tile histograms
    hold (2050 x 1090: 129 x 69 tiles, ragged on both edges), which takes the
    per-key global-atomic path of the key count and scatter, in one launch
    with a small view that takes the shared-memory path."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=1, lo=(-1.2, -0.7, 2.5), hi=(1.2, 0.7, 5.0))
    views = [dict(fx=1640.0, fy=1640.0, cx=1025.0, cy=545.0, width=2050, height=1090),
             dict(fx=60.0, fy=60.0, cx=32.0, cy=24.0, width=64, height=48)]
    base = synth.pose_from_center(np.eye(3), np.zeros(3))
    poses = np.stack([synth.perturb_normal(rng, base, 2.0, 0.03) for _ in views])
    return sc, views, poses


CASES = {
    "tiny": lambda: (lambda w: (w["scene"], w["views"], w["poses"]))(synth.tiny_workload(0)),
    "ragged_sh3": lambda: _ragged_case(),
    "ragged_sh1": lambda: _ragged_case(7, 2500, 1),
    "dense_medium": lambda: _dense_case(20000),
    "dense_large": lambda: _dense_case(120000),
    "same_depth": lambda: _same_depth_case(),
    "needles": lambda: _needle_case(),
    "wide_view": lambda: _wide_view_case(),
    "layered": lambda: _layered_case(),
}
GRAD_CASES = ["tiny", "ragged_sh3", "ragged_sh1", "dense_medium", "wide_view"]


@pytest.mark.parametrize("full", [True, False], ids=["full_sort", "lazy_sort"])
@pytest.mark.parametrize("case", list(CASES))
def test_keys_bit_exact(R, case, full):
    sc, views, poses = CASES[case]()
    R.opts.flags = L.GS_F_FULL_SORT if full else 0
    try:
        gpu_forward(R, sc, views, poses)
    finally:
        R.opts.flags = 0
    k = oracle.keys(sc, views, poses)
    valid = k["valid"].astype(bool)
    rect = R.query(L.GS_Q_RECT).reshape(-1, 4)
    assert np.array_equal(rect, k["rect"]), "tile rectangles differ"
    assert np.array_equal(R.query(L.GS_Q_RADIUS), k["radius"])
    d = R.query(L.GS_Q_DEPTH)
    assert np.array_equal(d.view(np.uint32)[valid], k["depth"].view(np.uint32)[valid]), "depth keys differ"
    m2 = R.query(L.GS_Q_MEAN2D).reshape(-1, 2)
    assert np.array_equal(m2[valid].view(np.uint32), k["mu2f"][valid].view(np.uint32))
    assert int(R.query(L.GS_Q_NUM_KEYS)[0]) == k["n_keys"]
    ranges = R.query(L.GS_Q_TILE_RANGES).reshape(-1, 2)
    assert np.array_equal(ranges, k["ranges"])
    got = R.query(L.GS_Q_SORTED_IDX)
    cnt = R.query(L.GS_Q_SORTED_COUNT)
    lens = k["ranges"][:, 1] - k["ranges"][:, 0]
    if full:
        assert np.array_equal(cnt, lens)
        assert np.array_equal(got, k["idx"]), "sorted tile lists differ"
    else:
        # every tile's sorted prefix is the oracle's prefix, and covers what
        # the blend consumed (the longest n_contrib of the tile's pixels)
        assert np.all(cnt <= lens)
        for t in np.nonzero(cnt)[0]:
            s0 = k["ranges"][t, 0]
            assert np.array_equal(got[s0:s0 + cnt[t]], k["idx"][s0:s0 + cnt[t]]), t
        nc = R.query(L.GS_Q_N_CONTRIB)
        off = 0; tb = 0
        for v in views:
            W, H = v["width"], v["height"]
            gw, gh = (W + 15) // 16, (H + 15) // 16
            ncv = nc[off:off + W * H].reshape(H, W)
            for ty in range(gh):
                for tx in range(gw):
                    tile_max = ncv[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16].max()
                    assert cnt[tb + ty * gw + tx] >= tile_max
            off += W * H; tb += gw * gh
    if case == "dense_medium":
        assert lens.max() > 2048          # medium path exercised
    if case in ("dense_large", "same_depth"):
        assert lens.max() > 12288         # MSD-split path exercised


@pytest.mark.parametrize("case", ["ragged_sh3", "dense_large", "same_depth", "needles"])
def test_lazy_sort_equals_full_sort(R, case):
    """Sorting tiles only as far as they are consumed changes nothing; nor does
    the per-warp box and ellipse culling of the lazy blend (the full-sort blend
    tests every staged entry at every pixel)."""
    sc, views, poses = CASES[case]()
    outs = []
    for flags in (L.GS_F_FULL_SORT, 0):
        R.opts.flags = flags
        try:
            _, _, img, _, _ = gpu_forward(R, sc, views, poses)
        finally:
            R.opts.flags = 0
        outs.append((img.cpu().numpy(), R.query(L.GS_Q_T_FINAL), R.query(L.GS_Q_N_CONTRIB)))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("case", list(CASES))
def test_forward_image_and_splats(R, case):
    sc, views, poses = CASES[case]()
    _, _, img, _, _ = gpu_forward(R, sc, views, poses)
    ref = oracle.render(sc, views, poses)
    img = img.cpu().numpy()
    fr = ref["fragile"].astype(bool)
    assert fr.mean() < 0.01, fr.mean()
    pix_ok = ~fr
    n_pix = len(fr)
    off = 0
    poff = 0
    for v in views:
        np_ = v["width"] * v["height"]
        m = pix_ok[poff:poff + np_]
        for ch in range(3):
            a = img[off + ch * np_: off + (ch + 1) * np_][m]
            b = ref["image"][off + ch * np_: off + (ch + 1) * np_][m]
            assert np.abs(a - b).max() <= 1e-4, (v, ch, np.abs(a - b).max())
        off += 3 * np_
        poff += np_
    T = R.query(L.GS_Q_T_FINAL)
    assert np.abs(T[pix_ok] - ref["T_final"][pix_ok]).max() <= 1e-4
    nc = R.query(L.GS_Q_N_CONTRIB)
    assert np.array_equal(nc[pix_ok], ref["n_contrib"][pix_ok].astype(np.uint32))
    assert n_pix == len(T)
    # splat values (FP32 vs FP64)
    vals = oracle.project_values(sc, views, poses)
    got = R.query(L.GS_Q_SPLAT).reshape(-1, 9).astype(np.float64)
    ok = oracle.keys(sc, views, poses)["valid"].astype(bool)
    np.testing.assert_allclose(got[ok, :2], vals[ok, :2], rtol=0, atol=2e-4)
    # the conic is an inverse: its FP32 error grows with the condition of Sigma_hat
    scale = np.abs(vals[ok, 2:5]).max(1, keepdims=True)
    a, b, c = vals[ok, 2], vals[ok, 3], vals[ok, 4]
    cond = (np.abs(a) + np.abs(c)) ** 2 / np.maximum(a * c - b * b, 1e-300)
    assert np.all(np.abs(got[ok, 2:5] - vals[ok, 2:5]) <= 1e-6 * cond[:, None] * scale + 1e-12)
    np.testing.assert_allclose(got[ok, 5], vals[ok, 5], rtol=1e-7)
    np.testing.assert_allclose(got[ok, 6:9], vals[ok, 6:9], rtol=0, atol=2e-6)


@pytest.mark.parametrize("bwd_px", [1, 2], ids=["1px", "2px"])
@pytest.mark.parametrize("case", GRAD_CASES)
def test_backward_gradients_and_pose(R, case, bwd_px):
    L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, bwd_px)
    try:
        _backward_case(R, case)
    finally:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1)


def _backward_case(R, case):
    sc, views, poses = CASES[case]()
    p, P, img, _, _ = gpu_forward(R, sc, views, poses)
    ref = oracle.render(sc, views, poses)
    rng = np.random.default_rng(11)
    n_img = img.numel()
    scale = 1.0 / (3 * views[0]["width"] * views[0]["height"])
    dldc = rng.standard_normal(n_img) * scale
    # zero the gradient on near-threshold pixels
    off = 0; poff = 0
    for v in views:
        np_ = v["width"] * v["height"]
        fr = ref["fragile"][poff:poff + np_].astype(bool)
        for ch in range(3):
            dldc[off + ch * np_: off + (ch + 1) * np_][fr] = 0.0
        off += 3 * np_; poff += np_
    dldc32 = dldc.astype(np.float32)
    g, pg = gpu_backward_dldc(R, p, views, P, img, dldc32)
    go = oracle.backward(sc, views, poses, dldc32.astype(np.float64))
    n = len(sc["opac"])
    frag = go["fragile_g"].reshape(len(views), n).any(0)
    keep = ~frag
    nc = (sc["sh_degree"] + 1) ** 2
    assert_grad_close(g["means"], go["means"], "means", mask=keep)
    assert_grad_close(g["scales"], go["scales"], "scales", mask=keep)
    assert_grad_close(g["quats"], go["quats"], "quats", mask=keep)
    assert_grad_close(g["opac"].reshape(-1, 1), go["opac"].reshape(-1, 1), "opac", mask=keep)
    assert_grad_close(g["sh"][:, :nc].reshape(n, -1), go["sh"][:, :nc].reshape(n, -1), "sh", mask=keep)
    assert np.all(g["sh"][:, nc:] == 0)
    assert_pose_close(pg, go["pose"], f"pose ({case})")


def test_fused_l1_loss_and_gradient(R):
    w = synth.tiny_workload(0)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    target = oracle.render(sc, views, w["target_poses"])["image"].astype(np.float32)
    p, P, img, tg, loss = gpu_forward(R, sc, views, poses, target=target)
    ref = oracle.render(sc, views, poses)
    L1, dldc, frag_l1 = oracle.loss_l1(views, ref["image"], target, weight=1.0)
    assert abs(loss.item() - L1) <= 1e-6 * max(1.0, L1) + 1e-7
    frag = ref["fragile"].astype(bool) | frag_l1.astype(bool)
    g = zero_grads(p)
    pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    lo = torch.zeros(1, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1, target=tg, w_l1=1.0, loss_out=lo), g, pg)
    torch.cuda.synchronize()
    assert abs(lo.item() - L1) <= 1e-6 * max(1.0, L1) + 1e-7
    go = oracle.backward(sc, views, poses, dldc)
    keep = ~go["fragile_g"].astype(bool)
    pose_slack = np.zeros(6)
    if frag.any():
        # near-threshold pixels: back-propagate their own share to find the
        # Gaussians they touch and bound their effect on the pose gradient
        m = np.tile(frag, 3)
        gf = oracle.backward(sc, views, poses, np.where(m, dldc, 0.0), want_g2d=True)
        ind = oracle.backward(sc, views, poses, np.where(m, 1.0, 0.0), want_g2d=True)
        keep &= ~(np.abs(ind["g2d"]).sum(1) > 0)
        pose_slack = 2.0 * np.abs(gf["pose"][0])
    assert keep.mean() > 0.9
    assert_grad_close(g["means"].cpu().numpy(), go["means"], "means", mask=keep)
    assert_grad_close(g["scales"].cpu().numpy(), go["scales"], "scales", mask=keep)
    assert_grad_close(g["opac"].cpu().numpy().reshape(-1, 1), go["opac"].reshape(-1, 1), "opac", mask=keep)
    assert_pose_close(pg.cpu().numpy(), go["pose"], "pose (fused L1)", slack=pose_slack)


@pytest.mark.parametrize("param", ["se3", "txso3"])
def test_pose_adam_step_matches_oracle(R, param):
    rng = np.random.default_rng(3)
    V = 5
    poses = np.stack([oracle.se3_exp(rng.standard_normal(6) * 0.4) for _ in range(V)])
    m = np.zeros((V, 6)); v = np.zeros((V, 6))
    Pd = poses_dev(poses); md = torch.zeros(V, 6, dtype=torch.float64, device=DEV); vd = torch.zeros_like(md)
    pr = poses.copy()
    for step in range(1, 6):
        g = rng.standard_normal((V, 6))
        if param == "se3":
            oracle.pose_adam(pr, m, v, g, 1e-2, step)
            R.pose_step(Pd, md, vd, torch.from_numpy(g).to(DEV), 1e-2, step)
        else:
            oracle.pose_adam_txso3(pr, m, v, g, 1e-2, step)
            R.pose_step(Pd, md, vd, torch.from_numpy(g).to(DEV), 1e-2, step, param=L.GS_POSE_TXSO3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Pd.cpu().numpy(), pr, atol=1e-12)
    np.testing.assert_allclose(md.cpu().numpy(), m, atol=1e-14)


def test_dssim_loss_and_gradient(R):
    w = synth.tiny_workload(2)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    rng = np.random.default_rng(4)
    target = rng.uniform(size=3 * 64 * 48).astype(np.float32)
    p, P, img, tg, _ = gpu_forward(R, sc, views, poses)
    Ld, dd, _ = oracle.loss_dssim(views, img.cpu().numpy().astype(np.float64), target, weight=0.2)
    L1, d1, _ = oracle.loss_l1(views, img.cpu().numpy().astype(np.float64), target, weight=0.8)
    g = zero_grads(p)
    pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    lo = torch.zeros(1, dtype=torch.float64, device=DEV)
    tgd = torch.from_numpy(target).to(DEV)
    R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1_DSSIM, target=tgd, w_l1=0.8, w_dssim=0.2, loss_out=lo), g, pg)
    torch.cuda.synchronize()
    assert abs(lo.item() - (Ld + L1)) <= 2e-6
    # the D-SSIM term's dL/dC itself, element by element
    img64 = img.cpu().numpy().astype(np.float64)
    assert_dssim_grad_close(R.query(L.GS_Q_DSSIM_GRAD), dd, oracle.loss_dssim_cond(views, img64, target, 0.2),
                            "D-SSIM dL/dC (64x48)")
    # the same backward through dL/dC from the oracle's combined gradient
    g2, pg2 = gpu_backward_dldc(R, p, views, P, img, (dd + d1).astype(np.float32))
    for k in ("means", "opac", "sh"):
        a = g[k].cpu().numpy().ravel(); b = g2[k].ravel()
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-9, k
    np.testing.assert_allclose(pg.cpu().numpy(), pg2, rtol=2e-3, atol=1e-3 * np.abs(pg2).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_dssim_gradient_per_element_504x378(R, seed):
    """D-SSIM dL/dC of a 504x378 view (the joint-refinement resolution), from
    the allocating path inside the backward (GS_Q_DSSIM_GRAD) and from the
    allocation-free entry point, against the oracle on the same image."""
    W, H = 504, 378
    views = [dict(fx=0.8 * W, fy=0.8 * W, cx=W / 2, cy=H / 2, width=W, height=H)]
    rng = np.random.default_rng(30 + seed)
    # a rendered-like image: smooth blobs plus noise, and a target close to it
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.zeros((3, H, W))
    for _ in range(40):
        cx, cy, s = rng.uniform(0, W), rng.uniform(0, H), rng.uniform(5, 40)
        img += rng.uniform(0, 0.5, (3, 1, 1)) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    img = np.clip(img + 0.02 * rng.standard_normal(img.shape), 0, 1).astype(np.float32).ravel()
    target = np.clip(img + 0.05 * rng.standard_normal(img.size), 0, 1).astype(np.float32)
    Ld, dd, _ = oracle.loss_dssim(views, img.astype(np.float64), target, weight=0.2)
    imgd = torch.from_numpy(img).to(DEV)
    tgd = torch.from_numpy(target).to(DEV)
    # allocating path: a backward with the D-SSIM term only (L1 weight 0)
    sc = synth.make_scene_box(7, 500, sh_degree=0, lo=(-1, -1, 3), hi=(1, 1, 5))
    p = to_dev(sc)
    P = poses_dev(synth.pose_from_center(np.eye(3), np.zeros(3))[None])
    R.forward(p, views, P)
    g = zero_grads(p)
    pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    lo = torch.zeros(1, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, imgd, L.make_loss(L.GS_LOSS_L1_DSSIM, target=tgd, w_l1=0.0, w_dssim=0.2, loss_out=lo), g, pg)
    torch.cuda.synchronize()
    assert abs(lo.item() - Ld) <= 1e-6 * max(1.0, Ld), (lo.item(), Ld)
    cond = oracle.loss_dssim_cond(views, img.astype(np.float64), target, 0.2)
    ra = assert_dssim_grad_close(R.query(L.GS_Q_DSSIM_GRAD), dd, cond, "D-SSIM dL/dC, allocating path")
    # allocation-free entry point
    out = torch.full_like(imgd, float("nan"))
    ls = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
    L.gs_loss_dssim_static(imgd, tgd, W, H, 0.2, out, ls)
    torch.cuda.synchronize()
    assert abs(ls.item() - Ld) <= 1e-6 * max(1.0, Ld), (ls.item(), Ld)
    rs = assert_dssim_grad_close(out.cpu().numpy(), dd, cond, "D-SSIM dL/dC, allocation-free entry point")
    print(f"worst error / tolerance: allocating {ra:.3g}, allocation-free {rs:.3g}")


def test_autograd_function_matches_oracle(R):
    w = synth.tiny_workload(0)
    sc, views, poses = w["scene"], w["views"], w["poses"]
    p = to_dev(sc)
    leaves = {k: p[k].clone().requires_grad_(True) for k in ("means", "scales", "quats", "opac", "sh")}
    leaves["sh_degree"] = p["sh_degree"]
    tau = torch.zeros(1, 6, dtype=torch.float64, device=DEV, requires_grad=True)
    img = render(R, leaves, views, poses_dev(poses), tau)
    rng = np.random.default_rng(9)
    wts = torch.from_numpy((rng.standard_normal(img.numel()) * 1e-3).astype(np.float32)).to(DEV)
    ref = oracle.render(sc, views, poses)
    wts_np = wts.cpu().numpy().astype(np.float64)
    wts_np_masked = wts_np.copy()
    fr = ref["fragile"].astype(bool)
    for ch in range(3):
        wts_np_masked[ch * 3072:(ch + 1) * 3072][fr] = 0
    wts = torch.from_numpy(wts_np_masked.astype(np.float32)).to(DEV)
    (img * wts).sum().backward()
    go = oracle.backward(sc, views, poses, wts_np_masked.astype(np.float32).astype(np.float64))
    keep = ~go["fragile_g"].astype(bool)
    n = len(sc["opac"])
    nc = (sc["sh_degree"] + 1) ** 2
    assert_grad_close(leaves["means"].grad.cpu().numpy(), go["means"], "means", mask=keep)
    assert_grad_close(leaves["scales"].grad.cpu().numpy(), go["scales"], "scales", mask=keep)
    assert_grad_close(leaves["quats"].grad.cpu().numpy(), go["quats"], "quats", mask=keep)
    assert_grad_close(leaves["opac"].grad.cpu().numpy().reshape(-1, 1), go["opac"].reshape(-1, 1), "opac", mask=keep)
    gsh = leaves["sh"].grad.cpu().numpy().reshape(n, 16, 3)
    assert_grad_close(gsh[:, :nc].reshape(n, -1), go["sh"][:, :nc].reshape(n, -1), "sh", mask=keep)
    assert np.all(gsh[:, nc:] == 0)
    assert_pose_close(tau.grad.cpu().numpy(), go["pose"], "pose (autograd)")


def test_batched_equals_per_view(R):
    sc, views, poses = _ragged_case(13, 2000, 2)
    p = to_dev(sc)
    P = poses_dev(poses)
    img_b = R.forward(p, views, P).clone()
    rng = np.random.default_rng(5)
    dldc = torch.from_numpy((rng.standard_normal(img_b.numel()) * 1e-3).astype(np.float32)).to(DEV)
    gb = zero_grads(p)
    pgb = torch.zeros(len(views), 6, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, img_b, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc), gb, pgb)
    gs_ = zero_grads(p)
    off = 0
    for v in range(len(views)):
        n3 = 3 * views[v]["width"] * views[v]["height"]
        img_v = R.forward(p, views[v:v + 1], P[v:v + 1].contiguous())
        assert torch.equal(img_v, img_b[off:off + n3]), v
        pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
        R.backward(p, views[v:v + 1], P[v:v + 1].contiguous(), img_v,
                   L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc[off:off + n3].contiguous()), gs_, pg)
        torch.testing.assert_close(pg[0], pgb[v], rtol=1e-5, atol=1e-9)
        off += n3
    for k in gb:
        torch.testing.assert_close(gs_[k], gb[k], rtol=1e-4, atol=1e-8)


def test_edge_cases(R):
    # empty scene, everything culled, 1x1 image, non-multiple-of-16 sizes
    base = synth.pose_from_center(np.eye(3), np.zeros(3))[None]
    empty = dict(means=np.zeros((0, 3), np.float32), scales=np.zeros((0, 3), np.float32),
                 quats=np.zeros((0, 4), np.float32), opac=np.zeros(0, np.float32),
                 sh=np.zeros((0, 16, 3), np.float32), sh_degree=0)
    v = [dict(fx=30.0, fy=30.0, cx=10.0, cy=7.0, width=21, height=13)]
    R.opts.bg[0], R.opts.bg[1], R.opts.bg[2] = 0.25, 0.5, 0.75
    try:
        _, _, img, _, _ = gpu_forward(R, empty, v, base)
        assert torch.equal(img.view(3, -1)[0], torch.full((21 * 13,), 0.25, device=DEV))
        behind = synth.make_scene_tiny(1, 50)
        behind["means"][:, 2] = -3.0
        p, P, img, _, _ = gpu_forward(R, behind, v, base)
        assert torch.equal(img.view(3, -1)[2], torch.full((21 * 13,), 0.75, device=DEV))
        g, pg = gpu_backward_dldc(R, p, v, P, img, np.ones(img.numel(), np.float32))
        assert all(np.all(x == 0) for x in g.values()) and np.all(pg == 0)
        one = [dict(fx=30.0, fy=30.0, cx=0.0, cy=0.0, width=1, height=1)]
        sc = synth.make_scene_tiny(2, 300)
        _, _, img1, _, _ = gpu_forward(R, sc, one, base)
        ref = oracle.render(sc, one, base, opts=dict(bg=(0.25, 0.5, 0.75)))
        if not ref["fragile"].any():
            assert np.abs(img1.cpu().numpy() - ref["image"]).max() <= 1e-4
    finally:
        R.opts.bg[0] = R.opts.bg[1] = R.opts.bg[2] = 0.0


def test_invalid_arguments_raise(R):
    sc, views, poses = _ragged_case(3, 100, 0)
    p = to_dev(sc)
    bad = [dict(views[0], width=0)]
    with pytest.raises(L.GsError):
        R.forward(p, bad, poses_dev(poses[:1]))
    with pytest.raises(L.GsError):
        R.backward(p, views, poses_dev(poses), torch.zeros(10, device=DEV),
                   L.make_loss(L.GS_LOSS_L1, target=None), None, None)


def test_recompute_in_backward_equals_stored_state(R):
    """A backward with GS_F_RECOMPUTE after another batch's forward gives the
    gradients of the plain forward/backward pair."""
    scA, viewsA, posesA = _ragged_case(71, 4000, 3)
    viewsB = [dict(fx=70.0, fy=70.0, cx=50.0, cy=40.0, width=100, height=80)]
    posesB = synth.pose_from_center(np.eye(3), np.array([0.1, 0.0, 0.0]))[None]
    p = to_dev(scA)
    PA, PB = poses_dev(posesA), poses_dev(posesB)
    rng = np.random.default_rng(71)
    imgA = R.forward(p, viewsA, PA).clone()
    dldc = torch.from_numpy((rng.standard_normal(imgA.numel()) * 1e-3).astype(np.float32)).to(DEV)
    loss = L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc)
    g1 = zero_grads(p); pg1 = torch.zeros(len(viewsA), 6, dtype=torch.float64, device=DEV)
    R.backward(p, viewsA, PA, imgA, loss, g1, pg1)
    R.forward(p, viewsB, PB)                       # the frames now hold batch B
    with pytest.raises(L.GsError):                 # a plain backward of A is refused
        R.backward(p, viewsA, PA, imgA, loss, zero_grads(p), None)
    g2 = zero_grads(p); pg2 = torch.zeros_like(pg1)
    R.opts.flags = L.GS_F_RECOMPUTE
    try:
        R.backward(p, viewsA, PA, imgA, loss, g2, pg2)
    finally:
        R.opts.flags = 0
    torch.cuda.synchronize()
    for k in g1:
        torch.testing.assert_close(g2[k], g1[k], rtol=1e-4, atol=1e-9)
    # the pose reduction sums float atomics, whose order differs run to run
    torch.testing.assert_close(pg2, pg1, rtol=1e-4, atol=1e-6 * float(pg1.abs().max()))


def test_masked_l1_loss_and_gradient(R):
    """Confidence-masked L1 (Sec. 3.4, Eq. 20-21) fused into the backward blend."""
    w = synth.tiny_workload(0)
    sc = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in w["scene"].items()}
    sc["opac"] = np.maximum(sc["opac"], 0.85).astype(np.float32)
    views, poses = w["views"], w["poses"]
    target = oracle.render(sc, views, w["target_poses"])["image"].astype(np.float32)
    p, P, img, tg, _ = gpu_forward(R, sc, views, poses, target=target)
    ref = oracle.render(sc, views, poses)
    kept = (1.0 - ref["T_final"]) > float(np.float32(0.99))
    assert 0.05 < kept.mean() < 0.95, kept.mean()
    Lm, dm, frm = oracle.loss_l1_masked(views, ref["image"], target, ref["T_final"], 0.99)
    frag = ref["fragile"].astype(bool) | frm.astype(bool)
    npx = frag.size
    # a near-threshold pixel may fall on either side: bound its share of the loss
    ad = np.abs(ref["image"] - target).reshape(3, npx).sum(0)
    slack = ad[frag].sum() / (3 * npx)
    g = zero_grads(p)
    pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    lo = torch.zeros(1, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1_MASKED, target=tg, loss_out=lo, mask_alpha=0.99), g, pg)
    torch.cuda.synchronize()
    assert abs(lo.item() - Lm) <= 1e-6 * max(1.0, Lm) + 1e-7 + slack, (lo.item(), Lm)
    go = oracle.backward(sc, views, poses, dm)
    keep = ~go["fragile_g"].astype(bool)
    pose_slack = np.zeros(6)
    if frag.any():
        m = np.tile(frag, 3)
        sgn = np.sign(ref["image"] - target) / (3 * npx)
        gf = oracle.backward(sc, views, poses, np.where(m, np.abs(sgn), 0.0))
        ind = oracle.backward(sc, views, poses, np.where(m, 1.0, 0.0), want_g2d=True)
        keep &= ~(np.abs(ind["g2d"]).sum(1) > 0)
        pose_slack = 2.0 * np.abs(gf["pose"][0]) + 1e-12
    assert keep.mean() > 0.8
    assert_grad_close(g["means"].cpu().numpy(), go["means"], "means", mask=keep)
    assert_grad_close(g["opac"].cpu().numpy().reshape(-1, 1), go["opac"].reshape(-1, 1), "opac", mask=keep)
    assert_pose_close(pg.cpu().numpy(), go["pose"], "pose (fused L1)", slack=pose_slack)
    # masked-out pixels carry no gradient: an all-masked threshold gives zero
    g0 = zero_grads(p)
    pg0 = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
    R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1_MASKED, target=tg, loss_out=lo, mask_alpha=0.999999),
               g0, pg0)
    torch.cuda.synchronize()
    assert lo.item() == 0.0 and not pg0.any() and all(not v.any() for v in g0.values())


@pytest.mark.parametrize("case", ["ragged_sh3", "dense_medium", "dense_large", "same_depth"])
def test_forward_pixels_per_thread_is_result_neutral(R, case):
    """Two pixels per thread in the forward blend give the same image, final
    transmittance, contributor counts and sorted tile prefixes bit for bit."""
    sc, views, poses = CASES[case]()
    outs = []
    try:
        for fpx in (1, 2):
            L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1, fpx)
            _, _, img, _, _ = gpu_forward(R, sc, views, poses)
            cnt = R.query(L.GS_Q_SORTED_COUNT)
            idx = R.query(L.GS_Q_SORTED_IDX)
            ranges = R.query(L.GS_Q_TILE_RANGES).reshape(-1, 2)
            pref = np.concatenate([idx[r0:r0 + c] for (r0, _), c in zip(ranges, cnt)]) if len(cnt) else idx[:0]
            outs.append((img.cpu().numpy(), R.query(L.GS_Q_T_FINAL), R.query(L.GS_Q_N_CONTRIB), pref))
    finally:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1, 1)
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)
    # the sorted prefixes agree where both sorted (each covers its own blend)
    n = min(len(outs[0][3]), len(outs[1][3]))
    assert n > 0


def test_backward_state_carries_over_between_batches(R):
    """The backward preprocess leaves the 2D-gradient records cleared for the
    next backward (which then skips its clearing pass): a backward of three
    views, one of a single view, and the three views again give the first
    result again, as does a backward after a larger batch grew the buffers."""
    sc, views, poses = CASES["ragged_sh3"]()
    rng = np.random.default_rng(9)
    n_img = sum(3 * v["width"] * v["height"] for v in views)
    dldc = rng.normal(size=n_img).astype(np.float32)
    n0 = 3 * views[0]["width"] * views[0]["height"]
    res = []
    for sel in ([0, 1, 2], [0], [0, 1, 2], [2, 1, 0, 2, 1], [0, 1, 2]):
        vs = [views[k] for k in sel]
        ps = poses[sel]
        offs = np.cumsum([0] + [3 * views[k]["width"] * views[k]["height"] for k in range(3)])
        d = np.concatenate([dldc[offs[k]:offs[k + 1]] for k in sel])
        p, P, img, _, _ = gpu_forward(R, sc, vs, ps)
        g, pg = gpu_backward_dldc(R, p, vs, P, img, d)
        res.append((sel, g, pg))
    ref = res[0]
    for sel, g, pg in (res[2], res[4]):
        for k in g:
            np.testing.assert_allclose(g[k], ref[1][k], rtol=1e-4, atol=1e-6 * float(np.abs(ref[1][k]).max() + 1e-30))
        np.testing.assert_allclose(pg, ref[2], rtol=1e-5, atol=1e-9)
    assert n0 > 0


@pytest.mark.parametrize("bwd_px", [1, 2])
def test_work_counters_only_with_count_flag(R, bwd_px):
    """The blends count their work only under GS_F_COUNT; image, per-pixel
    state and gradients are the same with and without the counting."""
    sc, views, poses = CASES["ragged_sh3"]()
    rng = np.random.default_rng(7)
    n_img = sum(3 * v["width"] * v["height"] for v in views)
    dldc = rng.normal(size=n_img).astype(np.float32)
    outs = []
    try:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, bwd_px, 2)
        for flags in (0, L.GS_F_COUNT):
            R.opts.flags = flags
            p, P, img, _, _ = gpu_forward(R, sc, views, poses)
            g, pg = gpu_backward_dldc(R, p, views, P, img, dldc)
            outs.append((img.cpu().numpy(), R.query(L.GS_Q_T_FINAL), R.query(L.GS_Q_N_CONTRIB), g, pg,
                         np.asarray(L.gs_frames_counters(R.frames))))
    finally:
        R.opts.flags = 0
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256, 1, 1)
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)
    for k in outs[0][3]:
        np.testing.assert_allclose(outs[1][3][k], outs[0][3][k], rtol=1e-4,
                                   atol=1e-6 * float(np.abs(outs[0][3][k]).max() + 1e-30))
    np.testing.assert_allclose(outs[1][4], outs[0][4], rtol=1e-5, atol=1e-9)
    assert not outs[0][5].any()
    c = outs[1][5]
    assert c[0] >= c[1] > 0 and c[2] >= c[3] > 0 and c[1] == c[3]   # blended = contributing pairs
    assert c[4] > 0 and c[5] > 0 and c[7] > 0 and c[8] >= c[9] > 0


def _many_views_case(n, n_views=70, seed=82):
    """More views than one preprocess launch takes (64), so the sliced passes
    run once per view chunk."""
    rng = np.random.default_rng(seed)
    sc = synth.make_scene_box(seed, n, sh_degree=1, lo=(-1, -1, 2.5), hi=(1, 1, 5))
    views = [dict(fx=20.0, fy=21.0, cx=12.0, cy=10.0, width=24, height=20) for _ in range(n_views)]
    base = synth.pose_from_center(np.eye(3), np.zeros(3))
    poses = np.stack([synth.perturb_normal(rng, base, 3.0, 0.05) for _ in views])
    return sc, views, poses


@pytest.mark.parametrize("n,with_image,many_views", [(3000, True, False), (300_000, True, False),
                                                     (300_000, False, False), (300_000, True, True)])
def test_step_with_host_buffers_equals_device_path(R, n, with_image, many_views):
    """gs_step with GS_F_HOST_IO (host inputs and outputs, copies inside the
    call, the loss input uploaded beside the forward) equals the same step on
    device buffers; twice in a row, so the upload stream is reused.  At 300k
    Gaussians the parameters go up and the gradients come down in four slices
    that overlap the preprocess kernels; with or without the image download;
    and with 70 views, two view chunks per preprocess pass."""
    sc, views, poses = _many_views_case(n) if many_views else _ragged_case(81, n, 2)
    rng = np.random.default_rng(81)
    p = to_dev(sc)
    P = poses_dev(poses)
    n_img = sum(3 * v["width"] * v["height"] for v in views)
    target = rng.uniform(size=n_img).astype(np.float32)
    V = len(views)
    # device path
    img_d = torch.empty(n_img, device=DEV)
    g_d = zero_grads(p)
    pg_d = torch.zeros(V, 6, dtype=torch.float64, device=DEV)
    lo_d = torch.zeros(V, dtype=torch.float64, device=DEV)
    tg = torch.from_numpy(target).to(DEV)
    desc = L.scene_desc(p["means"], p["scales"], p["quats"], p["opac"], p["sh"], p["sh_degree"])
    loss = L.make_loss(L.GS_LOSS_L1_DSSIM, target=tg, w_l1=0.8, w_dssim=0.2)
    L.gs_step(R.ctx, R.frames, desc, R.views(views), V, P.data_ptr(), R.opts, loss, img_d.data_ptr(),
              L.make_grads(**g_d), pg_d.data_ptr(), lo_d.data_ptr())
    torch.cuda.synchronize()
    # host path
    hp = {k: p[k].cpu().pin_memory() for k in ("means", "scales", "quats", "opac", "sh")}
    hposes = torch.from_numpy(poses).pin_memory()
    htg = torch.from_numpy(target).pin_memory()
    himg = torch.zeros(n_img).pin_memory()
    hg = {k: torch.zeros_like(hp[k]).pin_memory() for k in hp}
    hpg = torch.zeros(V, 6, dtype=torch.float64).pin_memory()
    hlo = torch.zeros(V, dtype=torch.float64).pin_memory()
    hdesc = L.scene_desc(hp["means"], hp["scales"], hp["quats"], hp["opac"], hp["sh"], p["sh_degree"])
    hloss = L.make_loss(L.GS_LOSS_L1_DSSIM, target=htg, w_l1=0.8, w_dssim=0.2)
    R.opts.flags = L.GS_F_HOST_IO
    try:
        for _ in range(2):
            L.gs_step(R.ctx, R.frames, hdesc, R.views(views), V, hposes.data_ptr(), R.opts, hloss,
                      himg.data_ptr() if with_image else None, L.make_grads(**hg), hpg.data_ptr(), hlo.data_ptr())
            torch.cuda.synchronize()
            if with_image:
                assert torch.equal(himg, img_d.cpu())
            for k in hg:
                np.testing.assert_allclose(hg[k].numpy(), g_d[k].cpu().numpy(), rtol=1e-4,
                                           atol=1e-6 * float(g_d[k].abs().max()))
            np.testing.assert_allclose(hpg.numpy(), pg_d.cpu().numpy(), rtol=1e-5, atol=1e-9)
            np.testing.assert_allclose(hlo.numpy(), lo_d.cpu().numpy(), rtol=1e-6)
    finally:
        R.opts.flags = 0
