"""Spatial (Morton) order of a scene's Gaussians (gs_spatial_order,
gs_gather_rows): the permutation equals numpy's ordering of the same FP32
grid codes, and rendering the reordered scene changes nothing but the order
of the per-Gaussian gradients (and of Gaussians at exactly equal depth)."""
import numpy as np
import pytest
import torch

from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import synth
from paper_2410_08743_gb300.render import Renderer

from .gpu_util import DEV, gpu_backward_dldc, poses_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def _spread(v):
    out = np.zeros_like(v, dtype=np.uint64)
    for b in range(10):
        out |= ((v.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def _morton_np(means):
    m = means.astype(np.float32)
    lo, hi = m.min(0), m.max(0)
    ext = (hi - lo).astype(np.float32)
    sc = np.where(ext > 0, np.float32(1024.0) / np.where(ext > 0, ext, np.float32(1)), np.float32(0)).astype(np.float32)
    q = np.floor(((m - lo).astype(np.float32) * sc).astype(np.float32))
    q = np.clip(q, 0, 1023).astype(np.uint64)
    return _spread(q[:, 0]) | (_spread(q[:, 1]) << np.uint64(1)) | (_spread(q[:, 2]) << np.uint64(2))


@pytest.mark.parametrize("n", [1, 1000, 100_003, 1_000_000])
def test_spatial_order_matches_numpy(R, n):
    rng = np.random.default_rng(n)
    means = rng.normal(0, 2, (n, 3)).astype(np.float32)
    means[: n // 10] = means[0]                         # many equal codes: ties go by index
    perm = torch.empty(n, dtype=torch.int32, device=DEV)
    L.gs_spatial_order(R.ctx, torch.from_numpy(means).to(DEV), perm)
    torch.cuda.synchronize()
    code = _morton_np(means)
    want = np.lexsort((np.arange(n), code))
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), want)


def test_reordered_scene_renders_the_same(R):
    rng = np.random.default_rng(9)
    sc = synth.make_scene_box(9, 20000, sh_degree=2, lo=(-1.5, -1, 3), hi=(1.5, 1, 6))
    # identity cameras see z_c = mu_z exactly: distinct mu_z leave no depth ties,
    # so the blending order cannot depend on the Gaussians' indices
    sc["means"][:, 2] = rng.permutation(np.linspace(3.0, 6.0, len(sc["opac"]))).astype(np.float32)
    assert len(np.unique(sc["means"][:, 2])) == len(sc["opac"])
    views = [dict(fx=60.0, fy=60.0, cx=48.0, cy=36.0, width=96, height=72),
             dict(fx=45.0, fy=47.0, cx=20.5, cy=16.0, width=40, height=33)]
    poses = np.stack([synth.pose_from_center(np.eye(3), np.zeros(3)) for _ in views])
    p = to_dev(sc)
    P = poses_dev(poses)
    img = R.forward(p, views, P).clone()
    dldc = (rng.standard_normal(img.numel()) * 1e-3).astype(np.float32)
    g, pg = gpu_backward_dldc(R, p, views, P, img, dldc)
    q, perm = L.spatially_ordered(R.ctx, p)
    img2 = R.forward(q, views, P).clone()
    assert torch.equal(img, img2)
    g2, pg2 = gpu_backward_dldc(R, q, views, P, img2, dldc)
    pm = perm.cpu().numpy().astype(np.int64)
    assert not np.array_equal(pm, np.arange(len(pm)))
    for k in g:
        np.testing.assert_allclose(g2[k], g[k][pm], rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(pg2, pg, rtol=1e-4, atol=1e-6 * np.abs(pg).max())
