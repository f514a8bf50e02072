"""Pins of the oracle's relative-pose initialisation (Sec. 3.4).

* Unprojection: projecting every returned point with the pinhole model gives
  back its grid pixel and depth (the inverse map), pixels without depth are
  skipped, and colours are the image's at those pixels.
* The neighbour scale equals scipy's k-d tree query (library routine).
* Depth maps of the synthetic room unproject onto the room's surfaces (the
  depth and pixel conventions agree with the renderer's)."""
import numpy as np
import scipy.spatial

import oracle
from paper_2410_08743_gb300 import synth


def test_unprojection_inverts_projection():
    rng = np.random.default_rng(0)
    view = dict(fx=70.0, fy=65.0, cx=31.5, cy=22.0, width=61, height=45)
    depth = rng.uniform(0.5, 4.0, (45, 61)).astype(np.float32)
    depth[rng.uniform(size=depth.shape) < 0.1] = 0.0
    depth[3, 4] = np.nan
    img = rng.uniform(size=3 * 61 * 45).astype(np.float32)
    pts, cols = oracle.unproject(view, depth, img, 3)
    vs, us = np.mgrid[0:45:3, 0:61:3]
    d = depth[vs, us].ravel()
    ok = d > 0
    assert len(pts) == ok.sum()
    u = view["fx"] * pts[:, 0] / pts[:, 2] + view["cx"]
    v = view["fy"] * pts[:, 1] / pts[:, 2] + view["cy"]
    np.testing.assert_allclose(u, us.ravel()[ok], atol=1e-9)
    np.testing.assert_allclose(v, vs.ravel()[ok], atol=1e-9)
    np.testing.assert_array_equal(pts[:, 2], d[ok].astype(np.float64))
    planes = img.reshape(3, 45, 61)
    for c in range(3):
        np.testing.assert_array_equal(cols[:, c], planes[c][vs, us].ravel()[ok].astype(np.float64))


def test_knn_mean_distance_matches_kdtree():
    rng = np.random.default_rng(1)
    pts = rng.standard_normal((3000, 3))
    pts[10] = pts[11]                                  # a coincident pair
    for k in (1, 3, 5):
        got = oracle.knn_mean_dist(pts, k)
        d, _ = scipy.spatial.cKDTree(pts).query(pts, k=k + 1)
        # the tree returns the point itself first (distance 0); for the
        # coincident pair either copy may come first, the distances agree
        want = np.sort(d, 1)[:, 1:].mean(1)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_room_depth_unprojects_onto_the_surfaces():
    w = synth.trajectory_workload(n=1000, n_frames=20, width=96, height=72, focal=50.0)
    geo = w["geometry"]
    for f in (2, 11):
        view, pose = w["views"][f], w["poses"][f]
        depth = synth.room_depth(geo, view, pose)
        pts, _ = oracle.unproject(view, depth, None, 4)
        R = pose[:9].reshape(3, 3)
        pw = (pts - pose[9:]) @ R                      # R^T (p - t)
        on_wall = np.isclose(np.abs(pw), geo["half"], atol=1e-4).any(1)
        on_box = np.zeros(len(pw), bool)
        for lo, hi in geo["boxes"]:
            inside = np.all((pw >= lo - 1e-4) & (pw <= hi + 1e-4), 1)
            face = np.isclose(pw, lo, atol=1e-4).any(1) | np.isclose(pw, hi, atol=1e-4).any(1)
            on_box |= inside & face
        assert np.all(on_wall | on_box)
