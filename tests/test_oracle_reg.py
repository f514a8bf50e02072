"""Pins of the oracle's joint-refinement regularisers and pruning rule
(Sec. 3.3, Eq. 17).

* Isotropic Gaussians have axis ratio 1: no anisotropy loss for r >= 1.
* A hand-checkable case: scales (1, 2, 4) with r = 3 give (4/1 - 3)/n.
* The gradient of the hinge matches central finite differences of the
  oracle's own value wherever the hinge and the axis order do not change.
* The opacity L1 is the mean opacity (closed form, numpy sum).
* The pruning threshold equals a numpy sort of the opacities (brute force):
  at most n_target opacities exceed it, and lowering it to the next smaller
  distinct opacity would keep more than n_target."""
import numpy as np

import oracle


def test_isotropic_and_closed_form():
    sc = np.full((5, 3), 0.3, np.float32)
    op = np.linspace(0.1, 0.9, 5).astype(np.float32)
    v, gs_, go = oracle.regularize(sc, op, 1.5, 1.0, 0.0)
    assert v == 0.0 and not gs_.any() and not go.any()
    sc = np.array([[1, 2, 4], [1, 1, 1]], np.float32)
    v, gs_, _ = oracle.regularize(sc, np.ones(2, np.float32), 3.0, 1.0, 0.0)
    assert v == (4.0 / 1.0 - 3.0) / 2
    # d/ds_max (s_max/s_min) = 1/s_min, d/ds_min = -s_max/s_min^2, times 1/n
    assert np.array_equal(gs_[0], np.array([-4.0, 0.0, 1.0]) / 2)
    assert not gs_[1].any()


def test_opacity_l1_is_the_mean():
    rng = np.random.default_rng(1)
    op = rng.uniform(0.01, 1, 1000).astype(np.float32)
    v, _, go = oracle.regularize(np.ones((1000, 3), np.float32), op, 10.0, 0.0, 0.7)
    assert abs(v - 0.7 * op.astype(np.float64).sum() / 1000) < 1e-12
    assert np.allclose(go, 0.7 / 1000)


def test_hinge_gradient_finite_differences():
    rng = np.random.default_rng(2)
    n = 300
    sc = np.exp(rng.normal(-3, 0.8, (n, 3))).astype(np.float32)
    op = rng.uniform(0.05, 0.95, n).astype(np.float32)
    r = 2.0
    _, g, _ = oracle.regularize(sc, op, r, 1.0, 0.0)
    checked = 0
    for _ in range(60):
        i, k = int(rng.integers(n)), int(rng.integers(3))
        h = 1e-3 * float(sc[i, k])
        sp, sm = sc.copy(), sc.copy()
        sp[i, k] = np.float32(sc[i, k] + h); sm[i, k] = np.float32(sc[i, k] - h)
        ratio = lambda s: s[i].max() / s[i].min()
        order = lambda s: (int(np.argmax(s[i])), int(np.argmin(s[i])))
        if (ratio(sp) > r) != (ratio(sm) > r) or order(sp) != order(sm):
            continue
        fd = (oracle.regularize(sp, op, r, 1.0, 0.0)[0] - oracle.regularize(sm, op, r, 1.0, 0.0)[0]) / (
            float(sp[i, k]) - float(sm[i, k]))
        assert abs(fd - g[i, k]) <= 1e-4 * abs(g[i, k]) + 1e-9, (i, k, fd, g[i, k])
        checked += 1
    assert checked >= 30


def test_prune_threshold_brute_force():
    rng = np.random.default_rng(3)
    for n, target, mn in ((1000, 300, 0.005), (1000, 1200, 0.005), (500, 100, 0.9), (64, 10, 0.0)):
        op = rng.uniform(0, 1, n).astype(np.float32)
        op[:20] = op[20]                       # ties
        t, keep = oracle.prune_threshold(op, target, mn)
        srt = np.sort(op)
        want = mn if n <= target else max(mn, float(srt[n - target - 1]))
        assert t == np.float32(want)
        assert keep == int((op > t).sum()) <= target
        below = srt[srt < t]
        if len(below) and t > mn:
            assert (op > below[-1]).sum() > target
