"""GPU tests of the optimisation kernels (Gaussian Adam, pose Adam), the
continuous-batching pose-solve server and CUDA-graph capture, through the C ABI.

The server's results are checked against the same solve done step by step
through gs_render_forward / gs_render_backward / gs_pose_step, against the
same request solved alone, and for convergence."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2410_08743_gb300 import _lib as L
from paper_2410_08743_gb300 import synth
from paper_2410_08743_gb300.render import Renderer

from .gpu_util import DEV, poses_dev, to_dev, zero_grads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2410_08743_gb300 import build
    build.build()
    r = Renderer(0)
    yield r
    r.close()


def test_gaussian_adam_matches_oracle(R):
    rng = np.random.default_rng(40)
    n, deg = 1500, 2
    raw = {"means": rng.standard_normal((n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
           "quats": rng.standard_normal((n, 4)), "logit_opac": rng.standard_normal((n, 1)),
           "sh": rng.standard_normal((n, 48))}
    raw = {k: a.astype(np.float32).astype(np.float64) for k, a in raw.items()}
    m = {k: np.zeros_like(a) for k, a in raw.items()}
    v = {k: np.zeros_like(a) for k, a in raw.items()}
    lrs = dict(means=1.6e-4, scales=5e-3, quats=1e-3, opac=5e-2, sh_dc=2.5e-3, sh_rest=1.25e-4)
    d = {k: torch.from_numpy(a.astype(np.float32)).to(DEV).contiguous() for k, a in raw.items()}
    dm = torch.zeros(59 * n, device=DEV)
    dv = torch.zeros(59 * n, device=DEV)
    act_s = torch.zeros(n, 3, device=DEV)
    act_o = torch.zeros(n, device=DEV)
    for step in range(1, 4):
        g = {"means": rng.standard_normal((n, 3)), "scales": rng.standard_normal((n, 3)),
             "quats": rng.standard_normal((n, 4)), "opac": rng.standard_normal((n, 1)),
             "sh": rng.standard_normal((n, 48))}
        g = {k: a.astype(np.float32) for k, a in g.items()}
        sc, op = oracle.gaussian_adam(raw, g, m, v, lrs, step, deg)
        gd = {k: torch.from_numpy(a).to(DEV).contiguous() for k, a in g.items()}
        gd["opac"] = gd["opac"].reshape(-1).contiguous()
        dr = dict(d)
        dr["logit_opac"] = d["logit_opac"].reshape(-1)
        L.gs_gaussian_adam(R.ctx, dr, act_s, act_o, gd, dm, dv, lrs, step, deg)
    torch.cuda.synchronize()
    for k in raw:
        np.testing.assert_allclose(d[k].cpu().numpy().astype(np.float64), raw[k], rtol=2e-5, atol=2e-6, err_msg=k)
    np.testing.assert_allclose(act_s.cpu().numpy(), sc, rtol=2e-5)
    np.testing.assert_allclose(act_o.cpu().numpy(), op, rtol=2e-5, atol=1e-7)


def _scene_and_targets(R, n_req, seed=50):
    """A 20k-Gaussian scene and n_req query images of mixed sizes rendered at
    ground-truth poses; initial poses off by a few degrees."""
    sc = synth.make_scene_box(seed, 20000, sh_degree=1, lo=(-1.5, -1.2, 3.0), hi=(1.5, 1.2, 6.0))
    p = to_dev(sc)
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        W = int(rng.integers(64, 160)); H = int(rng.integers(48, 120))
        view = synth.intrinsics(W, H)
        gt = synth.pose_from_center(synth.yaw_pitch(rng.uniform(-4, 4), rng.uniform(-4, 4)),
                                    np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.0]))
        img = R.forward(p, [view], poses_dev(gt[None])).cpu().numpy().copy()
        init = synth.perturb_normal(rng, gt, 3.0, 0.03)
        reqs.append(dict(view=view, image=img, gt=gt, init=init))
    return sc, p, reqs


def _rot_err_deg(a, b):
    Ra = np.asarray(a)[:9].reshape(3, 3); Rb = np.asarray(b)[:9].reshape(3, 3)
    c = (np.trace(Ra @ Rb.T) - 1) / 2
    return math.degrees(math.acos(min(1.0, max(-1.0, c))))


def _server(p, sc, slots, maxw=256, maxh=192, budget=0, qcap=1024, mask_alpha=0.0, pose_param=0):
    sh = L.gs_scene_borrow(p["means"], p["scales"], p["quats"], p["opac"], p["sh"], p["sh_degree"])
    srv = L.gs_server_create(0, sh, L.gs_default_opts(), slots, maxw, maxh, budget, qcap, mask_alpha, pose_param)
    return sh, srv


@pytest.mark.parametrize("mask_alpha,param", [(0.0, 0), (0.99, 0), (0.0, 1)], ids=["l1", "masked_l1", "txso3"])
def test_server_matches_step_by_step_solve(R, mask_alpha, param):
    sc, p, reqs = _scene_and_targets(R, 1, seed=51)
    rq = reqs[0]
    steps, lr0, lr1 = 12, 1e-2, 1e-3
    sh, srv = _server(p, sc, 4, mask_alpha=mask_alpha, pose_param=param)
    try:
        t = L.gs_solve_submit(srv, rq["view"], rq["image"], rq["init"], steps, lr0, lr1)
        res = L.gs_solve_wait(srv, t, 60000)
    finally:
        L.gs_server_destroy(srv)
        L.gs_scene_free(sh)
    assert res["status"] == 0 and res["steps_done"] == steps
    # the same solve through the public render / pose-step entry points
    P = poses_dev(rq["init"][None])
    m = torch.zeros(1, 6, dtype=torch.float64, device=DEV); v = torch.zeros_like(m)
    tgt = torch.from_numpy(rq["image"]).to(DEV)
    for k in range(steps):
        img = R.forward(p, [rq["view"]], P)
        pg = torch.zeros(1, 6, dtype=torch.float64, device=DEV)
        kind = L.GS_LOSS_L1_MASKED if mask_alpha > 0 else L.GS_LOSS_L1
        R.backward(p, [rq["view"]], P, img, L.make_loss(kind, target=tgt, w_l1=1.0, mask_alpha=mask_alpha), None, pg)
        lr = lr1 + 0.5 * (lr0 - lr1) * (1 + math.cos(math.pi * k / steps))
        R.pose_step(P, m, v, pg, lr, k + 1, param=param)
    torch.cuda.synchronize()
    np.testing.assert_allclose(np.array(res["pose"]), P.cpu().numpy()[0], atol=1e-6)


def test_server_result_same_alone_and_in_the_mix(R):
    sc, p, reqs = _scene_and_targets(R, 6, seed=52)
    steps = 30
    sh, srv = _server(p, sc, 8)
    try:
        t0 = L.gs_solve_submit(srv, reqs[0]["view"], reqs[0]["image"], reqs[0]["init"], steps, 1e-2, 1e-3)
        alone = L.gs_solve_wait(srv, t0, 60000)
        ts = [L.gs_solve_submit(srv, r["view"], r["image"], r["init"], steps, 1e-2, 1e-3) for r in reqs]
        mixed = [L.gs_solve_wait(srv, t, 60000) for t in ts]
        stats = L.gs_server_stats_get(srv)
    finally:
        L.gs_server_destroy(srv)
        L.gs_scene_free(sh)
    assert alone["status"] == 0 and all(r["status"] == 0 for r in mixed)
    assert stats["views_per_iteration"] > 1.5          # solves really shared iterations
    np.testing.assert_allclose(np.array(mixed[0]["pose"]), np.array(alone["pose"]), atol=1e-5)
    assert abs(mixed[0]["loss"] - alone["loss"]) <= 1e-5 * max(1.0, alone["loss"])
    # every solve lowered its photometric loss (rotation and translation are
    # coupled in SE(3), so a pose-error component alone may rise)
    for r, q in zip(mixed, reqs):
        tg = torch.from_numpy(q["image"]).to(DEV)
        l0 = torch.zeros(1, dtype=torch.float64, device=DEV)
        R.forward(p, [q["view"]], poses_dev(q["init"][None]), target=tg, loss_out=l0)
        assert r["loss"] < l0.item()


def test_server_admission_by_memory_budget(R):
    sc, p, reqs = _scene_and_targets(R, 4, seed=53)
    # a budget below two solves' modelled working set admits one at a time
    sh, srv = _server(p, sc, 8, budget=1)
    try:
        ts = [L.gs_solve_submit(srv, r["view"], r["image"], r["init"], 5, 1e-3, 1e-4) for r in reqs]
        out = [L.gs_solve_wait(srv, t, 60000) for t in ts]
        st = L.gs_server_stats_get(srv)
    finally:
        L.gs_server_destroy(srv)
        L.gs_scene_free(sh)
    assert all(o["status"] == 0 for o in out)
    assert st["views_per_iteration"] == pytest.approx(1.0)
    assert st["completed"] == 4


def test_server_admission_by_free_device_memory(R):
    """With the default budget the server admits solves while the modelled
    working set of the batch fits the device memory that is free (less a
    reserve): with most of the device taken by another allocation, a burst of
    requests is served a few at a time, none fails, and each result equals the
    same solve run alone."""
    sc = synth.make_scene_box(55, 1_000_000, sh_degree=1, lo=(-1.5, -1.2, 3.0), hi=(1.5, 1.2, 6.0))
    p = to_dev(sc)
    rng = np.random.default_rng(55)
    reqs = []
    for k in range(12):
        view = synth.intrinsics(504, 378)
        gt = synth.pose_from_center(synth.yaw_pitch(rng.uniform(-3, 3), rng.uniform(-3, 3)),
                                    np.array([rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), 0.0]))
        img = R.forward(p, [view], poses_dev(gt[None])).cpu().numpy().copy()
        reqs.append(dict(view=view, image=img, init=synth.perturb_normal(rng, gt, 2.0, 0.02)))
    steps = 4
    sh, srv = _server(p, sc, 1, maxw=504, maxh=378)
    try:                                    # reference: the first solve alone
        alone = L.gs_solve_wait(srv, L.gs_solve_submit(srv, reqs[0]["view"], reqs[0]["image"], reqs[0]["init"],
                                                       steps, 1e-2, 1e-3), 120000)
    finally:
        L.gs_server_destroy(srv)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info()
    reserve = max(256 << 20, int(0.02 * total))
    # leave the reserve plus about 1.5 GB: room for a handful of these views
    # (each about 0.25 GB modelled) but not for twelve
    take = free - reserve - (1536 << 20)
    filler = torch.empty(max(0, take), dtype=torch.uint8, device=DEV) if take > 0 else None
    srv = None
    try:
        free1, _ = torch.cuda.mem_get_info()
        srv = L.gs_server_create(0, sh, L.gs_default_opts(), 12, 504, 378, 0, 1024)
        ts = [L.gs_solve_submit(srv, r["view"], r["image"], r["init"], steps, 1e-2, 1e-3) for r in reqs]
        out = [L.gs_solve_wait(srv, t, 300000) for t in ts]
        st = L.gs_server_stats_get(srv)
    finally:
        if srv:
            L.gs_server_destroy(srv)
        L.gs_scene_free(sh)
        del filler
        torch.cuda.empty_cache()
    assert all(o["status"] == 0 for o in out), [o["status"] for o in out]
    assert 2 <= st["max_active"] < 12, st
    assert 0 < st["budget_bytes"] <= free1, (st["budget_bytes"], free1)
    np.testing.assert_allclose(np.array(out[0]["pose"]), np.array(alone["pose"]), atol=1e-5)


def test_server_requeues_solves_when_workspaces_cannot_grow(R):
    """A failed workspace growth (GS_ENOMEM, injected on the host) sends the
    iteration's new solves back to the queue; they finish later with the
    results of an undisturbed run.  A solve that fails alone three times in a
    row ends with GS_ENOMEM."""
    sc, p, reqs = _scene_and_targets(R, 3, seed=56)
    steps = 6
    sh, srv = _server(p, sc, 4)
    try:
        ref = [L.gs_solve_wait(srv, L.gs_solve_submit(srv, r["view"], r["image"], r["init"], steps, 1e-2, 1e-3),
                               60000) for r in reqs]
        L.gs_server_inject_enomem(srv, 2)
        ts = [L.gs_solve_submit(srv, r["view"], r["image"], r["init"], steps, 1e-2, 1e-3) for r in reqs]
        out = [L.gs_solve_wait(srv, t, 60000) for t in ts]
        st = L.gs_server_stats_get(srv)
        L.gs_server_inject_enomem(srv, 3)
        lone = L.gs_solve_wait(srv, L.gs_solve_submit(srv, reqs[0]["view"], reqs[0]["image"], reqs[0]["init"],
                                                      steps, 1e-2, 1e-3), 60000)
    finally:
        L.gs_server_destroy(srv)
        L.gs_scene_free(sh)
    assert all(o["status"] == 0 and o["steps_done"] == steps for o in out)
    assert st["requeued"] >= 1 and st["failed"] == 0
    for a, b in zip(out, ref):
        np.testing.assert_allclose(np.array(a["pose"]), np.array(b["pose"]), atol=1e-5)
    assert lone["status"] == L.GS_ENOMEM


def test_server_errors_cancel_and_timeout(R):
    sc, p, reqs = _scene_and_targets(R, 3, seed=54)
    sh, srv = _server(p, sc, 1, maxw=160, maxh=120, qcap=1)
    try:
        big = dict(reqs[0]["view"], width=300, height=200)
        with pytest.raises(L.GsError) as ei:
            L.gs_solve_submit(srv, big, np.zeros(3 * 300 * 200, np.float32), reqs[0]["init"], 5, 1e-3, 1e-4)
        assert ei.value.code == L.GS_EINVAL
        bad = reqs[0]["init"].copy(); bad[3] = np.nan
        with pytest.raises(L.GsError):
            L.gs_solve_submit(srv, reqs[0]["view"], reqs[0]["image"], bad, 5, 1e-3, 1e-4)
        long_t = L.gs_solve_submit(srv, reqs[0]["view"], reqs[0]["image"], reqs[0]["init"], 100000, 1e-3, 1e-4)
        with pytest.raises(L.GsError) as ei:
            L.gs_solve_wait(srv, long_t, 50)
        assert ei.value.code == L.GS_ETIMEOUT
        t2 = L.gs_solve_submit(srv, reqs[1]["view"], reqs[1]["image"], reqs[1]["init"], 5, 1e-3, 1e-4)
        with pytest.raises(L.GsError) as ei:      # queue capacity 1, slot busy
            L.gs_solve_submit(srv, reqs[2]["view"], reqs[2]["image"], reqs[2]["init"], 5, 1e-3, 1e-4)
        assert ei.value.code == L.GS_EBUSY
        L.gs_solve_cancel(srv, long_t)
        r = L.gs_solve_wait(srv, long_t, 60000)
        assert r["status"] == L.GS_EBUSY and r["steps_done"] < 100000
        r2 = L.gs_solve_wait(srv, t2, 60000)
        assert r2["status"] == 0
        with pytest.raises(L.GsError):
            L.gs_solve_poll(srv, 987654321)
    finally:
        L.gs_server_destroy(srv)
        L.gs_scene_free(sh)


def test_cuda_graph_capture_of_fwd_bwd_and_pose_step(R):
    """A captured forward + L1 backward + pose step replays like the eager
    sequence (poses updated on the device between replays)."""
    w = synth.tiny_workload(0)
    sc, views = w["scene"], w["views"]
    p = to_dev(sc)
    tgt = torch.from_numpy(oracle.render(sc, views, w["target_poses"])["image"].astype(np.float32)).to(DEV)
    r = Renderer(0)
    try:
        def run(P, m, v, img, pg, step):
            r.forward(p, views, P, image=img)
            r.backward(p, views, P, img, L.make_loss(L.GS_LOSS_L1, target=tgt, w_l1=1.0), None, pg)
            r.pose_step(P, m, v, pg, 1e-3, step)

        def fresh():
            return (poses_dev(w["poses"]), torch.zeros(1, 6, dtype=torch.float64, device=DEV),
                    torch.zeros(1, 6, dtype=torch.float64, device=DEV),
                    torch.empty(3 * 64 * 48, device=DEV), torch.zeros(1, 6, dtype=torch.float64, device=DEV))

        P, m, v, img, pg = fresh()
        eager = []
        for k in range(3):
            run(P, m, v, img, pg, 1)
            eager.append(P.cpu().numpy().copy())
        P, m, v, img, pg = fresh()
        run(P, m, v, img, pg, 1)            # grows the workspaces (step 1 of the sequence)
        torch.cuda.synchronize()
        r.set_flags(L.GS_F_NO_SYNC)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            pass
        torch.cuda.current_stream().wait_stream(s)
        Pc = P.clone()
        with torch.cuda.graph(g):
            run(P, m, v, img, pg, 1)
        # capture ran nothing; restore the state after step 1 and replay twice
        P.copy_(Pc)
        got = [Pc.cpu().numpy().copy()]
        for k in range(2):
            g.replay()
            torch.cuda.synchronize()
            got.append(P.cpu().numpy().copy())
        assert L.gs_status(r.ctx) == 0
        for a, b in zip(got, eager):
            np.testing.assert_allclose(a, b, atol=1e-9)
    finally:
        r.set_flags(0)
        r.close()


def test_tuning_is_result_neutral_and_autotune_caches(R, tmp_path):
    from paper_2410_08743_gb300 import tune
    sc = synth.make_scene_box(61, 40000, sh_degree=2, lo=(-1.2, -0.9, 3.0), hi=(1.2, 0.9, 6.0))
    views = [synth.intrinsics(96, 72), synth.intrinsics(40, 30), synth.intrinsics(160, 120)]
    rng = np.random.default_rng(61)
    poses = np.stack([synth.perturb_normal(rng, synth.pose_from_center(np.eye(3), np.zeros(3)), 2.0, 0.05)
                      for _ in views])
    p = to_dev(sc)
    P = poses_dev(poses)
    n_img = Renderer.image_numel(views)
    dldc = torch.from_numpy((rng.standard_normal(n_img) * 1e-3).astype(np.float32)).to(DEV)
    outs = []
    try:
        for t in ((4096, 2048, 256, 1), (1024, 1024, 128, 2), (8192, 1024, 256, 2), (2048, 2048, 128, 1)):
            L.gs_ctx_set_tuning(R.ctx, *t)
            img = R.forward(p, views, P).clone()
            g = zero_grads(p)
            pg = torch.zeros(len(views), 6, dtype=torch.float64, device=DEV)
            R.backward(p, views, P, img, L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc), g, pg)
            torch.cuda.synchronize()
            outs.append((img.cpu().numpy(), {k: v.cpu().numpy() for k, v in g.items()}, pg.cpu().numpy()))
        for img, g, pg in outs[1:]:
            assert np.array_equal(img, outs[0][0])
            for k in g:
                # equal up to the FP32 order of the gradient sums
                ref = outs[0][1][k]
                np.testing.assert_allclose(g[k], ref, rtol=1e-3, atol=1e-6 * np.abs(ref).max())
                assert np.linalg.norm(g[k] - ref) <= 1e-5 * np.linalg.norm(ref), k
            np.testing.assert_allclose(pg, outs[0][2], rtol=1e-5, atol=1e-12)
        with pytest.raises(L.GsError):
            L.gs_ctx_set_tuning(R.ctx, 3000, 2048, 256)
        img = torch.empty(n_img, device=DEV)
        loss = L.make_loss(L.GS_LOSS_DLDC, dl_dimage=dldc)
        cache = str(tmp_path / "tuning.json")
        r1 = tune.autotune(R, p, views, P, img, loss, repeats=1, cache_path=cache)
        assert not r1["cached"] and r1["tuning"]["sort_chunk"] in (1024, 2048)
        assert L.gs_ctx_get_tuning(R.ctx) == r1["tuning"]
        r2 = tune.autotune(R, p, views, P, img, loss, repeats=1, cache_path=cache)
        assert r2["cached"] and r2["tuning"] == r1["tuning"]
    finally:
        L.gs_ctx_set_tuning(R.ctx, 4096, 2048, 256)


def test_regularize_prune_compact_match_oracle(R):
    """Eq. 17 anisotropy hinge + opacity L1 (Sec. 3.3), the adaptive pruning
    threshold and the stable compaction, against the oracle / numpy."""
    rng = np.random.default_rng(60)
    n = 200_003
    sc = np.exp(rng.normal(-3, 0.8, (n, 3))).astype(np.float32)
    sc[:50] = 0.02                                     # isotropic rows
    op = rng.uniform(0.001, 0.999, n).astype(np.float32)
    op[100:400] = op[400]                              # ties
    r, la, lo = 2.5, 0.3, 0.05
    v_ref, gs_ref, go_ref = oracle.regularize(sc, op, r, la, lo)
    ds, do = torch.from_numpy(sc).to(DEV), torch.from_numpy(op).to(DEV)
    gs_ = torch.zeros(n, 3, device=DEV)
    go = torch.zeros(n, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    L.gs_regularize(R.ctx, ds, do, r, la, lo, gs_, go, loss)
    torch.cuda.synchronize()
    g1s, g1o = gs_.clone(), go.clone()
    L.gs_regularize(R.ctx, ds, do, r, la, lo, gs_, go, None)   # gradients are added
    torch.cuda.synchronize()
    assert torch.equal(gs_, 2 * g1s) and torch.equal(go, 2 * g1o)
    gs_, go = g1s, g1o
    ratio = sc.max(1).astype(np.float64) / sc.min(1)
    clear = np.abs(ratio - r) > 1e-5 * r               # FP32 and FP64 agree on the hinge there
    assert clear.mean() > 0.999
    assert abs(loss.item() - v_ref) <= 1e-5 * abs(v_ref) + 1e-3 * la / n * (~clear).sum()
    np.testing.assert_allclose(gs_.cpu().numpy()[clear], gs_ref[clear], rtol=2e-5, atol=1e-12)
    np.testing.assert_allclose(go.cpu().numpy(), go_ref, rtol=1e-5)
    for target, mn in ((60_000, 0.005), (300_000, 0.005), (150_000, 0.9)):
        t_ref, k_ref = oracle.prune_threshold(op, target, mn)
        t, k = L.gs_prune_threshold(R.ctx, do, target, mn)
        assert t == t_ref and k == k_ref
    t, k = L.gs_prune_threshold(R.ctx, do, 60_000, 0.005)
    keep = op > t
    means = rng.standard_normal((n, 3)).astype(np.float32)
    shv = rng.standard_normal((n, 48)).astype(np.float32)
    src = [torch.from_numpy(means).to(DEV), do, torch.from_numpy(shv).to(DEV)]
    dst = [torch.empty(k, 3, device=DEV), torch.empty(k, device=DEV), torch.empty(k, 48, device=DEV)]
    assert L.gs_compact(R.ctx, do, t, src, dst, [3, 1, 48]) == k
    assert np.array_equal(dst[0].cpu().numpy(), means[keep])
    assert np.array_equal(dst[1].cpu().numpy(), op[keep])
    assert np.array_equal(dst[2].cpu().numpy(), shv[keep])
