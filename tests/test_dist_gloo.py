"""Multi-rank host logic on CPU ranks (gloo, world size 2, 127.0.0.1): view
sharding, the flat gradient buffer and its all-reduce, max-over-ranks timing,
and that a rank which dies before a collective makes its peer's collective
fail after the timeout instead of hanging."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2410_08743_gb300 import dist as D
from paper_2410_08743_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_views_disjoint_covering_balanced():
    w = synth.batched_workload(seed=3, n=10, n_views=64)
    px = [v["width"] * v["height"] for v in w["views"]]
    for world in (1, 2, 3, 4, 8):
        parts = [D.shard_views(px, world, r) for r in range(world)]
        flat = [k for p in parts for k in p]
        assert flat == list(range(64))
        loads = [sum(px[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= 2 * max(px), (world, loads)   # each cut is off by <= half a view
    assert D.shard_views([5], 2, 1) == [] or D.shard_views([5], 2, 0) == []
    with pytest.raises(ValueError):
        D.shard_views(px, 2, 2)


def test_flat_grads_layout():
    g = D.FlatGrads(7, "cpu")
    assert g.buf.numel() == 59 * 7
    shapes = {k: tuple(v.shape) for k, v in g.items()}
    assert shapes == {"means": (7, 3), "scales": (7, 3), "quats": (7, 4), "opac": (7,), "sh": (7, 16, 3)}
    ptrs = sorted((v.data_ptr(), v.numel()) for _, v in g.items())
    base = g.buf.data_ptr()
    off = 0
    for p, n in ptrs:
        assert p == base + 4 * off
        off += n
    assert off == g.buf.numel()
    g["sh"][2, 5, 1] = 3.0
    assert g.buf[(3 + 3 + 4 + 1) * 7 + 2 * 48 + 5 * 3 + 1] == 3.0


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    try:
        r, w = D.init_from_env("gloo", timeout_s=5.0)
        if mode == "sum":
            g = D.FlatGrads(5, "cpu")
            rng = np.random.default_rng(100 + r)
            for _, v in g.items():
                v.copy_(torch.from_numpy(rng.standard_normal(tuple(v.shape)).astype(np.float32)))
            mine = g.buf.clone()
            D.allreduce_grads(g)
            m = D.max_over_ranks(1.5 + r)
            q.put((r, mine.numpy(), g.buf.numpy(), m))
        elif mode == "dies":
            if r == 1:
                raise SystemExit(3)      # leaves before the collective
            g = D.FlatGrads(3, "cpu")
            try:
                D.allreduce_grads(g)
                q.put((r, "returned"))
            except Exception as e:      # noqa: BLE001 - any error is the detection
                q.put((r, "raised " + type(e).__name__))
    finally:
        import torch.distributed as td
        if td.is_initialized():
            try:
                td.destroy_process_group()
            except Exception:
                pass


def _run(mode, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = []
    for p in ps:
        p.join(60)
        if p.is_alive():
            p.kill()
            pytest.fail("rank did not finish")
    while not q.empty():
        out.append(q.get())
    return out


def test_allreduce_sums_flat_gradients_and_max_over_ranks():
    out = sorted(_run("sum"), key=lambda t: t[0])
    assert [t[0] for t in out] == [0, 1]
    total = out[0][1].astype(np.float64) + out[1][1].astype(np.float64)
    for r, mine, red, m in out:
        np.testing.assert_allclose(red, total, rtol=1e-6, atol=1e-6)
        assert m == 2.5
    assert np.array_equal(out[0][2], out[1][2])    # identical replicas after the exchange


def test_dead_peer_makes_collective_fail_not_hang():
    out = _run("dies")
    assert len(out) == 1 and out[0][0] == 0
    assert out[0][1].startswith("raised"), out
