"""Multi-GPU plumbing for the renderer: one process per GPU, the scene
replicated on every rank, the views sharded.

What shards and what is exchanged:
* Views are independent in the forward, the loss and the backward: each rank
  renders its own views and computes their pose gradients (Sec. 3.2; a pose
  gradient depends on its own view only), so neither needs an exchange.
* The per-Gaussian gradient of a joint step (Sec. 3.3) is a sum over all views,
  so ranks that optimise one shared set of Gaussians sum their gradient buffers
  once per step (one all-reduce of 59 floats per Gaussian) and then take the
  same Adam step, which keeps the replicas identical.
* Independent pose solves (serving) exchange nothing: replicas only.

The collective is torch.distributed (NCCL between GPUs, gloo on CPU ranks).
Gradients live in one flat buffer so that the exchange is one call."""
from __future__ import annotations

import datetime
import os

import torch
import torch.distributed as dist

GRAD_WIDTHS = (("means", 3), ("scales", 3), ("quats", 4), ("opac", 1), ("sh", 48))
FLOATS_PER_GAUSSIAN = sum(w for _, w in GRAD_WIDTHS)


def shard_views(pixels, world: int, rank: int) -> list[int]:
    """Contiguous block of view indices for `rank`, cut so that every rank gets
    about the same number of pixels (pixels: per-view pixel counts).  The
    blocks are disjoint, ordered, and cover every view."""
    n = len(pixels)
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    total = float(sum(pixels))
    cuts = [0]
    acc = 0.0
    k = 0
    for r in range(1, world):
        goal = total * r / world
        while k < n and acc + pixels[k] / 2.0 < goal:
            acc += pixels[k]
            k += 1
        cuts.append(max(k, cuts[-1]))
    cuts.append(n)
    return list(range(cuts[rank], cuts[rank + 1]))


class FlatGrads:
    """The renderer's five per-Gaussian gradient arrays as views of one flat
    float32 buffer [59 N] (means [N,3], scales [N,3], quats [N,4], opac [N],
    sh [N,16,3], in that order)."""

    def __init__(self, n: int, device) -> None:
        self.n = int(n)
        self.buf = torch.zeros(FLOATS_PER_GAUSSIAN * self.n, dtype=torch.float32, device=device)
        self.views = {}
        off = 0
        for name, w in GRAD_WIDTHS:
            v = self.buf[off:off + w * self.n]
            if name == "sh":
                v = v.view(self.n, 16, 3)
            elif w > 1:
                v = v.view(self.n, w)
            self.views[name] = v
            off += w * self.n

    def __getitem__(self, k):
        return self.views[k]

    def items(self):
        return self.views.items()

    def as_dict(self) -> dict:
        return dict(self.views)

    def zero_(self) -> None:
        self.buf.zero_()


def init_from_env(backend: str | None = None, timeout_s: float = 60.0):
    """torch.distributed from RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT
    (torchrun's variables).  Returns (rank, world); (0, 1) without them.  A
    collective whose peer died or never joined raises after timeout_s instead
    of waiting forever."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
    return rank, world


def allreduce_grads(g: FlatGrads, group=None) -> None:
    """Sum the flat gradient buffer over the ranks of `group` (in place)."""
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(g.buf, op=dist.ReduceOp.SUM, group=group)


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Largest value of x over the ranks (the timing rule of a weak-scaling
    step: the job is as slow as its slowest rank)."""
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
