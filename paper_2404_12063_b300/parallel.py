"""Element-sharded loss + gradient across ranks (one GPU per rank).

The variational loss is a sum over elements (Algorithm 3: mean over test
functions, then a sum over elements), so contiguous blocks of elements are
independent: each rank evaluates its block with the parameters replicated,
and one sum all-reduce of (L, Lv, Lb, Ls, dL/deps, dL/dtheta) gives the
unsharded result.  The boundary and sensor terms (means over their points)
are evaluated whole on rank 0, so their normalisation stays global.  This
holds for the default normalisation (FV_NORM_TEST); the per-element
normalisation of Eq. (loss) divides by the global element count and is not
sharded.

The per-shard evaluator is supplied by the caller: ``cuda_evaluator`` runs the
CUDA library on this rank's GPU.
"""
from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np


def shard_ranges(n_elements: int, world: int) -> List[Tuple[int, int]]:
    """Balanced contiguous element blocks [lo, hi) for world ranks."""
    base, extra = divmod(n_elements, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def shard_problem(prob, rank: int, world: int):
    """This rank's sub-problem: its element block; boundary / sensor data on rank 0 only."""
    import dataclasses
    lo, hi = shard_ranges(prob.mesh.n_elements, world)[rank]
    mesh = prob.mesh.subset(lo, hi)
    kw = {"mesh": mesh}
    if rank != 0:
        kw.update(bd_xy=np.zeros((0, 2)), bd_g=np.zeros(0), sensor_xy=np.zeros((0, 2)), sensor_u=np.zeros(0))
    return dataclasses.replace(prob, **kw)


def cuda_evaluator(precision: str = "fp32", device: int = 0):
    """Evaluator factory using the CUDA library: returns f(sub_problem) ->
    g(params ndarray) -> (out[5], grad) as float64 numpy arrays."""
    def make(sub):
        import torch
        from . import api
        ctx = api.Context(device)
        pb = api.problem_from_inputs(ctx, sub, precision)

        def ev(params):
            p = torch.tensor(np.asarray(params), dtype=pb.dtype, device="cuda:%d" % device)
            out, grad = pb.loss_grad(p)
            return out.cpu().numpy().copy(), grad.cpu().double().numpy()
        ev._keep = (ctx, pb)
        return ev
    return make


class ShardedLoss:
    """loss_grad(params) on this rank's shard, summed over the process group."""

    def __init__(self, prob, rank: int, world: int, make_evaluator: Callable, group=None):
        if getattr(prob, "norm", "test") not in ("test", 0):
            raise ValueError("only the Algorithm 3 normalisation shards exactly")
        self.rank, self.world, self.group = rank, world, group
        self.sub = shard_problem(prob, rank, world)
        self.ev = make_evaluator(self.sub)

    def loss_grad(self, params) -> Tuple[np.ndarray, np.ndarray]:
        out, grad = self.ev(params)
        if self.world == 1:
            return out, grad
        import torch
        import torch.distributed as dist
        buf = torch.from_numpy(np.concatenate([out[:5], grad]).astype(np.float64))
        if dist.get_backend(self.group) == "nccl":
            buf = buf.cuda()
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
        buf = buf.cpu().numpy()
        return buf[:5], buf[5:]
