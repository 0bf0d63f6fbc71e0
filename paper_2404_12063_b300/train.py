"""Training driver: Adam on the FastVPINNs loss (paper Sec. 4.5-4.7: Adam,
learning rate 1e-3, one loss + gradient evaluation per iteration).

Each iteration is one ``fv_inverse_step``: the fused loss + gradient pass and
the Adam update of the parameters (and of eps when it is trainable) on the
device.  The solution error is the relative L2 error of u against the exact
solution at every quadrature point, evaluated with the same FP32 network
evaluation for every precision so that the precision forms are compared on
one yardstick.

    python -m paper_2404_12063_b300.train --compare --workload annulus --epochs 20000 --every 1000 --lr 5e-3

compares plain FP32 with the 16-bit tensor-core forms from one
initialisation (gear-like annulus, or the skewed disc with --workload disc)
and prints one JSON line: epochs/s, final error, and epochs and seconds to
reach 1.05 x the FP32 run's final error.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np
import torch

from . import api


def relative_l2(ctx, widths, params: torch.Tensor, xy_dev: torch.Tensor, u_exact: torch.Tensor) -> float:
    p32 = params.detach().to(torch.float32).contiguous()
    out = api.mlp_eval(ctx, widths, p32, xy_dev, "fp32")
    return float(torch.linalg.norm(out[0].double() - u_exact) / torch.linalg.norm(u_exact))


def train(ctx, prob, precision: str, epochs: int, lr: float = 1e-3, every: int = 250, storage=None,
          train_eps: bool = False, mesh=None):
    """Returns a list of (epoch, train_seconds, loss, rel_l2[, eps])."""
    pb = api.problem_from_inputs(ctx, prob, precision, storage=storage, mesh=mesh)
    dt = pb.dtype
    params = torch.tensor(prob.params, dtype=dt, device="cuda")
    eps = torch.tensor([prob.eps], dtype=torch.float64, device="cuda")
    adam = api.Adam(ctx, pb.net.n_params, precision, with_eps=train_eps)
    grad = torch.empty_like(params)
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    X = torch.tensor(pb.mesh.quad_points(), device="cuda")
    ue = torch.tensor(prob.u_exact(X[:, 0].cpu().numpy(), X[:, 1].cpu().numpy()), device="cuda")
    hist = [(0, 0.0, float("nan"), relative_l2(ctx, prob.widths, params, X, ue), float(eps.item()))]
    stream = ctx.stream
    t_train = 0.0
    done = 0
    while done < epochs:
        n = min(every, epochs - done)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            pb.inverse_step(params, eps, adam, lr, grad, out)
        e1.record(stream)
        torch.cuda.synchronize()
        t_train += e0.elapsed_time(e1) / 1e3
        done += n
        hist.append((done, t_train, float(out[0]), relative_l2(ctx, prob.widths, params, X, ue), float(eps.item())))
    return hist


def time_to_target(hist, target):
    for e, t, _, l2, _ in hist:
        if l2 <= target:
            return e, t
    return None, None


def final_error(hist, n=3):
    """Median relative L2 error over the last n checkpoints (damps Adam's fluctuation)."""
    return float(np.median([h[3] for h in hist[-n:]]))


def compare(workload: str, epochs: int, every: int, lr: float, variants=("fp32", "bf16", "fp16")):
    """Train each precision form from the same initialisation; the target error
    is 1.05 x the FP32 run's final error."""
    import fv_inputs as fi
    ctx = api.Context(0)
    prob = {"annulus": fi.gear_annulus, "disc": fi.skewed_disc}[workload]()
    res = {}
    for v in variants:
        res[v] = train(ctx, prob, v, epochs, lr, every, storage="bf16" if v in ("bf16", "fp16") else "fp32")
    target = 1.05 * final_error(res["fp32"])
    out = {"workload": prob.name, "epochs": epochs, "lr": lr, "target_rel_l2": target, "variants": {}}
    for v, h in res.items():
        e, t = time_to_target(h, target)
        out["variants"][v] = {"epochs_per_s": h[-1][0] / h[-1][1], "final_rel_l2": final_error(h),
                              "final_loss": h[-1][2], "epochs_to_target": e, "seconds_to_target": t,
                              "history": [(a, round(b, 4), c, d) for a, b, c, d, _ in h]}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--compare", action="store_true")
    ap.add_argument("--workload", default="annulus", choices=["annulus", "disc"])
    ap.add_argument("--epochs", type=int, default=4000)
    ap.add_argument("--every", type=int, default=250)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args(argv)
    if args.compare:
        print(json.dumps(compare(args.workload, args.epochs, args.every, args.lr)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
