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

    python -m paper_2404_12063_b300.train --claim --seeds 0 1 2 --lrs 1e-3 5e-3 --epochs 20000 --every 500

repeats that comparison over network initialisations (Glorot seeds) and
learning rates; a target counts as reached only from the first checkpoint
after which the error stays at or below it for two consecutive checkpoints.
It prints one JSON line; --markdown prints the summary tables instead.
"""
from __future__ import annotations

import argparse
import dataclasses
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
          train_eps: bool = False, mesh=None, max_seconds=None):
    """Returns a list of (epoch, train_seconds, loss, rel_l2[, eps]); stops
    after `epochs`, or at the first checkpoint past `max_seconds` of training."""
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
    while done < epochs and (max_seconds is None or t_train < max_seconds):
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


def sustained_time_to_target(hist, target, k=2):
    """(epoch, seconds) of the first checkpoint from which the error stays at
    or below target for k consecutive checkpoints; (None, None) if never."""
    for i in range(len(hist) - k + 1):
        if all(h[3] <= target for h in hist[i:i + k]):
            return hist[i][0], hist[i][1]
    return None, None


def error_at(hist, seconds):
    """Error at the last checkpoint within `seconds` of training."""
    best = hist[0]
    for h in hist:
        if h[1] <= seconds:
            best = h
    return best[3]


def claim(workload: str, epochs: int, every: int, lrs, seeds, variants=("fp32", "fp16", "bf16")):
    """The comparison of compare() for every (learning rate, Glorot seed), at
    equal wall-clock budgets: FP32 trains `epochs` epochs, the other forms
    train until they have used the same training time.  Per run the target
    is 1.05 x that run's FP32 final error (a run whose FP32 error ends above
    its initial error did not train and is reported, not counted); per
    (lr, form) the median and range over seeds of the sustained time to
    target and of the error at FP32's budget."""
    import fv_inputs as fi
    ctx = api.Context(0)
    make = {"annulus": fi.gear_annulus, "disc": fi.skewed_disc}[workload]
    runs = []
    for lr in lrs:
        for seed in seeds:
            prob = make()
            prob = dataclasses.replace(prob, params=fi.glorot_params(prob.widths, seed, 1))
            hs = {"fp32": train(ctx, prob, "fp32", epochs, lr, every, storage="fp32")}
            budget = hs["fp32"][-1][1]
            for v in variants:
                if v != "fp32":
                    hs[v] = train(ctx, prob, v, 50 * epochs, lr, every, storage="bf16", max_seconds=budget)
            target = 1.05 * final_error(hs["fp32"])
            trained = final_error(hs["fp32"]) < hs["fp32"][0][3]
            run = {"lr": lr, "seed": seed, "target_rel_l2": target, "fp32_trained": trained,
                   "budget_s": budget, "variants": {}}
            for v, h in hs.items():
                e, t = sustained_time_to_target(h, target) if trained else (None, None)
                run["variants"][v] = {"epochs_per_s": h[-1][0] / h[-1][1], "epochs": h[-1][0],
                                      "final_rel_l2": final_error(h), "rel_l2_at_budget": error_at(h, budget),
                                      "epochs_to_target": e, "seconds_to_target": t,
                                      "history": [(a, round(b, 3), round(d, 4)) for a, b, c, d, _ in h]}
            runs.append(run)
    summary = []
    for lr in lrs:
        for v in variants:
            rs = [r for r in runs if r["lr"] == lr and r["fp32_trained"]]
            ts = [r["variants"][v]["seconds_to_target"] for r in rs]
            reached = [t for t in ts if t is not None]
            errs = [r["variants"][v]["rel_l2_at_budget"] for r in rs]
            summary.append({"lr": lr, "form": v, "runs": len(rs), "reached": "%d/%d" % (len(reached), len(ts)),
                            "median_s": float(np.median(reached)) if reached else None,
                            "min_s": min(reached) if reached else None, "max_s": max(reached) if reached else None,
                            "median_rel_l2_at_budget": float(np.median(errs)) if errs else None,
                            "min_rel_l2_at_budget": min(errs) if errs else None,
                            "max_rel_l2_at_budget": max(errs) if errs else None,
                            "epochs_per_s": float(np.median([r["variants"][v]["epochs_per_s"] for r in runs
                                                             if r["lr"] == lr]))})
    return {"workload": workload, "epochs": epochs, "every": every, "seeds": list(seeds), "lrs": list(lrs),
            "rule": "target = 1.05 x the run's FP32 final error; reached when two consecutive checkpoints are below it",
            "summary": summary, "runs": runs}


def claim_markdown(res) -> str:
    lines = ["| lr | form | epochs/s | rel. L2 at FP32's budget: median (range) | reached target | "
             "median s to target | range (s) |", "|---|---|---|---|---|---|---|"]
    for r in res["summary"]:
        rng = "-" if r["min_s"] is None else "%.1f - %.1f" % (r["min_s"], r["max_s"])
        med = "-" if r["median_s"] is None else "%.1f" % r["median_s"]
        err = "-" if r["median_rel_l2_at_budget"] is None else "%.4f (%.4f - %.4f)" % (
            r["median_rel_l2_at_budget"], r["min_rel_l2_at_budget"], r["max_rel_l2_at_budget"])
        lines.append("| %g | %s | %.0f | %s | %s | %s | %s |" % (r["lr"], r["form"], r["epochs_per_s"], err,
                                                                r["reached"], med, rng))
    lines.append("")
    vs = list(res["runs"][0]["variants"])
    lines.append("| lr | seed | FP32 budget (s) | target | " +
                 " | ".join("%s epochs / error at budget / s to target" % v for v in vs) + " |")
    lines.append("|---|---|---|---|" + "---|" * len(vs))
    for run in res["runs"]:
        cells = []
        for v in vs:
            d = run["variants"][v]
            t = "-" if d["seconds_to_target"] is None else "%.1f (%d ep)" % (d["seconds_to_target"], d["epochs_to_target"])
            cells.append("%d / %.4f / %s" % (d["epochs"], d["rel_l2_at_budget"], t))
        tgt = "%.4f" % run["target_rel_l2"] if run["fp32_trained"] else "FP32 did not train"
        lines.append("| %g | %d | %.1f | %s | %s |" % (run["lr"], run["seed"], run["budget_s"], tgt, " | ".join(cells)))
    return "\n".join(lines)


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
    ap.add_argument("--claim", action="store_true")
    ap.add_argument("--seeds", type=int, nargs="+", default=[0, 1, 2])
    ap.add_argument("--lrs", type=float, nargs="+", default=[1e-3, 5e-3])
    ap.add_argument("--markdown", default=None, help="with --claim: a JSON file of an earlier run to summarise")
    args = ap.parse_args(argv)
    if args.markdown:
        with open(args.markdown) as fh:
            print(claim_markdown(json.loads(fh.read())))
    elif args.claim:
        print(json.dumps(claim(args.workload, args.epochs, args.every, args.lrs, args.seeds)))
    elif args.compare:
        print(json.dumps(compare(args.workload, args.epochs, args.every, args.lr)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
