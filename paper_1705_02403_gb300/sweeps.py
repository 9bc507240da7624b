"""Synthetic sweeps in the manner of Table 1 (cost error of GMT* against FMT*
over lambda and dimension) and Table 3 (time and cost against sample count
and obstacle resolution, double integrator and Dubins airplane), run on the
GPU planner.

FMT* is GMT* at lambda = 0 (the limit of Sec. III: every group is the set of
open nodes of minimum cost; the oracle tests pin this against a heap FMT*), so
both arms run through the same library on the same graph.  The environments
are synthetic analogues (envgen.rectangles, envgen.maze, envgen.forest_boxes,
envgen.di6_scaled, envgen.dubins_forest); the paper gives their figures, not
their geometry.

    python -m paper_1705_02403_gb300.sweeps --out sweeps.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import _native as N
from . import envgen
from .planner import Planner

LAMBDAS = (0.2, 0.5, 1.0)


def table1(runs: int = 50, n: int = 5000, lambdas=LAMBDAS, log=print):
    """Mean cost error c_GMT* / c_FMT* - 1 per environment, dimension and
    lambda, over the runs that both arms solve (Table 1: 50 runs, n = 5000)."""
    cases = [("rectangles", d) for d in (2, 3, 6, 10)] + [("maze", d) for d in (3, 5)]
    rows = []
    for env, d in cases:
        errs = {lam: [] for lam in lambdas}
        solved = 0
        t0 = time.time()
        for seed in range(runs):
            pb = envgen.rectangles(seed, d, n) if env == "rectangles" else envgen.maze(seed, d, n)
            pl = Planner(pb).build()
            base = pl.plan(allow_errors=True, lambda_=0.0)
            if base["status"] != N.GMT_OK:
                continue
            solved += 1
            for lam in lambdas:
                info = pl.plan(allow_errors=True, lambda_=lam)
                if info["status"] == N.GMT_OK:
                    errs[lam].append(info["path_cost"] / base["path_cost"] - 1.0)
        row = {"env": env, "d": d, "n": n, "runs": runs, "fmt_solved": solved,
               "radius": float(np.float32(N.gmt_connection_radius(n, d, 0.0, 1.0))),
               "cost_error": {str(lam): (float(np.mean(e)) if e else None) for lam, e in errs.items()},
               "cost_error_max": {str(lam): (float(np.max(e)) if e else None) for lam, e in errs.items()},
               "gmt_solved": {str(lam): len(e) for lam, e in errs.items()}, "wall_s": time.time() - t0}
        rows.append(row)
        if log:
            log(f"  {env} {d}D: " + ", ".join(f"lambda {lam}: {100 * row['cost_error'][str(lam)]:.2f}%"
                                             if row["cost_error"][str(lam)] is not None else f"lambda {lam}: -"
                                             for lam in lambdas) + f" ({solved}/{runs} solved)")
    return rows


def _timed_runs(problems, lam, reps=3):
    """Plan time (kernel, CUDA events) and graph-build time per problem, median
    of `reps` builds + plans each; plus status and cost of the last plan."""
    plan_ms, build_ms, costs, ok = [], [], [], 0
    for pb in problems:
        pl = Planner(pb.with_(lam=lam)).build()
        N.gmt_graph_set_profiling(pl.graph, True)
        pt, bt = [], []
        info = None
        for _ in range(reps):
            pl.build()
            info = pl.plan(allow_errors=True)
            torch.cuda.synchronize()
            p = N.gmt_graph_get_profile(pl.graph)
            pt.append(p["plan_ms"])
            bt.append(p["sample_ms"] + p["pair_ms"] + p["transpose_ms"] + p["scan_ms"] + p["fill_ms"])
        plan_ms.append(float(np.median(pt)))
        build_ms.append(float(np.median(bt)))
        if info["status"] == N.GMT_OK:
            ok += 1
            costs.append(info["path_cost"])
    return {"plan_ms_p50": float(np.median(plan_ms)), "plan_ms_p99": float(np.percentile(plan_ms, 99)),
            "build_ms_p50": float(np.median(build_ms)), "success": ok / len(problems),
            "mean_cost": float(np.mean(costs)) if costs else None}


def table3(runs: int = 20, lam: float = 1.0, log=print):
    """Double integrator (lambda = 1 as in Sec. V): time and cost against the
    sample count with 300 boxes, and time against the number of boxes that
    represent the same ten trunks at n = 5000."""
    rows = []
    for n in (1000, 2000, 5000, 10000):
        res = _timed_runs([envgen.di6_scaled(seed, n, nbox=300) for seed in range(runs)], lam)
        res.update({"sweep": "samples", "n": n, "boxes": 300})
        rows.append(res)
        if log:
            log(f"  n={n}, 300 boxes: plan {res['plan_ms_p50']:.3f} ms, build {res['build_ms_p50']:.3f} ms, "
                f"success {res['success']:.2f}, mean cost {res['mean_cost']}")
    for strips in (15, 50, 150, 500):
        probs = [envgen.di6_scaled(seed, 5000, boxes=envgen.forest_boxes(seed, 10, strips)) for seed in range(runs)]
        res = _timed_runs(probs, lam)
        res.update({"sweep": "boxes", "n": 5000, "boxes": 10 * strips})
        rows.append(res)
        if log:
            log(f"  n=5000, {10 * strips} boxes: plan {res['plan_ms_p50']:.3f} ms, build {res['build_ms_p50']:.3f} ms, "
                f"success {res['success']:.2f}")
    return rows


def table3_dubins(runs: int = 20, lam: float = 1.0, sampler: int = 1, log=print):
    """Dubins airplane in the forest analogue (lambda = 1, Halton samples as in
    Sec. V): time against the number of boxes at n = 5000 (150, 500, 1500,
    5000: the same ten trunks cut into 15, 50, 150, 500 strips, Table 3's box
    counts), then n = 10000 with 150 boxes (radius scaled for about the same
    mean out-degree)."""
    rows = []
    for n, strips in ((5000, 15), (5000, 50), (5000, 150), (5000, 500), (10000, 15)):
        r = float(np.float32(0.2 * (5000.0 / n) ** 0.2))
        probs = [envgen.dubins_forest(seed, n=n, r=r, strips=strips, sampler=sampler) for seed in range(runs)]
        res = _timed_runs(probs, lam)
        res.update({"sweep": "boxes" if n == 5000 else "samples", "n": n, "boxes": 10 * strips, "r": r})
        rows.append(res)
        if log:
            log(f"  n={n}, {10 * strips} boxes: plan {res['plan_ms_p50']:.3f} ms (p99 {res['plan_ms_p99']:.3f}), "
                f"build {res['build_ms_p50']:.3f} ms, success {res['success']:.2f}, mean cost {res['mean_cost']}")
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs1", type=int, default=50, help="runs per Table 1 cell")
    ap.add_argument("--runs3", type=int, default=20, help="problems per Table 3 row")
    ap.add_argument("--out", default="sweeps.json")
    ap.add_argument("--only", choices=["table1", "table3", "dubins"], default=None)
    a = ap.parse_args()
    t0 = time.time()
    out = {}
    if a.only in (None, "table1"):
        print("Table 1 analogue (cost error of GMT* against FMT* = GMT* at lambda 0, n = 5000):")
        out["table1"] = table1(a.runs1)
    if a.only in (None, "table3"):
        print("Table 3 analogue (double integrator, lambda = 1):")
        out["table3"] = table3(a.runs3)
    if a.only in (None, "dubins"):
        print("Table 3 analogue (Dubins airplane in the forest, lambda = 1, Halton samples):")
        out["table3_dubins"] = table3_dubins(a.runs3)
    out.update({"wall_s": time.time() - t0,
           "device": torch.cuda.get_device_name(0) if torch.cuda.is_available() else None})
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
