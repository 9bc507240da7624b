"""Freeze the connection radius of the 6D double-integrator workload.

The radius is an input of both the planner and the oracle.  It is chosen so
that the seed-0 instance (n = 4096, 30 boxes) has a mean out-degree of 40:
r is the (40 N)-th smallest directed connection cost over all ordered pairs,
evaluated by the oracle with a wide arrival-time bracket, rounded to four
significant digits.  Writes paper_1705_02403_gb300/configs/double_integrator_6d_n4096.json.

Run:  python oracle/calibrate_di_radius.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1705_02403_gb300 import envgen  # noqa: E402


def main():
    n, nbox, target_deg = 4096, 30, 40
    pb = envgen.di6(seed=0, n=n, nbox=nbox, r=4.0)
    X, goal = O.sample(pb)
    t = time.time()
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, 4.0)
    costs = np.sort(g.csr().out_cost.astype(np.float64))
    N = n + 1
    r = float(f"{costs[target_deg * N - 1]:.4g}")
    g2 = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r)
    E = g2.num_edges
    print(f"r={r} E={E} mean out-degree={E / N:.2f} ({time.time() - t:.1f}s)")
    out = {
        "name": "double_integrator_6d_n4096",
        "description": "6D double integrator GMT*: position [0,1]^3, velocity [-1,1]^3, n=4096 Philox samples, "
                       "30 random boxes, cost = arrival time + control effort, 20 trajectory points per edge, "
                       "lambda=0.5, r frozen so that the seed-0 instance has mean out-degree 40",
        "n": n, "boxes": nbox, "r": r, "lambda": 0.5, "traj_points": 20,
        "calibration": {"seed": 0, "edges": int(E), "mean_out_degree": round(E / N, 3)},
    }
    path = os.path.join(ROOT, "paper_1705_02403_gb300", "configs", "double_integrator_6d_n4096.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
