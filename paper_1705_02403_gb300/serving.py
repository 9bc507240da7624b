"""Replanning stream against gmt_server: sessions of 6D double-integrator
problems (n uniform in [2048, 8192]) whose 30 boxes translate every tick at
random speeds up to 0.02 per tick, one request per session per tick at a fixed
rate (100 Hz), latency percentiles over all requests.

    python -m paper_1705_02403_gb300.serving --sessions 100 --ticks 100
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import _native as N
from . import envgen
from .planner import goal_struct, params_struct, space_struct

R_4096 = 2.428  # frozen radius of the 4096-sample workload (mean out-degree 40)


def session_problem(seed: int, n: int) -> envgen.Problem:
    """DI problem whose radius keeps the mean out-degree near 40 at any n."""
    return envgen.di6(seed=seed, n=n, nbox=30, r=R_4096 * (4096.0 / n) ** (1.0 / 6.0))


class MovingBoxes:
    """Boxes translating at constant random velocities (|v| <= vmax per tick),
    reflected at the walls of [0,1]^3."""

    def __init__(self, pb: envgen.Problem, seed: int, vmax: float = 0.02):
        rng = np.random.default_rng([seed, 1705, 5])
        self.c = ((pb.box_lo + pb.box_hi) / 2).astype(np.float64)
        self.h = ((pb.box_hi - pb.box_lo) / 2).astype(np.float64)
        d = rng.normal(size=self.c.shape)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        self.v = d * rng.uniform(0, vmax, (len(self.c), 1))

    def step(self):
        self.c += self.v
        for a in range(3):
            lo = self.c[:, a] - self.h[:, a] < 0
            hi = self.c[:, a] + self.h[:, a] > 1
            self.v[lo | hi, a] *= -1
            self.c[:, a] = np.clip(self.c[:, a], self.h[:, a], 1 - self.h[:, a])
        return (self.c - self.h).astype(np.float32), (self.c + self.h).astype(np.float32)


def run_stream(sessions=100, ticks=100, hz=100.0, slots=32, cluster=4, threads=512, seed=0, n_range=(2048, 8192),
               log=print):
    rng = np.random.default_rng([seed, 1705, 6])
    server = N.Server(slots=slots, cluster=cluster, threads=threads, max_nodes=n_range[1] + 1, max_boxes=30)
    sids, movers = [], []
    t0 = time.time()
    for k in range(sessions):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        pb = session_problem(seed * 100000 + k, n)
        sid, _ = server.open_session(space_struct(pb), pb.x_init, goal_struct(pb), params_struct(pb), pb.box_lo,
                                     pb.box_hi)
        sids.append(sid)
        movers.append(MovingBoxes(pb, seed * 100000 + k))
    t_open = time.time() - t0
    results = []
    rid = 0
    start = time.perf_counter()
    for t in range(ticks):
        target = start + t / hz
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            results += server.poll(4096, 0)
            time.sleep(min(0.0005, target - now))
        for sid, mv in zip(sids, movers):
            lo, hi = mv.step()
            server.submit(sid, rid, lo, hi)
            rid += 1
    while len(results) < rid:
        results += server.poll(4096, 100)
    span = time.perf_counter() - start
    for sid in sids:
        server.close_session(sid)
    server.close()
    lat = np.array([r["latency_ms"] for r in results])
    out = {"sessions": sessions, "ticks": ticks, "rate_hz": hz, "requests": len(results), "slots": slots,
           "cluster": cluster, "threads": threads,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
           "queue_ms_p50": float(np.percentile([r["queue_ms"] for r in results], 50)),
           "requests_per_s": len(results) / span, "span_s": span, "session_setup_s": t_open,
           "edges_checked_per_s": float(sum(r["edges_checked"] for r in results) / span),
           "success_rate": float(np.mean([r["status"] == 0 for r in results])),
           "errors": int(sum(r["status"] < 0 for r in results)),
           "verdict_cache_hit_rate": float(1 - sum(r["checks_computed"] for r in results)
                                           / max(1, sum(r["checks"] for r in results)))}
    if log:
        log(json.dumps(out, indent=1))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sessions", type=int, default=100)
    ap.add_argument("--ticks", type=int, default=100)
    ap.add_argument("--hz", type=float, default=100.0)
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--cluster", type=int, default=4)
    ap.add_argument("--threads", type=int, default=512)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    out = run_stream(a.sessions, a.ticks, a.hz, a.slots, a.cluster, a.threads)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
