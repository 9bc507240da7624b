#!/usr/bin/env python
"""Benchmark of the GMT* hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmt|reference] [--workload di6|geo2d]

A step is one pass of the whole hot path over one synthetic problem: SampleFree
(Philox), the r-disk neighbour CSR (all-pairs cost filter) and the group
wavefront of Algorithm 1, through the C ABI.  Every step plans a different
seed.  The default workload is the 6D double integrator (n = 4096, 30 random
boxes, r frozen for mean out-degree 40, lambda = 0.5).

Metric: edges checked per second (CSR entries scanned by the frontier push and
the lazy parent selection), beside ms per plan p50/p99.  Inputs are resident in
HBM before the timed region; L2 is flushed (256 MiB write) between steps and
the flush is outside the per-step CUDA-event timings.

Under torchrun (N > 1) each rank plans its own seeds (replicas, no collective
on the data path); value = edges of all ranks / the slowest rank's time.

--impl reference times the CPU oracle (oracle/) as the reference arm: one full
oracle step (SampleFree, all-pairs CSR, wavefront) per step, on the GPU arm's
seeds, on one host core.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms/plan p50/p99 & edges checked/s; learned+batched vs plain at equal path cost"

# DRAM bytes (read + write) of one plan_kernel launch on this workload, from the
# ncu captures summarised in profiles/plan_kernel_double_integrator_6d_n4096.md
# and profiles/plan_kernel_geometric_2d_n1024.md.
# Set to None whenever plan_kernel changes until it is captured again.
PLAN_KERNEL_DRAM_BYTES = {"di6": 2225408, "geo2d": None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gmt", choices=["gmt", "reference"])
    ap.add_argument("--workload", default="di6", choices=["di6", "geo2d"])
    ap.add_argument("--seed-base", type=int, default=1000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    return ap.parse_args()


def make_problem(workload, seed):
    from paper_1705_02403_gb300 import envgen
    return envgen.cfg2_di6(seed) if workload == "di6" else envgen.cfg1_2d(seed)


def workload_config(workload):
    from paper_1705_02403_gb300 import envgen
    if workload == "di6":
        c = envgen.load_config("double_integrator_6d_n4096")
        return {"workload": "double_integrator_6d_n4096_30boxes", "kind": "double_integrator", "dim": 6,
                "n": c["n"], "boxes": c["boxes"], "r": c["r"], "lambda": c["lambda"],
                "traj_points": c["traj_points"]}
    c = envgen.load_config("geometric_2d_n1024")
    return {"workload": "geometric_2d_n1024_10boxes", "kind": "euclidean", "dim": 2, "n": c["n"],
            "boxes": c["boxes"], "r": c["r"], "lambda": c["lambda"], "seg_spacing": c["seg_spacing"]}


def pct(a, q):
    return float(np.percentile(np.asarray(a, dtype=np.float64), q)) if len(a) else None


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"gmt_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- oracle
def oracle_step(O, pb):
    """One full oracle step on one problem, timed: SampleFree, the all-pairs
    neighbour CSR and the wavefront.  Returns (seconds, edges checked)."""
    t0 = time.perf_counter()
    X, goal = O.sample(pb)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
    _, _, info = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing, pb.traj_points)
    sec = time.perf_counter() - t0
    return sec, info["push_edges"] + info["pull_edges"]


def cpu_baseline(workload, seeds):
    """The oracle, one full step per seed (single thread).  Returns
    (edges/s, seconds per step)."""
    from oracle import oracle as O
    O.build()
    tot_s, tot_e = 0.0, 0
    for s in seeds:
        sec, edges = oracle_step(O, make_problem(workload, s))
        tot_s += sec
        tot_e += edges
    return tot_e / tot_s, tot_s / len(seeds)


def plan_bytes(info, d, N):
    """Algorithmic bytes of one wavefront: 4 B per pushed out-edge (its column),
    12 B per scanned in-edge (column, cost, gathered snapshot cost), both end
    states of every collision check (2 d floats), the open/closed/unexplored and
    group masks touched once per iteration (5 N / 8 B) and the cost and parent
    writes (8 B per node)."""
    return (4 * info["push_edges"] + 12 * info["pull_edges"] + 8 * d * info["checks"] + info["iters"] * 5 * N / 8
            + 8 * N)


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = workload_config(args.workload)
    from oracle import oracle as O
    O.build()
    secs, edges = [], []
    # the GPU arm's seeds: warm-up steps first, then one seed per timed step
    seeds = [args.seed_base + k for k in range(args.warmup + args.steps)]
    for k, s in enumerate(seeds):
        sec, e = oracle_step(O, make_problem(args.workload, s))
        if k >= args.warmup:
            secs.append(sec); edges.append(e)
    value = float(np.sum(edges) / np.sum(secs))
    sample = (f"every step one full oracle step (SampleFree, all-pairs neighbour CSR, wavefront) on one problem; "
              f"seeds {seeds[args.warmup]}..{seeds[-1]} timed, as in the GPU arm; single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(cfg, seeds=f"{seeds[args.warmup]}..{seeds[-1]} (one seed per step)"),
            "ms_per_plan": {"p50": 1e3 * pct(secs, 50), "p99": 1e3 * pct(secs, 99)},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- ranks
def aggregate_ranks(time_ms, edges, world, device="cpu"):
    """Whole-job totals across replicas: the slowest rank's time (MAX) and the
    edges of all ranks (SUM); value = edges / time."""
    if world <= 1:
        return time_ms, edges
    import torch
    t = torch.tensor([time_ms, edges], dtype=torch.float64, device=device)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import boxes_on_device, goal_struct, params_struct, space_struct

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    cfg = workload_config(args.workload)
    total = args.warmup + args.steps
    seeds = [args.seed_base + 1_000_000 * rank + k for k in range(total)]
    probs = [make_problem(args.workload, s) for s in seeds]
    pb0 = probs[0]
    space, goal = space_struct(pb0), goal_struct(pb0)
    boxes = [boxes_on_device(pb, dev) for pb in probs]
    params = [params_struct(pb) for pb in probs]
    Nn = pb0.N
    parent = torch.empty(Nn, dtype=torch.int32, device=dev)
    cost = torch.empty(Nn, dtype=torch.float32, device=dev)
    path = torch.empty(Nn, dtype=torch.int32, device=dev)
    graph = N.Graph()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # sample, pair filter (the double integrator's also writes the transposed
    # matrix), row scans (both directions in one launch), fill, plan
    launches_per_step = 5

    def step(k, level):
        # the build is queued without a host wait (gmt_plan confirms it; the
        # first build of the handle sizes its edge arrays synchronously)
        N.gmt_build_graph_async(space, boxes[k][0], [float(v) for v in probs[k].x_init], goal, params[k], graph,
                                stream)
        N.gmt_graph_set_profiling(graph, level)
        # the plan's result is on the host when gmt_plan returns (its info
        # struct); turning it into a dict is left outside the timed region
        return N.gmt_plan(graph, boxes[k][0], params[k], parent.data_ptr(), cost.data_ptr(), path.data_ptr(),
                          stream)

    # ---- warm-up (untimed)
    for k in range(args.warmup):
        step(k, 0).as_dict()
    torch.cuda.synchronize()

    # ---- timed: inputs resident, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos, profs = [], []
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # no Python garbage collection inside the timed region (a collection is a
    # host pause of milliseconds during which the GPU would idle between steps)
    gc.collect()
    gc.disable()
    clocks.start()
    t_wall = time.perf_counter()
    for j in range(args.steps):
        k = args.warmup + j
        flush.zero_()
        ev[j][0].record(stream)
        info = step(k, 2)  # events around the plan kernel only (each event costs the device time)
        ev[j][1].record(stream)
        infos.append(info.as_dict())
        profs.append(N.gmt_graph_get_profile(graph))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    gc.enable()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    edges = [i["push_edges"] + i["pull_edges"] for i in infos]
    sum_ms = float(np.sum(step_ms))
    tot_edges = float(np.sum(edges))
    sum_ms_all, tot_edges_all = aggregate_ranks(sum_ms, tot_edges, world, dev)
    value = tot_edges_all / (sum_ms_all / 1e3)

    # ---- end to end: host inputs (pinned), H2D of the boxes and D2H of the tree each step
    h_lo = [torch.as_tensor(np.ascontiguousarray(pb.box_lo, np.float32)).pin_memory() for pb in probs]
    h_hi = [torch.as_tensor(np.ascontiguousarray(pb.box_hi, np.float32)).pin_memory() for pb in probs]
    d_lo = torch.empty_like(boxes[0][1][0]); d_hi = torch.empty_like(boxes[0][1][1])
    h_parent = torch.empty(Nn, dtype=torch.int32).pin_memory()
    h_cost = torch.empty(Nn, dtype=torch.float32).pin_memory()
    e2e_ms, e2e_edges = [], []
    bi = bo = 0
    N.gmt_graph_set_profiling(graph, 0)
    for j in range(args.steps):
        k = args.warmup + j
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        d_lo.copy_(h_lo[k], non_blocking=True); d_hi.copy_(h_hi[k], non_blocking=True)
        bx = N.gmt_boxes(); bx.count = d_lo.shape[0]; bx.lo = d_lo.data_ptr(); bx.hi = d_hi.data_ptr()
        N.gmt_build_graph_async(space, bx, [float(v) for v in probs[k].x_init], goal, params[k], graph, stream)
        info = N.gmt_plan(graph, bx, params[k], parent.data_ptr(), cost.data_ptr(), path.data_ptr(), stream)
        h_parent.copy_(parent, non_blocking=True); h_cost.copy_(cost, non_blocking=True)
        b.record(stream)
        b.synchronize()
        info = info.as_dict()
        e2e_ms.append(a.elapsed_time(b))
        e2e_edges.append(info["push_edges"] + info["pull_edges"])
        bi = h_lo[k].numel() * 4 + h_hi[k].numel() * 4
        bo = Nn * 8 + 64
    e2e_ms_all, e2e_edges_all = aggregate_ranks(float(np.sum(e2e_ms)), float(np.sum(e2e_edges)), world, dev)
    e2e_value = e2e_edges_all / (e2e_ms_all / 1e3)

    # ---- per-stage device times: an untimed pass over the first timed seeds
    # with events around every stage; the plan kernel's own time is the timed
    # region's
    stage_profs = []
    for j in range(min(args.steps, 20)):
        flush.zero_()
        step(args.warmup + j, 1)
        stage_profs.append(N.gmt_graph_get_profile(graph))
    torch.cuda.synchronize()

    # ---- roofline of the dominant kernel
    kern = {k: float(np.mean([p[k] for p in stage_profs])) for k in
            ("sample_ms", "pair_ms", "transpose_ms", "scan_ms", "fill_ms")}
    kern["plan_ms"] = float(np.mean([p["plan_ms"] for p in profs]))
    dominant = max(kern, key=kern.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    pbytes = [plan_bytes(i, pb0.d, Nn) for i in infos]
    roof = {"kernel": "plan_kernel (wavefront, Alg. 1)", "bound": "hbm",
            "achieved": float(np.mean(pbytes)) / (kern["plan_ms"] / 1e3) / 1e9,
            "peak": hbm, "unit": "GB/s", "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "traffic": PLAN_KERNEL_DRAM_BYTES.get(args.workload),
            "algorithmic_bytes_per_launch": float(np.mean(pbytes)),
            "launch_ms": kern["plan_ms"]}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if dominant != "plan_ms":
        roof["note"] = f"dominant stage is {dominant}; plan kernel reported"

    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(cfg, seeds=f"{seeds[args.warmup]}..{seeds[-1]} (one seed per step, per rank)",
                       parallelism=f"replicas x{world}", l2="flushed between steps (256 MiB write)"),
        "ms_per_plan": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99),
                        "plan_only_p50": pct([p["plan_ms"] for p in profs], 50),
                        "plan_only_p99": pct([p["plan_ms"] for p in profs], 99)},
        "plans_per_s": world * args.steps / (sum_ms_all / 1e3),
        "kernel_ms_mean": kern,
        "kernel_ms_note": "plan_ms: live in the timed steps; other stages: an untimed pass with every stage's events",
        "plan_launch": {"blocks": profs[-1]["plan_blocks"], "threads": profs[-1]["plan_threads"]},
        "success_rate": float(np.mean([i["status"] == 0 for i in infos])),
        "mean_edges_checked": float(np.mean(edges)),
        "wall_s": wall,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "edges/s", "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "ms_per_plan_p50": pct(e2e_ms, 50)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if not args.no_extras:
        line["batched"] = bench_batched(dev, flush)
        line["serving"] = bench_serving(local_rank)
        line["dubins"] = bench_dubins(dev, flush)
        line["learned"] = bench_learned()
        line["gpu_launches_extras"] = ("batched: 7 launches per group per batch (replayed CUDA graph); serving: 3 per "
                                       "request; dubins: 7-8 per build, 1 per plan")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nb = min(args.steps, 8 if args.workload == "di6" else 20)
        seeds_cpu = [seeds[args.warmup + j] for j in range(nb)]
        v, sec = cpu_baseline(args.workload, seeds_cpu)
        line["cpu_baseline"] = {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"the first {nb} timed seeds ({seeds_cpu[0]}..{seeds_cpu[-1]}), one full "
                                          f"oracle step each (SampleFree, all-pairs CSR, wavefront), measured, not "
                                          f"scaled; {1e3 * sec:.0f} ms per step"}
    if rank == 0:
        print(json.dumps(line), flush=True)


# DRAM bytes (read + write) of one launch of the batched plan kernel on the
# 256-query batch in its autotuned shape, from the ncu capture summarised in
# profiles/plan_batch_kernel_uneven_256.md.  None until that kernel is
# captured again after a change.
PLAN_BATCH_DRAM_BYTES = 1_712_398_848


def bench_batched(dev, flush, reps=5, cpu_queries=8):
    """The 256-query uneven batch (2D/3D, n log-uniform in [512, 16384], 5-80
    boxes, Theorem 1 radii): prepared once, plan-stage scheme and shape
    autotuned, then whole batches (sampling + CSR + wavefront) replayed from
    the captured CUDA graph, L2 flushed before each.  End to end: the boxes of
    every query are copied from pinned host memory before each batch and
    every parent and cost array back after it, inside the timed region.  CPU
    baseline: the oracle's full step on `cpu_queries` of the queries."""
    import torch
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import envgen
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = envgen.batch_queries(seed=0, q=256)
    bp = BatchPlanner(qs, device=dev)
    # every query's boxes in one device buffer (one host-to-device copy per batch)
    counts = [pb.nbox * pb.dp for pb in qs]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    h_lo = torch.as_tensor(np.concatenate([np.ascontiguousarray(pb.box_lo, np.float32).ravel() for pb in qs]))
    h_hi = torch.as_tensor(np.concatenate([np.ascontiguousarray(pb.box_hi, np.float32).ravel() for pb in qs]))
    h_lo, h_hi = h_lo.pin_memory(), h_hi.pin_memory()
    d_lo, d_hi = h_lo.to(dev), h_hi.to(dev)
    for k in range(len(qs)):
        if counts[k]:
            bp.queries[k].boxes.lo = d_lo.data_ptr() + 4 * int(off[k])
            bp.queries[k].boxes.hi = d_hi.data_ptr() + 4 * int(off[k])
    infos = bp.plan()
    N.gmt_batch_autotune(bp.batch)
    mode, cluster, threads = N.gmt_batch_get_launch(bp.batch)
    st = torch.cuda.current_stream()
    ms, plan_ms = [], []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        raw = bp.plan(raw=True)  # info dicts are built after the timed region
        b.record(st)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        plan_ms.append(N.gmt_batch_last_plan_ms(bp.batch))
    infos = N.infos_as_dicts(raw)
    edges = sum(i["push_edges"] + i["pull_edges"] for i in infos)
    t = float(np.median(ms))
    tp = float(np.median(plan_ms))
    # end to end: host boxes in, parent and cost arrays out
    h_parent = torch.empty(bp.parent.numel(), dtype=torch.int32).pin_memory()
    h_cost = torch.empty(bp.cost.numel(), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        d_lo.copy_(h_lo, non_blocking=True)
        d_hi.copy_(h_hi, non_blocking=True)
        raw = bp.plan(raw=True)
        h_parent.copy_(bp.parent, non_blocking=True)
        h_cost.copy_(bp.cost, non_blocking=True)
        b.record(st)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    infos_e = N.infos_as_dicts(raw)
    assert [i["status"] for i in infos_e] == [i["status"] for i in infos]
    te = float(np.median(e2e_ms))
    # plan-stage roofline: algorithmic bytes of every query's wavefront (the
    # per-plan formula of the main line) over the plan-stage time
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    pbytes = sum(plan_bytes(i, pb.d, pb.N) for i, pb in zip(infos, qs))
    achieved = pbytes / (tp / 1e3) / 1e9
    # CPU baseline: the oracle's full step (SampleFree, all-pairs CSR,
    # wavefront) on queries spread over the sizes, single thread
    from oracle import oracle as O
    O.build()
    pick = sorted(range(len(qs)), key=lambda k: qs[k].n)[::max(1, len(qs) // cpu_queries)][:cpu_queries]
    cpu_s, cpu_e = 0.0, 0
    for k in pick:
        pb = qs[k]
        t0 = time.perf_counter()
        X, goal = O.sample(pb)
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, np.float32(O.radius_thm1(pb.n, pb.d)))
        _, _, oi = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                          pb.traj_points)
        cpu_s += time.perf_counter() - t0
        cpu_e += oi["push_edges"] + oi["pull_edges"]
        assert oi["push_edges"] == infos[k]["push_edges"] and oi["pull_edges"] == infos[k]["pull_edges"]
    scheme = {N.BATCH_TEAMS: "teams", N.BATCH_LOCKSTEP: "lockstep", N.BATCH_POOL: "pool"}.get(mode, str(mode))
    return {"workload": "256 uneven 2D/3D geometric queries, n log-uniform in [512, 16384], 5-80 boxes",
            "ms_per_batch_p50": t, "plans_per_s": 256 / (t / 1e3), "edges_checked_per_s": edges / (t / 1e3),
            "sum_nodes": int(sum(pb.N for pb in qs)), "edges_checked_per_batch": int(edges),
            "success_rate": float(np.mean([i["status"] == 0 for i in infos])),
            "plan_stage_ms_p50": tp,
            "autotuned": {"scheme": scheme, "cluster": cluster, "threads": threads},
            "gpu_launches_per_batch": "build kernels per (kind, dimension) group, then one plan-stage launch",
            "plan_stage_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                    "frac": achieved / hbm, "algorithmic_bytes": pbytes,
                                    "traffic": PLAN_BATCH_DRAM_BYTES},
            "e2e": {"value": edges / (te / 1e3), "unit": "edges/s", "ms_per_batch_p50": te,
                    "h2d_bytes_per_step": int(h_lo.numel() * 8), "d2h_bytes_per_step": int(bp.parent.numel() * 8)},
            "cpu_baseline": {"value": cpu_e / cpu_s, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(pick)} of the 256 queries (n {min(qs[k].n for k in pick)}.."
                                       f"{max(qs[k].n for k in pick)}), one full oracle step each (SampleFree, "
                                       f"all-pairs CSR, wavefront); {1e3 * cpu_s / len(pick):.0f} ms per query"}}


def bench_learned(train_envs=3000, test_envs=200, epochs=20):
    """The learned proposal against uniform sampling at equal path cost (3D box
    environments, 30 boxes, Theorem 1 radii): the network is trained on the
    plain-GMT* solutions (n = 16384) of `train_envs` seeded environments, then
    every arm plans `test_envs` held-out environments at n in 512 .. 4096; per
    arm the smallest n within 2% of uniform sampling's mean cost at n = 4096,
    with its p50 step and plan times; then the mixture in batched form (all
    held-out environments in one gmt_propose_batch + gmt_plan_batch call per
    n) against plain uniform sampling at n = 4096, batched and single-plan."""
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    t0 = time.time()
    X, SG, T, kept = learned.generate_dataset([1_000_000 + k for k in range(train_envs)], n=16384, log=None)
    t_data = time.time() - t0
    model = N.Model(learned.GRID, learned.HIDDEN, learned.CELLS, 256, seed=7)
    t1 = time.time()
    losses = learned.train(model, X, SG, T, epochs=epochs, log=None)
    t_train = time.time() - t1
    test = [2_000_000 + k for k in range(test_envs)]
    Xt, SGt, Tt, _ = learned.generate_dataset(test, n=16384, log=None)
    held_out = learned.mean_loss(model, Xt, SGt, Tt)
    ev = learned.evaluate(model, test, log=None)
    cross = ev["within_2pct_of_reference"]
    evb = learned.evaluate_batched(model, test, ns=(384, 512, 640, 768, 1024), n_ref=4096,
                                   plain_step_ms_p50=ev["reference"]["step_ms_p50"], log=None)
    return {"workload": f"3D boxes, {train_envs} training / {test_envs} held-out environments, n in {list(learned.NS)}",
            "reference": ev["reference"], "within_2pct_of_reference": cross,
            "batched": {"workload": f"all {test_envs} held-out environments as one batch per arm "
                                    "(gmt_propose_batch + gmt_plan_batch, autotuned, graph-replayed)",
                        "within_2pct_of_plain": evb["within_2pct_of_plain"],
                        "plain_batched": evb["plain_batched"],
                        "plain_single_step_ms_p50": evb["plain_single_step_ms_p50"],
                        "environments_compared": evb["environments_compared"],
                        "mixture_batched": evb["mixture_batched"]},
            "cost_vs_reference": {arm: {n: ev[arm][n]["cost_vs_uniform_ref"] for n in ev[arm]}
                                  for arm in ("uniform", "mixture", "uniform_mixture_radius")},
            "success": {arm: {n: ev[arm][n]["success"] for n in ev[arm]}
                        for arm in ("uniform", "mixture", "uniform_mixture_radius")},
            "training": {"solved_envs": len(kept), "epochs": epochs, "dataset_s": t_data, "train_s": t_train,
                         "final_loss": losses[-1], "held_out_loss": held_out,
                         "uniform_cell_loss": float(np.log(learned.CELLS ** 3))}}


def bench_dubins(dev, flush, reps=20):
    """Dubins airplane forest (n = 5000, lambda = 1, Halton samples, rho = 0.05,
    r = 0.2; ten trunks as 150 and as 5000 boxes): per repetition the L2 is
    flushed, then the graph is built and planned; library event times of the
    build stages and of the plan kernel, p50 over the repetitions."""
    import torch
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import envgen
    from paper_1705_02403_gb300.planner import Planner
    out = {"workload": "Dubins airplane forest, n=5000, lambda=1, Halton, rho=0.05, r=0.2"}
    for strips in (15, 500):
        pb = envgen.dubins_forest(0, n=5000, strips=strips, sampler=1)
        pl = Planner(pb, device=dev).build()
        N.gmt_graph_set_profiling(pl.graph, True)
        plan_ms, build_ms, infos = [], [], []
        for _ in range(reps):
            flush.zero_()
            pl.build()
            infos.append(pl.plan())
            torch.cuda.synchronize()
            p = N.gmt_graph_get_profile(pl.graph)
            plan_ms.append(p["plan_ms"])
            build_ms.append(p["sample_ms"] + p["pair_ms"] + p["transpose_ms"] + p["scan_ms"] + p["fill_ms"])
        edges = float(np.mean([i["push_edges"] + i["pull_edges"] for i in infos]))
        out[f"boxes_{10 * strips}"] = {
            "plan_ms_p50": pct(plan_ms, 50), "plan_ms_p99": pct(plan_ms, 99), "build_ms_p50": pct(build_ms, 50),
            "edges_checked_per_s_plan": edges / (pct(plan_ms, 50) / 1e3), "E": int(pl.view().E),
            "path_cost": float(infos[-1]["path_cost"]), "status": int(infos[-1]["status"])}
    return out


def bench_serving(local_rank):
    """10,000 requests at 100 Hz: 100 double-integrator sessions (n uniform in
    [2048, 8192], 30 boxes moving up to 0.02 per tick), 100 ticks."""
    from paper_1705_02403_gb300.serving import run_stream
    out = run_stream(sessions=100, ticks=100, hz=100.0, slots=32, cluster=4, threads=512, seed=local_rank, log=None)
    return {"workload": "100 Hz replanning stream, 100 DI sessions x 100 ticks, n in [2048, 8192], 30 moving boxes",
            "latency_ms_p50": out["latency_ms"]["p50"], "latency_ms_p99": out["latency_ms"]["p99"],
            "requests": out["requests"], "requests_per_s": out["requests_per_s"],
            "edges_checked_per_s": out["edges_checked_per_s"], "verdict_cache_hit_rate": out["verdict_cache_hit_rate"],
            "success_rate": out["success_rate"], "errors": out["errors"]}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
