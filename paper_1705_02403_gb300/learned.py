"""Learned sampling proposal: data from plain GMT* solutions, training, and
evaluation of the 50/50 mixture (learned + uniform) against uniform sampling.

All computation runs in libgmt.so (batched planner, voxeliser, path
histograms, tcgen05 forward/backward, AdamW, proposal sampler); this module
sequences the calls and keeps the tensors.

Mixture rule: a plan with n samples draws n/2 with SampleFree (uniform, node 1
in the goal) and n/2 from the proposal; the connection radius is Theorem 1's
for the n/2 uniform samples alone, so the uniform half keeps the paper's
guarantee (Theorem 3 needs only the uniform samples and that radius).

    python -m paper_1705_02403_gb300.learned --train-envs 10000 --test-envs 1000 --out learned.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import _native as N
from . import envgen
from .planner import BatchPlanner, boxes_on_device, goal_struct, params_struct, space_struct

GRID, HIDDEN, CELLS = 32, 512, 16


def env(seed: int, n: int, nbox: int = 30) -> envgen.Problem:
    """3D box environment with its own start (near the origin corner) and goal
    ball (near the opposite corner); r = 0 selects Theorem 1's radius."""
    rng = np.random.default_rng([seed, 1705, 4])
    x0 = rng.uniform(0.02, 0.25, 3)
    gc = rng.uniform(0.75, 0.98, 3)
    bl, bh = envgen.random_boxes(rng, nbox, 3, x0, gc, 0.05, side=(0.05, 0.3))
    return envgen.Problem(kind=envgen.EUCLID, d=3, dp=3, lo=np.zeros(3, np.float32), hi=np.ones(3, np.float32),
                          box_lo=bl, box_hi=bh, x_init=x0.astype(np.float32), goal_center=gc.astype(np.float32),
                          goal_radius=0.05, goal_pos_only=False, n=n, r=0.0, lam=0.5, seed=seed, tag="learned3d")


def start_goal(pbs):
    return torch.tensor(np.stack([np.concatenate([pb.x_init[:3], pb.goal_center[:3]]) for pb in pbs]),
                        dtype=torch.float32, device="cuda")


def voxelize(pbs):
    X = torch.empty(len(pbs), GRID ** 3, dtype=torch.bfloat16, device="cuda")
    keep = [boxes_on_device(pb) for pb in pbs]
    N.gmt_voxelize([k[0] for k in keep], GRID, X.data_ptr())
    return X


def generate_dataset(seeds, n=16384, chunk=256, log=print):
    """Plain GMT* on every environment; targets = path histograms over cells."""
    Xs, SGs, Ts, kept = [], [], [], []
    t0 = time.time()
    for c in range(0, len(seeds), chunk):
        pbs = [env(s, n) for s in seeds[c:c + chunk]]
        bp = BatchPlanner(pbs)
        infos = bp.plan()
        ok = [k for k, i in enumerate(infos) if i["status"] == 0]
        T = torch.empty(len(ok), CELLS ** 3, dtype=torch.float32, device="cuda")
        for row, k in enumerate(ok):
            v = bp.view(k)
            N.gmt_path_histogram(v["X"].data_ptr(), v["X"].stride(0), v["path"].data_ptr(), infos[k]["path_len"],
                                 CELLS, 0.01, 1e-4, T[row].data_ptr())
        sel = [pbs[k] for k in ok]
        Xs.append(voxelize(sel))
        SGs.append(start_goal(sel))
        Ts.append(T)
        kept += [seeds[c + k] for k in ok]
        del bp
        if log:
            log(f"  dataset {c + len(pbs)}/{len(seeds)} solved {len(kept)} ({time.time() - t0:.1f}s)")
    return torch.cat(Xs), torch.cat(SGs), torch.cat(Ts), kept


def train(model: N.Model, X, SG, T, epochs=20, batch=256, lr=1e-3, wd=1e-4, seed=0, log=print):
    n = X.shape[0]
    g = torch.Generator().manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch].cuda()
            xb, sgb, tb = X[idx].contiguous(), SG[idx].contiguous(), T[idx].contiguous()
            loss = model.train_step(batch, xb.data_ptr(), sgb.data_ptr(), tb.data_ptr(), lr, wd)
            tot += loss
            cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"  epoch {ep}: mean loss {losses[-1]:.4f}")
    return losses


def mean_loss(model: N.Model, X, SG, T, batch=256):
    tot, cnt = 0.0, 0
    for s in range(0, X.shape[0], batch):
        b = min(batch, X.shape[0] - s)
        tot += model.backward(b, X[s:s + b].contiguous().data_ptr(), SG[s:s + b].contiguous().data_ptr(),
                              T[s:s + b].contiguous().data_ptr()) * b
        cnt += b
    return tot / cnt


def _timed(fn):
    """Runs fn() (which queues device work on the current stream and returns
    (info dict, graph)); returns (info, step ms from the first queued kernel to
    the plan's end, plan-kernel ms)."""
    st = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    info, g = fn()
    b.record(st)
    b.synchronize()
    plan_ms = N.gmt_graph_get_profile(g)["plan_ms"]
    return info, a.elapsed_time(b), plan_ms, g


def plan_uniform(pb: envgen.Problem, graph: N.Graph | None = None):
    """SampleFree + CSR + wavefront for one environment (single-plan API).
    Returns ((status, cost), step ms, plan ms, graph)."""
    space, goal = space_struct(pb), goal_struct(pb)
    boxes, keep = boxes_on_device(pb)
    params = params_struct(pb)
    g = graph if graph is not None else N.Graph()
    parent = torch.empty(pb.N, dtype=torch.int32, device="cuda")
    cost = torch.empty(pb.N, dtype=torch.float32, device="cuda")

    def run():
        N.gmt_build_graph_async(space, boxes, [float(v) for v in pb.x_init], goal, params, g)
        N.gmt_graph_set_profiling(g, 2)
        return N.gmt_plan(g, boxes, params, parent.data_ptr(), cost.data_ptr()).as_dict(), g

    info, step_ms, plan_ms, g = _timed(run)
    return (info["status"], info["path_cost"]), step_ms, plan_ms, g


def plan_mixture(model: N.Model, pb: envgen.Problem, graph: N.Graph | None = None):
    """n/2 uniform (SampleFree) + n/2 learned samples, radius for n/2: the
    proposal's forward pass and draws, the CSR and the wavefront.  Returns
    ((status, cost), step ms, plan ms, graph)."""
    n_u = pb.n // 2
    n_l = pb.n - n_u
    r = np.float32(N.gmt_connection_radius(n_u, 3, 0.0, 1.0))
    upb = pb.with_(n=n_u, r=float(r))
    space, goal = space_struct(upb), goal_struct(upb)
    boxes, keep = boxes_on_device(upb)
    params = params_struct(upb)
    samples = torch.empty(3, n_l, dtype=torch.float32, device="cuda")
    Nn = n_u + 1 + n_l
    parent = torch.empty(Nn, dtype=torch.int32, device="cuda")
    cost = torch.empty(Nn, dtype=torch.float32, device="cuda")

    def run():
        N.gmt_propose(model, space, boxes, upb.x_init, upb.goal_center, n_l, int(pb.seed) ^ 0x5A5A5A5A,
                      samples.data_ptr(), n_l)
        g = N.gmt_build_graph_ex(space, boxes, [float(v) for v in upb.x_init], goal, params, samples.data_ptr(), n_l,
                                 n_l, graph)
        N.gmt_graph_set_profiling(g, 2)
        return N.gmt_plan(g, boxes, params, parent.data_ptr(), cost.data_ptr()).as_dict(), g

    info, step_ms, plan_ms, g = _timed(run)
    return (info["status"], info["path_cost"]), step_ms, plan_ms, g


class MixtureBatch:
    """The mixture planned for many environments at once: gmt_propose_batch
    draws every environment's n/2 learned samples (one forward pass per
    max_batch environments, one sampling launch, one host synchronisation),
    and gmt_plan_batch plans every query with its learned samples appended
    after its n/2 + 1 SampleFree nodes (replayed from its CUDA graph from the
    second call on).  Every query's tree equals a single gmt_plan on the same
    sample set."""

    def __init__(self, model: N.Model, problems):
        self.model = model
        n = problems[0].n
        assert all(pb.n == n for pb in problems)
        self.n_u = n // 2
        self.n_l = n - self.n_u
        r = float(np.float32(N.gmt_connection_radius(self.n_u, 3, 0.0, 1.0)))
        self.upbs = [pb.with_(n=self.n_u, r=r) for pb in problems]
        self.spaces = [space_struct(u) for u in self.upbs]
        self._keep = [boxes_on_device(u) for u in self.upbs]
        self.boxes = [k[0] for k in self._keep]
        self.sg = [np.concatenate([u.x_init[:3], u.goal_center[:3]]) for u in self.upbs]
        self.seeds = [int(pb.seed) ^ 0x5A5A5A5A for pb in problems]
        self.samples = torch.empty(len(problems), 3, self.n_l, dtype=torch.float32, device="cuda")
        self.planner = BatchPlanner(self.upbs, extra=self.samples, extra_count=self.n_l)
        self.args = N.ProposeBatchArgs(self.spaces, self.boxes, self.sg, self.seeds)

    def propose(self):
        N.gmt_propose_batch(self.model, None, None, None, self.n_l, None, self.samples.data_ptr(), self.n_l,
                            args=self.args)

    def run(self, allow_errors=True, raw=False):
        self.propose()
        return self.planner.plan(allow_errors=allow_errors, raw=raw)


def _batch_timed(run, reps):
    """p50 of CUDA-event times around run() (which synchronises and returns
    the ctypes info array, or None), and the info dicts of the last call
    (converted outside the timed region)."""
    st = torch.cuda.current_stream()
    times, infos = [], None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        infos = run()
        b.record(st)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times)), (N.infos_as_dicts(infos) if infos is not None else None)


def evaluate_batched(model: N.Model, seeds, ns, n_ref=4096, reps=5, plain_step_ms_p50=None, log=print):
    """The mixture in batched form against plain GMT* at equal path cost.
    For every n in ns, all environments as one batch (gmt_propose_batch +
    gmt_plan_batch, autotuned, then graph-replayed): batch time p50
    over reps calls (and of the proposal and the batched plan alone) and mean
    path cost; the plain method is uniform sampling
    at n_ref, both batched (gmt_plan_batch) and, if given, the single-plan p50
    step time.  Costs are compared over the environments every arm solves.
    The crossing is the smallest n whose mean cost is within 2% of plain
    uniform@n_ref and whose success rate is within 2 points of it."""
    pbs_ref = [env(s, n_ref) for s in seeds]
    plain = BatchPlanner(pbs_ref)
    plain.plan(allow_errors=True)
    N.gmt_batch_autotune(plain.batch)
    plain_ms, plain_infos = _batch_timed(lambda: plain.plan(allow_errors=True, raw=True), reps + 1)
    arms = {}
    for n in ns:
        mb = MixtureBatch(model, [env(s, n) for s in seeds])
        mb.run()
        N.gmt_batch_autotune(mb.planner.batch)
        ms, infos = _batch_timed(lambda: mb.run(raw=True), reps + 1)
        prop_ms, _ = _batch_timed(mb.propose, reps + 1)
        plan_ms, _ = _batch_timed(lambda: mb.planner.plan(allow_errors=True, raw=True), reps + 1)
        arms[n] = (ms, infos, prop_ms, plan_ms)
    B = len(seeds)
    both = [i for i in range(B) if plain_infos[i]["status"] == 0 and all(a[1][i]["status"] == 0 for a in arms.values())]
    ref = float(np.mean([plain_infos[i]["path_cost"] for i in both])) if both else float("nan")
    ref_success = float(np.mean([x["status"] == 0 for x in plain_infos]))
    res = {"environments": B, "environments_compared": len(both),
           "plain_batched": {"n": n_ref, "batch_ms_p50": plain_ms, "ms_per_plan": plain_ms / B,
                             "mean_cost": ref, "success": ref_success},
           "plain_single_step_ms_p50": plain_step_ms_p50, "mixture_batched": {}}
    for n, (ms, infos, prop_ms, plan_ms) in arms.items():
        costs = [infos[i]["path_cost"] for i in both]
        res["mixture_batched"][str(n)] = {
            "batch_ms_p50": ms, "ms_per_plan": ms / B, "propose_ms_p50": prop_ms, "plan_batch_ms_p50": plan_ms,
            "success": float(np.mean([x["status"] == 0 for x in infos])),
            "mean_cost": float(np.mean(costs)) if costs else None,
            "cost_vs_plain": (float(np.mean(costs)) / ref) if costs else None}
    ok = [n for n in ns if res["mixture_batched"][str(n)]["cost_vs_plain"] is not None
          and res["mixture_batched"][str(n)]["cost_vs_plain"] <= 1.02
          and res["mixture_batched"][str(n)]["success"] >= ref_success - 0.02]
    n0 = min(ok) if ok else None
    cross = {"n": n0, "sample_reduction": (n_ref / n0) if n0 else None}
    if n0:
        mpp = res["mixture_batched"][str(n0)]["ms_per_plan"]
        cross["ms_per_plan"] = mpp
        cross["speedup_vs_plain_batched"] = res["plain_batched"]["ms_per_plan"] / mpp
        cross["speedup_vs_plain_single_p50"] = (plain_step_ms_p50 / mpp) if plain_step_ms_p50 else None
    res["within_2pct_of_plain"] = cross
    if log:
        log(json.dumps(res, indent=1))
    return res


NS = (256, 384, 512, 640, 768, 1024, 1365, 2048, 4096)


def evaluate(model: N.Model, seeds, ns=NS, n_ref=4096, log=print):
    """Mean path cost of three arms at each n, over the environments every arm
    solves at every n, relative to uniform sampling at n_ref:
      uniform                 SampleFree with Theorem 1's radius for n;
      mixture                 n/2 SampleFree + n/2 learned, Theorem 1's radius for n/2;
      uniform_mixture_radius  SampleFree with the mixture's radius (n/2), which
                              isolates what the learned samples add.
    Per arm: the smallest n whose mean cost is within 2% of the reference (and
    whose success rate is within 2 points of it), with the p50 step and plan
    times there (CUDA events; the step includes sampling, the proposal's
    forward pass and draws, and the CSR)."""
    arms = ("uniform", "mixture", "uniform_mixture_radius")
    per = {}
    g = None
    for n in sorted(set(ns) | {n_ref}):
        r_half = float(np.float32(N.gmt_connection_radius(n // 2, 3, 0.0, 1.0)))
        for arm in arms:
            if arm != "uniform" and n not in ns:
                continue
            out = []
            for s in seeds:
                pb = env(s, n)
                if arm == "mixture":
                    r, step, plan, g = plan_mixture(model, pb, g)
                else:
                    r, step, plan, g = plan_uniform(pb.with_(r=r_half) if arm != "uniform" else pb, g)
                out.append((r[0], r[1], step, plan))
            per[(arm, n)] = out
    keys = list(per)
    both = [i for i in range(len(seeds)) if all(per[k][i][0] == 0 for k in keys)]
    ref_rows = per[("uniform", n_ref)]
    ref = float(np.mean([ref_rows[i][1] for i in both])) if both else float("nan")
    ref_success = float(np.mean([x[0] == 0 for x in ref_rows]))
    res = {arm: {} for arm in arms}
    for (arm, n), rows in per.items():
        costs = [rows[i][1] for i in both]
        res[arm][str(n)] = {"success": float(np.mean([x[0] == 0 for x in rows])),
                            "mean_cost": float(np.mean(costs)) if costs else None,
                            "cost_vs_uniform_ref": (float(np.mean(costs)) / ref) if costs else None,
                            "step_ms_p50": float(np.median([x[2] for x in rows])),
                            "plan_ms_p50": float(np.median([x[3] for x in rows]))}
    res["reference"] = {"arm": "uniform", "n": n_ref, "mean_cost": ref, "success": ref_success,
                        "environments_compared": len(both), "environments": len(seeds),
                        "step_ms_p50": res["uniform"][str(n_ref)]["step_ms_p50"],
                        "plan_ms_p50": res["uniform"][str(n_ref)]["plan_ms_p50"]}
    crossing = {}
    for arm in arms:
        ok = [n for n in ns if res[arm][str(n)]["cost_vs_uniform_ref"] is not None
              and res[arm][str(n)]["cost_vs_uniform_ref"] <= 1.02
              and res[arm][str(n)]["success"] >= ref_success - 0.02]
        n0 = min(ok) if ok else None
        crossing[arm] = {"n": n0, "sample_reduction": (n_ref / n0) if n0 else None,
                         "step_ms_p50": res[arm][str(n0)]["step_ms_p50"] if n0 else None,
                         "plan_ms_p50": res[arm][str(n0)]["plan_ms_p50"] if n0 else None}
    res["within_2pct_of_reference"] = crossing
    if log:
        log(json.dumps(res, indent=1))
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-envs", type=int, default=10000)
    ap.add_argument("--test-envs", type=int, default=1000)
    ap.add_argument("--train-n", type=int, default=16384)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--out", default="learned.json")
    ap.add_argument("--checkpoint", default="")
    a = ap.parse_args()
    t0 = time.time()
    train_seeds = [1_000_000 + k for k in range(a.train_envs)]
    test_seeds = [2_000_000 + k for k in range(a.test_envs)]
    X, SG, T, kept = generate_dataset(train_seeds, n=a.train_n)
    t_data = time.time() - t0
    model = N.Model(GRID, HIDDEN, CELLS, 256, seed=7)
    t1 = time.time()
    losses = train(model, X, SG, T, epochs=a.epochs)
    t_train = time.time() - t1
    if a.checkpoint:
        model.save(a.checkpoint)
    Xt, SGt, Tt, _ = generate_dataset(test_seeds[:256], n=a.train_n, log=None)
    test_loss = mean_loss(model, Xt, SGt, Tt)
    ev = evaluate(model, test_seeds)
    out = {"train_envs": a.train_envs, "solved_train_envs": len(kept), "train_n": a.train_n, "epochs": a.epochs,
           "losses": losses, "held_out_loss": test_loss, "dataset_s": t_data, "train_s": t_train, "eval": ev,
           "total_s": time.time() - t0}
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "losses"}, indent=1))


if __name__ == "__main__":
    main()
