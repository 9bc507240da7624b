"""Batched planning (gmt_plan_batch) against the CPU oracle, query by query.

Every query of a mixed batch (2D and 3D geometric, double integrator; uneven
n, own seeds, own boxes, Theorem 1 radii) must produce the same samples, CSR,
parents, costs and counters as the oracle on that query alone; a repeated call
(replayed from the captured CUDA graph) must give the same bits again; every
plan-stage scheme (pool, teams, lockstep) and every launch shape give the same
trees.
"""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

INFO_KEYS = ["status", "goal_node", "iters", "final_i", "push_edges", "pull_edges", "checks", "failed", "tree_size"]


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def mixed_batch(seed=0, q=14, n_max=1500):
    qs = envgen.batch_queries(seed=seed, q=q - 4, n_min=200, n_max=n_max)
    qs += [envgen.di6(seed=50 + k, n=300 + 97 * k, r=2.8) for k in range(3)]
    qs += [envgen.geometric(77, d=2, n=1, nbox=3, r=0.12)]   # the smallest query
    return qs


def oracle_of(O, pb):
    X, goal = O.sample_halton(pb) if pb.sampler == 1 else O.sample(pb)
    r0 = O.radius_halton(pb.n, pb.d) if pb.sampler == 1 else O.radius_thm1(pb.n, pb.d)
    r = pb.r if pb.r > 0 else np.float32(r0)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r, rho=pb.rho)
    parent, cost, info = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                                pb.traj_points)
    return X, goal, g, parent, cost, info


def check_query(O, bp, k, infos, ref=None):
    pb = bp.problems[k]
    X, goal, g, parent, cost, info = ref if ref is not None else oracle_of(O, pb)
    v = bp.view(k)
    assert np.array_equal(bits(v["X"].cpu().numpy()), bits(X))
    assert np.array_equal(v["is_goal"].cpu().numpy(), goal)
    c = g.csr()
    assert v["E"] == g.num_edges
    assert np.array_equal(v["out_row"].cpu().numpy(), c.out_row)
    assert np.array_equal(v["out_col"].cpu().numpy(), c.out_col)
    assert np.array_equal(bits(v["out_cost"].cpu().numpy()), bits(c.out_cost))
    assert np.array_equal(v["in_col"].cpu().numpy(), c.in_col)
    p, cs = bp.result(k)
    assert np.array_equal(p.cpu().numpy(), parent), k
    assert np.array_equal(bits(cs.cpu().numpy()), bits(cost)), k
    for key in INFO_KEYS:
        assert infos[k][key] == info[key], (k, key)
    if info["status"] == O.OK:
        n = infos[k]["path_len"]
        assert list(v["path"][:n].cpu().numpy()) == O.path_to(parent, info["goal_node"])
    return X, goal, g, parent, cost, info


def test_mixed_batch_matches_oracle_and_replays(O):
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch())
    infos = bp.plan()
    refs = [check_query(O, bp, k, infos) for k in range(len(bp.problems))]
    # second identical call: replayed from the captured graph; outputs cleared first
    bp.parent.fill_(-9)
    bp.cost.fill_(-9.0)
    infos2 = bp.plan()
    for k in range(len(bp.problems)):
        check_query(O, bp, k, infos2, refs[k])
    # a third call replays the same graph again
    infos3 = bp.plan()
    assert infos3 == infos2
    from paper_1705_02403_gb300 import _native as N
    assert N.gmt_batch_last_plan_ms(bp.batch) > 0.0


@pytest.mark.parametrize("shape", [(1, 256), (1, 1024), (2, 512), (4, 512), (8, 1024), (16, 512)])
def test_every_team_shape_gives_the_same_trees(O, shape):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch(seed=1, q=10))
    infos = bp.plan()
    N.gmt_batch_set_mode(bp.batch, N.BATCH_TEAMS)
    N.gmt_batch_set_launch(bp.batch, *shape)
    assert N.gmt_batch_get_launch(bp.batch) == (N.BATCH_TEAMS, shape[0], shape[1])
    infos = bp.plan()            # prepared once; this call replays with the shape
    for k in range(len(bp.problems)):
        check_query(O, bp, k, infos)


@pytest.mark.parametrize("threads", [128, 256])
def test_every_pool_shape_gives_the_same_trees(O, threads):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch(seed=5, q=12))
    bp.plan()
    N.gmt_batch_set_mode(bp.batch, N.BATCH_POOL)
    N.gmt_batch_set_launch(bp.batch, 0, threads)
    assert N.gmt_batch_get_launch(bp.batch) == (N.BATCH_POOL, 0, threads)
    for rep in range(3):   # prepared, then replayed twice from the captured graph
        bp.parent.fill_(-9)
        bp.cost.fill_(-9.0)
        infos = bp.plan()
        for k in range(len(bp.problems)):
            check_query(O, bp, k, infos)


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_every_lockstep_shape_gives_the_same_trees(O, threads):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch(seed=4, q=12))
    bp.plan()
    N.gmt_batch_set_mode(bp.batch, N.BATCH_LOCKSTEP)
    N.gmt_batch_set_launch(bp.batch, 0, threads)
    assert N.gmt_batch_get_launch(bp.batch) == (N.BATCH_LOCKSTEP, 0, threads)
    infos = bp.plan()
    for k in range(len(bp.problems)):
        check_query(O, bp, k, infos)


def test_pool_lockstep_and_teams_agree_bit_for_bit(O):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch(seed=3, q=16))
    infos_p = bp.plan()
    assert N.gmt_batch_get_launch(bp.batch)[0] == N.BATCH_TEAMS   # the untuned default
    for k in range(len(bp.problems)):
        check_query(O, bp, k, infos_p)
    p_p, c_p = bp.parent.clone(), bp.cost.clone()
    for mode in (N.BATCH_POOL, N.BATCH_LOCKSTEP):
        N.gmt_batch_set_mode(bp.batch, mode)
        bp.parent.fill_(-9)
        bp.cost.fill_(-9.0)
        infos = bp.plan()
        assert infos == infos_p
        assert torch.equal(bp.parent, p_p)
        assert torch.equal(bp.cost.view(torch.int32), c_p.view(torch.int32))


@pytest.mark.parametrize("flags", ["cells", "cells_list", "pairs"])
def test_neighbour_build_choice_gives_the_same_queries(O, flags):
    # Every geometric query forced onto the cell-list neighbour build (or onto
    # the all-pairs test), small queries, a dense one whose rows outgrow the cell
    # list's sort buffer (the batch is prepared again with all pairs for it) and
    # double-integrator queries beside them: each equals the oracle.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = mixed_batch(seed=8, q=12) + [envgen.geometric(41, d=2, n=3000, nbox=4, r=1.3),
                                      envgen.geometric(56, d=3, n=5000, nbox=20, r=0.0)]
    bp = BatchPlanner(qs)
    f = {"cells": N.GMT_DEBUG_PAIRS_CELLS, "cells_list": N.GMT_DEBUG_PAIRS_CELLS | N.GMT_DEBUG_CELLS_LIST,
         "pairs": N.GMT_DEBUG_PAIRS_ALL}[flags]
    for k, pb in enumerate(qs):
        if pb.kind == envgen.EUCLID:
            bp.queries[k].params.debug_flags = f
    infos = bp.plan()
    for k in range(len(qs)):
        check_query(O, bp, k, infos)
    infos2 = bp.plan()          # replayed
    assert infos2 == infos


def test_halton_queries_in_a_batch(O):
    # Halton and Philox queries side by side (2D, 3D, double integrator, one
    # large enough for the cell list): each equals the oracle on its own.
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = mixed_batch(seed=9, q=10)
    qs = [pb.with_(sampler=k % 2) for k, pb in enumerate(qs)]
    qs.append(envgen.geometric(76, d=2, n=6000, nbox=20, r=0.0).with_(sampler=1))
    bp = BatchPlanner(qs)
    infos = bp.plan()
    for k in range(len(qs)):
        check_query(O, bp, k, infos)


@pytest.mark.parametrize("mode", ["pool", "teams", "lockstep"])
def test_dubins_queries_in_a_batch(O, mode):
    # Dubins airplane queries (Philox and Halton, 30 to 500 boxes, two turning
    # radii) next to geometric and double-integrator ones, under both plan-stage
    # schemes: each equals the oracle on its own.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = mixed_batch(seed=11, q=8)
    qs += [envgen.dubins_forest(31, n=900, r=0.3, trunks=3, strips=10),
           envgen.dubins_forest(32, n=1400, r=0.28, strips=15, sampler=1),
           envgen.dubins_forest(33, n=700, r=0.35, rho=0.1, strips=50),
           envgen.dubins_forest(34, n=64, r=0.6, trunks=2)]
    bp = BatchPlanner(qs)
    bp.plan()
    N.gmt_batch_set_mode(bp.batch, {"pool": N.BATCH_POOL, "teams": N.BATCH_TEAMS, "lockstep": N.BATCH_LOCKSTEP}[mode])
    infos = bp.plan()
    for k in range(len(qs)):
        check_query(O, bp, k, infos)
    v, _ = N.gmt_batch_get_view(bp.batch, len(qs) - 1)
    assert v.turn_radius == np.float32(qs[-1].rho) and v.in_path is not None


@pytest.mark.parametrize("mode", ["pool", "lockstep"])
def test_600_small_queries(O, mode):
    # 600 small queries: the lockstep scheme runs them as two launches, the
    # pool scheme in one
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = envgen.batch_queries(seed=5, q=600, n_min=16, n_max=200)
    bp = BatchPlanner(qs)
    bp.plan()
    N.gmt_batch_set_mode(bp.batch, N.BATCH_POOL if mode == "pool" else N.BATCH_LOCKSTEP)
    infos = bp.plan()
    for k in range(len(qs)):
        check_query(O, bp, k, infos)


@pytest.mark.parametrize("mode", ["pool", "lockstep"])
def test_nearly_complete_graphs_in_a_batch(O, mode):
    # Nearly complete graphs: x_init alone claims more candidates in its first
    # iteration than a lockstep block's shared-memory queue holds (the pushing
    # warp pulls the rest itself), and in the pool scheme one group node
    # produces over a thousand PULL items.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = [envgen.geometric(600 + k, d=2, n=1500, nbox=4, r=1.0) for k in range(2)]
    qs += [envgen.geometric(610, d=3, n=1400, nbox=6, r=1.2)]
    qs += envgen.batch_queries(seed=6, q=5, n_min=200, n_max=800)
    bp = BatchPlanner(qs)
    bp.plan()
    N.gmt_batch_set_mode(bp.batch, N.BATCH_POOL if mode == "pool" else N.BATCH_LOCKSTEP)
    infos = bp.plan()
    for k in range(len(qs)):
        check_query(O, bp, k, infos)
    assert max(bp.view(k)["E"] / qs[k].N for k in range(3)) > 1024


@pytest.mark.parametrize("mode", ["lockstep", "teams", "pool"])
def test_iteration_limit_per_query(O, mode):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = mixed_batch(seed=7, q=10)
    bp = BatchPlanner(qs)
    limits = {1: 1, 3: 4, 5: 2, 8: 6}
    for k, m in limits.items():
        bp.queries[k].params.max_iters = m
    bp.plan(allow_errors=True)
    N.gmt_batch_set_mode(bp.batch, {"pool": N.BATCH_POOL, "teams": N.BATCH_TEAMS, "lockstep": N.BATCH_LOCKSTEP}[mode])
    infos = bp.plan(allow_errors=True)
    for k, pb in enumerate(qs):
        X, goal = O.sample(pb)
        r = pb.r if pb.r > 0 else np.float32(O.radius_thm1(pb.n, pb.d))
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r)
        parent, cost, info = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                                    pb.traj_points, max_iters=limits.get(k))
        p, c = bp.result(k)
        assert np.array_equal(p.cpu().numpy(), parent), k
        assert np.array_equal(bits(c.cpu().numpy()), bits(cost)), k
        for key in INFO_KEYS:
            assert infos[k][key] == info[key], (k, key)
    assert any(infos[k]["status"] == N.GMT_ERR_ITER_LIMIT for k in limits)


def test_autotune_keeps_results(O):
    # The autotuner times every scheme and shape on the prepared batch; its
    # runs leave the CSR and the later trees equal to the oracle's.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner(mixed_batch(seed=2, q=12))
    infos = bp.plan()
    refs = [oracle_of(O, pb) for pb in bp.problems]
    c, t, ms = N.gmt_batch_autotune(bp.batch)
    # the autotuner ran the build's back half (fill, plan) many times on the
    # same samples and masks: the CSR it leaves is still the oracle's
    for k in range(len(bp.problems)):
        v = bp.view(k)
        g = refs[k][2].csr()
        assert v["E"] == refs[k][2].num_edges, k
        assert np.array_equal(v["out_col"].cpu().numpy(), g.out_col), k
        assert np.array_equal(bits(v["out_cost"].cpu().numpy()), bits(g.out_cost)), k
    mode, c2, t2 = N.gmt_batch_get_launch(bp.batch)
    assert mode in (N.BATCH_TEAMS, N.BATCH_LOCKSTEP, N.BATCH_POOL) and t2 == t and c2 == c
    assert (c == 0) == (mode in (N.BATCH_LOCKSTEP, N.BATCH_POOL))
    assert c in (0, 1, 2, 4, 8, 16) and t in (128, 256, 512, 1024) and ms > 0
    infos2 = bp.plan()
    for k in range(len(bp.problems)):
        check_query(O, bp, k, infos2, ref=refs[k])


@pytest.mark.parametrize("mode", ["pool", "teams", "lockstep"])
def test_full_size_batch_sampled_queries(O, mode):
    # The 256-query workload (n up to 16384): every query's tree is checked for
    # the paper's invariants on the GPU result, and a sample of queries, the
    # largest included, against the oracle bit for bit.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = envgen.batch_queries(seed=0, q=256)
    bp = BatchPlanner(qs)
    infos = bp.plan()
    if mode != "teams":
        N.gmt_batch_set_mode(bp.batch, N.BATCH_LOCKSTEP if mode == "lockstep" else N.BATCH_POOL)
        infos = bp.plan()
    assert N.gmt_batch_get_launch(bp.batch)[0] == {"pool": N.BATCH_POOL, "teams": N.BATCH_TEAMS,
                                                   "lockstep": N.BATCH_LOCKSTEP}[mode]
    sizes = np.array([pb.n for pb in qs])
    pick = sorted(set([int(np.argmax(sizes)), int(np.argmin(sizes))] + list(range(0, 256, 37))))
    for k in pick:
        check_query(O, bp, k, infos)
    for k in range(256):
        p, c = bp.result(k)
        p = p.cpu().numpy(); c = c.cpu().numpy()
        tree = p >= 0
        assert tree.sum() + 1 == np.isfinite(c).sum() == infos[k]["tree_size"]
        assert np.all(c[p[tree]] < c[tree])          # costs grow along tree edges


def test_invalid_batch_arguments(O):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    bp = BatchPlanner([envgen.geometric(1, d=4, n=100, nbox=2, r=0.3)])
    with pytest.raises(N.GmtError) as e:
        bp.plan()
    assert e.value.status == N.GMT_ERR_INVALID


def free_points(pb, count, seed):
    """`count` seeded uniform states of X outside every box: [d][count]."""
    rng = np.random.default_rng([seed, 1705, 77])
    out = []
    while len(out) < count:
        x = rng.uniform(pb.lo, pb.hi).astype(np.float32)
        p = x[:pb.dp]
        if len(pb.box_lo) and np.any(np.all((pb.box_lo <= p) & (p <= pb.box_hi), axis=1)):
            continue
        out.append(x)
    return np.stack(out, 1)


def appended_oracle(O, pb, extra):
    """The oracle on SampleFree's n + 1 nodes followed by `extra` [d][m]."""
    X, goal = O.sample_halton(pb) if pb.sampler == 1 else O.sample(pb)
    gd = pb.dp if pb.goal_pos_only else pb.d
    g_extra = np.array([O.in_goal(extra[:, j], gd, pb.goal_center, pb.goal_radius) for j in range(extra.shape[1])],
                       np.uint8)
    X = np.concatenate([X, extra], 1)
    goal = np.concatenate([goal, g_extra])
    r0 = O.radius_halton(pb.n, pb.d) if pb.sampler == 1 else O.radius_thm1(pb.n, pb.d)
    r = pb.r if pb.r > 0 else np.float32(r0)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r, rho=pb.rho)
    parent, cost, info = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                                pb.traj_points)
    return X, goal, g, parent, cost, info


def test_appended_samples_match_oracle_and_replay(O):
    # gmt_query.extra: caller samples appended after each query's n + 1
    # SampleFree nodes (the batched form of the learned mixture) give the
    # oracle's samples, CSR, tree and counters on the same node set; a replay
    # reads the appended samples again, so contents rewritten in place plan
    # anew, and a replayed sample in an obstacle fails only its own query.
    from paper_1705_02403_gb300 import learned
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import BatchPlanner
    qs = [learned.env(900 + k, 300 + 41 * k).with_(r=0.0) for k in range(3)]
    qs += [envgen.geometric(910, d=2, n=350, nbox=8, r=0.0), envgen.geometric(911, d=2, n=257, nbox=8, r=0.0)
           .with_(sampler=1)]
    qs += [envgen.di6(seed=920 + k, n=280 + 53 * k, r=2.8) for k in range(2)]
    m, pitch = 150, 160
    ext = np.zeros((len(qs), 6, pitch), np.float32)
    for k, pb in enumerate(qs):
        ext[k, :pb.d, :m] = free_points(pb, m, k)
    extra = torch.tensor(ext, device="cuda")
    bp = BatchPlanner(qs, extra=extra, extra_count=m)
    infos = bp.plan()
    for k, pb in enumerate(qs):
        check_query(O, bp, k, infos, ref=appended_oracle(O, pb, ext[k, :pb.d, :m]))
    # appended samples rewritten in place (permuted: the same edge count, so
    # the replayed arena still fits; new node indices, so new CSR order and
    # tie-breaks): the replay plans the new contents
    for k, pb in enumerate(qs):
        perm = np.random.default_rng(k).permutation(m)
        ext[k, :pb.d, :m] = ext[k, :pb.d, :m][:, perm]
    extra.copy_(torch.tensor(ext))
    bp.parent.fill_(-9)
    infos2 = bp.plan()
    for k, pb in enumerate(qs):
        check_query(O, bp, k, infos2, ref=appended_oracle(O, pb, ext[k, :pb.d, :m]))
    # an appended sample inside a box of query 0: that query reports the error
    pb0 = qs[0]
    inside = (pb0.box_lo[0] + pb0.box_hi[0]) / 2
    bad = ext.copy()
    bad[0, :3, 7] = inside
    extra.copy_(torch.tensor(bad))
    infos3 = bp.plan(allow_errors=True)
    assert infos3[0]["status"] == N.GMT_ERR_INVALID
    assert all(infos3[k]["status"] in (0, N.GMT_NO_PATH) for k in range(1, len(qs)))
    # the same call on a fresh handle fails before planning
    bp2 = BatchPlanner(qs, extra=extra, extra_count=m)
    with pytest.raises(RuntimeError):
        bp2.plan()
