"""Pins of the oracle's Algorithm 1 (GMT*), FMT* and Dijkstra.

Hand traces use dyadic coordinates so that every cost is exact in FP32; the
expected values in the tests were worked out by hand from Alg. 1 (Sec. III-A)
with the readings: group rule cost <= i*delta, V_open taken at the start of an
iteration, lazy failures stay unexplored, termination after the group is
expanded, result = minimum-cost goal node.
"""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra as sp_dijkstra

from paper_1705_02403_gb300 import envgen

F = np.float32
NOBOX = np.zeros((0, 2), F)


def graph2d(O, pts, goal_idx, r):
    X = np.array(pts, F).T.copy()
    goal = np.zeros(len(pts), np.uint8)
    goal[goal_idx] = 1
    return O.Graph(0, 2, 2, X, goal, r)


def test_trace_threshold_and_skip(O):
    # 0 = x_init (0,0), 1 = goal (0.5,0), 2 = a (0.125,0), 3 = b (0,0.1875),
    # 4 = c (0.3125,0); r = 0.25, lambda = 0.5, delta = 0.125.
    # Edges (< r): 0-2 .125, 0-3 .1875, 2-3 .2253, 2-4 .1875, 4-1 .1875.
    # i=0: G={0}; X_near={2,3}; 2<-0 (.125), 3<-0 (.1875).       next i=1
    # i=1 (theta .125): G={2} (cost equal to theta is in); X_near={4};
    #      4<-2 (.3125).                                          next i=2
    # i=2 (theta .25): G={3}; nothing unexplored.                 next i=3
    # i=3 (theta .375): G={4}; X_near={1}; 1<-4 (.5).             next i=4
    # i=4 (theta .5): G={1} holds the goal -> success, cost 0.5.
    g = graph2d(O, [(0, 0), (0.5, 0), (0.125, 0), (0, 0.1875), (0.3125, 0)], [1], 0.25)
    parent, cost, info, added, closed = g.plan(NOBOX, NOBOX, [0, 0], [1, 1], 0.5, trace=True)
    assert list(parent) == [-1, 4, 0, 0, 2]
    assert list(cost) == [0.0, 0.5, 0.125, 0.1875, 0.3125]
    assert info["status"] == O.OK and info["goal_node"] == 1 and info["path_cost"] == 0.5
    assert (info["iters"], info["final_i"]) == (5, 4)
    assert (info["push_edges"], info["pull_edges"], info["checks"], info["failed"]) == (10, 8, 4, 0)
    assert info["tree_size"] == 5
    assert list(added) == [-1, 3, 0, 0, 1] and list(closed) == [0, 4, 1, 2, 3]
    assert O.path_to(parent, 1) == [0, 2, 4, 1]
    # stepping through the empty groups gives the same result
    p2, c2, i2 = g.plan(NOBOX, NOBOX, [0, 0], [1, 1], 0.5, skip_empty=False)
    assert np.array_equal(p2, parent) and np.array_equal(c2, cost) and i2 == info


def trace_b(O):
    # 0 = x_init (0,0), 1 = d (0.125,0.375), 2 = a (0.1875,0), 3 = b (0,0.1875),
    # 4 = goal c (0.1875,0.1875); one box [0.15,0.25]x[0.05,0.1] blocks a->c.
    # Edges: 0-2 .1875, 0-3 .1875, 2-4 .1875, 3-4 .1875, 3-1 .2253, 4-1 .1976.
    g = graph2d(O, [(0, 0), (0.125, 0.375), (0.1875, 0), (0, 0.1875), (0.1875, 0.1875)], [4], 0.25)
    box_lo = np.array([[0.15, 0.05]], F)
    box_hi = np.array([[0.25, 0.1]], F)
    return g, box_lo, box_hi


def test_trace_lazy_failure_and_retry(O):
    # i=0: G={0}; 2<-0, 3<-0 (both .1875).                       next i=2
    # i=2 (theta .25): G={2,3}; X_near={1,4}.  1<-3 (.1875+.2253).
    #      4: parents 2 and 3 tie at .375, the lower index 2 wins, and the edge
    #      2->4 crosses the box: the check fails, 4 stays unexplored.
    #      G closes; V_open = {1}.                               next i=4
    # i=4 (theta .5): G={1}; 4 is retried: 4<-1.                  next i=5
    # i=5: G={4} holds the goal -> success.
    g, bl, bh = trace_b(O)
    parent, cost, info, added, closed = g.plan(bl, bh, [0, 0], [1, 1], 0.5, trace=True)
    c1 = F(F(0.1875) + np.sqrt(F(0.05078125)))
    c4 = F(c1 + np.sqrt(F(0.0390625)))
    assert list(parent) == [-1, 3, 0, 0, 1]
    assert cost[1] == c1 and cost[4] == c4
    assert info["status"] == O.OK and info["goal_node"] == 4 and info["path_cost"] == float(c4)
    assert (info["iters"], info["final_i"]) == (4, 5)
    assert (info["push_edges"], info["pull_edges"], info["checks"], info["failed"]) == (12, 13, 5, 1)
    assert list(added) == [-1, 2, 0, 0, 4] and list(closed) == [0, 4, 2, 2, 5]


def test_trace_fmt_star(O):
    # FMT* expands one node at a time: 0, then 2 (tie with 3 broken by index;
    # 4<-2 fails), then 3 (1<-3, and 4<-3 along y = 0.1875 is free), then the
    # goal 4 is the cheapest open node: cost .375 < GMT*'s, the group effect.
    g, bl, bh = trace_b(O)
    parent, cost, info = g.plan(bl, bh, [0, 0], [1, 1], 0.5, which="fmt")
    assert info["goal_node"] == 4 and info["path_cost"] == 0.375 and parent[4] == 3
    assert (info["iters"], info["push_edges"], info["pull_edges"], info["checks"], info["failed"]) == (3, 7, 13, 5, 1)
    best, _ = g.dijkstra(bl, bh, [0, 0], [1, 1])
    assert best == 0.375


def test_no_path_when_goal_unreachable(O):
    g = graph2d(O, [(0, 0), (0.9, 0.9), (0.125, 0)], [1], 0.25)
    parent, cost, info = g.plan(NOBOX, NOBOX, [0, 0], [1, 1], 0.5)
    assert info["status"] == O.NO_PATH and info["goal_node"] == -1
    assert list(parent) == [-1, -1, 0] and np.isinf(cost[1])


def test_iteration_cap(O):
    g = graph2d(O, [(0, 0), (0.5, 0), (0.125, 0), (0, 0.1875), (0.3125, 0)], [1], 0.25)
    _, _, info = g.plan(NOBOX, NOBOX, [0, 0], [1, 1], 0.5, max_iters=3)
    assert info["status"] == O.ERR_ITER_LIMIT


# ---------------------------------------------------------------- properties
def problems():
    yield envgen.geometric(0, d=2, n=500, nbox=10, r=0.12)
    yield envgen.geometric(1, d=3, n=600, nbox=20, r=0.25)
    yield envgen.geometric(2, d=2, n=400, nbox=0, r=0.15)
    yield envgen.di6(seed=1, n=300, r=2.8)


def tree_invariants(O, pb, g, parent, cost, added, closed, lam):
    csr = g.csr()
    N = g.N
    delta = F(F(lam) * F(pb.r))
    for x in range(1, N):
        p = parent[x]
        if p < 0:
            assert np.isinf(cost[x])
            continue
        row = csr.in_col[csr.in_row[x]:csr.in_row[x + 1]]
        k = np.searchsorted(row, p)
        assert k < len(row) and row[k] == p, "tree edge must be a graph edge"
        e = csr.in_cost[csr.in_row[x] + k]
        assert cost[x] == F(cost[p] + e), "cost recurrence"
        assert g.edge_free(p, x, e, pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.seg_spacing,
                           pb.traj_points), "tree edge must be collision-free"
        assert added[p] < added[x], "a parent is open before its child is added"
    for v in range(N):
        if closed[v] >= 0:
            i = closed[v]
            assert F(F(i) * delta) >= cost[v]
            assert i - 1 <= added[v] or F(F(i - 1) * delta) < cost[v], "closes at the first eligible i"
            assert closed[v] > added[v]


def test_properties_on_random_instances(O):
    for pb in problems():
        X, goal = O.sample(pb)
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
        args = (pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp])
        best, dist = g.dijkstra(*args, pb.seg_spacing, pb.traj_points)
        for lam in (0.2, 0.5, 1.0):
            parent, cost, info, added, closed = g.plan(*args, lam, pb.seg_spacing, pb.traj_points, trace=True)
            p2, c2, i2 = g.plan(*args, lam, pb.seg_spacing, pb.traj_points, skip_empty=False)
            assert np.array_equal(parent, p2) and np.array_equal(cost, c2) and info == i2
            tree_invariants(O, pb, g, parent, cost, added, closed, lam)
            if info["status"] == O.OK:
                assert np.isfinite(best)
                assert info["path_cost"] >= best                       # Dijkstra is exact
                if pb.nbox == 0 and pb.kind == O.EUCLID:               # Theorem 2
                    assert info["path_cost"] <= (1 + 2 * lam) * best * (1 + 1e-6)
                path = O.path_to(parent, info["goal_node"])
                assert path[0] == 0 and goal[path[-1]] == 1
            else:
                assert info["status"] == O.NO_PATH
        # lambda = 0 is the FMT* limit
        pg, cg, ig = g.plan(*args, 0.0, pb.seg_spacing, pb.traj_points)
        pf, cf, i_f = g.plan(*args, 0.0, pb.seg_spacing, pb.traj_points, which="fmt")
        assert ig["status"] == i_f["status"]
        if ig["status"] == O.OK:
            assert ig["goal_node"] == i_f["goal_node"] and ig["path_cost"] == i_f["path_cost"]
            assert O.path_to(pg, ig["goal_node"]) == O.path_to(pf, i_f["goal_node"])
        in_fmt = np.isfinite(cf)
        assert np.array_equal(pg[in_fmt], pf[in_fmt]) and np.array_equal(cg[in_fmt], cf[in_fmt])


def test_oracle_dijkstra_matches_scipy(O):
    pb = envgen.geometric(4, d=2, n=250, nbox=8, r=0.15)
    X, goal = O.sample(pb)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
    csr = g.csr()
    rows, cols, w = [], [], []
    for y in range(g.N):
        for e in range(csr.out_row[y], csr.out_row[y + 1]):
            x = int(csr.out_col[e])
            if g.edge_free(y, x, csr.out_cost[e], pb.box_lo, pb.box_hi, pb.lo, pb.hi):
                rows.append(y); cols.append(x); w.append(float(csr.out_cost[e]))
    M = csr_matrix((w, (rows, cols)), shape=(g.N, g.N))
    ref = sp_dijkstra(M, directed=True, indices=0)
    best, dist = g.dijkstra(pb.box_lo, pb.box_hi, pb.lo, pb.hi)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(dist))
    assert np.allclose(dist[fin], ref[fin], rtol=1e-5)
    assert best == pytest.approx(np.min(ref[goal.astype(bool)]), rel=1e-5)


def test_fp64_rerun_close(O):
    pb = envgen.geometric(5, d=2, n=500, nbox=10, r=0.12)
    X, goal = O.sample(pb)
    args = (pb.box_lo, pb.box_hi, pb.lo, pb.hi, pb.lam)
    g32 = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
    g64 = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r, precision=64)
    p32, c32, i32 = g32.plan(*args)
    p64, c64, i64 = g64.plan(*args)
    if np.array_equal(p32, p64) and i32["status"] == O.OK:
        assert i32["path_cost"] == pytest.approx(i64["path_cost"], rel=1e-5)
    fin = np.isfinite(c32) & np.isfinite(c64) & (p32 == p64)
    assert np.allclose(c32[fin], c64[fin], rtol=1e-5)


def test_group_suboptimality_is_small(O):
    # Table 1 reports cost errors of GMT* vs FMT* of a few percent at
    # lambda = 0.5 in 2D/3D; a soft check of the magnitude on random boxes.
    errs = []
    for seed in range(4):
        pb = envgen.geometric(seed, d=2, n=1500, nbox=10, r=0.08)
        X, goal = O.sample(pb)
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
        args = (pb.box_lo, pb.box_hi, pb.lo, pb.hi)
        _, _, ig = g.plan(*args, 0.5)
        _, _, i_f = g.plan(*args, 0.5, which="fmt")
        if ig["status"] == O.OK and i_f["status"] == O.OK:
            errs.append(ig["path_cost"] / i_f["path_cost"] - 1)
    assert errs and np.mean(errs) < 0.1 and min(errs) > -0.1
