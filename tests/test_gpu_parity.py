"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer arrays (CSR, parents, counters) and every FP32 value (samples, edge
costs, tree costs) must match bit for bit: both sides evaluate the same IEEE
FP32 expressions in the same order without FMA.  Sizes: the 2D workload at its
full size (n = 1024) over many seeds; the 6D double integrator at its full size
(n = 4096) for a few seeds and at n = 600 for more; plus edge cases.
"""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    from paper_1705_02403_gb300 import planner
    return planner


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def gpu_run(P, pb, launch=None, build_only=False, **over):
    pl = P.Planner(pb).build()
    v = pl.view()
    out = {"X": v.X.cpu().numpy(), "goal": v.is_goal.cpu().numpy(), "E": v.E,
           "out_row": v.out_row.cpu().numpy(), "out_col": v.out_col.cpu().numpy(),
           "out_cost": v.out_cost.cpu().numpy(), "in_row": v.in_row.cpu().numpy(),
           "in_col": v.in_col.cpu().numpy(), "in_cost": v.in_cost.cpu().numpy(), "planner": pl}
    if build_only:
        return out
    if launch is not None:
        pl.set_launch(*launch)
    info = pl.plan(**over)
    out.update(parent=pl.parent.cpu().numpy(), cost=pl.cost.cpu().numpy(), info=info,
               path=pl.path.cpu().numpy()[:info["path_len"]])
    return out


def oracle_run(O, pb, X=None, goal=None, **kw):
    if X is None:
        X, goal = O.sample_halton(pb) if pb.sampler == 1 else O.sample(pb)
    r0 = O.radius_halton(pb.n, pb.d) if pb.sampler == 1 else O.radius_thm1(pb.n, pb.d)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r if pb.r > 0 else np.float32(r0), rho=pb.rho)
    parent, cost, info = g.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                                pb.traj_points, **kw)
    return X, goal, g, parent, cost, info


INFO_KEYS = ["status", "goal_node", "iters", "final_i", "push_edges", "pull_edges", "checks", "failed", "tree_size"]


def assert_same(O, G, X, goal, g, parent, cost, info, check_graph=True):
    assert np.array_equal(bits(G["X"]), bits(X)), "samples differ"
    assert np.array_equal(G["goal"], goal), "goal flags differ"
    if check_graph:
        c = g.csr()
        assert G["E"] == g.num_edges
        assert np.array_equal(G["out_row"], c.out_row) and np.array_equal(G["out_col"], c.out_col)
        assert np.array_equal(bits(G["out_cost"]), bits(c.out_cost))
        assert np.array_equal(G["in_row"], c.in_row) and np.array_equal(G["in_col"], c.in_col)
        assert np.array_equal(bits(G["in_cost"]), bits(c.in_cost))
    assert np.array_equal(G["parent"], parent), "parent arrays differ"
    assert np.array_equal(bits(G["cost"]), bits(cost)), "cost arrays differ"
    for k in INFO_KEYS:
        assert G["info"][k] == info[k], (k, G["info"][k], info[k])
    if info["status"] == O.OK:
        assert np.float32(G["info"]["path_cost"]) == np.float32(info["path_cost"])
        assert list(G["path"]) == O.path_to(parent, info["goal_node"])


def test_geometric_2d_full_size_many_seeds(O, P):
    for seed in range(40):
        pb = envgen.cfg1_2d(seed)
        G = gpu_run(P, pb)
        assert_same(O, G, *oracle_run(O, pb), check_graph=seed < 10)


def test_double_integrator_small_many_seeds(O, P):
    for seed in range(6):
        pb = envgen.di6(seed=seed, n=600, r=2.8)
        G = gpu_run(P, pb)
        assert_same(O, G, *oracle_run(O, pb))


def test_double_integrator_arrival_times(O, P):
    # The build stores each edge's arrival time tau*; it must be the oracle's
    # tau for that pair, bit for bit, on out- and in-edges.
    pb = envgen.di6(seed=7, n=500, r=2.8)
    G = gpu_run(P, pb, build_only=True)
    v = G["planner"].view()
    raw = v.raw
    from paper_1705_02403_gb300.planner import wrap_device
    out_tau = wrap_device(raw.out_tau, (v.E,), "f4", G["planner"].graph).cpu().numpy()
    in_tau = wrap_device(raw.in_tau, (v.E,), "f4", G["planner"].graph).cpu().numpy()
    X = G["X"]
    r = np.float32(pb.r)
    for y in range(0, pb.N, 7):
        for e in range(G["out_row"][y], G["out_row"][y + 1]):
            x = G["out_col"][e]
            J, tau = O.cost_di(X[:, y], X[:, x], r)
            assert bits(J) == bits(G["out_cost"][e]) and bits(tau) == bits(out_tau[e])
    for x in range(0, pb.N, 7):
        for e in range(G["in_row"][x], G["in_row"][x + 1]):
            y = G["in_col"][e]
            J, tau = O.cost_di(X[:, y], X[:, x], r)
            assert bits(tau) == bits(in_tau[e])


def test_double_integrator_full_size(O, P):
    for seed in (1, 2):
        pb = envgen.cfg2_di6(seed)
        G = gpu_run(P, pb)
        assert_same(O, G, *oracle_run(O, pb))


def csr_of(P, pb, flags):
    v = P.Planner(pb).build(debug_flags=flags).view()
    return {k: getattr(v, k).cpu().numpy() for k in ("out_row", "out_col", "out_cost", "in_row", "in_col", "in_cost")}


def same_csr(a, b):
    return all(np.array_equal(a[k] if "cost" not in k else bits(a[k]), b[k] if "cost" not in k else bits(b[k]))
               for k in a)


@pytest.mark.parametrize("case", ["2d_small_r", "2d_ragged", "3d_thm1", "3d_boxes", "2d_dense_fallback",
                                  "3d_dense_fallback", "2d_two_nodes", "2d_tiled_fill", "3d_tiled_fill"])
def test_cell_list_and_all_pairs_give_the_oracle_csr(O, P, case):
    # The 2D/3D geometric neighbour build picks a cell list when the radius is
    # small against the domain.  Forced either way, and with either way of
    # ordering a row (bitmap or sorted list), it must give the oracle's CSR bit
    # for bit; rows longer than the list (dense graphs) fall back to the
    # all-pairs test.  All-pairs builds of at least 4096 nodes fill the CSR
    # by mask tiles (per-tile prefixes), smaller ones row by row.
    from paper_1705_02403_gb300 import _native as N
    pb = {"2d_small_r": envgen.geometric(51, d=2, n=3000, nbox=8, r=0.03),
          "2d_ragged": envgen.geometric(52, d=2, n=1777, nbox=5, r=0.05),
          "3d_thm1": envgen.geometric(53, d=3, n=4000, nbox=12, r=0.0),
          "3d_boxes": envgen.geometric(54, d=3, n=2500, nbox=40, r=0.11),
          "2d_dense_fallback": DENSE[0],
          "3d_dense_fallback": DENSE[1],
          "2d_two_nodes": envgen.geometric(55, d=2, n=1, nbox=0, r=0.05),
          # all-pairs builds of at least 4096 nodes fill the CSR by mask tiles
          "2d_tiled_fill": envgen.geometric(57, d=2, n=6100, nbox=10, r=0.0),
          "3d_tiled_fill": envgen.geometric(58, d=3, n=4500, nbox=20, r=0.0)}[case]
    cells = csr_of(P, pb, N.GMT_DEBUG_PAIRS_CELLS)
    listed = csr_of(P, pb, N.GMT_DEBUG_PAIRS_CELLS | N.GMT_DEBUG_CELLS_LIST)
    pairs = csr_of(P, pb, N.GMT_DEBUG_PAIRS_ALL)
    auto = csr_of(P, pb, 0)
    assert same_csr(cells, pairs) and same_csr(listed, pairs) and same_csr(auto, pairs)
    X, goal = O.sample(pb)
    r = pb.r if pb.r > 0 else np.float32(O.radius_thm1(pb.n, pb.d))
    c = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r).csr()
    ref = {"out_row": c.out_row, "out_col": c.out_col, "out_cost": c.out_cost, "in_row": c.in_row,
           "in_col": c.in_col, "in_cost": c.in_cost}
    assert same_csr(cells, ref)


def test_double_integrator_filters_keep_every_edge_on_adversarial_states(O, P):
    # The pair filter tests every pair with conservative bounds before the exact
    # procedure.  States appended in tight families (tiny position changes,
    # equal or nearly equal velocities, slow motion, exact duplicates of the
    # position) stress the bounds where their margins are thinnest; the CSR must
    # still equal the oracle's, which evaluates the definition for every pair.
    import torch
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import GraphView, boxes_on_device, goal_struct, params_struct, space_struct
    pb = envgen.di6(seed=11, n=200, nbox=0, r=2.0)
    rng = np.random.default_rng(5)
    states = []
    for b in np.concatenate([rng.uniform(0.2, 0.8, (40, 3)), rng.uniform(-0.8, 0.8, (40, 3))], axis=1):
        for kind in range(10):
            s = b.copy()
            if kind in (0, 1, 2):
                s[:3] += rng.uniform(-1e-3, 1e-3, 3)
                s[3:] = rng.uniform(-1, 1, 3)
            elif kind in (3, 4):
                s[:3] += rng.uniform(-0.1, 0.1, 3)
                s[3:] += rng.uniform(-1e-4, 1e-4, 3)
            elif kind == 5:
                s[3:] = rng.uniform(-1, 1, 3)
            elif kind in (6, 7):
                s[:3] += rng.uniform(-0.05, 0.05, 3)
                s[3:] = rng.uniform(-0.02, 0.02, 3)
            else:
                s[:3] += rng.uniform(-1e-5, 1e-5, 3)
                s[3:] += rng.uniform(-1e-5, 1e-5, 3)
            states.append(np.clip(s, [0, 0, 0, -1, -1, -1], [1, 1, 1, 1, 1, 1]))
    extra = torch.tensor(np.array(states, np.float32).T.copy(), device="cuda")
    boxes, keep = boxes_on_device(pb)
    g = N.gmt_build_graph_ex(space_struct(pb), boxes, [float(v) for v in pb.x_init], goal_struct(pb), params_struct(pb),
                             extra.data_ptr(), len(states), len(states))
    v = GraphView(g)
    X, goal = v.X.cpu().numpy(), v.is_goal.cpu().numpy()
    og = O.Graph(pb.kind, pb.d, pb.dp, X, goal, np.float32(pb.r))
    c = og.csr()
    assert v.E == og.num_edges and v.E > 0
    assert np.array_equal(v.out_row.cpu().numpy(), c.out_row) and np.array_equal(v.out_col.cpu().numpy(), c.out_col)
    assert np.array_equal(bits(v.out_cost.cpu().numpy()), bits(c.out_cost))
    assert np.array_equal(v.in_row.cpu().numpy(), c.in_row) and np.array_equal(v.in_col.cpu().numpy(), c.in_col)
    assert np.array_equal(bits(v.in_cost.cpu().numpy()), bits(c.in_cost))


@pytest.mark.parametrize("launch", [(1, 1024), (1, 256), (2, 512), (7, 256), (0, 0), (152, 1024), (0, 1024, 2),
                                    (0, 512, 4), (0, 1024, 8), (0, 1024, 16)])
def test_every_launch_shape_gives_the_same_tree(O, P, launch):
    for pb in (envgen.cfg1_2d(5), envgen.di6(seed=3, n=600, r=2.8)):
        G = gpu_run(P, pb, launch=launch)
        assert_same(O, G, *oracle_run(O, pb), check_graph=False)


DENSE = [envgen.geometric(41, d=2, n=3000, nbox=4, r=1.3), envgen.geometric(42, d=3, n=2600, nbox=6, r=1.6)]


@pytest.fixture(scope="module")
def dense_oracle(O):
    return [oracle_run(O, pb) for pb in DENSE]


@pytest.mark.parametrize("launch", [(1, 256), (1, 1024), (0, 1024, 16), (4, 256)])
def test_nearly_complete_graphs(O, P, dense_oracle, launch):
    # Nearly complete graphs: one warp's push of x_init claims thousands of
    # candidates in the first iteration, and every in-row scan spans many
    # warp-wide chunks.
    for pb, ref in zip(DENSE, dense_oracle):
        G = gpu_run(P, pb, launch=launch)
        assert G["out_row"][1] - G["out_row"][0] > 2048
        assert_same(O, G, *ref, check_graph=False)


@pytest.mark.parametrize("case", ["2d", "3d_thm", "di6", "4d", "ragged_small"])
def test_halton_sampling_matches_the_oracle(O, P, case):
    # Halton SampleFree (the paper's sampler): samples, goal flags, CSR and tree
    # equal the oracle's; r = 0 selects the low-dispersion radius.
    pb = {"2d": envgen.geometric(71, d=2, n=2000, nbox=10, r=0.05),
          "3d_thm": envgen.geometric(72, d=3, n=3000, nbox=30, r=0.0),
          "di6": envgen.di6(seed=73, n=600, r=2.8),
          "4d": envgen.geometric(74, d=4, n=1500, nbox=6, r=0.0),
          "ragged_small": envgen.geometric(75, d=2, n=37, nbox=3, r=0.3)}[case].with_(sampler=1)
    G = gpu_run(P, pb)
    assert_same(O, G, *oracle_run(O, pb))


def test_halton_free_points_over_many_chunks(O, P):
    # The free Halton points are gathered over many blocks, a chunk of 256
    # points each, in the order of k.  A box over 64% of the square leaves
    # about one point in three free, so the blocks loop for more chunks; the
    # samples must still be the oracle's, node for node.
    from paper_1705_02403_gb300 import _native as N
    box = (np.array([[0.1, 0.1]], np.float32), np.array([[0.9, 0.9]], np.float32))
    pb = envgen.geometric(76, d=2, n=60000, nbox=0, r=0.004).with_(box_lo=box[0], box_hi=box[1], sampler=1)
    G = gpu_run(P, pb, build_only=True)
    X, goal = O.sample_halton(pb)
    assert np.array_equal(bits(G["X"]), bits(X)) and np.array_equal(G["goal"], goal)
    # n = 1 and 2: x_init and the goal node only, then one free point
    for n in (1, 2):
        pb = envgen.geometric(77, d=2, n=n, nbox=4, r=0.5).with_(sampler=1)
        G = gpu_run(P, pb, build_only=True)
        X, goal = O.sample_halton(pb)
        assert np.array_equal(bits(G["X"]), bits(X)) and np.array_equal(G["goal"], goal)
    # too few free points within the attempt cap: an error on both sides
    pb = envgen.geometric(78, d=2, n=5000, nbox=0, r=0.05).with_(
        box_lo=np.array([[0.001, 0.0]], np.float32), box_hi=np.array([[1.0, 1.0]], np.float32),
        x_init=np.array([0.0005, 0.5], np.float32), goal_center=np.array([0.0005, 0.9], np.float32),
        goal_radius=0.0004, sampler=1)
    with pytest.raises(ValueError):
        O.sample_halton(pb)
    with pytest.raises(N.GmtError) as e:
        P.Planner(pb).build()
    assert e.value.status == N.GMT_ERR_INVALID


@pytest.mark.parametrize("case", ["2d_600", "3d_300", "di_forest_1500", "2d_outside", "2d_big_and_degenerate"])
def test_many_boxes_use_the_box_grid(O, P, case):
    # From 128 boxes the plan and SampleFree list each box in the grid cells
    # it overlaps on the first two position axes (boxes over more than 32
    # cells in a list scanned for every point); samples and tree must stay the
    # oracle's.
    rng = np.random.default_rng(81)
    if case == "2d_600":
        pb = envgen.geometric(81, d=2, n=2000, nbox=0, r=0.06)
        bl, bh = envgen.random_boxes(rng, 600, 2, pb.x_init, pb.goal_center, 0.05, side=(0.005, 0.03))
    elif case == "3d_300":
        pb = envgen.geometric(82, d=3, n=2500, nbox=0, r=0.12)
        bl, bh = envgen.random_boxes(rng, 300, 3, pb.x_init, pb.goal_center, 0.05, side=(0.01, 0.06))
    elif case == "di_forest_1500":
        pb = envgen.di6(seed=83, n=700, nbox=0, r=2.8)
        bl, bh = envgen.forest_boxes(83, 10, 150)
    elif case == "2d_big_and_degenerate":
        # 200 small boxes (16 x 16 cells), 4 boxes over ~40 cells each (the
        # big-box list), zero-width boxes (lo == hi on an axis: they still hold
        # the points on them) and empty ones (lo > hi: they hold nothing)
        pb = envgen.geometric(85, d=2, n=2500, nbox=0, r=0.06)
        bl, bh = envgen.random_boxes(rng, 200, 2, pb.x_init, pb.goal_center, 0.05, side=(0.01, 0.04))
        big_lo = np.array([[0.2, 0.3], [0.55, 0.1], [0.1, 0.6], [0.5, 0.5]], np.float32)
        big_hi = big_lo + np.array([[0.38, 0.36], [0.36, 0.37], [0.35, 0.2], [0.37, 0.36]], np.float32)
        flat_lo = np.array([[0.3, 0.05], [0.05, 0.9]], np.float32)
        flat_hi = np.array([[0.3, 0.3], [0.4, 0.9]], np.float32)          # x == 0.3 and y == 0.9 segments
        empty_lo = np.array([[0.6, 0.6], [0.1, 0.2]], np.float32)
        empty_hi = np.array([[0.5, 0.9], [0.3, 0.1]], np.float32)
        bl = np.concatenate([bl, big_lo, flat_lo, empty_lo])
        bh = np.concatenate([bh, big_hi, flat_hi, empty_hi])
    else:  # boxes reaching outside the domain on both sides
        pb = envgen.geometric(84, d=2, n=1500, nbox=0, r=0.07)
        bl, bh = envgen.random_boxes(rng, 300, 2, pb.x_init, pb.goal_center, 0.05, side=(0.01, 0.05))
        bl = bl.copy(); bh = bh.copy()
        bl[:20] -= 0.3; bh[20:40] += 0.3
        keep = ~(np.all(bl <= pb.x_init, axis=1) & np.all(pb.x_init <= bh, axis=1))
        bl, bh = bl[keep], bh[keep]
    pb = pb.with_(box_lo=bl, box_hi=bh)
    assert pb.nbox >= 128
    G = gpu_run(P, pb)
    assert_same(O, G, *oracle_run(O, pb), check_graph=False)
    assert G["info"]["checks"] > 0


@pytest.mark.parametrize("d", [3, 4, 10])
def test_geometric_higher_dimensions(O, P, d):
    pb = envgen.geometric(seed=d, d=d, n=700, nbox=12, r={3: 0.3, 4: 0.45, 10: 1.0}[d])
    G = gpu_run(P, pb, launch=(4, 256))
    assert_same(O, G, *oracle_run(O, pb))


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_lambda_values(O, P, lam):
    pb = envgen.cfg1_2d(7).with_(lam=lam)
    assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))
    pb = envgen.di6(seed=4, n=500, r=2.8, lam=lam)
    assert_same(O, gpu_run(P, pb, launch=(3, 512)), *oracle_run(O, pb))


def test_edge_cases(O, P):
    # n = 1: x_init plus the goal sample only
    pb = envgen.geometric(1, d=2, n=1, nbox=3, r=0.12)
    assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))
    # no obstacles, ragged N (not a multiple of 32), Theorem 1 radius
    pb = envgen.geometric(2, d=2, n=777, nbox=0, r=0.0)
    assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))
    # x_init inside the goal ball: success at cost 0 after the first group
    pb = envgen.geometric(3, d=2, n=200, nbox=4, r=0.12).with_(x_init=np.array([0.94, 0.95], np.float32))
    G = gpu_run(P, pb)
    assert G["info"]["status"] == O.OK and G["info"]["path_cost"] == 0.0
    assert_same(O, G, *oracle_run(O, pb))
    # goal unreachable: a closed wall around the goal ball
    wall_lo = np.array([[0.8, 0.8]], np.float32)
    wall_hi = np.array([[1.0, 0.82]], np.float32)
    wall2_lo = np.array([[0.8, 0.8]], np.float32)
    wall2_hi = np.array([[0.82, 1.0]], np.float32)
    pb = envgen.geometric(4, d=2, n=400, nbox=0, r=0.12).with_(
        box_lo=np.concatenate([wall_lo, wall2_lo]), box_hi=np.concatenate([wall_hi, wall2_hi]))
    G = gpu_run(P, pb)
    assert G["info"]["status"] == O.NO_PATH
    assert_same(O, G, *oracle_run(O, pb))
    # many boxes: beyond what the plan kernel stages in shared memory
    rng = np.random.default_rng(0)
    c = rng.random((3000, 2)); s = rng.uniform(0.001, 0.004, (3000, 2))
    lo, hi = (c - s).astype(np.float32), (c + s).astype(np.float32)
    keep = ~(np.all((lo <= 0.05) & (0.05 <= hi), 1) | np.all((lo <= 1.0) & (0.9 <= hi), 1))
    pb = envgen.geometric(5, d=2, n=900, nbox=0, r=0.1).with_(box_lo=lo[keep], box_hi=hi[keep])
    assert_same(O, gpu_run(P, pb, launch=(8, 512)), *oracle_run(O, pb))


def test_iteration_cap(O, P):
    pb = envgen.cfg1_2d(0)
    G = gpu_run(P, pb, allow_errors=True, max_iters=3)
    assert G["info"]["status"] == -5


def test_bad_x_init_is_an_error(O, P):
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.cfg1_2d(0)
    c = (pb.box_lo[0] + pb.box_hi[0]) / 2
    with pytest.raises(N.GmtError) as e:
        P.Planner(pb.with_(x_init=c.astype(np.float32))).build()
    assert e.value.status == N.GMT_ERR_INVALID


def test_bounded_barrier_wait_times_out(O, P):
    # A barrier that waits for one CTA more than the grid has: every wait runs
    # out after spin_limit polls and the call returns GMT_ERR_TIMEOUT; the
    # context stays usable and the next plan is correct.
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.cfg1_2d(1)
    pl = P.Planner(pb).build()
    pl.set_launch(4, 256)
    info = pl.plan(allow_errors=True, debug_flags=N.GMT_DEBUG_UNREACHABLE_BARRIER, spin_limit=2000)
    assert info["status"] == N.GMT_ERR_TIMEOUT
    torch.cuda.synchronize()
    info = pl.plan()
    X, goal, g, parent, cost, oinfo = oracle_run(O, pb)
    assert np.array_equal(pl.parent.cpu().numpy(), parent) and info["goal_node"] == oinfo["goal_node"]


def test_fp64_rerun_within_1e5(O, P):
    # (i) every GPU tree node's cost, re-accumulated in FP64 along the GPU's own
    # parent pointers with FP64 edge costs, agrees to 1e-5 relative.
    # (ii) the full FP64 oracle: where its tree equals the FP32 one, the goal
    # costs agree to 1e-5.
    for pb in (envgen.cfg1_2d(2), envgen.di6(seed=2, n=600, r=2.8)):
        G = gpu_run(P, pb)
        X, parent, cost = G["X"], G["parent"], G["cost"]
        c64 = np.full(len(parent), np.inf)
        c64[0] = 0.0
        order = np.argsort(cost)
        for v in order:
            p = parent[v]
            if p < 0:
                continue
            if pb.kind == O.EUCLID:
                e = np.linalg.norm(X[:, v].astype(np.float64) - X[:, p].astype(np.float64))
            else:
                e, _ = O.cost_di_f64(X[:, p].astype(np.float64), X[:, v].astype(np.float64), 2 * pb.r, 64, 60)
            c64[v] = c64[p] + e
        fin = np.isfinite(cost)
        assert np.all(np.abs(cost[fin] - c64[fin]) <= 1e-5 * np.maximum(c64[fin], 1e-30))
        g64 = O.Graph(pb.kind, pb.d, pb.dp, X, G["goal"], pb.r, precision=64)
        p64, cst64, i64 = g64.plan(pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing,
                                   pb.traj_points)
        if np.array_equal(p64, parent) and i64["status"] == O.OK:
            assert abs(i64["path_cost"] - G["info"]["path_cost"]) <= 1e-5 * i64["path_cost"]


def test_asynchronous_builds(O, P):
    # gmt_build_graph_async on a reused handle: no host wait in the build; the
    # plan confirms the edge count.  A graph with more edges than the arrays of
    # earlier builds is rebuilt synchronously by the plan; a bad x_init is
    # reported by the plan; a view confirms the build too.  Every result equals
    # the synchronous build's and the oracle's.
    from paper_1705_02403_gb300 import _native as N
    small = envgen.di6(seed=31, n=300, r=2.4)
    big = envgen.di6(seed=32, n=900, r=2.8)
    geo = envgen.geometric(33, d=2, n=700, nbox=8, r=0.1)
    pl = P.Planner(small).build()                       # sizes the edge arrays (synchronous)
    for pb in (big, small, big):                        # grows past them, then fits, then fits
        pl.pb = pb
        pl.space, pl.goal, pl.params = P.space_struct(pb), P.goal_struct(pb), P.params_struct(pb)
        pl.boxes, pl._box_tensors = P.boxes_on_device(pb)
        pl.parent = torch.empty(pb.N, dtype=torch.int32, device="cuda")
        pl.cost = torch.empty(pb.N, dtype=torch.float32, device="cuda")
        pl.path = torch.empty(pb.N, dtype=torch.int32, device="cuda")
        pl.build(asynchronous=True)
        info = pl.plan()
        G = {"parent": pl.parent.cpu().numpy(), "cost": pl.cost.cpu().numpy(), "info": info,
             "path": pl.path.cpu().numpy()[:info["path_len"]]}
        v = pl.view()
        G.update(X=v.X.cpu().numpy(), goal=v.is_goal.cpu().numpy(), E=v.E, out_row=v.out_row.cpu().numpy(),
                 out_col=v.out_col.cpu().numpy(), out_cost=v.out_cost.cpu().numpy(), in_row=v.in_row.cpu().numpy(),
                 in_col=v.in_col.cpu().numpy(), in_cost=v.in_cost.cpu().numpy())
        assert_same(O, G, *oracle_run(O, pb))
    # the same with all-pairs geometric graphs filled by mask tiles (3D, at
    # least 4096 nodes): a growing graph is rebuilt by the plan, a smaller one fits
    t_small = envgen.geometric(35, d=3, n=4200, nbox=12, r=0.0)
    t_big = envgen.geometric(36, d=3, n=6000, nbox=12, r=0.0)
    pt = P.Planner(t_small).build()
    for pb in (t_big, t_small):
        pt.pb = pb
        pt.space, pt.goal, pt.params = P.space_struct(pb), P.goal_struct(pb), P.params_struct(pb)
        pt.boxes, pt._box_tensors = P.boxes_on_device(pb)
        pt.parent = torch.empty(pb.N, dtype=torch.int32, device="cuda")
        pt.cost = torch.empty(pb.N, dtype=torch.float32, device="cuda")
        pt.path = torch.empty(pb.N, dtype=torch.int32, device="cuda")
        pt.build(asynchronous=True)
        info = pt.plan()
        G = {"parent": pt.parent.cpu().numpy(), "cost": pt.cost.cpu().numpy(), "info": info,
             "path": pt.path.cpu().numpy()[:info["path_len"]]}
        v = pt.view()
        G.update(X=v.X.cpu().numpy(), goal=v.is_goal.cpu().numpy(), E=v.E, out_row=v.out_row.cpu().numpy(),
                 out_col=v.out_col.cpu().numpy(), out_cost=v.out_cost.cpu().numpy(), in_row=v.in_row.cpu().numpy(),
                 in_col=v.in_col.cpu().numpy(), in_cost=v.in_cost.cpu().numpy())
        assert_same(O, G, *oracle_run(O, pb))
    # a view right after an asynchronous build confirms it
    g2 = P.Planner(geo).build()
    g2.build(asynchronous=True)
    v = g2.view()
    ref = gpu_run(P, geo, build_only=True)
    assert v.E == ref["E"] and np.array_equal(v.out_col.cpu().numpy(), ref["out_col"])
    # x_init in a box: the plan reports what the synchronous build would have
    bad = big.with_(x_init=((big.box_lo[0] + big.box_hi[0]) / 2).tolist() + [0.0, 0.0, 0.0])
    pl.pb = bad
    pl.space, pl.goal, pl.params = P.space_struct(bad), P.goal_struct(bad), P.params_struct(bad)
    pl.build(asynchronous=True)
    with pytest.raises(N.GmtError) as e:
        pl.plan()
    assert e.value.status == N.GMT_ERR_INVALID



def _retarget(P, pl, pb):
    """Points a planner (and its graph handle) at another problem."""
    pl.pb = pb
    pl.space, pl.goal, pl.params = P.space_struct(pb), P.goal_struct(pb), P.params_struct(pb)
    pl.boxes, pl._box_tensors = P.boxes_on_device(pb)
    pl.parent = torch.empty(pb.N, dtype=torch.int32, device="cuda")
    pl.cost = torch.empty(pb.N, dtype=torch.float32, device="cuda")
    pl.path = torch.empty(pb.N, dtype=torch.int32, device="cuda")


def test_double_integrator_listed_edges(O, P):
    # A rebuild of a double-integrator graph on a handle whose edge arrays are
    # already sized takes its costs and arrival times from the pair filter's
    # edge list (placed by rank) instead of solving for them again, in the
    # synchronous and the asynchronous build; CSR, costs, arrival times and the
    # tree must equal the oracle's bit for bit.  The last problem has more
    # edges than the list holds: the synchronous rebuild then fills row by row.
    from paper_1705_02403_gb300.planner import wrap_device
    first = envgen.cfg2_di6(20)
    pl = P.Planner(first).build()
    cases = [(envgen.cfg2_di6(21), False), (envgen.cfg2_di6(22), True), (envgen.di6(seed=23, n=600, r=2.8), False),
             (envgen.di6(seed=24, n=4500, r=2.5), True)]
    for pb, asynchronous in cases:
        _retarget(P, pl, pb)
        pl.build(asynchronous=asynchronous)
        info = pl.plan()
        v = pl.view()
        G = {"parent": pl.parent.cpu().numpy(), "cost": pl.cost.cpu().numpy(), "info": info,
             "path": pl.path.cpu().numpy()[:info["path_len"]], "X": v.X.cpu().numpy(),
             "goal": v.is_goal.cpu().numpy(), "E": v.E, "out_row": v.out_row.cpu().numpy(),
             "out_col": v.out_col.cpu().numpy(), "out_cost": v.out_cost.cpu().numpy(),
             "in_row": v.in_row.cpu().numpy(), "in_col": v.in_col.cpu().numpy(), "in_cost": v.in_cost.cpu().numpy()}
        X, goal, g, parent, cost, oinfo = oracle_run(O, pb)
        assert_same(O, G, X, goal, g, parent, cost, oinfo)
        out_tau = wrap_device(v.raw.out_tau, (v.E,), "f4", pl.graph).cpu().numpy()
        in_tau = wrap_device(v.raw.in_tau, (v.E,), "f4", pl.graph).cpu().numpy()
        r = np.float32(pb.r)
        for y in range(0, pb.N, 97):
            for e in range(G["out_row"][y], G["out_row"][y + 1]):
                J, tau = O.cost_di(X[:, y], X[:, G["out_col"][e]], r)
                assert bits(tau) == bits(out_tau[e])
        for x in range(0, pb.N, 97):
            for e in range(G["in_row"][x], G["in_row"][x + 1]):
                J, tau = O.cost_di(X[:, G["in_col"][e]], X[:, x], r)
                assert bits(tau) == bits(in_tau[e])


def test_large_graph(O, P):
    # 40001 nodes in 2D (Theorem 1 radius, 5.4 M edges, about 100 group
    # expansions): the cell-list build, a wavefront over a large graph and the
    # path walk from global memory (the parent array exceeds the 48 KB of
    # shared memory); everything equals the oracle
    pb = envgen.geometric(91, d=2, n=40000, nbox=40, r=0.0)
    G = gpu_run(P, pb)
    assert G["E"] > 5_000_000 and G["info"]["iters"] > 50
    assert_same(O, G, *oracle_run(O, pb))
