"""GPU parity for the Dubins airplane (Sec. V-A): samples, the directed CSR
(out- and in-rows), every edge cost, the tree, the counters and the path must
equal the oracle's bit for bit (both sides evaluate the same FP32 expressions,
with their own trigonometry written out in the same order).  Workloads: the
forest analogue (full-height trunks) at the paper's n = 5000 and smaller,
Philox and Halton samples, few boxes (scanned) and many (box grid), tight and
wide turning radii, ragged and tiny graphs, every launch shape.
"""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen
from test_gpu_parity import assert_same, bits, gpu_run, oracle_run

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def P():
    from paper_1705_02403_gb300 import planner
    return planner


def test_forest_many_seeds(O, P):
    for seed in range(8):
        pb = envgen.dubins_forest(seed, n=1000, r=0.3)
        G = gpu_run(P, pb)
        ref = oracle_run(O, pb)
        assert G["E"] > 5 * pb.N
        assert_same(O, G, *ref)


def test_forest_full_size(O, P):
    # n = 5000 as in the paper's forest problem (Table 2), lambda = 1
    for seed in (0, 1):
        pb = envgen.dubins_forest(seed, n=5000)
        G = gpu_run(P, pb)
        assert_same(O, G, *oracle_run(O, pb))
        assert G["info"]["status"] == 0


@pytest.mark.parametrize("case", ["halton", "many_boxes", "tight_turns", "wide_turns", "lambda0", "lambda05"])
def test_variants(O, P, case):
    pb = {
        "halton": envgen.dubins_forest(2, n=2000, r=0.25, sampler=1),
        "many_boxes": envgen.dubins_forest(3, n=1500, r=0.3, strips=50),        # 500 boxes: box grid
        "tight_turns": envgen.dubins_forest(4, n=1200, r=0.25, rho=0.02),
        "wide_turns": envgen.dubins_forest(5, n=1200, r=0.35, rho=0.2),
        "lambda0": envgen.dubins_forest(6, n=900, r=0.3, lam=0.0),
        "lambda05": envgen.dubins_forest(7, n=900, r=0.3, lam=0.5),
    }[case]
    if case == "many_boxes":
        assert pb.nbox >= 128
    assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))


@pytest.mark.parametrize("launch", [(1, 1024), (1, 256), (7, 256), (0, 0), (152, 1024), (0, 1024, 4),
                                    (0, 1024, 16)])
def test_every_launch_shape(O, P, launch):
    pb = envgen.dubins_forest(9, n=1500, r=0.28)
    assert_same(O, gpu_run(P, pb, launch=launch), *oracle_run(O, pb), check_graph=False)


def test_small_and_ragged(O, P):
    for n in (1, 2, 31, 32, 33, 95):
        pb = envgen.dubins_forest(n, n=n, r=0.6, trunks=2)
        assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))
    # no obstacles at all: only the walls constrain the turns
    pb = envgen.dubins_forest(11, n=700, r=0.3, trunks=0)
    assert_same(O, gpu_run(P, pb), *oracle_run(O, pb))


def test_static_plan_on_a_dubins_view(O, P):
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.dubins_forest(12, n=1800, r=0.27)
    pl = P.Planner(pb).build()
    view = N.gmt_graph_get_view(pl.graph)
    assert view.turn_radius == np.float32(pb.rho) and view.out_tau is None
    parent = torch.full_like(pl.parent, -7)
    cost = torch.full_like(pl.cost, -7.0)
    info = N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, parent.data_ptr(), cost.data_ptr(), None).as_dict()
    torch.cuda.synchronize()
    X, goal, g, ref_parent, ref_cost, ref_info = oracle_run(O, pb)
    assert np.array_equal(parent.cpu().numpy(), ref_parent)
    assert np.array_equal(bits(cost.cpu().numpy()), bits(ref_cost))
    assert info["status"] == ref_info["status"] and info["goal_node"] == ref_info["goal_node"]
    # a view without the turning radius is refused
    view.turn_radius = 0.0
    with pytest.raises(N.GmtError) as e:
        N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, parent.data_ptr(), cost.data_ptr(), None)
    assert e.value.status == N.GMT_ERR_INVALID


def test_bad_arguments(O, P):
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.dubins_forest(0, n=200)
    for bad in (pb.with_(rho=0.0), pb.with_(r=0.0)):
        with pytest.raises(N.GmtError) as e:
            P.Planner(bad).build()
        assert e.value.status == N.GMT_ERR_INVALID
    # the batched path checks the same
    bp = P.BatchPlanner([pb, pb.with_(rho=0.0)])
    with pytest.raises(N.GmtError) as e:
        bp.plan()
    assert e.value.status == N.GMT_ERR_INVALID


def test_aligned_states_and_recomputed_words(O, P):
    # Families of states along their own heading (a straight path whose end
    # turns round to near-full loops and are taken as small negative turns),
    # near-duplicates and pure sideways offsets, appended to a sparse forest
    # sample set; the CSR (every cost), the stored words (through the plan's
    # checks) and a plan that recomputes the words must all equal the oracle.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import GraphView, boxes_on_device, goal_struct, params_struct, space_struct
    pb = envgen.dubins_forest(21, n=300, r=0.3, trunks=3)
    rng = np.random.default_rng(8)
    states = []
    for _ in range(60):
        b = np.array([*rng.uniform(0.15, 0.85, 3), rng.uniform(-3.1, 3.1)])
        for kind in range(8):
            s = b.copy()
            if kind < 4:        # along the heading, same heading
                u = rng.uniform(0.005, 0.2)
                s[0] += u * np.cos(b[3]); s[1] += u * np.sin(b[3]); s[2] += rng.uniform(-0.05, 0.05)
            elif kind < 6:      # near-duplicates
                s[:3] += rng.uniform(-1e-4, 1e-4, 3); s[3] += rng.uniform(-1e-4, 1e-4)
            else:               # sideways, same heading
                u = rng.uniform(-0.1, 0.1)
                s[0] -= u * np.sin(b[3]); s[1] += u * np.cos(b[3])
            s = np.clip(s, pb.lo, pb.hi).astype(np.float32)
            if not np.any(np.all((pb.box_lo <= s[:3]) & (s[:3] <= pb.box_hi), axis=1)):
                states.append(s)
    extra = torch.tensor(np.array(states, np.float32).T.copy(), device="cuda")
    boxes, keep = boxes_on_device(pb)
    params = params_struct(pb)
    g = N.gmt_build_graph_ex(space_struct(pb), boxes, [float(v) for v in pb.x_init], goal_struct(pb), params,
                             extra.data_ptr(), len(states), len(states))
    v = GraphView(g)
    X, goal = v.X.cpu().numpy(), v.is_goal.cpu().numpy()
    og = O.Graph(pb.kind, pb.d, pb.dp, X, goal, np.float32(pb.r), rho=pb.rho)
    c = og.csr()
    assert v.E == og.num_edges and v.E > 0
    assert np.array_equal(v.out_row.cpu().numpy(), c.out_row) and np.array_equal(v.out_col.cpu().numpy(), c.out_col)
    assert np.array_equal(bits(v.out_cost.cpu().numpy()), bits(c.out_cost))
    assert np.array_equal(v.in_row.cpu().numpy(), c.in_row) and np.array_equal(v.in_col.cpu().numpy(), c.in_col)
    assert np.array_equal(bits(v.in_cost.cpu().numpy()), bits(c.in_cost))
    # stored words: the oracle's shortest word for every in-edge
    raw = v.raw
    words = P.wrap_device(raw.in_path, (v.E, 4), "f4", g).cpu().numpy()
    wid = words[:, 3].copy().view(np.int32)
    neg = 0
    for x in range(v.N):
        for e in range(c.in_row[x], c.in_row[x + 1]):
            y = int(c.in_col[e])
            ref, best = O.dubins_words(X[:, y], X[:, x], pb.rho, precision=32)
            assert wid[e] == best and np.array_equal(bits(words[e, :3]), bits(ref[best, 1:4]))
            neg += int(ref[best, 1] < 0 or ref[best, 3] < 0)
    assert neg > 0, "some stored words carry a negative end turn"
    # plans: stored words (gmt_plan) and recomputed ones (a view without them)
    n_total = v.N
    parent = torch.empty(n_total, dtype=torch.int32, device="cuda")
    cost = torch.empty(n_total, dtype=torch.float32, device="cuda")
    ref_parent, ref_cost, ref_info = og.plan(pb.box_lo, pb.box_hi, pb.lo[:3], pb.hi[:3], pb.lam, pb.seg_spacing)
    for recompute in (False, True):
        view = N.gmt_graph_get_view(g)
        if recompute:
            view.in_path = None
            info = N.gmt_plan_static(space_struct(pb), view, boxes, params, parent.data_ptr(), cost.data_ptr(),
                                     None).as_dict()
        else:
            info = N.gmt_plan(g, boxes, params, parent.data_ptr(), cost.data_ptr(), None).as_dict()
        torch.cuda.synchronize()
        assert np.array_equal(parent.cpu().numpy(), ref_parent)
        assert np.array_equal(bits(cost.cpu().numpy()), bits(ref_cost))
        assert info["checks"] == ref_info["checks"] and info["failed"] == ref_info["failed"]


def test_rebuilds_take_listed_words(O, P):
    # Rebuilds on a handle whose edge arrays are already sized take each edge's
    # cost and shortest word from the pair filter's list (placed by rank), in
    # the synchronous and the asynchronous build; a graph with more edges than
    # the list holds is rebuilt row by row.  CSR, stored words, tree and path
    # must equal the oracle's.
    from test_gpu_parity import _retarget
    pl = P.Planner(envgen.dubins_forest(30, n=1500, r=0.3)).build()
    for pb, asynchronous in ((envgen.dubins_forest(31, n=1500, r=0.3), False),
                             (envgen.dubins_forest(32, n=1400, r=0.3), True),
                             (envgen.dubins_forest(33, n=2500, r=0.35), True)):
        _retarget(P, pl, pb)
        pl.build(asynchronous=asynchronous)
        info = pl.plan()
        v = pl.view()
        G = {"parent": pl.parent.cpu().numpy(), "cost": pl.cost.cpu().numpy(), "info": info,
             "path": pl.path.cpu().numpy()[:info["path_len"]], "X": v.X.cpu().numpy(),
             "goal": v.is_goal.cpu().numpy(), "E": v.E, "out_row": v.out_row.cpu().numpy(),
             "out_col": v.out_col.cpu().numpy(), "out_cost": v.out_cost.cpu().numpy(),
             "in_row": v.in_row.cpu().numpy(), "in_col": v.in_col.cpu().numpy(), "in_cost": v.in_cost.cpu().numpy()}
        ref = oracle_run(O, pb)
        assert_same(O, G, *ref)
        X = G["X"]
        words = P.wrap_device(v.raw.in_path, (v.E, 4), "f4", pl.graph).cpu().numpy()
        wid = words[:, 3].copy().view(np.int32)
        for x in range(0, pb.N, 37):
            for e in range(G["in_row"][x], G["in_row"][x + 1]):
                y = int(G["in_col"][e])
                w, best = O.dubins_words(X[:, y], X[:, x], pb.rho, precision=32)
                assert wid[e] == best and np.array_equal(bits(words[e, :3]), bits(w[best, 1:4]))
