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
    # the batched path covers geometric and double-integrator queries only
    bp = P.BatchPlanner([pb])
    with pytest.raises(N.GmtError) as e:
        bp.plan()
    assert e.value.status == N.GMT_ERR_INVALID
