"""The sweep driver runs end to end on the GPU (small sizes): every Table 1
cell reports a cost error for the runs both arms solve; on small cells of
Table 1 each arm's plans equal the CPU oracle's (lambda = 0 against the
oracle's heap FMT*, lambda > 0 against its GMT*), bit for bit on the goal node
and its cost, and the reported cost errors are the oracle's."""
import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_table1_small():
    from paper_1705_02403_gb300 import sweeps
    rows = sweeps.table1(runs=3, n=400, log=None)
    assert len(rows) == 6
    for row in rows:
        for lam in ("0.2", "0.5", "1.0"):
            e = row["cost_error"][lam]
            assert e is None or (np.isfinite(e) and e > -0.5)


@pytest.mark.parametrize("env,d", [("rectangles", 2), ("maze", 3), ("rectangles", 6)])
def test_table1_cells_rest_on_the_oracle(O, env, d):
    from paper_1705_02403_gb300 import envgen, sweeps
    runs, n = 3, 400
    row = [r for r in sweeps.table1(runs=runs, n=n, log=None) if r["env"] == env and r["d"] == d][0]
    errs = {lam: [] for lam in sweeps.LAMBDAS}
    for seed in range(runs):
        pb = envgen.rectangles(seed, d, n) if env == "rectangles" else envgen.maze(seed, d, n)
        X, goal = O.sample(pb)
        r = np.float32(O.radius_thm1(pb.n, pb.d))
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r)
        args = (pb.box_lo, pb.box_hi, pb.lo[:pb.dp], pb.hi[:pb.dp])
        _, _, fmt = g.plan(*args, 0.0, pb.seg_spacing, pb.traj_points, which="fmt")
        _, _, gmt0 = g.plan(*args, 0.0, pb.seg_spacing, pb.traj_points)
        # the lambda -> 0 limit of GMT* is FMT*: same goal node and cost
        assert (gmt0["status"], gmt0["goal_node"]) == (fmt["status"], fmt["goal_node"])
        if fmt["status"] != O.OK:
            continue
        assert np.float32(gmt0["path_cost"]) == np.float32(fmt["path_cost"])
        for lam in sweeps.LAMBDAS:
            _, _, info = g.plan(*args, lam, pb.seg_spacing, pb.traj_points)
            if info["status"] == O.OK:
                errs[lam].append(float(np.float32(info["path_cost"])) / float(np.float32(fmt["path_cost"])) - 1.0)
    for lam in sweeps.LAMBDAS:
        got = row["cost_error"][str(lam)]
        assert row["gmt_solved"][str(lam)] == len(errs[lam])
        if errs[lam]:
            assert got == pytest.approx(float(np.mean(errs[lam])), rel=1e-9, abs=1e-12), lam
        else:
            assert got is None


def test_table3_small():
    from paper_1705_02403_gb300 import sweeps
    rows = sweeps.table3(runs=2, log=None)
    assert [r["boxes"] for r in rows] == [300, 300, 300, 300, 150, 500, 1500, 5000]
    assert all(r["plan_ms_p50"] > 0 and r["build_ms_p50"] > 0 for r in rows)


def test_table3_dubins_small():
    from paper_1705_02403_gb300 import sweeps
    rows = sweeps.table3_dubins(runs=1, log=None)
    assert [(r["n"], r["boxes"]) for r in rows] == [(5000, 150), (5000, 500), (5000, 1500), (5000, 5000),
                                                    (10000, 150)]
    assert all(r["plan_ms_p50"] > 0 and r["build_ms_p50"] > 0 for r in rows)
    assert all(r["success"] == 1.0 for r in rows)
