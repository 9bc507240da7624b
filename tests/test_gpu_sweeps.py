"""The sweep driver runs end to end on the GPU (small sizes): every Table 1
cell reports a cost error for the runs both arms solve, and the lambda = 0 arm
is the FMT* limit, so no error is below the rounding of a path cost."""
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
