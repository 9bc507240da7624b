"""gmt_plan_static, the allocation-free plan entry point, against gmt_plan.

Callers that must not allocate device memory while planning (a replanning loop
inside a control cycle, where an allocation can stall the device; systems
whose memory is fixed at start-up) use gmt_plan_static: the same wavefront
kernel, with its scratch in a fixed array inside the library.  Its results must
equal gmt_plan's bit for bit, on consecutive calls that share that array, up to
graphs that fill the array; and calls after the first on a device must not
change the device's free memory or the caching allocator's counts.
"""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def plan_both(pb, drop_tau=False):
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import Planner
    pl = Planner(pb).build()
    ref = pl.plan()
    ref_parent, ref_cost, ref_path = pl.parent.clone(), pl.cost.clone(), pl.path.clone()
    view = N.gmt_graph_get_view(pl.graph)
    if drop_tau:
        view.in_tau = view.out_tau = None   # the kernel recomputes arrival times
    parent = torch.full_like(ref_parent, -7)
    cost = torch.full_like(ref_cost, -7.0)
    path = torch.full_like(ref_path, -7)
    info = N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, parent.data_ptr(), cost.data_ptr(),
                             path.data_ptr()).as_dict()
    torch.cuda.synchronize()
    return ref, ref_parent, ref_cost, ref_path, info, parent, cost, path


def test_static_plan_equals_gmt_plan_on_consecutive_calls():
    # First call: 6D double integrator, N = 4097 (multi-CTA grid, barrier words
    # in the static array); second call: 2D, N = 1025 (one CTA), which must not
    # see anything left over from the first; third: a view without the stored
    # arrival times.
    for pb, drop in ((envgen.cfg2_di6(1), False), (envgen.cfg1_2d(3), False), (envgen.di6(2, n=700, r=2.8), True)):
        ref, rp, rc, rpath, info, parent, cost, path = plan_both(pb, drop)
        assert torch.equal(parent, rp)
        assert torch.equal(cost.view(torch.int32), rc.view(torch.int32))   # bit for bit
        n = ref["path_len"]
        assert info["path_len"] == n and torch.equal(path[:n], rpath[:n])
        for k in ("status", "goal_node", "path_cost", "iters", "final_i", "push_edges", "pull_edges", "checks",
                  "failed", "tree_size"):
            assert info[k] == ref[k], k


def test_static_plan_on_large_graphs_and_without_allocation():
    # A 2D graph of about 20000 nodes (its parent array no longer fits the
    # shared memory that the path walk reads it from) and one close to the
    # 65536-node limit, which uses nearly all of the fixed array.
    from paper_1705_02403_gb300 import _native as N
    for n in (20000, 65000):
        pb = envgen.geometric(seed=11, d=2, n=n, nbox=20, r=0.0)
        ref, rp, rc, rpath, info, parent, cost, path = plan_both(pb)
        assert torch.equal(parent, rp)
        assert torch.equal(cost.view(torch.int32), rc.view(torch.int32))
        for k in ("status", "goal_node", "iters", "push_edges", "pull_edges", "checks", "tree_size"):
            assert info[k] == ref[k], k
    # repeated calls allocate nothing: free device memory and the caching
    # allocator's counters are unchanged (outputs allocated beforehand)
    from paper_1705_02403_gb300.planner import Planner
    pl = Planner(envgen.cfg2_di6(4)).build()
    view = N.gmt_graph_get_view(pl.graph)
    parent = torch.empty_like(pl.parent)
    cost = torch.empty_like(pl.cost)
    N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, parent.data_ptr(), cost.data_ptr(), None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, parent.data_ptr(), cost.data_ptr(), None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = torch.cuda.memory_stats()
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k


def test_static_plan_rejects_graphs_beyond_capacity():
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import Planner
    pl = Planner(envgen.cfg1_2d(0)).build()
    view = N.gmt_graph_get_view(pl.graph)
    view.N = 65537
    info = N.gmt_plan_static(pl.space, view, pl.boxes, pl.params, pl.parent.data_ptr(), pl.cost.data_ptr(),
                             None, allow_errors=True)
    assert info.rc == N.GMT_ERR_INVALID
    assert "65536" in N.gmt_last_error()
