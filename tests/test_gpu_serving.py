"""The replanning server: every request's tree is the same alone and in a mix
of overlapping requests (bit for bit, verdict cache included; geometric,
double-integrator and Dubins-airplane sessions with moving boxes), sessions are
admitted by device memory, and the verdict cache only recomputes what moved
boxes can change."""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def structs(pb):
    from paper_1705_02403_gb300.planner import goal_struct, params_struct, space_struct
    return space_struct(pb), goal_struct(pb), params_struct(pb)


def alone(server, sid, pb, lo, hi):
    """The same request planned by itself: gmt_plan_static on the session's
    resident graph, with the boxes of that request, and no verdict cache."""
    from paper_1705_02403_gb300 import _native as N
    sp, g, p = structs(pb)
    v = server.session_view(sid)
    dlo = torch.tensor(np.asarray(lo, np.float32), device="cuda")
    dhi = torch.tensor(np.asarray(hi, np.float32), device="cuda")
    b = N.gmt_boxes(); b.count = dlo.shape[0]; b.lo = dlo.data_ptr(); b.hi = dhi.data_ptr()
    parent = torch.empty(v.N, dtype=torch.int32, device="cuda")
    cost = torch.empty(v.N, dtype=torch.float32, device="cuda")
    info = N.gmt_plan_static(sp, v, b, p, parent.data_ptr(), cost.data_ptr(), None).as_dict()
    return info, parent, cost


def test_same_alone_and_in_the_mix():
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.serving import MovingBoxes
    pbs = [envgen.di6(seed=1, n=700, r=2.8), envgen.geometric(2, d=2, n=900, nbox=10, r=0.12),
           envgen.di6(seed=3, n=1200, r=2.6), envgen.geometric(4, d=3, n=800, nbox=12, r=0.3),
           envgen.di6(seed=5, n=2500, r=2.5),
           envgen.dubins_forest(6, n=800, r=0.3, trunks=3, strips=10),
           envgen.dubins_forest(7, n=1500, r=0.28, trunks=2, strips=15, sampler=1)]
    server = N.Server(slots=3, cluster=2, threads=512, max_nodes=2501, max_boxes=30)
    sids = [server.open_session(*structs(pb)[:1], pb.x_init, *structs(pb)[1:], pb.box_lo, pb.box_hi)[0] for pb in pbs]
    movers = [MovingBoxes(pb, k, vmax=0.05) if pb.dp == 3 else None for k, pb in enumerate(pbs)]
    reqs, outs = [], {}
    rid = 0
    for tick in range(4):
        for k, (pb, sid) in enumerate(zip(pbs, sids)):
            if movers[k] is not None:
                lo, hi = movers[k].step()
            else:
                lo, hi = pb.box_lo + 0.01 * tick, pb.box_hi + 0.01 * tick
            parent = torch.full((pb.N,), -7, dtype=torch.int32, device="cuda")
            cost = torch.full((pb.N,), -7.0, dtype=torch.float32, device="cuda")
            server.submit(sid, rid, lo, hi, parent.data_ptr(), cost.data_ptr())
            reqs.append((rid, k, lo.copy(), hi.copy(), parent, cost))
            rid += 1
    res = {}
    while len(res) < rid:
        for r in server.poll(64, 200):
            res[r["request_id"]] = r
    torch.cuda.synchronize()
    overlapped = sum(r["queue_ms"] > 0.0 for r in res.values())
    assert overlapped > 0
    for rid_, k, lo, hi, parent, cost in reqs:
        r = res[rid_]
        info, p2, c2 = alone(server, sids[k], pbs[k], lo, hi)
        assert r["status"] == info["status"] and r["goal_node"] == info["goal_node"]
        assert torch.equal(parent, p2)
        assert torch.equal(cost.view(torch.int32), c2.view(torch.int32))
        if info["status"] == 0:
            assert r["path_cost"] == info["path_cost"]
    server.close()


def test_admission_by_device_memory():
    # A 60 MB budget holds two sessions of n = 2000 (each estimated at about
    # 24 MB: bit matrices plus CSR space for up to 256 edges per node); the
    # third is refused with GMT_ERR_ADMISSION, and fits again after a close.
    from paper_1705_02403_gb300 import _native as N
    pbs = [envgen.di6(seed=20 + k, n=2000, r=2.6) for k in range(4)]
    server = N.Server(slots=1, cluster=0, max_nodes=2001, max_boxes=30, memory_budget=60 << 20)
    opened = []
    for pb in pbs[:3]:
        sid, st = server.open_session(*structs(pb)[:1], pb.x_init, *structs(pb)[1:], pb.box_lo, pb.box_hi,
                                      allow_errors=True)
        if sid is not None:
            opened.append(sid)
        else:
            assert st == N.GMT_ERR_ADMISSION
    assert len(opened) == 2
    server.close_session(opened[0])
    sid, st = server.open_session(*structs(pbs[3])[:1], pbs[3].x_init, *structs(pbs[3])[1:], pbs[3].box_lo,
                                  pbs[3].box_hi, allow_errors=True)
    assert sid is not None and st == N.GMT_OK
    server.close()


def test_verdict_cache_reuse():
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.di6(seed=9, n=1500, r=2.6)
    server = N.Server(slots=2, cluster=2, max_nodes=1501, max_boxes=30)
    sid, _ = server.open_session(*structs(pb)[:1], pb.x_init, *structs(pb)[1:], pb.box_lo, pb.box_hi)
    server.submit(sid, 0, pb.box_lo, pb.box_hi)
    r0 = server.poll(4, 5000)[0]
    server.submit(sid, 1, pb.box_lo, pb.box_hi)          # nothing moved: every check is cached
    r1 = server.poll(4, 5000)[0]
    assert r1["checks_computed"] == 0 and r1["checks"] == r0["checks"] and r1["path_cost"] == r0["path_cost"]
    lo, hi = pb.box_lo.copy(), pb.box_hi.copy()
    lo[0] += 0.3; hi[0] += 0.3                           # one box moves
    lo[0] = np.clip(lo[0], 0, 0.9); hi[0] = np.clip(hi[0], 0.05, 1.0)
    server.submit(sid, 2, lo, hi)
    r2 = server.poll(4, 5000)[0]
    assert 0 < r2["checks_computed"] < r2["checks"]
    info, _, _ = alone(server, sid, pb, lo, hi)
    assert r2["status"] == info["status"] and r2["goal_node"] == info["goal_node"]
    server.close()


@pytest.mark.parametrize("kind", ["di", "dubins"])
def test_start_move_rebuilds_the_session(kind):
    # After gmt_server_move_start the session plans exactly as a graph built
    # fresh at the new start (same seed, the boxes of its last request) and
    # planned with the request's boxes; a move into a box is refused and the
    # session keeps planning on its previous graph.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300.planner import Planner, boxes_on_device
    from paper_1705_02403_gb300.serving import MovingBoxes
    pb = envgen.di6(seed=8, n=900, r=2.8) if kind == "di" else envgen.dubins_forest(8, n=900, r=0.3, trunks=3,
                                                                                      strips=10)
    server = N.Server(slots=2, cluster=2, threads=512, max_nodes=pb.N, max_boxes=pb.nbox)
    sid, _ = server.open_session(*structs(pb)[:1], pb.x_init, *structs(pb)[1:], pb.box_lo, pb.box_hi)
    mover = MovingBoxes(pb, 3, vmax=0.03)

    def request(rid, lo, hi):
        parent = torch.full((pb.N,), -7, dtype=torch.int32, device="cuda")
        cost = torch.full((pb.N,), -7.0, dtype=torch.float32, device="cuda")
        server.submit(sid, rid, lo, hi, parent.data_ptr(), cost.data_ptr())
        while True:
            got = server.poll(8, 200)
            if got:
                assert len(got) == 1 and got[0]["request_id"] == rid
                torch.cuda.synchronize()
                return got[0], parent, cost

    lo1, hi1 = mover.step()
    request(0, lo1, hi1)
    # a start inside one of the current boxes is refused
    inside = (lo1[0] + hi1[0]) / 2
    x_bad = pb.x_init.copy()
    x_bad[:3] = inside[:3]
    with pytest.raises(N.GmtError) as e:
        server.move_start(sid, x_bad)
    assert e.value.status == N.GMT_ERR_INVALID
    r, parent, cost = request(1, lo1, hi1)
    info, p2, c2 = alone(server, sid, pb, lo1, hi1)
    assert torch.equal(parent, p2) and torch.equal(cost.view(torch.int32), c2.view(torch.int32))
    # a valid move, then requests with moving boxes
    x_new = None
    for cand in ([0.03, 0.04, 0.3], [0.1, 0.03, 0.2], [0.04, 0.12, 0.1], [0.2, 0.05, 0.05]):
        c = np.array(cand, np.float32)
        if not np.any(np.all((lo1 <= c) & (c <= hi1), axis=1)):
            x_new = pb.x_init.copy()
            x_new[:3] = c
            break
    assert x_new is not None
    server.move_start(sid, x_new)
    fresh = Planner(pb.with_(x_init=x_new, box_lo=lo1, box_hi=hi1)).build()
    for rid in (2, 3):
        lo, hi = mover.step()
        r, parent, cost = request(rid, lo, hi)
        b, keep = boxes_on_device(pb.with_(box_lo=lo, box_hi=hi))
        fresh.boxes = b
        ref = fresh.plan()
        torch.cuda.synchronize()
        assert r["status"] == ref["status"] and r["goal_node"] == ref["goal_node"]
        assert torch.equal(parent, fresh.parent)
        assert torch.equal(cost.view(torch.int32), fresh.cost.view(torch.int32))
    v = server.session_view(sid)
    assert v.X is not None
    server.close()
