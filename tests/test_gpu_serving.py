"""The replanning server: every served tree equals the CPU oracle's plan on the
session's samples with that request's boxes (and start), bit for bit, with the
verdict cache warm; it is also the same alone and in a mix of overlapping
requests (geometric, double-integrator and Dubins-airplane sessions with moving
boxes); sessions are admitted by device memory, and the verdict cache only
recomputes what moved boxes can change."""
import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def structs(pb):
    from paper_1705_02403_gb300.planner import goal_struct, params_struct, space_struct
    return space_struct(pb), goal_struct(pb), params_struct(pb)


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def oracle_graph(O, pb):
    """The oracle's samples and r-disk graph of a session's problem (the
    samples are drawn against the boxes the session was opened with)."""
    X, goal = O.sample_halton(pb) if pb.sampler == 1 else O.sample(pb)
    return O.graph_for(pb, X, goal)


def session_samples(server, sid):
    from paper_1705_02403_gb300.planner import wrap_device
    v = server.session_view(sid)
    return wrap_device(v.X, (v.dim, v.x_pitch), "f4", server)[:, :v.N].cpu().numpy()


def assert_oracle(O, g, pb, lo, hi, r, parent, cost):
    """A served result against the oracle's plan with the request's boxes."""
    op, oc, oi = g.plan(lo, hi, pb.lo[:pb.dp], pb.hi[:pb.dp], pb.lam, pb.seg_spacing, pb.traj_points)
    assert r["status"] == oi["status"] and r["goal_node"] == oi["goal_node"]
    assert np.array_equal(parent.cpu().numpy(), op), "served parents differ from the oracle's"
    assert np.array_equal(bits(cost.cpu().numpy()), bits(oc)), "served costs differ from the oracle's"
    assert r["iters"] == oi["iters"] and r["checks"] == oi["checks"]
    assert r["edges_checked"] == oi["push_edges"] + oi["pull_edges"]
    if oi["status"] == O.OK:
        assert np.float32(r["path_cost"]) == np.float32(oi["path_cost"])


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


def test_same_alone_and_in_the_mix(O):
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
    graphs = [oracle_graph(O, pb) for pb in pbs]
    for k, (pb, sid) in enumerate(zip(pbs, sids)):   # resident samples are the oracle's
        assert np.array_equal(bits(session_samples(server, sid)), bits(graphs[k].X))
    warm = 0
    for rid_, k, lo, hi, parent, cost in reqs:
        r = res[rid_]
        assert_oracle(O, graphs[k], pbs[k], lo, hi, r, parent, cost)
        warm += r["checks_computed"] < r["checks"]
        info, p2, c2 = alone(server, sids[k], pbs[k], lo, hi)
        assert r["status"] == info["status"] and r["goal_node"] == info["goal_node"]
        assert torch.equal(parent, p2)
        assert torch.equal(cost.view(torch.int32), c2.view(torch.int32))
        if info["status"] == 0:
            assert r["path_cost"] == info["path_cost"]
    assert warm > 0   # later ticks answered checks from the verdict cache
    server.close()


def test_admission_by_device_memory():
    # An 80 MiB budget holds two sessions of n = 2000 (each estimated at about
    # 33 MB: bit matrices and their word prefixes plus CSR and edge-list space
    # for up to 256 edges per node); the third is refused with
    # GMT_ERR_ADMISSION, and fits again after a close.
    from paper_1705_02403_gb300 import _native as N
    pbs = [envgen.di6(seed=20 + k, n=2000, r=2.6) for k in range(4)]
    server = N.Server(slots=1, cluster=0, max_nodes=2001, max_boxes=30, memory_budget=80 << 20)
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


def test_verdict_cache_reuse(O):
    from paper_1705_02403_gb300 import _native as N
    pb = envgen.di6(seed=9, n=1500, r=2.6)
    g = oracle_graph(O, pb)
    server = N.Server(slots=2, cluster=2, max_nodes=1501, max_boxes=30)
    sid, _ = server.open_session(*structs(pb)[:1], pb.x_init, *structs(pb)[1:], pb.box_lo, pb.box_hi)

    def request(rid, lo, hi):
        parent = torch.full((pb.N,), -7, dtype=torch.int32, device="cuda")
        cost = torch.full((pb.N,), -7.0, dtype=torch.float32, device="cuda")
        server.submit(sid, rid, lo, hi, parent.data_ptr(), cost.data_ptr())
        r = server.poll(4, 5000)[0]
        torch.cuda.synchronize()
        assert_oracle(O, g, pb, lo, hi, r, parent, cost)
        return r

    r0 = request(0, pb.box_lo, pb.box_hi)
    r1 = request(1, pb.box_lo, pb.box_hi)                # nothing moved: every check is cached
    assert r1["checks_computed"] == 0 and r1["checks"] == r0["checks"] and r1["path_cost"] == r0["path_cost"]
    lo, hi = pb.box_lo.copy(), pb.box_hi.copy()
    lo[0] += 0.3; hi[0] += 0.3                           # one box moves
    lo[0] = np.clip(lo[0], 0, 0.9); hi[0] = np.clip(hi[0], 0.05, 1.0)
    r2 = request(2, lo, hi)
    assert 0 < r2["checks_computed"] < r2["checks"]
    server.close()


@pytest.mark.parametrize("kind", ["di", "dubins"])
def test_start_move_rebuilds_the_session(O, kind):
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
    assert_oracle(O, oracle_graph(O, pb), pb, lo1, hi1, r, parent, cost)   # still the first start's graph
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
    # the rebuilt session: the same seed drawn at the new start against the
    # boxes of its last request
    moved = pb.with_(x_init=x_new, box_lo=lo1, box_hi=hi1)
    g_new = oracle_graph(O, moved)
    fresh = Planner(moved).build()
    for rid in (2, 3):
        lo, hi = mover.step()
        r, parent, cost = request(rid, lo, hi)
        assert_oracle(O, g_new, moved, lo, hi, r, parent, cost)
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
