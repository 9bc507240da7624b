"""The learned proposal on the GPU: tensor-core forward/backward against the
CPU MLP oracle (same BF16 rounding points), the voxeliser and path histogram
against numpy, the proposal sampler's samples and distribution, training and
checkpoints."""
import os
import tempfile

import numpy as np
import pytest
import torch

from paper_1705_02403_gb300 import envgen

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

G, H, C = 32, 512, 16


def dev(ptr, shape, dtype, owner):
    from paper_1705_02403_gb300.planner import wrap_device
    return wrap_device(ptr, shape, dtype, owner)


def model_params(m):
    v = m.view()
    Din, Dz, Nc = v.in_features, v.z_features, v.n_cells
    f = lambda p, shape: dev(p, shape, "f4", m).cpu().numpy().astype(np.float32)
    P = {"W1": f(v.W1, (v.hidden, Din)), "b1": f(v.b1, (v.hidden,)), "W2": f(v.W2, (v.hidden, v.hidden)),
         "b2": f(v.b2, (v.hidden,)), "W3": f(v.W3, (Nc, Dz)), "b3": f(v.b3, (Nc,))}
    g = {"gW1": f(v.gW1, (v.hidden, Din)), "gb1": f(v.gb1, (v.hidden,)), "gW2": f(v.gW2, (v.hidden, v.hidden)),
         "gb2": f(v.gb2, (v.hidden,)), "gW3": f(v.gW3, (Nc, Dz)), "gb3": f(v.gb3, (Nc,))}
    return P, g, v


def batch_inputs(B, seed=0):
    from paper_1705_02403_gb300 import learned
    pbs = [learned.env(seed * 1000 + k, 100) for k in range(B)]
    X = learned.voxelize(pbs)
    SG = learned.start_goal(pbs)
    rng = np.random.default_rng(seed)
    T = rng.random((B, C ** 3)).astype(np.float32) ** 8
    T /= T.sum(1, keepdims=True)
    return pbs, X, SG, torch.tensor(T, device="cuda")


def test_voxelize_matches_numpy():
    pbs, X, _, _ = batch_inputs(4)
    g = (np.arange(G) + 0.5) / G
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    for b, pb in enumerate(pbs):
        occ = np.zeros(len(P), bool)
        for lo, hi in zip(pb.box_lo, pb.box_hi):
            occ |= np.all((lo <= P) & (P <= hi), axis=1)
        assert np.array_equal(X[b].float().cpu().numpy() > 0.5, occ)


def read_bf16(ptr, shape, owner):
    """A device BF16 array as exact FP32 values."""
    bits = dev(ptr, shape, "i2", owner).cpu().numpy().astype(np.uint16).astype(np.uint32)
    return (bits << 16).view(np.float32)


def test_forward_and_gradients_match_cpu_oracle():
    """Every element of every stage of the forward and backward pass against
    the oracle's definition of that stage, evaluated on the stage's own GPU
    inputs (mlp_oracle.stage_violations): a BF16 activation must be a value that
    rounding the exact result, moved by at most its FP32 sum's accumulation
    error, can give; the logits and all six gradients must lie within that
    error of the exact result.  Chained from the true inputs this checks the
    whole computation element by element.  Then the logits and gradients
    against the oracle run from the true inputs: they differ at most by what
    the BF16 intermediates that differ (rounded on either side of a rounding
    boundary that the two FP32 sums straddle) carry through the last product."""
    from oracle import mlp_oracle as M
    from paper_1705_02403_gb300 import _native as N
    B = 8
    m = N.Model(G, H, C, 16, seed=3)
    pbs, Xd, SGd, Td = batch_inputs(B, seed=1)
    loss = m.backward(B, Xd.data_ptr(), SGd.data_ptr(), Td.data_ptr())
    P, g, v = model_params(m)
    X = Xd.float().cpu().numpy()
    SG, T = SGd.cpu().numpy(), Td.cpu().numpy()
    Din, Dz, Nc = v.in_features, v.z_features, v.n_cells
    V = dict(g, loss=loss, logits=dev(v.logits, (B, Nc), "f4", m).cpu().numpy(),
             W1b=read_bf16(v.W1_bf16, (H, Din), m), W2b=read_bf16(v.W2_bf16, (H, H), m),
             W3b=read_bf16(v.W3_bf16, (Nc, Dz), m),
             H1=read_bf16(v.H1, (B, H), m), H2=read_bf16(v.H2, (B, H), m), Z=read_bf16(v.Z, (B, Dz), m),
             dlog=read_bf16(v.dlog, (B, Nc), m), dH2=read_bf16(v.dH2, (B, H), m), dH1=read_bf16(v.dH1, (B, H), m))
    bad = M.stage_violations(P, X, SG, T, V)
    assert not any(bad.values()), bad
    e2e, frac = M.end_to_end_violations(P, X, SG, T, V)
    assert not any(e2e.values()), e2e
    print("fraction of BF16 intermediates that differ from the oracle's:", frac)


def test_training_reduces_loss_and_checkpoints():
    from paper_1705_02403_gb300 import _native as N
    m = N.Model(G, H, C, 32, seed=4)
    pbs, X, SG, T = batch_inputs(32, seed=2)
    first = m.backward(32, X.data_ptr(), SG.data_ptr(), T.data_ptr())
    for _ in range(30):
        last = m.train_step(32, X.data_ptr(), SG.data_ptr(), T.data_ptr(), 1e-3, 1e-4)
    assert last < 0.9 * first
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "m.ckpt")
        m.save(path)
        m2 = N.Model(G, H, C, 32, seed=99)
        m2.load(path)
        l1 = m.backward(32, X.data_ptr(), SG.data_ptr(), T.data_ptr())
        l2 = m2.backward(32, X.data_ptr(), SG.data_ptr(), T.data_ptr())
        assert l1 == l2 and m2.view().step == m.view().step
        # resume: one more step from either gives the same loss
        a = m.train_step(32, X.data_ptr(), SG.data_ptr(), T.data_ptr(), 1e-3, 1e-4)
        b = m2.train_step(32, X.data_ptr(), SG.data_ptr(), T.data_ptr(), 1e-3, 1e-4)
        assert a == b


def test_path_histogram_matches_numpy():
    from paper_1705_02403_gb300 import _native as N
    rng = np.random.default_rng(0)
    Xn = rng.random((3, 50)).astype(np.float32)
    path = np.array([0, 7, 13, 21, 49], np.int32)
    X = torch.tensor(Xn, device="cuda")
    p = torch.tensor(path, device="cuda")
    h = torch.empty(C ** 3, device="cuda")
    N.gmt_path_histogram(X.data_ptr(), 50, p.data_ptr(), len(path), C, 0.01, 1e-4, h.data_ptr())
    ref = np.zeros(C ** 3)
    for a, b in zip(path[:-1], path[1:]):
        L = np.linalg.norm(Xn[:, b] - Xn[:, a])
        m = max(1, int(np.ceil(L / 0.01)))
        for k in range(m):
            x = Xn[:, a] + (k / m) * (Xn[:, b] - Xn[:, a])
            c = np.clip((x * C).astype(int), 0, C - 1)
            ref[(c[0] * C + c[1]) * C + c[2]] += 1
    c = np.clip((Xn[:, path[-1]] * C).astype(int), 0, C - 1)
    ref[(c[0] * C + c[1]) * C + c[2]] += 1
    ref = (ref + 1e-4) / (ref.sum() + 1e-4 * C ** 3)
    assert np.allclose(h.cpu().numpy(), ref, rtol=1e-3, atol=1e-7)


def test_proposal_samples_follow_the_softmax():
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    from paper_1705_02403_gb300.planner import boxes_on_device, space_struct
    m = N.Model(G, H, C, 4, seed=5)
    pb = learned.env(11, 100).with_(box_lo=np.zeros((0, 3), np.float32), box_hi=np.zeros((0, 3), np.float32))
    boxes, keep = boxes_on_device(pb)
    n = 400000
    S = torch.empty(3, n, device="cuda")
    N.gmt_propose(m, space_struct(pb), boxes, pb.x_init, pb.goal_center, n, 123, S.data_ptr(), n)
    logits = dev(m.view().logits, (1, C ** 3), "f4", m).cpu().numpy()[0].astype(np.float64)
    p = np.exp(logits - logits.max()); p /= p.sum()
    s = S.cpu().numpy()
    assert s.min() >= 0.0 and s.max() <= 1.0          # closed state space [0,1]^3
    c = np.clip((s * C).astype(int), 0, C - 1)
    counts = np.bincount((c[0] * C + c[1]) * C + c[2], minlength=C ** 3)
    # coarse chi^2 over 64 groups of 64 cells
    obs = counts.reshape(64, -1).sum(1); exp = n * p.reshape(64, -1).sum(1)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < 120.0          # 63 dof: the 99.99% quantile is about 115
    # with boxes: every sample is collision-free
    pb2 = learned.env(12, 100)
    boxes2, keep2 = boxes_on_device(pb2)
    S2 = torch.empty(3, 5000, device="cuda")
    N.gmt_propose(m, space_struct(pb2), boxes2, pb2.x_init, pb2.goal_center, 5000, 7, S2.data_ptr(), 5000)
    P2 = S2.cpu().numpy().T
    inside = np.any(np.all((pb2.box_lo[None] <= P2[:, None]) & (P2[:, None] <= pb2.box_hi[None]), axis=2), axis=1)
    assert not inside.any()


def test_batched_proposal_follows_each_softmax_and_agrees_with_single_calls():
    # gmt_propose_batch: every environment's samples follow the softmax of its
    # own logits row (chi^2 over 64 groups of cells), stay in X and out of its
    # boxes, and agree with one gmt_propose call per environment (same seed)
    # except where a draw falls within rounding of a CDF cell boundary; 6
    # environments with max_batch 4 take two chunks.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    from paper_1705_02403_gb300.planner import boxes_on_device, space_struct
    m = N.Model(G, H, C, 4, seed=8)
    empty = np.zeros((0, 3), np.float32)
    pbs = [learned.env(40 + k, 100).with_(box_lo=empty, box_hi=empty) for k in range(3)]
    keep = [boxes_on_device(pb) for pb in pbs]
    n = 200000
    S = torch.empty(3, 3, n, device="cuda")
    sg = [np.concatenate([pb.x_init, pb.goal_center]) for pb in pbs]
    N.gmt_propose_batch(m, [space_struct(pb) for pb in pbs], [k[0] for k in keep], sg, n, [5, 6, 7], S.data_ptr(), n)
    logits = dev(m.view().logits, (3, C ** 3), "f4", m).cpu().numpy().astype(np.float64)
    for b in range(3):
        p = np.exp(logits[b] - logits[b].max()); p /= p.sum()
        s = S[b].cpu().numpy()
        assert s.min() >= 0.0 and s.max() <= 1.0
        c = np.clip((s * C).astype(int), 0, C - 1)
        counts = np.bincount((c[0] * C + c[1]) * C + c[2], minlength=C ** 3)
        obs = counts.reshape(64, -1).sum(1); exp = n * p.reshape(64, -1).sum(1)
        assert ((obs - exp) ** 2 / exp).sum() < 120.0, b
    # different environments give different logits rows
    assert np.abs(logits[0] - logits[1]).max() > 1e-3
    # with boxes, two chunks, against single calls
    pbs = [learned.env(60 + k, 100) for k in range(6)]
    keep = [boxes_on_device(pb) for pb in pbs]
    cnt, pitch = 3000, 3008
    S = torch.full((6, 3, pitch), -1.0, device="cuda")
    seeds = [1000 + 3 * k for k in range(6)]
    N.gmt_propose_batch(m, [space_struct(pb) for pb in pbs], [k[0] for k in keep],
                        [np.concatenate([pb.x_init, pb.goal_center]) for pb in pbs], cnt, seeds, S.data_ptr(), pitch)
    Sb = S.cpu().numpy()
    assert np.all(Sb[:, :, cnt:] == -1.0)          # nothing past count is written
    for b, pb in enumerate(pbs):
        one = torch.empty(3, cnt, device="cuda")
        N.gmt_propose(m, space_struct(pb), keep[b][0], pb.x_init, pb.goal_center, cnt, seeds[b], one.data_ptr(), cnt)
        P = Sb[b, :, :cnt].T
        assert P.min() >= 0.0 and P.max() <= 1.0
        inside = np.any(np.all((pb.box_lo[None] <= P[:, None]) & (P[:, None] <= pb.box_hi[None]), axis=2), axis=1)
        assert not inside.any(), b
        same = np.all(one.cpu().numpy().T == P, axis=1).mean()
        assert same >= 0.99, (b, same)


def test_batched_mixture_plans_equal_single_plans():
    # The mixture in batched form (gmt_propose_batch + gmt_plan_batch with the
    # learned samples appended to every query) gives each environment the
    # tree that gmt_build_graph_ex + gmt_plan give on the same sample set, and
    # a replay (same seeds) gives the same bits again.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    m = N.Model(G, H, C, 4, seed=9)
    pbs = [learned.env(80 + k, 500) for k in range(5)]
    mb = learned.MixtureBatch(m, pbs)
    infos = mb.run(allow_errors=False)
    for k, upb in enumerate(mb.upbs):
        v = mb.planner.view(k)
        assert v["N"] == upb.n + 1 + mb.n_l
        X = v["X"].cpu().numpy()
        assert np.array_equal(X[:, upb.n + 1:], mb.samples[k].cpu().numpy())
        g = N.gmt_build_graph_ex(learned.space_struct(upb), mb.boxes[k], [float(x) for x in upb.x_init],
                                 learned.goal_struct(upb), learned.params_struct(upb), mb.samples[k].data_ptr(),
                                 mb.n_l, mb.n_l)
        parent = torch.empty(v["N"], dtype=torch.int32, device="cuda")
        cost = torch.empty(v["N"], dtype=torch.float32, device="cuda")
        info = N.gmt_plan(g, mb.boxes[k], learned.params_struct(upb), parent.data_ptr(), cost.data_ptr(),
                          allow_errors=True).as_dict()
        p, c = mb.planner.result(k)
        assert np.array_equal(p.cpu().numpy(), parent.cpu().numpy()), k
        assert np.array_equal(c.cpu().numpy().view(np.uint32), cost.cpu().numpy().view(np.uint32)), k
        assert infos[k]["status"] == info["status"] and infos[k]["path_cost"] == info["path_cost"]
    p0 = mb.planner.parent.clone()
    mb.planner.parent.fill_(-9)
    infos2 = mb.run(allow_errors=False)
    assert torch.equal(mb.planner.parent, p0)
    assert [i["path_cost"] for i in infos2] == [i["path_cost"] for i in infos]


def test_mixture_graph_appends_learned_samples(O):
    # gmt_build_graph_ex: the appended samples become nodes n+1.. and the graph
    # and tree equal the oracle's on the same sample set.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    m = N.Model(G, H, C, 4, seed=6)
    pb = learned.env(21, 600)
    res, _, _, g = learned.plan_mixture(m, pb)
    v = N.gmt_graph_get_view(g)
    X = dev(v.X, (3, v.x_pitch), "f4", g)[:, :v.N].cpu().numpy()
    goal = dev(v.is_goal, (v.N,), "u1", g).cpu().numpy()
    r = np.float32(N.gmt_connection_radius(300, 3, 0.0, 1.0))
    og = O.Graph(0, 3, 3, X, goal, r)
    assert og.num_edges == v.E
    parent, cost, info = og.plan(pb.box_lo, pb.box_hi, pb.lo, pb.hi, pb.lam)
    assert info["status"] == res[0]
    if res[0] == 0:
        assert np.float32(info["path_cost"]) == np.float32(res[1])


def test_trained_proposal_gains_over_uniform_sampling():
    # What the network adds: trained on plain-GMT* solutions of 768 environments
    # (n = 4096), on 64 held-out environments its cell distribution explains the
    # held-out solution paths far better than uniform sampling (cross-entropy
    # well below log(16^3)), and the 50/50 mixture at n = 1024 finds cheaper
    # paths than uniform sampling at n = 1024 with the same radius.
    from paper_1705_02403_gb300 import _native as N
    from paper_1705_02403_gb300 import learned
    X, SG, T, kept = learned.generate_dataset([3_000_000 + k for k in range(768)], n=4096, log=None)
    m = N.Model(G, H, C, 256, seed=8)
    learned.train(m, X, SG, T, epochs=8, log=None)
    test = [4_000_000 + k for k in range(64)]
    Xt, SGt, Tt, _ = learned.generate_dataset(test, n=4096, log=None)
    assert learned.mean_loss(m, Xt, SGt, Tt) < np.log(C ** 3) - 1.0
    ev = learned.evaluate(m, test, ns=(1024,), n_ref=4096, log=None)
    mix = ev["mixture"]["1024"]["mean_cost"]
    ctrl = ev["uniform_mixture_radius"]["1024"]["mean_cost"]
    assert mix < ctrl, (mix, ctrl)
