"""Pins of the oracle's SampleFree (Section III-B) and goal membership."""
import numpy as np

from paper_1705_02403_gb300 import envgen

F = np.float32


def rebuild_node(O, pb, k):
    """Node k rebuilt with numpy float32 arithmetic from Philox words."""
    key = (pb.seed & 0xFFFFFFFF, pb.seed >> 32)
    gd = pb.dp if pb.goal_pos_only else pb.d
    for t in range(65536):
        words = np.concatenate([O.philox4x32_10((k, t, 0, b), key) for b in range((pb.d + 3) // 4)])
        x = np.zeros(pb.d, F)
        for a in range(pb.d):
            u = F(int(words[a]) >> 8) * F(2.0 ** -24)
            lo, hi = F(pb.lo[a]), F(pb.hi[a])
            if k == 1 and a < gd:
                lo, hi = F(F(pb.goal_center[a]) - F(pb.goal_radius)), F(F(pb.goal_center[a]) + F(pb.goal_radius))
            x[a] = F(lo + F(u * F(hi - lo)))
        if k == 1:
            diff = x[:gd] - pb.goal_center[:gd].astype(F)
            s = F(0)
            for v in diff:
                s = F(s + F(v * v))
            if not (s <= F(F(pb.goal_radius) * F(pb.goal_radius))):
                continue
            if np.any(x < pb.lo) or np.any(x > pb.hi):
                continue
        p = x[:pb.dp]
        if np.any(np.all((pb.box_lo <= p) & (p <= pb.box_hi), axis=1)):
            continue
        return x
    raise AssertionError("no sample")


def test_sample_invariants(O):
    for pb in [envgen.cfg1_2d(3), envgen.di6(seed=2, n=500)]:
        X, goal = O.sample(pb)
        N = pb.N
        assert X.shape == (pb.d, N)
        assert np.array_equal(X[:, 0], pb.x_init)
        assert np.all(X >= pb.lo[:, None]) and np.all(X <= pb.hi[:, None])
        P = X[:pb.dp].T
        inside = np.all((pb.box_lo[None] <= P[:, None]) & (P[:, None] <= pb.box_hi[None]), axis=2)
        assert not inside.any(), "a sample lies in an obstacle"
        assert goal[1] == 1, "node 1 must lie in the goal region"
        gd = pb.dp if pb.goal_pos_only else pb.d
        for k in range(N):
            assert goal[k] == O.in_goal(X[:gd, k], gd, pb.goal_center[:gd], pb.goal_radius)
        X2, goal2 = O.sample(pb)
        assert np.array_equal(X, X2) and np.array_equal(goal, goal2)


def test_sample_matches_independent_rebuild(O):
    for pb in [envgen.cfg1_2d(11), envgen.di6(seed=5, n=64)]:
        X, _ = O.sample(pb)
        for k in list(range(1, 12)) + [pb.n]:
            ref = rebuild_node(O, pb, k)
            assert np.array_equal(X[:, k].view(np.uint32), ref.view(np.uint32)), k


def test_sample_seed_changes_samples(O):
    a, _ = O.sample(envgen.cfg1_2d(1))
    b, _ = O.sample(envgen.cfg1_2d(2))
    assert not np.array_equal(a[:, 2:], b[:, 2:])


def test_sample_uniform_chi2(O):
    # No obstacles: nodes 2..n must be uniform on the unit square.  10x10
    # cells, 99 dof; the 99.9% quantile of chi^2_99 is 148.2.
    pb = envgen.geometric(7, d=2, n=20000, nbox=0)
    X, _ = O.sample(pb)
    P = X[:, 2:]
    idx = np.minimum((P * 10).astype(int), 9)
    counts = np.bincount(idx[0] * 10 + idx[1], minlength=100)
    exp = P.shape[1] / 100
    assert ((counts - exp) ** 2 / exp).sum() < 148.2


def test_sample_rejects_bad_x_init(O):
    pb = envgen.cfg1_2d(0)
    bad = pb.with_(x_init=np.array([1.5, 0.5], np.float32))
    try:
        O.sample(bad)
    except ValueError:
        pass
    else:
        raise AssertionError("x_init outside X must be rejected")
    c = (pb.box_lo[0] + pb.box_hi[0]) / 2
    try:
        O.sample(pb.with_(x_init=c.astype(np.float32)))
    except ValueError:
        pass
    else:
        raise AssertionError("x_init inside an obstacle must be rejected")
