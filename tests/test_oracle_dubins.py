"""Pins of the oracle's Dubins airplane (Sec. V-A: a planar Dubins car with a
single integrator in altitude and Euclidean path-length cost).

The oracle's words are checked against an independent construction written
here from the circle geometry (tangent lines between turning circles, the
circle touching both end circles), every word's segments are walked here in
closed form and must land on the target pose, and the oracle's own sine,
cosine, arctangent and arccosine are checked against numpy.
"""
import math

import numpy as np
import pytest

from paper_1705_02403_gb300 import envgen

F = np.float32
WORDS = ("LSL", "RSR", "LSR", "RSL", "RLR", "LRL")
TWO_PI = 2 * math.pi


def mod2pi(a):
    return a - TWO_PI * math.floor(a / TWO_PI)


def ang_diff(a, b):
    d = mod2pi(a - b)
    return min(d, TWO_PI - d)


def walk(pose, word, lengths, rho):
    """End pose of the word's segments (t, p, q in units of rho) from pose."""
    x, y, th = pose
    for seg, u in zip(word, lengths):
        if seg == "S":
            x, y = x + rho * u * math.cos(th), y + rho * u * math.sin(th)
        elif seg == "L":
            x, y = x + rho * (math.sin(th + u) - math.sin(th)), y + rho * (math.cos(th) - math.cos(th + u))
            th += u
        else:
            x, y = x + rho * (math.sin(th) - math.sin(th - u)), y + rho * (math.cos(th - u) - math.cos(th))
            th -= u
    return x, y, th


def circle(pose, side, rho):
    x, y, th = pose
    if side == "L":
        return np.array([x - rho * math.sin(th), y + rho * math.cos(th)])
    return np.array([x + rho * math.sin(th), y - rho * math.cos(th)])


def turn(side, h0, h1):
    return mod2pi(h1 - h0) if side == "L" else mod2pi(h0 - h1)


def geometric_lengths(p0, p1, rho):
    """Word lengths from the circle construction: CSC via the common tangent
    of the two turning circles, CCC via the circle of radius rho touching both
    (both positions of it)."""
    out = {}
    for w in ("LSL", "RSR", "LSR", "RSL"):
        c0, c1 = circle(p0, w[0], rho), circle(p1, w[2], rho)
        v = c1 - c0
        D = float(np.hypot(*v))
        ang = math.atan2(v[1], v[0])
        if w[0] == w[2]:
            ell, psi = D, ang
        else:
            if D < 2 * rho:
                continue
            ell = math.sqrt(D * D - 4 * rho * rho)
            psi = ang + math.atan2(2 * rho, ell) if w == "LSR" else ang - math.atan2(2 * rho, ell)
        out[w] = rho * (turn(w[0], p0[2], psi) + turn(w[2], psi, p1[2])) + ell
    for w in ("RLR", "LRL"):
        c0, c1 = circle(p0, w[0], rho), circle(p1, w[2], rho)
        v = c1 - c0
        D = float(np.hypot(*v))
        if D > 4 * rho:
            continue
        m = (c0 + c1) / 2
        h = math.sqrt(max(4 * rho * rho - D * D / 4, 0.0))
        nrm = np.array([-v[1], v[0]]) / D if D > 0 else np.array([0.0, 1.0])
        best = math.inf
        for sgn in (1, -1):
            c2 = m + sgn * h * nrm
            t0, t1 = (c0 + c2) / 2, (c1 + c2) / 2
            off = math.pi / 2 if w[0] == "L" else -math.pi / 2
            h0 = math.atan2(t0[1] - c0[1], t0[0] - c0[0]) + off     # heading at the first contact
            h1 = math.atan2(t1[1] - c1[1], t1[0] - c1[0]) + off     # heading at the second contact
            total = turn(w[0], p0[2], h0) + turn(w[1], h0, h1) + turn(w[2], h1, p1[2])
            best = min(best, rho * total)
        out[w] = best
    return out


def random_pairs(rng, count, spread=0.4):
    for _ in range(count):
        a = np.array([*rng.uniform(0, 1, 3), rng.uniform(-math.pi, math.pi)])
        b = np.array([*(a[:3] + rng.uniform(-spread, spread, 3)), rng.uniform(-math.pi, math.pi)])
        yield a, b


# ------------------------------------------------------------------ trigonometry
def test_trig_matches_numpy(O):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-40, 40, 4000), np.linspace(-7, 7, 2001), [0.0, math.pi / 4, -math.pi / 2]])
    for prec, tol in ((64, 1e-11), (32, None)):
        xs = x if prec == 64 else x.astype(F).astype(np.float64)
        s, c = O.dub_trig(0, xs, precision=prec)
        # float: the argument's own spacing bounds the reduction error
        t = tol if tol else 2.5e-7 + 2 * np.spacing(np.abs(xs).astype(F)).astype(np.float64)
        assert np.all(np.abs(s - np.sin(xs)) <= t) and np.all(np.abs(c - np.cos(xs)) <= t)
    y, xx = rng.normal(size=5000), rng.normal(size=5000)
    y[:4], xx[:4] = [0.0, 1.0, 0.0, -1.0], [1.0, 0.0, -1.0, 0.0]
    for prec, tol in ((64, 1e-10), (32, 4e-7)):
        yy, xv = (y, xx) if prec == 64 else (y.astype(F).astype(np.float64), xx.astype(F).astype(np.float64))
        a = O.dub_trig(1, xv, yy, precision=prec)
        assert np.all(np.abs(a - np.arctan2(yy, xv)) <= tol)
    assert O.dub_trig(1, [0.0], [0.0])[0] == 0.0
    u = np.concatenate([rng.uniform(-1, 1, 3000), [-1.0, 0.0, 1.0]])
    for prec, tol in ((64, 1e-10), (32, 5e-7)):
        uu = u if prec == 64 else u.astype(F).astype(np.float64)
        assert np.all(np.abs(O.dub_trig(2, uu, precision=prec) - np.arccos(uu)) <= tol)


# ------------------------------------------------------------------ words
def test_every_word_lands_on_the_target_pose(O):
    rng = np.random.default_rng(2)
    seen = set()
    for rho in (0.05, 0.2):
        for a, b in random_pairs(rng, 400, spread=0.5):
            words, best = O.dubins_words(a, b, rho, precision=64)
            for k in range(6):
                w, t, p, q, L = words[k]
                if not np.isfinite(L):
                    continue
                x, y, th = walk((a[0], a[1], a[3]), WORDS[k], (t, p, q), rho)
                assert abs(x - b[0]) < 1e-9 and abs(y - b[1]) < 1e-9 and ang_diff(th, b[3]) < 1e-9, WORDS[k]
                assert L == pytest.approx(rho * (t + p + q), rel=1e-14)
                if WORDS[k] in ("RLR", "LRL"):
                    assert p >= math.pi - 1e-12     # the middle arc of a CCC word exceeds a half turn
            seen.add(best)
    assert seen == set(range(6)), "every word is the shortest for some pair"


def test_words_match_the_circle_construction(O):
    rng = np.random.default_rng(3)
    for rho in (0.05, 0.15):
        for a, b in random_pairs(rng, 400, spread=0.5):
            words, best = O.dubins_words(a, b, rho, precision=64)
            geo = geometric_lengths((a[0], a[1], a[3]), (b[0], b[1], b[3]), rho)
            for k, w in enumerate(WORDS[:4]):
                if w in geo and np.isfinite(words[k, 4]):
                    assert words[k, 4] == pytest.approx(geo[w], abs=1e-9), w
            Lmin = min(geo.values())
            assert words[best, 4] == pytest.approx(Lmin, abs=1e-9), "shortest path"


def test_closed_forms(O):
    rho = 0.1
    # headings along the line: the straight segment
    for phi in (0.0, 0.7, -2.0, math.pi - 0.01):
        a = np.array([0.3, 0.4, 0.2, phi])
        for D, dz in ((0.25, 0.0), (0.6, 0.3), (0.05, -0.1)):
            b = np.array([a[0] + D * math.cos(phi), a[1] + D * math.sin(phi), a[2] + dz, phi])
            assert O.cost_dubins(a, b, rho, 10.0, precision=64) == pytest.approx(math.hypot(D, dz), abs=1e-12)
            assert O.cost_dubins(a, b, rho, 10.0) == pytest.approx(math.hypot(D, dz), rel=2e-6)
    # north at the origin to south at (4 rho, 0): a right quarter turn, 2 rho
    # east along the top of the two right circles, a right quarter turn
    # (Dubins' RSR with t = q = pi/2, p = 2); its mirror image and reversal
    for prec, tol in ((64, 1e-12), (32, 1e-6)):
        for dz in (0.0, 0.5):
            L = (math.pi + 2) * rho
            for a, b in (([0, 0, 0, math.pi / 2], [4 * rho, 0, dz, -math.pi / 2]),
                         ([0, 0, 0, -math.pi / 2], [4 * rho, 0, dz, math.pi / 2]),
                         ([4 * rho, 0, dz, math.pi / 2], [0, 0, 0, -math.pi / 2])):
                assert O.cost_dubins(a, b, rho, 10.0, precision=prec) == pytest.approx(math.hypot(L, dz), abs=tol)
    words, best = O.dubins_words([0, 0, 0, math.pi / 2], [4 * rho, 0, 0, -math.pi / 2], rho, precision=64)
    assert WORDS[best] == "RSR" and np.allclose(words[best, 1:4], [math.pi / 2, 2, math.pi / 2], atol=1e-12)


def test_symmetries_and_bounds(O):
    rng = np.random.default_rng(4)
    rho = 0.08
    for a, b in random_pairs(rng, 300, spread=0.4):
        c = O.cost_dubins(a, b, rho, 10.0, precision=64)
        d3 = float(np.linalg.norm(b[:3] - a[:3]))
        assert c >= d3 - 1e-12
        # rigid motion of the plane (positions and headings together)
        w, tx, ty = rng.uniform(-math.pi, math.pi), rng.uniform(-1, 1), rng.uniform(-1, 1)
        R = np.array([[math.cos(w), -math.sin(w)], [math.sin(w), math.cos(w)]])
        mv = lambda s: np.array([*(R @ s[:2] + [tx, ty]), s[2], s[3] + w])
        assert O.cost_dubins(mv(a), mv(b), rho, 10.0, precision=64) == pytest.approx(c, abs=1e-9)
        # mirror y -> -y, heading -> -heading: same length, left and right swapped
        mr = lambda s: np.array([s[0], -s[1], s[2], -s[3]])
        assert O.cost_dubins(mr(a), mr(b), rho, 10.0, precision=64) == pytest.approx(c, abs=1e-9)
        # the reversed trajectory (end to start, headings turned around)
        rv = lambda s: np.array([s[0], s[1], s[2], s[3] + math.pi])
        assert O.cost_dubins(rv(b), rv(a), rho, 10.0, precision=64) == pytest.approx(c, abs=1e-9)
        # float against double
        assert O.cost_dubins(a, b, rho, 10.0) == pytest.approx(c, abs=2e-4 * rho + 1e-5 * c)


def test_prefilter_never_decides(O):
    # pairs just past the prefilter's bound: the raw float cost is >= r anyway
    rng = np.random.default_rng(5)
    r, rho = 0.2, 0.05
    for _ in range(3000):
        a = np.array([*rng.uniform(0.2, 0.8, 3), rng.uniform(-math.pi, math.pi)])
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        b = np.array([*(a[:3] + u * r * rng.uniform(1.0, 1.02)), rng.uniform(-math.pi, math.pi)])
        d2 = float(np.sum((b[:3].astype(F) - a[:3].astype(F)).astype(np.float64) ** 2))
        raw = O.cost_dubins(a, b, rho, 100.0)
        if d2 >= 1.015625 * r * r:
            assert raw >= r
            assert math.isinf(O.cost_dubins(a, b, rho, r))
        else:
            assert O.cost_dubins(a, b, rho, r) == raw


# ------------------------------------------------------------------ trajectory points and checks
def test_points_follow_the_path(O):
    rng = np.random.default_rng(6)
    rho = 0.07
    for a, b in random_pairs(rng, 100, spread=0.3):
        words, best = O.dubins_words(a, b, rho, precision=64)
        L = words[best, 4]
        p0 = O.dubins_point(a, b, rho, 0.0, precision=64)
        p1 = O.dubins_point(a, b, rho, 1.0, precision=64)
        assert np.allclose(p0[:3], a[:3], atol=1e-12) and ang_diff(p0[3], a[3]) < 1e-12
        assert np.allclose(p1[:3], b[:3], atol=1e-9) and ang_diff(p1[3], b[3]) < 1e-9
        pts = np.array([O.dubins_point(a, b, rho, k / 64, precision=64) for k in range(65)])
        seg = np.hypot(np.diff(pts[:, 0]), np.diff(pts[:, 1]))
        assert np.all(seg <= L / 64 * (1 + 1e-9)) and seg.sum() >= L * 0.995   # unit planar speed
        assert np.allclose(pts[:, 2], a[2] + np.arange(65) / 64 * (b[2] - a[2]), atol=1e-12)
        # midpoints against this file's closed-form walk of the chosen word
        for s in (0.25, 0.5, 0.75):
            ell = s * L / rho
            lens, rest = [], ell
            for u in words[best, 1:4]:
                lens.append(min(rest, u))
                rest -= lens[-1]
            x, y, th = walk((a[0], a[1], a[3]), WORDS[best], lens, rho)
            q = O.dubins_point(a, b, rho, s, precision=64)
            assert abs(q[0] - x) < 1e-9 and abs(q[1] - y) < 1e-9 and ang_diff(q[3], th) < 1e-9


def test_check_against_independent_walk(O):
    """The float check against a double walk of the same points (boxes and
    walls), skipping points within 1e-4 of a face."""
    rng = np.random.default_rng(7)
    rho, spacing = 0.06, 0.01
    lo, hi = np.zeros(3, F), np.ones(3, F)
    agree = 0
    for trial in range(300):
        a = np.array([*rng.uniform(0.05, 0.95, 3), rng.uniform(-math.pi, math.pi)], F)
        b = np.array([*(a[:3] + rng.uniform(-0.25, 0.25, 3)), rng.uniform(-math.pi, math.pi)], F)
        c = O.cost_dubins(a, b, rho, 100.0)
        blo = rng.uniform(0, 1, (4, 3)).astype(F)
        bhi = (blo + rng.uniform(0.02, 0.2, (4, 3))).astype(F)
        words, best = O.dubins_words(a, b, rho, precision=64)
        L = words[best, 4]
        m = max(2, math.ceil(F(c) / F(spacing)) + 1)
        hit, near = False, False
        for k in range(m):
            s = k / (m - 1)
            ell, lens = s * L / rho, []
            for u in words[best, 1:4]:
                lens.append(min(ell, u))
                ell -= lens[-1]
            x, y, _ = walk((a[0], a[1], a[3]), WORDS[best], lens, rho)
            p = np.array([x, y, a[2] + s * (b[2] - a[2])])
            inside = np.all((blo <= p) & (p <= bhi), axis=1)
            out = np.any(p < lo) or np.any(p > hi)
            gap = min(np.min(np.abs(np.concatenate([(p - blo).ravel(), (p - bhi).ravel()]))),
                      np.min(np.abs(np.concatenate([p - lo, p - hi]))))
            near |= gap < 1e-4
            hit |= bool(np.any(inside)) or out
        if near:
            continue
        assert O.edge_free_dubins(a, b, c, rho, spacing, lo, hi, blo, bhi) == (not hit)
        agree += 1
    assert agree > 200


# ------------------------------------------------------------------ graph and plan
def test_dubins_graph_matches_pairwise_costs(O):
    pb = envgen.dubins_forest(3, n=250, r=0.3)
    X, goal = O.sample(pb)
    g = O.graph_for(pb, X, goal)
    csr = g.csr()
    N = X.shape[1]
    E = 0
    for i in range(N):
        cols = []
        for j in range(N):
            if j != i:
                c = O.cost_dubins(X[:, i], X[:, j], pb.rho, pb.r)
                if F(c) < F(pb.r):
                    cols.append((j, F(c)))
        row = list(zip(csr.out_col[csr.out_row[i]:csr.out_row[i + 1]], csr.out_cost[csr.out_row[i]:csr.out_row[i + 1]]))
        assert [(int(j), F(c)) for j, c in row] == cols
        E += len(cols)
    assert E == g.num_edges > 0
    # in-rows hold the same edges, transposed
    pairs_out = {(i, int(j)) for i in range(N) for j in csr.out_col[csr.out_row[i]:csr.out_row[i + 1]]}
    pairs_in = {(int(j), x) for x in range(N) for j in csr.in_col[csr.in_row[x]:csr.in_row[x + 1]]}
    assert pairs_out == pairs_in
    assert any((j, i) not in pairs_out for i, j in pairs_out), "the Dubins cost is not symmetric"


def test_dubins_plans(O):
    from test_oracle_plan import tree_invariants
    for seed, n, r in ((1, 400, 0.35), (2, 600, 0.3)):
        pb = envgen.dubins_forest(seed, n=n, r=r)
        X, goal = O.sample(pb)
        g = O.graph_for(pb, X, goal)
        args = (pb.box_lo, pb.box_hi, pb.lo[:3], pb.hi[:3])
        best, _ = g.dijkstra(*args, pb.seg_spacing)
        for lam in (0.5, 1.0):
            parent, cost, info, added, closed = g.plan(*args, lam, pb.seg_spacing, trace=True)
            tree_invariants(O, pb, g, parent, cost, added, closed, lam)
            assert info["status"] == O.OK and info["path_cost"] >= best
            assert info["path_cost"] >= float(np.linalg.norm(pb.goal_center[:3] - pb.x_init[:3])) - pb.goal_radius
        pg, cg, ig = g.plan(*args, 0.0, pb.seg_spacing)
        pf, cf, i_f = g.plan(*args, 0.0, pb.seg_spacing, which="fmt")
        assert ig["path_cost"] == i_f["path_cost"] and O.path_to(pg, ig["goal_node"]) == O.path_to(pf, i_f["goal_node"])
