"""Pins of the oracle's lazy edge collision check (Alg. 1, Sec. III-A)."""
import numpy as np

F = np.float32


def slab_chord(y, x, lo, hi):
    """Length of the part of segment y->x inside the closed box [lo, hi]
    (exact slab method in float64), 0 if it misses."""
    y = y.astype(float); x = x.astype(float)
    d = x - y
    t0, t1 = 0.0, 1.0
    for a in range(len(y)):
        if abs(d[a]) < 1e-300:
            if y[a] < lo[a] or y[a] > hi[a]:
                return 0.0
            continue
        ta, tb = (lo[a] - y[a]) / d[a], (hi[a] - y[a]) / d[a]
        ta, tb = min(ta, tb), max(ta, tb)
        t0, t1 = max(t0, ta), min(t1, tb)
        if t0 > t1:
            return 0.0
    return (t1 - t0) * np.linalg.norm(d)


def seg_box_distance(y, x, lo, hi, samples=2001):
    t = np.linspace(0, 1, samples)[:, None]
    P = y.astype(float) + t * (x.astype(float) - y.astype(float))
    q = np.clip(P, lo, hi)
    return np.min(np.linalg.norm(P - q, axis=1))


def test_geometric_check_agrees_with_exact_slab_test(O):
    rng = np.random.default_rng(0)
    spacing = 0.005
    decided = 0
    for trial in range(600):
        d = 2 if trial % 2 == 0 else 3
        y = rng.random(d).astype(F)
        x = (y + rng.uniform(-0.2, 0.2, d)).astype(F)
        c = rng.random(d); s = rng.uniform(0.005, 0.08, d)
        lo, hi = (c - s / 2).astype(F), (c + s / 2).astype(F)
        if np.all((lo <= y) & (y <= hi)) or np.all((lo <= x) & (x <= hi)):
            continue
        L = O.cost_euclid(y, x)
        free = O.edge_free_geometric(y, x, L, spacing, lo[None], hi[None])
        chord = slab_chord(y, x, lo.astype(float), hi.astype(float))
        if chord > spacing + 1e-6:
            assert not free, "a chord longer than the point spacing must be detected"
            decided += 1
        elif chord == 0.0 and seg_box_distance(y, x, lo, hi) > 1e-6:
            assert free, "a segment that misses the box must be free"
            decided += 1
    assert decided > 300


def test_geometric_hand_placed():
    from oracle import oracle as O
    wall_lo = np.array([[0.5, 0.0]], F); wall_hi = np.array([[0.51, 0.6]], F)
    y, x = np.array([0.4, 0.3], F), np.array([0.6, 0.3], F)
    assert not O.edge_free_geometric(y, x, O.cost_euclid(y, x), 0.005, wall_lo, wall_hi)
    y2, x2 = np.array([0.4, 0.7], F), np.array([0.6, 0.7], F)      # passes above the wall
    assert O.edge_free_geometric(y2, x2, O.cost_euclid(y2, x2), 0.005, wall_lo, wall_hi)
    # closed boxes: touching the boundary collides
    y3, x3 = np.array([0.25, 0.6], F), np.array([0.75, 0.6], F)
    assert not O.edge_free_geometric(y3, x3, O.cost_euclid(y3, x3), 0.005, wall_lo, wall_hi)
    # a wall thinner than the spacing can be missed; a zero-length edge tests its endpoint
    assert O.edge_free_geometric(y, y, 0.0, 0.005, wall_lo, wall_hi)


def test_di_rest_to_rest_is_the_straight_segment(O):
    # v0 = v1 = 0: the Hermite curve is the segment p0->p1 traversed with
    # h01(s) = 3s^2 - 2s^3; consecutive points are at most 1.5/19 of the length
    # apart, so any chord longer than that is detected.
    rng = np.random.default_rng(1)
    plo, phi = np.zeros(3, F), np.ones(3, F)
    decided = 0
    for _ in range(400):
        p0 = rng.uniform(0.1, 0.9, 3); p1 = rng.uniform(0.1, 0.9, 3)
        s0 = np.r_[p0, 0, 0, 0].astype(F); s1 = np.r_[p1, 0, 0, 0].astype(F)
        c = rng.random(3); s = rng.uniform(0.02, 0.2, 3)
        lo, hi = (c - s / 2).astype(F), (c + s / 2).astype(F)
        if np.all((lo <= s0[:3]) & (s0[:3] <= hi)) or np.all((lo <= s1[:3]) & (s1[:3] <= hi)):
            continue
        J, tau = O.cost_di(s0, s1, F(8.0))
        free = O.edge_free_di(s0, s1, tau, 20, plo, phi, lo[None], hi[None])
        chord = slab_chord(s0[:3], s1[:3], lo.astype(float), hi.astype(float))
        L = np.linalg.norm(p1 - p0)
        if chord > 1.5 / 19 * L + 1e-6:
            assert not free
            decided += 1
        elif chord == 0.0 and seg_box_distance(s0[:3], s1[:3], lo, hi) > 1e-6:
            assert free
            decided += 1
    assert decided > 200


def test_di_leaving_the_workspace_collides(O):
    # Start and end at the same point near the ceiling, leaving upwards and
    # arriving from above: the trajectory rises past z = 1.
    s0 = np.array([0.5, 0.5, 0.9, 0, 0, 1.0], F)
    s1 = np.array([0.5, 0.5, 0.9, 0, 0, -1.0], F)
    J, tau = O.cost_di(s0, s1, F(8.0))
    assert np.isfinite(J)
    none = np.zeros((0, 3), F)
    assert not O.edge_free_di(s0, s1, tau, 20, np.zeros(3, F), np.ones(3, F), none, none)
    assert O.edge_free_di(s0, s1, tau, 20, np.zeros(3, F), np.full(3, 2.0, F), none, none)


def test_geometric_point_count(O):
    # L = 0.125, spacing 0.005: in FP32 L/spacing rounds to exactly 25, so
    # m = ceil(.)+1 = 26 points with step L/25 = 0.005, at x = 0.25 + 0.005k.
    # A sliver box [0.2549, 0.2551] holds the point x = 0.255 but no point of a
    # 25-point discretisation (step 0.0052083: 0.25, 0.2552083, ...).
    y, x = np.array([0.25, 0.5], F), np.array([0.375, 0.5], F)
    L = O.cost_euclid(y, x)
    assert L == F(0.125)
    lo, hi = np.array([[0.2549, 0.4]], F), np.array([[0.2551, 0.6]], F)
    assert not O.edge_free_geometric(y, x, L, 0.005, lo, hi)
    lo2, hi2 = np.array([[0.2552, 0.4]], F), np.array([[0.2598, 0.6]], F)   # strictly between two points
    assert O.edge_free_geometric(y, x, L, 0.005, lo2, hi2)
