"""Pins of the oracle's Halton SampleFree (Sec. V's low-dispersion sampler):
radical inverses against their closed form and an exact rational rebuild,
the sample set against the definition rebuilt in numpy, and the
low-dispersion radius against its relation to Theorem 1's."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1705_02403_gb300 import envgen

PRIMES = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]


def radical_inverse(k, p):
    x, f = Fraction(0), Fraction(1, p)
    while k > 0:
        x += (k % p) * f
        f /= p
        k //= p
    return np.float32(float(x))


def test_radical_inverse_closed_forms(O):
    assert [O.halton_unit(k, 2) for k in range(1, 9)] == [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875, 0.0625]
    third = [Fraction(1, 3), Fraction(2, 3), Fraction(1, 9), Fraction(4, 9), Fraction(7, 9), Fraction(2, 9),
             Fraction(5, 9), Fraction(8, 9)]
    assert [O.halton_unit(k, 3) for k in range(1, 9)] == [np.float32(float(x)) for x in third]
    # powers of the base map to their reciprocals; p^m - 1 to 1 - p^-m
    for p in PRIMES:
        assert O.halton_unit(p, p) == np.float32(1.0 / (p * p))
        assert O.halton_unit(p ** 3 - 1, p) == np.float32(float(1 - Fraction(1, p ** 3)))


def test_radical_inverse_matches_exact_rationals(O):
    rng = np.random.default_rng(3)
    for k in list(rng.integers(1, 1 << 24, 300)) + [1, 2, (1 << 24) - 1]:
        for p in PRIMES:
            assert O.halton_unit(int(k), p) == radical_inverse(int(k), p), (k, p)


def halton_rebuild(pb, count, goal_mapped=False):
    d = pb.d
    gd = pb.dp if pb.goal_pos_only else d
    pts = []
    for k in range(1, count + 1):
        u = np.array([radical_inverse(k, PRIMES[a]) for a in range(d)], np.float32)
        lo, hi = pb.lo.astype(np.float32).copy(), pb.hi.astype(np.float32).copy()
        if goal_mapped:
            lo[:gd] = np.float32(pb.goal_center[:gd]) - np.float32(pb.goal_radius)
            hi[:gd] = np.float32(pb.goal_center[:gd]) + np.float32(pb.goal_radius)
        pts.append(lo + u * (hi - lo))
    return np.array(pts, np.float32)


def in_boxes(P, pb):
    return np.any(np.all((pb.box_lo[None] <= P[:, None, :pb.dp]) & (P[:, None, :pb.dp] <= pb.box_hi[None]), axis=2),
                  axis=1)


@pytest.mark.parametrize("case", ["2d", "3d", "di6"])
def test_halton_sample_set_follows_the_definition(O, case):
    pb = {"2d": envgen.geometric(3, d=2, n=300, nbox=10, r=0.1),
          "3d": envgen.geometric(4, d=3, n=250, nbox=30, r=0.2),
          "di6": envgen.di6(seed=5, n=200, nbox=30, r=2.0)}[case]
    X, goal = O.sample_halton(pb)
    N = pb.N
    assert np.array_equal(X[:, 0], pb.x_init.astype(np.float32))
    # nodes 2..n: the free Halton points in index order
    P = halton_rebuild(pb, 4 * N)
    free = P[~in_boxes(P, pb)]
    assert np.array_equal(X[:, 2:].T, free[:N - 2])
    # node 1: the first goal-mapped Halton point in X, in the goal ball, outside the boxes
    G = halton_rebuild(pb, 2000, goal_mapped=True)
    gd = pb.dp if pb.goal_pos_only else pb.d
    ok = (np.all((pb.lo <= G) & (G <= pb.hi), axis=1) & ~in_boxes(G, pb)
          & np.array([O.in_goal(g, gd, pb.goal_center, pb.goal_radius) for g in G]))
    assert np.array_equal(X[:, 1], G[np.argmax(ok)])
    assert goal[1] == 1 and goal[0] == 0


def test_halton_radius_drops_the_log_factor(O):
    for d in (2, 3, 6):
        for n in (100, 4096, 100000):
            assert O.radius_halton(n, d) == pytest.approx(O.radius_thm1(n, d) / np.log(n) ** (1.0 / d), rel=1e-12)
