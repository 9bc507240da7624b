"""The sweep environments (synthetic analogues of Tables 1 and 3) are valid
planning problems: x_init outside every box, no box touching the goal ball,
boxes inside the domain; the maze leaves a door in every wall and the forest
strips cover each trunk's disk."""
import numpy as np
import pytest

from paper_1705_02403_gb300 import envgen


def inside(p, lo, hi):
    return np.all((lo <= p) & (p <= hi), axis=-1)


@pytest.mark.parametrize("d", [2, 3, 6, 10])
def test_rectangles(d):
    for seed in range(20):
        pb = envgen.rectangles(seed, d, n=100)
        assert pb.box_lo.shape == (10, d)
        assert not inside(pb.x_init, pb.box_lo, pb.box_hi).any()
        near = np.clip(pb.goal_center, pb.box_lo, pb.box_hi)
        assert np.all(np.linalg.norm(near - pb.goal_center, axis=1) > 0.05)
        assert np.all(pb.box_lo[:, 2:] == 0) and np.all(pb.box_hi[:, 2:] == 1)


@pytest.mark.parametrize("d", [3, 5])
def test_maze_walls_have_doors(d):
    rng = np.random.default_rng(0)
    for seed in range(10):
        pb = envgen.maze(seed, d, n=100)
        assert not inside(pb.x_init, pb.box_lo, pb.box_hi).any()
        for w in range(3):
            lo, hi = pb.box_lo[4 * w:4 * w + 4], pb.box_hi[4 * w:4 * w + 4]
            x0 = 0.5 * (lo[0, 0] + hi[0, 0])
            pts = rng.uniform(0, 1, (20000, d))
            pts[:, 0] = x0
            blocked = np.zeros(len(pts), bool)
            for k in range(4):
                blocked |= inside(pts, lo[k], hi[k])
            frac_open = 1 - blocked.mean()
            assert 0.04 < frac_open < 0.09            # a door of side 0.25 in two axes: 1/16 of the wall


def test_forest_strips_cover_each_disk():
    rng = np.random.default_rng(1)
    for strips in (15, 50, 150, 500):
        lo, hi = envgen.forest_boxes(3, 10, strips)
        assert lo.shape == (10 * strips, 3)
        for t in range(10):
            L, H = lo[t * strips:(t + 1) * strips], hi[t * strips:(t + 1) * strips]
            c = np.array([0.5 * (L[0, 0] + H[0, 0]), 0.5 * (L[0, 1] + H[-1, 1])])
            rad = 0.5 * (H[-1, 1] - L[0, 1])
            a = rng.uniform(0, 2 * np.pi, 2000)
            rr = rad * np.sqrt(rng.uniform(0, 0.98, 2000))
            p = np.stack([c[0] + rr * np.cos(a), c[1] + rr * np.sin(a), rng.uniform(0, 1, 2000)], axis=1)
            covered = np.zeros(len(p), bool)
            for k in range(strips):
                covered |= inside(p, L[k], H[k])
            assert covered.all()


def test_dubins_forest():
    for seed in range(10):
        for strips in (15, 500):
            pb = envgen.dubins_forest(seed, n=100, strips=strips)
            assert (pb.kind, pb.d, pb.dp) == (envgen.DUBINS, 4, 3) and pb.rho > 0
            assert pb.box_lo.shape == (10 * strips, 3)
            assert not inside(pb.x_init[:3], pb.box_lo, pb.box_hi).any()
            near = np.clip(pb.goal_center[:3], pb.box_lo, pb.box_hi)
            assert np.all(np.linalg.norm(near - pb.goal_center[:3], axis=1) > pb.goal_radius)
            assert np.all(pb.box_lo[:, 2] == 0) and np.all(pb.box_hi[:, 2] == 1)   # full-height trunks
            assert pb.lo[3] < -3.14 and pb.hi[3] > 3.14                              # every heading
