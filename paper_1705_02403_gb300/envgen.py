"""Seeded synthetic planning problems (inputs only).

This module draws the environments both the CUDA planner and the CPU oracle
consume: state bounds, obstacle boxes, x_init, goal ball, n, r, lambda and the
Philox seed.  It contains none of the planner's arithmetic (no sampling, cost,
neighbour or wavefront code); the obstacle boxes are drawn with numpy's PCG64
from the problem seed.

The paper's own workloads (an S3DIS-derived indoor map, a two-level cave and a
forest, Section V-B) are not available; seeded random-box environments with box
counts and sample counts in the paper's ranges (Table 3) stand in for them.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field, replace

import numpy as np

EUCLID, DI, DUBINS = 0, 1, 2
HERE = os.path.dirname(os.path.abspath(__file__))
CONFIG_DIR = os.path.join(HERE, "configs")


@dataclass
class Problem:
    """One planning query (Problem 1 of the paper plus Alg. 1's inputs)."""
    kind: int                 # EUCLID (arc length), DI (double integrator time + effort) or DUBINS (airplane path length)
    d: int                    # state dimension
    dp: int                   # position dimension (obstacles live here)
    lo: np.ndarray            # [d] state lower bounds
    hi: np.ndarray            # [d] state upper bounds
    box_lo: np.ndarray        # [B, dp] closed obstacle boxes
    box_hi: np.ndarray        # [B, dp]
    x_init: np.ndarray        # [d]
    goal_center: np.ndarray   # [d] (first dp used when goal_pos_only)
    goal_radius: float
    goal_pos_only: bool
    n: int                    # number of samples; N = n + 1 nodes
    r: float                  # connection radius (0 = Theorem 1 radius, computed by the planner)
    lam: float                # group cost threshold factor lambda
    seed: int                 # Philox key for SampleFree
    seg_spacing: float = 0.005
    traj_points: int = 20
    eta: float = 0.0          # Theorem 1 tuning parameter (only when r == 0)
    mu_free: float = 1.0      # Lebesgue measure bound used by Theorem 1 (only when r == 0)
    tag: str = ""
    sampler: int = 0          # 0: Philox i.i.d. uniform; 1: Halton sequence (seed unused)
    rho: float = 0.0          # Dubins airplane turning radius (DUBINS only)

    @property
    def N(self) -> int:
        return self.n + 1

    @property
    def nbox(self) -> int:
        return int(self.box_lo.shape[0])

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def random_boxes(rng, count, dp, x_init_pos, goal_center_pos, goal_radius, side=(0.05, 0.2)):
    """Boxes with per-axis side lengths U[side] and centres U[0,1]^dp; a box that
    contains x_init or touches the goal ball is redrawn."""
    lo = np.zeros((count, dp)); hi = np.zeros((count, dp))
    k = 0
    while k < count:
        s = rng.uniform(side[0], side[1], size=dp)
        c = rng.uniform(0.0, 1.0, size=dp)
        bl, bh = c - s / 2, c + s / 2
        if np.all(bl <= x_init_pos) and np.all(x_init_pos <= bh):
            continue
        nearest = np.clip(goal_center_pos, bl, bh)
        if np.linalg.norm(nearest - goal_center_pos) <= goal_radius:
            continue
        lo[k], hi[k] = bl, bh
        k += 1
    return _f32(lo), _f32(hi)


def geometric(seed: int, d: int = 2, n: int = 1024, nbox: int = 10, r: float = 0.12, lam: float = 0.5,
              tag: str = "") -> Problem:
    """Unit hypercube, Euclidean cost, x_init at 0.05, goal ball radius 0.05 at 0.95."""
    rng = np.random.default_rng([seed, 1705, d])
    x0 = np.full(d, 0.05)
    gc = np.full(d, 0.95)
    bl, bh = random_boxes(rng, nbox, d, x0, gc, 0.05)
    return Problem(kind=EUCLID, d=d, dp=d, lo=_f32(np.zeros(d)), hi=_f32(np.ones(d)), box_lo=bl, box_hi=bh,
                   x_init=_f32(x0), goal_center=_f32(gc), goal_radius=0.05, goal_pos_only=False, n=n, r=r,
                   lam=lam, seed=seed, tag=tag)


def load_config(name: str) -> dict:
    with open(os.path.join(CONFIG_DIR, name + ".json")) as f:
        return json.load(f)


def cfg1_2d(seed: int = 0) -> Problem:
    """2D geometric GMT*: n=1024, 10 boxes, r=0.12, lambda=0.5."""
    c = load_config("geometric_2d_n1024")
    return geometric(seed, d=2, n=c["n"], nbox=c["boxes"], r=c["r"], lam=c["lambda"], tag="geometric_2d_n1024")


def di6(seed: int = 0, n: int = 4096, nbox: int = 30, r: float | None = None, lam: float = 0.5) -> Problem:
    """6D double integrator: position [0,1]^3, velocity [-1,1]^3, x_init at rest
    at (0.05,0.05,0.05), goal = position ball radius 0.05 at (0.95,0.95,0.95)."""
    if r is None:
        r = load_config("double_integrator_6d_n4096")["r"]
    rng = np.random.default_rng([seed, 1705, 6])
    x0 = np.array([0.05, 0.05, 0.05, 0.0, 0.0, 0.0])
    gc = np.array([0.95, 0.95, 0.95, 0.0, 0.0, 0.0])
    bl, bh = random_boxes(rng, nbox, 3, x0[:3], gc[:3], 0.05)
    return Problem(kind=DI, d=6, dp=3, lo=_f32([0, 0, 0, -1, -1, -1]), hi=_f32([1, 1, 1, 1, 1, 1]),
                   box_lo=bl, box_hi=bh, x_init=_f32(x0), goal_center=_f32(gc), goal_radius=0.05,
                   goal_pos_only=True, n=n, r=float(np.float32(r)), lam=lam, seed=seed,
                   tag="double_integrator_6d")


def cfg2_di6(seed: int = 0) -> Problem:
    c = load_config("double_integrator_6d_n4096")
    return di6(seed, n=c["n"], nbox=c["boxes"], r=c["r"], lam=c["lambda"])


def batch_queries(seed: int = 0, q: int = 256, n_min: int = 512, n_max: int = 16384, lam: float = 0.5):
    """Uneven batch: each query 2D or 3D geometric (coin flip), n log-uniform in
    [n_min, n_max], its own seed, 5..80 boxes; r = 0 asks for the Theorem 1
    radius (eta = 0, mu(X_free) <= 1)."""
    rng = np.random.default_rng([seed, 1705, 3])
    out = []
    for k in range(q):
        d = int(rng.integers(2, 4))
        n = int(round(n_min * (n_max / n_min) ** rng.uniform()))
        nbox = int(rng.integers(5, 81))
        qseed = int(rng.integers(0, 2**63 - 1))
        pb = geometric(qseed, d=d, n=n, nbox=nbox, r=0.0, lam=lam, tag=f"batch{seed}_{k}")
        out.append(pb)
    return out

# ---------------------------------------------------------------- sweeps
# Synthetic analogues of the environments of Tables 1 and 3 (the paper gives
# their figures, not their geometry).

def rectangles(seed: int, d: int, n: int = 5000, nbox: int = 10, lam: float = 0.5) -> Problem:
    """Table 1 "Rectangles" analogue: the unit d-cube with nbox rectangles in the
    first two axes (sides U[0.1, 0.3], centres U[0.15, 0.85]^2) extruded over
    every other axis, so they obstruct equally in every dimension; x_init at
    0.05, goal ball radius 0.05 at 0.95; Theorem 1 radius."""
    rng = np.random.default_rng([seed, 1705, 100 + d])
    x0, gc = np.full(d, 0.05), np.full(d, 0.95)
    lo = np.zeros((nbox, d)); hi = np.ones((nbox, d))
    k = 0
    while k < nbox:
        c = rng.uniform(0.15, 0.85, 2)
        s = rng.uniform(0.1, 0.3, 2)
        bl, bh = c - s / 2, c + s / 2
        if np.all(bl <= x0[:2]) and np.all(x0[:2] <= bh):
            continue                                   # would contain x_init
        if np.linalg.norm(np.clip(gc[:2], bl, bh) - gc[:2]) <= 0.05:
            continue                                   # would touch the goal ball
        lo[k, :2], hi[k, :2] = bl, bh
        k += 1
    return Problem(kind=EUCLID, d=d, dp=d, lo=_f32(np.zeros(d)), hi=_f32(np.ones(d)), box_lo=_f32(lo),
                   box_hi=_f32(hi), x_init=_f32(x0), goal_center=_f32(gc), goal_radius=0.05, goal_pos_only=False,
                   n=n, r=0.0, lam=lam, seed=seed, tag=f"rectangles_{d}d")


def maze(seed: int, d: int, n: int = 5000, walls: int = 3, door: float = 0.25, lam: float = 0.5) -> Problem:
    """Table 1 "Maze" analogue: walls of thickness 0.05 across axis 0 at
    x0 = k / (walls + 1), each spanning every other axis except one square door
    (side `door` in axes 1 and 2, at a random place), as 4 boxes per wall
    around the door; d >= 3."""
    rng = np.random.default_rng([seed, 1705, 200 + d])
    x0, gc = np.full(d, 0.05), np.full(d, 0.95)
    lo, hi = [], []
    for w in range(walls):
        xc = (w + 1) / (walls + 1)
        dc = rng.uniform(door / 2 + 0.05, 1 - door / 2 - 0.05, 2)
        d_lo, d_hi = dc - door / 2, dc + door / 2
        for part in range(4):
            bl, bh = np.zeros(d), np.ones(d)
            bl[0], bh[0] = xc - 0.025, xc + 0.025
            if part == 0: bh[1] = d_lo[0]                               # below the door in axis 1
            elif part == 1: bl[1] = d_hi[0]                             # above it
            elif part == 2: bl[1], bh[1], bh[2] = d_lo[0], d_hi[0], d_lo[1]
            else: bl[1], bh[1], bl[2] = d_lo[0], d_hi[0], d_hi[1]
            lo.append(bl); hi.append(bh)
    return Problem(kind=EUCLID, d=d, dp=d, lo=_f32(np.zeros(d)), hi=_f32(np.ones(d)), box_lo=_f32(np.array(lo)),
                   box_hi=_f32(np.array(hi)), x_init=_f32(x0), goal_center=_f32(gc), goal_radius=0.05,
                   goal_pos_only=False, n=n, r=0.0, lam=lam, seed=seed, tag=f"maze_{d}d")


def forest_boxes(seed: int, trunks: int, strips: int):
    """Table 3 obstacle-resolution analogue: `trunks` vertical cylinders in
    the unit cube (radius U[0.03, 0.06], axis at U[0.15, 0.8]^2, full height),
    each cross-section approximated by `strips` axis-aligned strips (each as
    wide as the disk's chord at the strip's edge nearest the axis, so the union
    covers the disk); the same trunks at every resolution."""
    rng = np.random.default_rng([seed, 1705, 300])
    lo, hi = [], []
    for _ in range(trunks):
        c = rng.uniform(0.15, 0.8, 2)
        rad = rng.uniform(0.03, 0.06)
        for k in range(strips):
            y0 = -rad + 2 * rad * k / strips
            y1 = -rad + 2 * rad * (k + 1) / strips
            yo = min(abs(y0), abs(y1)) if y0 * y1 > 0 else 0.0   # the strip's edge nearest the centre
            half = np.sqrt(max(rad * rad - yo * yo, 0.0))
            lo.append([c[0] - half, c[1] + y0, 0.0])
            hi.append([c[0] + half, c[1] + y1, 1.0])
    return _f32(np.array(lo)), _f32(np.array(hi))


def di6_scaled(seed: int, n: int, nbox: int = 300, lam: float = 0.5, boxes=None) -> Problem:
    """Table 3 analogue for the double integrator: the bench workload's setting
    at sample count n with the radius scaled as r_4096 (4096 / n)^(1/6) (about
    the same mean out-degree); boxes: `nbox` random boxes (sides U[0.02, 0.08])
    or the given (lo, hi) arrays."""
    c = load_config("double_integrator_6d_n4096")
    r = float(np.float32(c["r"] * (4096.0 / n) ** (1.0 / 6.0)))
    pb = di6(seed, n=n, nbox=0, r=r, lam=lam)
    if boxes is None:
        rng = np.random.default_rng([seed, 1705, 400])
        bl, bh = random_boxes(rng, nbox, 3, pb.x_init[:3], pb.goal_center[:3], 0.05, side=(0.02, 0.08))
    else:
        bl, bh = boxes
    return pb.with_(box_lo=bl, box_hi=bh, tag=f"di6_n{n}_b{bl.shape[0]}")


def dubins_forest(seed: int, n: int = 5000, trunks: int = 10, strips: int = 15, rho: float = 0.05,
                  r: float = 0.2, lam: float = 1.0, sampler: int = 0) -> Problem:
    """Dubins airplane in a forest (the Sec. V-B forest analogue): state
    (x, y, z, heading), position in the unit cube, heading in [-pi, pi];
    obstacles: forest_boxes(seed, trunks, strips) (full-height trunks); x_init
    at (0.05, 0.05, 0.2) heading 0; goal = position ball radius 0.05 at
    (0.95, 0.95, 0.8); turning radius rho; lambda = 1 as in Sec. V."""
    bl, bh = forest_boxes(seed, trunks, strips) if trunks > 0 else (_f32(np.zeros((0, 3))), _f32(np.zeros((0, 3))))
    pi = float(np.float32(np.pi))
    return Problem(kind=DUBINS, d=4, dp=3, lo=_f32([0, 0, 0, -pi]), hi=_f32([1, 1, 1, pi]), box_lo=bl, box_hi=bh,
                   x_init=_f32([0.05, 0.05, 0.2, 0.0]), goal_center=_f32([0.95, 0.95, 0.8, 0.0]), goal_radius=0.05,
                   goal_pos_only=True, n=n, r=float(np.float32(r)), lam=lam, seed=seed, sampler=sampler,
                   rho=float(np.float32(rho)), tag=f"dubins_forest_n{n}_b{bl.shape[0]}")
