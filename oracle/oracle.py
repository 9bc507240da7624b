"""ctypes wrapper of the GMT* CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
import this module.  The planner library never does.  The C++ source is
``oracle/gmt_oracle.cpp``; it is built with IEEE semantics and FMA contraction
off (``-O2 -ffp-contract=off -fno-fast-math``) so that its FP32 results are
reproducible bit for bit on x86-64 and aarch64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gmt_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

OK, NO_PATH, ERR_INVALID, ERR_ITER_LIMIT = 0, 1, -1, -5
EUCLID, DI, DUBINS = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain g++)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("goal_node", C.c_int32), ("path_cost", C.c_double),
                ("iters", C.c_int64), ("final_i", C.c_int64), ("push_edges", C.c_int64),
                ("pull_edges", C.c_int64), ("checks", C.c_int64), ("failed", C.c_int64),
                ("tree_size", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P, I32, I64, F32, F64, U64, U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_uint64, C.c_uint32
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_word_to_unit.argtypes = [U32]; L.orc_word_to_unit.restype = F32
        L.orc_sample.argtypes = [I32, I32, P, P, I32, P, P, P, P, F32, I32, I32, U64, U32, I32, P, P]
        L.orc_sample.restype = I32
        L.orc_in_goal.argtypes = [P, I32, P, F32]; L.orc_in_goal.restype = I32
        L.orc_cost_euclid_f32.argtypes = [P, P, I32]; L.orc_cost_euclid_f32.restype = F32
        L.orc_cost_euclid_f64.argtypes = [P, P, I32]; L.orc_cost_euclid_f64.restype = F64
        L.orc_cost_di_f32.argtypes = [P, P, F32, P]; L.orc_cost_di_f32.restype = F32
        L.orc_cost_di_f64.argtypes = [P, P, F64, I32, I32, P]; L.orc_cost_di_f64.restype = F64
        L.orc_di_coeffs_f64.argtypes = [P, P, P]
        L.orc_hermite_point_f64.argtypes = [P, P, F64, F64, P]
        L.orc_edge_free_geometric_f32.argtypes = [P, P, I32, F32, F32, I32, P, P]
        L.orc_edge_free_geometric_f32.restype = I32
        L.orc_edge_free_di_f32.argtypes = [P, P, F32, I32, P, P, I32, P, P]
        L.orc_edge_free_di_f32.restype = I32
        L.orc_radius_thm1.argtypes = [I32, I32, F64, F64]; L.orc_radius_thm1.restype = F64
        L.orc_radius_halton.argtypes = [I32, I32, F64, F64]; L.orc_radius_halton.restype = F64
        L.orc_halton_unit.argtypes = [C.c_uint32, C.c_uint32]; L.orc_halton_unit.restype = F32
        L.orc_sample_halton.argtypes = [I32, I32, P, P, I32, P, P, P, P, F32, I32, I32, C.c_int64, P, P]
        L.orc_sample_halton.restype = I32
        L.orc_graph_build.argtypes = [I32, I32, I32, I32, I32, P, P, F32]; L.orc_graph_build.restype = P
        L.orc_graph_build_dubins.argtypes = [I32, I32, P, P, F32, F32]; L.orc_graph_build_dubins.restype = P
        L.orc_dubins_words.argtypes = [I32, P, P, F64, P]; L.orc_dubins_words.restype = I32
        L.orc_cost_dubins.argtypes = [I32, P, P, F64, F64]; L.orc_cost_dubins.restype = F64
        L.orc_dubins_point.argtypes = [I32, P, P, F64, F64, P]
        L.orc_dub_trig.argtypes = [I32, I32, I32, P, P, P, P]
        L.orc_edge_free_dubins_f32.argtypes = [P, P, F32, F32, F32, P, P, I32, P, P]
        L.orc_edge_free_dubins_f32.restype = I32
        L.orc_graph_free.argtypes = [I32, P]
        L.orc_graph_num_edges.argtypes = [I32, P]; L.orc_graph_num_edges.restype = I64
        L.orc_graph_copy.argtypes = [I32, P, P, P, P, P, P, P]
        L.orc_plan.argtypes = [I32, I32, P, I32, P, P, P, P, F32, F32, I32, I32, I32, P, P, P, P, P]
        L.orc_plan.restype = I32
        L.orc_dijkstra.argtypes = [I32, P, I32, P, P, P, P, F32, I32, P]; L.orc_dijkstra.restype = F64
        L.orc_graph_edge_free.argtypes = [I32, P, I32, I32, F64, I32, P, P, P, P, F32, I32]
        L.orc_graph_edge_free.restype = I32
        L.orc_count_edges_rows.argtypes = [I32, I32, I32, P, F32, I32, I32]
        L.orc_count_edges_rows.restype = I64
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# --------------------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def word_to_unit(w: int) -> float:
    return lib().orc_word_to_unit(int(w))


def cost_euclid(a, b, precision=32):
    if precision == 64:
        a = np.ascontiguousarray(a, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
        return lib().orc_cost_euclid_f64(_p(a), _p(b), len(a))
    a = _f32(a); b = _f32(b)
    return np.float32(lib().orc_cost_euclid_f32(_p(a), _p(b), len(a)))


def cost_di(s0, s1, r):
    """FP32 double-integrator cost J and arrival time tau (both +inf if no root in (0, r])."""
    s0 = _f32(s0); s1 = _f32(s1)
    tau = np.zeros(1, dtype=np.float32)
    J = lib().orc_cost_di_f32(_p(s0), _p(s1), np.float32(r), _p(tau))
    return np.float32(J), tau[0]


def cost_di_f64(s0, s1, span, grid=32, bisect=52):
    s0 = np.ascontiguousarray(s0, dtype=np.float64); s1 = np.ascontiguousarray(s1, dtype=np.float64)
    tau = np.zeros(1, dtype=np.float64)
    J = lib().orc_cost_di_f64(_p(s0), _p(s1), float(span), grid, bisect, _p(tau))
    return J, tau[0]


def di_coeffs_f64(s0, s1):
    s0 = np.ascontiguousarray(s0, dtype=np.float64); s1 = np.ascontiguousarray(s1, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_di_coeffs_f64(_p(s0), _p(s1), _p(out))
    return out


def hermite_point_f64(s0, s1, tau, s):
    s0 = np.ascontiguousarray(s0, dtype=np.float64); s1 = np.ascontiguousarray(s1, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_hermite_point_f64(_p(s0), _p(s1), float(tau), float(s), _p(out))
    return out


def edge_free_geometric(y, x, L, spacing, box_lo, box_hi):
    y = _f32(y); x = _f32(x); bl = _f32(box_lo); bh = _f32(box_hi)
    return bool(lib().orc_edge_free_geometric_f32(_p(y), _p(x), len(y), np.float32(L), np.float32(spacing),
                                                   bl.shape[0], _p(bl), _p(bh)))


def edge_free_di(y, x, tau, points, pos_lo, pos_hi, box_lo, box_hi):
    y = _f32(y); x = _f32(x); bl = _f32(box_lo).reshape(-1, 3); bh = _f32(box_hi).reshape(-1, 3)
    pl = _f32(pos_lo); ph = _f32(pos_hi)
    return bool(lib().orc_edge_free_di_f32(_p(y), _p(x), np.float32(tau), points, _p(pl), _p(ph),
                                            bl.shape[0], _p(bl), _p(bh)))


def radius_thm1(n: int, d: int, eta: float = 0.0, mu: float = 1.0) -> float:
    return lib().orc_radius_thm1(n, d, eta, mu)


def radius_halton(n: int, d: int, eta: float = 0.0, mu: float = 1.0) -> float:
    return lib().orc_radius_halton(n, d, eta, mu)


def halton_unit(k: int, p: int) -> float:
    return lib().orc_halton_unit(k, p)


def sample_halton(problem, max_candidates: int | None = None):
    """Halton SampleFree for a problem: (X [d][N] float32, is_goal [N] uint8)."""
    pb = problem
    d, dp, n = pb.d, pb.dp, pb.n
    N = n + 1
    X = np.zeros((d, N), dtype=np.float32)
    goal = np.zeros(N, dtype=np.uint8)
    lo, hi = _f32(pb.lo), _f32(pb.hi)
    bl, bh = _f32(pb.box_lo).reshape(-1, dp), _f32(pb.box_hi).reshape(-1, dp)
    xi, gc = _f32(pb.x_init), _f32(pb.goal_center)
    cap = max_candidates if max_candidates is not None else 64 * N + 65536
    st = lib().orc_sample_halton(d, dp, _p(lo), _p(hi), bl.shape[0], _p(bl), _p(bh), _p(xi), _p(gc),
                                 np.float32(pb.goal_radius), int(pb.goal_pos_only), n, cap, _p(X), _p(goal))
    if st != OK:
        raise ValueError(f"oracle Halton sampling failed with status {st}")
    return X, goal


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------- Dubins airplane
DUBINS_WORDS = ("LSL", "RSR", "LSR", "RSL", "RLR", "LRL")


def dubins_words(s0, s1, rho, precision=32):
    """All six Dubins words of the pair (x, y, z, theta) -> (x, y, z, theta):
    array [6][5] of (word, t, p, q, L) (+inf L where a word does not exist) and
    the index of the shortest.  precision 32 computes in float."""
    a, b = _f64(s0), _f64(s1)
    out = np.zeros((6, 5), np.float64)
    best = lib().orc_dubins_words(precision, _p(a), _p(b), float(rho), _p(out))
    return out, best


def cost_dubins(s0, s1, rho, r, precision=32):
    """Edge cost of s0 -> s1 (+inf when the distance prefilter rejects it)."""
    a, b = _f64(s0), _f64(s1)
    return lib().orc_cost_dubins(precision, _p(a), _p(b), float(rho), float(r))


def dubins_point(s0, s1, rho, s, precision=32):
    a, b = _f64(s0), _f64(s1)
    out = np.zeros(4, np.float64)
    lib().orc_dubins_point(precision, _p(a), _p(b), float(rho), float(s), _p(out))
    return out


def dub_trig(which, x, y=None, precision=32):
    """The oracle's own trigonometry over arrays: which 0 = (sin, cos) of x,
    1 = atan2(y, x), 2 = acos(x)."""
    x = _f64(x).ravel()
    y = _f64(y).ravel() if y is not None else np.zeros_like(x)
    o0, o1 = np.zeros_like(x), np.zeros_like(x)
    lib().orc_dub_trig(precision, which, x.size, _p(x), _p(y), _p(o0), _p(o1))
    return (o0, o1) if which == 0 else o0


def edge_free_dubins(s0, s1, c, rho, spacing, pos_lo, pos_hi, box_lo, box_hi):
    a, b = _f32(s0), _f32(s1)
    bl, bh = _f32(box_lo).reshape(-1, 3), _f32(box_hi).reshape(-1, 3)
    pl, ph = _f32(pos_lo), _f32(pos_hi)
    return bool(lib().orc_edge_free_dubins_f32(_p(a), _p(b), np.float32(c), np.float32(rho), np.float32(spacing),
                                               _p(pl), _p(ph), bl.shape[0], _p(bl), _p(bh)))


def in_goal(x, gd, c, rho):
    x = _f32(x); c = _f32(c)
    return bool(lib().orc_in_goal(_p(x), gd, _p(c), np.float32(rho)))


# --------------------------------------------------------------------------- problems
def sample(problem, stream: int = 0, max_attempts: int = 65536):
    """SampleFree for a problem (see paper_1705_02403_gb300.envgen.Problem).

    Returns (X [d][N] float32, is_goal [N] uint8)."""
    pb = problem
    d, dp, n = pb.d, pb.dp, pb.n
    N = n + 1
    X = np.zeros((d, N), dtype=np.float32)
    goal = np.zeros(N, dtype=np.uint8)
    lo, hi = _f32(pb.lo), _f32(pb.hi)
    bl, bh = _f32(pb.box_lo).reshape(-1, dp), _f32(pb.box_hi).reshape(-1, dp)
    xi, gc = _f32(pb.x_init), _f32(pb.goal_center)
    st = lib().orc_sample(d, dp, _p(lo), _p(hi), bl.shape[0], _p(bl), _p(bh), _p(xi), _p(gc),
                          np.float32(pb.goal_radius), int(pb.goal_pos_only), n, int(pb.seed), stream,
                          max_attempts, _p(X), _p(goal))
    if st != OK:
        raise ValueError(f"oracle sampling failed with status {st}")
    return X, goal


@dataclass
class CSR:
    out_row: np.ndarray
    out_col: np.ndarray
    out_cost: np.ndarray
    in_row: np.ndarray
    in_col: np.ndarray
    in_cost: np.ndarray


class Graph:
    """Brute-force r-disk neighbour graph of a sample set (FP32 or FP64)."""

    def __init__(self, kind, d, dp, X, goal, r, precision=32, rho=0.0):
        X = _f32(X)
        self.kind, self.d, self.dp, self.N, self.r, self.precision = kind, d, dp, X.shape[1], float(np.float32(r)), precision
        self.X, self.goal = X, np.ascontiguousarray(goal, dtype=np.uint8)
        if kind == DUBINS:
            if (d, dp) != (4, 3) or not rho > 0:
                raise ValueError("Dubins airplane graphs need d = 4, dp = 3 and a turning radius > 0")
            self._h = lib().orc_graph_build_dubins(precision, self.N, _p(X), _p(self.goal), np.float32(r),
                                                   np.float32(rho))
        else:
            self._h = lib().orc_graph_build(precision, kind, d, dp, self.N, _p(X), _p(self.goal), np.float32(r))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_graph_free(self.precision, h)
            self._h = None

    @property
    def num_edges(self) -> int:
        return lib().orc_graph_num_edges(self.precision, self._h)

    def csr(self) -> CSR:
        E, N = self.num_edges, self.N
        a = [np.zeros(N + 1, np.int32), np.zeros(E, np.int32), np.zeros(E, np.float64),
             np.zeros(N + 1, np.int32), np.zeros(E, np.int32), np.zeros(E, np.float64)]
        lib().orc_graph_copy(self.precision, self._h, *[_p(x) for x in a])
        if self.precision == 32:
            a[2] = a[2].astype(np.float32)
            a[5] = a[5].astype(np.float32)
        return CSR(*a)

    def _boxargs(self, box_lo, box_hi, pos_lo, pos_hi):
        bl = _f32(box_lo).reshape(-1, self.dp); bh = _f32(box_hi).reshape(-1, self.dp)
        pl = _f32(pos_lo); ph = _f32(pos_hi)
        return bl, bh, pl, ph

    def plan(self, box_lo, box_hi, pos_lo, pos_hi, lam, seg_spacing=0.005, traj_points=20,
             skip_empty=True, max_iters=None, which="gmt", trace=False):
        """Run GMT* (Alg. 1) or FMT*.  Returns (parent, cost, info) and, with
        trace=True, also (added_i, closed_i) per node."""
        bl, bh, pl, ph = self._boxargs(box_lo, box_hi, pos_lo, pos_hi)
        parent = np.zeros(self.N, np.int32)
        cost = np.zeros(self.N, np.float64)
        info = Info()
        added = np.zeros(self.N, np.int64) if trace else None
        closed = np.zeros(self.N, np.int64) if trace else None
        lib().orc_plan(self.precision, 0 if which == "gmt" else 1, self._h, bl.shape[0], _p(bl), _p(bh), _p(pl),
                       _p(ph), np.float32(lam), np.float32(seg_spacing), traj_points, int(skip_empty),
                       int(max_iters if max_iters is not None else self.N + 1), _p(parent), _p(cost),
                       C.byref(info), _p(added), _p(closed))
        if self.precision == 32:
            cost = cost.astype(np.float32)
        if trace:
            return parent, cost, info.as_dict(), added, closed
        return parent, cost, info.as_dict()

    def dijkstra(self, box_lo, box_hi, pos_lo, pos_hi, seg_spacing=0.005, traj_points=20):
        bl, bh, pl, ph = self._boxargs(box_lo, box_hi, pos_lo, pos_hi)
        dist = np.zeros(self.N, np.float64)
        best = lib().orc_dijkstra(self.precision, self._h, bl.shape[0], _p(bl), _p(bh), _p(pl), _p(ph),
                                  np.float32(seg_spacing), traj_points, _p(dist))
        return best, dist

    def edge_free(self, y, x, c, box_lo, box_hi, pos_lo, pos_hi, seg_spacing=0.005, traj_points=20):
        bl, bh, pl, ph = self._boxargs(box_lo, box_hi, pos_lo, pos_hi)
        return bool(lib().orc_graph_edge_free(self.precision, self._h, int(y), int(x), float(c), bl.shape[0],
                                              _p(bl), _p(bh), _p(pl), _p(ph), np.float32(seg_spacing),
                                              traj_points))


def count_edges_rows(problem, X, row0, row1):
    """Edges leaving nodes row0..row1-1 (a slice of the neighbour-set build)."""
    X = _f32(X)
    if problem.kind == DUBINS:
        raise ValueError("count_edges_rows covers the Euclidean and double-integrator costs")
    return lib().orc_count_edges_rows(problem.kind, problem.d, X.shape[1], _p(X), np.float32(problem.r), row0, row1)


def graph_for(problem, X=None, goal=None, precision=32):
    if X is None:
        X, goal = sample(problem)
    return Graph(problem.kind, problem.d, problem.dp, X, goal, problem.r, precision, rho=getattr(problem, "rho", 0.0))


def plan_problem(problem, X=None, goal=None, precision=32, **kw):
    g = graph_for(problem, X, goal, precision)
    parent, cost, info = g.plan(problem.box_lo, problem.box_hi, problem.lo[:problem.dp], problem.hi[:problem.dp],
                                problem.lam, problem.seg_spacing, problem.traj_points, **kw)
    return g, parent, cost, info


def path_to(parent, goal_node):
    """Walk parent pointers from the goal node back to node 0."""
    if goal_node < 0:
        return []
    path = [int(goal_node)]
    while path[-1] != 0:
        path.append(int(parent[path[-1]]))
        if len(path) > len(parent) + 1:
            raise RuntimeError("cycle in parent array")
    return path[::-1]
