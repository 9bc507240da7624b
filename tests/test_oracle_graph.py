"""Pins of the oracle's r-disk neighbour graph (Section III-A: neighbours are
samples whose connection cost is below r)."""
import numpy as np
from scipy.spatial import cKDTree

from paper_1705_02403_gb300 import envgen

F = np.float32


def check_csr_shape(csr, N):
    assert csr.out_row[0] == 0 and csr.in_row[0] == 0
    assert np.all(np.diff(csr.out_row) >= 0) and np.all(np.diff(csr.in_row) >= 0)
    for v in range(N):
        row = csr.out_col[csr.out_row[v]:csr.out_row[v + 1]]
        assert np.all(np.diff(row) > 0) and v not in row
        row = csr.in_col[csr.in_row[v]:csr.in_row[v + 1]]
        assert np.all(np.diff(row) > 0) and v not in row


def edge_set(csr, N):
    s = {}
    for v in range(N):
        for e in range(csr.out_row[v], csr.out_row[v + 1]):
            s[(v, int(csr.out_col[e]))] = csr.out_cost[e]
    return s


def test_euclid_graph_matches_kdtree(O):
    for seed, d in [(0, 2), (1, 3), (2, 2)]:
        pb = envgen.geometric(seed, d=d, n=800, nbox=5, r=0.15 if d == 2 else 0.25)
        X, goal = O.sample(pb)
        g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, pb.r)
        csr = g.csr()
        check_csr_shape(csr, g.N)
        E = edge_set(csr, g.N)
        P = X.T.astype(np.float64)
        tree = cKDTree(P)
        inner = tree.query_pairs(pb.r - 1e-6)
        outer = tree.query_pairs(pb.r + 1e-6)
        und = {(min(i, j), max(i, j)) for (i, j) in E}
        assert {(i, j) for i, j in inner} <= und <= {(i, j) for i, j in outer}
        # symmetric cost, in-arrays equal out-arrays
        for (i, j), c in E.items():
            assert E[(j, i)] == c
        assert np.array_equal(csr.in_row, csr.out_row) and np.array_equal(csr.in_col, csr.out_col)
        assert np.array_equal(csr.in_cost, csr.out_cost)


def test_di_graph_matches_pairwise_costs(O):
    pb = envgen.di6(seed=3, n=60)
    X, goal = O.sample(pb)
    r = F(1.6)
    g = O.Graph(pb.kind, pb.d, pb.dp, X, goal, r)
    csr = g.csr()
    check_csr_shape(csr, g.N)
    E = edge_set(csr, g.N)
    count = 0
    for i in range(g.N):
        for j in range(g.N):
            if i == j:
                continue
            J, _ = O.cost_di(X[:, i], X[:, j], r)
            if J < r:
                assert E[(i, j)] == J
                count += 1
            else:
                assert (i, j) not in E
    assert count == len(E) > 0
    # the cost is not symmetric, and the in-CSR is the transpose of the out-CSR
    assert any((j, i) not in E for (i, j) in E)
    for v in range(g.N):
        for e in range(csr.in_row[v], csr.in_row[v + 1]):
            assert E[(int(csr.in_col[e]), v)] == csr.in_cost[e]
    assert len(csr.in_col) == len(csr.out_col)


def test_neighbour_predicate_is_strict(O):
    # Section III-A: neighbours have connection cost *less than* r.  Dyadic
    # points at exactly r = 0.25 apart are not neighbours; 0.1875 apart are.
    X = np.array([[0.0, 0.25, 0.0], [0.0, 0.0, 0.1875]], F)
    g = O.Graph(0, 2, 2, X, np.zeros(3, np.uint8), 0.25)
    csr = g.csr()
    E = edge_set(csr, 3)
    assert (0, 1) not in E and (1, 0) not in E
    assert E[(0, 2)] == F(0.1875) and E[(2, 0)] == F(0.1875)
