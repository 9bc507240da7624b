"""Pins of the oracle's connection costs (Euclidean; double integrator)."""
import numpy as np
import pytest
from scipy.integrate import quad
from scipy.linalg import expm
from scipy.optimize import minimize_scalar

F = np.float32


def test_euclid_matches_numpy_and_is_symmetric(O):
    rng = np.random.default_rng(0)
    for d in (2, 3, 6, 10):
        for _ in range(200):
            a, b = rng.random(d, dtype=np.float32), rng.random(d, dtype=np.float32)
            c = O.cost_euclid(a, b)
            assert c == O.cost_euclid(b, a)          # bitwise symmetric
            ref = np.linalg.norm(a.astype(np.float64) - b.astype(np.float64))
            assert abs(float(c) - ref) <= 2e-7 * max(ref, 1e-30) + 1e-12
            assert O.cost_euclid(a, b, 64) == pytest.approx(ref, rel=1e-14)


def rand_state(rng):
    return np.concatenate([rng.random(3), rng.uniform(-1, 1, 3)])


def test_di_closed_form_at_rest(O):
    # v0 = v1 = 0: tau* = sqrt(6 |dp|), J = (4/3) tau*.
    rng = np.random.default_rng(1)
    for _ in range(50):
        p0, p1 = rng.random(3), rng.random(3)
        s0 = np.r_[p0, 0, 0, 0]; s1 = np.r_[p1, 0, 0, 0]
        L = np.linalg.norm(p1 - p0)
        tau = np.sqrt(6 * L)
        J64, t64 = O.cost_di_f64(s0, s1, span=10.0, grid=64, bisect=60)
        assert t64 == pytest.approx(tau, rel=1e-12)
        assert J64 == pytest.approx(4 * tau / 3, rel=1e-12)
        J32, t32 = O.cost_di(s0.astype(F), s1.astype(F), 8.0)
        ref = 4 * np.sqrt(6 * np.linalg.norm(s1[:3].astype(F).astype(float) - s0[:3].astype(F).astype(float))) / 3
        assert float(J32) == pytest.approx(ref, rel=2e-6)


def test_di_closed_form_same_velocity(O):
    # dp = 0, v0 = v1 = v: tau* = sqrt(12) |v|, J = 4 sqrt(3) |v|.
    rng = np.random.default_rng(2)
    for _ in range(50):
        p = rng.random(3); v = rng.uniform(-1, 1, 3)
        s = np.r_[p, v]
        J64, t64 = O.cost_di_f64(s, s, span=10.0, grid=64, bisect=60)
        assert t64 == pytest.approx(np.sqrt(12) * np.linalg.norm(v), rel=1e-12)
        assert J64 == pytest.approx(4 * np.sqrt(3) * np.linalg.norm(v), rel=1e-12)


def gramian_J(s0, s1, tau):
    """tau + d^T G(tau)^-1 d with G built by numerical quadrature of
    e^{As} B B^T e^{A^T s} (per axis, A = [[0,1],[0,0]], B = [0,1]^T) and
    d = x1 - e^{A tau} x0: the minimum control effort of a linear system."""
    A = np.array([[0.0, 1.0], [0.0, 0.0]])
    B = np.array([[0.0], [1.0]])
    G = np.zeros((2, 2))
    for i in range(2):
        for j in range(2):
            G[i, j] = quad(lambda s: (expm(A * s) @ B @ B.T @ expm(A.T * s))[i, j], 0, tau, epsabs=1e-13, epsrel=1e-13)[0]
    Phi = expm(A * tau)
    e = 0.0
    for ax in range(3):
        x0 = np.array([s0[ax], s0[3 + ax]]); x1 = np.array([s1[ax], s1[3 + ax]])
        dd = x1 - Phi @ x0
        e += dd @ np.linalg.solve(G, dd)
    return tau + e


def test_di_J_matches_gramian(O):
    rng = np.random.default_rng(3)
    for _ in range(12):
        s0, s1 = rand_state(rng), rand_state(rng)
        abc = O.di_coeffs_f64(s0, s1)
        for tau in (0.3, 1.1, 2.7):
            J_formula = tau + abc[0] / tau - abc[1] / tau ** 2 + abc[2] / tau ** 3
            assert J_formula == pytest.approx(gramian_J(s0, s1, tau), rel=1e-8)


def test_di_tau_is_minimiser_on_dense_scan(O):
    # The smallest positive root of the quartic is a local minimiser of J; it is
    # the global one for almost every pair.  J >= the scanned global minimum
    # always; equal (to 1e-9 rel) for >= 98% of pairs.
    rng = np.random.default_rng(4)
    agree = 0
    M = 300
    for _ in range(M):
        s0, s1 = rand_state(rng), rand_state(rng)
        abc = O.di_coeffs_f64(s0, s1)
        Jf = lambda t: t + abc[0] / t - abc[1] / t ** 2 + abc[2] / t ** 3
        grid = np.linspace(1e-3, 12.0, 24000)
        k = int(np.argmin(Jf(grid)))
        res = minimize_scalar(Jf, bounds=(grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]), method="bounded",
                              options={"xatol": 1e-13})
        J64, _ = O.cost_di_f64(s0, s1, span=12.0, grid=2048, bisect=60)
        assert J64 >= res.fun * (1 - 1e-9)
        if abs(J64 - res.fun) <= 1e-9 * res.fun:
            agree += 1
    assert agree >= 0.98 * M


def test_di_fp32_close_to_fp64(O):
    rng = np.random.default_rng(5)
    r = F(2.428)
    n = 0
    while n < 300:
        s0, s1 = rand_state(rng).astype(F), rand_state(rng).astype(F)
        J32, t32 = O.cost_di(s0, s1, r)
        if not np.isfinite(J32) or J32 >= r:
            continue
        J64, t64 = O.cost_di_f64(s0.astype(float), s1.astype(float), float(r), 32, 52)
        assert float(J32) == pytest.approx(J64, rel=1e-5)
        n += 1


def test_di_hermite_is_the_min_effort_trajectory(O):
    # The oracle's Hermite position curve must start/end at p0/p1 with
    # velocities v0/v1 (in time t = s tau), and its control effort
    # int ||p''(t)||^2 dt must equal J(tau) - tau.
    rng = np.random.default_rng(6)
    for _ in range(20):
        s0, s1 = rand_state(rng), rand_state(rng)
        tau = rng.uniform(0.3, 3.0)
        ss = np.array([0.0, 1 / 3, 2 / 3, 1.0])
        pts = np.array([O.hermite_point_f64(s0, s1, tau, s) for s in ss])
        coef = [np.polyfit(ss, pts[:, a], 3) for a in range(3)]
        assert np.allclose(pts[0], s0[:3], atol=1e-14) and np.allclose(pts[-1], s1[:3], atol=1e-14)
        for a in range(3):
            d1 = np.polyder(coef[a])
            assert np.polyval(d1, 0.0) / tau == pytest.approx(s0[3 + a], abs=1e-9)
            assert np.polyval(d1, 1.0) / tau == pytest.approx(s1[3 + a], abs=1e-9)
        effort = 0.0
        for a in range(3):
            d2 = np.polyder(coef[a], 2)
            sq = np.polyint(np.polymul(d2, d2))
            effort += (np.polyval(sq, 1.0) - np.polyval(sq, 0.0)) / tau ** 3
        abc = O.di_coeffs_f64(s0, s1)
        assert effort == pytest.approx(abc[0] / tau - abc[1] / tau ** 2 + abc[2] / tau ** 3, rel=1e-8)


def test_di_no_edge_when_no_root_in_range(O):
    s0 = np.array([0.0, 0, 0, 0, 0, 0], F)
    s1 = np.array([1.0, 1, 1, 0, 0, 0], F)   # tau* = sqrt(6 sqrt 3) = 3.22
    J, tau = O.cost_di(s0, s1, F(2.0))
    assert np.isinf(J) and np.isinf(tau)
    J, tau = O.cost_di(s0, s1, F(4.5))
    assert float(tau) == pytest.approx(np.sqrt(6 * np.sqrt(3)), rel=1e-6)


def test_radius_thm1_closed_forms(O):
    for n in (512, 1000, 16384):
        r2 = 4 * np.sqrt(0.5) * np.sqrt(1 / np.pi) * np.sqrt(np.log(n) / n)
        assert O.radius_thm1(n, 2) == pytest.approx(r2, rel=1e-13)
        r3 = 4 * (1 / 3) ** (1 / 3) * (1 / (4 * np.pi / 3)) ** (1 / 3) * (np.log(n) / n) ** (1 / 3)
        assert O.radius_thm1(n, 3) == pytest.approx(r3, rel=1e-13)
        assert O.radius_thm1(n, 2, eta=1.0, mu=0.5) == pytest.approx(r2 * (2 * 0.5) ** 0.5, rel=1e-13)
