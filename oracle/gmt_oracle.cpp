// GMT* CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of what the Group Marching Tree
// hot path computes (Ichter, Schmerling, Pavone, "Group Marching Tree:
// Sampling-Based Approximately Optimal Motion Planning on GPUs", 2017).
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
// load this library.  It shares no code, header, table or constant generator
// with the CUDA path under paper_1705_02403_gb300/csrc/, and includes none of
// its files.
//
// Compile with IEEE semantics and no contraction:
//   g++ -std=c++17 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC
//
// Every function is templated on the real type R (float for the bit-exact
// parity path, double for the FP64 rerun).  Evaluation order of every
// floating-point expression is written out explicitly (left to right) and
// stated in the comment above it; the GPU path follows the same readings.
//
// Pins (what checks this file against something other than itself) live in
// tests/test_oracle_*.py:
//   philox4x32_10   -> Triton's Philox run in its CPU interpreter (library)
//   sample_free     -> invariants, chi^2 uniformity, independent rebuild
//   cost_euclid     -> numpy float64 norm, bitwise symmetry
//   cost_di         -> closed forms, dense FP64 scan of J, Hermite quadrature,
//                      Gramian built by numerical integration
//   edge_free       -> exact slab segment/box test (superset detector),
//                      hand-placed boxes
//   build_graph     -> scipy cKDTree pair query (Euclidean), brute force
//   gmt_plan        -> hand-traced graphs, skip == stepping, lambda=0 == heap
//                      FMT*, Dijkstra lower bound, (1+2 lambda) upper bound
//                      without obstacles (Theorem 2), tree invariants
//   fmt_plan        -> hand-traced graph, Dijkstra lower bound
//   dijkstra        -> scipy.sparse.csgraph.dijkstra
//   radius_thm1     -> closed form of Theorem 1 for d = 2, 3

#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>
#include <queue>
#include <limits>
#include <algorithm>

namespace {

enum { ORC_OK = 0, ORC_NO_PATH = 1, ORC_ERR_INVALID = -1, ORC_ERR_ITER_LIMIT = -5 };
enum { ORC_EUCLID = 0, ORC_DI = 1, ORC_DUBINS = 2 };
enum { UNEXPLORED = 0, OPEN = 1, CLOSED = 2 };
const int MAXD = 12;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers:
// as easy as 1, 2, 3").  One round maps the counter (c0,c1,c2,c3) with key
// (k0,k1) to (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)) with the
// round multipliers A = 0xD2511F53, B = 0xCD9E8D57; between rounds the key is
// bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t A = 0xD2511F53u, B = 0xCD9E8D57u;
    const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)A * (uint64_t)c0;
        uint64_t pb = (uint64_t)B * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += WA; k1 += WB;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// A 32-bit Philox word becomes a float in [0,1): its top 24 bits times 2^-24
// (exact in FP32).
float word_to_unit(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------------------
// Obstacles: a union of closed axis-aligned boxes in position space
// (Section V-B: obstacles are unions of axis-aligned bounding boxes).
// ---------------------------------------------------------------------------
struct Boxes {
    int count, dp;
    const float* lo;  // [count][dp]
    const float* hi;  // [count][dp]
};

template <typename R>
bool point_in_obstacle(const R* p, const Boxes& B) {
    for (int b = 0; b < B.count; ++b) {
        bool inside = true;
        for (int a = 0; a < B.dp; ++a) {
            R l = (R)B.lo[b * B.dp + a], h = (R)B.hi[b * B.dp + a];
            if (!(l <= p[a] && p[a] <= h)) { inside = false; break; }
        }
        if (inside) return true;
    }
    return false;
}

// Goal region: a closed ball of radius rho around c, over the position axes
// only (pos_only) or over the whole state.  Membership: sum over axes, in
// axis order starting from 0, of (x_a - c_a)^2, compared <= rho*rho.
bool in_goal(const float* x, int gd, const float* c, float rho) {
    float s = 0.0f;
    for (int a = 0; a < gd; ++a) {
        float t = x[a] - c[a];
        s = s + t * t;
    }
    return s <= rho * rho;
}

// ---------------------------------------------------------------------------
// Connection costs.
// ---------------------------------------------------------------------------

// Euclidean arc length (Section II): c = sqrt(((dx0*dx0)+dx1*dx1)+...),
// dx_a = x_to[a] - x_from[a], summed in axis order from 0.
template <typename R>
R cost_euclid(const R* from, const R* to, int d) {
    R s = 0;
    for (int a = 0; a < d; ++a) {
        R t = to[a] - from[a];
        s = s + t * t;
    }
    return std::sqrt(s);
}

// Double integrator xdd = u in 3 axes, cost = arrival time tau plus control
// effort, the "mixed time / quadratic control effort" cost of Section V-A.
// For fixed tau the minimum-effort control gives
//   J(tau) = tau + a/tau - b/tau^2 + c/tau^3,
//   a = 4(|v0|^2 + v0.v1 + |v1|^2), b = 12 dp.(v0+v1), c = 12 |dp|^2,
// and dJ/dtau = 0 is the quartic q(tau) = tau^4 - a tau^2 + 2b tau - 3c.
// The optimal arrival time is the smallest positive root of q, bracketed on the
// grid tau_k = r*(k/G), k = 1..G (first k with q(tau_k) >= 0; none -> no edge,
// because J(tau) >= tau), then refined by `bisect` halvings of
// [tau_{k-1}, tau_k] (mid = lo + (hi-lo)*0.5; q(mid) < 0 -> lo = mid else hi =
// mid; tau* = hi).  q is evaluated as ((tau*tau - a)*tau + 2b)*tau - 3c with
// 2b = 2*b and 3c = 3*c rounded once each; J as ((c/tau - b)/tau + a)/tau + tau.
// State layout: [p0 p1 p2 v0 v1 v2].
template <typename R>
struct DICoeffs { R a, b, c, b2, c3; };

template <typename R>
DICoeffs<R> di_coeffs(const R* s0, const R* s1) {
    R n00 = 0, n01 = 0, n11 = 0, bs = 0, cs = 0;
    for (int ax = 0; ax < 3; ++ax) {
        R p0 = s0[ax], v0 = s0[3 + ax], p1 = s1[ax], v1 = s1[3 + ax];
        R dp = p1 - p0;
        n00 = n00 + v0 * v0;
        n01 = n01 + v0 * v1;
        n11 = n11 + v1 * v1;
        bs = bs + dp * (v0 + v1);
        cs = cs + dp * dp;
    }
    DICoeffs<R> k;
    k.a = (R)4 * ((n00 + n01) + n11);
    k.b = (R)12 * bs;
    k.c = (R)12 * cs;
    k.b2 = (R)2 * k.b;
    k.c3 = (R)3 * k.c;
    return k;
}

template <typename R>
R di_quartic(const DICoeffs<R>& k, R t) { return ((t * t - k.a) * t + k.b2) * t - k.c3; }

template <typename R>
R di_J(const DICoeffs<R>& k, R t) { return ((k.c / t - k.b) / t + k.a) / t + t; }

// Returns J (+inf when no root lies in (0, span]) and the arrival time.
template <typename R>
R cost_di(const R* s0, const R* s1, R span, int grid, int bisect, R* tau_out) {
    DICoeffs<R> k = di_coeffs(s0, s1);
    R prev = 0;
    int found = 0;
    R t_hi = 0;
    for (int g = 1; g <= grid; ++g) {
        R tg = span * ((R)g / (R)grid);
        if (di_quartic(k, tg) >= (R)0) { found = g; t_hi = tg; break; }
        prev = tg;
    }
    if (!found) { if (tau_out) *tau_out = std::numeric_limits<R>::infinity(); return std::numeric_limits<R>::infinity(); }
    R lo = prev, hi = t_hi;
    for (int s = 0; s < bisect; ++s) {
        R mid = lo + (hi - lo) * (R)0.5;
        if (di_quartic(k, mid) < (R)0) lo = mid; else hi = mid;
    }
    if (tau_out) *tau_out = hi;
    return di_J(k, hi);
}

const int DI_GRID = 32;
template <typename R> int di_bisect_steps();
template <> int di_bisect_steps<float>() { return 24; }
template <> int di_bisect_steps<double>() { return 52; }

// ---------------------------------------------------------------------------
// Dubins airplane (Sec. V-A): a planar Dubins car of turning radius rho with a
// single integrator in altitude (unbounded climb rate) and the Euclidean
// length of the trajectory as cost.  State (x, y, z, theta).  Reading: the
// trajectory follows the shortest planar Dubins path (the best of the words
// LSL, RSR, LSR, RSL, RLR, LRL; Dubins 1957) with altitude linear in planar arc
// length, so its length is sqrt(L^2 + dz^2) with L the planar path length: the
// shortest trajectory, because any altitude profile over a planar path of
// length L is at least that long and the bound grows with L.
//
// Sine, cosine and arctangent are this file's own (range reduction and Taylor
// series evaluated in a fixed order), so results do not depend on a math
// library; the float and double instantiations use their own constants.
// ---------------------------------------------------------------------------
template <typename R> struct DubK;
template <> struct DubK<float> {
    static constexpr float pi = 3.14159265358979f, two_pi = 6.28318530717959f, pi_2 = 1.57079632679490f,
                           pi_4 = 0.785398163397448f;
    static constexpr float pi_2_hi = 1.57079637050628662109375f;  // fl(pi/2)
    static constexpr float pi_2_lo = -4.37113900018624e-8f;       // pi/2 - fl(pi/2)
    static constexpr float two_over_pi = 0.636619772367581f, tan_pi_8 = 0.414213562373095f;
};
template <> struct DubK<double> {
    static constexpr double pi = 3.14159265358979323846, two_pi = 6.28318530717958647692,
                            pi_2 = 1.57079632679489661923, pi_4 = 0.785398163397448309616;
    static constexpr double pi_2_hi = 1.57079632679489655800;  // fl64(pi/2)
    static constexpr double pi_2_lo = 6.12323399573676603587e-17;
    static constexpr double two_over_pi = 0.636619772367581343076, tan_pi_8 = 0.414213562373095048802;
};

// sin r, cos r for |r| <= pi/4 (+ rounding): Taylor polynomials through r^11
// and r^12, Horner form.
template <typename R> R dub_sin_poly(R r) {
    const R r2 = r * r;
    return r + r * (r2 * ((R)(-1.0 / 6) + r2 * ((R)(1.0 / 120) + r2 * ((R)(-1.0 / 5040) +
                    r2 * ((R)(1.0 / 362880) + r2 * (R)(-1.0 / 39916800))))));
}
template <typename R> R dub_cos_poly(R r) {
    const R r2 = r * r;
    return (R)1 + r2 * ((R)(-1.0 / 2) + r2 * ((R)(1.0 / 24) + r2 * ((R)(-1.0 / 720) +
                  r2 * ((R)(1.0 / 40320) + r2 * ((R)(-1.0 / 3628800) + r2 * (R)(1.0 / 479001600))))));
}
// x = k pi/2 + r with k the nearest integer to 2x/pi (ties to even); the
// quadrant k mod 4 picks +-sin r or +-cos r.
template <typename R> void dub_sincos(R x, R* s, R* c) {
    const R kf = std::nearbyint(x * DubK<R>::two_over_pi);
    const R r = (x - kf * DubK<R>::pi_2_hi) - kf * DubK<R>::pi_2_lo;
    const R sr = dub_sin_poly(r), cr = dub_cos_poly(r);
    const int q = (int)((long long)kf & 3);
    if (q == 0) { *s = sr; *c = cr; }
    else if (q == 1) { *s = cr; *c = -sr; }
    else if (q == 2) { *s = -sr; *c = -cr; }
    else { *s = -cr; *c = sr; }
}
template <typename R> R dub_cos(R x) { R s, c; dub_sincos(x, &s, &c); return c; }
// atan z, 0 <= z <= 1: above tan(pi/8), atan z = pi/4 + atan u with
// u = (z - 1)/(z + 1); then the series u - u^3/3 + u^5/5 - ... through u^21
// (|u| <= tan(pi/8)).
template <typename R> R dub_atan01(R z) {
    R base = 0, u = z;
    if (z > DubK<R>::tan_pi_8) { base = DubK<R>::pi_4; u = (z - (R)1) / (z + (R)1); }
    const R u2 = u * u;
    R poly = (R)(-1.0 / 21);
    poly = (R)(1.0 / 19) + u2 * poly;
    poly = (R)(-1.0 / 17) + u2 * poly;
    poly = (R)(1.0 / 15) + u2 * poly;
    poly = (R)(-1.0 / 13) + u2 * poly;
    poly = (R)(1.0 / 11) + u2 * poly;
    poly = (R)(-1.0 / 9) + u2 * poly;
    poly = (R)(1.0 / 7) + u2 * poly;
    poly = (R)(-1.0 / 5) + u2 * poly;
    poly = (R)(1.0 / 3) + u2 * poly;
    poly = -(u2 * poly);
    return base + (u + u * poly);
}
// Angle of (x, y) in (-pi, pi]; (0, 0) -> 0.
template <typename R> R dub_atan2(R y, R x) {
    const R ax = std::fabs(x), ay = std::fabs(y);
    if (ax == (R)0 && ay == (R)0) return 0;
    R a = ay <= ax ? dub_atan01(ay / ax) : DubK<R>::pi_2 - dub_atan01(ax / ay);
    if (x < (R)0) a = DubK<R>::pi - a;
    return y < (R)0 ? -a : a;
}
template <typename R> R dub_acos(R x) { return dub_atan2(std::sqrt(((R)1 - x) * ((R)1 + x)), x); }
template <typename R> R dub_mod2pi(R a) { return a - DubK<R>::two_pi * std::floor(a / DubK<R>::two_pi); }
// An end turn (t or q) within 2^-13 of a full circle is the small negative
// turn it differs by: a full loop is never part of a shortest path, and the
// turn is that close to 2 pi only when its exact value is a rounding error
// away from 0.
template <typename R> R dub_end_turn(R a) {
    return a > DubK<R>::two_pi - (R)(1.0 / 8192) ? a - DubK<R>::two_pi : a;
}

enum { DUB_LSL = 0, DUB_RSR, DUB_LSR, DUB_RSL, DUB_RLR, DUB_LRL, DUB_NONE };

template <typename R>
struct DubinsPath { int word; R t, p, q; R L; };   // t, p, q: segment lengths / rho; L = rho ((t + p) + q)

// Lengths of all six words (+inf where a word does not exist), in the order of
// the enum.  Frame: the line from start to end, scaled by 1/rho: the start is
// at the origin with heading alpha, the end at (d, 0) with heading beta.  A CSC
// word's straight part is the common tangent of its two turning circles; a CCC
// word's middle circle touches both (it exists only for circles at most 4 rho
// apart).
template <typename R>
void dubins_words(R x0, R y0, R th0, R x1, R y1, R th1, R rho, DubinsPath<R> out[6]) {
    const R dx = x1 - x0, dy = y1 - y0;
    const R D = std::sqrt(dx * dx + dy * dy);
    const R d = D / rho;
    const R phi = dub_atan2(dy, dx);
    const R al = dub_mod2pi(th0 - phi), be = dub_mod2pi(th1 - phi);
    R sa, ca, sb, cb;
    dub_sincos(al, &sa, &ca);
    dub_sincos(be, &sb, &cb);
    const R cab = dub_cos(al - be);
    const R dd = d * d;
    const R inf = std::numeric_limits<R>::infinity();
    for (int w = 0; w < 6; ++w) out[w] = DubinsPath<R>{w, 0, 0, 0, inf};
    auto set = [&](int w, R t, R p, R q) {
        t = dub_end_turn(t);
        q = dub_end_turn(q);
        out[w] = DubinsPath<R>{w, t, p, q, ((t + p) + q) * rho};
    };
    {   // LSL
        const R p2 = (((R)2 + dd) - (R)2 * cab) + ((R)2 * d) * (sa - sb);
        if (p2 >= (R)0) {
            const R psi = dub_atan2(cb - ca, (d + sa) - sb);
            set(DUB_LSL, dub_mod2pi(psi - al), std::sqrt(p2), dub_mod2pi(be - psi));
        }
    }
    {   // RSR
        const R p2 = (((R)2 + dd) - (R)2 * cab) + ((R)2 * d) * (sb - sa);
        if (p2 >= (R)0) {
            const R psi = dub_atan2(ca - cb, (d - sa) + sb);
            set(DUB_RSR, dub_mod2pi(al - psi), std::sqrt(p2), dub_mod2pi(psi - be));
        }
    }
    {   // LSR
        const R p2 = ((dd - (R)2) + (R)2 * cab) + ((R)2 * d) * (sa + sb);
        if (p2 >= (R)0) {
            const R p = std::sqrt(p2);
            const R psi = dub_atan2(-ca - cb, (d + sa) + sb) - dub_atan2((R)-2, p);
            set(DUB_LSR, dub_mod2pi(psi - al), p, dub_mod2pi(psi - be));
        }
    }
    {   // RSL
        const R p2 = ((dd - (R)2) + (R)2 * cab) - ((R)2 * d) * (sa + sb);
        if (p2 >= (R)0) {
            const R p = std::sqrt(p2);
            const R psi = dub_atan2(ca + cb, (d - sa) - sb) - dub_atan2((R)2, p);
            set(DUB_RSL, dub_mod2pi(al - psi), p, dub_mod2pi(be - psi));
        }
    }
    {   // RLR
        const R c = ((((R)6 - dd) + (R)2 * cab) + ((R)2 * d) * (sa - sb)) / (R)8;
        if (std::fabs(c) <= (R)1) {
            const R p = dub_mod2pi(DubK<R>::two_pi - dub_acos(c));
            const R t = dub_mod2pi((al - dub_atan2(ca - cb, (d - sa) + sb)) + p / (R)2);
            set(DUB_RLR, t, p, dub_mod2pi(((al - be) - t) + p));
        }
    }
    {   // LRL
        const R c = ((((R)6 - dd) + (R)2 * cab) + ((R)2 * d) * (sb - sa)) / (R)8;
        if (std::fabs(c) <= (R)1) {
            const R p = dub_mod2pi(DubK<R>::two_pi - dub_acos(c));
            const R t = dub_mod2pi(((-al) - dub_atan2(ca - cb, (d + sa) - sb)) + p / (R)2);
            set(DUB_LRL, t, p, dub_mod2pi(((be - al) - t) + p));
        }
    }
}

// The shortest word (ties: the earliest in enum order).
template <typename R>
DubinsPath<R> dubins_path(const R* s0, const R* s1, R rho) {
    DubinsPath<R> w[6];
    dubins_words(s0[0], s0[1], s0[3], s1[0], s1[1], s1[3], rho, w);
    DubinsPath<R> best{DUB_NONE, 0, 0, 0, std::numeric_limits<R>::infinity()};
    for (int k = 0; k < 6; ++k)
        if (w[k].L < best.L) best = w[k];
    return best;
}

// Prefilter: the cost is at least the 3D distance, so a pair whose squared
// distance reaches (1 + 2^-6) r^2 has no edge; the margin keeps the test from
// deciding any pair the rounded cost could put below r.
template <typename R>
bool dubins_near(const R* s0, const R* s1, R r) {
    const R dx = s1[0] - s0[0], dy = s1[1] - s0[1], dz = s1[2] - s0[2];
    return ((dx * dx + dy * dy) + dz * dz) < (r * r) * (R)1.015625;
}

template <typename R>
R cost_dubins(const R* s0, const R* s1, R rho) {
    const DubinsPath<R> P = dubins_path(s0, s1, rho);
    const R dz = s1[2] - s0[2];
    return std::sqrt(P.L * P.L + dz * dz);
}

// Pose at fraction s of the trajectory: planar arc length ell = s L walked
// through the word's segments (a left turn by angle a from heading th moves by
// rho (sin(th + a) - sin th, cos th - cos(th + a)), a right turn by
// rho (sin th - sin(th - a), cos(th - a) - cos th), a straight part of length l
// by l (cos th, sin th)); altitude z0 + s dz.
template <typename R>
void dubins_point(const R* s0, const R* s1, const DubinsPath<R>& P, R rho, R s, R* out) {
    static const int kSeg[6][3] = {{0, 1, 0}, {2, 1, 2}, {0, 1, 2}, {2, 1, 0}, {2, 0, 2}, {0, 2, 0}};  // 0 L, 1 S, 2 R
    R x = s0[0], y = s0[1], th = s0[3];
    R ell = s * P.L;
    const R len[3] = {P.t * rho, P.p * rho, P.q * rho};
    for (int k = 0; k < 3; ++k) {
        const R a = ell < len[k] ? ell : len[k];
        const int type = kSeg[P.word][k];
        R s_th, c_th;
        dub_sincos(th, &s_th, &c_th);
        if (type == 1) {
            x = x + a * c_th;
            y = y + a * s_th;
        } else {
            const R ang = a / rho;
            const R th2 = type == 0 ? th + ang : th - ang;
            R s_2, c_2;
            dub_sincos(th2, &s_2, &c_2);
            if (type == 0) {
                x = x + rho * (s_2 - s_th);
                y = y + rho * (c_th - c_2);
            } else {
                x = x + rho * (s_th - s_2);
                y = y + rho * (c_2 - c_th);
            }
            th = th2;
        }
        ell = ell - a;
    }
    out[0] = x;
    out[1] = y;
    out[2] = s0[2] + s * (s1[2] - s0[2]);
    out[3] = th;
}

// Cost of the directed connection from -> to, both states of dimension d.
template <typename R>
R edge_cost(int kind, const R* from, const R* to, int d, R r, R* tau, R rho = 0) {
    if (kind == ORC_EUCLID) { if (tau) *tau = 0; return cost_euclid(from, to, d); }
    if (kind == ORC_DUBINS) {
        if (tau) *tau = 0;
        return dubins_near(from, to, r) ? cost_dubins(from, to, rho) : std::numeric_limits<R>::infinity();
    }
    return cost_di(from, to, r, DI_GRID, di_bisect_steps<R>(), tau);
}

// ---------------------------------------------------------------------------
// Edge collision check (Alg. 1's lazy check, Sec. III-A): one connection.
// Geometric: m = max(2, ceil(L/spacing)+1) points p_k = y + t_k (x - y),
//   t_k = k/(m-1), endpoints included; a point in a closed box collides.
// Double integrator: the minimum-effort trajectory is the cubic Hermite curve
//   p(s) = h00 p0 + h10 tau v0 + h01 p1 + h11 tau v1, s in [0,1],
//   h00 = 2s^3-3s^2+1, h10 = s^3-2s^2+s, h01 = 3s^2-2s^3, h11 = s^3-s^2,
//   evaluated at s_k = k/(P-1), k = 0..P-1; a point in a box or outside the
//   position bounds collides.
// ---------------------------------------------------------------------------
template <typename R>
bool edge_free_geometric(const R* y, const R* x, int dp, R L, R spacing, const Boxes& B) {
    int m = (int)std::ceil(L / spacing) + 1;
    if (m < 2) m = 2;
    R p[MAXD];
    for (int k = 0; k < m; ++k) {
        R t = (R)k / (R)(m - 1);
        for (int a = 0; a < dp; ++a) p[a] = y[a] + t * (x[a] - y[a]);
        if (point_in_obstacle(p, B)) return false;
    }
    return true;
}

template <typename R>
void hermite_point(const R* s0, const R* s1, R tau, R s, R* p) {
    R s2 = s * s;
    R s3 = s2 * s;
    R h00 = ((R)2 * s3 - (R)3 * s2) + (R)1;
    R h10 = (s3 - (R)2 * s2) + s;
    R h01 = (R)3 * s2 - (R)2 * s3;
    R h11 = s3 - s2;
    R h10t = h10 * tau, h11t = h11 * tau;
    for (int a = 0; a < 3; ++a)
        p[a] = ((h00 * s0[a] + h10t * s0[3 + a]) + h01 * s1[a]) + h11t * s1[3 + a];
}

template <typename R>
bool edge_free_di(const R* y, const R* x, R tau, int points, const float* plo, const float* phi, const Boxes& B) {
    R p[3];
    for (int k = 0; k < points; ++k) {
        R s = (R)k / (R)(points - 1);
        hermite_point(y, x, tau, s, p);
        for (int a = 0; a < 3; ++a)
            if (p[a] < (R)plo[a] || p[a] > (R)phi[a]) return false;
        if (point_in_obstacle(p, B)) return false;
    }
    return true;
}

// Dubins airplane edge of cost c: m = max(2, ceil(c/spacing)+1) points at
// s_k = k/(m-1) of the path; a point in a box or outside the position bounds
// collides.
template <typename R>
bool edge_free_dubins(const R* y, const R* x, R c, R rho, R spacing, const float* plo, const float* phi,
                      const Boxes& B) {
    const DubinsPath<R> P = dubins_path(y, x, rho);
    int m = (int)std::ceil(c / spacing) + 1;
    if (m < 2) m = 2;
    R q[4];
    for (int k = 0; k < m; ++k) {
        const R s = (R)k / (R)(m - 1);
        dubins_point(y, x, P, rho, s, q);
        for (int a = 0; a < 3; ++a)
            if (q[a] < (R)plo[a] || q[a] > (R)phi[a]) return false;
        if (point_in_obstacle(q, B)) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Neighbour graph: y -> x is an edge iff y != x and c(y,x) < r (Section III-A:
// neighbours are samples whose connection cost is less than r).  Out-lists are
// ascending in x, in-lists ascending in y.
// ---------------------------------------------------------------------------
template <typename R>
struct Graph {
    int kind = 0, d = 0, dp = 0, N = 0;
    R r = 0;
    R rho = 0;   // Dubins airplane: turning radius
    std::vector<R> X;            // [d][N]
    std::vector<uint8_t> goal;   // [N]
    std::vector<int32_t> out_row, out_col, in_row, in_col;
    std::vector<R> out_cost, in_cost;
    void state(int v, R* s) const { for (int a = 0; a < d; ++a) s[a] = X[(size_t)a * N + v]; }
};

template <typename R>
Graph<R>* build_graph(int kind, int d, int dp, int N, const float* X, const uint8_t* goal, float r, float rho = 0.0f) {
    Graph<R>* g = new Graph<R>();
    g->kind = kind; g->d = d; g->dp = dp; g->N = N; g->r = (R)r;
    g->rho = (R)rho;
    g->X.resize((size_t)d * N);
    for (size_t i = 0; i < (size_t)d * N; ++i) g->X[i] = (R)X[i];
    g->goal.assign(goal, goal + N);
    std::vector<std::vector<std::pair<int, R>>> out(N), in(N);
    R si[MAXD], sj[MAXD];
    for (int i = 0; i < N; ++i) {
        g->state(i, si);
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            g->state(j, sj);
            R c = edge_cost<R>(kind, si, sj, d, g->r, nullptr, g->rho);
            if (c < g->r) out[i].push_back({j, c});
        }
    }
    for (int y = 0; y < N; ++y)
        for (auto& e : out[y]) in[e.first].push_back({y, e.second});
    auto flatten = [N](const std::vector<std::vector<std::pair<int, R>>>& L,
                       std::vector<int32_t>& row, std::vector<int32_t>& col, std::vector<R>& cost) {
        row.assign(N + 1, 0);
        for (int v = 0; v < N; ++v) row[v + 1] = row[v] + (int32_t)L[v].size();
        col.clear(); cost.clear();
        for (int v = 0; v < N; ++v)
            for (auto& e : L[v]) { col.push_back(e.first); cost.push_back(e.second); }
    };
    flatten(out, g->out_row, g->out_col, g->out_cost);
    flatten(in, g->in_row, g->in_col, g->in_cost);
    return g;
}

// ---------------------------------------------------------------------------
// Planner inputs shared by GMT*, FMT* and Dijkstra.
// ---------------------------------------------------------------------------
struct PlanCfg {
    Boxes boxes;
    const float* pos_lo;   // position bounds (double-integrator wall test)
    const float* pos_hi;
    float lambda, seg_spacing;
    int traj_points, skip_empty, max_iters;
};

}  // namespace

extern "C" {

struct orc_info {
    int32_t status, goal_node;
    double path_cost;
    int64_t iters, final_i, push_edges, pull_edges, checks, failed, tree_size;
};

}

namespace {

// Collision verdict for the tree edge parent y -> child x with cost c.
template <typename R>
bool check_edge(const Graph<R>& g, int y, int x, R c, const PlanCfg& P) {
    R sy[MAXD], sx[MAXD];
    g.state(y, sy); g.state(x, sx);
    if (g.kind == ORC_EUCLID) return edge_free_geometric(sy, sx, g.dp, c, (R)P.seg_spacing, P.boxes);
    if (g.kind == ORC_DUBINS)
        return edge_free_dubins(sy, sx, c, g.rho, (R)P.seg_spacing, P.pos_lo, P.pos_hi, P.boxes);
    R tau;
    cost_di<R>(sy, sx, g.r, DI_GRID, di_bisect_steps<R>(), &tau);
    return edge_free_di(sy, sx, tau, P.traj_points, P.pos_lo, P.pos_hi, P.boxes);
}

template <typename R>
void finish(const Graph<R>& g, const std::vector<R>& cost, bool success, orc_info* info) {
    info->goal_node = -1;
    info->path_cost = std::numeric_limits<double>::infinity();
    if (!success) { info->status = ORC_NO_PATH; return; }
    // Result (Alg. 1's returned path, Sec. III-A): the minimum-cost tree node in
    // X_goal, ties by index.
    int best = -1;
    for (int v = 0; v < g.N; ++v)
        if (g.goal[v] && cost[v] < std::numeric_limits<R>::infinity())
            if (best < 0 || cost[v] < cost[best]) best = v;
    info->status = ORC_OK;
    info->goal_node = best;
    info->path_cost = (double)cost[best];
}

// ---------------------------------------------------------------------------
// Group Marching Tree (Sec. III-A, Algorithm 1), one threshold index at a time.
//
// Every node is in one of three sets: unexplored (not yet in the tree), open
// (in the tree, its out-neighbours not yet expanded) or closed (expanded).
// The tree starts as x_init alone, open, at cost 0.  At threshold index i the
// group is every open node whose cost is at most theta_i = fl(fl(i) * delta),
// delta = fl(lambda r); lambda = 0 is the FMT* limit, where the group is the
// open nodes at the minimum open cost.  The group's unexplored out-neighbours
// are the candidates.  Each candidate x looks for its cheapest connection
// among its open in-neighbours y, by (cost(y) + c(y, x), y) -- "open" as it
// stood before this index's additions -- and checks only that one edge for
// collisions (the lazy check).  A free edge puts x in the tree, open from the
// next index on; a blocked one leaves x unexplored, to be tried again when a
// later group reaches it.  Then the group closes.  The plan succeeds as soon
// as a closed group held a goal node and fails once nothing is open.
// With skip_empty, threshold indices whose group would be empty (no-ops) are
// skipped: the next index is the smallest i' > i with theta_{i'} >= the
// minimum open cost.
// ---------------------------------------------------------------------------
namespace gmt_steps {

// Open nodes with cost <= theta, ascending.
template <typename R>
std::vector<int> open_group(const std::vector<int>& set, const std::vector<R>& cost, R theta) {
    std::vector<int> grp;
    for (int v = 0; v < (int)set.size(); ++v)
        if (set[v] == OPEN && cost[v] <= theta) grp.push_back(v);
    return grp;
}

// Smallest cost among open nodes (+inf if none is open).
template <typename R>
R min_open_cost(const std::vector<int>& set, const std::vector<R>& cost) {
    R m = std::numeric_limits<R>::infinity();
    for (int v = 0; v < (int)set.size(); ++v)
        if (set[v] == OPEN && cost[v] < m) m = cost[v];
    return m;
}

// Unexplored out-neighbours of the group's nodes, each once, ascending.
template <typename R>
std::vector<int> candidates_of(const Graph<R>& g, const std::vector<int>& grp, const std::vector<int>& set,
                               int64_t* scanned) {
    std::vector<char> seen(g.N, 0);
    std::vector<int> cand;
    for (int z : grp) {
        *scanned += g.out_row[z + 1] - g.out_row[z];
        for (int e = g.out_row[z]; e < g.out_row[z + 1]; ++e) {
            const int x = g.out_col[e];
            if (set[x] == UNEXPLORED && !seen[x]) { seen[x] = 1; cand.push_back(x); }
        }
    }
    std::sort(cand.begin(), cand.end());
    return cand;
}

// The lexicographically smallest (cost(y) + c(y, x), y) over open in-neighbours
// y of x.  Returns y (-1 if none), its connection cost and the edge's cost.
template <typename R>
int best_open_parent(const Graph<R>& g, int x, const std::vector<int>& set, const std::vector<R>& cost, R* via,
                     R* edge, int64_t* scanned) {
    *scanned += g.in_row[x + 1] - g.in_row[x];
    int best = -1;
    R cbest = std::numeric_limits<R>::infinity(), ebest = 0;
    for (int e = g.in_row[x]; e < g.in_row[x + 1]; ++e) {
        const int y = g.in_col[e];
        if (set[y] != OPEN) continue;
        const R c = cost[y] + g.in_cost[e];
        if (best < 0 || c < cbest || (c == cbest && y < best)) { best = y; cbest = c; ebest = g.in_cost[e]; }
    }
    *via = cbest;
    *edge = ebest;
    return best;
}

// The threshold index after i, given the minimum open cost m > theta_i.  The
// index stays below 2^24 (exact in FP32); returns -1 beyond that.
template <typename R>
int64_t next_index(int64_t i, R m, R delta, bool skip_empty) {
    if (delta == (R)0) return i + 1;
    if (!(m / delta < (R)16777216)) return -1;
    if (!skip_empty) return i + 1;
    int64_t k = (int64_t)std::ceil(m / delta);
    if (k < i + 1) k = i + 1;
    while (k > i + 1 && (R)(k - 1) * delta >= m) --k;
    while ((R)k * delta < m) ++k;
    return k;
}

}  // namespace gmt_steps

template <typename R>
int gmt_plan(const Graph<R>& g, const PlanCfg& P, int32_t* parent_out, R* cost_out, orc_info* info,
             int64_t* added_i = nullptr, int64_t* closed_i = nullptr) {
    using namespace gmt_steps;
    const int N = g.N;
    const R INF = std::numeric_limits<R>::infinity();
    std::memset(info, 0, sizeof(*info));
    std::vector<int> set(N, UNEXPLORED);
    std::vector<R> cost(N, INF);
    std::vector<int32_t> parent(N, -1);
    set[0] = OPEN;
    cost[0] = 0;
    if (added_i) for (int v = 0; v < N; ++v) added_i[v] = v == 0 ? -1 : -2;
    if (closed_i) for (int v = 0; v < N; ++v) closed_i[v] = -2;
    const R delta = (R)P.lambda * g.r;    // fl(lambda * r)
    int64_t i = 0;
    bool success = false;
    int status = ORC_OK;
    struct Link { int x, y; R c; };
    for (;;) {
        const R theta = delta == (R)0 ? min_open_cost(set, cost) : (R)i * delta;
        const std::vector<int> grp = open_group(set, cost, theta);
        if (!grp.empty()) {
            if (info->iters >= P.max_iters) { status = ORC_ERR_ITER_LIMIT; break; }
            info->iters++;
        }
        // every candidate is decided against the open set as it stands now;
        // the new tree edges are applied together afterwards
        std::vector<Link> links;
        for (int x : candidates_of(g, grp, set, &info->push_edges)) {
            R via, edge;
            const int y = best_open_parent(g, x, set, cost, &via, &edge, &info->pull_edges);
            // x was reached from a node of the group, which is open, so y exists
            info->checks++;
            if (check_edge(g, y, x, edge, P)) links.push_back({x, y, via});
            else info->failed++;
        }
        for (const Link& l : links) {
            set[l.x] = OPEN; parent[l.x] = l.y; cost[l.x] = l.c;
            if (added_i) added_i[l.x] = i;
        }
        bool goal_in_group = false;
        for (int z : grp) {
            set[z] = CLOSED;
            if (g.goal[z]) goal_in_group = true;
            if (closed_i) closed_i[z] = i;
        }
        if (goal_in_group) { success = true; break; }
        const R m = min_open_cost(set, cost);
        if (m == INF) { success = false; break; }
        const int64_t nxt = next_index(i, m, delta, P.skip_empty);
        if (nxt < 0) {  // the index would leave the exact FP32 range
            if (!P.skip_empty) i = i + 1;
            status = ORC_ERR_ITER_LIMIT;
            break;
        }
        i = nxt;
    }
    info->final_i = i;
    int64_t tree = 0;
    for (int v = 0; v < N; ++v) if (cost[v] < INF) ++tree;
    info->tree_size = tree;
    for (int v = 0; v < N; ++v) { parent_out[v] = parent[v]; cost_out[v] = cost[v]; }
    if (status != ORC_OK) { info->status = status; info->goal_node = -1; info->path_cost = INFINITY; return status; }
    finish(g, cost, success, info);
    return info->status;
}

// ---------------------------------------------------------------------------
// FMT* (Janson, Schmerling, Clark, Pavone 2015), the comparator of Section III:
// expand only the single minimum-cost open node z (ties by index) per step,
// connect each unexplored out-neighbour x of z to argmin over open
// in-neighbours of cost(y) + c(y,x), lazily checked; stop when z is a goal node
// or the open set is empty.  Open nodes are kept in a binary heap.
// ---------------------------------------------------------------------------
template <typename R>
int fmt_plan(const Graph<R>& g, const PlanCfg& P, int32_t* parent_out, R* cost_out, orc_info* info) {
    const int N = g.N;
    const R INF = std::numeric_limits<R>::infinity();
    std::memset(info, 0, sizeof(*info));
    std::vector<int> set(N, UNEXPLORED);
    std::vector<R> cost(N, INF);
    std::vector<int32_t> parent(N, -1);
    typedef std::pair<R, int> Key;
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    set[0] = OPEN; cost[0] = 0; heap.push({(R)0, 0});
    int found = -1;
    while (!heap.empty()) {
        Key top = heap.top(); heap.pop();
        int z = top.second;
        if (set[z] != OPEN) continue;
        if (g.goal[z]) { found = z; break; }
        info->iters++;
        std::vector<std::pair<int, std::pair<int, R>>> added;
        info->push_edges += g.out_row[z + 1] - g.out_row[z];
        for (int e = g.out_row[z]; e < g.out_row[z + 1]; ++e) {
            int x = g.out_col[e];
            if (set[x] != UNEXPLORED) continue;
            info->pull_edges += g.in_row[x + 1] - g.in_row[x];
            int yb = -1; R cb = INF, eb = 0;
            for (int f = g.in_row[x]; f < g.in_row[x + 1]; ++f) {
                int y = g.in_col[f];
                if (set[y] != OPEN) continue;
                R c = cost[y] + g.in_cost[f];
                if (yb < 0 || c < cb || (c == cb && y < yb)) { yb = y; cb = c; eb = g.in_cost[f]; }
            }
            info->checks++;
            if (check_edge(g, yb, x, eb, P)) added.push_back({x, {yb, cb}});
            else info->failed++;
        }
        for (auto& a : added) {
            set[a.first] = OPEN; parent[a.first] = a.second.first; cost[a.first] = a.second.second;
            heap.push({cost[a.first], a.first});
        }
        set[z] = CLOSED;
    }
    int64_t tree = 0;
    for (int v = 0; v < N; ++v) if (cost[v] < INF) ++tree;
    info->tree_size = tree;
    for (int v = 0; v < N; ++v) { parent_out[v] = parent[v]; cost_out[v] = cost[v]; }
    info->goal_node = -1;
    info->path_cost = INFINITY;
    if (found < 0) { info->status = ORC_NO_PATH; return ORC_NO_PATH; }
    info->status = ORC_OK; info->goal_node = found; info->path_cost = (double)cost[found];
    return ORC_OK;
}

// Exact shortest path (Dijkstra) from x_init over the directed r-disk graph
// restricted to collision-free edges (every edge checked).  dist uses the same
// recurrence fl(dist(y) + c(y,x)) as the planners.
template <typename R>
double dijkstra(const Graph<R>& g, const PlanCfg& P, R* dist_out) {
    const int N = g.N;
    const R INF = std::numeric_limits<R>::infinity();
    std::vector<R> dist(N, INF);
    std::vector<char> done(N, 0);
    typedef std::pair<R, int> Key;
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    dist[0] = 0; heap.push({(R)0, 0});
    while (!heap.empty()) {
        Key t = heap.top(); heap.pop();
        int y = t.second;
        if (done[y]) continue;
        done[y] = 1;
        for (int e = g.out_row[y]; e < g.out_row[y + 1]; ++e) {
            int x = g.out_col[e];
            if (done[x]) continue;
            R c = dist[y] + g.out_cost[e];
            if (c < dist[x] && check_edge(g, y, x, g.out_cost[e], P)) { dist[x] = c; heap.push({c, x}); }
        }
    }
    R best = INF;
    for (int v = 0; v < N; ++v) if (g.goal[v] && dist[v] < best) best = dist[v];
    if (dist_out) for (int v = 0; v < N; ++v) dist_out[v] = dist[v];
    return (double)best;
}

PlanCfg make_cfg(int nbox, int dp, const float* blo, const float* bhi, const float* pos_lo, const float* pos_hi,
                 float lambda, float seg_spacing, int traj_points, int skip_empty, int max_iters) {
    PlanCfg P;
    P.boxes.count = nbox; P.boxes.dp = dp; P.boxes.lo = blo; P.boxes.hi = bhi;
    P.pos_lo = pos_lo; P.pos_hi = pos_hi;
    P.lambda = lambda; P.seg_spacing = seg_spacing; P.traj_points = traj_points;
    P.skip_empty = skip_empty; P.max_iters = max_iters;
    return P;
}

}  // namespace

// ===========================================================================
// C interface (loaded with ctypes by the tests).
// ===========================================================================
extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }
float orc_word_to_unit(uint32_t w) { return word_to_unit(w); }

// SampleFree(n) (Section III-B) with V = {x_init} U SampleFree(n): node 0 is
// x_init, node 1 is drawn uniformly in X_goal n X_free (so at least one sample
// lies in the goal region, Alg. 1 input), nodes 2..n uniformly in X_free.
// Node k, attempt t draws Philox4x32-10 blocks with counter (k, t, stream, blk)
// and key (seed lo 32 bits, seed hi 32 bits); coordinate a uses word a%4 of
// block a/4, mapped to lo_a + u*(hi_a - lo_a).  The first attempt that is
// accepted (not in any closed box; for node 1 also inside the goal ball and the
// state bounds) is the sample.  For node 1 the goal axes draw from the ball's
// bounding box [c - rho, c + rho].  Returns 0, or -1 on invalid input or when a
// node exhausts max_attempts.
int orc_sample(int d, int dp, const float* lo, const float* hi, int nbox, const float* blo, const float* bhi,
               const float* x_init, const float* goal_c, float goal_r, int goal_pos_only, int n, uint64_t seed,
               uint32_t stream, int max_attempts, float* X, uint8_t* is_goal) {
    if (d < 1 || d > MAXD || dp < 1 || dp > d || n < 1) return ORC_ERR_INVALID;
    Boxes B{nbox, dp, blo, bhi};
    const int N = n + 1;
    const int gd = goal_pos_only ? dp : d;
    for (int a = 0; a < d; ++a)
        if (!(lo[a] <= x_init[a] && x_init[a] <= hi[a])) return ORC_ERR_INVALID;
    if (point_in_obstacle(x_init, B)) return ORC_ERR_INVALID;
    for (int a = 0; a < d; ++a) X[(size_t)a * N + 0] = x_init[a];
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    float x[MAXD];
    for (int k = 1; k < N; ++k) {
        bool ok = false;
        for (int t = 0; t < max_attempts && !ok; ++t) {
            uint32_t words[MAXD];
            for (int blk = 0; blk * 4 < d; ++blk) {
                uint32_t ctr[4] = {(uint32_t)k, (uint32_t)t, stream, (uint32_t)blk};
                philox4x32_10(ctr, key, words + 4 * blk);
            }
            for (int a = 0; a < d; ++a) {
                float u = word_to_unit(words[a]);
                float l = lo[a], h = hi[a];
                if (k == 1 && a < gd) { l = goal_c[a] - goal_r; h = goal_c[a] + goal_r; }
                x[a] = l + u * (h - l);
            }
            if (k == 1) {
                bool inb = true;
                for (int a = 0; a < d; ++a) if (!(lo[a] <= x[a] && x[a] <= hi[a])) inb = false;
                if (!inb || !in_goal(x, gd, goal_c, goal_r)) continue;
            }
            if (point_in_obstacle(x, B)) continue;
            ok = true;
        }
        if (!ok) return ORC_ERR_INVALID;
        for (int a = 0; a < d; ++a) X[(size_t)a * N + k] = x[a];
    }
    for (int k = 0; k < N; ++k) {
        for (int a = 0; a < d; ++a) x[a] = X[(size_t)a * N + k];
        is_goal[k] = in_goal(x, gd, goal_c, goal_r) ? 1 : 0;
    }
    return ORC_OK;
}

// ---- Halton SampleFree (the low-dispersion sequence of Sec. V, "Halton
// sequence"; our reading of how it meets SampleFree's contract) ----
// Point k >= 1 of the Halton sequence has coordinate a equal to the radical
// inverse of k in the a-th prime base: writing k = sum_i d_i p^i, it is
// sum_i d_i p^-(i+1).  It is evaluated exactly as the fraction R / p^m (R the
// digits of k reversed, m their count), rounded to double and then to float.
static const uint32_t kHaltonPrimes[MAXD] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29};

float halton_unit(uint32_t k, uint32_t p) {
    uint64_t R = 0, P = 1;
    while (k > 0) {
        R = R * p + k % p;
        P *= p;
        k /= p;
    }
    return (float)((double)R / (double)P);
}

// Node 0 = x_init.  Node 1 = the first Halton point (k = 1, 2, ...), mapped into
// the goal ball's bounding box on the goal axes and into X on the others, that
// lies in X, in the goal ball and outside every box.  Nodes 2..n = the Halton
// points mapped into X that lie outside every box, in the order of k.  At most
// max_candidates points are tried for node 1 and for nodes 2..n each.
int orc_sample_halton(int d, int dp, const float* lo, const float* hi, int nbox, const float* blo, const float* bhi,
                      const float* x_init, const float* goal_c, float goal_r, int goal_pos_only, int n,
                      long long max_candidates, float* X, uint8_t* is_goal) {
    if (d < 1 || d > MAXD || dp < 1 || dp > d || n < 1) return ORC_ERR_INVALID;
    Boxes B{nbox, dp, blo, bhi};
    const int N = n + 1;
    const int gd = goal_pos_only ? dp : d;
    for (int a = 0; a < d; ++a)
        if (!(lo[a] <= x_init[a] && x_init[a] <= hi[a])) return ORC_ERR_INVALID;
    if (point_in_obstacle(x_init, B)) return ORC_ERR_INVALID;
    for (int a = 0; a < d; ++a) X[(size_t)a * N + 0] = x_init[a];
    float x[MAXD];
    if (N > 1) {
        bool found = false;
        for (long long k = 1; k <= max_candidates && !found; ++k) {
            for (int a = 0; a < d; ++a) {
                const float u = halton_unit((uint32_t)k, kHaltonPrimes[a]);
                float l = lo[a], h = hi[a];
                if (a < gd) { l = goal_c[a] - goal_r; h = goal_c[a] + goal_r; }
                x[a] = l + u * (h - l);
            }
            bool inb = true;
            for (int a = 0; a < d; ++a) if (!(lo[a] <= x[a] && x[a] <= hi[a])) inb = false;
            if (!inb || !in_goal(x, gd, goal_c, goal_r) || point_in_obstacle(x, B)) continue;
            for (int a = 0; a < d; ++a) X[(size_t)a * N + 1] = x[a];
            found = true;
        }
        if (!found) return ORC_ERR_INVALID;
    }
    int v = 2;
    for (long long k = 1; v < N; ++k) {
        if (k > max_candidates) return ORC_ERR_INVALID;
        for (int a = 0; a < d; ++a) {
            const float u = halton_unit((uint32_t)k, kHaltonPrimes[a]);
            x[a] = lo[a] + u * (hi[a] - lo[a]);
        }
        if (point_in_obstacle(x, B)) continue;
        for (int a = 0; a < d; ++a) X[(size_t)a * N + v] = x[a];
        ++v;
    }
    for (int k = 0; k < N; ++k) {
        for (int a = 0; a < d; ++a) x[a] = X[(size_t)a * N + k];
        is_goal[k] = in_goal(x, gd, goal_c, goal_r) ? 1 : 0;
    }
    return ORC_OK;
}

float orc_halton_unit(uint32_t k, uint32_t p) { return halton_unit(k, p); }

// Connection radius for low-dispersion samples (Sec. III-B: a smaller r than
// Theorem 1's may be used; our reading drops Theorem 1's log n factor):
// 4 ((1 + eta) (1/d) (mu / zeta_d) (1/n))^(1/d).
double orc_radius_halton(int n, int d, double eta, double mu) {
    const double pi = 3.14159265358979323846;
    double zeta = std::pow(pi, (double)d / 2.0) / std::tgamma((double)d / 2.0 + 1.0);
    double base = (1.0 + eta) * (1.0 / (double)d) * (mu / zeta) * (1.0 / (double)n);
    return 4.0 * std::pow(base, 1.0 / (double)d);
}

int orc_in_goal(const float* x, int gd, const float* c, float rho) { return in_goal(x, gd, c, rho) ? 1 : 0; }

float orc_cost_euclid_f32(const float* from, const float* to, int d) { return cost_euclid(from, to, d); }
double orc_cost_euclid_f64(const double* from, const double* to, int d) { return cost_euclid(from, to, d); }

float orc_cost_di_f32(const float* s0, const float* s1, float r, float* tau) {
    return cost_di<float>(s0, s1, r, DI_GRID, 24, tau);
}
double orc_cost_di_f64(const double* s0, const double* s1, double span, int grid, int bisect, double* tau) {
    return cost_di<double>(s0, s1, span, grid, bisect, tau);
}
void orc_di_coeffs_f64(const double* s0, const double* s1, double* abc) {
    DICoeffs<double> k = di_coeffs(s0, s1);
    abc[0] = k.a; abc[1] = k.b; abc[2] = k.c;
}
void orc_hermite_point_f64(const double* s0, const double* s1, double tau, double s, double* p) {
    hermite_point(s0, s1, tau, s, p);
}

int orc_edge_free_geometric_f32(const float* y, const float* x, int dp, float L, float spacing, int nbox,
                                const float* blo, const float* bhi) {
    Boxes B{nbox, dp, blo, bhi};
    return edge_free_geometric(y, x, dp, L, spacing, B) ? 1 : 0;
}
int orc_edge_free_di_f32(const float* y, const float* x, float tau, int points, const float* plo, const float* phi,
                         int nbox, const float* blo, const float* bhi) {
    Boxes B{nbox, 3, blo, bhi};
    return edge_free_di(y, x, tau, points, plo, phi, B) ? 1 : 0;
}

// Theorem 1 radius r = 4 (1+eta)^(1/d) (1/d)^(1/d) (mu/zeta_d)^(1/d) (log n/n)^(1/d),
// zeta_d = pi^(d/2) / Gamma(d/2 + 1), evaluated in double as
// 4 * pow((1+eta) * (1/d) * (mu/zeta_d) * (log(n)/n), 1/d).
double orc_radius_thm1(int n, int d, double eta, double mu) {
    const double pi = 3.14159265358979323846;
    double zeta = std::pow(pi, (double)d / 2.0) / std::tgamma((double)d / 2.0 + 1.0);
    double base = (1.0 + eta) * (1.0 / (double)d) * (mu / zeta) * (std::log((double)n) / (double)n);
    return 4.0 * std::pow(base, 1.0 / (double)d);
}

// ---- graphs ----
void* orc_graph_build_dubins(int precision, int N, const float* X, const uint8_t* goal, float r, float rho) {
    if (precision == 64) return build_graph<double>(ORC_DUBINS, 4, 3, N, X, goal, r, rho);
    return build_graph<float>(ORC_DUBINS, 4, 3, N, X, goal, r, rho);
}

// Dubins words of a pair (float or double, by `precision`): six entries of
// (word, t, p, q, L) in enum order; returns the index of the shortest (6 if
// none exists).  States are (x, y, z, theta).
int orc_dubins_words(int precision, const double* s0, const double* s1, double rho, double* out) {
    auto run = [&](auto zero) {
        typedef decltype(zero) R;
        const R a[4] = {(R)s0[0], (R)s0[1], (R)s0[2], (R)s0[3]}, b[4] = {(R)s1[0], (R)s1[1], (R)s1[2], (R)s1[3]};
        DubinsPath<R> w[6];
        dubins_words(a[0], a[1], a[3], b[0], b[1], b[3], (R)rho, w);
        for (int k = 0; k < 6; ++k) {
            out[5 * k + 0] = w[k].word; out[5 * k + 1] = w[k].t; out[5 * k + 2] = w[k].p;
            out[5 * k + 3] = w[k].q; out[5 * k + 4] = w[k].L;
        }
        return dubins_path(a, b, (R)rho).word;
    };
    return precision == 64 ? run(0.0) : run(0.0f);
}
// Cost of the connection s0 -> s1 (r: the prefilter's radius; +inf when the
// prefilter rejects the pair).
double orc_cost_dubins(int precision, const double* s0, const double* s1, double rho, double r) {
    auto run = [&](auto zero) {
        typedef decltype(zero) R;
        const R a[4] = {(R)s0[0], (R)s0[1], (R)s0[2], (R)s0[3]}, b[4] = {(R)s1[0], (R)s1[1], (R)s1[2], (R)s1[3]};
        return (double)edge_cost<R>(ORC_DUBINS, a, b, 4, (R)r, nullptr, (R)rho);
    };
    return precision == 64 ? run(0.0) : run(0.0f);
}
// Pose at fraction s of the trajectory s0 -> s1.
void orc_dubins_point(int precision, const double* s0, const double* s1, double rho, double s, double* out) {
    auto run = [&](auto zero) {
        typedef decltype(zero) R;
        const R a[4] = {(R)s0[0], (R)s0[1], (R)s0[2], (R)s0[3]}, b[4] = {(R)s1[0], (R)s1[1], (R)s1[2], (R)s1[3]};
        R q[4];
        dubins_point(a, b, dubins_path(a, b, (R)rho), (R)rho, (R)s, q);
        for (int k = 0; k < 4; ++k) out[k] = (double)q[k];
    };
    if (precision == 64) run(0.0); else run(0.0f);
}
// The trigonometric building blocks over arrays (float or double).
void orc_dub_trig(int precision, int which, int n, const double* x, const double* y, double* out0, double* out1) {
    for (int i = 0; i < n; ++i) {
        if (precision == 64) {
            if (which == 0) dub_sincos(x[i], &out0[i], &out1[i]);
            else out0[i] = which == 1 ? dub_atan2(y[i], x[i]) : dub_acos(x[i]);
        } else {
            float a, b;
            if (which == 0) { dub_sincos((float)x[i], &a, &b); out0[i] = a; out1[i] = b; }
            else out0[i] = which == 1 ? dub_atan2((float)y[i], (float)x[i]) : dub_acos((float)x[i]);
        }
    }
}
// Collision verdict of the trajectory s0 -> s1 of cost c (float).
int orc_edge_free_dubins_f32(const float* s0, const float* s1, float c, float rho, float spacing, const float* pos_lo,
                             const float* pos_hi, int nbox, const float* blo, const float* bhi) {
    Boxes B{nbox, 3, blo, bhi};
    return edge_free_dubins<float>(s0, s1, c, rho, spacing, pos_lo, pos_hi, B) ? 1 : 0;
}

void* orc_graph_build(int precision, int kind, int d, int dp, int N, const float* X, const uint8_t* goal, float r) {
    if (precision == 64) return build_graph<double>(kind, d, dp, N, X, goal, r);
    return build_graph<float>(kind, d, dp, N, X, goal, r);
}
void orc_graph_free(int precision, void* g) {
    if (precision == 64) delete (Graph<double>*)g; else delete (Graph<float>*)g;
}
int64_t orc_graph_num_edges(int precision, const void* g) {
    if (precision == 64) return (int64_t)((const Graph<double>*)g)->out_col.size();
    return (int64_t)((const Graph<float>*)g)->out_col.size();
}
// Copies the CSR arrays out; costs are widened to double.
void orc_graph_copy(int precision, const void* gv, int32_t* out_row, int32_t* out_col, double* out_cost,
                    int32_t* in_row, int32_t* in_col, double* in_cost) {
    auto copy = [&](auto* g) {
        std::copy(g->out_row.begin(), g->out_row.end(), out_row);
        std::copy(g->out_col.begin(), g->out_col.end(), out_col);
        for (size_t e = 0; e < g->out_cost.size(); ++e) out_cost[e] = (double)g->out_cost[e];
        std::copy(g->in_row.begin(), g->in_row.end(), in_row);
        std::copy(g->in_col.begin(), g->in_col.end(), in_col);
        for (size_t e = 0; e < g->in_cost.size(); ++e) in_cost[e] = (double)g->in_cost[e];
    };
    if (precision == 64) copy((const Graph<double>*)gv); else copy((const Graph<float>*)gv);
}

// Number of directed edges y -> x with y in rows [row0, row1): the row-slice of
// the neighbour-set computation, used to time a bounded sample of it.
int64_t orc_count_edges_rows(int kind, int d, int N, const float* X, float r, int row0, int row1) {
    int64_t count = 0;
    float si[MAXD], sj[MAXD];
    for (int i = row0; i < row1 && i < N; ++i) {
        for (int a = 0; a < d; ++a) si[a] = X[(size_t)a * N + i];
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int a = 0; a < d; ++a) sj[a] = X[(size_t)a * N + j];
            if (edge_cost<float>(kind, si, sj, d, r, nullptr) < r) ++count;
        }
    }
    return count;
}

// ---- planners ----
// which: 0 = GMT* (Alg. 1), 1 = FMT*.  cost_out is double regardless of precision.
// added_i / closed_i (GMT* only, may be NULL): threshold index i of the
// iteration that added / closed each node (-1 for x_init, -2 never).
int orc_plan(int precision, int which, const void* gv, int nbox, const float* blo, const float* bhi,
             const float* pos_lo, const float* pos_hi, float lambda, float seg_spacing, int traj_points,
             int skip_empty, int max_iters, int32_t* parent, double* cost_out, orc_info* info,
             int64_t* added_i, int64_t* closed_i) {
    auto run = [&](auto* g, auto zero) {
        typedef decltype(zero) R;
        PlanCfg P = make_cfg(nbox, g->dp, blo, bhi, pos_lo, pos_hi, lambda, seg_spacing, traj_points, skip_empty, max_iters);
        std::vector<R> c(g->N);
        int st = which == 0 ? gmt_plan<R>(*g, P, parent, c.data(), info, added_i, closed_i)
                            : fmt_plan<R>(*g, P, parent, c.data(), info);
        for (int v = 0; v < g->N; ++v) cost_out[v] = (double)c[v];
        return st;
    };
    if (precision == 64) return run((const Graph<double>*)gv, 0.0);
    return run((const Graph<float>*)gv, 0.0f);
}

double orc_dijkstra(int precision, const void* gv, int nbox, const float* blo, const float* bhi,
                    const float* pos_lo, const float* pos_hi, float seg_spacing, int traj_points, double* dist_out) {
    auto run = [&](auto* g, auto zero) {
        typedef decltype(zero) R;
        PlanCfg P = make_cfg(nbox, g->dp, blo, bhi, pos_lo, pos_hi, 0.0f, seg_spacing, traj_points, 1, 0);
        std::vector<R> dist(g->N);
        double best = dijkstra<R>(*g, P, dist.data());
        if (dist_out) for (int v = 0; v < g->N; ++v) dist_out[v] = (double)dist[v];
        return best;
    };
    if (precision == 64) return run((const Graph<double>*)gv, 0.0);
    return run((const Graph<float>*)gv, 0.0f);
}

// Collision verdict of one directed graph edge y -> x of a built graph.
int orc_graph_edge_free(int precision, const void* gv, int y, int x, double c, int nbox, const float* blo,
                        const float* bhi, const float* pos_lo, const float* pos_hi, float seg_spacing,
                        int traj_points) {
    auto run = [&](auto* g, auto zero) {
        typedef decltype(zero) R;
        PlanCfg P = make_cfg(nbox, g->dp, blo, bhi, pos_lo, pos_hi, 0.0f, seg_spacing, traj_points, 1, 0);
        return check_edge<R>(*g, y, x, (R)c, P) ? 1 : 0;
    };
    if (precision == 64) return run((const Graph<double>*)gv, 0.0);
    return run((const Graph<float>*)gv, 0.0f);
}

}  // extern "C"
