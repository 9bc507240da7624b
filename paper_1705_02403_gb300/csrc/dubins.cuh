// Dubins airplane (Sec. V-A): a planar Dubins car of turning radius rho with a
// single integrator in altitude, cost = Euclidean length of the trajectory.
// State (x, y, z, theta).  The trajectory follows the shortest planar Dubins
// path (words LSL, RSR, LSR, RSL, RLR, LRL; Dubins 1957) with the altitude
// linear in planar arc length, so its length is sqrt(L^2 + dz^2) for a planar
// path of length L.
//
// Every function is IEEE FP32 in a fixed evaluation order (the library is
// built without FMA contraction and with IEEE division and square root), and
// sine, cosine and arctangent are written out here (range reduction plus
// Taylor series), so an edge's cost and its trajectory points are the same
// bits wherever they are computed.
#pragma once

#include <cstdint>

namespace gmtk {

namespace dub {
constexpr float kPi = 3.14159265358979f;
constexpr float kTwoPi = 6.28318530717959f;
constexpr float kPi2 = 1.57079632679490f;
constexpr float kPi4 = 0.785398163397448f;
constexpr float kPi2Hi = 1.57079637050628662109375f;  // fl(pi/2)
constexpr float kPi2Lo = -4.37113900018624e-8f;       // pi/2 - fl(pi/2)
constexpr float kTwoOverPi = 0.636619772367581f;
constexpr float kTanPi8 = 0.414213562373095f;
constexpr float kLoopSnap = (float)(1.0 / 8192);      // end turns within this of 2 pi are small negative turns
}  // namespace dub

enum { kDubLSL = 0, kDubRSR, kDubLSR, kDubRSL, kDubRLR, kDubLRL, kDubNone };

// sin r and cos r for |r| <= pi/4 (+ rounding): Taylor polynomials through
// r^11 and r^12 in Horner form.
__device__ __forceinline__ float dub_sin_poly(float r) {
    const float r2 = r * r;
    return r + r * (r2 * ((float)(-1.0 / 6) +
                          r2 * ((float)(1.0 / 120) +
                                r2 * ((float)(-1.0 / 5040) + r2 * ((float)(1.0 / 362880) + r2 * (float)(-1.0 / 39916800))))));
}
__device__ __forceinline__ float dub_cos_poly(float r) {
    const float r2 = r * r;
    return 1.0f + r2 * ((float)(-1.0 / 2) +
                        r2 * ((float)(1.0 / 24) +
                              r2 * ((float)(-1.0 / 720) +
                                    r2 * ((float)(1.0 / 40320) +
                                          r2 * ((float)(-1.0 / 3628800) + r2 * (float)(1.0 / 479001600))))));
}

// x = k pi/2 + r, k the nearest integer to 2x/pi (ties to even); the quadrant
// k mod 4 selects +-sin r or +-cos r.
__device__ __forceinline__ void dub_sincos(float x, float* s, float* c) {
    const float kf = rintf(x * dub::kTwoOverPi);
    const float r = (x - kf * dub::kPi2Hi) - kf * dub::kPi2Lo;
    const float sr = dub_sin_poly(r), cr = dub_cos_poly(r);
    const int q = __float2int_rz(kf) & 3;  // kf is integral and small: its quadrant mod 4
    if (q == 0) { *s = sr; *c = cr; }
    else if (q == 1) { *s = cr; *c = -sr; }
    else if (q == 2) { *s = -sr; *c = -cr; }
    else { *s = -cr; *c = sr; }
}

// atan z for 0 <= z <= 1: above tan(pi/8), pi/4 + atan((z - 1)/(z + 1)); then
// the series u - u^3/3 + ... - u^21/21.
__device__ __forceinline__ float dub_atan01(float z) {
    float base = 0.0f, u = z;
    if (z > dub::kTanPi8) {
        base = dub::kPi4;
        u = (z - 1.0f) / (z + 1.0f);
    }
    const float u2 = u * u;
    float poly = (float)(-1.0 / 21);
    poly = (float)(1.0 / 19) + u2 * poly;
    poly = (float)(-1.0 / 17) + u2 * poly;
    poly = (float)(1.0 / 15) + u2 * poly;
    poly = (float)(-1.0 / 13) + u2 * poly;
    poly = (float)(1.0 / 11) + u2 * poly;
    poly = (float)(-1.0 / 9) + u2 * poly;
    poly = (float)(1.0 / 7) + u2 * poly;
    poly = (float)(-1.0 / 5) + u2 * poly;
    poly = (float)(1.0 / 3) + u2 * poly;
    poly = -(u2 * poly);
    return base + (u + u * poly);
}

// Angle of (x, y) in (-pi, pi]; (0, 0) -> 0.
__device__ __forceinline__ float dub_atan2(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    if (ax == 0.0f && ay == 0.0f) return 0.0f;
    float a = ay <= ax ? dub_atan01(ay / ax) : dub::kPi2 - dub_atan01(ax / ay);
    if (x < 0.0f) a = dub::kPi - a;
    return y < 0.0f ? -a : a;
}

__device__ __forceinline__ float dub_acos(float x) { return dub_atan2(__fsqrt_rn((1.0f - x) * (1.0f + x)), x); }
__device__ __forceinline__ float dub_mod2pi(float a) { return a - dub::kTwoPi * floorf(a / dub::kTwoPi); }
// A first or last turn within kLoopSnap of a full circle is the small
// negative turn it differs by (a full loop never belongs to a shortest path).
__device__ __forceinline__ float dub_end_turn(float a) {
    return a > dub::kTwoPi - dub::kLoopSnap ? a - dub::kTwoPi : a;
}

struct DubPath {
    int word;
    float t, p, q;  // segment lengths / rho
    float L;        // planar length rho ((t + p) + q)
};

// Shortest of the six words (ties: the earlier word).  Frame: the line from
// start to end scaled by 1/rho, start at the origin with heading alpha, end at
// (d, 0) with heading beta; CSC words run along a common tangent of their two
// turning circles, CCC words along a third circle touching both.
__device__ __forceinline__ DubPath dubins_path(const float* s0, const float* s1, float rho) {
    const float dx = s1[0] - s0[0], dy = s1[1] - s0[1];
    const float D = __fsqrt_rn(dx * dx + dy * dy);
    const float d = D / rho;
    const float phi = dub_atan2(dy, dx);
    const float al = dub_mod2pi(s0[3] - phi), be = dub_mod2pi(s1[3] - phi);
    float sa, ca, sb, cb, scab, cab;
    dub_sincos(al, &sa, &ca);
    dub_sincos(be, &sb, &cb);
    dub_sincos(al - be, &scab, &cab);
    const float dd = d * d;
    DubPath best{kDubNone, 0.0f, 0.0f, 0.0f, __int_as_float(0x7f800000)};
    auto consider = [&](int w, float t, float p, float q) {
        t = dub_end_turn(t);
        q = dub_end_turn(q);
        const float L = ((t + p) + q) * rho;
        if (L < best.L) best = DubPath{w, t, p, q, L};
    };
    {  // LSL
        const float p2 = ((2.0f + dd) - 2.0f * cab) + (2.0f * d) * (sa - sb);
        if (p2 >= 0.0f) {
            const float psi = dub_atan2(cb - ca, (d + sa) - sb);
            consider(kDubLSL, dub_mod2pi(psi - al), __fsqrt_rn(p2), dub_mod2pi(be - psi));
        }
    }
    {  // RSR
        const float p2 = ((2.0f + dd) - 2.0f * cab) + (2.0f * d) * (sb - sa);
        if (p2 >= 0.0f) {
            const float psi = dub_atan2(ca - cb, (d - sa) + sb);
            consider(kDubRSR, dub_mod2pi(al - psi), __fsqrt_rn(p2), dub_mod2pi(psi - be));
        }
    }
    {  // LSR
        const float p2 = ((dd - 2.0f) + 2.0f * cab) + (2.0f * d) * (sa + sb);
        if (p2 >= 0.0f) {
            const float p = __fsqrt_rn(p2);
            const float psi = dub_atan2(-ca - cb, (d + sa) + sb) - dub_atan2(-2.0f, p);
            consider(kDubLSR, dub_mod2pi(psi - al), p, dub_mod2pi(psi - be));
        }
    }
    {  // RSL
        const float p2 = ((dd - 2.0f) + 2.0f * cab) - (2.0f * d) * (sa + sb);
        if (p2 >= 0.0f) {
            const float p = __fsqrt_rn(p2);
            const float psi = dub_atan2(ca + cb, (d - sa) - sb) - dub_atan2(2.0f, p);
            consider(kDubRSL, dub_mod2pi(al - psi), p, dub_mod2pi(be - psi));
        }
    }
    {  // RLR
        const float c = (((6.0f - dd) + 2.0f * cab) + (2.0f * d) * (sa - sb)) / 8.0f;
        if (fabsf(c) <= 1.0f) {
            const float p = dub_mod2pi(dub::kTwoPi - dub_acos(c));
            const float t = dub_mod2pi((al - dub_atan2(ca - cb, (d - sa) + sb)) + p / 2.0f);
            consider(kDubRLR, t, p, dub_mod2pi(((al - be) - t) + p));
        }
    }
    {  // LRL
        const float c = (((6.0f - dd) + 2.0f * cab) + (2.0f * d) * (sb - sa)) / 8.0f;
        if (fabsf(c) <= 1.0f) {
            const float p = dub_mod2pi(dub::kTwoPi - dub_acos(c));
            const float t = dub_mod2pi(((-al) - dub_atan2(ca - cb, (d + sa) - sb)) + p / 2.0f);
            consider(kDubLRL, t, p, dub_mod2pi(((be - al) - t) + p));
        }
    }
    return best;
}

// The cost is at least the 3D distance: pairs with squared distance at or
// above (1 + 2^-6) r^2 have no edge (the margin keeps this test from deciding
// a pair whose rounded cost could fall below r).
__device__ __forceinline__ bool dubins_near(const float* s0, const float* s1, float r) {
    const float dx = s1[0] - s0[0], dy = s1[1] - s0[1], dz = s1[2] - s0[2];
    return ((dx * dx + dy * dy) + dz * dz) < (r * r) * 1.015625f;
}

__device__ __forceinline__ float dubins_length(const DubPath& P, const float* s0, const float* s1) {
    const float dz = s1[2] - s0[2];
    return __fsqrt_rn(P.L * P.L + dz * dz);
}

__device__ __forceinline__ float dubins_cost(const float* s0, const float* s1, float rho) {
    return dubins_length(dubins_path(s0, s1, rho), s0, s1);
}

// Trajectory points.  The pose at fraction s walks planar arc length s L
// through the word's segments: segment k advances by a_k = min(ell_k, len_k)
// with ell_0 = s L and ell_{k+1} = ell_k - a_k (a left turn by a from heading
// th moves by rho (sin(th + a) - sin th, cos th - cos(th + a)), a right turn by
// rho (sin th - sin(th - a), cos(th - a) - cos th), a straight part by
// a (cos th, sin th)); the altitude is z0 + s dz.  DubSegs holds the pose at
// the start of each segment (the segments before it walked in full), so a
// point costs one partial segment: after it, a segment of length >= 0 advances
// by exactly 0, and only a negative last turn (an end turn taken as a small
// negative turn) still applies in full.
struct DubSegs {
    float x[3], y[3], th[3], sn[3], cs[3];  // start pose of each segment, sin and cos of its heading
    float len[3];                           // segment lengths (rho t, rho p, rho q)
    unsigned types;                         // 2 bits per segment: 0 L, 1 S, 2 R
    float L, rho;
};

// the partial (or full) segment of type `type` from a pose
__device__ __forceinline__ void dub_advance(unsigned type, float a, float rho, float& x, float& y, float& th, float s_th,
                                            float c_th) {
    if (type == 1u) {
        x = x + a * c_th;
        y = y + a * s_th;
    } else {
        const float ang = a / rho;
        const float th2 = type == 0u ? th + ang : th - ang;
        float s_2, c_2;
        dub_sincos(th2, &s_2, &c_2);
        if (type == 0u) {
            x = x + rho * (s_2 - s_th);
            y = y + rho * (c_th - c_2);
        } else {
            x = x + rho * (s_th - s_2);
            y = y + rho * (c_2 - c_th);
        }
        th = th2;
    }
}

__device__ __forceinline__ DubSegs dubins_segments(const float* s0, const DubPath& P, float rho) {
    // segment types by word, 2 bits each: LSL RSR LSR RSL RLR LRL
    constexpr unsigned kSeg[6] = {0u | 1u << 2 | 0u << 4, 2u | 1u << 2 | 2u << 4, 0u | 1u << 2 | 2u << 4,
                                  2u | 1u << 2 | 0u << 4, 2u | 0u << 2 | 2u << 4, 0u | 2u << 2 | 0u << 4};
    DubSegs G;
    G.types = kSeg[P.word < 6 ? P.word : 0];
    G.len[0] = P.t * rho;
    G.len[1] = P.p * rho;
    G.len[2] = P.q * rho;
    G.L = P.L;
    G.rho = rho;
    float x = s0[0], y = s0[1], th = s0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float s_th, c_th;
        dub_sincos(th, &s_th, &c_th);
        G.x[k] = x; G.y[k] = y; G.th[k] = th; G.sn[k] = s_th; G.cs[k] = c_th;
        if (k < 2) dub_advance((G.types >> (2 * k)) & 3u, G.len[k], rho, x, y, th, s_th, c_th);
    }
    return G;
}

__device__ __forceinline__ void dubins_point(const float* s0, const float* s1, const DubSegs& G, float s, float* out) {
    float ell = s * G.L;
    int k = 0;
    float a = ell;
    if (!(ell < G.len[0])) {      // segment 0 walked in full
        ell = ell - G.len[0];
        k = 1;
        a = ell;
        if (!(ell < G.len[1])) {  // segment 1 walked in full
            ell = ell - G.len[1];
            k = 2;
            a = ell < G.len[2] ? ell : G.len[2];
        }
    }
    float x = G.x[k], y = G.y[k], th = G.th[k];
    dub_advance((G.types >> (2 * k)) & 3u, a, G.rho, x, y, th, G.sn[k], G.cs[k]);
    if (k < 2 && G.len[2] < 0.0f) {  // a negative last turn applies whatever the point
        float s_th, c_th;
        dub_sincos(th, &s_th, &c_th);
        dub_advance((G.types >> 4) & 3u, G.len[2], G.rho, x, y, th, s_th, c_th);
    }
    out[0] = x;
    out[1] = y;
    out[2] = s0[2] + s * (s1[2] - s0[2]);
}

}  // namespace gmtk
