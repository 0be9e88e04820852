// FP32 device geometry of GPU-friendly stroke expansion (Levien & Uguray,
// arXiv 2405.00127).  Shared by the count and write passes, which must take
// identical decisions: the library is compiled with -fmad=false, so every
// expression below rounds the same way wherever it is inlined, and FMAs appear
// only where written explicitly.
#pragma once

#include <cmath>
#include <cstdint>

#include "../../include/stroke_expand.h"

// Every routine is __host__ __device__: the kernels run them on the GPU, and a
// host build of the same source lets the library's own tests step through a
// single tag on the CPU.
#ifdef __CUDACC__
#define SE_HD __host__ __device__ __forceinline__
// the large per-vertex routines keep a single compiled copy: lanes of a warp
// that diverge into different primitive kinds then share instruction cache
#define SE_NOINL static __host__ __device__ __noinline__
#else
#define SE_HD inline
#define SE_NOINL inline
#endif

namespace se {

// ---------------------------------------------------------------------------
// configuration shared by both passes
// ---------------------------------------------------------------------------
constexpr int kMaxDepth = 16;              // subdivision depth cap (Algorithm 2)
constexpr float kDerivEps = 1e-5f;         // |B'| below this * control-polygon length is a cusp (Section 7.3)
constexpr float kDerivDt = 1.0f / 1024.0f; // re-sampling step toward the piece interior
constexpr float kCMin = 0.25f;             // smallest accepted chord/arc ratio of an ES piece
constexpr float kPi = 3.14159265358979323846f;

struct Params {
    float tol_fit, tol_flat;
    bool arcs;
};

SE_HD float2 f2(float x, float y) { return make_float2(x, y); }

// Division for vertex placement only (never for a decision, never for a vertex
// that two threads compute): the hardware's fast division (within 2 ulp) on the
// device, exact division on the host.
SE_HD float vdiv(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
SE_HD float2 sub2(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
SE_HD float2 add2(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
SE_HD float2 mul2(float2 a, float s) { return f2(a.x * s, a.y * s); }
SE_HD float dot2(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
SE_HD float cross2(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
SE_HD float len2(float2 a) { return sqrtf(a.x * a.x + a.y * a.y); }
SE_HD float2 cmul(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
SE_HD float2 cdiv(float2 a, float2 b) {
    float d = b.x * b.x + b.y * b.y;
    return f2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// The accurate FP32 sine, cosine, arctangent and arcsine of the decision
// arithmetic (fits, counts, subdivision), each compiled once, out of line: the
// library's range reductions and slow paths otherwise repeat at every call site
// in every kernel and crowd the instruction cache.  The same functions, so the
// same results.
#ifdef __CUDA_ARCH__
static __device__ __noinline__ float acc_sin(float x) { return sinf(x); }
static __device__ __noinline__ float acc_cos(float x) { return cosf(x); }
static __device__ __noinline__ float acc_atan2(float y, float x) { return atan2f(y, x); }
static __device__ __noinline__ float acc_asin(float x) { return asinf(x); }
#else
inline float acc_sin(float x) { return sinf(x); }
inline float acc_cos(float x) { return cosf(x); }
inline float acc_atan2(float y, float x) { return atan2f(y, x); }
inline float acc_asin(float x) { return asinf(x); }
#endif

// Sine and cosine for vertex positions only (never for a decision): the
// hardware approximations after a Cody-Waite reduction by 2 pi (2 pi split as
// 6.28125 + 1.9353071795864769e-3, the first part exact in a few bits), which
// keeps the absolute error near 4e-7 for the angles of an Euler-spiral piece.
SE_HD void vsincos(float x, float* s, float* c) {
#ifdef __CUDA_ARCH__
    float k = rintf(x * 0.15915494309189535f);
    float r = (x - k * 6.28125f) - k * 1.9353071795864769e-3f;
    *s = __sinf(r);
    *c = __cosf(r);
#else
    sincosf(x, s, c);
#endif
}

// ---------------------------------------------------------------------------
// cubic segment
// ---------------------------------------------------------------------------
struct Cubic {
    float2 p[4];
    float2 d[4];  // control points relative to p[0] (d[0] = 0)
    bool line;
};

SE_HD void cubic_local(Cubic& c) {
    c.d[0] = f2(0.0f, 0.0f);
    c.d[1] = sub2(c.p[1], c.p[0]);
    c.d[2] = sub2(c.p[2], c.p[0]);
    c.d[3] = sub2(c.p[3], c.p[0]);
}

// B(t) - p[0], evaluated from the differences so that the chords of small
// pieces keep FP32 precision at the segment's own scale rather than at the
// scale of the absolute coordinates
SE_HD float2 cubic_eval_local(const Cubic& c, float t) {
    float mt = 1.0f - t;
    float b1 = 3.0f * mt * mt * t, b2 = 3.0f * mt * t * t, b3 = t * t * t;
    return f2(b1 * c.d[1].x + b2 * c.d[2].x + b3 * c.d[3].x, b1 * c.d[1].y + b2 * c.d[2].y + b3 * c.d[3].y);
}

SE_HD float2 cubic_deriv(const Cubic& c, float t) {
    float mt = 1.0f - t;
    float2 d01 = sub2(c.p[1], c.p[0]), d12 = sub2(c.p[2], c.p[1]), d23 = sub2(c.p[3], c.p[2]);
    float a = mt * mt, b = 2.0f * mt * t, d = t * t;
    return f2(3.0f * (d01.x * a + d12.x * b + d23.x * d), 3.0f * (d01.y * a + d12.y * b + d23.y * d));
}

// Section 7.3: a derivative below kDerivEps * (control polygon length) is
// re-sampled kDerivDt toward the inside of the piece that ends at t (or, at
// t = 0, starts there).
SE_HD float2 deriv_robust(const Cubic& c, float t) {
    if (c.line) {
        const float2 d = sub2(c.p[3], c.p[0]);
        // a line whose end points coincide in FP32 (a dash part shorter than the
        // coordinates' resolution): the direction of a dot, +x
        return (d.x == 0.0f && d.y == 0.0f) ? f2(1.0f, 0.0f) : d;
    }
    float2 d = cubic_deriv(c, t);
    float S = len2(sub2(c.p[1], c.p[0])) + len2(sub2(c.p[2], c.p[1])) + len2(sub2(c.p[3], c.p[2]));
    float thr = kDerivEps * S;
    if (len2(d) < thr) {
        float tt = t > 0.0f ? t - kDerivDt : t + kDerivDt;
        d = cubic_deriv(c, tt);
        if (d.x == 0.0f && d.y == 0.0f) d = sub2(c.p[3], c.p[0]);
        if (d.x == 0.0f && d.y == 0.0f) d = f2(1.0f, 0.0f);
    }
    return d;
}

// The single formula for every offset point at a sampled (point, derivative):
// P + sh * unit right normal of q.  Segment ends, joins and caps all use it, so
// shared outline vertices are bit-identical across threads.
SE_HD float2 shared_offset(float2 P, float2 q, float sh) {
    if (sh == 0.0f) return P;  // a fill's own vertices
    // vertex placement only: one fast reciprocal (every vertex that two
    // primitives share comes from this one function, so they stay bit-identical)
    const float il = vdiv(1.0f, sqrtf(q.x * q.x + q.y * q.y));
    return f2(P.x + sh * (q.y * il), P.y + sh * (-q.x * il));
}

// ---------------------------------------------------------------------------
// Appendix A: geometric Hermite interpolation (k = th0 + th1, d = th1 - th0)
// ---------------------------------------------------------------------------
SE_HD void gh(float k, float d, float& k1, float& c) {
    float d2 = d * d, k2 = k * k;
    k1 = 6.0f * d - d * d2 * (1.0f / 70.0f) - d * d2 * d2 * (1.0f / 10780.0f) +
         d * d2 * d2 * d2 * 2.769178184818219e-7f - k2 * d * 0.1f + k2 * d * d2 * (1.0f / 4200.0f) +
         k2 * d * d2 * d2 * 1.6959677820260655e-5f - k2 * k2 * d * (1.0f / 1400.0f) +
         k2 * k2 * d * d2 * 6.84915970574303e-5f - k2 * k2 * k2 * d * 7.936475029053326e-6f;
    c = 1.0f - d2 * (1.0f / 40.0f) + d2 * d2 * 0.00034226190482569864f - d2 * d2 * d2 * 1.9349474568904524e-6f -
        k2 * (1.0f / 24.0f) + k2 * d2 * 0.0024702380951963226f - k2 * d2 * d2 * 3.7297408997537985e-5f +
        k2 * k2 * (1.0f / 1920.0f) - k2 * k2 * d2 * 4.87350869747975e-5f - k2 * k2 * k2 * 3.1001936068463107e-6f;
}

// ---------------------------------------------------------------------------
// Section 7.1: error of the cubic -> ES fit, in input units.  Angles: start
// tangent at -th0 and end tangent at +th1 relative to the chord.
// ---------------------------------------------------------------------------
// (with the sines of t0, t1 and t0 + t1 given: the fit evaluates the area for
// two handle-length pairs at the same angles, and an out-of-line sine is not
// merged by the compiler)
SE_HD float es_area(float d0, float d1, float sin_t0, float sin_t1, float sin_t01) {
    return 0.15f * (2.0f * d0 * sin_t0 + 2.0f * d1 * sin_t1 - d0 * d1 * sin_t01);
}

struct Fit {
    float th0, th1, chord, err;
};

// kInlineTrig: the arctangents, cosines and sines inline (the plan pass, whose
// subdivision loop runs the fit many times per segment: 0.32 -> 0.30 ms on
// map-like) or through the out-of-line copies (the piece pass, one fit per
// piece, where the smaller code measured faster).  The same functions either
// way, so the same values.
template <bool kInlineTrig>
static __host__ __device__ __noinline__ Fit fit_es_t(float2 ch, float2 q0, float2 q1, float dt) {
    Fit f;
    f.chord = len2(ch);
    if (f.chord == 0.0f) {
        f.th0 = f.th1 = 0.0f;
        f.err = INFINITY;
        return f;
    }
    f.th0 = kInlineTrig ? atan2f(cross2(q0, ch), dot2(q0, ch)) : acc_atan2(cross2(q0, ch), dot2(q0, ch));
    f.th1 = kInlineTrig ? atan2f(cross2(ch, q1), dot2(ch, q1)) : acc_atan2(cross2(ch, q1), dot2(ch, q1));
    float d0 = len2(q0) * dt / (3.0f * f.chord);
    float d1 = len2(q1) * dt / (3.0f * f.chord);
    float den0 = 1.0f + (kInlineTrig ? cosf(f.th0) : acc_cos(f.th0));
    float den1 = 1.0f + (kInlineTrig ? cosf(f.th1) : acc_cos(f.th1));
    if (!(den0 > 0.0f) || !(den1 > 0.0f)) {
        f.err = INFINITY;
        return f;
    }
    float db0 = 2.0f / (3.0f * den0), db1 = 2.0f / (3.0f * den1);
    float k = f.th0 + f.th1, dd = f.th0 - f.th1;
    float ak = fabsf(k);
    float e1 = 4.6255e-6f * (ak * ak * ak * ak * ak) + 7.5e-3f * k * k * fabsf(dd);
    const float s0 = kInlineTrig ? sinf(f.th0) : acc_sin(f.th0);
    const float s1 = kInlineTrig ? sinf(f.th1) : acc_sin(f.th1);
    const float s01 = kInlineTrig ? sinf(f.th0 + f.th1) : acc_sin(f.th0 + f.th1);
    float e2 = 1.55f * fabsf(es_area(d0, d1, s0, s1, s01) - es_area(db0, db1, s0, s1, s01));
    float e3 = (0.005f * ak + 0.07f * fabsf(dd)) * sqrtf((db0 - d0) * (db0 - d0) + (db1 - d1) * (db1 - d1));
    f.err = (e1 + e2 + e3) * f.chord;
    return f;
}

// ---------------------------------------------------------------------------
// Euler-spiral piece
// ---------------------------------------------------------------------------
struct ES {
    float2 p0, p1, q0, q1;
    float2 rot;  // maps the unit ES (arc length 1) onto the chord
    float th0, th1, k0, k1, L;
    uint32_t degenerate;  // zero chord (64 bytes in all: no padding)
};

SE_HD float es_theta(const ES& e, float s) {
    return -e.th0 + e.k0 * s + 0.5f * e.k1 * (s * s - s);
}

// int_0^s exp(i theta(u)) du by composite 4-point Gauss-Legendre, panels of at
// most 2 rad of turning.  Fast = true uses vsincos (vertex positions).
template <bool Fast>
SE_HD float2 es_unit_pos_t(const ES& e, float s) {
    if (s == 0.0f) return f2(0.0f, 0.0f);
    const float gx[4] = {-0.8611363115940526f, -0.3399810435848563f, 0.3399810435848563f, 0.8611363115940526f};
    const float gw[4] = {0.3478548451374538f, 0.6521451548625461f, 0.6521451548625461f, 0.3478548451374538f};
    float A = (fabsf(e.k0) + fabsf(e.k1)) * fabsf(s);
    int m = 1 + (int)(A * 0.5f);
    if (m > 64) m = 64;
    float h = s / (float)m;
    float ax = 0.0f, ay = 0.0f;
    for (int j = 0; j < m; j++) {
        float base = (float)j * h;
#pragma unroll
        for (int g = 0; g < 4; g++) {
            float sg = base + 0.5f * h * (gx[g] + 1.0f);
            float sn, cs;
            if (Fast) vsincos(es_theta(e, sg), &sn, &cs);
            else sincosf(es_theta(e, sg), &sn, &cs);
            ax += gw[g] * cs;
            ay += gw[g] * sn;
        }
    }
    return f2(0.5f * h * ax, 0.5f * h * ay);
}

// Vertex positions (never a decision): int_s0^s1 exp(i theta(u)) du by
// 3-point Gauss-Legendre on panels of at most 1 rad of turning, with the
// hardware sine and cosine.  Against the exact integral its error stays below
// 3e-6 of the piece length (4 points on 2 rad panels: 3e-7), within the FP32
// resolution of the piece's own angles, and it takes three sines and cosines
// per panel instead of four.
SE_NOINL float2 es_unit_span(const ES& e, float s0, float s1) {
    const float gx[3] = {-0.7745966692414834f, 0.0f, 0.7745966692414834f};
    const float gw[3] = {0.5555555555555556f, 0.8888888888888889f, 0.5555555555555556f};
    const float len = s1 - s0;
    float A = (fabsf(e.k0) + fabsf(e.k1)) * len;
    int m = 1 + (int)A;
    if (m > 128) m = 128;
    float h = m == 1 ? len : vdiv(len, (float)m);
    float ax = 0.0f, ay = 0.0f;
    for (int j = 0; j < m; j++) {
        float base = s0 + (float)j * h;
#pragma unroll
        for (int g = 0; g < 3; g++) {
            float sg = base + 0.5f * h * (gx[g] + 1.0f);
            float sn, cs;
            vsincos(es_theta(e, sg), &sn, &cs);
            ax += gw[g] * cs;
            ay += gw[g] * sn;
        }
    }
    return f2(0.5f * h * ax, 0.5f * h * ay);
}

// Appendix A: the unit ES is scaled, rotated and translated so its ends land on
// the chord; the arc length comes from the same quadrature (|P(1)|).  The
// quadrature takes the hardware sine and cosine: their ~4e-7 absolute error
// moves |P(1)|, and with it L and every count, by under 1e-6 relative, far inside
// the 1e-4 relative distance from an integer below which a count is not resolved.
// The result comes back by value (an ES passed by reference to an out-of-line
// function would have to live in local memory).
struct ESSetup {
    float k0, k1, L;
    float2 rot;
};

SE_NOINL ESSetup es_setup(float th0, float th1, float2 chord, float chord_len) {
    ES e;
    e.th0 = th0;
    e.th1 = th1;
    float c;
    e.k0 = th0 + th1;
    gh(e.k0, th1 - th0, e.k1, c);
    float2 u1 = es_unit_pos_t<true>(e, 1.0f);
    float m = len2(u1);
    ESSetup r;
    r.k0 = e.k0;
    r.k1 = e.k1;
    r.L = chord_len / (m > 0.05f ? m : 0.05f);
    r.rot = cdiv(chord, u1);
    return r;
}

SE_HD float es_kn(const ES& e, float s) { return e.k0 + e.k1 * (s - 0.5f); }

// Point at parameter s, integrated from the nearer end of the piece: from p0
// for s <= 1/2, back from p1 otherwise (p0 + chord = p1 up to the rounding of
// the coordinates), so no vertex integrates over more than half the piece's
// turning -- half the panels in the worst case, where a warp waits for its
// slowest lane.
SE_HD float2 es_pos(const ES& e, float s) {
    const bool back = s > 0.5f;
    const float2 d = cmul(es_unit_span(e, back ? s : 0.0f, back ? 1.0f : s), e.rot);
    return back ? sub2(e.p1, d) : add2(e.p0, d);
}

SE_HD float2 es_tangent(const ES& e, float s) {
    float sn, cs;
    vsincos(es_theta(e, s), &sn, &cs);
    float2 t = cmul(f2(cs, sn), e.rot);
    float il = vdiv(1.0f, len2(t));
    return f2(t.x * il, t.y * il);
}

SE_NOINL float2 es_offset(const ES& e, float s, float sh) {
    if (s == 0.0f) return shared_offset(e.p0, e.q0, sh);
    if (s == 1.0f) return shared_offset(e.p1, e.q1, sh);
    float2 T = es_tangent(e, s);
    float2 P = es_pos(e, s);
    return f2(P.x + sh * T.y, P.y + sh * (-T.x));
}

// Centre of curvature P + N / kappa on an evolute range of the parallel curve at
// signed offset sh.  There 1 + sh kappa <= 0, so the radius 1 / kappa has the
// sign of -sh and magnitude at most |sh|, reaching -sh at the parallel curve's
// cusp (where the evolute meets it); FP32 can round kappa to zero at that end
// of a very short piece, so the radius is held to that bound.
SE_NOINL float2 es_evolute(const ES& e, float s, float sh) {
    float2 T = es_tangent(e, s);
    float2 P = es_pos(e, s);
    float r = vdiv(e.L, es_kn(e, s));  // the radius 1 / kappa
    if (!(fabsf(r) <= fabsf(sh))) r = -sh;
    return f2(P.x + (-T.y) * r, P.y + T.x * r);
}

// ---------------------------------------------------------------------------
// Section 4.2: piecewise approximation F of the density integral, handled as
// divided differences over "anchored" abscissae u with e = |u| - 1 carried
// separately, so that FP32 keeps full relative precision near the inflection
// (u = -1) and the offset cusp (u = +1) and when curvature is nearly constant.
// ---------------------------------------------------------------------------
constexpr float kC1 = 1.0976991822760038f;
constexpr float kC2 = 0.9148117935952064f;
constexpr float kC3 = 0.16145779359520596f;
constexpr float kK = 0.9428090415820634f;  // sqrt(8) / 3

struct UA {
    float u, e;
};

// u = -1 - 2 sh_n kappa (inflection -> -1, offset cusp -> +1)
SE_HD UA make_ua(float sh_n, float kap) {
    float t = 2.0f * sh_n * kap;
    UA r;
    r.u = -1.0f - t;
    r.e = (r.u < 0.0f) ? t : -2.0f * (1.0f + sh_n * kap);
    return r;
}

SE_HD int region(float u) {
    float a = fabsf(u);
    int p = a < 0.8f ? 0 : (a < 1.25f ? 1 : (a < 2.1f ? 2 : 3));
    return (p == 0) ? 0 : (u < 0.0f ? -p : p);
}

SE_HD float sincf(float x) {
    float ax = fabsf(x);
    if (ax < 1e-3f) return 1.0f - x * x * (1.0f / 6.0f);
    return acc_sin(x) / x;
}

// divided difference of g(e) = e |e|^0.5
SE_HD float dd_g(float ea, float eb) {
    float a = fabsf(ea), b = fabsf(eb);
    if (a + b == 0.0f) return 0.0f;
    if ((ea >= 0.0f) == (eb >= 0.0f) || a == 0.0f || b == 0.0f) {
        float ra = sqrtf(a), rb = sqrtf(b);
        return (a + ra * rb + b) / (ra + rb);
    }
    return (a * sqrtf(a) + b * sqrtf(b)) / (a + b);
}

// divided difference of F over [x, y] within one region (x, y anchored)
SE_HD float dd_region(int r, UA x, UA y) {
    int p = r < 0 ? -r : r;
    if (p == 0) {
        float m = 0.5f * (x.u + y.u), d = y.u - x.u;
        return acc_cos(kC1 * m) * sincf(0.5f * kC1 * d);
    }
    if (p == 1) return kK * dd_g(x.e, y.e);
    if (p == 2) return 0.6406f * (fabsf(x.u) + fabsf(y.u)) - 0.81f;
    return 0.5f * (fabsf(x.u) + fabsf(y.u)) - 0.156f;
}

SE_HD UA boundary_ua(float b) {
    UA r;
    r.u = b;
    r.e = fabsf(b) - 1.0f;
    return r;
}

// next region boundary strictly between cur and the target, in the direction of travel
SE_HD bool next_boundary(float cur, float target, float& b) {
    const float bs[6] = {-2.1f, -1.25f, -0.8f, 0.8f, 1.25f, 2.1f};
    if (target > cur) {
        for (int i = 0; i < 6; i++)
            if (bs[i] > cur && bs[i] < target) { b = bs[i]; return true; }
    } else {
        for (int i = 5; i >= 0; i--)
            if (bs[i] < cur && bs[i] > target) { b = bs[i]; return true; }
    }
    return false;
}

// divided difference of F over [a, b] (any order); each sub-interval between
// region boundaries takes the region of its midpoint
SE_NOINL float dd_F(UA a, UA b) {
    const bool single = region(a.u) == region(b.u);
    float num = 0.0f, den = 0.0f, bnd;
    UA x = a;
    if (!single) {
        while (next_boundary(x.u, b.u, bnd)) {
            UA y = boundary_ua(bnd);
            float w = y.u - x.u;
            num += dd_region(region(0.5f * (x.u + y.u)), x, y) * w;
            den += w;
            x = y;
        }
    }
    // the last sub-interval (for a range inside one region, the only one) at one
    // call site: a warp whose ranges cross boundaries and ranges that do not
    // evaluates it once
    const float d = dd_region(single ? region(a.u) : region(0.5f * (x.u + b.u)), x, b);
    if (single) return d;
    float w = b.u - x.u;
    num += d * w;
    den += w;
    return num / den;
}

// Section 4.1: lines needed for the parallel curve at normalised signed offset
// sh_n over [a, b] of the unit ES: (b - a) * DD_F / (2 sqrt|sh_n|) / sqrt(8 tol_n).
SE_NOINL float line_count(float k0, float k1, float sh_n, float a, float b, float tol_n) {
    UA ua = make_ua(sh_n, k0 + k1 * (a - 0.5f));
    UA ub = make_ua(sh_n, k0 + k1 * (b - 0.5f));
    float I = (b - a) * dd_F(ua, ub) / (2.0f * sqrtf(fabsf(sh_n)));
    return fabsf(I) / sqrtf(8.0f * tol_n);
}

// --- vertex placement (never a decision): the same inverse with the hardware
// sine/cosine, from a per-range precomputation ---------------------------------
SE_HD float sincf_v(float x) {
    float ax = fabsf(x);
    if (ax < 1e-3f) return 1.0f - x * x * (1.0f / 6.0f);
    float sn, cs;
    vsincos(x, &sn, &cs);
    return vdiv(sn, x);
}

// dd_g for vertex placement (fast division)
SE_HD float dd_g_v(float ea, float eb) {
    float a = fabsf(ea), b = fabsf(eb);
    if (a + b == 0.0f) return 0.0f;
    if ((ea >= 0.0f) == (eb >= 0.0f) || a == 0.0f || b == 0.0f) {
        float ra = sqrtf(a), rb = sqrtf(b);
        return vdiv(a + ra * rb + b, ra + rb);
    }
    return vdiv(a * sqrtf(a) + b * sqrtf(b), a + b);
}

SE_HD float dd_region_v(int r, UA x, UA y) {
    int p = r < 0 ? -r : r;
    if (p == 0) {
        float m = 0.5f * (x.u + y.u), d = y.u - x.u;
        float sn, cs;
        vsincos(kC1 * m, &sn, &cs);
        return cs * sincf_v(0.5f * kC1 * d);
    }
    if (p == 1) return kK * dd_g_v(x.e, y.e);
    if (p == 2) return 0.6406f * (fabsf(x.u) + fabsf(y.u)) - 0.81f;
    return 0.5f * (fabsf(x.u) + fabsf(y.u)) - 0.156f;
}

// first region boundary strictly between cur and target, in the direction of travel
SE_HD bool next_bnd(float cur, float target, float& b) {
    if (target > cur) {
        b = cur < -2.1f ? -2.1f : cur < -1.25f ? -1.25f : cur < -0.8f ? -0.8f : cur < 0.8f ? 0.8f : cur < 1.25f ? 1.25f
                                                                                                      : 2.1f;
        return cur < 2.1f && b < target;
    }
    b = cur > 2.1f ? 2.1f : cur > 1.25f ? 1.25f : cur > 0.8f ? 0.8f : cur > -0.8f ? -0.8f : cur > -1.25f ? -1.25f
                                                                                                   : -2.1f;
    return cur > -2.1f && b > target;
}

// ginv(G) = sign(G) |G|^(2/3), the inverse of g(e) = e |e|^0.5
SE_HD float ginv(float G) { return copysignf(cbrtf(G * G), G); }

// Solve F(x + d) - F(x) = y for d inside region r (x anchored).
SE_HD float solve_region(int r, UA x, float y) {
    int p = r < 0 ? -r : r;
    float su = (r < 0) ? -1.0f : 1.0f;
    if (p == 0) {
        float s0 = acc_sin(kC1 * x.u) + kC1 * y;
        s0 = fminf(1.0f, fmaxf(-1.0f, s0));
        float d = acc_asin(s0) / kC1 - x.u;
        // refine: d = y / DD(x, x + d), insensitive to the error in d
        for (int it = 0; it < 2; it++) {
            UA z;
            z.u = x.u + d;
            z.e = 0.0f;
            float dd = dd_region(0, x, z);
            if (dd > 0.0f) d = y / dd;
        }
        return d;
    }
    if (p == 1) {
        float ys = su * y / kK;  // change of g(e)
        float ex = x.e;
        float e2 = ginv(ex * sqrtf(fabsf(ex)) + ys);
        float ddg = dd_g(ex, e2);
        float de = (ddg > 0.0f) ? ys / ddg : e2 - ex;
        return su * de;
    }
    float A = (p == 2) ? 0.6406f : 0.5f;
    float B = (p == 2) ? -0.81f : -0.156f;
    float a = fabsf(x.u);
    float yp = su * y;
    float Bq = 2.0f * A * a + B;
    float disc = fmaxf(Bq * Bq + 4.0f * A * yp, 0.0f);
    float da = 2.0f * yp / (Bq + sqrtf(disc));
    return su * da;
}

// The region-local solve of solve_region for vertex placement (its arcsine
// inline: the emit's hot path, where an out-of-line call cost more than the
// code it saves).  In region 0,
// F(u) = sin(c1 u) / c1, so with S, C = sin, cos(c1 x) and t = S + c1 y the
// step is c1 d = asin(t C - S sqrt(1 - t^2)); writing t C - S sqrt(1 - t^2) as
// c1 y (C + S (t + S) / (C + sqrt(1 - t^2))) removes the cancellation between
// the two products (C >= cos(0.8 c1) > 0.6 in region 0), so one hardware
// sine/cosine and one arcsine place the vertex.
SE_HD float solve_region_v(int r, UA x, float y) {
    int p = r < 0 ? -r : r;
    if (p == 0) {
        float S, C;
        vsincos(kC1 * x.u, &S, &C);
        const float t = fminf(1.0f, fmaxf(-1.0f, S + kC1 * y));
        const float rt = sqrtf(fmaxf(0.0f, (1.0f - t) * (1.0f + t)));
        const float q = kC1 * y * (C + vdiv(S * (t + S), C + rt));
        return asinf(fminf(1.0f, fmaxf(-1.0f, q))) * (1.0f / kC1);
    }
    // regions 1-3: the steps of solve_region with fast division
    const float su = (r < 0) ? -1.0f : 1.0f;
    if (p == 1) {
        const float ys = su * y * (1.0f / kK);  // change of g(e)
        const float ex = x.e;
        const float e2 = ginv(ex * sqrtf(fabsf(ex)) + ys);
        const float ddg = dd_g_v(ex, e2);
        const float de = (ddg > 0.0f) ? vdiv(ys, ddg) : e2 - ex;
        return su * de;
    }
    const float A = (p == 2) ? 0.6406f : 0.5f;
    const float B = (p == 2) ? -0.81f : -0.156f;
    const float yp = su * y;
    const float Bq = 2.0f * A * fabsf(x.u) + B;
    const float disc = fmaxf(Bq * Bq + 4.0f * A * yp, 0.0f);
    return su * vdiv(2.0f * yp, Bq + sqrtf(disc));
}

// Per-range data of the vertex placement below, computed once per range by the
// piece pass: the anchored start abscissa, u(b), du and the F difference.
struct LineInv {
    float ua_u, ua_e, ub_u, du, total;
};

SE_NOINL LineInv line_inv(const ES& e, float sh_n, float a, float b) {
    UA ua = make_ua(sh_n, es_kn(e, a));
    UA ub = make_ua(sh_n, es_kn(e, b));
    LineInv li;
    li.ua_u = ua.u;
    li.ua_e = ua.e;
    li.ub_u = ub.u;
    li.du = -2.0f * sh_n * e.k1 * (b - a);
    li.total = li.du == 0.0f ? 0.0f : dd_F(ua, ub) * li.du;
    return li;
}

// line_s from a LineInv (vertex placement; inline in its one caller, the emit's
// vertex routine: 1.38 against 1.40 ms out of line)
SE_HD float line_s_v(const LineInv& li, float a, float b, int i, int n) {
    if (i == 0) return a;
    if (i == n) return b;
    float fr = vdiv((float)i, (float)n);
    if (li.du == 0.0f) return a + (b - a) * fr;
    float y = fr * li.total;
    UA x;
    x.u = li.ua_u;
    x.e = li.ua_e;
    float end_u = li.ub_u, walked = 0.0f, bnd;
    while (next_bnd(x.u, li.ub_u, bnd)) {
        UA yb = boundary_ua(bnd);
        float w = yb.u - x.u;
        float inc = dd_region_v(region(0.5f * (x.u + yb.u)), x, yb) * w;
        if (fabsf(y) <= fabsf(inc)) {
            end_u = yb.u;
            break;
        }
        y -= inc;
        walked += w;
        x = yb;
    }
    float d = solve_region_v(region(0.5f * (x.u + end_u)), x, y);
    float lam = vdiv(walked + d, li.du);
    lam = fminf(1.0f, fmaxf(0.0f, lam));
    return a + (b - a) * lam;
}

// Fill flattening (offset 0): parameter of vertex i of n at equal steps of
// g(k) = k |k|^(1/2) between the range's curvatures (LineInv holds k_a, k_b,
// k_b - k_a and g(k_b) - g(k_a)), solved relative to k_a.
SE_NOINL float fill_s_v(const LineInv& li, float a, float b, int i, int n) {
    if (i == 0) return a;
    if (i == n) return b;
    float fr = (float)i / (float)n;
    if (li.du == 0.0f) return a + (b - a) * fr;
    const float ka = li.ua_u;
    const float y = fr * li.total;
    const float k2 = ginv(ka * sqrtf(fabsf(ka)) + y);
    const float ddg = dd_g(ka, k2);
    const float dk = ddg > 0.0f ? y / ddg : k2 - ka;
    float lam = dk / li.du;
    lam = fminf(1.0f, fmaxf(0.0f, lam));
    return a + (b - a) * lam;
}

// --- refined mode (Section 4.2): the exact integral f of Section 4.1 --------
// f(u) = int_0^u sqrt|v^2 - 1| dv, odd.  Divided differences are formed without
// subtracting nearby values of f, in three classes by |u|:
//   zero  |u| <= 1/2   closed form; differences of u sqrt(1 - u^2) and asin u
//                       rewritten with c = sqrt(1 - u^2) and the sine of a difference
//   cusp  1/2 < |u| <= 3/2   f = sign(u) (pi/4 + sqrt2 g(e) P(e)), e = |u| - 1,
//                       g(e) = e |e|^(1/2) and P the binomial series of
//                       sqrt(1 + e/2) integrated against t^(1/2) (|e/2| <= 1/4)
//   far   |u| > 3/2    closed form; differences of u sqrt(u^2 - 1) and acosh u
//                       rewritten with s = sqrt(u^2 - 1) and the log of a ratio
constexpr int kSerTerms = 11;  // |e/2|^11 / 12.5 < 1e-9 at the class edge
struct SerCoef {
    float p[kSerTerms];
};
// p_k = binom(1/2, k) 2^-k / (k + 3/2)
__host__ __device__ constexpr SerCoef ser_coef() {
    SerCoef c{};
    double b = 1.0;
    double two = 1.0;
    for (int k = 0; k < kSerTerms; k++) {
        c.p[k] = (float)(b / two / (k + 1.5));
        b = b * (0.5 - k) / (k + 1);
        two *= 2.0;
    }
    return c;
}
constexpr float kSqrt2 = 1.41421356237309505f;

// P(y) and the divided difference (P(y) - P(x)) / (y - x), by synthetic division
SE_HD void ser_eval(float x, float y, float& Py, float& dP) {
    constexpr SerCoef kSer = ser_coef();
    float v = kSer.p[kSerTerms - 1], d = 0.0f;
#pragma unroll
    for (int k = kSerTerms - 2; k >= 0; k--) {
        d = d * x + v;
        v = v * y + kSer.p[k];
    }
    Py = v;
    dP = d;
}

SE_HD int xregion(float u) {
    float a = fabsf(u);
    int p = a <= 0.5f ? 0 : (a <= 1.5f ? 1 : 2);
    return (p == 0) ? 0 : (u < 0.0f ? -p : p);
}

// first class boundary strictly between cur and target, in the direction of travel
SE_HD bool next_xbnd(float cur, float target, float& b) {
    if (target > cur) {
        b = cur < -1.5f ? -1.5f : cur < -0.5f ? -0.5f : cur < 0.5f ? 0.5f : 1.5f;
        return cur < 1.5f && b < target;
    }
    b = cur > 1.5f ? 1.5f : cur > 0.5f ? 0.5f : cur > -0.5f ? -0.5f : -1.5f;
    return cur > -1.5f && b > target;
}

// divided difference of f over [x, y] within one class (x == y gives f'(x))
SE_HD float ddx_region(int r, UA x, UA y) {
    int p = r < 0 ? -r : r;
    if (p == 0) {
        const float cx = sqrtf(-x.e * (2.0f + x.e)), cy = sqrtf(-y.e * (2.0f + y.e));
        const float q = x.u * (x.u + y.u) / (cx + cy);
        const float w = cx + q;
        const float z = (y.u - x.u) * w;
        const float A = z == 0.0f ? 1.0f : acc_asin(z) / z;
        return 0.5f * (cy - q + A * w);
    }
    if (p == 1) {
        float Py, dP;
        ser_eval(x.e, y.e, Py, dP);
        return kSqrt2 * (dd_g(x.e, y.e) * Py + x.e * sqrtf(fabsf(x.e)) * dP);
    }
    const float a = fabsf(x.u), b = fabsf(y.u);
    const float sa = sqrtf(x.e * (2.0f + x.e)), sb = sqrtf(y.e * (2.0f + y.e));
    const float q = (a + b) / (sa + sb);
    const float w = (1.0f + q) / (a + sa);
    const float z = (b - a) * w;
    const float Lz = z == 0.0f ? 1.0f : log1pf(z) / z;
    return 0.5f * (sb + a * q - Lz * w);
}

// divided difference of f over [a, b] (any order), class by class
SE_NOINL float dd_Fx(UA a, UA b) {
    if (xregion(a.u) == xregion(b.u)) return ddx_region(xregion(a.u), a, b);
    float num = 0.0f, den = 0.0f, bnd;
    UA x = a;
    while (next_xbnd(x.u, b.u, bnd)) {
        UA y = boundary_ua(bnd);
        float w = y.u - x.u;
        num += ddx_region(xregion(0.5f * (x.u + y.u)), x, y) * w;
        den += w;
        x = y;
    }
    float w = b.u - x.u;
    num += ddx_region(xregion(0.5f * (x.u + b.u)), x, b) * w;
    den += w;
    return num / den;
}

// f itself (for the starting value only)
SE_HD float fx_abs(UA x) {
    const float a = fabsf(x.u);
    float r;
    const int p = xregion(a);
    if (p == 0) r = 0.5f * (a * sqrtf(-x.e * (2.0f + x.e)) + acc_asin(a));
    else if (p == 1) {
        float Py, dP;
        ser_eval(x.e, x.e, Py, dP);
        r = 0.25f * kPi + kSqrt2 * x.e * sqrtf(fabsf(x.e)) * Py;
    } else r = 0.5f * (a * sqrtf(x.e * (2.0f + x.e)) - acoshf(a)) + 0.25f * kPi;
    return copysignf(r, x.u);
}

// inverse of the approximation of Section 4.2, piece by piece (odd)
SE_HD float fa_inv(float y) {
    const float a = fabsf(y);
    const float y08 = sinf(kC1 * 0.8f) / kC1;
    const float y125 = kK * 0.125f + 0.25f * kPi;
    const float y21 = 0.6406f * 2.1f * 2.1f - 0.81f * 2.1f + kC2;
    float x;
    if (a < y08) x = acc_asin(fminf(1.0f, kC1 * a)) / kC1;
    else if (a < y125) x = 1.0f + ginv((a - 0.25f * kPi) / kK);
    else if (a < y21) x = (0.81f + sqrtf(fmaxf(0.81f * 0.81f - 4.0f * 0.6406f * (kC2 - a), 0.0f))) / (2.0f * 0.6406f);
    else x = 0.156f + sqrtf(fmaxf(0.156f * 0.156f - 2.0f * (kC3 - a), 0.0f));
    return copysignf(x, y);
}

// the point u(x) + d, keeping e = |u| - 1 anchored while the sign of u holds
SE_HD UA ua_step(UA x, float d) {
    UA r;
    r.u = x.u + d;
    if (x.u != 0.0f && (r.u >= 0.0f) == (x.u >= 0.0f)) r.e = x.e + (x.u > 0.0f ? d : -d);
    else r.e = fabsf(r.u) - 1.0f;
    return r;
}

// Refined vertex placement: li.total holds the exact integral's difference
// f(ub) - f(ua) (du times its divided difference).  The starting value is the
// approximation's inverse of the target f(ua) + fr (f(ub) - f(ua)); two Newton
// steps on lam in [0, 1], with f(u(lam)) - f(ua) formed as a divided difference
// from ua, refine it (Section 4.2).
SE_NOINL float line_s_refined(const LineInv& li, float a, float b, int i, int n) {
    if (i == 0) return a;
    if (i == n) return b;
    const float fr = (float)i / (float)n;
    if (li.du == 0.0f) return a + (b - a) * fr;
    UA ua;
    ua.u = li.ua_u;
    ua.e = li.ua_e;
    const float D = li.total / li.du;
    const float u0 = fa_inv(fx_abs(ua) + fr * li.total);
    float lam = fminf(1.0f, fmaxf(0.0f, (u0 - ua.u) / li.du));
    for (int it = 0; it < 2; it++) {
        const UA x = ua_step(ua, lam * li.du);
        const float fp = sqrtf(fabsf(x.e * (2.0f + x.e)));
        if (fp > 0.0f) {
            const float res = dd_Fx(ua, x) * lam - fr * D;
            lam = fminf(1.0f, fmaxf(0.0f, lam - res / fp));
        }
    }
    return a + (b - a) * lam;
}

// Parameter s in [a, b] of vertex i of n on the line-flattened parallel curve:
// equal steps of F between u(a) and u(b) (Section 4.1), inverted region by
// region relative to the current anchor.
SE_NOINL float line_s(const ES& e, float sh_n, float a, float b, int i, int n) {
    if (i == 0) return a;
    if (i == n) return b;
    float fr = (float)i / (float)n;
    UA ua = make_ua(sh_n, es_kn(e, a));
    UA ub = make_ua(sh_n, es_kn(e, b));
    // u is linear in s: du = -2 sh_n k1 (b - a) exactly, whereas ub.u - ua.u
    // loses the digits that u = -1 - 2 sh_n kappa rounds away near |u| = 1
    float du = -2.0f * sh_n * e.k1 * (b - a);
    if (du == 0.0f) return a + (b - a) * fr;
    float total = dd_F(ua, ub) * du;
    float y = fr * total;
    UA x = ua;
    UA end = ub;
    float walked = 0.0f, bnd;
    while (next_boundary(x.u, ub.u, bnd)) {
        UA yb = boundary_ua(bnd);
        float w = yb.u - x.u;
        float inc = dd_region(region(0.5f * (x.u + yb.u)), x, yb) * w;
        if (fabsf(y) <= fabsf(inc)) {
            end = yb;
            break;
        }
        y -= inc;
        walked += w;
        x = yb;
    }
    float d = solve_region(region(0.5f * (x.u + end.u)), x, y);
    float lam = (walked + d) / du;
    lam = fminf(1.0f, fmaxf(0.0f, lam));
    return a + (b - a) * lam;
}

// Section 5: arcs for the ES parallel curve over arc length S, curvature slope kp
SE_HD float arc_count(float S, float kp, float h, float tol) {
    return S * cbrtf(fabsf(kp) * (1.0f + 0.4f * fabsf(h * S * kp)) / (120.0f * tol));
}

// Section 6: evolute lines over [a, b] (density |s - s_infl|^-1/2)
SE_NOINL float evolute_count(float k0, float k1, float L, float a, float b, float tol) {
    if (k1 == 0.0f) return 0.0f;
    float s0 = 0.5f - k0 / k1;
    float ga = sqrtf(fabsf(a - s0)), gb = sqrtf(fabsf(b - s0));
    return 2.0f * sqrtf(L) * (b - a) / (ga + gb) / sqrtf(8.0f * tol);
}

SE_NOINL float evolute_s(const ES& e, float a, float b, int i, int n) {
    if (i == 0) return a;
    if (i == n) return b;
    float fr = vdiv((float)i, (float)n);
    if (e.k1 == 0.0f) return a + (b - a) * fr;
    float s0 = 0.5f - vdiv(e.k0, e.k1);
    float ga = sqrtf(fabsf(a - s0)), gb = sqrtf(fabsf(b - s0));
    float gi = ga + fr * (gb - ga);
    return a + vdiv((b - a) * fr * (gi + ga), ga + gb);
}

// Section 2.1: exact arc metric, lines for a circular arc of radius r turning by ang
SE_HD float round_N(float ang, float r, float tol) {
    float x = 1.0f - tol / r;
    x = fminf(1.0f, fmaxf(-1.0f, x));
    return ang / (2.0f * acosf(x));
}

// ceil with the max(1, .) floor used for every count; clamps to SE_MAX_RANGE_COUNT
SE_HD uint32_t count_of(float N, uint32_t& flags) {
    if (!(N == N)) N = 1.0f;
    float c = ceilf(N);
    if (c < 1.0f) c = 1.0f;
    if (c > (float)SE_MAX_RANGE_COUNT) {
        flags |= 1u;
        c = (float)SE_MAX_RANGE_COUNT;
    }
    return (uint32_t)c;
}

SE_HD float menger(float2 a, float2 m, float2 b) {
    float cr = cross2(sub2(m, a), sub2(b, m));
    float d = len2(sub2(m, a)) * len2(sub2(b, m)) * len2(sub2(b, a));
    return d > 0.0f ? 2.0f * cr / d : 0.0f;
}

SE_HD float2 rotate(float2 v, float ang) {
    float sn, cs;
    vsincos(ang, &sn, &cs);
    return f2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
}

}  // namespace se
