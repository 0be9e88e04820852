// Device dashing (SVG dash semantics; the paper dashes on the CPU, Section 9.3,
// and leaves GPU dashing to future work, Section 10).
//
// A dashed subpath becomes a sequence of open subpaths, one per "on" interval
// of the pattern, each made of the parts of the source segments that the
// interval covers.  The pass works per segment:
//
//   * the FP32 arc length of each segment, by adaptive Gauss-Legendre
//     quadrature of |B'(t)| (fixed panels resolve the sharp minimum of |B'| at
//     a near-cusp only to ~1e-5; the adaptive rule reaches ~2e-7);
//   * a segmented scan of the lengths, in exact fixed point (units of 2^-32),
//     gives each segment the arc length at which it ends within its subpath;
//     integer sums do not depend on the order of the scan, so a subpath gets
//     the same positions whichever scene or batch it is expanded in;
//   * each segment owns the pattern boundaries that fall inside it, found
//     from its two end positions; a boundary position is one canonical
//     function of (period index, pattern index), and the end of segment j is
//     the same stored value as the start of segment j + 1, so every boundary
//     belongs to exactly one segment;
//   * a cut at arc length s becomes a parameter t by inverting the same
//     quadrature, and each part [ta, tb] of a cubic becomes the sub-cubic with
//     the blossom values B(ta,ta,ta), B(ta,ta,tb), B(ta,tb,tb), B(tb,tb,tb).
#pragma once

#include "launch.h"
#include "pipeline.cuh"
#include "stroke_math.cuh"

namespace se {

// ---------------------------------------------------------------------------
// double-float arithmetic: a value is the unevaluated sum hi + lo
// (Dekker 1971; Knuth's TwoSum; the "accurate" sum of Hida, Li and Bailey)
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

SE_HD DF df_make(float a) {
    DF r;
    r.hi = a;
    r.lo = 0.0f;
    return r;
}

// s + e == a + b exactly
SE_HD DF two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    DF r;
    r.hi = s;
    r.lo = e;
    return r;
}

// exact when |a| >= |b| (or a == 0)
SE_HD DF quick_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    DF r;
    r.hi = s;
    r.lo = e;
    return r;
}

SE_HD DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    DF t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

SE_HD DF df_neg(DF a) {
    a.hi = -a.hi;
    a.lo = -a.lo;
    return a;
}

SE_HD DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

// a * b for a float b; the product of the high parts is exact through a fused
// multiply-add (an explicit fmaf is fused whatever the contraction setting)
SE_HD DF df_mul_f(DF a, float b) {
    float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e += a.lo * b;
    return quick_two_sum(p, e);
}

// arc length in fixed point: units of 2^-32 (exact for lengths >= 2^-9; a
// subpath may hold up to 2^30 units of length)
constexpr float kFixScale = 4294967296.0f;
constexpr long long kFixMax = 1ll << 62;

SE_HD long long fix_of(float len) {
#ifdef __CUDA_ARCH__
    return __float2ll_rn(len * kFixScale);
#else
    return llrintf(len * kFixScale);
#endif
}

// a fixed-point length as a double-float (relative error 2^-48)
SE_HD DF df_of_fix(long long q) {
    float h = (float)q;
    long long hq = (long long)h;
    float l = (float)(q - hq);
    DF r;
    r.hi = h * (1.0f / kFixScale);
    r.lo = l * (1.0f / kFixScale);
    return quick_two_sum(r.hi, r.lo);
}

SE_HD bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
SE_HD bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
SE_HD float df_float(DF a) { return a.hi + a.lo; }

// ---------------------------------------------------------------------------
// arc length of a cubic: adaptive 8-point Gauss-Legendre on |B'(t)|
// ---------------------------------------------------------------------------
constexpr int kArcDepth = 12;       // finest panel: 2^-12 of the parameter range
constexpr float kArcTol = 1e-6f;    // accept a panel when its halves agree to kArcTol * poly * width

struct Speed {
    float2 a, b, c;  // B'(t) = 3 ((1-t)^2 a + 2 (1-t) t b + t^2 c)
};

SE_HD Speed speed_of(const Cubic& cu) {
    Speed s;
    s.a = sub2(cu.p[1], cu.p[0]);
    s.b = sub2(cu.p[2], cu.p[1]);
    s.c = sub2(cu.p[3], cu.p[2]);
    return s;
}

SE_HD float speed_at(const Speed& s, float t) {
    float mt = 1.0f - t;
    float A = mt * mt, B = 2.0f * mt * t, C = t * t;
    float x = 3.0f * (s.a.x * A + s.b.x * B + s.c.x * C);
    float y = 3.0f * (s.a.y * A + s.b.y * B + s.c.y * C);
    return sqrtf(x * x + y * y);
}

// int_lo^hi |B'(t)| dt by the 8-point rule
SE_HD float speed_gl(const Speed& s, float lo, float hi) {
    const float X[8] = {0.019855071751231912f, 0.10166676129318664f, 0.2372337950418355f, 0.40828267875217511f,
                        0.59171732124782483f,  0.7627662049581645f,  0.89833323870681336f, 0.98014492824876809f};
    const float W[8] = {0.050614268145188532f, 0.11119051722668721f, 0.15685332293894344f, 0.18134189168918083f,
                        0.18134189168918083f,  0.15685332293894344f, 0.11119051722668721f, 0.050614268145188532f};
    float w = hi - lo, acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; i++) acc += W[i] * speed_at(s, lo + w * X[i]);
    return acc * w;
}

// Depth-first walk over the accepted panels, left to right.  Each accepted
// panel is a pair of halves [lo, mid], [mid, hi] with integrals L, R; the
// running total is a compensated (Kahan) sum of L + R.  The length of the
// segment is the total after the last pair; t_at() inverts the walk's own
// partial sums, so a cut and the segment length use the same numbers.
struct ArcWalk {
    Speed sp;
    float poly;
    float st_lo[kArcDepth + 2], st_hi[kArcDepth + 2], st_w[kArcDepth + 2];
    int st_d[kArcDepth + 2];
    int top;
    float tot, comp;          // sum of the accepted pairs before the current one
    float lo, mid, hi, L, R;  // current pair
    bool have;

    SE_HD void init(const Cubic& cu) {
        sp = speed_of(cu);
        poly = len2(sp.a) + len2(sp.b) + len2(sp.c);
        top = 0;
        st_lo[0] = 0.0f;
        st_hi[0] = 1.0f;
        st_w[0] = speed_gl(sp, 0.0f, 1.0f);
        st_d[0] = 0;
        top = 1;
        tot = 0.0f;
        comp = 0.0f;
        have = false;
    }

    // advance to the next accepted pair; false when the walk is over
    SE_HD bool next() {
        while (top > 0) {
            top--;
            float a = st_lo[top], b = st_hi[top], whole = st_w[top];
            int d = st_d[top];
            float m = 0.5f * (a + b);
            float l = speed_gl(sp, a, m), r = speed_gl(sp, m, b);
            if (d >= kArcDepth || fabsf((l + r) - whole) <= kArcTol * poly * (b - a)) {
                lo = a;
                mid = m;
                hi = b;
                L = l;
                R = r;
                return true;
            }
            // right half first so that the left half is walked first
            st_lo[top] = m;
            st_hi[top] = b;
            st_w[top] = r;
            st_d[top] = d + 1;
            top++;
            st_lo[top] = a;
            st_hi[top] = m;
            st_w[top] = l;
            st_d[top] = d + 1;
            top++;
        }
        return false;
    }

    SE_HD void accept() {
        float y = (L + R) - comp;
        float t = tot + y;
        comp = (t - tot) - y;
        tot = t;
    }

    // parameter in [x0, x1] at which x0's partial integral reaches g (0 <= g <= whole):
    // safeguarded Newton, stopped once the residual is within the FP32 resolution
    // of the segment's arc length (~1e-7 of its control polygon) or the bracket
    // is a few ulps wide
    SE_HD float solve(float x0, float x1, float g, float whole) const {
        if (!(g > 0.0f)) return x0;
        if (!(g < whole)) return x1;
        const float ftol = 1e-7f * poly;
        float a = x0, b = x1;
        float t = x0 + (x1 - x0) * (g / whole);
        for (int it = 0; it < 40; it++) {
            float f = speed_gl(sp, x0, t) - g;
            if (fabsf(f) <= ftol) break;
            if (f > 0.0f) b = t;
            else a = t;
            if (!(b - a > 4.8e-7f * fmaxf(fabsf(t), 1e-30f))) break;
            float v = speed_at(sp, t);
            float tn = v > 0.0f ? t - f / v : 0.5f * (a + b);
            if (!(tn > a && tn < b)) tn = 0.5f * (a + b);
            t = tn;
        }
        return t;
    }

    // parameter at arc length s; calls must come with non-decreasing s
    SE_HD float t_at(float s) {
        for (;;) {
            if (!have) {
                if (!next()) return 1.0f;
                have = true;
            }
            if (s < tot + (L + R) || top == 0) break;
            accept();
            have = false;
        }
        float g = s - tot;
        if (g <= L) return solve(lo, mid, g, L);
        return solve(mid, hi, g - L, R);
    }
};

// The accepted panels of a walk, recorded once per segment so that each of its
// cuts can be solved on its own: per pair the bounds, the integrals of the two
// halves and the (compensated) sum of the pairs before it.
constexpr int kPanelMax = 24;

struct PanelPair {
    float lo, hi, L, R, tot;
};

// Records the walk's pairs; false when the segment has more than kPanelMax.
SE_HD bool record_panels(const Cubic& cu, PanelPair* out, uint32_t& n) {
    ArcWalk w;
    w.init(cu);
    n = 0;
    while (w.next()) {
        if (n == (uint32_t)kPanelMax) return false;
        PanelPair& q = out[n++];
        q.lo = w.lo;
        q.hi = w.hi;
        q.L = w.L;
        q.R = w.R;
        q.tot = w.tot;
        w.accept();
    }
    return true;
}

// Parameter at arc length s from a recorded walk: the pair holding s (the
// last pair whose running sum is <= s), then the same solve as ArcWalk::t_at.
SE_HD float t_from_panels(const Cubic& cu, const PanelPair* pp, uint32_t n, float s) {
    if (n == 0) return 1.0f;
    uint32_t j = 0;
    for (uint32_t step = 16; step > 0; step >>= 1)
        if (j + step < n && pp[j + step].tot <= s) j += step;
    // ArcWalk::t_at moves on while s >= tot + (L + R) and pairs remain
    while (j + 1 < n && !(s < pp[j].tot + (pp[j].L + pp[j].R))) j++;
    ArcWalk w;
    w.sp = speed_of(cu);
    w.poly = len2(w.sp.a) + len2(w.sp.b) + len2(w.sp.c);
    const PanelPair& q = pp[j];
    const float mid = 0.5f * (q.lo + q.hi);
    const float g = s - q.tot;
    if (g <= q.L) return w.solve(q.lo, mid, g, q.L);
    return w.solve(mid, q.hi, g - q.L, q.R);
}

// FP32 arc length of a segment
SE_HD float seg_arc_length(const Cubic& cu) {
    if (cu.line) return len2(cu.d[3]);
    ArcWalk w;
    w.init(cu);
    while (w.next()) w.accept();
    return w.tot;
}

// point of the blossom B(u1, u2, u3), from the local control points
SE_HD float2 blossom(const Cubic& cu, float u1, float u2, float u3) {
    float2 b0 = cu.d[0], b1 = cu.d[1], b2 = cu.d[2], b3 = cu.d[3];
    b0 = add2(mul2(b0, 1.0f - u1), mul2(b1, u1));
    b1 = add2(mul2(b1, 1.0f - u1), mul2(b2, u1));
    b2 = add2(mul2(b2, 1.0f - u1), mul2(b3, u1));
    b0 = add2(mul2(b0, 1.0f - u2), mul2(b1, u2));
    b1 = add2(mul2(b1, 1.0f - u2), mul2(b2, u2));
    b0 = add2(mul2(b0, 1.0f - u3), mul2(b1, u3));
    return add2(cu.p[0], b0);
}

// point of the segment at t (the end points exactly)
SE_HD float2 seg_point_at(const Cubic& cu, float t) {
    if (t <= 0.0f) return cu.p[0];
    if (t >= 1.0f) return cu.p[3];
    if (cu.line) return add2(cu.p[0], mul2(cu.d[3], t));
    return blossom(cu, t, t, t);
}

// ---------------------------------------------------------------------------
// dash pattern and the boundary walk
// ---------------------------------------------------------------------------
constexpr uint32_t kDashMaxCuts = 1u << 22;  // boundaries one segment may hold
constexpr float kDashMaxPeriods = 8388608.0f; // 2^23 periods along one subpath

struct DashPattern {
    const float* d;
    uint32_t n;   // entries given
    uint32_t np;  // entries walked: n, or 2n when n is odd
    DF period;
    DF ph0;       // dash offset reduced into [0, period)
    bool valid;   // entries finite and >= 0, period finite and > 0

    SE_HD float at(uint32_t k) const { return d[k % n]; }
};

SE_HD DashPattern make_pattern(const float* dashes, uint32_t first, uint32_t count, float offset, bool& bad) {
    DashPattern p;
    p.d = dashes + first;
    p.n = count;
    p.np = (count & 1u) ? 2u * count : count;
    p.period = df_make(0.0f);
    p.ph0 = df_make(0.0f);
    p.valid = false;
    bool ok = isfinite(offset);
    for (uint32_t k = 0; k < count; k++) {
        float v = p.d[k];
        if (!(v >= 0.0f) || !isfinite(v)) ok = false;
    }
    if (!ok) {
        bad = true;
        return p;
    }
    for (uint32_t k = 0; k < p.np; k++) p.period = df_add(p.period, df_make(p.at(k)));
    if (!(p.period.hi > 0.0f) || !isfinite(p.period.hi)) return p;  // zero period: nothing is drawn
    // offset mod period, in [0, period)
    float q = floorf(offset / p.period.hi);
    DF r = df_sub(df_make(offset), df_mul_f(p.period, q));
    for (int it = 0; it < 4 && df_lt(r, df_make(0.0f)); it++) r = df_add(r, p.period);
    for (int it = 0; it < 4 && df_le(p.period, r); it++) r = df_sub(r, p.period);
    p.ph0 = r;
    p.valid = true;
    return p;
}

// Canonical boundary position m * period + (d_0 + ... + d_{k-1}): callers
// advance (m, k, Bk) only through dash_next so that every caller computes the
// same value for the same boundary.
struct DashCursor {
    float m;     // period index
    uint32_t k;  // pattern index of the interval the boundary starts
    DF Bk;       // d_0 + ... + d_{k-1}
};

SE_HD DF dash_pos(const DashPattern& p, const DashCursor& c) { return df_add(df_mul_f(p.period, c.m), c.Bk); }

SE_HD void dash_next(const DashPattern& p, DashCursor& c) {
    c.Bk = df_add(c.Bk, df_make(p.at(c.k)));
    c.k++;
    if (c.k == p.np) {
        c.k = 0;
        c.m += 1.0f;
        c.Bk = df_make(0.0f);
    }
}

// first boundary at or after z (strictly after when `after`)
SE_HD DashCursor dash_first_at(const DashPattern& p, DF z, bool after) {
    DashCursor c;
    float m = floorf(z.hi / p.period.hi) - 1.0f;
    c.m = m > 0.0f ? m : 0.0f;
    c.k = 0;
    c.Bk = df_make(0.0f);
    for (uint32_t it = 0; it < 3u * p.np + 3u; it++) {
        DF b = dash_pos(p, c);
        if (after ? df_lt(z, b) : df_le(z, b)) break;
        dash_next(p, c);
    }
    return c;
}

// An interval is "on" when its pattern index is even (np is even).
SE_HD bool interval_on(const DashPattern& p, uint32_t k_start_of_next) {
    uint32_t cur = k_start_of_next == 0u ? p.np - 1u : k_start_of_next - 1u;
    return (cur & 1u) == 0u;
}

// Walk the boundaries of a segment covering phase positions [z0, z1) (the
// first segment of a subpath: (z0, z1), a boundary at its start having been
// passed before the walk).  Calls, in order along the segment:
//   sink.cut(s)        a boundary at local arc length s
//   sink.part(sa, sb)  an "on" part [sa, sb] (sb < 0: up to the segment end)
//   sink.end()         the dash ends at the latest cut
//   sink.start(first)  a dash starts at the latest cut (or at the subpath start)
// Returns whether the segment ends inside an "on" interval; `overflow` is set
// when the segment holds more than kDashMaxCuts boundaries.
template <class Sink>
SE_HD bool dash_walk(const DashPattern& p, DF z0, DF z1, bool first, Sink& sink, bool& overflow) {
    DashCursor c = dash_first_at(p, z0, first);
    bool on = interval_on(p, c.k);
    if (first && on) sink.start(true);
    float prev = 0.0f;
    for (uint32_t n = 0;; n++) {
        DF b = dash_pos(p, c);
        if (!df_lt(b, z1)) break;
        if (n >= kDashMaxCuts) {
            overflow = true;
            break;
        }
        float s = df_float(df_sub(b, z0));
        if (s < prev) s = prev;
        sink.cut(s);
        if (on && s > prev) sink.part(prev, s);
        if (on) sink.end();
        on = (c.k & 1u) == 0u;
        if (on) sink.start(false);
        prev = s;
        dash_next(p, c);
    }
    if (on) sink.part(prev, -1.0f);
    return on;
}

// The k-th boundary a segment owns (the one dash_walk meets after k others),
// as the same canonical value dash_walk computes for it.
SE_HD DF dash_kth(const DashPattern& p, DF z0, bool first, uint64_t k) {
    DashCursor c = dash_first_at(p, z0, first);
    uint64_t K = (uint64_t)c.k + k;
    c.m += (float)(K / p.np);
    c.k = (uint32_t)(K % p.np);
    c.Bk = df_make(0.0f);
    for (uint32_t j = 0; j < c.k; j++) c.Bk = df_add(c.Bk, df_make(p.at(j)));
    return dash_pos(p, c);
}

// A sink that only counts the output tags and points.
struct DashCounter {
    uint32_t cc;  // points per part: 1 for a line, 3 for a curve (parts of quadratics are cubics)
    uint64_t tags = 0, pts = 0, cuts = 0;
    SE_HD void cut(float) { cuts++; }
    SE_HD void part(float, float) {
        tags += 1;
        pts += cc;
    }
    SE_HD void end() {
        tags += 1;
        pts += 2;
    }
    SE_HD void start(bool) { pts += 1; }
};

struct DashNull {
    SE_HD void cut(float) {}
    SE_HD void part(float, float) {}
    SE_HD void end() {}
    SE_HD void start(bool) {}
};

// ---------------------------------------------------------------------------
// buffers of the device dash pass (dash.cu)
// ---------------------------------------------------------------------------
struct DashBufs {
    // input stream
    const uint8_t* tags;
    uint64_t n_tags;
    const uint32_t* words;  // path data stream of the input (32- or 16-bit points per tag)
    uint64_t n_words;
    const se_style* styles;
    uint32_t n_styles;
    uint32_t n_paths;
    const float* dashes;
    uint32_t n_dashes;
    TagInfo info;         // tag scan of the input
    float* len;           // per tag: arc length of a dashed segment (0 otherwise)
    long long* end_pos;   // per tag: arc length from its subpath start to the tag's end (units of 2^-32)
    uint2* cnt;           // per tag: output (tags, points)
    ulonglong2* off;      // per tag + 1: exclusive scan of cnt
    uint32_t* nonempty;   // per path: 1 when it has output
    uint8_t* out_tags;
    uint64_t cap_tags;
    float2* out_pts;
    uint64_t cap_pts;
    se_style* out_styles;
    uint64_t* out_n;      // [0] tags, [1] points (0, 0 when over capacity); [2], [3] the totals needed;
                          // [4] cuts of dashed cubics needed
    uint32_t* ncut;       // per tag: boundaries inside a dashed cubic (their parameters are solved in parallel)
    ulonglong2* cut_off;  // per tag + 1: exclusive scan of (ncut, ncut > 0): first cut, panel slot
    PanelPair* panels;    // per cubic with cuts: kPanelMax recorded pairs
    uint32_t* n_panels;   // per cubic with cuts: pairs recorded (kPanelMax + 1: too many)
    uint64_t cap_slots;
    float* cut_t;         // per cut: its parameter on the source cubic
    uint64_t cap_cuts;
    uint32_t* status;
};

// What a tag is, for the dash pass.
struct DashTag {
    uint8_t tag;
    uint32_t cc;
    bool end, seg, curve, dashed, ok;  // curve: a quadratic or cubic segment (its parts are cubics)
    uint32_t base;
    DashPattern pat;
};

SE_HD DashTag classify(const DashBufs& b, uint64_t i, uint32_t& flags) {
    DashTag d;
    d.tag = b.tags[i];
    d.cc = d.tag & SE_TAG_COUNT_MASK;
    d.end = (d.tag & SE_TAG_SUBPATH_END) != 0u;
    d.seg = !d.end && d.cc != 0u;
    d.curve = d.seg && d.cc != 1u;
    d.base = b.info.pt_base[i];
    d.dashed = false;
    d.ok = true;
    // the tag's points 0 .. cc (its first is the previous tag's last, or its subpath's
    // start); a marker's two data points follow its first
    const uint64_t w = tag_wpp(d.tag);
    const uint64_t npt = d.cc + 1u;
    if (d.cc != 0u && (uint64_t)d.base + npt * w > b.n_words) {
        flags |= kStatusBadTag;
        d.ok = false;
        return d;
    }
    uint32_t sid = b.info.style[i];
    if (sid >= b.n_styles) {
        flags |= kStatusBadTag;
        d.ok = false;
        return d;
    }
    const se_style st = b.styles[sid];
    if (st.dash_count == 0u || st.fill) return d;  // fills are not dashed
    d.dashed = true;
    bool bad = false;
    if (!b.dashes || (uint64_t)st.dash_first + st.dash_count > b.n_dashes) bad = true;
    else d.pat = make_pattern(b.dashes, st.dash_first, st.dash_count, st.dash_offset, bad);
    if (bad) {
        flags |= kStatusBadTag;
        d.pat.valid = false;
    }
    return d;
}

// phase positions of a dashed segment; false when the subpath is too long for the pattern
SE_HD bool seg_span(const DashBufs& b, const DashPattern& p, uint64_t i, DF& z0, DF& z1, bool& first) {
    first = b.info.sub_first[i] == (uint32_t)i;
    long long q0 = first ? 0ll : b.end_pos[i - 1], q1 = b.end_pos[i];
    if (q1 >= kFixMax || q0 < 0) return false;
    z0 = df_add(p.ph0, df_of_fix(q0));
    z1 = df_add(p.ph0, df_of_fix(q1));
    return z1.hi / p.period.hi <= kDashMaxPeriods;
}

// Writes the output of one dashed segment as the boundary walk visits it.
struct DashWriter {
    const float* cut_t;   // this segment's cut parameters (cubics), in order
    uint32_t n_cut;
    const Cubic* cu;
    ArcWalk* walk;
    bool walk_ready;
    float len;
    uint8_t* tags;
    float2* pts;
    uint64_t T, Q, T_end, Q_end;
    float t_before, t_cur;
    float2 p_cur;
    bool overrun;

    SE_HD void put_tag(uint8_t t) {
        if (T < T_end) tags[T] = t;
        else overrun = true;
        T++;
    }
    SE_HD void put_pt(float2 p) {
        if (Q < Q_end) pts[Q] = p;
        else overrun = true;
        Q++;
    }
    SE_HD void cut(float s) {
        t_before = t_cur;
        float t;
        if (cu->line) {
            t = len > 0.0f ? s / len : 0.0f;
        } else if (cut_t) {
            t = n_cut ? *cut_t : 1.0f;  // solved by the cut pass
            if (n_cut) {
                cut_t++;
                n_cut--;
            }
        } else {
            if (!walk_ready) {
                walk->init(*cu);
                walk_ready = true;
            }
            t = walk->t_at(s);
        }
        t = fminf(fmaxf(t, t_before), 1.0f);
        t_cur = t;
        p_cur = seg_point_at(*cu, t);
    }
    SE_HD void part(float, float sb) {
        float ta = sb < 0.0f ? t_cur : t_before;
        float tb = sb < 0.0f ? 1.0f : t_cur;
        if (cu->line) {
            put_tag((uint8_t)(1u | SE_TAG_F32));
            put_pt(seg_point_at(*cu, tb));
        } else {
            put_tag((uint8_t)(3u | SE_TAG_F32));
            if (ta <= 0.0f && tb >= 1.0f) {
                put_pt(cu->p[1]);
                put_pt(cu->p[2]);
                put_pt(cu->p[3]);
            } else {
                put_pt(blossom(*cu, ta, ta, tb));
                put_pt(blossom(*cu, ta, tb, tb));
                put_pt(seg_point_at(*cu, tb));
            }
        }
    }
    SE_HD void end() {
        put_tag((uint8_t)(2u | SE_TAG_SUBPATH_END | SE_TAG_F32));
        put_pt(p_cur);
        put_pt(p_cur);
    }
    SE_HD void start(bool) { put_pt(p_cur); }
};

// Output (tags, points) of input tag i, before the empty tag of an empty path.
SE_HD void dash_tag_count(const DashBufs& b, uint64_t i, uint64_t& nt, uint64_t& np, uint64_t& nc,
                          uint32_t& flags) {
    DashTag d = classify(b, i, flags);
    nt = 0;
    np = 0;
    nc = 0;
    if (!d.ok) {
    } else if (!d.dashed) {
        if (d.cc != 0u) {
            nt = 1;
            np = d.cc + (d.end ? 1u : 0u);
        }
    } else if (d.pat.valid && d.seg) {
        DF z0, z1;
        bool first, overflow = false;
        if (!seg_span(b, d.pat, i, z0, z1, first)) {
            flags |= kStatusBadTag;
        } else {
            DashCounter c;
            c.cc = d.curve ? 3u : 1u;
            dash_walk(d.pat, z0, z1, first, c, overflow);
            if (overflow) flags |= kStatusBadTag;
            nt = c.tags;
            np = c.pts;
            nc = d.curve ? c.cuts : 0u;
        }
    } else if (d.pat.valid && d.end && b.info.sub_first[i] != (uint32_t)i) {
        // the marker closes the last dash when the subpath ends inside one
        DF z0, z1;
        bool first, overflow = false;
        if (seg_span(b, d.pat, i - 1, z0, z1, first)) {
            DashNull nul;
            if (dash_walk(d.pat, z0, z1, first, nul, overflow)) {
                nt = 1;
                np = 2;
            }
        }
    }
    if (nt > 0xffffffffull || np > 0xffffffffull || nc > 0xffffffffull) {
        flags |= kStatusBadTag;
        nt = np = nc = 0;
    }
}

// Writes the output of input tag i at its offsets o (and ends before o1).
SE_HD void dash_tag_write(const DashBufs& b, uint64_t i, ulonglong2 o, ulonglong2 o1, uint32_t& flags) {
    DashTag d = classify(b, i, flags);
    uint64_t T = o.x, Q = o.y;
    if (!d.ok) {
    } else if (!d.dashed) {
        if (d.cc != 0u && T < o1.x) {
            // the rewritten stream is 32-bit; the points are written in stream order
            // (each tag from its first point up to, not including, its last, and a
            // marker its first point and two data points)
            b.out_tags[T++] = (uint8_t)((d.tag & ~(SE_TAG_PATH | SE_TAG_STYLE | SE_TAG_TRANSFORM)) | SE_TAG_F32);
            uint32_t inc = d.cc + (d.end ? 1u : 0u);
            for (uint32_t k = 0; k < inc && Q < o1.y; k++) b.out_pts[Q++] = load_pt(b.words, d.base, k, d.tag);
        }
    } else if (d.pat.valid && d.seg) {
        DF z0, z1;
        bool first, overflow = false;
        if (seg_span(b, d.pat, i, z0, z1, first)) {
            Cubic cu = load_seg(b.words, d.tag, d.base);
            ArcWalk walk;
            DashWriter w;
            w.cut_t = b.cut_t ? b.cut_t + b.cut_off[i].x : nullptr;
            w.n_cut = b.cut_t ? (uint32_t)(b.cut_off[i + 1].x - b.cut_off[i].x) : 0u;
            w.cu = &cu;
            w.walk = &walk;
            w.walk_ready = false;
            w.len = b.len[i];
            w.tags = b.out_tags;
            w.pts = b.out_pts;
            w.T = T;
            w.Q = Q;
            w.T_end = o1.x;
            w.Q_end = o1.y;
            w.t_before = 0.0f;
            w.t_cur = 0.0f;
            w.p_cur = cu.p[0];
            w.overrun = false;
            dash_walk(d.pat, z0, z1, first, w, overflow);
            if (w.overrun) flags |= kStatusBadTag;
            T = w.T < o1.x ? w.T : o1.x;
        }
    } else if (d.pat.valid && d.end && b.info.sub_first[i] != (uint32_t)i) {
        DF z0, z1;
        bool first, overflow = false;
        if (seg_span(b, d.pat, i - 1, z0, z1, first)) {
            DashNull nul;
            if (dash_walk(d.pat, z0, z1, first, nul, overflow) && T < o1.x && Q + 2 <= o1.y) {
                float2 e = load_pt(b.words, d.base, 0u, d.tag);  // end point of the subpath's last segment
                b.out_tags[T++] = (uint8_t)(2u | SE_TAG_SUBPATH_END | SE_TAG_F32);
                b.out_pts[Q++] = e;
                b.out_pts[Q++] = e;
            }
        }
    }
    // a path without output keeps one empty tag (its path id stays in the stream)
    if (T < o1.x && (b.tags[i] & SE_TAG_PATH)) b.out_tags[T] = (uint8_t)SE_TAG_F32;
}

cudaError_t launch_dash(const DashBufs& b, ScanState tag_state, ScanState seg_state, ScanState out_state,
                        ScanState cut_state, cudaStream_t s);

}  // namespace se
