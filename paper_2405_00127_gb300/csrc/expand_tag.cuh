// Per-tag stroke expansion (Algorithms 1 and 2 of Levien & Uguray), shared by
// the count pass (W = false: decisions and counts only) and the write pass
// (W = true: the same decisions, plus the primitives).  Host + device so the
// library's tests can run a tag on the CPU with the identical source.
#pragma once

#include "launch.h"
#include "stroke_math.cuh"

namespace se {

SE_HD int ctz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __ffs((int)x) - 1;
#else
    return __builtin_ctz(x);
#endif
}

// ---------------------------------------------------------------------------
// expansion (Algorithms 1 and 2)
// ---------------------------------------------------------------------------
struct Out {
    float4* prims;
    float* curv;
    uint32_t* pid;
    uint64_t pos;
    uint64_t lim;    // end of this tag's output range (never written past)
    uint32_t path;
    uint32_t overflow;

    SE_HD void put_at(uint64_t at, float2 a, float2 b, float k, bool flip) {
        if (at >= lim) {
            overflow = 1;
            return;
        }
        if (flip) {
            float2 t = a;
            a = b;
            b = t;
            k = -k;
        }
        prims[at] = make_float4(a.x, a.y, b.x, b.y);
        if (curv) curv[at] = k;
        if (pid) pid[at] = path;
    }
    SE_HD void put(float2 a, float2 b, float k, bool flip) { put_at(pos++, a, b, k, flip); }
};

struct Ctx {
    float tol_fit, tol_flat;
    bool arcs;
    uint32_t flags;
};

SE_HD uint32_t offset_n(Ctx& c, const ES& e, float sh, float a, float b) {
    if (c.arcs) return count_of(arc_count((b - a) * e.L, e.k1 / (e.L * e.L), fabsf(sh), c.tol_flat), c.flags);
    return count_of(line_count(e.k0, e.k1, sh / e.L, a, b, c.tol_flat / e.L), c.flags);
}

SE_HD float offset_sample(const ES& e, float sh, bool arcs, float a, float b, int i, int n) {
    if (arcs) {
        if (i == 0) return a;
        if (i == n) return b;
        return a + (b - a) * ((float)i / (float)n);
    }
    return line_s(e, sh / e.L, a, b, i, n);
}

// parallel curve over [a, b] in n primitives, forward or reversed
template <bool W>
SE_HD void offset_range(Ctx& c, const ES& e, float sh, float a, float b, bool reverse,
                                             uint32_t n, Out& o, bool flip) {
    if (!W) return;
    float2 prev = es_offset(e, a, sh);
    float sprev = a;
    for (uint32_t j = 1; j <= n; j++) {
        float s = offset_sample(e, sh, c.arcs, a, b, (int)j, (int)n);
        float2 cur = es_offset(e, s, sh);
        float k = c.arcs ? menger(prev, es_offset(e, 0.5f * (sprev + s), sh), cur) : 0.0f;
        if (!reverse) o.put_at(o.pos + (j - 1), prev, cur, k, flip);
        else o.put_at(o.pos + (n - j), cur, prev, -k, flip);
        prev = cur;
        sprev = s;
    }
    o.pos += n;
}

// Section 6: offset(a) -> evolute(a..b) -> offset(b), twice, then the offset reversed
template <bool W>
SE_HD uint32_t evolute_patch(Ctx& c, const ES& e, float sh, float a, float b, Out& o,
                                                  bool flip) {
    uint32_t n_o = offset_n(c, e, sh, a, b);
    uint32_t n_e = count_of(evolute_count(e.k0, e.k1, e.L, a, b, c.tol_flat), c.flags);
    if (W) {
        float2 oa = es_offset(e, a, sh), ob = es_offset(e, b, sh);
        float2 prev = es_evolute(e, a);
        uint64_t r0 = o.pos, r1 = o.pos + n_e + 2;
        o.put_at(r0, oa, prev, 0.0f, flip);
        o.put_at(r1, oa, prev, 0.0f, flip);
        for (uint32_t j = 1; j <= n_e; j++) {
            float2 cur = es_evolute(e, evolute_s(e, a, b, (int)j, (int)n_e));
            o.put_at(r0 + j, prev, cur, 0.0f, flip);
            o.put_at(r1 + j, prev, cur, 0.0f, flip);
            prev = cur;
        }
        o.put_at(r0 + n_e + 1, prev, ob, 0.0f, flip);
        o.put_at(r1 + n_e + 1, prev, ob, 0.0f, flip);
        o.pos += 2 * (n_e + 2);
        offset_range<W>(c, e, sh, a, b, true, n_o, o, flip);
    }
    return 2 * (n_e + 2) + n_o;
}

template <bool W>
SE_HD uint32_t piece_side(Ctx& c, const ES& e, float sh, Out& o) {
    bool flip = sh < 0.0f;
    if (e.degenerate) {
        if (W) o.put(shared_offset(e.p0, e.q0, sh), shared_offset(e.p1, e.q1, sh), 0.0f, flip);
        return 1;
    }
    float sh_n = sh / e.L;
    float x0 = sh_n * es_kn(e, 0.0f), x1 = sh_n * es_kn(e, 1.0f);
    float w0 = 1.0f + x0, w1 = 1.0f + x1;
    float ts = (w0 * w1 >= 0.0f) ? 1.0f : w0 / (w0 - w1);
    uint32_t cnt = 0;
    if (w0 >= 0.0f) {
        uint32_t n = offset_n(c, e, sh, 0.0f, ts);
        offset_range<W>(c, e, sh, 0.0f, ts, false, n, o, flip);
        cnt += n;
        if (ts < 1.0f) cnt += evolute_patch<W>(c, e, sh, ts, 1.0f, o, flip);
    } else {
        cnt += evolute_patch<W>(c, e, sh, 0.0f, ts, o, flip);
        if (ts < 1.0f) {
            uint32_t n = offset_n(c, e, sh, ts, 1.0f);
            offset_range<W>(c, e, sh, ts, 1.0f, false, n, o, flip);
            cnt += n;
        }
    }
    return cnt;
}

// Algorithm 2: adaptive cubic -> ES subdivision with the (t0_u, dt) stack; each
// accepted piece is emitted on side +h, then side -h.  Returns the count and
// the derivative sampled at t = 1 (the end tangent).
template <bool W>
SE_HD uint32_t stroke_pieces(Ctx& c, const Cubic& cu, float h, Out& o, float2& q_end) {
    uint32_t t0_u = 0;
    float dt = 1.0f;
    int depth = 0;
    float2 p0 = cu.p[0];
    float2 lp0 = f2(0.0f, 0.0f);
    float2 q0 = deriv_robust(cu, 0.0f);
    q_end = q0;
    uint32_t cnt = 0;
    for (;;) {
        float t0 = (float)t0_u * dt;
        if (t0 >= 1.0f) break;
        float t1 = t0 + dt;
        float2 lp1, p1;
        if (t1 == 1.0f) {
            lp1 = cu.d[3];
            p1 = cu.p[3];
        } else {
            lp1 = cubic_eval_local(cu, t1);
            p1 = add2(cu.p[0], lp1);
        }
        float2 q1 = cu.line ? q0 : deriv_robust(cu, t1);
        float2 chord = sub2(lp1, lp0);
        Fit f = fit_es(chord, q0, q1, dt);
        bool ok = f.err <= c.tol_fit;
        if (ok && f.chord > 0.0f) {
            float k1, cc;
            gh(f.th0 + f.th1, f.th1 - f.th0, k1, cc);
            if (cc < kCMin) ok = false;
        }
        if (!ok && depth < kMaxDepth) {
            t0_u *= 2u;
            dt *= 0.5f;
            depth++;
            continue;
        }
        ES e;
        e.p0 = p0;
        e.p1 = p1;
        e.q0 = q0;
        e.q1 = q1;
        e.th0 = f.th0;
        e.th1 = f.th1;
        e.degenerate = (f.chord == 0.0f);
        e.k0 = e.k1 = 0.0f;
        e.L = 0.0f;
        e.rot = f2(0.0f, 0.0f);
        if (!e.degenerate) es_setup(e, chord, f.chord);
        cnt += piece_side<W>(c, e, h, o);
        cnt += piece_side<W>(c, e, -h, o);
        t0_u += 1u;
        int shift = ctz32(t0_u);
        t0_u >>= shift;
        dt *= (float)(1u << shift);
        depth -= shift;
        p0 = p1;
        lp0 = lp1;
        q0 = q1;
        q_end = q1;
    }
    return cnt;
}

// polyline of a circular arc about P from A by signed angle ang in n steps, ending exactly at B
template <bool W>
SE_HD void round_poly(float2 P, float2 A, float2 B, float ang, uint32_t n, Out& o, bool flip) {
    if (!W) return;
    float2 prev = A, ra = sub2(A, P);
    for (uint32_t i = 1; i <= n; i++) {
        float2 cur = (i == n) ? B : add2(P, rotate(ra, ang * ((float)i / (float)n)));
        o.put(prev, cur, 0.0f, flip);
        prev = cur;
    }
}

template <bool W>
SE_HD uint32_t join(Ctx& c, float2 P, float2 Ti, float2 To, float h, int style, float ml,
                                         Out& o) {
    float2 AR = shared_offset(P, Ti, h), BR = shared_offset(P, To, h);
    float2 AL = shared_offset(P, Ti, -h), BL = shared_offset(P, To, -h);
    float cr = cross2(Ti, To), dp = dot2(Ti, To);
    float li = len2(Ti), lo = len2(To);
    bool left = cr >= 0.0f;
    float alpha = atan2f(fabsf(cr), dp);
    int sig_out = left ? 1 : -1;
    uint32_t cnt = 0;
    for (int pass = 0; pass < 2; pass++) {
        int sigma = pass == 0 ? 1 : -1;
        bool flip = sigma < 0;
        float2 A = sigma > 0 ? AR : AL, B = sigma > 0 ? BR : BL;
        if (sigma != sig_out) {
            if (W) {
                o.put(A, P, 0.0f, flip);
                o.put(P, B, 0.0f, flip);
            }
            cnt += 2;
            continue;
        }
        if (style == SE_JOIN_MITER) {
            float cosa = dp / (li * lo);
            float q = (1.0f + cosa) * ml * ml * 0.5f;
            if (q >= 1.0f) {
                if (W) {
                    float sc = (float)sigma * h / (1.0f + cosa);
                    float2 Ri = f2(Ti.y / li, -Ti.x / li), Ro = f2(To.y / lo, -To.x / lo);
                    float2 M = f2(P.x + sc * (Ri.x + Ro.x), P.y + sc * (Ri.y + Ro.y));
                    o.put(A, M, 0.0f, flip);
                    o.put(M, B, 0.0f, flip);
                }
                cnt += 2;
            } else {
                if (W) o.put(A, B, 0.0f, flip);
                cnt += 1;
            }
        } else if (style == SE_JOIN_ROUND) {
            if (c.arcs) {
                if (W) o.put(A, B, (float)sigma / h, flip);
                cnt += 1;
            } else {
                uint32_t n = count_of(round_N(alpha, h, c.tol_flat), c.flags);
                round_poly<W>(P, A, B, (float)sigma * alpha, n, o, flip);
                cnt += n;
            }
        } else {
            if (W) o.put(A, B, 0.0f, flip);
            cnt += 1;
        }
    }
    return cnt;
}

template <bool W>
SE_HD uint32_t end_cap(Ctx& c, float2 P, float2 T, float h, int cap, Out& o) {
    float2 AR = shared_offset(P, T, h), AL = shared_offset(P, T, -h);
    if (cap == SE_CAP_BUTT) {
        if (W) o.put(AR, AL, 0.0f, false);
        return 1;
    }
    if (cap == SE_CAP_SQUARE) {
        if (W) {
            float l = len2(T);
            float2 E = f2(h * T.x / l, h * T.y / l);
            float2 a = add2(AR, E), b = add2(AL, E);
            o.put(AR, a, 0.0f, false);
            o.put(a, b, 0.0f, false);
            o.put(b, AL, 0.0f, false);
        }
        return 3;
    }
    if (c.arcs) {
        if (W) o.put(AR, AL, 1.0f / h, false);
        return 1;
    }
    uint32_t n = count_of(round_N(kPi, h, c.tol_flat), c.flags);
    round_poly<W>(P, AR, AL, kPi, n, o, false);
    return n;
}

template <bool W>
SE_HD uint32_t start_cap(Ctx& c, float2 P, float2 T, float h, int cap, Out& o) {
    float2 BR = shared_offset(P, T, h), BL = shared_offset(P, T, -h);
    if (cap == SE_CAP_BUTT) {
        if (W) o.put(BL, BR, 0.0f, false);
        return 1;
    }
    if (cap == SE_CAP_SQUARE) {
        if (W) {
            float l = len2(T);
            float2 E = f2(-h * T.x / l, -h * T.y / l);
            float2 a = add2(BL, E), b = add2(BR, E);
            o.put(BL, a, 0.0f, false);
            o.put(a, b, 0.0f, false);
            o.put(b, BR, 0.0f, false);
        }
        return 3;
    }
    if (c.arcs) {
        if (W) o.put(BL, BR, 1.0f / h, false);
        return 1;
    }
    uint32_t n = count_of(round_N(kPi, h, c.tol_flat), c.flags);
    round_poly<W>(P, BL, BR, kPi, n, o, false);
    return n;
}

SE_HD Cubic load_seg(const float2* pts, uint8_t tag, uint32_t base) {
    Cubic cu;
    if ((tag & SE_TAG_COUNT_MASK) == 1u) {
        cu.line = true;
        cu.p[0] = pts[base];
        cu.p[3] = pts[base + 1];
        cu.p[1] = cu.p[0];
        cu.p[2] = cu.p[3];
    } else {
        cu.line = false;
        cu.p[0] = pts[base];
        cu.p[1] = pts[base + 1];
        cu.p[2] = pts[base + 2];
        cu.p[3] = pts[base + 3];
    }
    cubic_local(cu);
    return cu;
}

// Algorithm 1 for one tag: a segment emits its pieces and its join or end
// cap; a cap marker emits its subpath's start cap (or the dot of a subpath
// with no segments).
// a segment tag's control points must lie inside the point stream
SE_HD bool seg_ok(const ExpandArgs& a, uint8_t tag, uint32_t base) {
    uint32_t cc = tag & SE_TAG_COUNT_MASK;
    return (cc == 1u || cc == 3u) && !(tag & SE_TAG_SUBPATH_END) && (uint64_t)base + cc < a.n_points;
}

// Algorithm 1 for one tag: a segment emits its pieces and its join or end
// cap; a cap marker emits its subpath's start cap (or the dot of a subpath
// with no segments).  Malformed streams set kStatusBadTag and emit nothing
// further for the tag; every index is checked before it is dereferenced.
template <bool W>
SE_HD uint32_t process_tag(const ExpandArgs& a, uint64_t i, Ctx& c, Out& o) {
    uint8_t tag = a.tags[i];
    uint32_t cc = tag & SE_TAG_COUNT_MASK;
    if (cc == 0u) return 0;
    uint32_t sid = a.info.style[i];
    if (sid >= a.n_styles) {
        c.flags |= kStatusBadTag;
        return 0;
    }
    const se_style st = a.styles[sid];
    float h = st.half_width;
    uint32_t base = a.info.pt_base[i];
    if (tag & SE_TAG_SUBPATH_END) {
        uint32_t first = a.info.sub_first[i];
        if (first == (uint32_t)i) {
            if (st.cap == SE_CAP_BUTT) return 0;
            if ((uint64_t)base >= a.n_points) {
                c.flags |= kStatusBadTag;
                return 0;
            }
            float2 P = a.pts[base];
            uint32_t n = end_cap<W>(c, P, f2(1.0f, 0.0f), h, st.cap, o);
            n += start_cap<W>(c, P, f2(1.0f, 0.0f), h, st.cap, o);
            return n;
        }
        if (tag & SE_TAG_CLOSED) return 0;
        uint8_t ft = a.tags[first];
        uint32_t fb = a.info.pt_base[first];
        if (first > (uint32_t)i || !seg_ok(a, ft, fb)) {
            c.flags |= kStatusBadTag;
            return 0;
        }
        Cubic f = load_seg(a.pts, ft, fb);
        return start_cap<W>(c, f.p[0], deriv_robust(f, 0.0f), h, st.cap, o);
    }
    if (!seg_ok(a, tag, base) || i + 1 >= a.n_tags) {
        c.flags |= kStatusBadTag;
        return 0;
    }
    Cubic cu = load_seg(a.pts, tag, base);
    float2 q_end;
    uint32_t n = stroke_pieces<W>(c, cu, h, o, q_end);
    float2 P = cu.p[3];
    uint8_t nt = a.tags[i + 1];
    if (nt & SE_TAG_SUBPATH_END) {
        if (nt & SE_TAG_CLOSED) {
            uint32_t first = a.info.sub_first[i];
            uint8_t ft = a.tags[first];
            uint32_t fb = a.info.pt_base[first];
            if (first > (uint32_t)i || !seg_ok(a, ft, fb)) {
                c.flags |= kStatusBadTag;
                return n;
            }
            Cubic f = load_seg(a.pts, ft, fb);
            n += join<W>(c, P, q_end, deriv_robust(f, 0.0f), h, st.join, st.miter_limit, o);
        } else {
            n += end_cap<W>(c, P, q_end, h, st.cap, o);
        }
    } else {
        if (!seg_ok(a, nt, base + cc)) {
            c.flags |= kStatusBadTag;
            return n;
        }
        Cubic nx = load_seg(a.pts, nt, base + cc);
        n += join<W>(c, P, q_end, deriv_robust(nx, 0.0f), h, st.join, st.miter_limit, o);
    }
    return n;
}

}  // namespace se
