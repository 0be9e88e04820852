// Load-balanced stroke expansion (Levien & Uguray, Algorithms 1 and 2),
// restated as four data-parallel phases:
//
//   plan    one thread per tag: the cubic -> Euler-spiral subdivision of
//           Algorithm 2, recording each accept/reject decision as one bit,
//           plus the tag's join / cap record (Algorithm 1);
//   decode  one thread per tag: replays the recorded decisions into one
//           compact reference (t0_u, depth) per accepted piece;
//   piece   one thread per piece: Euler-spiral setup (Appendix A) and, per
//           side, the parallel-curve / evolute ranges and their primitive
//           counts (Sections 4-7);
//   emit    one lane per output primitive, consecutive lanes writing
//           consecutive primitives, each evaluating its own vertices.
//
// Every routine is __host__ __device__ (SE_HD) so the same source can be
// stepped on the CPU.  The library is built with -fmad=false: a value that two
// threads compute independently (a vertex shared by two primitives, a piece
// end point shared by two pieces) is the same function of the same inputs and
// therefore bit-identical.
#pragma once

#include <cstring>

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

// Affine transform of a point (Section 8.2): x' = a x + c y + e, y' = b x + d y + f.
// Every point goes through this one expression, so a point shared by two
// segments maps to the same value in both.
SE_HD float2 xf_point(const float* m, float2 p) {
    return f2((m[0] * p.x + m[2] * p.y) + m[4], (m[1] * p.x + m[3] * p.y) + m[5]);
}

// the half-width scale of a transform: sqrt|det| of its linear part (exact for a
// similarity; an isotropic pen otherwise)
SE_HD float xf_scale(const float* m) { return m ? sqrtf(fabsf(m[0] * m[3] - m[1] * m[2])) : 1.0f; }

// Point k of a tag whose points start at word `base` (Table 1 bit 3): two words
// (float x, float y) for a 32-bit tag, one (int16 x low, int16 y high) for a
// 16-bit tag.  A 32-bit point at an even word is one 8-byte load.
SE_HD uint32_t tag_wpp(uint8_t tag) { return (tag & SE_TAG_F32) ? 2u : 1u; }

SE_HD float bits_float(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(v);
#else
    float f;
    std::memcpy(&f, &v, 4);
    return f;
#endif
}

SE_HD float2 load_pt(const uint32_t* w, uint32_t base, uint32_t k, uint8_t tag) {
    if (tag & SE_TAG_F32) {
        const uint32_t i = base + 2u * k;
        if ((i & 1u) == 0u) return reinterpret_cast<const float2*>(w)[i >> 1];
        return f2(bits_float(w[i]), bits_float(w[i + 1]));
    }
    const uint32_t v = w[base + k];
    return f2((float)(int16_t)(uint16_t)(v & 0xffffu), (float)(int16_t)(uint16_t)(v >> 16));
}

// A segment's control points (transformed by m when m is not NULL), as a cubic:
// lines and quadratics are degree-elevated (Section 8.1); a quadratic's cubic
// control points are P0 + 2/3 (Q1 - P0) and P2 + 2/3 (Q1 - P2).
// the tag's points 0 .. n-1 with one width test (32-bit points at an even word
// are 8-byte loads)
SE_HD void load_pts(const uint32_t* w, uint32_t base, uint32_t n, uint8_t tag, float2* out) {
    if (tag & SE_TAG_F32) {
        if ((base & 1u) == 0u) {
            const float2* p2 = reinterpret_cast<const float2*>(w) + (base >> 1);
            for (uint32_t k = 0; k < n; k++) out[k] = p2[k];
        } else {
            for (uint32_t k = 0; k < n; k++) out[k] = f2(bits_float(w[base + 2 * k]), bits_float(w[base + 2 * k + 1]));
        }
    } else {
        for (uint32_t k = 0; k < n; k++) {
            const uint32_t v = w[base + k];
            out[k] = f2((float)(int16_t)(uint16_t)(v & 0xffffu), (float)(int16_t)(uint16_t)(v >> 16));
        }
    }
}

SE_HD Cubic load_seg(const uint32_t* w, uint8_t tag, uint32_t base, const float* m = nullptr) {
    Cubic cu;
    const uint32_t cc = tag & SE_TAG_COUNT_MASK;
    float2 q[4];
    load_pts(w, base, cc == 1u ? 2u : (cc == 2u && !(tag & SE_TAG_SUBPATH_END)) ? 3u : 4u, tag, q);
    if (cc == 1u) {
        cu.line = true;
        cu.p[0] = q[0];
        cu.p[3] = q[1];
        if (m) {
            cu.p[0] = xf_point(m, cu.p[0]);
            cu.p[3] = xf_point(m, cu.p[3]);
        }
        cu.p[1] = cu.p[0];
        cu.p[2] = cu.p[3];
    } else if (cc == 2u && !(tag & SE_TAG_SUBPATH_END)) {
        cu.line = false;
        float2 p0 = q[0], q1 = q[1], p3 = q[2];
        if (m) {
            p0 = xf_point(m, p0);
            q1 = xf_point(m, q1);
            p3 = xf_point(m, p3);
        }
        cu.p[0] = p0;
        cu.p[3] = p3;
        cu.p[1] = add2(p0, mul2(sub2(q1, p0), 2.0f / 3.0f));
        cu.p[2] = add2(p3, mul2(sub2(q1, p3), 2.0f / 3.0f));
    } else {
        cu.line = false;
        for (uint32_t k = 0; k < 4u; k++) cu.p[k] = q[k];
        if (m)
            for (int k = 0; k < 4; k++) cu.p[k] = xf_point(m, cu.p[k]);
    }
    cubic_local(cu);
    return cu;
}

// a segment tag's control points must lie inside the path data stream
SE_HD bool seg_ok(const ExpandArgs& a, uint8_t tag, uint32_t base) {
    uint32_t cc = tag & SE_TAG_COUNT_MASK;
    return cc != 0u && !(tag & SE_TAG_SUBPATH_END) && (uint64_t)base + (uint64_t)(cc + 1u) * tag_wpp(tag) <= a.n_words;
}

// the transform of tag i (NULL: identity); an index past the stream is left to tag_xform_ok
SE_HD const float* tag_xform(const ExpandArgs& a, uint64_t i) {
    if (!a.info.xform) return nullptr;
    const uint32_t x = a.info.xform[i];
    return x < a.n_xforms ? a.xforms + 6ull * x : nullptr;
}

SE_HD bool tag_xform_ok(const ExpandArgs& a, uint64_t i) {
    if (!a.info.xform) return true;
    const uint32_t x = a.info.xform[i];
    return x == ~0u || x < a.n_xforms;
}

// point and local point (relative to p[0]) at a dyadic parameter
SE_HD void seg_point(const Cubic& cu, float t, float2& p, float2& lp) {
    if (t == 0.0f) {
        p = cu.p[0];
        lp = f2(0.0f, 0.0f);
    } else if (t == 1.0f) {
        p = cu.p[3];
        lp = cu.d[3];
    } else {
        lp = cubic_eval_local(cu, t);
        p = add2(cu.p[0], lp);
    }
}

// derivative sampled at a piece boundary t: the start of the segment samples
// toward the inside (t + dt), every later boundary toward the piece ending there
SE_HD float2 seg_deriv(const Cubic& cu, float t) { return deriv_robust(cu, t); }

// ---------------------------------------------------------------------------
// plan: Algorithm 2 with the two-word stack; decision bits (1 = accept)
// ---------------------------------------------------------------------------
struct PlanOut {
    uint32_t n_pieces;
    uint64_t bits;
    bool overflow;  // more than 64 recorded decisions: decode recomputes the fits
};

// One fit decision of Algorithm 2 (shared by plan and the overflow replay).  It
// takes only values: a segment passed by reference to an out-of-line function
// would have to live in local memory for the whole subdivision loop.
SE_NOINL bool accept_piece(float2 lp0, float2 lp1, float2 q0, float2 q1, float dt, float tol_fit) {
    Fit f = fit_es_t<true>(sub2(lp1, lp0), q0, q1, dt);
    bool ok = f.err <= tol_fit;
    if (ok && f.chord > 0.0f) {
        float k1, cc;
        gh(f.th0 + f.th1, f.th1 - f.th0, k1, cc);
        if (cc < kCMin) ok = false;
    }
    return ok;
}

// a segment whose control points all coincide (in FP32): its chord is zero at
// every depth, so no fit can succeed and Algorithm 2 would halve it down to the
// depth cap; it is one degenerate piece instead
SE_HD bool seg_is_point(const Cubic& cu) {
    return cu.d[1].x == 0.0f && cu.d[1].y == 0.0f && cu.d[2].x == 0.0f && cu.d[2].y == 0.0f && cu.d[3].x == 0.0f &&
           cu.d[3].y == 0.0f;
}

SE_HD PlanOut plan_segment(const Cubic& cu, float tol_fit) {
    PlanOut po;
    po.n_pieces = 0;
    po.bits = 0;
    po.overflow = false;
    if (seg_is_point(cu)) {  // one piece, accepted at depth 0 (decision bit 0 set)
        po.n_pieces = 1;
        po.bits = 1ull;
        return po;
    }
    uint32_t nbits = 0;
    uint32_t t0_u = 0;
    int depth = 0;
    float dt = 1.0f;
    float2 lp0 = f2(0.0f, 0.0f);
    float2 q0 = seg_deriv(cu, 0.0f);
    for (;;) {
        float t0 = (float)t0_u * dt;
        if (t0 >= 1.0f) break;
        float t1 = t0 + dt;
        float2 p1, lp1;
        seg_point(cu, t1, p1, lp1);
        float2 q1 = cu.line ? q0 : seg_deriv(cu, t1);
        bool ok = true;
        if (depth < kMaxDepth) {
            ok = accept_piece(lp0, lp1, q0, q1, dt, tol_fit);
            if (nbits < 64u) {
                if (ok) po.bits |= (1ull << nbits);
            } else {
                po.overflow = true;
            }
            nbits++;
        }
        if (!ok) {
            t0_u *= 2u;
            dt *= 0.5f;
            depth++;
            continue;
        }
        po.n_pieces++;
        t0_u += 1u;
        int shift = ctz32(t0_u);
        t0_u >>= shift;
        dt *= (float)(1u << shift);
        depth -= shift;
        lp0 = lp1;
        q0 = q1;
    }
    return po;
}

// Piece references: t0_u (dyadic start numerator, < 2^17) and depth (<= 16).
SE_HD uint32_t pack_ref(uint32_t t0_u, int depth) { return (t0_u << 5) | (uint32_t)depth; }
SE_HD void unpack_ref(uint32_t r, uint32_t& t0_u, int& depth) {
    t0_u = r >> 5;
    depth = (int)(r & 31u);
}
constexpr uint32_t kTailRef = 0xffffffffu;

// Replay the recorded decisions (or, after an overflow, recompute them) and
// hand each accepted piece's reference to `sink(k, ref)`.
template <class Sink>
SE_HD void decode_segment(const Cubic& cu, const PlanOut& po, float tol_fit, Sink sink) {
    if (seg_is_point(cu)) {
        sink(0u, pack_ref(0u, 0));
        return;
    }
    uint32_t nbits = 0, k = 0;
    uint32_t t0_u = 0;
    int depth = 0;
    float dt = 1.0f;
    float2 lp0 = f2(0.0f, 0.0f);
    float2 q0 = seg_deriv(cu, 0.0f);
    for (;;) {
        float t0 = (float)t0_u * dt;
        if (t0 >= 1.0f) break;
        bool ok = true;
        float t1 = t0 + dt;
        float2 p1, lp1;
        float2 q1 = q0;
        if (po.overflow) {
            seg_point(cu, t1, p1, lp1);
            q1 = cu.line ? q0 : seg_deriv(cu, t1);
        }
        if (depth < kMaxDepth) {
            ok = po.overflow ? accept_piece(lp0, lp1, q0, q1, dt, tol_fit) : ((po.bits >> nbits) & 1ull) != 0;
            nbits++;
        }
        if (!ok) {
            t0_u *= 2u;
            dt *= 0.5f;
            depth++;
            continue;
        }
        sink(k++, pack_ref(t0_u, depth));
        t0_u += 1u;
        int shift = ctz32(t0_u);
        t0_u >>= shift;
        dt *= (float)(1u << shift);
        depth -= shift;
        if (po.overflow) {
            lp0 = lp1;
            q0 = q1;
        }
    }
}

// ---------------------------------------------------------------------------
// piece: ES setup and per-side ranges (Sections 4-7, Algorithm 2 body)
// ---------------------------------------------------------------------------
struct SideRanges {
    float ts;          // parallel-curve cusp parameter (1 = none)
    uint32_t first_normal;  // 1: [normal 0..ts][patch ts..1]; 0: [patch 0..ts][normal ts..1]
    uint32_t n_norm;   // primitives of the normal range (0 if absent)
    uint32_t n_e;      // evolute lines of the patch
    uint32_t n_o;      // reversed parallel-curve primitives of the patch
    uint32_t has_patch;
    LineInv inv_norm, inv_patch;  // vertex placement of the two parallel-curve ranges (line output)
};

SE_HD uint32_t side_total(const SideRanges& r) { return r.n_norm + (r.has_patch ? 2u * (r.n_e + 2u) + r.n_o : 0u); }

struct PieceRec {
    ES es;
    SideRanges side[2];  // [0]: +h, [1]: -h
    float h;             // 0 for a fill
    uint32_t total;
    uint32_t sides;      // 2 for a stroke, 1 for a fill (the source curve itself)
    uint32_t item;       // the piece's item (its primitive offset is item_off[item])
    uint32_t path;       // path id of its tag
};

// A piece's shape as plain values: the range counts take these by value, so the
// piece's ES never has to live in local memory.
struct ESShape {
    float k0, k1, L;
    uint32_t degenerate;
};

SE_HD uint32_t offset_count(ESShape e, float sh, float a, float b, float tol_flat, bool arcs, uint32_t& flags) {
    if (arcs) return count_of(arc_count((b - a) * e.L, e.k1 / (e.L * e.L), fabsf(sh), tol_flat), flags);
    return count_of(line_count(e.k0, e.k1, sh / e.L, a, b, tol_flat / e.L), flags);
}

// Line output: the count of a parallel-curve range (Section 4.1) and the data of
// its vertex placement, from one divided difference of F.  The same expressions
// as line_count and line_inv, so the values are those two would give.  The
// refined mode takes the exact integral instead of its approximation (Section
// 4.2); fills are exact in both.  The placement data goes straight to *li (the
// piece record).  One compiled copy (out of line, everything by value); the
// returned count carries kCountLimit when it was clamped.
constexpr uint32_t kCountLimit = 0x80000000u;

template <bool refine>
static __host__ __device__ __noinline__ uint32_t offset_range_lines(ESShape e, float sh, float a, float b,
                                                                    float tol_flat, LineInv* li) {
    uint32_t flags = 0;
    LineInv v;
    uint32_t n;
    if (sh == 0.0f) {
        // a fill: density sqrt|kappa| (the 2/3-power law of Section 2.2), as the
        // divided difference of g(k) = k |k|^(1/2) over the range's curvatures
        const float ka = e.k0 + e.k1 * (a - 0.5f), kb = e.k0 + e.k1 * (b - 0.5f);
        const float dd = dd_g(ka, kb);
        const float I = (b - a) * (2.0f / 3.0f) * dd;
        n = count_of(fabsf(I) / sqrtf(8.0f * (tol_flat / e.L)), flags);
        v.ua_u = ka;
        v.ua_e = 0.0f;
        v.ub_u = kb;
        v.du = e.k1 * (b - a);
        v.total = dd * v.du;
    } else {
        const float sh_n = sh / e.L;
        UA ua = make_ua(sh_n, e.k0 + e.k1 * (a - 0.5f));
        UA ub = make_ua(sh_n, e.k0 + e.k1 * (b - 0.5f));
        const float dd = refine ? dd_Fx(ua, ub) : dd_F(ua, ub);
        const float I = (b - a) * dd / (2.0f * sqrtf(fabsf(sh_n)));
        n = count_of(fabsf(I) / sqrtf(8.0f * (tol_flat / e.L)), flags);
        v.ua_u = ua.u;
        v.ua_e = ua.e;
        v.ub_u = ub.u;
        v.du = -2.0f * sh_n * e.k1 * (b - a);
        v.total = v.du == 0.0f ? 0.0f : dd * v.du;
    }
    if (n <= 1u) v.ua_u = v.ua_e = v.ub_u = v.du = v.total = 0.0f;
    *li = v;
    return flags ? (n | kCountLimit) : n;
}

// a count from offset_range_lines, its limit bit moved into flags
SE_HD uint32_t take_count(uint32_t c, uint32_t& flags) {
    if (c & kCountLimit) flags |= kStatusLimit;
    return c & ~kCountLimit;
}

// Counts of one side: primitives, chain vertices, status flags.
struct SideCounts {
    uint32_t total, verts, flags;
};

// One side's ranges (the parallel curve, and an evolute patch where the curve
// has a cusp: Sections 4-7), written to *out (the piece record).
template <bool arcs, bool refine>
static __host__ __device__ __noinline__ SideCounts side_ranges(ESShape e, float sh, float tol_flat,
                                                               SideRanges* out) {
    uint32_t flags = 0;
    SideRanges r;
    r.ts = 1.0f;
    r.first_normal = 1;
    r.n_norm = r.n_e = r.n_o = r.has_patch = 0;
    const LineInv zero = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    SideCounts out_c;
    if (e.degenerate) {
        r.n_norm = 1;
        r.inv_norm = r.inv_patch = zero;
        *out = r;
        out_c.total = 1u;
        out_c.verts = 2u;
        out_c.flags = 0u;
        return out_c;
    }
    float sh_n = sh / e.L;
    float x0 = sh_n * (e.k0 + e.k1 * (0.0f - 0.5f)), x1 = sh_n * (e.k0 + e.k1 * (1.0f - 0.5f));
    float w0 = 1.0f + x0, w1 = 1.0f + x1;
    float ts = (w0 * w1 >= 0.0f) ? 1.0f : w0 / (w0 - w1);
    r.ts = ts;
    r.first_normal = w0 >= 0.0f ? 1u : 0u;
    float pa, pb, na, nb;
    bool has_norm;
    if (w0 >= 0.0f) {
        na = 0.0f;
        nb = ts;
        has_norm = true;
        r.has_patch = ts < 1.0f;
        pa = ts;
        pb = 1.0f;
    } else {
        r.has_patch = 1;
        pa = 0.0f;
        pb = ts;
        has_norm = ts < 1.0f;
        na = ts;
        nb = 1.0f;
    }
    // the range placement data is written straight into the record; a range that
    // is absent keeps zero data
    if (!has_norm || arcs) out->inv_norm = zero;
    if (!r.has_patch || arcs) out->inv_patch = zero;
    if (arcs) {
        if (has_norm) r.n_norm = offset_count(e, sh, na, nb, tol_flat, true, flags);
        if (r.has_patch) r.n_o = offset_count(e, sh, pa, pb, tol_flat, true, flags);
    } else {
        if (has_norm) r.n_norm = take_count(offset_range_lines<refine>(e, sh, na, nb, tol_flat, &out->inv_norm), flags);
        if (r.has_patch) r.n_o = take_count(offset_range_lines<refine>(e, sh, pa, pb, tol_flat, &out->inv_patch), flags);
    }
    if (r.has_patch) r.n_e = count_of(evolute_count(e.k0, e.k1, e.L, pa, pb, tol_flat), flags);
    out->ts = r.ts;
    out->first_normal = r.first_normal;
    out->n_norm = r.n_norm;
    out->n_e = r.n_e;
    out->n_o = r.n_o;
    out->has_patch = r.has_patch;
    out_c.total = r.n_norm + (r.has_patch ? 2u * (r.n_e + 2u) + r.n_o : 0u);
    out_c.verts = (r.n_norm ? r.n_norm + 1u : 0u) + (r.has_patch ? (r.n_e + 3u) + (r.n_o + 1u) : 0u);
    out_c.flags = flags;
    return out_c;
}

// Build the piece (t0_u, depth) of segment cu: the same values the sequential
// Algorithm 2 computes for it, written into pr (on the device: the piece record
// staged in shared memory).  In two steps, so that a block can regroup its
// pieces between them: the Euler-spiral fit and shape (build_piece_shape), then
// both sides' ranges and counts (build_piece_sides), which return the piece's
// primitives and write its chain vertices to *verts.
SE_HD void build_piece_shape(const Cubic& cu, uint32_t t0_u, int depth, float h, PieceRec& pr) {
    float dt = 1.0f / (float)(1u << depth);
    float t0 = (float)t0_u * dt, t1 = t0 + dt;
    float2 p0, lp0, p1, lp1;
    seg_point(cu, t0, p0, lp0);
    seg_point(cu, t1, p1, lp1);
    float2 q0 = seg_deriv(cu, t0);
    float2 q1 = cu.line ? q0 : seg_deriv(cu, t1);
    float2 chord = sub2(lp1, lp0);
    Fit f = fit_es_t<false>(chord, q0, q1, dt);
    ES e;
    e.p0 = p0;
    e.p1 = p1;
    e.q0 = q0;
    e.q1 = q1;
    e.th0 = f.th0;
    e.th1 = f.th1;
    e.degenerate = f.chord == 0.0f ? 1u : 0u;
    e.k0 = e.k1 = 0.0f;
    e.L = 0.0f;
    e.rot = f2(0.0f, 0.0f);
    if (!e.degenerate) {
        const ESSetup su = es_setup(f.th0, f.th1, chord, f.chord);
        e.k0 = su.k0;
        e.k1 = su.k1;
        e.L = su.L;
        e.rot = su.rot;
    }
    pr.es = e;
    pr.h = h;
    pr.sides = h == 0.0f ? 1u : 2u;
}

// Which side of the shaped piece will hold an evolute patch (its parallel curve
// has a cusp: |h kappa| > 1 at an end), the costlier work of build_piece_sides,
// done in the call for that side.  Scheduling only: no result depends on it.
// 2: the +h side (and maybe the other) has a patch, 1: only the -h side,
// 0: neither.  On side sh the parallel curve has a cusp where 1 + sh kappa
// changes sign, kappa = kn / L with kn = k0 + k1 (s - 1/2) linear in s: a patch
// on +h needs kn <= -L / h at an end, on -h kn >= L / h.
SE_HD uint32_t piece_patch_class(const PieceRec& pr) {
    const ES& e = pr.es;
    if (e.degenerate || pr.h == 0.0f) return 0u;
    const float kn0 = e.k0 - 0.5f * e.k1, kn1 = e.k0 + 0.5f * e.k1;
    if (fminf(kn0, kn1) * pr.h <= -e.L) return 2u;
    return fmaxf(kn0, kn1) * pr.h >= e.L ? 1u : 0u;
}

template <bool arcs, bool refine>
SE_HD uint32_t build_piece_sides(PieceRec& pr, float tol_flat, uint32_t& flags, uint32_t* verts = nullptr) {
    ESShape shp;
    shp.k0 = pr.es.k0;
    shp.k1 = pr.es.k1;
    shp.L = pr.es.L;
    shp.degenerate = pr.es.degenerate;
    const float h = pr.h;
    SideCounts c0 = side_ranges<arcs, refine>(shp, h, tol_flat, &pr.side[0]);
    SideCounts c1;
    c1.total = c1.verts = c1.flags = 0u;
    if (pr.sides == 2u) {
        c1 = side_ranges<arcs, refine>(shp, -h, tol_flat, &pr.side[1]);
    } else {
        // a fill has one side; the other holds no ranges
        SideRanges z;
        z.ts = 1.0f;
        z.first_normal = 1u;
        z.n_norm = z.n_e = z.n_o = z.has_patch = 0u;
        z.inv_norm = z.inv_patch = LineInv{0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        pr.side[1] = z;
    }
    flags |= c0.flags | c1.flags;
    pr.total = c0.total + c1.total;
    if (verts) *verts = c0.verts + c1.verts;
    return pr.total;
}

template <bool arcs, bool refine>
SE_HD uint32_t build_piece(const Cubic& cu, uint32_t t0_u, int depth, float h, float tol_flat, PieceRec& pr,
                           uint32_t& flags, uint32_t* verts = nullptr) {
    build_piece_shape(cu, t0_u, depth, h, pr);
    return build_piece_sides<arcs, refine>(pr, tol_flat, flags, verts);
}

SE_HD uint32_t side_verts(const ES& e, const SideRanges& r) {
    if (e.degenerate) return 2u;
    return (r.n_norm ? r.n_norm + 1u : 0u) + (r.has_patch ? (r.n_e + 3u) + (r.n_o + 1u) : 0u);
}

SE_HD uint32_t piece_verts(const PieceRec& pr) {
    return side_verts(pr.es, pr.side[0]) + (pr.sides == 2u ? side_verts(pr.es, pr.side[1]) : 0u);
}

// ---------------------------------------------------------------------------
// tails: joins and caps (Algorithm 1, SVG semantics)
// ---------------------------------------------------------------------------
enum : uint32_t { kTailNone = 0, kTailJoin = 1, kTailEndCap = 2, kTailStartCap = 3, kTailDot = 4 };

struct TailRec {
    float2 P, Ti, To;  // joint / cap point; incoming and outgoing tangents
    float2 P0;         // a line segment's start point (when `line`)
    float h, ml;
    uint32_t kind;
    uint32_t style;    // join or cap style
    uint32_t n0, n1;   // primitives on the +h / -h pass (joins), or of the cap (n0)
    float alpha;       // join turn angle
    uint32_t left;     // join turns left
    uint32_t line;     // 1: the tag is a line whose two offsets lead the item (no piece item)
};

// A line segment's whole expansion is one Euler-spiral piece of zero curvature
// whose two parallel curves are one primitive each, between the offsets of its
// end points (Section 8.1: lines are degree-elevated cubics).  Its tail item
// emits those two primitives ahead of the join or cap, so a line needs no
// piece item at all.
constexpr uint32_t kLinePrims = 2u, kLineVerts = 4u;

SE_HD uint32_t tail_total(const TailRec& t) { return t.n0 + t.n1 + (t.line ? kLinePrims : 0u); }

SE_HD uint32_t tail_verts(const TailRec& t) {
    const uint32_t lead = t.line ? kLineVerts : 0u;
    if (t.kind == kTailNone) return lead;
    if (t.kind == kTailEndCap || t.kind == kTailStartCap) return lead + t.n0 + 1u;
    return lead + t.n0 + t.n1 + 2u;
}

SE_HD uint32_t cap_count(uint32_t cap, float h, float tol_flat, bool arcs, uint32_t& flags) {
    if (cap == SE_CAP_BUTT) return 1;
    if (cap == SE_CAP_SQUARE) return 3;
    if (arcs) return 1;
    return count_of(round_N(kPi, h, tol_flat), flags);
}

SE_HD void make_join(TailRec& t, float tol_flat, bool arcs, uint32_t& flags) {
    float cr = cross2(t.Ti, t.To), dp = dot2(t.Ti, t.To);
    t.left = cr >= 0.0f ? 1u : 0u;
    t.alpha = acc_atan2(fabsf(cr), dp);
    uint32_t outer;
    if (t.style == SE_JOIN_MITER) {
        float cosa = dp / (len2(t.Ti) * len2(t.To));
        float q = (1.0f + cosa) * t.ml * t.ml * 0.5f;
        outer = q >= 1.0f ? 2u : 1u;
    } else if (t.style == SE_JOIN_ROUND) {
        outer = arcs ? 1u : count_of(round_N(t.alpha, t.h, tol_flat), flags);
    } else {
        outer = 1u;
    }
    // the outer contour is on the +h side for a left turn
    t.n0 = t.left ? outer : 2u;
    t.n1 = t.left ? 2u : outer;
}

// ---------------------------------------------------------------------------
// emission as chains: every item is a short list of polylines ("chains");
// chain c has n primitives and n + 1 vertices, primitive i joining vertex i
// to vertex i + 1 (flipped chains -- the -h side -- store it as i + 1 -> i).
// The emit pass gives each vertex one lane, which writes it into the
// primitives that share it, so no vertex is evaluated twice.
// ---------------------------------------------------------------------------
enum : uint32_t {
    kChOffset = 0,      // parallel curve over [a, b], vertices in parameter order
    kChOffsetRev = 1,   // parallel curve over [a, b], vertices in reverse order
    kChEvolute = 2,     // offset(a) -> evolute(a .. b) -> offset(b); emitted twice
    kChDegen = 3,       // one primitive between the offsets of a zero-chord piece
    kChPoly = 4,        // join / cap contour: explicit vertices (see tail_vertex)
    kChLine = 5,        // a line segment's parallel curve: one primitive between its end offsets
};

struct Chain {
    uint32_t type;
    uint32_t n;        // primitives (n + 1 vertices); kChEvolute: n = n_e + 2 per copy
    uint32_t p_off;    // first primitive, relative to the item
    uint32_t v_off;    // first vertex, relative to the item
    float a, b;        // parameter range (offset / evolute chains)
    float sh;          // signed offset (offset chains), or the cap/join side
    uint32_t flip;
    uint32_t aux;      // kChEvolute: n_e; kChPoly: sub-kind
    const LineInv* inv;  // offset chains in line output: the range's vertex placement
};

constexpr int kMaxChains = 6;

struct ChainList {
    Chain c[kMaxChains];
    int n;
    uint32_t prims, verts;
};

SE_HD void chain_push(ChainList& L, uint32_t type, uint32_t n, float a, float b, float sh, uint32_t flip,
                      uint32_t aux, uint32_t copies) {
    Chain& c = L.c[L.n++];
    c.type = type;
    c.n = n;
    c.p_off = L.prims;
    c.v_off = L.verts;
    c.a = a;
    c.b = b;
    c.sh = sh;
    c.flip = flip;
    c.aux = aux;
    c.inv = nullptr;
    L.prims += n * copies;
    L.verts += n + 1u;
}

SE_HD void side_chains(ChainList& L, const ES& e, const SideRanges& r, float sh) {
    uint32_t flip = sh < 0.0f ? 1u : 0u;
    if (e.degenerate) {
        chain_push(L, kChDegen, 1u, 0.0f, 1.0f, sh, flip, 0u, 1u);
        return;
    }
    float na = r.first_normal ? 0.0f : r.ts, nb = r.first_normal ? r.ts : 1.0f;
    float pa = r.first_normal ? r.ts : 0.0f, pb = r.first_normal ? 1.0f : r.ts;
    if (r.first_normal && r.n_norm) chain_push(L, kChOffset, r.n_norm, na, nb, sh, flip, 0u, 1u);
    if (r.has_patch) {
        chain_push(L, kChEvolute, r.n_e + 2u, pa, pb, sh, flip, r.n_e, 2u);
        chain_push(L, kChOffsetRev, r.n_o, pa, pb, sh, flip, 0u, 1u);
    }
    if (!r.first_normal && r.n_norm) chain_push(L, kChOffset, r.n_norm, na, nb, sh, flip, 0u, 1u);
}

// The chain holding vertex `local` of an item, found by walking the chain
// counts (no chain array is materialised).
struct ChainFinder {
    uint32_t local, prims, verts;
    bool found;
    Chain out;
    const LineInv* inv;
    SE_HD void push(uint32_t type, uint32_t n, float a, float b, float sh, uint32_t flip, uint32_t aux,
                    uint32_t copies) {
        if (found) return;
        if (local < verts + n + 1u) {
            out.inv = inv;
            out.type = type;
            out.n = n;
            out.p_off = prims;
            out.v_off = verts;
            out.a = a;
            out.b = b;
            out.sh = sh;
            out.flip = flip;
            out.aux = aux;
            found = true;
        }
        prims += n * copies;
        verts += n + 1u;
    }
};

template <class Sink>
SE_HD void side_walk(Sink& L, const ES& e, const SideRanges& r, float sh) {
    uint32_t flip = sh < 0.0f ? 1u : 0u;
    if (e.degenerate) {
        L.push(kChDegen, 1u, 0.0f, 1.0f, sh, flip, 0u, 1u);
        return;
    }
    float na = r.first_normal ? 0.0f : r.ts, nb = r.first_normal ? r.ts : 1.0f;
    float pa = r.first_normal ? r.ts : 0.0f, pb = r.first_normal ? 1.0f : r.ts;
    L.inv = &r.inv_norm;
    if (r.first_normal && r.n_norm) L.push(kChOffset, r.n_norm, na, nb, sh, flip, 0u, 1u);
    if (r.has_patch) {
        L.inv = nullptr;
        L.push(kChEvolute, r.n_e + 2u, pa, pb, sh, flip, r.n_e, 2u);
        L.inv = &r.inv_patch;
        L.push(kChOffsetRev, r.n_o, pa, pb, sh, flip, 0u, 1u);
    }
    L.inv = &r.inv_norm;
    if (!r.first_normal && r.n_norm) L.push(kChOffset, r.n_norm, na, nb, sh, flip, 0u, 1u);
}

// A piece whose two sides are one parallel-curve range each (no evolute patch,
// not degenerate): the common case, whose chains need no walk.
SE_HD bool piece_is_simple(const PieceRec& pr) {
    return pr.sides == 2u && !pr.es.degenerate && !pr.side[0].has_patch && !pr.side[1].has_patch;
}

// Chain `side` (0: +h, 1: -h) of a simple piece; `interior` selects how v_off
// counts (interior vertices only, or all vertices).
SE_HD void simple_chain(const PieceRec& pr, uint32_t side, bool interior, Chain& c) {
    const uint32_t n0 = pr.side[0].n_norm;
    c.type = kChOffset;
    c.n = pr.side[side].n_norm;
    c.p_off = side ? n0 : 0u;
    c.v_off = side ? (interior ? n0 - 1u : n0 + 1u) : 0u;
    c.a = 0.0f;
    c.b = pr.side[side].ts;
    c.sh = side ? -pr.h : pr.h;
    c.flip = side;
    c.aux = 0u;
    c.inv = &pr.side[side].inv_norm;
}

SE_HD bool piece_find_chain(const PieceRec& pr, uint32_t local, Chain& c) {
    ChainFinder f;
    f.local = local;
    f.prims = f.verts = 0;
    f.found = false;
    f.inv = nullptr;
    side_walk(f, pr.es, pr.side[0], pr.h);
    if (pr.sides == 2u) side_walk(f, pr.es, pr.side[1], -pr.h);
    c = f.out;
    return f.found;
}

// The chain holding vertex `local` of any piece, computed from the sides'
// counts in the order side_walk pushes them (one side: [normal][evolute,
// reversed offset] or [evolute, reversed offset][normal]; a degenerate side is
// one kDegen chain) with selects instead of a walk: the same Chain
// piece_find_chain returns.  `local` must be below piece_verts(pr).
SE_HD void piece_chain_at(const PieceRec& pr, uint32_t local, Chain& c) {
    const uint32_t v0 = side_verts(pr.es, pr.side[0]);
    const uint32_t side = local >= v0 ? 1u : 0u;
    const SideRanges& r = pr.side[side];
    const uint32_t l = side ? local - v0 : local;
    const uint32_t v_base = side ? v0 : 0u;
    const uint32_t p_base = side ? side_total(pr.side[0]) : 0u;
    c.sh = side ? -pr.h : pr.h;
    c.flip = c.sh < 0.0f ? 1u : 0u;
    if (pr.es.degenerate) {
        c.type = kChDegen;
        c.n = 1u;
        c.p_off = p_base;
        c.v_off = v_base;
        c.a = 0.0f;
        c.b = 1.0f;
        c.aux = 0u;
        c.inv = nullptr;
        return;
    }
    const bool fn = r.first_normal != 0u;
    const bool patch = r.has_patch != 0u;
    const uint32_t vN = r.n_norm ? r.n_norm + 1u : 0u;
    const uint32_t vE = patch ? r.n_e + 3u : 0u, vO = patch ? r.n_o + 1u : 0u;
    const uint32_t pE = patch ? 2u * (r.n_e + 2u) : 0u, pO = patch ? r.n_o : 0u;
    // 0: normal range, 1: evolute, 2: reversed offset of the patch
    const uint32_t which = fn ? (l < vN ? 0u : (l < vN + vE ? 1u : 2u)) : (l < vE ? 1u : (l < vE + vO ? 2u : 0u));
    const uint32_t e_v = fn ? vN : 0u, e_p = fn ? r.n_norm : 0u;  // the evolute's first vertex / primitive
    const float ts = r.ts;
    if (which == 0u) {
        c.type = kChOffset;
        c.n = r.n_norm;
        c.v_off = fn ? 0u : vE + vO;
        c.p_off = fn ? 0u : pE + pO;
        c.a = fn ? 0.0f : ts;
        c.b = fn ? ts : 1.0f;
        c.aux = 0u;
        c.inv = &r.inv_norm;
    } else {
        c.type = which == 1u ? kChEvolute : kChOffsetRev;
        c.n = which == 1u ? r.n_e + 2u : r.n_o;
        c.v_off = which == 1u ? e_v : e_v + vE;
        c.p_off = which == 1u ? e_p : e_p + pE;
        c.a = fn ? ts : 0.0f;
        c.b = fn ? 1.0f : ts;
        c.aux = which == 1u ? r.n_e : 0u;
        c.inv = which == 1u ? nullptr : &r.inv_patch;
    }
    c.v_off += v_base;
    c.p_off += p_base;
}

// A vertex whose position has a closed form: a chain end at a piece end
// (parameter 0 or 1: the offset of the piece's end point along its end
// tangent's normal) or a degenerate piece's vertex.  The value is the one
// chain_vertex returns for it; every other vertex needs the density inverse
// and the arc-length quadrature.
SE_HD bool end_vertex(const ES& e, uint32_t type, uint32_t n, float a, float b, float sh, uint32_t k, float2& pos) {
    float s;
    if (type == kChDegen) {
        s = k == 0u ? 0.0f : 1.0f;
    } else {
        const uint32_t i = type == kChOffsetRev ? n - k : k;
        if (i != 0u && i != n) return false;
        s = i == 0u ? a : b;
    }
    if (s != 0.0f && s != 1.0f) return false;
    const bool at0 = s == 0.0f;  // one call site: the arithmetic is compiled once
    pos = shared_offset(at0 ? e.p0 : e.p1, at0 ? e.q0 : e.q1, sh);
    return true;
}

SE_HD void piece_chains(const PieceRec& pr, ChainList& L) {
    L.n = 0;
    L.prims = L.verts = 0;
    side_chains(L, pr.es, pr.side[0], pr.h);
    if (pr.sides == 2u) side_chains(L, pr.es, pr.side[1], -pr.h);
}

// Tail sub-kinds (kChPoly aux)
enum : uint32_t { kPolyJoinOuter = 0, kPolyJoinInner = 1, kPolyEndCap = 2, kPolyStartCap = 3 };

template <class Sink>
SE_HD void tail_walk(Sink& L, const TailRec& t) {
    if (t.line) {  // the +h offset, then the -h offset reversed, as a piece item orders them
        L.push(kChLine, 1u, 0.0f, 1.0f, t.h, 0u, 0u, 1u);
        L.push(kChLine, 1u, 0.0f, 1.0f, -t.h, 1u, 0u, 1u);
    }
    if (t.kind == kTailJoin) {
        for (int pass = 0; pass < 2; pass++) {
            uint32_t n = pass == 0 ? t.n0 : t.n1;
            float sh = pass == 0 ? t.h : -t.h;
            bool outer = (pass == 0) == (t.left != 0u);
            L.push(kChPoly, n, 0.0f, 0.0f, sh, pass == 1 ? 1u : 0u, outer ? kPolyJoinOuter : kPolyJoinInner, 1u);
        }
    } else if (t.kind == kTailEndCap) {
        L.push(kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyEndCap, 1u);
    } else if (t.kind == kTailStartCap) {
        L.push(kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyStartCap, 1u);
    } else if (t.kind == kTailDot) {
        L.push(kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyEndCap, 1u);
        L.push(kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyStartCap, 1u);
    }
}

SE_HD bool tail_find_chain(const TailRec& t, uint32_t local, Chain& c) {
    ChainFinder f;
    f.local = local;
    f.prims = f.verts = 0;
    f.found = false;
    f.inv = nullptr;
    tail_walk(f, t);
    c = f.out;
    return f.found;
}

SE_HD void tail_chains(const TailRec& t, ChainList& L) {
    L.n = 0;
    L.prims = L.verts = 0;
    if (t.line) {
        chain_push(L, kChLine, 1u, 0.0f, 1.0f, t.h, 0u, 0u, 1u);
        chain_push(L, kChLine, 1u, 0.0f, 1.0f, -t.h, 1u, 0u, 1u);
    }
    if (t.kind == kTailJoin) {
        for (int pass = 0; pass < 2; pass++) {
            uint32_t n = pass == 0 ? t.n0 : t.n1;
            float sh = pass == 0 ? t.h : -t.h;
            bool outer = (pass == 0) == (t.left != 0u);
            chain_push(L, kChPoly, n, 0.0f, 0.0f, sh, pass == 1 ? 1u : 0u, outer ? kPolyJoinOuter : kPolyJoinInner, 1u);
        }
    } else if (t.kind == kTailEndCap) {
        chain_push(L, kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyEndCap, 1u);
    } else if (t.kind == kTailStartCap) {
        chain_push(L, kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyStartCap, 1u);
    } else if (t.kind == kTailDot) {
        chain_push(L, kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyEndCap, 1u);
        chain_push(L, kChPoly, t.n0, 0.0f, 0.0f, t.h, 0u, kPolyStartCap, 1u);
    }
}

SE_HD float offset_param(const ES& e, float sh, bool arcs, float a, float b, int i, int n) {
    if (arcs) {
        if (i == 0) return a;
        if (i == n) return b;
        return a + (b - a) * ((float)i / (float)n);
    }
    return line_s(e, sh / e.L, a, b, i, n);
}

// parameter of vertex k of an offset chain (the reversed chain visits o_n .. o_0)
template <bool refine = false>
SE_HD float chain_param(const ES& e, const Chain& c, bool arcs, uint32_t k) {
    int i = c.type == kChOffsetRev ? (int)(c.n - k) : (int)k;
    if (!arcs && c.inv && c.sh == 0.0f) return fill_s_v(*c.inv, c.a, c.b, i, (int)c.n);
    if (!arcs && c.inv) return refine ? line_s_refined(*c.inv, c.a, c.b, i, (int)c.n)
                                      : line_s_v(*c.inv, c.a, c.b, i, (int)c.n);
    return offset_param(e, c.sh, arcs, c.a, c.b, i, (int)c.n);
}

// piece_vertex for one output kind (the kernels are instantiated per kind, so
// each carries only its own code).  The chain's fields come by value: a chain
// passed by reference to an out-of-line function would live in local memory.
template <bool kArcs, bool kRefine>
static __host__ __device__ __noinline__ float2 chain_vertex(const ES& e, uint32_t type, uint32_t n, uint32_t aux,
                                                           float a, float b, float sh, const LineInv* inv,
                                                           uint32_t k) {
    if (type == kChDegen) return k == 0u ? shared_offset(e.p0, e.q0, sh) : shared_offset(e.p1, e.q1, sh);
    // The vertex's parameter s, and whether it lies on the evolute (the interior
    // of an evolute chain) rather than on the parallel curve.
    float s;
    bool evo = false;
    if (type == kChEvolute) {
        evo = k != 0u && k != n;
        s = k == 0u ? a : (k == n ? b : evolute_s(e, a, b, (int)k - 1, (int)aux));
    } else {
        // the offset chain's vertex parameter (the reversed chain visits o_n .. o_0).
        // Line output: every parallel-curve chain carries its range's inverse (the
        // piece pass writes one per range), so the emit never recomputes the density
        // integral; arc output places its vertices uniformly in the parameter.
        const int i = type == kChOffsetRev ? (int)(n - k) : (int)k;
        if constexpr (kArcs) {
            s = offset_param(e, sh, true, a, b, i, (int)n);
        } else {
            if (sh == 0.0f) s = fill_s_v(*inv, a, b, i, (int)n);
            else s = kRefine ? line_s_refined(*inv, a, b, i, (int)n) : line_s_v(*inv, a, b, i, (int)n);
        }
    }
    // One evaluation of the spiral's point and tangent serves both kinds (the
    // same expressions as es_offset and es_evolute, so the same values): a warp
    // placing evolute and parallel-curve vertices together integrates once.
    if (!evo && (s == 0.0f || s == 1.0f)) return shared_offset(s == 0.0f ? e.p0 : e.p1, s == 0.0f ? e.q0 : e.q1, sh);
    const float2 T = es_tangent(e, s);
    const float2 P = es_pos(e, s);
    if (evo) {
        float r = vdiv(e.L, es_kn(e, s));  // the radius 1 / kappa, held to the cusp's bound
        if (!(fabsf(r) <= fabsf(sh))) r = -sh;
        return f2(P.x + (-T.y) * r, P.y + T.x * r);
    }
    return f2(P.x + sh * T.y, P.y + sh * (-T.x));
}

template <bool kArcs, bool kRefine>
SE_HD float2 piece_vertex_t(const ES& e, const Chain& c, uint32_t k) {
    return chain_vertex<kArcs, kRefine>(e, c.type, c.n, c.aux, c.a, c.b, c.sh, c.inv, k);
}

SE_NOINL float2 piece_vertex(const ES& e, const Chain& c, bool arcs, uint32_t k) {
    if (c.type == kChDegen) return k == 0u ? shared_offset(e.p0, e.q0, c.sh) : shared_offset(e.p1, e.q1, c.sh);
    if (c.type == kChEvolute) {
        if (k == 0u) return es_offset(e, c.a, c.sh);
        if (k == c.n) return es_offset(e, c.b, c.sh);
        return es_evolute(e, evolute_s(e, c.a, c.b, (int)k - 1, (int)c.aux), c.sh);
    }
    return es_offset(e, chain_param(e, c, arcs, k), c.sh);
}

// vertex i of n of a circular arc about P from A by signed angle ang, ending exactly at B
SE_NOINL float2 round_vertex(float2 P, float2 A, float2 B, float ang, uint32_t i, uint32_t n) {
    if (i == 0u) return A;
    if (i == n) return B;
    return add2(P, rotate(sub2(A, P), ang * ((float)i / (float)n)));
}

// Vertex k of a tail chain (the chain's fields by value: a chain passed by
// reference to an out-of-line function would live in local memory).
//   - a line's parallel curve: the offsets of its end points, the same
//     expression as a piece's end vertices (es_offset at s = 0 and 1), whose
//     point and derivative are the line's end point and P - P0;
//   - a cap contour: end cap from +h to -h bulging along T, start cap from -h to
//     +h bulging against T (a dot's T is +x); square caps extend both offsets by
//     h along the bulge, round caps turn by pi about P;
//   - a join from the incoming side's offset A to the outgoing side's B: the
//     inner contour through P, a miter tip, or a round arc about P.
// Every vertex starts from one offset point, computed at one call site, and
// every arc vertex comes from one rotation call: a warp holding caps, joins and
// lines evaluates each once.
SE_NOINL float2 tail_vertex_f(const TailRec& t, uint32_t type, uint32_t n, uint32_t aux, float sh, bool arcs,
                              uint32_t k) {
    (void)arcs;
    const bool line = type == kChLine;
    const bool cap = !line && (aux == kPolyEndCap || aux == kPolyStartCap);
    const bool start = aux == kPolyStartCap;
    const float2 Tc = (cap && t.kind == kTailDot) ? f2(1.0f, 0.0f) : t.Ti;
    // the offset point the vertex starts from: a cap's last vertex and the second
    // corner of a square cap start from B, its others from A; a join's last
    // vertex from B (the outgoing side), its others from A
    float2 bp = t.P, bq = t.Ti;
    float bsh = sh;
    if (line) {
        bp = k == 0u ? t.P0 : t.P;
    } else if (cap) {
        const bool from_b = k == n || (t.style == SE_CAP_SQUARE && k != 0u && k != 1u);
        bq = Tc;
        bsh = (start != from_b) ? -t.h : t.h;
    } else if (k == n) {
        bq = t.To;
    }
    const float2 O = shared_offset(bp, bq, bsh);
    if (line || k == 0u || k == n) return O;
    float ang;
    if (cap) {
        if (t.style == SE_CAP_SQUARE) {
            float l = len2(Tc);
            float sg = start ? -t.h : t.h;
            float2 E = f2(sg * Tc.x / l, sg * Tc.y / l);
            return add2(O, E);
        }
        ang = kPi;
    } else {
        if (aux == kPolyJoinInner) return t.P;
        if (t.style == SE_JOIN_MITER) {
            float li = len2(t.Ti), lo = len2(t.To);
            float cosa = dot2(t.Ti, t.To) / (li * lo);
            float sc = sh / (1.0f + cosa);
            float2 Ri = f2(t.Ti.y / li, -t.Ti.x / li), Ro = f2(t.To.y / lo, -t.To.x / lo);
            return f2(t.P.x + sc * (Ri.x + Ro.x), t.P.y + sc * (Ri.y + Ro.y));
        }
        ang = (sh > 0.0f ? 1.0f : -1.0f) * t.alpha;
    }
    return round_vertex(t.P, O, O, ang, k, n);  // interior: its end B is not read
}

SE_HD float2 tail_vertex(const TailRec& t, const Chain& c, bool arcs, uint32_t k) {
    return tail_vertex_f(t, c.type, c.n, c.aux, c.sh, arcs, k);
}

// curvature of primitive i of a chain, before any flip (arc output)
SE_HD float tail_prim_curvature(const TailRec& t, const Chain& c, bool arcs) {
    if (!arcs || c.type == kChLine) return 0.0f;
    if (c.aux == kPolyEndCap || c.aux == kPolyStartCap) return t.style == SE_CAP_ROUND ? 1.0f / t.h : 0.0f;
    if (c.aux == kPolyJoinOuter && t.style == SE_JOIN_ROUND) return (c.sh > 0.0f ? 1.0f : -1.0f) / t.h;
    return 0.0f;
}

// ---------------------------------------------------------------------------
// per-tag plan (Algorithm 1): pieces of a segment, and the tag's tail
// ---------------------------------------------------------------------------
SE_HD void plan_tag(const ExpandArgs& a, uint64_t i, PlanOut& po, TailRec& t, uint32_t& flags) {
    po.n_pieces = 0;
    po.bits = 0;
    po.overflow = false;
    t.kind = kTailNone;
    t.n0 = t.n1 = 0;
    t.line = 0;
    t.P = t.Ti = t.To = t.P0 = f2(0.0f, 0.0f);
    t.h = 1.0f;
    t.ml = 1.0f;
    t.style = 0;
    t.alpha = 0.0f;
    t.left = 0;
    uint8_t tag = a.tags[i];
    uint32_t cc = tag & SE_TAG_COUNT_MASK;
    if (cc == 0u) return;
    uint32_t sid = a.info.style[i];
    if (sid >= a.n_styles) {
        flags |= kStatusBadTag;
        return;
    }
    const se_style st = a.styles[sid];
    if (st.dash_count != 0u && !st.fill) {
        flags |= kStatusBadTag;  // dashed styles must be expanded by the dash pass first
        return;
    }
    if (!tag_xform_ok(a, i)) {
        flags |= kStatusBadTag;  // more transform bits than transform entries
        return;
    }
    const float* m = tag_xform(a, i);
    t.h = st.half_width * xf_scale(m);
    t.ml = st.miter_limit;
    uint32_t base = a.info.pt_base[i];
    // every tag of a subpath has its subpath's coordinate width (Table 1 bit 3):
    // each tag after the first matches its predecessor
    if (a.info.sub_first[i] != (uint32_t)i && i > 0 && ((a.tags[i - 1] ^ tag) & SE_TAG_F32)) {
        flags |= kStatusBadTag;
        return;
    }
    if (st.fill) {
        // Algorithm 1, fill branch: the segment itself; no join, cap or marker output
        t.h = 0.0f;
        if (tag & SE_TAG_SUBPATH_END) return;
        if (!seg_ok(a, tag, base)) {
            flags |= kStatusBadTag;
            return;
        }
        Cubic cu = load_seg(a.words, tag, base, m);
        po = plan_segment(cu, a.tol_fit);
        return;
    }
    if (tag & SE_TAG_SUBPATH_END) {
        uint32_t first = a.info.sub_first[i];
        if (first == (uint32_t)i) {
            if (st.cap == SE_CAP_BUTT) return;
            if ((uint64_t)base + tag_wpp(tag) > a.n_words) {
                flags |= kStatusBadTag;
                return;
            }
            t.kind = kTailDot;
            t.style = st.cap;
            const float2 P = load_pt(a.words, base, 0u, tag);
            t.P = m ? xf_point(m, P) : P;
            t.n0 = cap_count(st.cap, t.h, a.tol_flat, a.arcs, flags);
            t.n1 = t.n0;
            return;
        }
        if (tag & SE_TAG_CLOSED) return;
        uint8_t ft = a.tags[first];
        uint32_t fb = a.info.pt_base[first];
        if (first > (uint32_t)i || !seg_ok(a, ft, fb)) {
            flags |= kStatusBadTag;
            return;
        }
        Cubic f = load_seg(a.words, ft, fb, tag_xform(a, first));
        t.kind = kTailStartCap;
        t.style = st.cap;
        t.P = f.p[0];
        t.Ti = seg_deriv(f, 0.0f);
        t.n0 = cap_count(st.cap, t.h, a.tol_flat, a.arcs, flags);
        return;
    }
    if (!seg_ok(a, tag, base) || i + 1 >= tag_count(a)) {
        flags |= kStatusBadTag;
        return;
    }
    Cubic cu = load_seg(a.words, tag, base, m);
    t.P = cu.p[3];
    t.Ti = seg_deriv(cu, 1.0f);
    if (cu.line && len2(cu.d[3]) > 0.0f && t.h != 0.0f) {
        // a line of nonzero chord: one accepted fit, zero curvature, one primitive
        // per side -- emitted by the tail item (see kLinePrims)
        t.line = 1u;
        t.P0 = cu.p[0];
    } else {
        po = plan_segment(cu, a.tol_fit);
    }
    uint8_t nt = a.tags[i + 1];
    if ((nt & SE_TAG_SUBPATH_END) && !(nt & SE_TAG_CLOSED)) {
        t.kind = kTailEndCap;
        t.style = st.cap;
        t.n0 = cap_count(st.cap, t.h, a.tol_flat, a.arcs, flags);
        return;
    }
    Cubic nx;
    if (nt & SE_TAG_SUBPATH_END) {
        uint32_t first = a.info.sub_first[i];
        uint8_t ft = a.tags[first];
        uint32_t fb = a.info.pt_base[first];
        if (first > (uint32_t)i || !seg_ok(a, ft, fb)) {
            flags |= kStatusBadTag;
            return;
        }
        nx = load_seg(a.words, ft, fb, tag_xform(a, first));
    } else {
        if (!seg_ok(a, nt, base + cc * tag_wpp(tag))) {
            flags |= kStatusBadTag;
            return;
        }
        nx = load_seg(a.words, nt, base + cc * tag_wpp(tag), tag_xform(a, i + 1));
    }
    t.kind = kTailJoin;
    t.style = st.join;
    t.To = seg_deriv(nx, 0.0f);
    make_join(t, a.tol_flat, a.arcs, flags);
}

// ---------------------------------------------------------------------------
// workspace of the plan / decode / piece / emit passes
// ---------------------------------------------------------------------------
struct PlanBufs {
    uint32_t* n_items;     // per tag: pieces + 1 (the tail item)
    uint64_t* bits;        // per tag: recorded fit decisions
    uint32_t* overflow;    // per tag: decisions did not fit in 64 bits
    TailRec* tails;        // per tag
    uint64_t* item_base;   // per tag + 1: exclusive scan of n_items
    uint64_t* items_total; // the item total (written by the item scan)
    uint64_t item_cap;     // capacity of the per-item arrays
    uint32_t* item_tag;    // per item: owning tag
    uint32_t* item_ref;    // per item: piece reference or kTailRef
    uint32_t* item_count;  // per item: primitives
    uint32_t* item_vcount; // per item: chain vertices
    uint64_t* item_off;    // per item + 1: exclusive scan of item_count
    PieceRec* pieces;      // per piece (pieces numbered densely: tag i's first piece is item_base[i] - i)
    uint32_t* piece_item;  // per piece: its item
};

cudaError_t launch_tag_scan(const uint8_t* tags, uint64_t n, const uint64_t* n_dev, TagInfo info, ScanState st,
                            uint32_t* status, cudaStream_t s);
cudaError_t launch_plan(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s);
cudaError_t launch_item_scan(const ExpandArgs& a, const PlanBufs& pb, ScanState st, cudaStream_t s);
cudaError_t launch_decode(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s);
cudaError_t launch_piece(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s);
cudaError_t launch_prim_scan(const ExpandArgs& a, const PlanBufs& pb, uint64_t* tag_offset, uint64_t* path_offset,
                             uint32_t n_paths, ScanState st, cudaStream_t s);
cudaError_t launch_emit(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s);
cudaError_t launch_chunk_bounds(const ExpandArgs& a, const PlanBufs& pb, uint32_t k_chunks, uint64_t* out,
                                cudaStream_t s);

}  // namespace se
