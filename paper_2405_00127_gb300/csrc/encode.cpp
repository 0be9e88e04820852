// Host encoder: SVG-style verbs -> tag / point / style streams
// (Levien & Uguray, Section 8.2 and Table 1).
//
// Per drawn subpath the point stream holds the start point, then the new
// points of each segment (1 for a line, 2 for a quadratic, 3 for a cubic),
// then the two data points of the cap marker; consecutive segments share
// their boundary point.  A path's transform, when given, goes to the
// transform stream; the first tag of a path whose transform differs from the
// previous path's starts a new entry (transform bit), as for styles.
// A tag's point increment is its coordinate count plus one when its
// subpath-end bit is set, so an exclusive scan of the increments gives every
// tag the index of its first control point.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/stroke_expand.h"

namespace {

struct Pt {
    float x, y;
};

inline bool same(Pt a, Pt b) { return a.x == b.x && a.y == b.y; }

// cc: 1 line (end point p[3]), 2 quadratic (control point p[1], end p[3]),
// 3 cubic (p[1], p[2], p[3]); p[0] is the current point
struct Seg {
    uint8_t cc;
    Pt p[4];
};

struct Sink {
    // either counts (tags / words) or writes into the caller's arrays
    bool write;
    uint8_t* tags;
    uint32_t* words;
    uint64_t n_tags = 0, n_words = 0;

    void tag(uint8_t t) {
        if (write) tags[n_tags] = t;
        n_tags++;
    }
    // a 32-bit point is two words (the floats' bits); a 16-bit point one word,
    // x in the low half and y in the high half
    void point(Pt p, bool f32) {
        if (f32) {
            if (write && words) {
                std::memcpy(&words[n_words], &p.x, 4);
                std::memcpy(&words[n_words + 1], &p.y, 4);
            }
            n_words += 2;
        } else {
            if (write && words) {
                const uint16_t x = (uint16_t)(int16_t)p.x, y = (uint16_t)(int16_t)p.y;
                words[n_words] = (uint32_t)x | ((uint32_t)y << 16);
            }
            n_words += 1;
        }
    }
};

// a coordinate a 16-bit tag can hold exactly
bool fits16(float v) { return v == std::floor(v) && v >= -32768.0f && v <= 32767.0f; }

struct PathState {
    bool first_tag_of_path = true;
    bool style_bit = false;
    bool xform_bit = false;
    bool f32 = true;  // the path's coordinate width (Table 1 bit 3)
    uint64_t last_tag = 0;  // index of the most recent tag (to set the path bit)
};

// Emit one drawn subpath.  `segs` already excludes zero-length segments and
// includes the closing line of a closed subpath.
void emit_subpath(Sink& s, PathState& ps, Pt start, const std::vector<Seg>& segs, bool closed) {
    auto push_tag = [&](uint8_t t) {
        if (ps.first_tag_of_path) {
            if (ps.style_bit) t |= SE_TAG_STYLE;
            if (ps.xform_bit) t |= SE_TAG_TRANSFORM;
            ps.first_tag_of_path = false;
        }
        ps.last_tag = s.n_tags;
        s.tag(t);
    };
    const uint8_t fbit = ps.f32 ? (uint8_t)SE_TAG_F32 : (uint8_t)0;
    const bool f32 = ps.f32;
    s.point(start, f32);
    for (const Seg& g : segs) {
        if (g.cc == 1) {
            push_tag(uint8_t(1u | fbit));
            s.point(g.p[3], f32);
        } else if (g.cc == 2) {
            push_tag(uint8_t(2u | fbit));
            s.point(g.p[1], f32);
            s.point(g.p[3], f32);
        } else {
            push_tag(uint8_t(3u | fbit));
            s.point(g.p[1], f32);
            s.point(g.p[2], f32);
            s.point(g.p[3], f32);
        }
    }
    // cap marker: coordinate count 2, subpath-end bit; its two data points are
    // the subpath start and the first segment's next control point
    uint8_t t = uint8_t(2u | SE_TAG_SUBPATH_END | fbit);
    if (closed) t |= SE_TAG_CLOSED;
    push_tag(t);
    s.point(start, f32);
    s.point(segs.empty() ? start : segs[0].p[1], f32);
}

bool finite_pt(const float* p) { return std::isfinite(p[0]) && std::isfinite(p[1]); }

// Walk the verbs of every path; `styles` may be NULL when only sizing.
se_status run(const uint8_t* verbs, uint64_t n_verbs, const float* pts, uint64_t n_pts,
              const uint32_t* path_verb_off, uint32_t n_paths, const se_style* styles, const float* xforms,
              const uint8_t* coord16, Sink& s, se_style* styles_out, uint32_t* n_styles_out, float* xforms_out,
              uint32_t* n_xforms_out) {
    if (!verbs && n_verbs) return SE_ERR_INVALID_ARG;
    if (!pts && n_pts) return SE_ERR_INVALID_ARG;
    if (!path_verb_off) return SE_ERR_INVALID_ARG;
    if (path_verb_off[0] != 0 || path_verb_off[n_paths] != n_verbs) return SE_ERR_INVALID_INPUT;
    uint64_t pc = 0;
    uint32_t n_styles = 0, n_xforms = 0;
    const se_style* prev_style = nullptr;
    const float* prev_xform = nullptr;
    std::vector<Seg> segs;
    for (uint32_t p = 0; p < n_paths; p++) {
        if (path_verb_off[p + 1] < path_verb_off[p]) return SE_ERR_INVALID_INPUT;
        PathState ps;
        bool fill = false;
        if (styles) {
            const se_style& st = styles[p];
            fill = st.fill != 0;
            if (!fill) {  // a fill's stroke fields are ignored
                if (!(std::isfinite(st.half_width) && st.half_width > 0.0f)) return SE_ERR_INVALID_INPUT;
                if (!(st.miter_limit >= 1.0f) || !std::isfinite(st.miter_limit)) return SE_ERR_INVALID_INPUT;
                if (st.join > SE_JOIN_ROUND || st.cap > SE_CAP_ROUND) return SE_ERR_INVALID_INPUT;
            }
            bool fresh = !prev_style || std::memcmp(prev_style, &st, sizeof(se_style)) != 0;
            if (fresh) {
                if (styles_out) styles_out[n_styles] = st;
                n_styles++;
                prev_style = &styles[p];
            }
            ps.style_bit = fresh;
        } else {
            ps.style_bit = (p == 0);
        }
        if (xforms) {
            const float* m = xforms + 6 * (uint64_t)p;
            for (int k = 0; k < 6; k++)
                if (!std::isfinite(m[k])) return SE_ERR_INVALID_INPUT;
            bool fresh = !prev_xform || std::memcmp(prev_xform, m, 6 * sizeof(float)) != 0;
            if (fresh) {
                if (xforms_out) std::memcpy(xforms_out + 6 * (uint64_t)n_xforms, m, 6 * sizeof(float));
                n_xforms++;
                prev_xform = m;
            }
            ps.xform_bit = fresh;
        }
        // 16-bit coordinates when asked for and every coordinate of the path fits
        ps.f32 = true;
        if (coord16 && coord16[p]) {
            uint64_t q = pc;
            bool fits = true;
            for (uint32_t vi = path_verb_off[p]; vi < path_verb_off[p + 1] && fits; vi++) {
                const uint8_t vb = verbs[vi];
                const uint64_t np = vb == SE_VERB_CUBIC ? 3 : vb == SE_VERB_QUAD ? 2 : vb == SE_VERB_CLOSE ? 0 : 1;
                for (uint64_t k = 0; k < np && fits; k++, q++)
                    fits = q < n_pts && fits16(pts[2 * q]) && fits16(pts[2 * q + 1]);
            }
            ps.f32 = !fits;
        }
        uint64_t tags_before = s.n_tags;
        bool have = false, drawn = false, closed = false;
        Pt start{0, 0}, cur{0, 0};
        segs.clear();
        auto flush = [&]() {
            if (have && drawn) {
                if (fill) closed = true;  // a filled subpath is closed whether or not it says so
                if (closed && !segs.empty() && !same(cur, start)) {
                    Seg l;
                    l.cc = 1;
                    l.p[0] = cur;
                    l.p[1] = cur;
                    l.p[2] = start;
                    l.p[3] = start;
                    segs.push_back(l);
                }
                emit_subpath(s, ps, start, segs, closed);
            }
            segs.clear();
            drawn = false;
            closed = false;
        };
        for (uint32_t vi = path_verb_off[p]; vi < path_verb_off[p + 1]; vi++) {
            uint8_t vb = verbs[vi];
            if (vb == SE_VERB_MOVE) {
                flush();
                if (pc + 1 > n_pts || !finite_pt(pts + 2 * pc)) return SE_ERR_INVALID_INPUT;
                start = cur = Pt{pts[2 * pc], pts[2 * pc + 1]};
                pc += 1;
                have = true;
            } else if (vb == SE_VERB_LINE || vb == SE_VERB_CUBIC || vb == SE_VERB_QUAD) {
                if (!have) return SE_ERR_INVALID_INPUT;
                if (closed) {  // drawing after closepath starts a new subpath at the start point
                    flush();
                    cur = start;
                }
                Seg g;
                g.p[0] = cur;
                if (vb == SE_VERB_LINE) {
                    if (pc + 1 > n_pts || !finite_pt(pts + 2 * pc)) return SE_ERR_INVALID_INPUT;
                    g.cc = 1;
                    g.p[3] = Pt{pts[2 * pc], pts[2 * pc + 1]};
                    g.p[1] = g.p[0];
                    g.p[2] = g.p[3];
                    pc += 1;
                } else if (vb == SE_VERB_QUAD) {
                    if (pc + 2 > n_pts || !finite_pt(pts + 2 * pc) || !finite_pt(pts + 2 * pc + 2))
                        return SE_ERR_INVALID_INPUT;
                    g.cc = 2;
                    g.p[1] = Pt{pts[2 * pc], pts[2 * pc + 1]};
                    g.p[3] = Pt{pts[2 * pc + 2], pts[2 * pc + 3]};
                    g.p[2] = g.p[3];
                    pc += 2;
                } else {
                    if (pc + 3 > n_pts) return SE_ERR_INVALID_INPUT;
                    for (int k = 0; k < 3; k++) {
                        if (!finite_pt(pts + 2 * (pc + k))) return SE_ERR_INVALID_INPUT;
                        g.p[k + 1] = Pt{pts[2 * (pc + k)], pts[2 * (pc + k) + 1]};
                    }
                    g.cc = 3;
                    pc += 3;
                }
                drawn = true;
                // zero-length segments (every control point at the current point) are dropped
                if (!(same(g.p[1], cur) && same(g.p[2], cur) && same(g.p[3], cur))) segs.push_back(g);
                cur = g.p[3];
            } else if (vb == SE_VERB_CLOSE) {
                if (!have) return SE_ERR_INVALID_INPUT;
                closed = true;
                drawn = true;
            } else {
                return SE_ERR_INVALID_INPUT;
            }
        }
        flush();
        if (s.n_tags == tags_before) {
            // nothing drawn: one empty tag keeps path ids aligned with input paths
            uint8_t t = uint8_t(SE_TAG_F32 | SE_TAG_PATH);
            if (ps.style_bit) t |= SE_TAG_STYLE;
            if (ps.xform_bit) t |= SE_TAG_TRANSFORM;
            s.tag(t);
        } else if (s.write) {
            s.tags[ps.last_tag] |= SE_TAG_PATH;
        }
    }
    if (pc != n_pts) return SE_ERR_INVALID_INPUT;
    if (n_styles_out) *n_styles_out = n_styles;
    if (n_xforms_out) *n_xforms_out = n_xforms;
    return SE_OK;
}

}  // namespace

extern "C" se_status se_encode_size(const uint8_t* verbs, uint64_t n_verbs, const float* pts, uint64_t n_pts,
                                    const uint32_t* path_verb_off, uint32_t n_paths, const se_style* styles,
                                    const uint8_t* coord16, uint64_t* n_tags, uint64_t* n_words) {
    if (!n_tags || !n_words) return SE_ERR_INVALID_ARG;
    Sink s;
    s.write = false;
    s.tags = nullptr;
    s.words = nullptr;
    se_status st = run(verbs, n_verbs, pts, n_pts, path_verb_off, n_paths, styles, nullptr, coord16, s, nullptr,
                       nullptr, nullptr, nullptr);
    if (st != SE_OK) return st;
    *n_tags = s.n_tags;
    *n_words = s.n_words;
    return SE_OK;
}

extern "C" se_status se_encode(const uint8_t* verbs, uint64_t n_verbs, const float* pts, uint64_t n_pts,
                               const uint32_t* path_verb_off, uint32_t n_paths, const se_style* styles_in,
                               const float* transforms_in, const uint8_t* coord16, uint8_t* tags_out,
                               uint32_t* words_out, se_style* styles_out, uint32_t* n_styles_out,
                               float* transforms_out, uint32_t* n_transforms_out) {
    if (!n_styles_out || (n_paths && (!styles_in || !tags_out || !styles_out))) return SE_ERR_INVALID_ARG;
    if (transforms_in && n_paths && !transforms_out) return SE_ERR_INVALID_ARG;
    Sink s;
    s.write = true;
    s.tags = tags_out;
    s.words = words_out;
    if (n_transforms_out) *n_transforms_out = 0;
    return run(verbs, n_verbs, pts, n_pts, path_verb_off, n_paths, styles_in, transforms_in, coord16, s, styles_out,
               n_styles_out, transforms_out, n_transforms_out);
}
