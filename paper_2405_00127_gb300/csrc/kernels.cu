// Device kernels of the stroke-expansion hot path (Levien & Uguray, arXiv 2405.00127).
//
//   tag_scan      Section 8.2: inclusive scan of the tag monoid over the tag
//                 stream, segmented at subpath ends -> per tag: first control
//                 point, path id, style id, first tag of its subpath.
//   expand<false> Algorithms 1 and 2: per tag, the number of output primitives.
//   count_scan    exclusive scan of the counts -> output offsets, per-path
//                 offsets and the total (replaces the paper's atomic bump
//                 allocation, so the output order is deterministic).
//   expand<true>  the same decisions again, now writing the primitives.
//
// Both scans are single-pass decoupled look-back scans: each block takes a
// ticket, scans its 4096-item tile in registers and shared memory with warp
// shuffles, publishes its aggregate, and walks back over its predecessors'
// published values.  Every wait is bounded; on timeout the block records
// kStatusTimeout and continues, so no launch can hang.
#include <cuda/atomic>

#include "launch.h"
#include "stroke_math.cuh"

namespace se {

// ---------------------------------------------------------------------------
// decoupled look-back scan
// ---------------------------------------------------------------------------
constexpr uint32_t kSpinLimit = 1u << 22;

template <class T, class Op>
__device__ __forceinline__ T warp_incl_scan(T v, Op op) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = Op::shfl_up(v, d);
        if (lane >= d) v = op.combine(o, v);
    }
    return v;
}

template <class Op>
__global__ void __launch_bounds__(kScanThreads) lookback_scan(Op op, uint64_t n, ScanState st, uint32_t* status) {
    using T = typename Op::T;
    __shared__ uint32_t s_tile;
    __shared__ T s_warp[kScanThreads / 32];
    __shared__ T s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(st.ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t base = (uint64_t)tile * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    op.load(base, n, v);
    T acc = op.identity();
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        acc = op.combine(acc, v[k]);
        v[k] = acc;  // thread-local inclusive
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T w = warp_incl_scan(acc, op);
    if (lane == 31) s_warp[warp] = w;
    __syncthreads();
    if (warp == 0) {
        T x = lane < kScanThreads / 32 ? s_warp[lane] : op.identity();
        x = warp_incl_scan(x, op);
        if (lane < kScanThreads / 32) s_warp[lane] = x;  // inclusive over warps
    }
    __syncthreads();
    T warp_excl = warp == 0 ? op.identity() : s_warp[warp - 1];
    T w_excl = Op::shfl_up(w, 1);
    if (lane == 0) w_excl = op.identity();
    T thread_excl = op.combine(warp_excl, w_excl);
    if (threadIdx.x == 0) {
        T tile_agg = s_warp[kScanThreads / 32 - 1];
        T* agg = reinterpret_cast<T*>(st.agg);
        T* incl = reinterpret_cast<T*>(st.incl);
        T ex = op.identity();
        if (tile == 0) {
            incl[0] = tile_agg;
            cuda::atomic_ref<uint32_t, cuda::thread_scope_device> f(st.flags[0]);
            f.store(2u, cuda::memory_order_release);
        } else {
            agg[tile] = tile_agg;
            cuda::atomic_ref<uint32_t, cuda::thread_scope_device> f(st.flags[tile]);
            f.store(1u, cuda::memory_order_release);
            int64_t t = (int64_t)tile - 1;
            while (t >= 0) {
                cuda::atomic_ref<uint32_t, cuda::thread_scope_device> ft(st.flags[t]);
                uint32_t fl = ft.load(cuda::memory_order_acquire);
                uint32_t spins = 0;
                while (fl == 0u && spins < kSpinLimit) {
                    __nanosleep(64);
                    fl = ft.load(cuda::memory_order_acquire);
                    spins++;
                }
                if (fl == 0u) {
                    atomicOr(status, (uint32_t)kStatusTimeout);
                    break;
                }
                if (fl == 2u) {
                    ex = op.combine(incl[t], ex);
                    break;
                }
                ex = op.combine(agg[t], ex);
                t--;
            }
            incl[tile] = op.combine(ex, tile_agg);
            f.store(2u, cuda::memory_order_release);
        }
        s_prefix = ex;
    }
    __syncthreads();
    T prefix = op.combine(s_prefix, thread_excl);
    op.store(base, n, v, prefix);
}

// Tag monoid (Table 1): point increment (coordinate count + subpath-end bit),
// path bits, style bits, and the subpath segmentation as a max of
// (index + 1) over subpath-end tags.
struct TagOp {
    using T = uint4;
    const uint8_t* tags;
    TagInfo info;

    __device__ __forceinline__ T identity() const { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ T combine(T a, T b) const {
        return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w > b.w ? a.w : b.w);
    }
    __device__ static __forceinline__ T shfl_up(T v, int d) {
        return make_uint4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                          __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
    }
    __device__ static __forceinline__ T value(uint8_t t, uint64_t i) {
        uint32_t end = (t & SE_TAG_SUBPATH_END) ? 1u : 0u;
        return make_uint4((t & SE_TAG_COUNT_MASK) + end, (t & SE_TAG_PATH) ? 1u : 0u, (t & SE_TAG_STYLE) ? 1u : 0u,
                          end ? (uint32_t)(i + 1) : 0u);
    }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
        uint8_t b[kScanItems];
        if (base + kScanItems <= n) {
            uint4 q = *reinterpret_cast<const uint4*>(tags + base);
            const uint8_t* qb = reinterpret_cast<const uint8_t*>(&q);
#pragma unroll
            for (int k = 0; k < kScanItems; k++) b[k] = qb[k];
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; k++) b[k] = (base + k < n) ? tags[base + k] : 0;
        }
#pragma unroll
        for (int k = 0; k < kScanItems; k++) v[k] = (base + k < n) ? value(b[k], base + k) : identity();
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            T ex = combine(prefix, k ? v[k - 1] : identity());
            T in = combine(prefix, v[k]);
            info.pt_base[i] = ex.x;
            info.path[i] = ex.y;
            info.style[i] = in.z - 1u;
            info.sub_first[i] = ex.w;
        }
    }
};

// Exclusive scan of per-tag primitive counts -> offsets; per-path offsets at
// path-bit tags; the total at the end.
struct CountOp {
    using T = unsigned long long;
    const uint32_t* counts;
    const uint8_t* tags;
    const uint32_t* path;
    uint64_t* offsets;
    uint64_t* path_offset;
    uint32_t n_paths;
    uint64_t* total;
    uint64_t capacity;
    uint32_t* status;

    __device__ __forceinline__ T identity() const { return 0ull; }
    __device__ __forceinline__ T combine(T a, T b) const { return a + b; }
    __device__ static __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) v[k] = (base + k < n) ? (T)counts[base + k] : 0ull;
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            T ex = prefix + (k ? v[k - 1] : 0ull);
            T in = prefix + v[k];
            offsets[i] = ex;
            if (path_offset && (tags[i] & SE_TAG_PATH)) {
                if (path[i] < n_paths) path_offset[path[i] + 1] = in;
                else atomicOr(status, (uint32_t)kStatusBadTag);
            }
            if (i == n - 1) {
                offsets[n] = in;
                *total = in;
                if (path_offset) path_offset[0] = 0ull;
                if (in > capacity) atomicOr(status, (uint32_t)kStatusCapacity);
            }
        }
    }
};

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

    __device__ __forceinline__ void put_at(uint64_t at, float2 a, float2 b, float k, bool flip) {
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
    __device__ __forceinline__ void put(float2 a, float2 b, float k, bool flip) { put_at(pos++, a, b, k, flip); }
};

struct Ctx {
    float tol_fit, tol_flat;
    bool arcs;
    uint32_t flags;
};

__device__ __forceinline__ uint32_t offset_n(Ctx& c, const ES& e, float sh, float a, float b) {
    if (c.arcs) return count_of(arc_count((b - a) * e.L, e.k1 / (e.L * e.L), fabsf(sh), c.tol_flat), c.flags);
    return count_of(line_count(e.k0, e.k1, sh / e.L, a, b, c.tol_flat / e.L), c.flags);
}

__device__ __forceinline__ float offset_sample(const ES& e, float sh, bool arcs, float a, float b, int i, int n) {
    if (arcs) {
        if (i == 0) return a;
        if (i == n) return b;
        return a + (b - a) * ((float)i / (float)n);
    }
    return line_s(e, sh / e.L, a, b, i, n);
}

// parallel curve over [a, b] in n primitives, forward or reversed
template <bool W>
__device__ __forceinline__ void offset_range(Ctx& c, const ES& e, float sh, float a, float b, bool reverse,
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
__device__ __forceinline__ uint32_t evolute_patch(Ctx& c, const ES& e, float sh, float a, float b, Out& o,
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
__device__ __forceinline__ uint32_t piece_side(Ctx& c, const ES& e, float sh, Out& o) {
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
__device__ __forceinline__ uint32_t stroke_pieces(Ctx& c, const Cubic& cu, float h, Out& o, float2& q_end) {
    uint32_t t0_u = 0;
    float dt = 1.0f;
    int depth = 0;
    float2 p0 = cu.p[0];
    float2 q0 = deriv_robust(cu, 0.0f);
    q_end = q0;
    uint32_t cnt = 0;
    for (;;) {
        float t0 = (float)t0_u * dt;
        if (t0 >= 1.0f) break;
        float t1 = t0 + dt;
        float2 p1 = (t1 == 1.0f) ? cu.p[3] : cubic_eval(cu, t1);
        float2 q1 = cu.line ? q0 : deriv_robust(cu, t1);
        Fit f = fit_es(p0, p1, q0, q1, dt);
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
        if (!e.degenerate) es_setup(e, f.chord);
        cnt += piece_side<W>(c, e, h, o);
        cnt += piece_side<W>(c, e, -h, o);
        t0_u += 1u;
        int shift = __ffs((int)t0_u) - 1;
        t0_u >>= shift;
        dt *= (float)(1u << shift);
        depth -= shift;
        p0 = p1;
        q0 = q1;
        q_end = q1;
    }
    return cnt;
}

// polyline of a circular arc about P from A by signed angle ang in n steps, ending exactly at B
template <bool W>
__device__ __forceinline__ void round_poly(float2 P, float2 A, float2 B, float ang, uint32_t n, Out& o, bool flip) {
    if (!W) return;
    float2 prev = A, ra = sub2(A, P);
    for (uint32_t i = 1; i <= n; i++) {
        float2 cur = (i == n) ? B : add2(P, rotate(ra, ang * ((float)i / (float)n)));
        o.put(prev, cur, 0.0f, flip);
        prev = cur;
    }
}

template <bool W>
__device__ __forceinline__ uint32_t join(Ctx& c, float2 P, float2 Ti, float2 To, float h, int style, float ml,
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
__device__ __forceinline__ uint32_t end_cap(Ctx& c, float2 P, float2 T, float h, int cap, Out& o) {
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
__device__ __forceinline__ uint32_t start_cap(Ctx& c, float2 P, float2 T, float h, int cap, Out& o) {
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

__device__ __forceinline__ Cubic load_seg(const float2* pts, uint8_t tag, uint32_t base) {
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
    return cu;
}

// Algorithm 1 for one tag: a segment emits its pieces and its join or end
// cap; a cap marker emits its subpath's start cap (or the dot of a subpath
// with no segments).
// a segment tag's control points must lie inside the point stream
__device__ __forceinline__ bool seg_ok(const ExpandArgs& a, uint8_t tag, uint32_t base) {
    uint32_t cc = tag & SE_TAG_COUNT_MASK;
    return (cc == 1u || cc == 3u) && !(tag & SE_TAG_SUBPATH_END) && (uint64_t)base + cc < a.n_points;
}

// Algorithm 1 for one tag: a segment emits its pieces and its join or end
// cap; a cap marker emits its subpath's start cap (or the dot of a subpath
// with no segments).  Malformed streams set kStatusBadTag and emit nothing
// further for the tag; every index is checked before it is dereferenced.
template <bool W>
__device__ __forceinline__ uint32_t process_tag(const ExpandArgs& a, uint64_t i, Ctx& c, Out& o) {
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

template <bool W>
__global__ void __launch_bounds__(128) expand_kernel(ExpandArgs a) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_tags) return;
    Ctx c;
    c.tol_fit = a.tol_fit;
    c.tol_flat = a.tol_flat;
    c.arcs = a.arcs;
    c.flags = 0;
    Out o;
    o.prims = a.prims;
    o.curv = a.curvature;
    o.pid = a.path_id;
    o.path = a.info.path[i];
    o.pos = 0;
    o.lim = 0;
    o.overflow = 0;
    if (W) {
        if (*a.total > a.capacity) return;
        o.pos = a.offsets[i];
        o.lim = a.offsets[i + 1];
    }
    uint32_t n = process_tag<W>(a, i, c, o);
    if (!W) a.counts[i] = n;
    if (W && o.overflow) c.flags |= kStatusBadTag;
    if (c.flags) atomicOr(a.status, c.flags);
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
static uint32_t n_tiles(uint64_t n) { return (uint32_t)((n + kScanTile - 1) / kScanTile); }

cudaError_t launch_tag_scan(const uint8_t* tags, uint64_t n, TagInfo info, ScanState st, uint32_t* status,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    TagOp op;
    op.tags = tags;
    op.info = info;
    lookback_scan<TagOp><<<n_tiles(n), kScanThreads, 0, s>>>(op, n, st, status);
    return cudaGetLastError();
}

cudaError_t launch_count_scan(const uint32_t* counts, const uint8_t* tags, const uint32_t* path, uint64_t n,
                              uint64_t* offsets, uint64_t* path_offset, uint32_t n_paths, uint64_t* total,
                              uint64_t capacity, ScanState st, uint32_t* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    CountOp op;
    op.counts = counts;
    op.tags = tags;
    op.path = path;
    op.offsets = offsets;
    op.path_offset = path_offset;
    op.n_paths = n_paths;
    op.total = total;
    op.capacity = capacity;
    op.status = status;
    lookback_scan<CountOp><<<n_tiles(n), kScanThreads, 0, s>>>(op, n, st, status);
    return cudaGetLastError();
}

cudaError_t launch_expand_count(const ExpandArgs& a, cudaStream_t s) {
    if (a.n_tags == 0) return cudaSuccess;
    uint32_t blocks = (uint32_t)((a.n_tags + 127) / 128);
    expand_kernel<false><<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_expand_write(const ExpandArgs& a, cudaStream_t s) {
    if (a.n_tags == 0) return cudaSuccess;
    uint32_t blocks = (uint32_t)((a.n_tags + 127) / 128);
    expand_kernel<true><<<blocks, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace se
