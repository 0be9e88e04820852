// Device kernels of the stroke-expansion hot path (Levien & Uguray, arXiv 2405.00127).
//
//   tag_scan     Section 8.2: inclusive scan of the tag monoid over the tag
//                stream, segmented at subpath ends -> per tag: first control
//                point, path id, style id, first tag of its subpath.
//   plan         per tag: Algorithm 2 subdivision (decisions recorded as bits)
//                and the tag's join / cap record (Algorithm 1).
//   item_scan    exclusive scan of (pieces + 1) per tag -> item base per tag.
//   decode       per tag: one reference per accepted piece, plus the tail item.
//   piece        per item: Euler-spiral setup and range counts (Sections 4-7).
//   prim_scan    exclusive scan of the item counts -> primitive offsets, per-tag
//                and per-path offsets, the total (replaces the paper's atomic
//                bump allocation, so the output order is deterministic).
//   emit         per output primitive: its vertices, written coalesced.
//
// Both scans are single-pass decoupled look-back scans: each block takes a
// ticket, scans its 4096-item tile in registers and shared memory with warp
// shuffles, publishes its aggregate, and walks back over its predecessors'
// published values.  Every wait is bounded; on timeout the block records
// kStatusTimeout and continues, so no launch can hang.
#include <mutex>

#include "bulk.cuh"
#include "pipeline.cuh"
#include "launch.h"
#include "scan.cuh"
#include "stroke_math.cuh"

namespace se {

// Tag monoid (Table 1): point increment (coordinate count + subpath-end bit),
// path bits, style bits, and the subpath segmentation as a max of
// (index + 1) over subpath-end tags.
struct TagOp {
    using T = TagVal;
    const uint8_t* tags;
    TagInfo info;

    __device__ __forceinline__ T identity() const { return T{0u, 0u, 0u, 0u, 0u, 0u}; }
    __device__ __forceinline__ T combine(T a, T b) const {
        return T{a.pt + b.pt, a.path + b.path, a.style + b.style, a.xf + b.xf, a.sub > b.sub ? a.sub : b.sub,
                 a.crv + b.crv};
    }
    __device__ static __forceinline__ T shfl_up(T v, int d) {
        return T{__shfl_up_sync(0xffffffffu, v.pt, d), __shfl_up_sync(0xffffffffu, v.path, d),
                 __shfl_up_sync(0xffffffffu, v.style, d), __shfl_up_sync(0xffffffffu, v.xf, d),
                 __shfl_up_sync(0xffffffffu, v.sub, d), __shfl_up_sync(0xffffffffu, v.crv, d)};
    }
    // a quadratic or cubic segment: Algorithm 2's subdivision loop in the plan pass
    __device__ static __forceinline__ bool is_curve(uint8_t t) {
        return !(t & SE_TAG_SUBPATH_END) && (t & SE_TAG_COUNT_MASK) >= 2u;
    }
    // subpaths end at subpath-end tags and never span paths, so a path bit
    // also starts a new segment of the scan.  A tag adds (count + 1 when it
    // starts a subpath) points of its own width to the path data stream; the
    // previous tag `p` tells whether it starts one.
    __device__ static __forceinline__ bool starts_subpath(uint8_t p, uint64_t i) {
        return i == 0 || (p & (SE_TAG_SUBPATH_END | SE_TAG_PATH));
    }
    __device__ static __forceinline__ uint32_t words_of(uint8_t t, uint8_t p, uint64_t i) {
        const uint32_t cc = t & SE_TAG_COUNT_MASK;
        if (cc == 0u) return 0u;
        return (cc + (starts_subpath(p, i) ? 1u : 0u)) * ((t & SE_TAG_F32) ? 2u : 1u);
    }
    __device__ static __forceinline__ T value(uint8_t t, uint8_t p, uint64_t i) {
        uint32_t brk = (t & (SE_TAG_SUBPATH_END | SE_TAG_PATH)) ? 1u : 0u;
        return T{words_of(t, p, i), (t & SE_TAG_PATH) ? 1u : 0u, (t & SE_TAG_STYLE) ? 1u : 0u,
                 (t & SE_TAG_TRANSFORM) ? 1u : 0u, brk ? (uint32_t)(i + 1) : 0u, is_curve(t) ? 1u : 0u};
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
        const uint8_t before = (base > 0 && base - 1 < n) ? tags[base - 1] : (uint8_t)0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++)
            v[k] = (base + k < n) ? value(b[k], k ? b[k - 1] : before, base + k) : identity();
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            T ex = combine(prefix, k ? v[k - 1] : identity());
            T in = combine(prefix, v[k]);
            // the tag's first point: its subpath's start (stored with it), else the
            // previous tag's last point, one point of this width back
            const uint8_t t = tags[i], p = i ? tags[i - 1] : (uint8_t)0;
            const uint32_t back = starts_subpath(p, i) ? 0u : ((t & SE_TAG_F32) ? 2u : 1u);
            info.pt_base[i] = ex.pt >= back ? ex.pt - back : 0u;
            info.path[i] = ex.path;
            info.style[i] = in.style - 1u;
            info.sub_first[i] = ex.sub;
            if (info.xform) info.xform[i] = in.xf - 1u;  // ~0u before the first transform entry
            if (info.curve_list) {
                // the plan pass's schedule: curves first, then the rest, each in stream order
                if (in.crv != ex.crv) info.curve_list[ex.crv] = (uint32_t)i;
                else info.line_list[i - ex.crv] = (uint32_t)i;
                if (i == n - 1) *info.n_curves = in.crv;
            }
        }
    }
};

// Exclusive scan of u32 counts into u64 offsets (offsets[n] = total).
struct OffsetOp {
    using T = unsigned long long;
    const uint32_t* counts;
    uint64_t* offsets;
    uint64_t* total;

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
            offsets[i] = prefix + (k ? v[k - 1] : 0ull);
            if (i == n - 1) {
                offsets[n] = prefix + v[k];
                if (total) *total = prefix + v[k];
            }
        }
    }
};

// Exclusive scan of the item counts into primitive offsets, with the per-tag
// and per-path offsets of the caller's outline and the capacity check.
struct PrimScanOp {
    using T = unsigned long long;
    const uint32_t* counts;
    const uint32_t* item_tag;
    const uint32_t* item_ref;
    const uint8_t* tags;
    const uint32_t* path;
    uint64_t n_tags;
    const uint64_t* n_tags_dev;
    uint32_t n_paths;
    uint64_t* offsets;
    uint64_t* tag_offset;
    uint64_t* path_offset;
    uint64_t* total;
    uint64_t capacity;
    uint32_t* status;
    const uint32_t* dash_status;
    const uint64_t* items_total;  // the item scan's total: above item_cap, decode wrote no owners
    uint64_t item_cap;

    __device__ __forceinline__ T identity() const { return 0ull; }
    __device__ __forceinline__ T combine(T a, T b) const { return a + b; }
    __device__ static __forceinline__ T shfl_up(T v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) v[k] = (base + k < n) ? (T)counts[base + k] : 0ull;
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
        // the owners and per-tag offsets come from the item scan and decode: not
        // trusted after a timeout, and not written when the items overflowed the
        // workspace (decode then recorded kStatusWorkspace and wrote nothing)
        if (scan_untrusted(status, dash_status) || *items_total > item_cap) return;
        // A tag's items are its pieces, then its tail item, so an item starts its
        // tag exactly when the item before it is a tail (or it is item 0): the
        // per-tag offsets need the owner only of first and tail items, and no
        // lookup of the tag's first item.
        const bool outline = tag_offset || path_offset;
        uint32_t ref_prev = kTailRef;
        if (outline && base > 0 && base - 1 < n) ref_prev = item_ref[base - 1];
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            T ex = prefix + (k ? v[k - 1] : 0ull);
            T in = prefix + v[k];
            offsets[i] = ex;
            if (outline) {
                const uint32_t ref = item_ref[i];
                const bool first = tag_offset && ref_prev == kTailRef, tail = path_offset && ref == kTailRef;
                ref_prev = ref;
                if (first || tail) {
                    const uint32_t t = item_tag[i];
                    if (first) tag_offset[t] = ex;
                    if (tail && (tags[t] & SE_TAG_PATH)) {
                        if (path[t] < n_paths) path_offset[path[t] + 1] = in;
                        else atomicOr(status, (uint32_t)kStatusBadTag);
                    }
                }
            }
            if (i == n - 1) {
                offsets[n] = in;
                *total = in;
                if (tag_offset) {
                    uint64_t nt = n_tags;
                    if (n_tags_dev && *n_tags_dev < nt) nt = *n_tags_dev;
                    tag_offset[nt] = in;
                }
                if (path_offset) path_offset[0] = 0ull;
                if (in > capacity || in >= (1ull << 32)) atomicOr(status, (uint32_t)kStatusCapacity);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// plan / decode / piece
// ---------------------------------------------------------------------------
// One thread per tag.  Curves (quadratics and cubics) carry the subdivision loop
// of Algorithm 2 while lines take one trivial fit, so the tag scan lists the
// curve tags first and the other tags after them, and the plan pass takes tags
// in that order: every block but one holds tags of one class, whose lanes run
// loops of similar length and whose warps finish together (sorting each block's
// tags instead left the line warps of a mixed block idle until its curve warps
// were done: 26% of the SM's warp slots busy against 50% possible).  Four
// 256-thread blocks per SM (64 registers) measured faster than the 78 registers
// the compiler takes unbounded (0.432 against 0.471 ms on map-like).
__global__ void __launch_bounds__(256, 4) plan_kernel(ExpandArgs a, PlanBufs pb) {
    const uint64_t n = tag_count(a);
    const uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= n || scan_untrusted(a.status, a.dash_status)) return;
    const uint64_t nc = *a.info.n_curves;
    const uint64_t i = slot < nc ? a.info.curve_list[slot] : a.info.line_list[slot - nc];
    uint32_t flags = 0;
    PlanOut po;
    TailRec t;
    plan_tag(a, i, po, t, flags);
    pb.n_items[i] = po.n_pieces + 1u;
    pb.bits[i] = po.bits;
    pb.overflow[i] = po.overflow ? 1u : 0u;
    pb.tails[i] = t;
    if (flags) atomicOr(a.status, flags);
}

__global__ void __launch_bounds__(256) decode_kernel(ExpandArgs a, PlanBufs pb) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tag_count(a)) return;
    if (scan_untrusted(a.status, a.dash_status)) return;
    if (*pb.items_total > pb.item_cap) {
        if (i == 0) atomicOr(a.status, (uint32_t)kStatusWorkspace);
        return;
    }
    uint64_t b = pb.item_base[i];
    uint32_t np = pb.n_items[i] - 1u;
    if (np > 0u) {
        // pieces are numbered densely (tag i's first piece is b - i), so the
        // piece passes run over pieces only and keep compact records
        const uint64_t p0 = b - i;
        Cubic cu = load_seg(a.words, a.tags[i], a.info.pt_base[i], tag_xform(a, i));
        PlanOut po;
        po.n_pieces = np;
        po.bits = pb.bits[i];
        po.overflow = pb.overflow[i] != 0u;
        uint32_t* refs = pb.item_ref;
        uint32_t* owner = pb.item_tag;
        uint32_t* pitem = pb.piece_item;
        decode_segment(cu, po, a.tol_fit, [&](uint32_t k, uint32_t ref) {
            if (k < np) {
                refs[b + k] = ref;
                owner[b + k] = (uint32_t)i;
                pitem[p0 + k] = (uint32_t)(b + k);
            }
        });
    }
    const TailRec t = pb.tails[i];
    pb.item_ref[b + np] = kTailRef;
    pb.item_tag[b + np] = (uint32_t)i;
    pb.item_count[b + np] = tail_total(t);
    pb.item_vcount[b + np] = tail_verts(t);
}
// One record per piece, built in shared memory (the piece's values go there
// field by field from registers, never through local memory); each warp then
// copies 32 consecutive records -- 6,912 contiguous bytes of the record array --
// to global memory with coalesced 8-byte stores, whole sectors at a time.  256-thread blocks, 55.3 KB of records each, four per
// SM: measured against the same staging in 128-thread blocks (1.20 ms) and the
// record built in local memory and stored per thread (1.17 ms), the piece stage
// takes 1.08 ms on map-like.
constexpr uint32_t kPieceWords2 = sizeof(PieceRec) / 8;  // 8-byte words per record
static_assert(sizeof(PieceRec) % 8 == 0, "piece records are copied as 8-byte words");

// kPieceThreads: the records one block stages (256: four blocks per SM; 128:
// eight) -- the piece pass's tile, a tuning knob.
//
// Each step fits its pieces (one per thread, in item order); for line output
// it then regroups them by work class before the range counts: pieces whose
// parallel curve has a cusp on the +h side (an evolute patch: an extra range,
// its count and the evolute count, done in that side's call), then those with
// one on the -h side only, then the rest, so a warp runs one side's patch code
// at a time and the warps without patches never wait on it (piece stage 1.08 ->
// 0.99 ms on map-like with two classes).
// The records stay in place in shared memory; only the thread that counts a
// record changes.
template <bool kArcs, bool kRefine, int kPieceThreads>
__global__ void __launch_bounds__(kPieceThreads, 1024 / kPieceThreads) piece_kernel(ExpandArgs a, PlanBufs pb) {
    __shared__ PieceRec s_rec[kPieceThreads];
    __shared__ uint32_t s_perm[kArcs ? 1 : kPieceThreads];
    __shared__ uint32_t s_wcount[kArcs ? 1 : 2 * (kPieceThreads / 32)];
    const uint64_t n_items = *pb.items_total;
    if (n_items > pb.item_cap || scan_untrusted(a.status, a.dash_status)) return;
    const uint64_t n_pieces = n_items - tag_count(a);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wib = tid >> 5;
    // the grid is sized from the tag count; a scene with more pieces than threads
    // loops (whole blocks at a time: every thread takes every step)
    for (uint64_t base = (uint64_t)blockIdx.x * kPieceThreads; base < n_pieces;
         base += (uint64_t)gridDim.x * kPieceThreads) {
        const uint32_t cnt = (uint32_t)(n_pieces - base < kPieceThreads ? n_pieces - base : kPieceThreads);
        uint32_t cls = 0;  // work class (line output): which side holds an evolute patch
        if (tid < cnt) {
            PieceRec& pr = s_rec[tid];
            const uint32_t j = pb.piece_item[base + tid];
            const uint32_t i = pb.item_tag[j];
            const se_style st = a.styles[a.info.style[i]];
            Cubic cu = load_seg(a.words, a.tags[i], a.info.pt_base[i], tag_xform(a, i));
            uint32_t t0_u;
            int depth;
            unpack_ref(pb.item_ref[j], t0_u, depth);
            const float h = st.fill ? 0.0f : st.half_width * xf_scale(tag_xform(a, i));
            pr.item = j;
            pr.path = a.info.path[i];
            if constexpr (!kArcs) {
                build_piece_shape(cu, t0_u, depth, h, pr);
                cls = piece_patch_class(pr);
            } else {
                // arc output: the whole piece at once (its range counts are closed forms)
                uint32_t flags = 0, verts = 0;
                const uint32_t total = build_piece<kArcs, kRefine>(cu, t0_u, depth, h, a.tol_flat, pr, flags, &verts);
                pb.item_count[j] = total;
                pb.item_vcount[j] = verts;
                if (flags) atomicOr(a.status, flags);
            }
        }
        // line output: patch pieces first (by side), then the others, each in item
        // order (threads past the end keep the block's last slots).  Arc output counts
        // a range in closed form, too cheap to pay for the block barriers: each
        // thread built its whole record above.
        if constexpr (!kArcs) {
            // classes in the order 2, 1, 0: each block-wide run holds one class
            const uint32_t m2 = __ballot_sync(0xffffffffu, cls == 2u), m1 = __ballot_sync(0xffffffffu, cls == 1u);
            if (lane == 0) {
                s_wcount[wib] = __popc(m2);
                s_wcount[kPieceThreads / 32 + wib] = __popc(m1);
            }
            __syncthreads();
            uint32_t b2 = 0, b1 = 0, t2 = 0, t1 = 0;
#pragma unroll
            for (uint32_t w = 0; w < kPieceThreads / 32; w++) {
                const uint32_t c2 = s_wcount[w], c1 = s_wcount[kPieceThreads / 32 + w];
                b2 += w < wib ? c2 : 0u;
                b1 += w < wib ? c1 : 0u;
                t2 += c2;
                t1 += c1;
            }
            const uint32_t below = (1u << lane) - 1u;
            const uint32_t r2 = __popc(m2 & below), r1 = __popc(m1 & below);
            const uint32_t b0 = wib * 32u - b2 - b1, r0 = lane - r2 - r1;
            s_perm[cls == 2u ? b2 + r2 : (cls == 1u ? t2 + b1 + r1 : t2 + t1 + b0 + r0)] = tid;
            __syncthreads();
            const uint32_t q = s_perm[tid];
            if (q < cnt) {
                PieceRec& pr = s_rec[q];
                uint32_t flags = 0, verts = 0;
                const uint32_t total = build_piece_sides<kArcs, kRefine>(pr, a.tol_flat, flags, &verts);
                pb.item_count[pr.item] = total;
                pb.item_vcount[pr.item] = verts;
                if (flags) atomicOr(a.status, flags);
            }
        }
        // every record the warp copies is complete
        if constexpr (!kArcs) __syncthreads();
        else __syncwarp();
        const uint32_t w0 = wib * 32u;
        if (w0 < cnt) {
            const uint32_t wc = cnt - w0 < 32u ? cnt - w0 : 32u;
            const uint2* src = reinterpret_cast<const uint2*>(&s_rec[w0]);
            uint2* dst = reinterpret_cast<uint2*>(pb.pieces + base + w0);
            for (uint32_t w = lane; w < wc * kPieceWords2; w += 32u) dst[w] = src[w];
        }
        // the next step overwrites the records
        if constexpr (!kArcs) __syncthreads();
        else __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// emit: one lane per chain vertex.  A persistent grid walks chunks of
// 32 * kEmitPer consecutive vertices per warp; lanes of a warp mostly share a
// chain, so they run the same code on neighbouring parameters.  Each lane
// writes its vertex into the one or two primitives that share it.
// ---------------------------------------------------------------------------
// largest j in [lo, hi) with off[j] <= p (off[lo] <= p is assumed)
__device__ __forceinline__ uint64_t find_item(const uint64_t* off, uint64_t lo, uint64_t hi, uint64_t p) {
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (off[mid] <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void put_vertex(const ExpandArgs& a, uint64_t prim, bool as_end, float2 v) {
    float2* p2 = reinterpret_cast<float2*>(a.prims);
    p2[2 * prim + (as_end ? 1 : 0)] = v;
}

// Index of the piece holding vertex w of a warp's chunk: the largest j with
// start[j] <= w (pieces without vertices share the next one's start).
__device__ __forceinline__ uint32_t vertex_piece(const uint32_t* start, uint32_t w) {
    uint32_t j = 0;
#pragma unroll
    for (uint32_t step = 16; step > 0; step >>= 1)
        if (start[j + step] <= w) j += step;
    return j;
}

// Line output: vertex kk of chain c goes to the primitives that share it (both
// copies of an evolute chain); pbase is the chain's first primitive.
__device__ __forceinline__ void write_line_vertex(float4* prims, uint32_t* path_id, uint64_t pbase, const Chain& c,
                                                  uint32_t kk, uint32_t path, float2 pos) {
    float2* p2 = reinterpret_cast<float2*>(prims);
    const int copies = c.type == kChEvolute ? 2 : 1;
    for (int cp = 0; cp < copies; cp++) {
        const uint64_t b0 = pbase + (uint64_t)cp * c.n;
        if (kk < c.n) {
            p2[2 * (b0 + kk) + (c.flip != 0u ? 1 : 0)] = pos;
            if (path_id) path_id[b0 + kk] = path;
        }
        if (kk > 0u) p2[2 * (b0 + kk - 1u) + (c.flip == 0u ? 1 : 0)] = pos;
    }
}

// Vertex w of a warp's chunk placed by the density inverse (lines) and the
// quadrature: the vertices without a closed form.  Out of line: one compiled
// copy serves the queue's flushes and its drain (instruction fetch, not
// arithmetic, bounds this kernel once its lanes are busy).
template <bool kArcs, bool kRefine>
static __device__ __noinline__ void place_vertex(float4* prims, uint32_t* path_id, const PieceRec* prs,
                                                 const uint32_t* start, const unsigned long long* off,
                                                 const uint32_t* paths, uint32_t w) {
    const uint32_t j = vertex_piece(start, w);
    const PieceRec& pr = prs[j];
    Chain c;
    piece_chain_at(pr, w - start[j], c);
    const uint32_t kk = w - start[j] - c.v_off;
    const float2 pos = piece_vertex_t<kArcs, kRefine>(pr.es, c, kk);
    write_line_vertex(prims, path_id, off[j] + c.p_off, c, kk, paths[j], pos);
}

// Signed curvature of arc primitive kk - 1 of parallel-curve chain c (stored as
// `prim`, its vertices in chain order unless the chain is flipped): the circle
// through its end points and the parallel curve's point at the mid parameter.
static __device__ __noinline__ float arc_curvature(const ES& es, Chain c, uint32_t kk, float4 prim) {
    const float2 lo = f2(prim.x, prim.y), hi = f2(prim.z, prim.w);
    const float2 prev = c.flip ? hi : lo, pos = c.flip ? lo : hi;
    const float s0 = chain_param(es, c, true, kk - 1u), s1 = chain_param(es, c, true, kk);
    return menger(prev, es_offset(es, 0.5f * (s0 + s1), c.sh), pos);
}

// Piece vertices, item-parallel.  Each warp takes 32 consecutive items, copies
// their piece records into shared memory with coalesced word loads, numbers
// their vertices with a warp scan and then sweeps that vertex list one vertex
// per lane: a lane finds its item in shared memory (5-step search over the
// warp's 32 starts), so no vertex searches global offsets or walks a record
// in global memory, and the lanes of one sweep mostly run the same
// parallel-curve code on neighbouring vertices.
static_assert(sizeof(PieceRec) % 4 == 0, "piece records are copied as words");

template <bool kArcs, bool kRefine, int kPieceEmitThreads>
__global__ void __launch_bounds__(kPieceEmitThreads) emit_pieces_kernel(ExpandArgs a, PlanBufs pb) {
    constexpr int kPieceEmitWarps = kPieceEmitThreads / 32;
    __shared__ __align__(16) PieceRec s_pr[kPieceEmitWarps][32];
    __shared__ __align__(8) uint64_t s_bar[kPieceEmitWarps];  // the warp's bulk-copy barrier
    __shared__ uint32_t s_vstart[kPieceEmitWarps][33];
    __shared__ unsigned long long s_off[kPieceEmitWarps][32];
    __shared__ uint32_t s_path[kPieceEmitWarps][32];
    __shared__ uint32_t s_queue[kPieceEmitWarps][64];  // line output: vertices waiting for a full warp
    const uint64_t total = *a.total;
    const uint64_t n_items = *pb.items_total;
    if (total > a.capacity || n_items > pb.item_cap || scan_untrusted(a.status, a.dash_status)) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t n_warps = (uint64_t)gridDim.x * kPieceEmitWarps;
    const uint64_t n_all = n_items - tag_count(a);
    const uint64_t p_begin = a.emit_piece_lo < n_all ? a.emit_piece_lo : n_all;
    const uint64_t n_pieces = a.emit_piece_hi < n_all ? a.emit_piece_hi : n_all;  // end of the range
    const uint64_t n_chunks = (n_pieces - (p_begin < n_pieces ? p_begin : n_pieces) + 31) / 32;
    constexpr uint32_t kWords = sizeof(PieceRec) / 4;
    if (lane == 0) bulk_bar_init(&s_bar[wib]);
    __syncwarp();
    uint32_t phase = 0;
    for (uint64_t chunk = (uint64_t)blockIdx.x * kPieceEmitWarps + wib; chunk < n_chunks; chunk += n_warps) {
        const uint64_t p0 = p_begin + chunk * 32;
        const uint32_t cnt = (uint32_t)(n_pieces - p0 < 32 ? n_pieces - p0 : 32);
        // The chunk's records are contiguous: one bulk copy on the copy engine when
        // the chunk starts on a 16-byte boundary (always, unless an emit range
        // starts at an odd piece), rounded up to 16 bytes (the record array has the
        // slack), else word copies by the lanes.
        if ((reinterpret_cast<uintptr_t>(pb.pieces + p0) & 15u) == 0u) {
            if (lane == 0)
                bulk_load(&s_pr[wib][0], pb.pieces + p0, (cnt * (uint32_t)sizeof(PieceRec) + 15u) & ~15u, &s_bar[wib]);
            if (!bulk_wait(&s_bar[wib], phase)) {
                // the copy did not land: record it, let it drain (bounded), stop
                if (lane == 0) atomicOr(a.status, (uint32_t)kStatusTimeout);
                bulk_wait(&s_bar[wib], phase);
                return;
            }
            phase ^= 1u;
        } else {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(pb.pieces + p0);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_pr[wib][0]);
            for (uint32_t w = lane; w < cnt * kWords; w += 32) dst[w] = src[w];
        }
        __syncwarp();  // the records are in shared memory
        uint32_t nv = 0;
        if ((uint32_t)lane < cnt) {
            // the record carries its item and path: one dependent load for the offset
            const PieceRec& pr = s_pr[wib][lane];
            nv = piece_verts(pr);
            s_off[wib][lane] = pb.item_off[pr.item];
            s_path[wib][lane] = pr.path;
        }
        uint32_t incl = nv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        s_vstart[wib][lane] = incl - nv;
        if (lane == 31) s_vstart[wib][32] = incl;
        __syncwarp();
        const uint32_t V = s_vstart[wib][32];
        // Vertices.  Each lane writes its vertex into the primitives that share it
        // (8-byte halves: vertex k ends primitive k - 1 and starts primitive k).
        // Most vertices of map-like scenes are chain ends at piece ends, whose
        // positions have a closed form; the rest need the density inverse (lines)
        // and the arc-length quadrature.  A sweep places its closed-form vertices
        // at once and queues the others in shared memory; whenever 32 are queued
        // the warp places them together, so the expensive code runs with full
        // warps instead of the quarter of a sweep's lanes that need it.  (One
        // sweep over all vertices with the expensive code inline measured 2.0 ms
        // on map-like lines, sweeping interior and end vertices apart 2.4 ms; the
        // queue 1.45 ms.)
        uint32_t qn = 0;  // queued vertices (warp-uniform, below 32 between sweeps)
        for (uint32_t w0 = 0; w0 < V; w0 += 32) {
            const uint32_t w = w0 + lane;
            bool deferred = false;
            if (w < V) {
                const uint32_t j = vertex_piece(s_vstart[wib], w);
                const PieceRec& pr = s_pr[wib][j];
                Chain c;
                piece_chain_at(pr, w - s_vstart[wib][j], c);
                const uint32_t kk = w - s_vstart[wib][j] - c.v_off;
                float2 pos;
                if (end_vertex(pr.es, c.type, c.n, c.a, c.b, c.sh, kk, pos))
                    write_line_vertex(a.prims, a.path_id, s_off[wib][j] + c.p_off, c, kk, s_path[wib][j], pos);
                else
                    deferred = true;
            }
            const uint32_t dm = __ballot_sync(0xffffffffu, deferred);
            if (deferred) s_queue[wib][qn + __popc(dm & ((1u << lane) - 1u))] = w;
            qn += __popc(dm);
            if (qn >= 32u) {
                __syncwarp();
                place_vertex<kArcs, kRefine>(a.prims, a.path_id, s_pr[wib], s_vstart[wib], s_off[wib], s_path[wib],
                                             s_queue[wib][lane]);
                __syncwarp();
                if ((uint32_t)lane < qn - 32u) s_queue[wib][lane] = s_queue[wib][32 + lane];
                __syncwarp();
                qn -= 32u;
            }
        }
        __syncwarp();
        if ((uint32_t)lane < qn)
            place_vertex<kArcs, kRefine>(a.prims, a.path_id, s_pr[wib], s_vstart[wib], s_off[wib], s_path[wib],
                                         s_queue[wib][lane]);
        if constexpr (kArcs) {
            // Arc output: each primitive's curvature, from the circle through its
            // two end points (written above by this warp, read back from L1) and
            // the parallel curve's point at its mid parameter.  Every primitive of
            // a parallel-curve chain evaluates one such point, so the lanes of this
            // sweep mostly run the same code.
            __syncwarp();  // the warp's vertex stores are visible to all its lanes
            if (a.curvature) {
                for (uint32_t w = lane; w < V; w += 32) {
                    const uint32_t j = vertex_piece(s_vstart[wib], w);
                    const PieceRec& pr = s_pr[wib][j];
                    Chain c;
                    piece_chain_at(pr, w - s_vstart[wib][j], c);
                    const uint32_t kk = w - s_vstart[wib][j] - c.v_off;
                    if (kk == 0u) continue;
                    const uint64_t q = s_off[wib][j] + c.p_off + kk - 1u;
                    float curv = 0.0f;
                    if (c.type == kChOffset || c.type == kChOffsetRev)
                        curv = arc_curvature(pr.es, c, kk, a.prims[q]);
                    if (c.flip) curv = -curv;
                    a.curvature[q] = curv;
                    if (c.type == kChEvolute) a.curvature[q + c.n] = curv;
                }
            }
        }
        __syncwarp();  // the next chunk overwrites this warp's shared records
    }
}

// Tail vertices (joins, caps), tag-parallel like the piece kernel: each warp
// takes 32 consecutive tags, stages their tail records in shared memory,
// numbers their vertices with a warp scan and sweeps that list one vertex per
// lane; instantiated per output kind.
static_assert(sizeof(TailRec) % 4 == 0, "tail records are copied as words");

template <bool kArcs, int kTailEmitThreads>
__global__ void __launch_bounds__(kTailEmitThreads) emit_tails_kernel(ExpandArgs a, PlanBufs pb) {
    constexpr int kTailEmitWarps = kTailEmitThreads / 32;
    __shared__ __align__(16) TailRec s_tr[kTailEmitWarps][32];
    __shared__ __align__(8) uint64_t s_bar[kTailEmitWarps];  // the warp's bulk-copy barrier
    __shared__ uint32_t s_vstart[kTailEmitWarps][33];
    __shared__ unsigned long long s_off[kTailEmitWarps][32];
    __shared__ uint32_t s_path[kTailEmitWarps][32];
    const uint64_t total = *a.total;
    const uint64_t n_items = *pb.items_total;
    if (total > a.capacity || n_items > pb.item_cap || scan_untrusted(a.status, a.dash_status)) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t n_warps = (uint64_t)gridDim.x * kTailEmitWarps;
    const uint64_t n_all = tag_count(a);
    const uint64_t t_begin = a.emit_tag_lo < n_all ? a.emit_tag_lo : n_all;
    const uint64_t n_tags = a.emit_tag_hi < n_all ? a.emit_tag_hi : n_all;  // end of the range
    const uint64_t n_chunks = (n_tags - (t_begin < n_tags ? t_begin : n_tags) + 31) / 32;
    constexpr uint32_t kWords = sizeof(TailRec) / 4;
    if (lane == 0) bulk_bar_init(&s_bar[wib]);
    __syncwarp();
    uint32_t phase = 0;
    for (uint64_t chunk = (uint64_t)blockIdx.x * kTailEmitWarps + wib; chunk < n_chunks; chunk += n_warps) {
        const uint64_t t0 = t_begin + chunk * 32;
        const uint32_t cnt = (uint32_t)(n_tags - t0 < 32 ? n_tags - t0 : 32);
        // one bulk copy of the chunk's contiguous records when it starts on a
        // 16-byte boundary (the record array has the slack for the rounding)
        if ((reinterpret_cast<uintptr_t>(pb.tails + t0) & 15u) == 0u) {
            if (lane == 0)
                bulk_load(&s_tr[wib][0], pb.tails + t0, (cnt * (uint32_t)sizeof(TailRec) + 15u) & ~15u, &s_bar[wib]);
            if (!bulk_wait(&s_bar[wib], phase)) {
                if (lane == 0) atomicOr(a.status, (uint32_t)kStatusTimeout);
                bulk_wait(&s_bar[wib], phase);
                return;
            }
            phase ^= 1u;
        } else {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(pb.tails + t0);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&s_tr[wib][0]);
            for (uint32_t w = lane; w < cnt * kWords; w += 32) dst[w] = src[w];
        }
        uint32_t nv = 0;
        if ((uint32_t)lane < cnt) {
            const uint64_t t = t0 + lane;
            const uint64_t item = pb.item_base[t + 1] - 1;  // the tag's tail item
            nv = pb.item_vcount[item];
            s_off[wib][lane] = pb.item_off[item];
            s_path[wib][lane] = a.info.path[t];
        }
        uint32_t incl = nv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        s_vstart[wib][lane] = incl - nv;
        if (lane == 31) s_vstart[wib][32] = incl;
        __syncwarp();
        const uint32_t V = s_vstart[wib][32];
        for (uint32_t w = lane; w < V; w += 32) {
            uint32_t j = 0;
#pragma unroll
            for (uint32_t step = 16; step > 0; step >>= 1)
                if (s_vstart[wib][j + step] <= w) j += step;
            const TailRec& tr = s_tr[wib][j];
            const uint32_t local = w - s_vstart[wib][j];
            Chain c;
            tail_find_chain(tr, local, c);
            const uint32_t kk = local - c.v_off;
            const float2 pos = tail_vertex(tr, c, kArcs, kk);
            float curv = kArcs ? tail_prim_curvature(tr, c, true) : 0.0f;
            if (c.flip) curv = -curv;
            const uint64_t b0 = s_off[wib][j] + c.p_off;
            if (kk < c.n) {
                put_vertex(a, b0 + kk, c.flip != 0u, pos);
                if (kArcs && a.curvature) a.curvature[b0 + kk] = curv;
                if (a.path_id) a.path_id[b0 + kk] = s_path[wib][j];
            }
            if (kk > 0u) put_vertex(a, b0 + kk - 1u, c.flip == 0u, pos);
        }
        __syncwarp();  // the next chunk overwrites this warp's shared records
    }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
static uint32_t n_tiles(uint64_t n) { return (uint32_t)((n + kScanTile - 1) / kScanTile); }
static uint32_t blocks_for(uint64_t n, uint32_t t) { return (uint32_t)((n + t - 1) / t); }

// Pieces a scene of n_tags tags is sized for on the host (the device count is
// known only after the item scan): 8 per tag, where the synthetic scenes take
// about 3.  The piece pass, the primitive scan and the emit grids are sized from
// it and loop when a scene has more, so a small document after a large one
// launches a grid of its own size rather than the workspace's.
static uint64_t pieces_bound(const ExpandArgs& a, const PlanBufs& pb) {
    const uint64_t est = 8ull * a.n_tags + 1024ull;
    return est < pb.item_cap ? est : pb.item_cap;
}

cudaError_t launch_tag_scan(const uint8_t* tags, uint64_t n, const uint64_t* n_dev, TagInfo info, ScanState st,
                            uint32_t* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    TagOp op;
    op.tags = tags;
    op.info = info;
    lookback_scan<TagOp><<<n_tiles(n), kScanThreads, 0, s>>>(op, n, n_dev, st, status);
    return cudaGetLastError();
}

cudaError_t launch_plan(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s) {
    if (a.n_tags == 0) return cudaSuccess;
    plan_kernel<<<blocks_for(a.n_tags, tu.plan_block), tu.plan_block, 0, s>>>(a, pb);
    return cudaGetLastError();
}

cudaError_t launch_item_scan(const ExpandArgs& a, const PlanBufs& pb, ScanState st, cudaStream_t s) {
    if (a.n_tags == 0) return cudaSuccess;
    OffsetOp op;
    op.counts = pb.n_items;
    op.offsets = pb.item_base;
    op.total = pb.items_total;
    lookback_scan<OffsetOp><<<n_tiles(a.n_tags), kScanThreads, 0, s>>>(op, a.n_tags, a.n_tags_dev, st, a.status);
    return cudaGetLastError();
}

cudaError_t launch_decode(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s) {
    if (a.n_tags == 0) return cudaSuccess;
    decode_kernel<<<blocks_for(a.n_tags, tu.plan_block), tu.plan_block, 0, s>>>(a, pb);
    return cudaGetLastError();
}

cudaError_t launch_piece(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s) {
    if (a.n_tags == 0 || pb.item_cap == 0) return cudaSuccess;
    // one thread per piece, up to pieces_bound of them (more loop); the block is
    // the tile of records staged in shared memory (128 or 256)
    const uint64_t want = pieces_bound(a, pb);
    if (tu.piece_block <= 128) {
        const unsigned pg = blocks_for(want, 128);
        if (a.arcs) piece_kernel<true, false, 128><<<pg, 128, 0, s>>>(a, pb);
        else if (a.refine) piece_kernel<false, true, 128><<<pg, 128, 0, s>>>(a, pb);
        else piece_kernel<false, false, 128><<<pg, 128, 0, s>>>(a, pb);
    } else {
        const unsigned pg = blocks_for(want, 256);
        if (a.arcs) piece_kernel<true, false, 256><<<pg, 256, 0, s>>>(a, pb);
        else if (a.refine) piece_kernel<false, true, 256><<<pg, 256, 0, s>>>(a, pb);
        else piece_kernel<false, false, 256><<<pg, 256, 0, s>>>(a, pb);
    }
    return cudaGetLastError();
}

cudaError_t launch_prim_scan(const ExpandArgs& a, const PlanBufs& pb, uint64_t* tag_offset, uint64_t* path_offset,
                             uint32_t n_paths, ScanState st, cudaStream_t s) {
    if (a.n_tags == 0 || pb.item_cap == 0) return cudaSuccess;
    PrimScanOp op;
    op.counts = pb.item_count;
    op.item_tag = pb.item_tag;
    op.item_ref = pb.item_ref;
    op.tags = a.tags;
    op.path = a.info.path;
    op.n_tags = a.n_tags;
    op.n_tags_dev = a.n_tags_dev;
    op.n_paths = n_paths;
    op.offsets = pb.item_off;
    op.tag_offset = tag_offset;
    op.path_offset = path_offset;
    op.total = const_cast<uint64_t*>(a.total);
    op.capacity = a.capacity;
    op.status = a.status;
    op.dash_status = a.dash_status;
    op.items_total = pb.items_total;
    op.item_cap = pb.item_cap;
    // items = pieces + tags; the scan loops over tiles past its grid
    const uint64_t items_bound = pieces_bound(a, pb) + a.n_tags;
    const uint32_t grid = n_tiles(items_bound < pb.item_cap ? items_bound : pb.item_cap);
    lookback_scan<PrimScanOp><<<grid, kScanThreads, 0, s>>>(op, pb.item_cap, pb.items_total, st, a.status);
    return cudaGetLastError();
}

// The persistent emit grids' shape on one device: its SM count and the blocks of
// each emit kernel that fit on an SM.  Computed once per device and kernel
// instantiation (std::call_once: the server's worker threads launch
// concurrently, and a shape read half-written launched empty grids).
struct EmitShape {
    int sms = 1, fit_p = 1, fit_t = 1;
};
constexpr int kMaxDevices = 64;

template <bool ARCS, bool REFINE, int T>
static EmitShape emit_shape() {
    static std::once_flag once[kMaxDevices];
    static EmitShape shape[kMaxDevices];
    int dev = 0;
    cudaGetDevice(&dev);
    auto measure = [dev] {
        EmitShape e;
        int sms = 0, fp = 0, ft = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) e.sms = sms;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fp, emit_pieces_kernel<ARCS, REFINE, T>, T, 0) == cudaSuccess &&
            fp > 0)
            e.fit_p = fp;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ft, emit_tails_kernel<ARCS, T>, T, 0) == cudaSuccess && ft > 0)
            e.fit_t = ft;
        return e;
    };
    if (dev < 0 || dev >= kMaxDevices) return measure();
    std::call_once(once[dev], [&] { shape[dev] = measure(); });
    return shape[dev];
}

template <bool ARCS, bool REFINE, int T>
static cudaError_t launch_emit_kind(const ExpandArgs& a, const PlanBufs& pb, uint32_t per_sm, cudaStream_t s) {
    const EmitShape sh = emit_shape<ARCS, REFINE, T>();
    const int sms = sh.sms, fit_p = sh.fit_p, fit_t = sh.fit_t;
    // the tuning's blocks per SM is in units of 256 threads
    const int scale = 256 / T;
    int pp = per_sm == 0 || scale * (int)per_sm > fit_p ? fit_p : scale * (int)per_sm;
    int pt = per_sm == 0 || scale * (int)per_sm > fit_t ? fit_t : scale * (int)per_sm;
    // persistent grids, but no more blocks than the scene has 32-item chunks for
    // (the kernels stride over chunks, so any grid size is complete)
    const uint64_t warps = T / 32;
    const uint64_t want_p = (pieces_bound(a, pb) / 32 + warps) / warps, want_t = (a.n_tags / 32 + warps) / warps;
    const uint32_t gp = (uint32_t)((uint64_t)(sms * pp) < want_p ? (uint64_t)(sms * pp) : want_p);
    const uint32_t gt = (uint32_t)((uint64_t)(sms * pt) < want_t ? (uint64_t)(sms * pt) : want_t);
    emit_pieces_kernel<ARCS, REFINE, T><<<gp, T, 0, s>>>(a, pb);
    emit_tails_kernel<ARCS, T><<<gt, T, 0, s>>>(a, pb);
    return cudaGetLastError();
}

template <bool ARCS, bool REFINE>
static cudaError_t launch_emit_arcs(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s) {
    // shared records of 32 items per warp: 128 threads is the largest block within
    // the 48 KB of static shared memory
    if (tu.emit_block <= 64) return launch_emit_kind<ARCS, REFINE, 64>(a, pb, tu.emit_blocks_per_sm, s);
    return launch_emit_kind<ARCS, REFINE, 128>(a, pb, tu.emit_blocks_per_sm, s);
}

// Chunk boundaries of an emit split into k_chunks tag ranges: for boundary k the
// tag t_k = k T / k_chunks (T the stream's tag count), its first piece and its
// first primitive -- out[3k], out[3k + 1], out[3k + 2].
__global__ void chunk_bounds_kernel(ExpandArgs a, PlanBufs pb, uint32_t k_chunks, uint64_t* out) {
    const uint32_t k = threadIdx.x;
    if (k > k_chunks) return;
    const uint64_t T = tag_count(a);
    const uint64_t t = k == k_chunks ? T : T * k / k_chunks;
    const uint64_t ib = pb.item_base[t];
    out[3 * k] = t;
    out[3 * k + 1] = ib - t;
    out[3 * k + 2] = pb.item_off[ib];
}

cudaError_t launch_chunk_bounds(const ExpandArgs& a, const PlanBufs& pb, uint32_t k_chunks, uint64_t* out,
                                cudaStream_t s) {
    chunk_bounds_kernel<<<1, 64, 0, s>>>(a, pb, k_chunks, out);
    return cudaGetLastError();
}

cudaError_t launch_emit(const ExpandArgs& a, const PlanBufs& pb, const Tuning& tu, cudaStream_t s) {
    if (a.n_tags == 0 || a.capacity == 0) return cudaSuccess;
    if (a.arcs) return launch_emit_arcs<true, false>(a, pb, tu, s);
    return a.refine ? launch_emit_arcs<false, true>(a, pb, tu, s) : launch_emit_arcs<false, false>(a, pb, tu, s);
}

}  // namespace se

namespace se {

// Test hook for the bulk copies' bounded wait: one warp initialises a barrier
// and waits on its first phase.  With copy = 0 nothing is issued, so the phase
// never completes and the wait gives up after `limit` polls (kStatusTimeout);
// with copy = 1 lane 0 copies 256 bytes of `src` (every byte 0x5A) into shared
// memory first, the wait succeeds and the lanes check the bytes (kStatusBadTag
// if they differ).  A copy that has not landed when its wait gives up is drained
// with a second bounded wait before the block exits.
__global__ void bulk_wait_probe_kernel(const uint4* src, uint32_t copy, uint32_t limit, uint32_t* status) {
    __shared__ __align__(16) uint4 s_buf[16];
    __shared__ __align__(8) uint64_t s_bar;
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) bulk_bar_init(&s_bar);
    __syncwarp();
    if (copy && lane == 0) bulk_load(s_buf, src, (uint32_t)sizeof(s_buf), &s_bar);
    if (!bulk_wait(&s_bar, 0u, limit)) {
        if (lane == 0) atomicOr(status, (uint32_t)kStatusTimeout);
        if (copy) bulk_wait(&s_bar, 0u);
        return;
    }
    const uint4 v = s_buf[lane & 15u];
    if (v.x != 0x5a5a5a5au || v.y != 0x5a5a5a5au || v.z != 0x5a5a5a5au || v.w != 0x5a5a5a5au)
        atomicOr(status, (uint32_t)kStatusBadTag);
}

cudaError_t launch_bulk_wait_probe(const void* src, uint32_t copy, uint32_t limit, uint32_t* status, cudaStream_t s) {
    bulk_wait_probe_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const uint4*>(src), copy, limit, status);
    return cudaGetLastError();
}

// Exclusive scan of u32 counts into u64 offsets with caller-supplied scan state
// (used by the entry point that allocates nothing).
cudaError_t launch_offsets_with_state(const uint32_t* counts, uint64_t n, uint64_t* offsets, ScanState st,
                                      uint32_t* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    OffsetOp op;
    op.counts = counts;
    op.offsets = offsets;
    op.total = nullptr;
    lookback_scan<OffsetOp><<<n_tiles(n), kScanThreads, 0, s>>>(op, n, nullptr, st, status);
    return cudaGetLastError();
}

}  // namespace se
