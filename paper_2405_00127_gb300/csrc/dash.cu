// Device dash pass: rewrites a scene whose styles carry dash patterns into a
// solid scene (tags, points, styles) that the expansion then strokes.  Every
// "on" interval of a dashed subpath becomes an open subpath of its own: the
// parts of the source segments it covers, then a cap marker.  Paths without
// a dash pattern are copied unchanged.  Output order follows the input: tag by
// tag, and within a tag along the segment, so the result is deterministic.
//
//   tag scan   (the expansion's tag-monoid scan, on the input tags)
//   len        per tag: FP32 arc length of a dashed segment
//   seg scan   compensated segmented sum of the lengths per subpath
//   count      per tag: output tags and points; marks paths with output
//   out scan   exclusive scan of the counts (+ one empty tag for a path left
//              without output), capacity check, totals
//   write      per tag: the output tags and points
//   fixup      path and style bits on the first / last output tag of each
//              path; copies the styles with the dash pattern removed
#include "dash.cuh"
#include "launch.h"
#include "pipeline.cuh"
#include "scan.cuh"

namespace se {

__global__ void __launch_bounds__(128) dash_len_kernel(DashBufs b) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_tags) return;
    uint32_t flags = 0;
    DashTag d = classify(b, i, flags);
    float L = 0.0f;
    if (d.ok && d.seg && d.dashed && d.pat.valid) {
        Cubic cu = load_seg(b.words, d.tag, d.base);
        L = seg_arc_length(cu);
    }
    b.len[i] = L;
}

// segmented sum of the arc lengths in fixed point (heads: first tag of a subpath)
struct SegLenOp {
    struct T {
        long long v;
        uint32_t head;
        uint32_t pad;
    };
    float* len;
    const uint32_t* sub_first;
    long long* end_pos;

    __device__ __forceinline__ T identity() const {
        T t;
        t.v = 0ll;
        t.head = 0u;
        t.pad = 0u;
        return t;
    }
    __device__ __forceinline__ T combine(T a, T b) const {
        if (b.head) return b;
        T r;
        r.v = a.v + b.v;
        if (r.v > kFixMax) r.v = kFixMax;  // saturate: such a subpath is rejected when walked
        r.head = a.head;
        r.pad = 0u;
        return r;
    }
    __device__ static __forceinline__ T shfl_up(T v, int d) {
        T r;
        r.v = __shfl_up_sync(0xffffffffu, v.v, d);
        r.head = __shfl_up_sync(0xffffffffu, v.head, d);
        r.pad = 0u;
        return r;
    }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i < n) {
                float l = len[i];
                v[k].v = l < 1073741824.0f ? fix_of(l) : kFixMax;
                v[k].head = sub_first[i] == (uint32_t)i ? 1u : 0u;
                v[k].pad = 0u;
            } else {
                v[k] = identity();
            }
        }
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            end_pos[i] = combine(prefix, v[k]).v;
        }
    }
};

__global__ void __launch_bounds__(128) dash_count_kernel(DashBufs b) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_tags) return;
    uint32_t flags = 0;
    uint64_t nt, np, nc;
    dash_tag_count(b, i, nt, np, nc, flags);
    b.cnt[i] = make_uint2((uint32_t)nt, (uint32_t)np);
    b.ncut[i] = (uint32_t)nc;
    if (nt) {
        uint32_t p = b.info.path[i];
        if (p < b.n_paths) atomicOr(&b.nonempty[p], 1u);
    }
    if (flags) atomicOr(b.status, flags);
}

// exclusive scan of the output counts, with one empty tag for every path left without output
struct DashOutOp {
    using T = ulonglong2;
    DashBufs b;

    __device__ __forceinline__ T identity() const { return make_ulonglong2(0ull, 0ull); }
    __device__ __forceinline__ T combine(T a, T c) const { return make_ulonglong2(a.x + c.x, a.y + c.y); }
    __device__ static __forceinline__ T shfl_up(T v, int d) {
        return make_ulonglong2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
    }
    __device__ __forceinline__ bool placeholder(uint64_t i) const {
        if (!(b.tags[i] & SE_TAG_PATH)) return false;
        uint32_t p = b.info.path[i];
        return p < b.n_paths && b.nonempty[p] == 0u;
    }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i < n) {
                uint2 c = b.cnt[i];
                v[k] = make_ulonglong2((unsigned long long)c.x + (placeholder(i) ? 1ull : 0ull), c.y);
            } else {
                v[k] = identity();
            }
        }
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            b.off[i] = combine(prefix, k ? v[k - 1] : identity());
            if (i == n - 1) {
                T in = combine(prefix, v[k]);
                b.off[n] = in;
                bool fits = in.x <= b.cap_tags && in.y <= b.cap_pts && in.x < (1ull << 31) && in.y < (1ull << 32);
                b.out_n[0] = fits ? in.x : 0ull;
                b.out_n[1] = fits ? in.y : 0ull;
                b.out_n[2] = in.x;
                b.out_n[3] = in.y;
                if (!fits) atomicOr(b.status, (uint32_t)kStatusWorkspace);
            }
        }
    }
};

// exclusive scan of the per-tag cut counts and of the cubics that have cuts
// (x: first cut, y: panel slot); over capacity, the rewrite is abandoned (tag
// and point totals zeroed) and reported as a workspace overflow
struct CutScanOp {
    using T = ulonglong2;
    DashBufs b;

    __device__ __forceinline__ T identity() const { return make_ulonglong2(0ull, 0ull); }
    __device__ __forceinline__ T combine(T a, T c) const { return make_ulonglong2(a.x + c.x, a.y + c.y); }
    __device__ static __forceinline__ T shfl_up(T v, int d) {
        return make_ulonglong2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
    }
    __device__ __forceinline__ void load(uint64_t base, uint64_t n, T* v) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint32_t c = (base + k < n) ? b.ncut[base + k] : 0u;
            v[k] = make_ulonglong2((unsigned long long)c, c ? 1ull : 0ull);
        }
    }
    __device__ __forceinline__ void store(uint64_t base, uint64_t n, const T* v, T prefix) const {
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            uint64_t i = base + k;
            if (i >= n) break;
            b.cut_off[i] = combine(prefix, k ? v[k - 1] : identity());
            if (i == n - 1) {
                T in = combine(prefix, v[k]);
                b.cut_off[n] = in;
                b.out_n[4] = in.x;
                b.out_n[5] = in.y;
                if (in.x > b.cap_cuts || in.y > b.cap_slots) {
                    b.out_n[0] = 0ull;
                    b.out_n[1] = 0ull;
                    atomicOr(b.status, (uint32_t)kStatusWorkspace);
                }
            }
        }
    }
};

// One thread per dashed cubic with cuts: its arc-length walk, recorded.
__global__ void __launch_bounds__(128) dash_panel_kernel(DashBufs b) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n_tags || b.out_n[0] == 0ull || b.ncut[i] == 0u || (*b.status & kStatusTimeout)) return;
    uint32_t flags = 0;
    DashTag d = classify(b, i, flags);
    if (!d.ok || !d.seg) return;
    const uint64_t slot = b.cut_off[i].y;
    Cubic cu = load_seg(b.words, d.tag, d.base);
    uint32_t n = 0;
    bool fits = record_panels(cu, b.panels + slot * kPanelMax, n);
    b.n_panels[slot] = fits ? n : (uint32_t)kPanelMax + 1u;
}

// One thread per cut inside a dashed cubic: its parameter, from the segment's
// recorded walk (or a fresh walk when it recorded too many pairs) at the
// cut's canonical position.
__global__ void __launch_bounds__(128) dash_cut_kernel(DashBufs b) {
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = b.out_n[4];
    if (c >= total || b.out_n[0] == 0ull || (*b.status & kStatusTimeout)) return;
    // segment: the largest i with cut_off[i].x <= c
    uint64_t lo = 0, hi = b.n_tags;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (b.cut_off[mid].x <= c) lo = mid;
        else hi = mid;
    }
    const uint64_t i = lo;
    uint32_t flags = 0;
    DashTag d = classify(b, i, flags);
    float t = 1.0f;
    DF z0, z1;
    bool first;
    if (d.ok && d.dashed && d.pat.valid && d.curve && seg_span(b, d.pat, i, z0, z1, first)) {
        const DF zb = dash_kth(d.pat, z0, first, c - b.cut_off[i].x);
        const float s = df_float(df_sub(zb, z0));
        Cubic cu = load_seg(b.words, d.tag, d.base);
        const uint64_t slot = b.cut_off[i].y;
        const uint32_t np = b.n_panels[slot];
        if (np <= (uint32_t)kPanelMax) {
            t = t_from_panels(cu, b.panels + slot * kPanelMax, np, s);
        } else {
            ArcWalk w;
            w.init(cu);
            t = w.t_at(s);
        }
    }
    b.cut_t[c] = t;
}

__global__ void __launch_bounds__(128) dash_write_kernel(DashBufs b) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // offsets from a scan whose wait gave up are not trusted: nothing is written
    if (i >= b.n_tags || (b.out_n[0] == 0ull && b.out_n[2] != 0ull) || (*b.status & kStatusTimeout)) return;
    uint32_t flags = 0;
    dash_tag_write(b, i, b.off[i], b.off[i + 1], flags);
    if (flags) atomicOr(b.status, flags);
}

__device__ __forceinline__ void or_byte(uint8_t* base, uint64_t idx, uint8_t bits) {
    uintptr_t addr = reinterpret_cast<uintptr_t>(base + idx);
    uint32_t* word = reinterpret_cast<uint32_t*>(addr & ~uintptr_t(3));
    atomicOr(word, (uint32_t)bits << (8u * (uint32_t)(addr & 3u)));
}

__global__ void __launch_bounds__(128) dash_fixup_kernel(DashBufs b) {
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.n_styles) {
        se_style st = b.styles[i];
        st.dash_first = 0u;
        st.dash_count = 0u;
        st.dash_offset = 0.0f;
        b.out_styles[i] = st;
    }
    if (i >= b.n_tags || (b.out_n[0] == 0ull && b.out_n[2] != 0ull)) return;
    uint8_t t = b.tags[i];
    ulonglong2 o = b.off[i], o1 = b.off[i + 1];
    const uint8_t head = (uint8_t)(t & (SE_TAG_STYLE | SE_TAG_TRANSFORM));
    if (head && o.x < b.out_n[0]) or_byte(b.out_tags, o.x, head);
    if ((t & SE_TAG_PATH) && o1.x > 0ull && o1.x <= b.out_n[0]) or_byte(b.out_tags, o1.x - 1, (uint8_t)SE_TAG_PATH);
}

static uint32_t blocks_of(uint64_t n, uint32_t t) { return (uint32_t)((n + t - 1) / t); }

// The dash pass on the stream: the caller has cleared `nonempty`, the scan
// states and the status word.  seg_state / out_state: look-back states for the
// two scans (16-byte tile slots).
cudaError_t launch_dash(const DashBufs& b, ScanState tag_state, ScanState seg_state, ScanState out_state,
                        ScanState cut_state, cudaStream_t s) {
    if (b.n_tags == 0) return cudaSuccess;
    cudaError_t e = launch_tag_scan(b.tags, b.n_tags, nullptr, b.info, tag_state, b.status, s);
    if (e != cudaSuccess) return e;
    uint32_t g = blocks_of(b.n_tags, 128);
    dash_len_kernel<<<g, 128, 0, s>>>(b);
    SegLenOp sop;
    sop.len = b.len;
    sop.sub_first = b.info.sub_first;
    sop.end_pos = b.end_pos;
    uint32_t tiles = (uint32_t)((b.n_tags + kScanTile - 1) / kScanTile);
    lookback_scan<SegLenOp><<<tiles, kScanThreads, 0, s>>>(sop, b.n_tags, nullptr, seg_state, b.status);
    dash_count_kernel<<<g, 128, 0, s>>>(b);
    DashOutOp oop;
    oop.b = b;
    lookback_scan<DashOutOp><<<tiles, kScanThreads, 0, s>>>(oop, b.n_tags, nullptr, out_state, b.status);
    CutScanOp cop;
    cop.b = b;
    lookback_scan<CutScanOp><<<tiles, kScanThreads, 0, s>>>(cop, b.n_tags, nullptr, cut_state, b.status);
    dash_panel_kernel<<<g, 128, 0, s>>>(b);
    if (b.cap_cuts) dash_cut_kernel<<<blocks_of(b.cap_cuts, 128), 128, 0, s>>>(b);
    dash_write_kernel<<<g, 128, 0, s>>>(b);
    uint64_t nf = b.n_tags > b.n_styles ? b.n_tags : b.n_styles;
    dash_fixup_kernel<<<blocks_of(nf, 128), 128, 0, s>>>(b);
    return cudaGetLastError();
}

}  // namespace se
