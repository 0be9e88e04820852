// Nonzero-rule coverage of an expanded outline on a pixel grid: the downstream
// use of the line soup (Section 8.1, whose renderer bins the soup into tiles
// and computes coverage with scanlines), here as a check and a consumer of the
// library's own output.
//
// For every path and every pixel centre (x + 1/2, y + 1/2) of a W x H grid the
// winding number of the path's primitives is the signed count of crossings of
// the centre's row to its left; a pixel is covered by the path when that is
// nonzero.  The result is, per pixel, the number of paths covering it, and per
// path the number of pixels it covers.
//
// Work is organised by (path, row) buckets -- the scanline form of tile
// binning, one row of pixels per bin:
//   bounds   rows each path's primitives cross (atomic min / max per path)
//   scan     bucket base per path
//   count    crossings per bucket
//   scan     crossing offsets per bucket
//   scatter  crossing records (x, direction) into their buckets
//   spans    per bucket: sort by x, accumulate the winding, add the covered
//            pixel runs to the image and the path's area
// Arcs are cut into equal-angle chords of sagitta at most 1e-3 px.  Every
// per-pixel value is an integer sum, so the image does not depend on the order
// of the atomic additions.
#include <cuda_runtime.h>

#include <climits>

#include "ctx.h"
#include "scan.cuh"

namespace se {

cudaError_t launch_offsets_with_state(const uint32_t* counts, uint64_t n, uint64_t* offsets, ScanState st,
                                      uint32_t* status, cudaStream_t s);

namespace {

constexpr float kArcFlat = 1e-3f;   // chord sagitta for arcs, pixels
constexpr int kMaxArcChords = 1024;
constexpr int kCovThreads = 256;

struct CovArgs {
    const float4* prims;
    const float* curv;      // NULL: lines
    const uint32_t* path_id;
    uint64_t n;
    uint32_t n_paths;
    uint32_t W, H;
    int* row_lo;            // per path
    int* row_hi;
    uint32_t* rows;         // per path: rows spanned (scan input)
    uint64_t* bucket_base;  // per path + 1
    uint32_t* bucket_cnt;   // per bucket
    uint32_t* bucket_cur;
    uint64_t* bucket_off;   // per bucket + 1
    float* cx;              // per crossing
    int8_t* cdir;
    uint32_t* count;        // W * H
    unsigned long long* area;  // per path (may be NULL)
    uint32_t* status;
};

// Chords of a primitive: a line is one; an arc of signed curvature k from A to B
// (its centre to the left of A -> B when k > 0) turns by 2 half, half =
// asin(c |k| / 2) for chord length c, and is cut into n equal-angle chords of
// sagitta at most kArcFlat (r theta^2 / 8 bounds the sagitta of a chord turning
// by theta).  Vertex j lies at distance c sin(phi / 2) / sin(half) from A in the
// direction of the chord turned by sgn (phi / 2 - half), phi = 2 half j / n: no
// centre or radius enters, so a nearly straight arc stays exact to FP32.
struct ArcChords {
    float2 a, b, u;  // u: unit chord direction
    float c, half, sgn, s_half;
    int n;
};

__device__ ArcChords arc_chords(float4 p, float k) {
    ArcChords ac;
    ac.a = make_float2(p.x, p.y);
    ac.b = make_float2(p.z, p.w);
    ac.n = 1;
    const float dx = p.z - p.x, dy = p.w - p.y;
    ac.c = sqrtf(dx * dx + dy * dy);
    if (k == 0.0f || !(ac.c > 0.0f) || !isfinite(k)) return ac;
    ac.u = make_float2(dx / ac.c, dy / ac.c);
    ac.half = asinf(fminf(1.0f, 0.5f * ac.c * fabsf(k)));
    ac.sgn = k > 0.0f ? 1.0f : -1.0f;
    ac.s_half = sinf(ac.half);
    const float theta = sqrtf(8.0f * kArcFlat * fabsf(k));
    const float nf = ceilf(2.0f * ac.half / theta);
    ac.n = nf < 1.0f ? 1 : (nf > (float)kMaxArcChords ? kMaxArcChords : (int)nf);
    if (!(ac.s_half > 0.0f)) ac.n = 1;
    return ac;
}

__device__ float2 arc_vertex(const ArcChords& ac, int j) {
    if (j == 0) return ac.a;
    if (j == ac.n) return ac.b;
    const float phi = 2.0f * ac.half * ((float)j / (float)ac.n);
    const float len = ac.c * (sinf(0.5f * phi) / ac.s_half);
    float sn, cs;
    sincosf(ac.sgn * (0.5f * phi - ac.half), &sn, &cs);
    return make_float2(ac.a.x + len * (ac.u.x * cs - ac.u.y * sn), ac.a.y + len * (ac.u.x * sn + ac.u.y * cs));
}

// Rows r in [0, H) whose centre line y = r + 1/2 the chord a -> b crosses, with
// the half-open rule lo <= r + 1/2 < hi (a vertex shared by two chords counts
// once where the path passes through it and twice or not at all at an extremum).
__device__ bool chord_rows(float2 a, float2 b, uint32_t H, int& r0, int& r1) {
    const float lo = fminf(a.y, b.y), hi = fmaxf(a.y, b.y);
    if (!(lo < hi) || !isfinite(lo) || !isfinite(hi)) return false;
    if (hi <= 0.5f || lo >= (float)H - 0.5f + 1.0f) return false;
    float f0 = ceilf(lo - 0.5f), f1 = ceilf(hi - 0.5f) - 1.0f;
    f0 = fmaxf(f0, 0.0f);
    f1 = fminf(f1, (float)H - 1.0f);
    if (f0 > f1) return false;
    r0 = (int)f0;
    r1 = (int)f1;
    while (r0 <= r1 && (float)r0 + 0.5f < lo) r0++;
    while (r1 >= r0 && !((float)r1 + 0.5f < hi)) r1--;
    return r0 <= r1;
}

__device__ float cross_x(float2 a, float2 b, int r) {
    const float yr = (float)r + 0.5f;
    return a.x + (yr - a.y) / (b.y - a.y) * (b.x - a.x);
}

template <class F>
__device__ void for_chords(const CovArgs& A, uint64_t i, F f) {
    const float4 p = A.prims[i];
    const float k = A.curv ? A.curv[i] : 0.0f;
    const ArcChords ac = arc_chords(p, k);
    float2 prev = ac.a;
    for (int j = 1; j <= ac.n; j++) {
        const float2 cur = arc_vertex(ac, j);
        f(prev, cur);
        prev = cur;
    }
}

__global__ void __launch_bounds__(kCovThreads) cov_init(CovArgs A) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.n_paths) {
        A.row_lo[i] = INT_MAX;
        A.row_hi[i] = -1;
    }
}

__global__ void __launch_bounds__(kCovThreads) cov_bounds(CovArgs A) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const uint32_t p = A.path_id[i];
    if (p >= A.n_paths) {
        atomicOr(A.status, (uint32_t)kStatusBadTag);
        return;
    }
    int lo = INT_MAX, hi = -1;
    for_chords(A, i, [&](float2 a, float2 b) {
        int r0, r1;
        if (chord_rows(a, b, A.H, r0, r1)) {
            lo = min(lo, r0);
            hi = max(hi, r1);
        }
    });
    if (hi >= 0) {
        atomicMin(&A.row_lo[p], lo);
        atomicMax(&A.row_hi[p], hi);
    }
}

__global__ void __launch_bounds__(kCovThreads) cov_rows(CovArgs A) {
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.n_paths) return;
    const int lo = A.row_lo[p], hi = A.row_hi[p];
    A.rows[p] = hi >= lo ? (uint32_t)(hi - lo + 1) : 0u;
}

__global__ void __launch_bounds__(kCovThreads) cov_count(CovArgs A) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const uint32_t p = A.path_id[i];
    if (p >= A.n_paths) return;
    const uint64_t base = A.bucket_base[p];
    const int lo = A.row_lo[p];
    for_chords(A, i, [&](float2 a, float2 b) {
        int r0, r1;
        if (!chord_rows(a, b, A.H, r0, r1)) return;
        for (int r = r0; r <= r1; r++) atomicAdd(&A.bucket_cnt[base + (uint64_t)(r - lo)], 1u);
    });
}

__global__ void __launch_bounds__(kCovThreads) cov_scatter(CovArgs A) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const uint32_t p = A.path_id[i];
    if (p >= A.n_paths) return;
    const uint64_t base = A.bucket_base[p];
    const int lo = A.row_lo[p];
    for_chords(A, i, [&](float2 a, float2 b) {
        int r0, r1;
        if (!chord_rows(a, b, A.H, r0, r1)) return;
        const int8_t dir = b.y > a.y ? (int8_t)1 : (int8_t)-1;
        for (int r = r0; r <= r1; r++) {
            const uint64_t bk = base + (uint64_t)(r - lo);
            const uint64_t slot = A.bucket_off[bk] + atomicAdd(&A.bucket_cur[bk], 1u);
            A.cx[slot] = cross_x(a, b, r);
            A.cdir[slot] = dir;
        }
    });
}

// largest path p with bucket_base[p] <= b
__device__ uint32_t bucket_path(const CovArgs& A, uint64_t b) {
    uint32_t lo = 0, hi = A.n_paths;
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (A.bucket_base[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ bool before(float xa, int8_t da, float xb, int8_t db) { return xa < xb || (xa == xb && da < db); }

__global__ void __launch_bounds__(kCovThreads) cov_spans(CovArgs A, uint64_t n_buckets) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_buckets) return;
    const uint64_t o0 = A.bucket_off[b], o1 = A.bucket_off[b + 1];
    if (o1 == o0) return;
    float* x = A.cx + o0;
    int8_t* d = A.cdir + o0;
    const int64_t n = (int64_t)(o1 - o0);
    // sort by (x, direction): Shell sort with gaps 3h + 1, insertion sort for short runs
    int64_t gap = 1;
    while (gap < n / 3) gap = 3 * gap + 1;
    for (; gap >= 1; gap /= 3) {
        for (int64_t i = gap; i < n; i++) {
            const float xv = x[i];
            const int8_t dv = d[i];
            int64_t j = i;
            while (j >= gap && before(xv, dv, x[j - gap], d[j - gap])) {
                x[j] = x[j - gap];
                d[j] = d[j - gap];
                j -= gap;
            }
            x[j] = xv;
            d[j] = dv;
        }
    }
    const uint32_t p = bucket_path(A, b);
    const int row = A.row_lo[p] + (int)(b - A.bucket_base[p]);
    uint32_t* img = A.count + (uint64_t)row * A.W;
    unsigned long long covered = 0;
    int w = 0;
    for (int64_t k = 0; k + 1 < n; k++) {
        w += d[k];
        if (w == 0) continue;
        // pixels whose centre lies in [x_k, x_{k+1})
        float f0 = fmaxf(ceilf(x[k] - 0.5f), 0.0f), f1 = fminf(ceilf(x[k + 1] - 0.5f), (float)A.W);
        if (!(f0 < f1)) continue;
        int j0 = (int)f0, j1 = (int)f1;
        while (j0 < j1 && (float)j0 + 0.5f < x[k]) j0++;
        while (j1 > j0 && !((float)(j1 - 1) + 0.5f < x[k + 1])) j1--;
        for (int j = j0; j < j1; j++) atomicAdd(&img[j], 1u);
        covered += (unsigned long long)(j1 - j0);
    }
    if (A.area && covered) atomicAdd(&A.area[p], covered);
}

uint32_t grid_of(uint64_t n) { return (uint32_t)((n + kCovThreads - 1) / kCovThreads); }

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace se

using namespace se;

extern "C" se_status se_coverage(se_ctx* c, const float* prims, const float* curvature, const uint32_t* path_id,
                                 uint64_t n_prims, uint32_t n_paths, uint32_t width, uint32_t height,
                                 uint32_t* count, uint64_t* path_area) {
    if (!c || !count || (n_prims && (!prims || !path_id)) || width == 0 || height == 0) return SE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(prims) & 15u) != 0) return se_fail(c, SE_ERR_INVALID_ARG, "prims must be 16-byte aligned");
    if ((uint64_t)width * height >= (1ull << 40)) return se_fail(c, SE_ERR_INVALID_ARG, "grid too large");
    settle_pending(c);
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)width * height * 4, s);
    if (e == cudaSuccess && path_area && n_paths) e = cudaMemsetAsync(path_area, 0, (size_t)n_paths * 8, s);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "coverage clear", e);
    if (n_prims == 0 || n_paths == 0) return cudaStreamSynchronize(s) == cudaSuccess ? SE_OK : SE_ERR_CUDA;

    // per-path stage: bounds, rows, bucket bases (+ scan state and status)
    const uint64_t tp = (n_paths + 1 + kScanTile - 1) / kScanTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = al256(off + bytes);
        return o;
    };
    size_t o_lo = take(n_paths * 4ull), o_hi = take(n_paths * 4ull), o_rows = take((n_paths + 1ull) * 4);
    size_t o_base = take((n_paths + 1ull) * 8), o_ctl = take((4 + tp) * 4), o_agg = take(tp * 8), o_incl = take(tp * 8);
    void* m1 = nullptr;
    e = cudaMallocAsync(&m1, off, s);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_OOM, "coverage workspace", e);
    char* b1 = static_cast<char*>(m1);
    CovArgs A{};
    A.prims = reinterpret_cast<const float4*>(prims);
    A.curv = curvature;
    A.path_id = path_id;
    A.n = n_prims;
    A.n_paths = n_paths;
    A.W = width;
    A.H = height;
    A.row_lo = reinterpret_cast<int*>(b1 + o_lo);
    A.row_hi = reinterpret_cast<int*>(b1 + o_hi);
    A.rows = reinterpret_cast<uint32_t*>(b1 + o_rows);
    A.bucket_base = reinterpret_cast<uint64_t*>(b1 + o_base);
    uint32_t* ctl = reinterpret_cast<uint32_t*>(b1 + o_ctl);
    A.status = ctl;
    A.count = count;
    A.area = reinterpret_cast<unsigned long long*>(path_area);
    ScanState st{ctl + 4, b1 + o_agg, b1 + o_incl, ctl + 1};
    void* m2 = nullptr;
    se_status result = SE_OK;
    uint64_t nb = 0, ncross = 0;
    uint32_t h_status = 0;
    e = cudaMemsetAsync(ctl, 0, (4 + tp) * 4, s);
    if (e == cudaSuccess) {
        cov_init<<<grid_of(n_paths), kCovThreads, 0, s>>>(A);
        cov_bounds<<<grid_of(n_prims), kCovThreads, 0, s>>>(A);
        cov_rows<<<grid_of(n_paths), kCovThreads, 0, s>>>(A);
        e = launch_offsets_with_state(A.rows, n_paths, A.bucket_base, st, A.status, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, A.bucket_base + n_paths, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeAsync(m1, s);
        return se_fail(c, SE_ERR_CUDA, "coverage bounds", e);
    }
    // per-bucket stage
    const uint64_t tb = (nb + 1 + kScanTile - 1) / kScanTile;
    off = 0;
    size_t o_cnt = take((nb + 1) * 4), o_cur = take((nb + 1) * 4), o_boff = take((nb + 1) * 8);
    size_t o_ctl2 = take((4 + tb) * 4), o_agg2 = take(tb * 8), o_incl2 = take(tb * 8);
    size_t part = off;
    e = cudaMallocAsync(&m2, part, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(m1, s);
        return se_fail(c, SE_ERR_OOM, "coverage buckets", e);
    }
    char* b2 = static_cast<char*>(m2);
    A.bucket_cnt = reinterpret_cast<uint32_t*>(b2 + o_cnt);
    A.bucket_cur = reinterpret_cast<uint32_t*>(b2 + o_cur);
    A.bucket_off = reinterpret_cast<uint64_t*>(b2 + o_boff);
    uint32_t* ctl2 = reinterpret_cast<uint32_t*>(b2 + o_ctl2);
    ScanState st2{ctl2 + 4, b2 + o_agg2, b2 + o_incl2, ctl2 + 1};
    e = cudaMemsetAsync(b2, 0, part, s);
    if (e == cudaSuccess && nb) {
        cov_count<<<grid_of(n_prims), kCovThreads, 0, s>>>(A);
        e = launch_offsets_with_state(A.bucket_cnt, nb, A.bucket_off, st2, A.status, s);
    }
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(&ncross, A.bucket_off + nb, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    void* m3 = nullptr;
    if (e == cudaSuccess && ncross) {
        e = cudaMallocAsync(&m3, al256(ncross * 4) + ncross + 16, s);
        if (e == cudaSuccess) {
            A.cx = static_cast<float*>(m3);
            A.cdir = reinterpret_cast<int8_t*>(static_cast<char*>(m3) + al256(ncross * 4));
            cov_scatter<<<grid_of(n_prims), kCovThreads, 0, s>>>(A);
            cov_spans<<<grid_of(nb), kCovThreads, 0, s>>>(A, nb);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, A.status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (m3) cudaFreeAsync(m3, s);
    cudaFreeAsync(m2, s);
    cudaFreeAsync(m1, s);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "coverage", e);
    if (h_status & kStatusTimeout) result = se_fail(c, SE_ERR_TIMEOUT, "coverage scan wait gave up");
    else if (h_status & kStatusBadTag) result = se_fail(c, SE_ERR_INVALID_INPUT, "a path id is out of range");
    return result;
}
