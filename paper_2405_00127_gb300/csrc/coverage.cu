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
//   paths    the path of each bucket
//   count    crossings per bucket
//   scan     crossing offsets per bucket
//   scatter  crossing records (x, direction) into their buckets
//   spans    per bucket: sort by x, accumulate the winding, add each covered
//            pixel run to the image as a difference (+1 at its first pixel,
//            -1 past its last) and its length to the path's area; one thread
//            per bucket of up to 16 crossings (a sorting network in registers),
//            one warp per bucket of up to 32 (a sort across the lanes), one
//            warp per larger one (a column histogram in place of the sort), one
//            block per bucket wider than the histogram
//   rowscan  per row: prefix sum of the differences, giving the counts
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
    uint32_t* bucket_path_id;  // per bucket: its path
    uint32_t* bucket_cnt;   // per bucket
    uint32_t* bucket_cur;
    uint64_t* bucket_off;   // per bucket + 1
    float* cx;              // per crossing
    int8_t* cdir;
    uint32_t* wl;           // buckets of kSmallMax + 1 (17) to 32 crossings (their ids)
    uint32_t* n_wl;         // their count
    uint32_t* mid;          // buckets of more than 32 crossings
    uint32_t* n_mid;
    uint32_t* big;          // of those, the buckets wider than kHistCap columns
    uint32_t* n_big;
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

// Row bounds per path.  Neighbouring primitives mostly belong to one path, so
// the lanes of a warp first combine their bounds with the lanes of the same path
// (a segmented min / max over shuffles; only lanes of equal path id are combined,
// which is correct in any order) and only the first lane of each run of equal
// ids updates the path's bounds: one pair of atomics per run instead of per lane.
__global__ void __launch_bounds__(kCovThreads) cov_bounds(CovArgs A) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t p = 0xffffffffu;  // no path: combines with nothing
    int lo = INT_MAX, hi = -1;
    if (i < A.n) {
        p = A.path_id[i];
        if (p >= A.n_paths) {
            atomicOr(A.status, (uint32_t)kStatusBadTag);
            p = 0xffffffffu;
        } else {
            for_chords(A, i, [&](float2 a, float2 b) {
                int r0, r1;
                if (chord_rows(a, b, A.H, r0, r1)) {
                    lo = min(lo, r0);
                    hi = max(hi, r1);
                }
            });
        }
    }
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const uint32_t pn = __shfl_down_sync(0xffffffffu, p, d);
        const int lon = __shfl_down_sync(0xffffffffu, lo, d);
        const int hin = __shfl_down_sync(0xffffffffu, hi, d);
        if (lane + d < 32u && pn == p) {
            lo = min(lo, lon);
            hi = max(hi, hin);
        }
    }
    const uint32_t pp = __shfl_up_sync(0xffffffffu, p, 1);
    const bool first = lane == 0u || pp != p;
    if (first && p != 0xffffffffu && hi >= 0) {
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

// The path of every bucket, one warp per path (its lanes stride over the path's rows).
__global__ void __launch_bounds__(kCovThreads) cov_bucket_paths(CovArgs A) {
    const uint64_t p = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= A.n_paths) return;
    const uint64_t b1 = A.bucket_base[p + 1];
    for (uint64_t b = A.bucket_base[p] + (threadIdx.x & 31u); b < b1; b += 32) A.bucket_path_id[b] = (uint32_t)p;
}

__device__ bool before(float xa, int8_t da, float xb, int8_t db) { return xa < xb || (xa == xb && da < db); }

// The first pixel column whose centre c + 1/2 is at or right of x, clamped to
// [0, W]: a crossing at x counts toward the winding of columns col_of(x) on.
__device__ __forceinline__ int col_of(float x, uint32_t W) {
    int c = (int)fminf(fmaxf(ceilf(x - 0.5f), 0.0f), (float)W);
    while (c < (int)W && (float)c + 0.5f < x) c++;
    while (c > 0 && (float)(c - 1) + 0.5f >= x) c--;
    return c;
}

__device__ __forceinline__ uint32_t* bucket_row(const CovArgs& A, uint64_t b, uint32_t& p) {
    p = A.bucket_path_id[b];
    const int row = A.row_lo[p] + (int)(b - A.bucket_base[p]);
    return A.count + (uint64_t)row * A.W;
}

// A covered run [j0, j1) of an image row, as a difference: +1 at j0, -1 at j1
// (the row scan sums it).
__device__ __forceinline__ void add_run(const CovArgs& A, uint32_t* img, int j0, int j1) {
    atomicAdd(&img[j0], 1u);
    if ((uint32_t)j1 < A.W) atomicAdd(&img[j1], 0xffffffffu);
}

// Small buckets, one thread each (most buckets hold a few crossings): the
// thread loads the bucket's crossings into registers at once (padded with +inf)
// and sorts them with a fixed network of 63 compare-exchanges (Batcher's
// odd-even merge sort of 16), so no step waits on a dependent memory access.  A
// bucket of more crossings goes on the list for cov_spans_warp (up to 32) or for
// cov_spans_mid.
constexpr int kSmallMax = 16;

__device__ __forceinline__ void cex(float* x, int* d, int i, int j) {
    if (before(x[j], (int8_t)d[j], x[i], (int8_t)d[i])) {
        const float tx = x[i];
        const int td = d[i];
        x[i] = x[j];
        d[i] = d[j];
        x[j] = tx;
        d[j] = td;
    }
}

__global__ void __launch_bounds__(kCovThreads) cov_spans(CovArgs A, uint64_t n_buckets) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_buckets) return;
    const uint64_t o0 = A.bucket_off[b], o1 = A.bucket_off[b + 1];
    if (o1 == o0) return;
    if (o1 - o0 > 32u) {
        A.mid[atomicAdd(A.n_mid, 1u)] = (uint32_t)b;
        return;
    }
    const int n = (int)(o1 - o0);
    if (n > kSmallMax) {
        A.wl[atomicAdd(A.n_wl, 1u)] = (uint32_t)b;
        return;
    }
    float x[kSmallMax];
    int d[kSmallMax];
#pragma unroll
    for (int k = 0; k < kSmallMax; k++) {
        x[k] = k < n ? A.cx[o0 + k] : INFINITY;
        d[k] = k < n ? (int)A.cdir[o0 + k] : 0;
    }
    // Batcher's odd-even merge sort of 16: 63 compare-exchanges
    constexpr int kNet16[63][2] = {
        {0, 1}, {2, 3}, {0, 2}, {1, 3}, {1, 2}, {4, 5}, {6, 7}, {4, 6},
        {5, 7}, {5, 6}, {0, 4}, {2, 6}, {2, 4}, {1, 5}, {3, 7}, {3, 5},
        {1, 2}, {3, 4}, {5, 6}, {8, 9}, {10, 11}, {8, 10}, {9, 11}, {9, 10},
        {12, 13}, {14, 15}, {12, 14}, {13, 15}, {13, 14}, {8, 12}, {10, 14}, {10, 12},
        {9, 13}, {11, 15}, {11, 13}, {9, 10}, {11, 12}, {13, 14}, {0, 8}, {4, 12},
        {4, 8}, {2, 10}, {6, 14}, {6, 10}, {2, 4}, {6, 8}, {10, 12}, {1, 9},
        {5, 13}, {5, 9}, {3, 11}, {7, 15}, {7, 11}, {3, 5}, {7, 9}, {11, 13},
        {1, 2}, {3, 4}, {5, 6}, {7, 8}, {9, 10}, {11, 12}, {13, 14}};
#pragma unroll
    for (int c = 0; c < 63; c++) cex(x, d, kNet16[c][0], kNet16[c][1]);
    uint32_t p;
    uint32_t* img = bucket_row(A, b, p);
    unsigned long long covered = 0;
    int w = 0;
#pragma unroll
    for (int k = 0; k + 1 < kSmallMax; k++) {
        w += d[k];
        if (k + 1 < n && w != 0) {
            const int j0 = col_of(x[k], A.W), j1 = col_of(x[k + 1], A.W);
            if (j0 < j1) {
                add_run(A, img, j0, j1);
                covered += (unsigned long long)(j1 - j0);
            }
        }
    }
    if (A.area && covered) atomicAdd(&A.area[p], covered);
}

// Buckets of kSmallMax + 1 to 32 crossings, one warp each (a persistent grid
// walks the list), one crossing per lane: a bitonic sort across the lanes with
// shuffles (lanes past the bucket hold +inf), a warp scan of the directions for
// the winding after each crossing, and lane k writes the run of columns from
// col_of(x_k) up to col_of(x_k+1).
constexpr int kWarpThreads = 256;

__global__ void __launch_bounds__(kWarpThreads) cov_spans_warp(CovArgs A) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t n_wl = *A.n_wl;
    const uint32_t n_warps = gridDim.x * (kWarpThreads / 32);
    for (uint32_t q = blockIdx.x * (kWarpThreads / 32) + (threadIdx.x >> 5); q < n_wl; q += n_warps) {
        const uint64_t b = A.wl[q];
        const uint64_t o0 = A.bucket_off[b];
        const uint32_t n = (uint32_t)(A.bucket_off[b + 1] - o0);
        float x = lane < n ? A.cx[o0 + lane] : INFINITY;
        int d = lane < n ? (int)A.cdir[o0 + lane] : 0;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const float ox = __shfl_xor_sync(0xffffffffu, x, j);
                const int od = __shfl_xor_sync(0xffffffffu, d, j);
                // the lower lane of a pair keeps the smaller key in ascending runs
                const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
                const bool take = keep_min ? before(ox, (int8_t)od, x, (int8_t)d) : before(x, (int8_t)d, ox, (int8_t)od);
                if (take) {
                    x = ox;
                    d = od;
                }
            }
        }
        int w = d;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        const float xn = __shfl_down_sync(0xffffffffu, x, 1);
        uint32_t p;
        uint32_t* img = bucket_row(A, b, p);
        unsigned long long covered = 0;
        if (lane + 1 < n && w != 0) {
            const int j0 = col_of(x, A.W), j1 = col_of(xn, A.W);
            if (j0 < j1) {
                add_run(A, img, j0, j1);
                covered = (unsigned long long)(j1 - j0);
            }
        }
        if (A.area) {
            for (uint32_t o = 16; o > 0; o >>= 1) covered += __shfl_down_sync(0xffffffffu, covered, o);
            if (lane == 0 && covered) atomicAdd(&A.area[p], covered);
        }
    }
}

// Buckets of more than 32 crossings, one warp each (a persistent grid walks the
// list), without a sort: the winding of column c is the sum of the directions of the crossings
// with col_of(x) <= c, so the warp bins the crossings by column into a histogram
// in shared memory over the bucket's column range [c_lo, c_hi) (from the first
// to the last crossing's column), takes its running sum and writes every run of
// nonzero columns.  A bucket wider than kHistCap columns goes on the list for
// cov_spans_big.
constexpr int kMidThreads = 256;
constexpr int kHistCap = 1024;

__global__ void __launch_bounds__(kMidThreads) cov_spans_mid(CovArgs A) {
    __shared__ int s_hist[kMidThreads / 32][kHistCap];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    int* hist = s_hist[wib];
    const uint32_t n_mid = *A.n_mid;
    const uint32_t n_warps = gridDim.x * (kMidThreads / 32);
    for (uint32_t q = blockIdx.x * (kMidThreads / 32) + wib; q < n_mid; q += n_warps) {
        const uint64_t b = A.mid[q];
        const uint64_t o0 = A.bucket_off[b];
        const uint32_t n = (uint32_t)(A.bucket_off[b + 1] - o0);
        int c_lo = INT_MAX, c_hi = 0;
        for (uint32_t k = lane; k < n; k += 32) {
            const int c = col_of(A.cx[o0 + k], A.W);
            c_lo = min(c_lo, c);
            c_hi = max(c_hi, c);
        }
        c_lo = __reduce_min_sync(0xffffffffu, c_lo);
        c_hi = __reduce_max_sync(0xffffffffu, c_hi);
        const int width = c_hi - c_lo;
        if (width <= 0) continue;
        if (width > kHistCap) {
            if (lane == 0) A.big[atomicAdd(A.n_big, 1u)] = (uint32_t)b;
            continue;
        }
        for (int c = (int)lane; c < width; c += 32) hist[c] = 0;
        __syncwarp();
        for (uint32_t k = lane; k < n; k += 32) {
            const int c = col_of(A.cx[o0 + k], A.W);
            if (c < c_hi) atomicAdd(&hist[c - c_lo], (int)A.cdir[o0 + k]);
        }
        __syncwarp();
        int carry = 0;
        for (int base = 0; base < width; base += 32) {
            const int c = base + (int)lane;
            int w = c < width ? hist[c] : 0;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            w += carry;
            if (c < width) hist[c] = w;
            carry = __shfl_sync(0xffffffffu, w, 31);
        }
        __syncwarp();
        uint32_t p;
        uint32_t* img = bucket_row(A, b, p);
        unsigned long long covered = 0;
        for (int c = (int)lane; c < width; c += 32) {
            if (hist[c] == 0) continue;
            covered++;
            // the ends of runs of nonzero columns, as in add_run
            if (c == 0 || hist[c - 1] == 0) atomicAdd(&img[c_lo + c], 1u);
            if ((c + 1 == width || hist[c + 1] == 0) && (uint32_t)(c_lo + c + 1) < A.W)
                atomicAdd(&img[c_lo + c + 1], 0xffffffffu);
        }
        if (A.area) {
            for (uint32_t o = 16; o > 0; o >>= 1) covered += __shfl_down_sync(0xffffffffu, covered, o);
            if (lane == 0 && covered) atomicAdd(&A.area[p], covered);
        }
        __syncwarp();  // the next bucket rewrites the histogram
    }
}

// The widest buckets, one block each (a persistent grid walks the list).  The
// block sorts the bucket with a bitonic network whose compare-exchanges all run
// ascending (each merge starts by comparing element i of a block of k with
// element k - 1 - i), so the pairs that reach past n -- a virtual +inf padding up
// to the power of two -- never exchange and are skipped.  The bucket is sorted
// in shared memory when it holds at most kBigCap crossings and in place in
// global memory otherwise.  A block scan of the directions then gives the
// winding after every crossing, and each thread writes the runs of the gaps it
// owns (the columns from col_of(x_k) up to col_of(x_k+1) have the winding after
// crossing k).
constexpr int kBigThreads = 256;
constexpr int kBigCap = 8192;

__device__ __forceinline__ void bitonic_sort(float* x, int8_t* d, uint32_t n) {
    uint32_t N = 1;
    while (N < n && N < 0x80000000u) N <<= 1;  // n < 2^31: the host checks the crossing total
    for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j >= 1; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                uint32_t lo, hi;
                if (j == (k >> 1)) {  // the merge's first step: mirror pairs
                    const uint32_t off = i & (j - 1);
                    lo = (i / j) * k + off;
                    hi = (i / j) * k + k - 1 - off;
                } else {
                    lo = (i / j) * 2 * j + (i & (j - 1));
                    hi = lo + j;
                }
                if (hi < n && before(x[hi], d[hi], x[lo], d[lo])) {
                    const float tx = x[lo];
                    const int8_t td = d[lo];
                    x[lo] = x[hi];
                    d[lo] = d[hi];
                    x[hi] = tx;
                    d[hi] = td;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void big_spans(const CovArgs& A, uint64_t b, float* x, int8_t* d, uint32_t n,
                                          int* s_scan, unsigned long long* s_area) {
    bitonic_sort(x, d, n);
    uint32_t p;
    uint32_t* img = bucket_row(A, b, p);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    unsigned long long covered = 0;
    int carry = 0;
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t k = base + tid;
        int incl = k < n ? (int)d[k] : 0;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31u) s_scan[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < (blockDim.x >> 5) ? s_scan[lane] : 0;
#pragma unroll
            for (uint32_t o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            if (lane < (blockDim.x >> 5)) s_scan[lane] = w;
        }
        __syncthreads();
        const int w = carry + (warp ? s_scan[warp - 1] : 0) + incl;  // winding after crossing k
        const int tile_total = s_scan[(blockDim.x >> 5) - 1];
        if (k + 1 < n && w != 0) {
            const int j0 = col_of(x[k], A.W), j1 = col_of(x[k + 1], A.W);
            if (j0 < j1) {
                add_run(A, img, j0, j1);
                covered += (unsigned long long)(j1 - j0);
            }
        }
        carry += tile_total;
        __syncthreads();  // s_scan is rewritten by the next tile
    }
    if (A.area) {
        for (uint32_t o = 16; o > 0; o >>= 1) covered += __shfl_down_sync(0xffffffffu, covered, o);
        if (lane == 0 && covered) atomicAdd(s_area, covered);
        __syncthreads();
        if (tid == 0 && *s_area) atomicAdd(&A.area[p], *s_area);
    }
}

__global__ void __launch_bounds__(kBigThreads) cov_spans_big(CovArgs A) {
    __shared__ float s_x[kBigCap];
    __shared__ int8_t s_d[kBigCap];
    __shared__ int s_scan[kBigThreads / 32];
    __shared__ unsigned long long s_area;
    const uint32_t n_big = *A.n_big;
    for (uint32_t q = blockIdx.x; q < n_big; q += gridDim.x) {
        const uint64_t b = A.big[q];
        const uint64_t o0 = A.bucket_off[b];
        const uint32_t n = (uint32_t)(A.bucket_off[b + 1] - o0);
        if (threadIdx.x == 0) s_area = 0;
        if (n <= (uint32_t)kBigCap) {
            for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
                s_x[k] = A.cx[o0 + k];
                s_d[k] = A.cdir[o0 + k];
            }
            __syncthreads();
            big_spans(A, b, s_x, s_d, n, s_scan, &s_area);
        } else {
            __syncthreads();
            big_spans(A, b, A.cx + o0, A.cdir + o0, n, s_scan, &s_area);
        }
        __syncthreads();  // the next bucket rewrites the shared arrays
    }
}

// Per row of the image: the inclusive prefix sum, in place, that turns the span
// differences written by cov_spans into per-pixel counts (modulo 2^32, so the
// intermediate -1 terms cancel exactly).  One block per row; each thread owns
// four consecutive pixels of a 4 * kRowScanThreads tile and the tile's carry
// moves left to right.
constexpr int kRowScanThreads = 1024;

__global__ void __launch_bounds__(kRowScanThreads) cov_rowscan(uint32_t* count, uint32_t W) {
    __shared__ uint32_t s_warp[kRowScanThreads / 32];
    __shared__ uint32_t s_carry;
    uint32_t* row = count + (uint64_t)blockIdx.x * W;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < W; base += 4u * kRowScanThreads) {
        const uint32_t j = base + 4u * tid;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = j + k < W ? row[j + k] : 0u;
        v[1] += v[0];
        v[2] += v[1];
        v[3] += v[2];
        uint32_t incl = v[3];
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31u) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_warp[lane];
#pragma unroll
            for (uint32_t d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += o;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const uint32_t before = s_carry + (warp ? s_warp[warp - 1] : 0u) + (incl - v[3]);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (j + k < W) row[j + k] = before + v[k];
        __syncthreads();  // every thread has read s_carry and s_warp
        if (tid == kRowScanThreads - 1) s_carry = before + v[3];
        __syncthreads();
    }
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
    if ((uint64_t)width * height >= (1ull << 40) || height > 0x7fffffffu || width > 0x7fffffffu)
        return se_fail(c, SE_ERR_INVALID_ARG, "grid too large");
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
    e = ctx_alloc(c, (void**)&m1, off, s);
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
        ctx_free(c, m1, s);
        return se_fail(c, SE_ERR_CUDA, "coverage bounds", e);
    }
    // per-bucket stage (bucket ids are 32-bit)
    if (nb >= 0xffffffffull) {
        ctx_free(c, m1, s);
        return se_fail(c, SE_ERR_INVALID_ARG, "coverage: 2^32 or more (path, row) buckets");
    }
    const uint64_t tb = (nb + 1 + kScanTile - 1) / kScanTile;
    off = 0;
    size_t o_cnt = take((nb + 1) * 4), o_cur = take((nb + 1) * 4), o_boff = take((nb + 1) * 8);
    size_t o_bp = take((nb + 1) * 4), o_wl = take((nb + 1) * 4), o_mid = take((nb + 1) * 4), o_big = take((nb + 1) * 4);
    size_t o_ctl2 = take((4 + tb) * 4), o_agg2 = take(tb * 8), o_incl2 = take(tb * 8);
    size_t part = off;
    e = ctx_alloc(c, (void**)&m2, part, s);
    if (e != cudaSuccess) {
        ctx_free(c, m1, s);
        return se_fail(c, SE_ERR_OOM, "coverage buckets", e);
    }
    char* b2 = static_cast<char*>(m2);
    A.bucket_cnt = reinterpret_cast<uint32_t*>(b2 + o_cnt);
    A.bucket_cur = reinterpret_cast<uint32_t*>(b2 + o_cur);
    A.bucket_off = reinterpret_cast<uint64_t*>(b2 + o_boff);
    uint32_t* ctl2 = reinterpret_cast<uint32_t*>(b2 + o_ctl2);
    ScanState st2{ctl2 + 4, b2 + o_agg2, b2 + o_incl2, ctl2 + 1};
    A.bucket_path_id = reinterpret_cast<uint32_t*>(b2 + o_bp);
    A.wl = reinterpret_cast<uint32_t*>(b2 + o_wl);
    A.n_wl = ctl2;
    A.mid = reinterpret_cast<uint32_t*>(b2 + o_mid);
    A.n_mid = ctl2 + 2;
    A.big = reinterpret_cast<uint32_t*>(b2 + o_big);
    A.n_big = ctl2 + 3;
    e = cudaMemsetAsync(b2, 0, part, s);
    if (e == cudaSuccess && nb) {
        cov_bucket_paths<<<grid_of(32ull * n_paths), kCovThreads, 0, s>>>(A);
        cov_count<<<grid_of(n_prims), kCovThreads, 0, s>>>(A);
        e = launch_offsets_with_state(A.bucket_cnt, nb, A.bucket_off, st2, A.status, s);
    }
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(&ncross, A.bucket_off + nb, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && ncross >= 0x80000000ull) {
        ctx_free(c, m2, s);
        ctx_free(c, m1, s);
        return se_fail(c, SE_ERR_INVALID_ARG, "coverage: 2^31 or more row crossings");
    }
    void* m3 = nullptr;
    if (e == cudaSuccess && ncross) {
        e = ctx_alloc(c, (void**)&m3, al256(ncross * 4) + ncross + 16, s);
        if (e == cudaSuccess) {
            A.cx = static_cast<float*>(m3);
            A.cdir = reinterpret_cast<int8_t*>(static_cast<char*>(m3) + al256(ncross * 4));
            cov_scatter<<<grid_of(n_prims), kCovThreads, 0, s>>>(A);
            cov_spans<<<grid_of(nb), kCovThreads, 0, s>>>(A, nb);
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
            const unsigned per = (unsigned)(sms > 0 ? sms : 1);
            cov_spans_warp<<<per * 8u, kWarpThreads, 0, s>>>(A);
            cov_spans_mid<<<per * 6u, kMidThreads, 0, s>>>(A);
            cov_spans_big<<<per * 4u, kBigThreads, 0, s>>>(A);
            cov_rowscan<<<height, kRowScanThreads, 0, s>>>(count, width);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, A.status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (m3) ctx_free(c, m3, s);
    ctx_free(c, m2, s);
    ctx_free(c, m1, s);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "coverage", e);
    if (h_status & kStatusTimeout) result = se_fail(c, SE_ERR_TIMEOUT, "coverage scan wait gave up");
    else if (h_status & kStatusBadTag) result = se_fail(c, SE_ERR_INVALID_INPUT, "a path id is out of range");
    return result;
}
