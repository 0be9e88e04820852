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

#include "expand_tag.cuh"
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
