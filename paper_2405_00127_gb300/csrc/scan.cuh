// Single-pass decoupled look-back scan shared by the expansion and dash passes.
//
// Each block takes a ticket, scans its kScanTile-item tile in registers and
// shared memory with warp shuffles, publishes its aggregate, and walks back
// over its predecessors' published values, 32 at a time with one warp (the
// flags in one round trip, the values combined in tile order with shuffles)
// up to the nearest inclusive prefix.  Every wait is bounded; on timeout the
// block records kStatusTimeout and continues, so no launch can hang.
#pragma once

#include <cuda/atomic>

#include <cstring>

#include "launch.h"

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

// a value of any 4-byte-multiple type shifted down the warp by d lanes
template <class T>
__device__ __forceinline__ T shfl_down_any(T v, int d) {
    static_assert(sizeof(T) % 4 == 0, "scan values are whole words");
    constexpr int kW = (int)(sizeof(T) / 4);
    uint32_t w[kW];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int k = 0; k < kW; k++) w[k] = __shfl_down_sync(0xffffffffu, w[k], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// n_dev (optional): the length is read on the device and clamped to n.  A block
// takes tickets until one lies past the last tile, so a grid of any size scans
// every tile (a grid smaller than the tile count makes blocks loop; tickets
// are handed out in order, so every tile a block waits on belongs to a block
// that is already running).
template <class Op>
__global__ void __launch_bounds__(kScanThreads) lookback_scan(Op op, uint64_t n, const uint64_t* n_dev, ScanState st,
                                                              uint32_t* status) {
    using T = typename Op::T;
    __shared__ uint32_t s_tile;
    __shared__ T s_warp[kScanThreads / 32];
    __shared__ T s_prefix;
    if (n_dev) {
        uint64_t m = *n_dev;
        n = m < n ? m : n;
    }
    if (n == 0) return;
    for (;;) {
        __syncthreads();  // the previous tile's shared values are consumed
        if (threadIdx.x == 0) s_tile = atomicAdd(st.ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if ((uint64_t)tile * kScanTile >= n) return;
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
        if (warp == 0) {
            // publish the tile's aggregate, then look back with the whole warp: lane i
            // reads the flag of tile top - i, so one round trip covers 32 predecessors
            const T tile_agg = s_warp[kScanThreads / 32 - 1];
            T* agg = reinterpret_cast<T*>(st.agg);
            T* incl = reinterpret_cast<T*>(st.incl);
            T ex = op.identity();
            cuda::atomic_ref<uint32_t, cuda::thread_scope_device> f(st.flags[tile]);
            if (tile == 0) {
                if (lane == 0) {
                    incl[0] = tile_agg;
                    f.store(2u, cuda::memory_order_release);
                }
            } else {
                if (lane == 0) {
                    agg[tile] = tile_agg;
                    f.store(1u, cuda::memory_order_release);
                }
                int64_t top = (int64_t)tile - 1;  // the newest predecessor of the window
                const uint32_t limit = st.spin_limit ? st.spin_limit : kSpinLimit;
                uint32_t spins = 0;
                bool timed_out = false;
                while (top >= 0) {
                    const int64_t t = top - lane;
                    uint32_t fl = 2u;  // lanes before tile 0 lie past its inclusive prefix: never used
                    if (t >= 0) {
                        cuda::atomic_ref<uint32_t, cuda::thread_scope_device> ft(st.flags[t]);
                        fl = ft.load(cuda::memory_order_acquire);
                    }
                    const uint32_t incl_lanes = __ballot_sync(0xffffffffu, fl == 2u);
                    const uint32_t zero_lanes = __ballot_sync(0xffffffffu, fl == 0u);
                    // the window ends at the nearest inclusive prefix (lane m), else it is all 32
                    const uint32_t m = incl_lanes ? (uint32_t)(__ffs(incl_lanes) - 1) : 31u;
                    const uint32_t need = m == 31u ? 0xffffffffu : ((1u << (m + 1u)) - 1u);
                    if (zero_lanes & need) {  // a predecessor has not published yet
                        if (++spins >= limit) {
                            timed_out = true;
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    T v = op.identity();
                    if ((uint32_t)lane <= m && t >= 0) v = fl == 2u ? incl[t] : agg[t];
                    // ordered reduction: lane 0 receives v[m] + ... + v[0], earlier tiles first
    #pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const T o = shfl_down_any(v, d);
                        if (lane + d < 32) v = op.combine(o, v);
                    }
                    if (lane == 0) ex = op.combine(v, ex);
                    if (incl_lanes) break;
                    top -= 32;
                }
                if (lane == 0) {
                    if (timed_out) atomicOr(status, (uint32_t)kStatusTimeout);
                    incl[tile] = op.combine(ex, tile_agg);
                    f.store(2u, cuda::memory_order_release);
                }
            }
            if (lane == 0) s_prefix = ex;
        }
        __syncthreads();
        T prefix = op.combine(s_prefix, thread_excl);
        op.store(base, n, v, prefix);
    }
}

}  // namespace se
