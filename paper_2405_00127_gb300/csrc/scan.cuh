// Single-pass decoupled look-back scan shared by the expansion and dash passes.
//
// Each block takes a ticket, scans its kScanTile-item tile in registers and
// shared memory with warp shuffles, publishes its aggregate, and walks back
// over its predecessors' published values.  Every wait is bounded; on timeout
// the block records kStatusTimeout and continues, so no launch can hang.
#pragma once

#include <cuda/atomic>

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

// n_dev (optional): the length is read on the device and clamped to n; blocks
// whose ticket lies past the last tile exit before touching any state.
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

}  // namespace se
