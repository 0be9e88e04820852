// One-dimensional bulk copies from global to shared memory on the copy engine
// (cp.async.bulk with an mbarrier counting the bytes), for the emit kernels'
// record staging: one lane issues the copy of a warp's 32 contiguous records,
// the warp waits on the barrier's phase, and no lane spends load and store
// instructions on the copy.
//
// Contract (checked by the callers before they take this path, else they copy
// with plain loads): source and destination 16-byte aligned, size a multiple of
// 16 bytes.  Every wait is bounded: a wait that runs out returns false, and the
// caller records kStatusTimeout and drains with a second bounded wait before the
// block may exit (a copy still in flight would write shared memory that the
// next block on the SM owns).
#pragma once

#include <cstdint>

namespace se {

constexpr uint32_t kBulkSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// one arrival (the issuing lane's) completes a phase, together with the bytes
__device__ __forceinline__ void bulk_bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issue the copy of `bytes` from global `src` to shared `dst`, completing the
// barrier's current phase when they have landed.  Shared memory the warp read
// through ordinary loads before this call is ordered ahead of the copy's writes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Wait until the barrier's phase `parity` has completed; false if it did not
// within `limit` polls.
__device__ __forceinline__ bool bulk_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kBulkSpinLimit) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace se
