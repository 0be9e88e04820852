// The count -> offset scan for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc: code running under a fixed device
// memory budget that was reserved up front, code that must not block on the
// allocator (which can synchronise the device) inside a latency-critical
// render loop, or a plugin running inside a host application that owns all
// device allocations.  For them this file keeps the scan's scratch -- the
// per-tile look-back flags, aggregates and inclusive prefixes, the tile ticket
// and a status word -- in one file-scope device array of fixed size, so the
// entry point allocates nothing.  The caller passes the counts and the output
// offsets; both are device memory the caller owns.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "../../include/stroke_expand.h"
#include "launch.h"

namespace se {
cudaError_t launch_offsets_with_state(const uint32_t* counts, uint64_t n, uint64_t* offsets, ScanState st,
                                      uint32_t* status, cudaStream_t s);
}

using namespace se;

namespace {

// one look-back slot per scan tile, rounded up so a limit that is not a
// multiple of the tile still has a slot for its last (partial) tile
constexpr uint64_t kTiles = (SE_NOALLOC_MAX_COUNTS + kScanTile - 1) / kScanTile;
static_assert(kTiles * kScanTile >= SE_NOALLOC_MAX_COUNTS, "a look-back slot for every tile");
// layout: [status, ticket, pad, pad] [flags: kTiles u32] [agg: kTiles u64] [incl: kTiles u64]
constexpr size_t kControlBytes = (4 + kTiles) * 4;
constexpr size_t kAggOffset = (kControlBytes + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kAggOffset + 2 * kTiles * 8;

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// the array's device address per device, resolved once under a per-device
// once-flag (host threads may make their first calls concurrently)
std::once_flag g_once[kMaxDevices];
std::atomic<void*> g_scratch_addr[kMaxDevices];

}  // namespace

extern "C" se_status se_scan_offsets_noalloc(const uint32_t* counts, uint64_t n, uint64_t* offsets,
                                             void* cuda_stream) {
    if (n > SE_NOALLOC_MAX_COUNTS) return SE_ERR_INVALID_ARG;
    if (n > 0 && (!counts || !offsets)) return SE_ERR_INVALID_ARG;
    if (!offsets) return SE_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SE_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // first call on this device: resolve the device address of the array
    // (host code cannot use the symbol itself as a device pointer)
    std::call_once(g_once[dev], [dev] {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) == cudaSuccess && p) g_scratch_addr[dev].store(p);
    });
    unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev].load());
    if (!base) return SE_ERR_CUDA;
    uint32_t* control = reinterpret_cast<uint32_t*>(base);
    // the array keeps the previous call's contents: flags, ticket and status must restart at zero
    if (cudaMemsetAsync(control, 0, kControlBytes, s) != cudaSuccess) return SE_ERR_CUDA;
    if (n == 0) {
        if (cudaMemsetAsync(offsets, 0, 8, s) != cudaSuccess) return SE_ERR_CUDA;
        return cudaStreamSynchronize(s) == cudaSuccess ? SE_OK : SE_ERR_CUDA;
    }
    ScanState st;
    st.spin_limit = 0;  // the default bound on every wait
    st.ticket = control + 1;
    st.flags = control + 4;
    st.agg = base + kAggOffset;
    st.incl = base + kAggOffset + kTiles * 8;
    if (launch_offsets_with_state(counts, n, offsets, st, control, s) != cudaSuccess) return SE_ERR_CUDA;
    // the status word comes back on the caller's stream only (a copy on the
    // legacy default stream would also wait for every other blocking stream)
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, control, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SE_ERR_CUDA;
    return (status & kStatusTimeout) ? SE_ERR_TIMEOUT : SE_OK;
}
