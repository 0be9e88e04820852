// Internal state of a library context (shared by api.cu and batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <string>

#include "../../include/stroke_expand.h"
#include "dash.cuh"
#include "launch.h"
#include "pipeline.cuh"

using namespace se;

// Workspace of the device dash pass: per input tag, per path and the
// rewritten (solid) output streams.
struct DashWs {
    void* mem = nullptr;
    size_t bytes = 0;
    uint64_t cap_in = 0;
    uint32_t cap_paths = 0, cap_styles = 0;
    uint64_t cap_tags = 0, cap_pts = 0, cap_cuts = 0, cap_slots = 0;
    se::DashBufs b{};
    se::ScanState tag_st{}, seg_st{}, out_st{}, cut_st{};
    uint32_t* control = nullptr;  // [status, 4 tickets (+ pad), 4 x tile flags]
    size_t control_bytes = 0;
};

struct se_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // the caller's device allocator (both NULL: the stream-ordered allocator)
    se_alloc_fn alloc_fn = nullptr;
    se_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string err;
    // device workspace: per-tag arrays for cap_tags tags, per-item arrays for item_cap items
    void* ws = nullptr;
    uint64_t cap_tags = 0;
    uint64_t item_cap = 0;
    TagInfo info{};
    uint32_t* xform_buf = nullptr;  // per-tag transform index (info.xform points here for scenes with transforms)
    PlanBufs pb{};
    uint32_t* control = nullptr;  // [status, 3 tickets, flags_tags[tt], flags_items[tt], flags_prims[ti]]
    size_t control_bytes = 0;
    uint32_t* status = nullptr;
    uint64_t* total = nullptr;
    ScanState scan_tags{}, scan_items{}, scan_prims{};
    uint64_t* items_total = nullptr;
    // pinned host read-back
    uint64_t* h_total = nullptr;
    uint32_t* h_status = nullptr;       // [0] expansion status, [1] dash status
    uint64_t* h_items = nullptr;
    uint64_t* h_dash = nullptr;         // dash out_n: tags, points, tags needed, points needed, cuts needed
    uint64_t last_tags = 0;             // tags (or the tag capacity of a dashed rewrite) of the last scene
    uint64_t last_input_tags = 0;
    bool last_dashed = false;
    DashWs dash;
    uint64_t dash_slots_need = 0;  // cubics with cuts the last count needed panel slots for
    Tuning tune;
    bool capturing = false;  // inside a stream capture: no workspace may be (re)allocated
    uint64_t ws_gen = 0;     // bumped whenever a workspace is reallocated (captured graphs hold its addresses)
    size_t ws_bytes = 0;
    // buffers of the host end-to-end entry point
    void* io = nullptr;
    size_t io_bytes = 0;
    // its pipelined download: a copy stream, one event per emit chunk, the chunk
    // boundaries (pinned)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t chunk_ev[16] = {};
    uint64_t* h_bounds = nullptr;
    // stage events: start, after tag scan, plan, pieces, primitive scan, emit;
    // ev[6], ev[7] around the dash pass
    bool profile = false;
    bool profiled = false;
    cudaEvent_t ev[8] = {};
    // the scene and params of the last se_count whose front half is still in the
    // workspace (an expansion may then run just the primitive scan and the emit)
    bool counted = false;
    se_scene_dev counted_scene{};
    se_params counted_params{};
    uint64_t counted_gen = 0;
    // read-back of a library-owned outline whose expansion is still in flight:
    // run before the context starts another expansion (the read-back state is
    // the context's own, so it must be taken first)
    std::function<void()> settle;
};

// Device memory for the context's work on stream s: from the caller's allocator
// when the context has one, else from the stream-ordered allocator.  A refused
// allocation is cudaErrorMemoryAllocation (the caller maps it to SE_ERR_OOM).
inline cudaError_t dev_alloc(se_alloc_fn fa, void* user, void** p, size_t bytes, cudaStream_t s) {
    if (!fa) return cudaMallocAsync(p, bytes, s);
    *p = fa(bytes, user, static_cast<void*>(s));
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
inline void dev_free(se_free_fn ff, void* user, void* p, cudaStream_t s) {
    if (!p) return;
    if (ff) ff(p, user, static_cast<void*>(s));
    else cudaFreeAsync(p, s);
}
inline cudaError_t ctx_alloc(se_ctx* c, void** p, size_t bytes, cudaStream_t s) {
    return dev_alloc(c->alloc_fn, c->alloc_user, p, bytes, s);
}
inline cudaError_t ctx_alloc(se_ctx* c, void** p, size_t bytes) { return ctx_alloc(c, p, bytes, c->stream); }
inline void ctx_free(se_ctx* c, void* p, cudaStream_t s) { dev_free(c->free_fn, c->alloc_user, p, s); }
inline void ctx_free(se_ctx* c, void* p) { ctx_free(c, p, c->stream); }

inline void settle_pending(se_ctx* c) {
    if (c && c->settle) {
        std::function<void()> f = std::move(c->settle);
        c->settle = nullptr;
        f();
    }
}

// Device bytes a batch holds (its gathered scene and tables).
size_t se_batch_device_bytes(const se_batch* b);

// Record an error message on the context and return st.
se_status se_fail(se_ctx* c, se_status st, const char* what, cudaError_t e = cudaSuccess);
