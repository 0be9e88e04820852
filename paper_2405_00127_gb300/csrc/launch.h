// Types shared by the host orchestration (api.cu) and the kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stroke_expand.h"

namespace se {

// Status bits a kernel may set in the workspace status word.
enum : uint32_t {
    kStatusLimit = 1u,      // a range count was clamped to SE_MAX_RANGE_COUNT
    kStatusBadTag = 2u,     // malformed tag stream, bad dash pattern (or a dashed style reached the expansion)
    kStatusTimeout = 4u,    // a bounded look-back wait gave up
    kStatusCapacity = 8u,   // outline buffers too small: nothing written
    kStatusWorkspace = 16u, // the context's piece workspace is too small for this scene
};

// Per-tag results of the tag-monoid scan (structure of arrays).
struct TagInfo {
    uint32_t* pt_base;    // word index of the tag's first control point
    uint32_t* path;       // path id
    uint32_t* style;      // style-stream index
    uint32_t* sub_first;  // first tag of the tag's subpath
    uint32_t* xform;      // transform-stream index (~0u: identity); NULL when the scene has no transforms
    // the plan pass's schedule (NULL when not wanted): curve tags (quadratics and
    // cubics, which carry Algorithm 2's subdivision loop) in stream order, the
    // other tags in stream order, and the curve count
    uint32_t* curve_list;
    uint32_t* line_list;
    uint32_t* n_curves;
};

// One element of the tag-monoid scan (Section 8.2): point offset, path,
// style and transform counts, the subpath start (a max), and the count of
// curve tags (the plan pass's schedule).
struct TagVal {
    uint32_t pt, path, style, xf, sub, crv;
};
constexpr size_t kTagValBytes = 32;  // per-tile aggregate slot (sizeof(TagVal) rounded up)
static_assert(sizeof(TagVal) <= kTagValBytes, "tag scan slot");

struct ScanState {
    uint32_t* flags;      // per tile: 0 none, 1 aggregate, 2 inclusive prefix
    void* agg;            // per tile aggregate
    void* incl;           // per tile inclusive prefix
    uint32_t* ticket;     // dynamic tile ticket
    uint32_t spin_limit;  // polls of a predecessor's flag before the wait gives up (0: the default limit)
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

struct ExpandArgs {
    const uint8_t* tags;
    uint64_t n_tags;             // tag count, or an upper bound of it when n_tags_dev is set
    const uint64_t* n_tags_dev;  // optional: the tag count in device memory (a stream rewritten on the device)
    const uint32_t* words;  // path data stream (Table 1: 32- or 16-bit coordinates per tag)
    uint64_t n_words;
    const se_style* styles;
    uint32_t n_styles;
    const float* xforms;  // 6 floats per entry (Section 8.2); NULL when n_xforms == 0
    uint32_t n_xforms;
    TagInfo info;
    float tol_fit, tol_flat;
    bool arcs;
    bool refine;  // refined line output (Section 4.2)
    // emit ranges (pieces and tags whose primitives the emit kernels write; all by default)
    uint64_t emit_piece_lo = 0, emit_piece_hi = ~0ull;
    uint64_t emit_tag_lo = 0, emit_tag_hi = ~0ull;
    // outline
    const uint64_t* total;
    uint64_t capacity;
    float4* prims;
    float* curvature;
    uint32_t* path_id;
    uint32_t* status;
    const uint32_t* dash_status;  // the dash pass's status word when the scene was dashed on the device, else NULL
};

// Launch shapes the autotuner chooses among (the results do not depend on them).
struct Tuning {
    uint32_t plan_block = 256;        // threads per block of plan / decode (256: 6% faster plan than 128 on map-like)
    uint32_t piece_block = 256;       // piece records staged per block (128 or 256; 256: 1.08 vs 1.20 ms on map-like)
    uint32_t emit_block = 64;         // threads per block of the emit kernels (64 or 128)
    uint32_t emit_blocks_per_sm = 0;  // resident emit blocks per SM (0: as many as fit)
};

// Offsets from a scan whose bounded wait gave up (here or in the dash pass that
// wrote the stream) are not trusted: kernels that index by them write nothing.
__device__ __forceinline__ bool scan_untrusted(const uint32_t* status, const uint32_t* dash_status) {
    return ((*status | (dash_status ? *dash_status : 0u)) & kStatusTimeout) != 0u;
}

// tag count of the stream being expanded (device side)
__host__ __device__ __forceinline__ uint64_t tag_count(const ExpandArgs& a) {
    if (!a.n_tags_dev) return a.n_tags;
    uint64_t n = *a.n_tags_dev;
    return n < a.n_tags ? n : a.n_tags;
}

}  // namespace se
