// Host-side launch wrappers for the stroke-expansion kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/stroke_expand.h"

namespace se {

// Status bits a kernel may set in the workspace status word.
enum : uint32_t {
    kStatusLimit = 1u,      // a range count was clamped to SE_MAX_RANGE_COUNT
    kStatusBadTag = 2u,     // malformed tag stream
    kStatusTimeout = 4u,    // a bounded look-back wait gave up
    kStatusCapacity = 8u,   // outline buffers too small: nothing written
};

// Per-tag results of the tag-monoid scan (structure of arrays).
struct TagInfo {
    uint32_t* pt_base;    // index of the tag's first control point
    uint32_t* path;       // path id
    uint32_t* style;      // style-stream index
    uint32_t* sub_first;  // first tag of the tag's subpath
};

struct ScanState {
    uint32_t* flags;      // per tile: 0 none, 1 aggregate, 2 inclusive prefix
    void* agg;            // per tile aggregate
    void* incl;           // per tile inclusive prefix
    uint32_t* ticket;     // dynamic tile ticket
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

struct ExpandArgs {
    const uint8_t* tags;
    uint64_t n_tags;
    const float2* pts;
    uint64_t n_points;
    const se_style* styles;
    uint32_t n_styles;
    TagInfo info;
    float tol_fit, tol_flat;
    bool arcs;
    // count pass
    uint32_t* counts;
    // write pass
    const uint64_t* offsets;
    const uint64_t* total;
    uint64_t capacity;
    float4* prims;
    float* curvature;
    uint32_t* path_id;
    uint32_t* status;
};

cudaError_t launch_tag_scan(const uint8_t* tags, uint64_t n, TagInfo info, ScanState st, uint32_t* status,
                            cudaStream_t s);
cudaError_t launch_count_scan(const uint32_t* counts, const uint8_t* tags, const uint32_t* path, uint64_t n,
                              uint64_t* offsets, uint64_t* path_offset, uint32_t n_paths, uint64_t* total,
                              uint64_t capacity, ScanState st, uint32_t* status, cudaStream_t s);
cudaError_t launch_expand_count(const ExpandArgs& a, cudaStream_t s);
cudaError_t launch_expand_write(const ExpandArgs& a, cudaStream_t s);

}  // namespace se
