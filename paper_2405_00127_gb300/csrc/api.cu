// C ABI of the stroke-expansion library: context, workspace and the
// scan -> count -> scan -> write pipeline on the context's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/stroke_expand.h"
#include "launch.h"

using namespace se;

struct se_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // device workspace, sized for cap_tags tags
    void* ws = nullptr;
    uint64_t cap_tags = 0;
    TagInfo info{};
    uint32_t* counts = nullptr;
    uint64_t* offsets = nullptr;  // cap_tags + 1
    uint32_t* control = nullptr;  // [status, ticket_a, ticket_b, pad, flags_a[tiles], flags_b[tiles]]
    size_t control_bytes = 0;
    uint32_t* status = nullptr;
    uint64_t* total = nullptr;
    ScanState scan_tags{}, scan_counts{};
    // pinned host read-back
    uint64_t* h_total = nullptr;
    uint32_t* h_status = nullptr;
    // buffers of the host end-to-end entry point
    void* io = nullptr;
    size_t io_bytes = 0;
    // stage events: [start, after tag scan, after count, after count scan, after write]
    bool profile = false;
    bool profiled = false;
    cudaEvent_t ev[5] = {};
};

namespace {

se_status fail(se_ctx* c, se_status st, const char* what, cudaError_t e = cudaSuccess) {
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
        }
    }
    return st;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// (Re)allocate the workspace for n tags.
se_status ensure_workspace(se_ctx* c, uint64_t n) {
    if (n <= c->cap_tags && c->ws) return SE_OK;
    uint64_t cap = n < 4096 ? 4096 : n + n / 4;
    uint64_t tiles = (cap + kScanTile - 1) / kScanTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_pt = take(cap * 4), o_path = take(cap * 4), o_style = take(cap * 4), o_sub = take(cap * 4);
    size_t o_counts = take(cap * 4), o_offsets = take((cap + 1) * 8), o_total = take(8);
    size_t o_agg_a = take(tiles * 16), o_incl_a = take(tiles * 16);
    size_t o_agg_b = take(tiles * 8), o_incl_b = take(tiles * 8);
    size_t control_bytes = (4 + 2 * tiles) * 4;
    size_t o_control = take(control_bytes);
    if (c->ws) {
        cudaFreeAsync(c->ws, c->stream);
        c->ws = nullptr;
        c->cap_tags = 0;
    }
    cudaError_t e = cudaMallocAsync(&c->ws, off, c->stream);
    if (e != cudaSuccess) {
        c->ws = nullptr;
        return fail(c, SE_ERR_OOM, "workspace allocation failed", e);
    }
    char* b = static_cast<char*>(c->ws);
    c->info.pt_base = reinterpret_cast<uint32_t*>(b + o_pt);
    c->info.path = reinterpret_cast<uint32_t*>(b + o_path);
    c->info.style = reinterpret_cast<uint32_t*>(b + o_style);
    c->info.sub_first = reinterpret_cast<uint32_t*>(b + o_sub);
    c->counts = reinterpret_cast<uint32_t*>(b + o_counts);
    c->offsets = reinterpret_cast<uint64_t*>(b + o_offsets);
    c->total = reinterpret_cast<uint64_t*>(b + o_total);
    c->control = reinterpret_cast<uint32_t*>(b + o_control);
    c->control_bytes = control_bytes;
    c->status = c->control;
    c->scan_tags.ticket = c->control + 1;
    c->scan_counts.ticket = c->control + 2;
    c->scan_tags.flags = c->control + 4;
    c->scan_counts.flags = c->control + 4 + tiles;
    c->scan_tags.agg = b + o_agg_a;
    c->scan_tags.incl = b + o_incl_a;
    c->scan_counts.agg = b + o_agg_b;
    c->scan_counts.incl = b + o_incl_b;
    c->cap_tags = cap;
    return SE_OK;
}

se_status check_scene(se_ctx* c, const se_scene_dev* s) {
    if (!s) return fail(c, SE_ERR_INVALID_ARG, "scene is NULL");
    if (s->n_tags && (!s->tags || !s->points || !s->styles)) return fail(c, SE_ERR_INVALID_ARG, "scene pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(s->tags) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "tags must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(s->points) & 7u) != 0) return fail(c, SE_ERR_INVALID_ARG, "points must be 8-byte aligned");
    if (s->n_tags >= (1ull << 32) || s->n_points >= (1ull << 32))
        return fail(c, SE_ERR_INVALID_ARG, "more than 2^32 tags or points");
    return SE_OK;
}

se_status check_params(se_ctx* c, const se_params* p) {
    if (!p) return fail(c, SE_ERR_INVALID_ARG, "params is NULL");
    if (!(p->tol > 0.0f) || !(p->fit_frac > 0.0f) || !(p->flat_frac > 0.0f))
        return fail(c, SE_ERR_INVALID_ARG, "tolerances must be positive");
    if (p->out_kind != SE_OUT_LINES && p->out_kind != SE_OUT_ARCS) return fail(c, SE_ERR_INVALID_ARG, "bad out_kind");
    return SE_OK;
}

ExpandArgs make_args(se_ctx* c, const se_scene_dev* s, const se_params* p) {
    ExpandArgs a{};
    a.tags = s->tags;
    a.n_tags = s->n_tags;
    a.pts = reinterpret_cast<const float2*>(s->points);
    a.n_points = s->n_points;
    a.styles = s->styles;
    a.n_styles = s->n_styles;
    a.info = c->info;
    a.tol_fit = p->tol * p->fit_frac;
    a.tol_flat = p->tol * p->flat_frac;
    a.arcs = p->out_kind == SE_OUT_ARCS;
    a.counts = c->counts;
    a.status = c->status;
    return a;
}

// scan + count + scan; the offsets go to `offsets`
se_status front_half(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* offsets, uint64_t* path_offset,
                     uint64_t capacity) {
    se_status st = ensure_workspace(c, s->n_tags);
    if (st != SE_OK) return st;
    cudaError_t e = cudaMemsetAsync(c->control, 0, c->control_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->total, 0, 8, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "memset", e);
    if (s->n_tags == 0) {
        if (path_offset && s->n_paths == 0) e = cudaMemsetAsync(path_offset, 0, 8, c->stream);
        if (offsets) e = cudaMemsetAsync(offsets, 0, 8, c->stream);
        return e == cudaSuccess ? SE_OK : fail(c, SE_ERR_CUDA, "memset", e);
    }
    if (c->profile) cudaEventRecord(c->ev[0], c->stream);
    e = launch_tag_scan(s->tags, s->n_tags, c->info, c->scan_tags, c->status, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "tag scan launch", e);
    if (c->profile) cudaEventRecord(c->ev[1], c->stream);
    ExpandArgs a = make_args(c, s, p);
    e = launch_expand_count(a, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "count launch", e);
    if (c->profile) cudaEventRecord(c->ev[2], c->stream);
    e = launch_count_scan(c->counts, s->tags, c->info.path, s->n_tags, offsets, path_offset, s->n_paths, c->total,
                          capacity, c->scan_counts, c->status, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "count scan launch", e);
    if (c->profile) cudaEventRecord(c->ev[3], c->stream);
    return SE_OK;
}

se_status map_status(uint32_t s) {
    if (s & kStatusTimeout) return SE_ERR_TIMEOUT;
    if (s & kStatusBadTag) return SE_ERR_INVALID_INPUT;
    if (s & kStatusCapacity) return SE_ERR_CAPACITY;
    if (s & kStatusLimit) return SE_ERR_LIMIT;
    return SE_OK;
}

}  // namespace

extern "C" se_status se_ctx_create(int device, void* cuda_stream, se_ctx** out) {
    if (!out) return SE_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) return SE_ERR_INVALID_ARG;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    se_ctx* c = new (std::nothrow) se_ctx();
    if (!c) return SE_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    e = cudaMallocHost(reinterpret_cast<void**>(&c->h_total), 16);
    if (e != cudaSuccess) {
        delete c;
        return SE_ERR_OOM;
    }
    c->h_status = reinterpret_cast<uint32_t*>(c->h_total + 1);
    *out = c;
    return SE_OK;
}

extern "C" se_status se_ctx_destroy(se_ctx* c) {
    if (!c) return SE_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->io) cudaFree(c->io);
    if (c->h_total) cudaFreeHost(c->h_total);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
    return SE_OK;
}

extern "C" const char* se_ctx_last_error(const se_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

extern "C" se_status se_expand(se_ctx* c, const se_scene_dev* s, const se_params* p, const se_outline_dev* out) {
    if (!c) return SE_ERR_INVALID_ARG;
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    if (!out || (out->capacity && !out->prims)) return fail(c, SE_ERR_INVALID_ARG, "outline buffers are NULL");
    if ((reinterpret_cast<uintptr_t>(out->prims) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "prims must be 16-byte aligned");
    if (p->out_kind == SE_OUT_ARCS && out->capacity && !out->curvature)
        return fail(c, SE_ERR_INVALID_ARG, "arc output needs a curvature buffer");
    cudaSetDevice(c->device);
    st = ensure_workspace(c, s->n_tags);
    if (st != SE_OK) return st;
    uint64_t* offsets = out->tag_offset ? out->tag_offset : c->offsets;
    st = front_half(c, s, p, offsets, out->path_offset, out->capacity);
    if (st != SE_OK || s->n_tags == 0) return st;
    ExpandArgs a = make_args(c, s, p);
    a.offsets = offsets;
    a.total = c->total;
    a.capacity = out->capacity;
    a.prims = reinterpret_cast<float4*>(out->prims);
    a.curvature = p->out_kind == SE_OUT_ARCS ? out->curvature : nullptr;
    a.path_id = out->path_id;
    cudaError_t e = launch_expand_write(a, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "write launch", e);
    if (c->profile) {
        cudaEventRecord(c->ev[4], c->stream);
        c->profiled = true;
    }
    return SE_OK;
}

extern "C" se_status se_profile_enable(se_ctx* c, int enable) {
    if (!c) return SE_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (enable && !c->ev[0]) {
        for (auto& e : c->ev) {
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return fail(c, SE_ERR_CUDA, "event create", r);
        }
    }
    c->profile = enable != 0;
    c->profiled = false;
    return SE_OK;
}

extern "C" se_status se_profile_read(se_ctx* c, float* ms) {
    if (!c || !ms) return SE_ERR_INVALID_ARG;
    if (!c->profiled) return fail(c, SE_ERR_INVALID_ARG, "no profiled expansion");
    cudaError_t e = cudaEventSynchronize(c->ev[4]);
    for (int k = 0; k < 4 && e == cudaSuccess; k++) e = cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "event read", e);
    return SE_OK;
}

extern "C" se_status se_count(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* n_prims) {
    if (!c || !n_prims) return SE_ERR_INVALID_ARG;
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    cudaSetDevice(c->device);
    st = ensure_workspace(c, s->n_tags);
    if (st != SE_OK) return st;
    st = front_half(c, s, p, c->offsets, nullptr, ~0ull);
    if (st != SE_OK) return st;
    return se_sync(c, n_prims);
}

extern "C" se_status se_sync(se_ctx* c, uint64_t* n_prims) {
    if (!c) return SE_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->ws) {
        if (n_prims) *n_prims = 0;
        return SE_OK;
    }
    cudaError_t e = cudaMemcpyAsync(c->h_total, c->total, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_status, c->status, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "sync", e);
    if (n_prims) *n_prims = *c->h_total;
    se_status st = map_status(*c->h_status);
    if (st != SE_OK) fail(c, st, "device status");
    return st;
}

extern "C" se_status se_total_device(se_ctx* c, const uint64_t** d_total) {
    if (!c || !d_total) return SE_ERR_INVALID_ARG;
    if (!c->ws) return fail(c, SE_ERR_INVALID_ARG, "no expansion has run");
    *d_total = c->total;
    return SE_OK;
}

extern "C" se_status se_expand_host(se_ctx* c, const uint8_t* tags, uint64_t n_tags, const float* points,
                                    uint64_t n_points, const se_style* styles, uint32_t n_styles, uint32_t n_paths,
                                    const float* dashes, uint32_t n_dashes, const se_params* p, float* host_prims,
                                    float* host_curvature, uint64_t capacity, uint64_t* n_prims) {
    if (!c || !n_prims || (n_tags && (!tags || !points || !styles)) || (capacity && !host_prims))
        return SE_ERR_INVALID_ARG;
    se_status st = check_params(c, p);
    if (st != SE_OK) return st;
    bool arcs = p->out_kind == SE_OUT_ARCS;
    if (arcs && capacity && !host_curvature) return fail(c, SE_ERR_INVALID_ARG, "arc output needs a curvature buffer");
    cudaSetDevice(c->device);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_tags = take(n_tags + 16), o_pts = take(n_points * 8 + 8), o_sty = take(size_t(n_styles) * sizeof(se_style) + 8);
    size_t o_dash = take(size_t(n_dashes) * 4 + 4), o_prims = take(capacity * 16 + 16), o_curv = take(arcs ? capacity * 4 + 4 : 4);
    if (off > c->io_bytes) {
        if (c->io) cudaFreeAsync(c->io, c->stream);
        c->io = nullptr;
        c->io_bytes = 0;
        cudaError_t e = cudaMallocAsync(&c->io, off, c->stream);
        if (e != cudaSuccess) {
            c->io = nullptr;
            return fail(c, SE_ERR_OOM, "host-path buffers", e);
        }
        c->io_bytes = off;
    }
    char* b = static_cast<char*>(c->io);
    cudaError_t e = cudaSuccess;
    if (n_tags) e = cudaMemcpyAsync(b + o_tags, tags, n_tags, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_points) e = cudaMemcpyAsync(b + o_pts, points, n_points * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_styles)
        e = cudaMemcpyAsync(b + o_sty, styles, size_t(n_styles) * sizeof(se_style), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_dashes) e = cudaMemcpyAsync(b + o_dash, dashes, size_t(n_dashes) * 4, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "upload", e);
    se_scene_dev s{};
    s.tags = reinterpret_cast<const uint8_t*>(b + o_tags);
    s.n_tags = n_tags;
    s.points = reinterpret_cast<const float*>(b + o_pts);
    s.n_points = n_points;
    s.styles = reinterpret_cast<const se_style*>(b + o_sty);
    s.n_styles = n_styles;
    s.n_paths = n_paths;
    s.dashes = n_dashes ? reinterpret_cast<const float*>(b + o_dash) : nullptr;
    s.n_dashes = n_dashes;
    se_outline_dev o{};
    o.prims = reinterpret_cast<float*>(b + o_prims);
    o.curvature = arcs ? reinterpret_cast<float*>(b + o_curv) : nullptr;
    o.capacity = capacity;
    st = se_expand(c, &s, p, &o);
    if (st != SE_OK) return st;
    uint64_t n = 0;
    st = se_sync(c, &n);
    *n_prims = n;
    if (st != SE_OK && st != SE_ERR_LIMIT) return st;
    if (n) {
        e = cudaMemcpyAsync(host_prims, b + o_prims, n * 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && arcs) e = cudaMemcpyAsync(host_curvature, b + o_curv, n * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "download", e);
    }
    return st;
}
