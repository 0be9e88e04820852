// C ABI of the stroke-expansion library: context, workspace and the
// scan -> count -> scan -> write pipeline on the context's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/stroke_expand.h"
#include "launch.h"
#include "pipeline.cuh"

using namespace se;

struct se_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // device workspace: per-tag arrays for cap_tags tags, per-item arrays for item_cap items
    void* ws = nullptr;
    uint64_t cap_tags = 0;
    uint64_t item_cap = 0;
    TagInfo info{};
    PlanBufs pb{};
    uint32_t* control = nullptr;  // [status, 3 tickets, flags_tags[tt], flags_items[tt], flags_prims[ti]]
    size_t control_bytes = 0;
    uint32_t* status = nullptr;
    uint64_t* total = nullptr;
    uint64_t* vtotal = nullptr;
    ScanState scan_tags{}, scan_items{}, scan_prims{};
    // pinned host read-back
    uint64_t* h_total = nullptr;
    uint32_t* h_status = nullptr;
    uint64_t* h_items = nullptr;
    uint64_t last_tags = 0;
    size_t ws_bytes = 0;
    // buffers of the host end-to-end entry point
    void* io = nullptr;
    size_t io_bytes = 0;
    // stage events: start, after tag scan, plan, pieces, primitive scan, emit
    bool profile = false;
    bool profiled = false;
    cudaEvent_t ev[6] = {};
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

// (Re)allocate the workspace for n tags and at least `items` piece items.
se_status ensure_workspace(se_ctx* c, uint64_t n, uint64_t items) {
    if (n <= c->cap_tags && items <= c->item_cap && c->ws) return SE_OK;
    uint64_t cap = n < 4096 ? 4096 : n + n / 4;
    if (cap < c->cap_tags) cap = c->cap_tags;
    uint64_t icap = items < 4 * cap ? 4 * cap : items + items / 4;
    if (icap < c->item_cap) icap = c->item_cap;
    uint64_t tt = (cap + kScanTile - 1) / kScanTile, ti = (icap + kScanTile - 1) / kScanTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_pt = take(cap * 4), o_path = take(cap * 4), o_style = take(cap * 4), o_sub = take(cap * 4);
    size_t o_nitems = take(cap * 4), o_bits = take(cap * 8), o_ovf = take(cap * 4);
    size_t o_tails = take(cap * sizeof(TailRec)), o_ibase = take((cap + 1) * 8);
    size_t o_itag = take(icap * 4), o_iref = take(icap * 4), o_icnt = take(icap * 4), o_ioff = take((icap + 1) * 8);
    size_t o_ivcnt = take(icap * 4), o_ivoff = take((icap + 1) * 8), o_vtotal = take(8);
    size_t o_pieces = take(icap * sizeof(PieceRec));
    size_t o_total = take(8);
    size_t o_agg_t = take(tt * 16), o_incl_t = take(tt * 16);
    size_t o_agg_i = take(tt * 8), o_incl_i = take(tt * 8);
    size_t o_agg_p = take(ti * 8), o_incl_p = take(ti * 8);
    size_t control_bytes = (4 + 2 * tt + ti) * 4;
    size_t o_control = take(control_bytes);
    if (c->ws) {
        cudaFreeAsync(c->ws, c->stream);
        c->ws = nullptr;
        c->cap_tags = 0;
        c->item_cap = 0;
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
    PlanBufs& pb = c->pb;
    pb.n_items = reinterpret_cast<uint32_t*>(b + o_nitems);
    pb.bits = reinterpret_cast<uint64_t*>(b + o_bits);
    pb.overflow = reinterpret_cast<uint32_t*>(b + o_ovf);
    pb.tails = reinterpret_cast<TailRec*>(b + o_tails);
    pb.item_base = reinterpret_cast<uint64_t*>(b + o_ibase);
    pb.item_cap = icap;
    pb.item_tag = reinterpret_cast<uint32_t*>(b + o_itag);
    pb.item_ref = reinterpret_cast<uint32_t*>(b + o_iref);
    pb.item_count = reinterpret_cast<uint32_t*>(b + o_icnt);
    pb.item_off = reinterpret_cast<uint64_t*>(b + o_ioff);
    pb.item_vcount = reinterpret_cast<uint32_t*>(b + o_ivcnt);
    pb.item_voff = reinterpret_cast<uint64_t*>(b + o_ivoff);
    c->vtotal = reinterpret_cast<uint64_t*>(b + o_vtotal);
    pb.pieces = reinterpret_cast<PieceRec*>(b + o_pieces);
    c->total = reinterpret_cast<uint64_t*>(b + o_total);
    c->control = reinterpret_cast<uint32_t*>(b + o_control);
    c->control_bytes = control_bytes;
    c->status = c->control;
    c->scan_tags.ticket = c->control + 1;
    c->scan_items.ticket = c->control + 2;
    c->scan_prims.ticket = c->control + 3;
    c->scan_tags.flags = c->control + 4;
    c->scan_items.flags = c->control + 4 + tt;
    c->scan_prims.flags = c->control + 4 + 2 * tt;
    c->scan_tags.agg = b + o_agg_t;
    c->scan_tags.incl = b + o_incl_t;
    c->scan_items.agg = b + o_agg_i;
    c->scan_items.incl = b + o_incl_i;
    c->scan_prims.agg = b + o_agg_p;
    c->scan_prims.incl = b + o_incl_p;
    c->cap_tags = cap;
    c->item_cap = icap;
    c->ws_bytes = off;
    return SE_OK;
}

se_status check_scene(se_ctx* c, const se_scene_dev* s) {
    if (!s) return fail(c, SE_ERR_INVALID_ARG, "scene is NULL");
    if (s->n_tags && (!s->tags || !s->points || !s->styles)) return fail(c, SE_ERR_INVALID_ARG, "scene pointer is NULL");
    if ((reinterpret_cast<uintptr_t>(s->tags) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "tags must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(s->points) & 7u) != 0) return fail(c, SE_ERR_INVALID_ARG, "points must be 8-byte aligned");
    if (s->n_tags >= (1ull << 31) || s->n_points >= (1ull << 32))
        return fail(c, SE_ERR_INVALID_ARG, "more than 2^31 tags or 2^32 points");
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
    a.total = c->total;
    a.status = c->status;
    return a;
}

void rec(se_ctx* c, int k) {
    if (c->profile) cudaEventRecord(c->ev[k], c->stream);
}

// tag scan, plan, item scan, decode, piece, primitive scan
se_status front_half(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* tag_offset,
                     uint64_t* path_offset, uint64_t capacity) {
    cudaError_t e = cudaMemsetAsync(c->control, 0, c->control_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->total, 0, 8, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "memset", e);
    if (s->n_tags == 0) {
        if (path_offset) e = cudaMemsetAsync(path_offset, 0, 8ull * (s->n_paths + 1), c->stream);
        if (e == cudaSuccess && tag_offset) e = cudaMemsetAsync(tag_offset, 0, 8, c->stream);
        return e == cudaSuccess ? SE_OK : fail(c, SE_ERR_CUDA, "memset", e);
    }
    ExpandArgs a = make_args(c, s, p);
    a.capacity = capacity;
    rec(c, 0);
    e = launch_tag_scan(s->tags, s->n_tags, c->info, c->scan_tags, c->status, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "tag scan launch", e);
    rec(c, 1);
    e = launch_plan(a, c->pb, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "plan launch", e);
    rec(c, 2);
    e = launch_item_scan(a, c->pb, c->scan_items, c->stream);
    if (e == cudaSuccess) e = launch_decode(a, c->pb, c->stream);
    if (e == cudaSuccess) e = launch_piece(a, c->pb, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "piece launch", e);
    rec(c, 3);
    e = launch_prim_scan(a, c->pb, tag_offset, path_offset, s->n_paths, c->vtotal, c->scan_prims, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "primitive scan launch", e);
    rec(c, 4);
    return SE_OK;
}

se_status map_status(uint32_t s) {
    if (s & kStatusTimeout) return SE_ERR_TIMEOUT;
    if (s & kStatusBadTag) return SE_ERR_INVALID_INPUT;
    if (s & kStatusWorkspace) return SE_ERR_WORKSPACE;
    if (s & kStatusCapacity) return SE_ERR_CAPACITY;
    if (s & kStatusLimit) return SE_ERR_LIMIT;
    return SE_OK;
}

se_status read_back(se_ctx* c, uint64_t* n_prims, uint64_t* n_items) {
    cudaError_t e = cudaMemcpyAsync(c->h_total, c->total, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_status, c->status, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && n_items) e = cudaMemcpyAsync(c->h_items, c->pb.item_base + c->last_tags, 8,
                                                         cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "sync", e);
    if (n_prims) *n_prims = *c->h_total;
    if (n_items) *n_items = c->last_tags ? *c->h_items : 0;
    se_status st = map_status(*c->h_status);
    if (st != SE_OK) fail(c, st, "device status");
    return st;
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
    e = cudaMallocHost(reinterpret_cast<void**>(&c->h_total), 32);
    if (e != cudaSuccess) {
        delete c;
        return SE_ERR_OOM;
    }
    c->h_status = reinterpret_cast<uint32_t*>(c->h_total + 1);
    c->h_items = c->h_total + 2;
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
    st = ensure_workspace(c, s->n_tags, 0);
    if (st != SE_OK) return st;
    c->last_tags = s->n_tags;
    st = front_half(c, s, p, out->tag_offset, out->path_offset, out->capacity);
    if (st != SE_OK || s->n_tags == 0) return st;
    ExpandArgs a = make_args(c, s, p);
    a.capacity = out->capacity;
    a.prims = reinterpret_cast<float4*>(out->prims);
    a.curvature = p->out_kind == SE_OUT_ARCS ? out->curvature : nullptr;
    a.path_id = out->path_id;
    cudaError_t e = launch_emit(a, c->pb, c->vtotal, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "emit launch", e);
    if (c->profile) {
        cudaEventRecord(c->ev[5], c->stream);
        c->profiled = true;
    }
    return SE_OK;
}

extern "C" se_status se_count(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* n_prims) {
    if (!c || !n_prims) return SE_ERR_INVALID_ARG;
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    cudaSetDevice(c->device);
    uint64_t need = 0;
    for (int attempt = 0; attempt < 2; attempt++) {
        st = ensure_workspace(c, s->n_tags, need);
        if (st != SE_OK) return st;
        c->last_tags = s->n_tags;
        st = front_half(c, s, p, nullptr, nullptr, ~0ull);
        if (st != SE_OK) return st;
        st = read_back(c, n_prims, &need);
        if (st != SE_ERR_WORKSPACE) return st;
    }
    return st;
}

extern "C" se_status se_sync(se_ctx* c, uint64_t* n_prims) {
    if (!c) return SE_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->ws) {
        if (n_prims) *n_prims = 0;
        return SE_OK;
    }
    return read_back(c, n_prims, nullptr);
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
    cudaError_t e = cudaEventSynchronize(c->ev[5]);
    for (int k = 0; k < 5 && e == cudaSuccess; k++) e = cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "event read", e);
    return SE_OK;
}

extern "C" se_status se_ctx_stats(se_ctx* c, se_stats* out) {
    if (!c || !out) return SE_ERR_INVALID_ARG;
    out->n_tags = c->last_tags;
    out->n_items = 0;
    out->n_prims = 0;
    out->piece_bytes = (uint32_t)sizeof(PieceRec);
    out->tail_bytes = (uint32_t)sizeof(TailRec);
    out->workspace_bytes = c->ws_bytes;
    if (!c->ws) return SE_OK;
    cudaSetDevice(c->device);
    se_status st = read_back(c, &out->n_prims, &out->n_items);
    return st == SE_ERR_CUDA ? st : SE_OK;
}
