// C ABI of the stroke-expansion library: context, workspace and the
// scan -> count -> scan -> write pipeline on the context's stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/stroke_expand.h"
#include "ctx.h"

using namespace se;

namespace {

se_status fail(se_ctx* c, se_status st, const char* what, cudaError_t e = cudaSuccess) {
    return se_fail(c, st, what, e);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// (Re)allocate the workspace for n tags and at least `items` piece items.
se_status ensure_workspace(se_ctx* c, uint64_t n, uint64_t items) {
    if (n <= c->cap_tags && items <= c->item_cap && c->ws) return SE_OK;
    if (c->capturing) return fail(c, SE_ERR_WORKSPACE, "workspace too small to capture: count the scene first");
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
    size_t o_tails = take(cap * sizeof(TailRec) + 16), o_ibase = take((cap + 1) * 8);
    size_t o_itag = take(icap * 4), o_iref = take(icap * 4), o_icnt = take(icap * 4), o_ioff = take((icap + 1) * 8);
    size_t o_ivcnt = take(icap * 4);
    // 16 bytes of slack: the emit's bulk copies round a partial chunk up to 16 bytes
    size_t o_pieces = take(icap * sizeof(PieceRec) + 16), o_pitem = take(icap * 4);
    size_t o_total = take(8), o_itot = take(8);
    size_t o_xf = take(cap * 4);
    size_t o_clist = take(cap * 4), o_llist = take(cap * 4), o_ncurve = take(8);
    size_t o_agg_t = take(tt * kTagValBytes), o_incl_t = take(tt * kTagValBytes);
    size_t o_agg_i = take(tt * 8), o_incl_i = take(tt * 8);
    size_t o_agg_p = take(ti * 8), o_incl_p = take(ti * 8);
    size_t control_bytes = (4 + 2 * tt + ti) * 4;
    size_t o_control = take(control_bytes);
    if (c->ws) {
        ctx_free(c, c->ws);
        c->ws = nullptr;
        c->cap_tags = 0;
        c->item_cap = 0;
    }
    cudaError_t e = ctx_alloc(c, &c->ws, off);
    c->ws_gen++;
    if (e != cudaSuccess) {
        c->ws = nullptr;
        return fail(c, SE_ERR_OOM, "workspace allocation failed", e);
    }
    char* b = static_cast<char*>(c->ws);
    c->info.pt_base = reinterpret_cast<uint32_t*>(b + o_pt);
    c->info.path = reinterpret_cast<uint32_t*>(b + o_path);
    c->info.style = reinterpret_cast<uint32_t*>(b + o_style);
    c->info.sub_first = reinterpret_cast<uint32_t*>(b + o_sub);
    c->xform_buf = reinterpret_cast<uint32_t*>(b + o_xf);
    c->info.xform = nullptr;  // set per scene: only a scene with transforms records them
    c->info.curve_list = reinterpret_cast<uint32_t*>(b + o_clist);
    c->info.line_list = reinterpret_cast<uint32_t*>(b + o_llist);
    c->info.n_curves = reinterpret_cast<uint32_t*>(b + o_ncurve);
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
    pb.pieces = reinterpret_cast<PieceRec*>(b + o_pieces);
    pb.piece_item = reinterpret_cast<uint32_t*>(b + o_pitem);
    c->total = reinterpret_cast<uint64_t*>(b + o_total);
    c->items_total = reinterpret_cast<uint64_t*>(b + o_itot);
    pb.items_total = c->items_total;
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
    if (s->n_tags && (!s->tags || !s->styles)) return fail(c, SE_ERR_INVALID_ARG, "scene pointer is NULL");
    if (s->n_words && !s->words) return fail(c, SE_ERR_INVALID_ARG, "scene path data is NULL");
    if ((reinterpret_cast<uintptr_t>(s->tags) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "tags must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(s->words) & 3u) != 0) return fail(c, SE_ERR_INVALID_ARG, "path data must be 4-byte aligned");
    if (s->n_tags >= (1ull << 31) || s->n_words >= (1ull << 32))
        return fail(c, SE_ERR_INVALID_ARG, "more than 2^31 tags or 2^32 path data words");
    if (s->n_transforms && !s->transforms) return fail(c, SE_ERR_INVALID_ARG, "scene transform array is NULL");
    if ((reinterpret_cast<uintptr_t>(s->transforms) & 3u) != 0)
        return fail(c, SE_ERR_INVALID_ARG, "transforms must be 4-byte aligned");
    return SE_OK;
}

se_status check_params(se_ctx* c, const se_params* p) {
    if (!p) return fail(c, SE_ERR_INVALID_ARG, "params is NULL");
    if (!(p->tol > 0.0f) || !(p->fit_frac > 0.0f) || !(p->flat_frac > 0.0f))
        return fail(c, SE_ERR_INVALID_ARG, "tolerances must be positive");
    if (p->out_kind != SE_OUT_LINES && p->out_kind != SE_OUT_ARCS) return fail(c, SE_ERR_INVALID_ARG, "bad out_kind");
    if (p->refine > 1u) return fail(c, SE_ERR_INVALID_ARG, "refine is 0 or 1");
    return SE_OK;
}

// (Re)allocate the dash workspace for the scene and at least (tags, pts) output.
se_status ensure_dash(se_ctx* c, const se_scene_dev* s, uint64_t need_tags, uint64_t need_pts, uint64_t need_cuts) {
    DashWs& d = c->dash;
    uint64_t n = s->n_tags;
    uint64_t want_t = need_tags ? need_tags + need_tags / 4 : (4 * n > 4096 ? 4 * n : 4096);
    uint64_t want_p = need_pts ? need_pts + need_pts / 4 : (4 * s->n_words > 4096 ? 4 * s->n_words : 4096);
    uint64_t want_c = need_cuts ? need_cuts + need_cuts / 4 : (4 * n > 4096 ? 4 * n : 4096);
    bool inputs_fit = d.mem && n <= d.cap_in && s->n_paths <= d.cap_paths && s->n_styles <= d.cap_styles;
    bool output_fits = (need_tags == 0 || need_tags <= d.cap_tags) && (need_pts == 0 || need_pts <= d.cap_pts) &&
                       (need_cuts == 0 || need_cuts <= d.cap_cuts) && c->dash_slots_need <= d.cap_slots;
    if (inputs_fit && output_fits) return SE_OK;  // an undersized output is reported by se_sync
    if (c->capturing) return fail(c, SE_ERR_WORKSPACE, "dash workspace too small to capture: count the scene first");
    uint64_t cin = n > d.cap_in ? n + n / 4 : d.cap_in;
    uint32_t cpaths = s->n_paths > d.cap_paths ? s->n_paths : d.cap_paths;
    uint32_t cstyles = s->n_styles > d.cap_styles ? s->n_styles : d.cap_styles;
    uint64_t ct = want_t > d.cap_tags ? want_t : d.cap_tags;
    uint64_t cp = want_p > d.cap_pts ? want_p : d.cap_pts;
    uint64_t ccut = want_c > d.cap_cuts ? want_c : d.cap_cuts;
    if (ccut > (1ull << 34)) ccut = 1ull << 34;
    if (ct > (1ull << 31) - 1) ct = (1ull << 31) - 1;
    if (cp > (1ull << 32) - 1) cp = (1ull << 32) - 1;
    uint64_t tiles = (cin + kScanTile - 1) / kScanTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    size_t o_pt = take(cin * 4), o_path = take(cin * 4), o_style = take(cin * 4), o_sub = take(cin * 4);
    size_t o_len = take(cin * 4), o_pos = take(cin * 8), o_cnt = take(cin * 8), o_off = take((cin + 1) * 16);
    size_t o_ne = take(size_t(cpaths) * 4 + 4);
    size_t o_otags = take(ct + 16), o_opts = take(cp * 8 + 8), o_osty = take(size_t(cstyles) * sizeof(se_style) + 8);
    size_t o_outn = take(64);
    uint64_t cslot = need_cuts ? (d.cap_slots > 4096 ? d.cap_slots : 4096) : d.cap_slots;
    if (c->dash_slots_need > cslot) cslot = c->dash_slots_need + c->dash_slots_need / 4;
    if (cslot < 4096) cslot = 4096;
    size_t o_ncut = take(cin * 4), o_cutoff = take((cin + 1) * 16), o_cutt = take(ccut * 4 + 4);
    size_t o_panels = take(cslot * kPanelMax * sizeof(PanelPair)), o_npan = take(cslot * 4);
    size_t o_agg[4], o_incl[4];
    for (int k = 0; k < 4; k++) {
        o_agg[k] = take(tiles * kTagValBytes);  // the largest scan element (the tag scan's)
        o_incl[k] = take(tiles * kTagValBytes);
    }
    size_t control_bytes = (8 + 4 * tiles) * 4;
    size_t o_ctl = take(control_bytes);
    if (d.mem) {
        ctx_free(c, d.mem);
        d.mem = nullptr;
        d.cap_in = d.cap_tags = d.cap_pts = d.cap_cuts = 0;
        d.cap_paths = d.cap_styles = 0;
    }
    cudaError_t e = ctx_alloc(c, &d.mem, off);
    c->ws_gen++;
    if (e != cudaSuccess) {
        d.mem = nullptr;
        return fail(c, SE_ERR_OOM, "dash workspace allocation failed", e);
    }
    char* b = static_cast<char*>(d.mem);
    DashBufs& B = d.b;
    B.info.pt_base = reinterpret_cast<uint32_t*>(b + o_pt);
    B.info.path = reinterpret_cast<uint32_t*>(b + o_path);
    B.info.style = reinterpret_cast<uint32_t*>(b + o_style);
    B.info.sub_first = reinterpret_cast<uint32_t*>(b + o_sub);
    B.info.xform = nullptr;  // dash positions are measured before the transform
    B.info.curve_list = B.info.line_list = B.info.n_curves = nullptr;  // no plan pass on the input stream
    B.len = reinterpret_cast<float*>(b + o_len);
    B.end_pos = reinterpret_cast<long long*>(b + o_pos);
    B.cnt = reinterpret_cast<uint2*>(b + o_cnt);
    B.off = reinterpret_cast<ulonglong2*>(b + o_off);
    B.nonempty = reinterpret_cast<uint32_t*>(b + o_ne);
    B.out_tags = reinterpret_cast<uint8_t*>(b + o_otags);
    B.cap_tags = ct;
    B.out_pts = reinterpret_cast<float2*>(b + o_opts);
    B.cap_pts = cp;
    B.out_styles = reinterpret_cast<se_style*>(b + o_osty);
    B.out_n = reinterpret_cast<uint64_t*>(b + o_outn);
    B.ncut = reinterpret_cast<uint32_t*>(b + o_ncut);
    B.cut_off = reinterpret_cast<ulonglong2*>(b + o_cutoff);
    B.panels = reinterpret_cast<PanelPair*>(b + o_panels);
    B.n_panels = reinterpret_cast<uint32_t*>(b + o_npan);
    B.cap_slots = cslot;
    B.cut_t = reinterpret_cast<float*>(b + o_cutt);
    B.cap_cuts = ccut;
    d.control = reinterpret_cast<uint32_t*>(b + o_ctl);
    d.control_bytes = control_bytes;
    B.status = d.control;
    ScanState* sts[4] = {&d.tag_st, &d.seg_st, &d.out_st, &d.cut_st};
    for (int k = 0; k < 4; k++) {
        sts[k]->ticket = d.control + 1 + k;
        sts[k]->flags = d.control + 8 + k * tiles;
        sts[k]->agg = b + o_agg[k];
        sts[k]->incl = b + o_incl[k];
    }
    d.bytes = off;
    d.cap_in = cin;
    d.cap_paths = cpaths;
    d.cap_styles = cstyles;
    d.cap_tags = ct;
    d.cap_pts = cp;
    d.cap_cuts = ccut;
    d.cap_slots = cslot;
    return SE_OK;
}

// Enqueue the dash pass; *out receives the rewritten scene, whose tag count is
// the device value c->dash.b.out_n[0] (n_tags holds the capacity bound).
se_status run_dash(se_ctx* c, const se_scene_dev* s, se_scene_dev* out) {
    DashWs& d = c->dash;
    DashBufs& B = d.b;
    B.tags = s->tags;
    B.n_tags = s->n_tags;
    B.words = s->words;
    B.n_words = s->n_words;
    B.styles = s->styles;
    B.n_styles = s->n_styles;
    B.n_paths = s->n_paths;
    B.dashes = s->dashes;
    B.n_dashes = s->n_dashes;
    cudaError_t e = cudaMemsetAsync(d.control, 0, d.control_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.nonempty, 0, size_t(s->n_paths) * 4 + 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.out_n, 0, 64, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "memset", e);
    if (c->profile) cudaEventRecord(c->ev[6], c->stream);
    e = launch_dash(B, d.tag_st, d.seg_st, d.out_st, d.cut_st, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "dash launch", e);
    if (c->profile) cudaEventRecord(c->ev[7], c->stream);
    *out = se_scene_dev{};
    out->tags = B.out_tags;
    out->n_tags = d.cap_tags;
    out->words = reinterpret_cast<const uint32_t*>(B.out_pts);  // the rewrite is 32-bit: two words a point
    out->n_words = 2 * d.cap_pts;
    out->styles = B.out_styles;
    out->n_styles = s->n_styles;
    out->n_paths = s->n_paths;
    out->transforms = s->transforms;  // the rewrite is in the paths' own coordinates
    out->n_transforms = s->n_transforms;
    return SE_OK;
}

bool has_dashes(const se_scene_dev* s) { return s->n_dashes > 0 && s->dashes && s->n_tags > 0; }

ExpandArgs make_args(se_ctx* c, const se_scene_dev* s, const se_params* p) {
    ExpandArgs a{};
    a.tags = s->tags;
    a.n_tags = s->n_tags;
    a.words = s->words;
    a.n_words = s->n_words;
    a.styles = s->styles;
    a.n_styles = s->n_styles;
    a.xforms = s->n_transforms ? s->transforms : nullptr;
    a.n_xforms = s->n_transforms;
    a.info = c->info;
    a.info.xform = s->n_transforms ? c->xform_buf : nullptr;
    a.tol_fit = p->tol * p->fit_frac;
    a.tol_flat = p->tol * p->flat_frac;
    a.arcs = p->out_kind == SE_OUT_ARCS;
    a.refine = !a.arcs && p->refine != 0u;
    a.total = c->total;
    a.status = c->status;
    a.n_tags_dev = c->last_dashed ? c->dash.b.out_n : nullptr;
    a.dash_status = c->last_dashed ? c->dash.b.status : nullptr;
    return a;
}

void rec(se_ctx* c, int k) {
    if (c->profile) cudaEventRecord(c->ev[k], c->stream);
}

// tag scan, plan, item scan, decode, piece, primitive scan
se_status front_half(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* tag_offset,
                     uint64_t* path_offset, uint64_t capacity) {
    c->counted = false;  // the workspace is about to hold this run's results
    cudaError_t e = cudaMemsetAsync(c->control, 0, c->control_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->total, 0, 8, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->items_total, 0, 8, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "memset", e);
    if (c->profile && !c->last_dashed) {
        cudaEventRecord(c->ev[6], c->stream);
        cudaEventRecord(c->ev[7], c->stream);
    }
    if (s->n_tags == 0) {
        if (path_offset) e = cudaMemsetAsync(path_offset, 0, 8ull * (s->n_paths + 1), c->stream);
        if (e == cudaSuccess && tag_offset) e = cudaMemsetAsync(tag_offset, 0, 8, c->stream);
        return e == cudaSuccess ? SE_OK : fail(c, SE_ERR_CUDA, "memset", e);
    }
    ExpandArgs a = make_args(c, s, p);
    a.capacity = capacity;
    rec(c, 0);
    e = launch_tag_scan(s->tags, s->n_tags, a.n_tags_dev, a.info, c->scan_tags, c->status, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "tag scan launch", e);
    rec(c, 1);
    e = launch_plan(a, c->pb, c->tune, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "plan launch", e);
    rec(c, 2);
    e = launch_item_scan(a, c->pb, c->scan_items, c->stream);
    if (e == cudaSuccess) e = launch_decode(a, c->pb, c->tune, c->stream);
    if (e == cudaSuccess) e = launch_piece(a, c->pb, c->tune, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "piece launch", e);
    rec(c, 3);
    e = launch_prim_scan(a, c->pb, tag_offset, path_offset, s->n_paths, c->scan_prims, c->stream);
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
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_items, c->items_total, 8, cudaMemcpyDeviceToHost, c->stream);
    c->h_status[1] = 0;
    if (e == cudaSuccess && c->last_dashed) {
        e = cudaMemcpyAsync(c->h_status + 1, c->dash.b.status, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_dash, c->dash.b.out_n, 48, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "sync", e);
    if (n_prims) *n_prims = *c->h_total;
    if (n_items) *n_items = c->last_tags ? *c->h_items : 0;
    se_status st = map_status(c->h_status[0] | c->h_status[1]);
    if (st != SE_OK) fail(c, st, "device status");
    return st;
}

}  // namespace

se_status se_fail(se_ctx* c, se_status st, const char* what, cudaError_t e) {
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
        }
    }
    return st;
}

extern "C" se_status se_ctx_create(int device, void* cuda_stream, se_alloc_fn alloc_fn, se_free_fn free_fn,
                                   void* user, se_ctx** out) {
    if (!out) return SE_ERR_INVALID_ARG;
    *out = nullptr;
    if ((alloc_fn == nullptr) != (free_fn == nullptr)) return SE_ERR_INVALID_ARG;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) return SE_ERR_INVALID_ARG;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return SE_ERR_CUDA;
    se_ctx* c = new (std::nothrow) se_ctx();
    if (!c) return SE_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->alloc_fn = alloc_fn;
    c->free_fn = free_fn;
    c->alloc_user = user;
    e = cudaMallocHost(reinterpret_cast<void**>(&c->h_total), 128);
    if (e != cudaSuccess) {
        delete c;
        return SE_ERR_OOM;
    }
    c->h_status = reinterpret_cast<uint32_t*>(c->h_total + 1);
    c->h_items = c->h_total + 2;
    c->h_dash = c->h_total + 3;
    *out = c;
    return SE_OK;
}

extern "C" se_status se_ctx_destroy(se_ctx* c) {
    if (!c) return SE_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    ctx_free(c, c->ws);
    ctx_free(c, c->dash.mem);
    ctx_free(c, c->io);
    cudaStreamSynchronize(c->stream);
    if (c->h_total) cudaFreeHost(c->h_total);
    if (c->h_bounds) cudaFreeHost(c->h_bounds);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : c->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    delete c;
    return SE_OK;
}

extern "C" const char* se_ctx_last_error(const se_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

// Everything of an expansion but the emit: validation, the dash pass, the
// workspace, and the front half; `a` receives the arguments of the emit.  `emit`
// is false when there is nothing to emit (an empty scene).
static se_status expand_front(se_ctx* c, const se_scene_dev* s, const se_params* p, const se_outline_dev* out,
                       ExpandArgs& a, bool& emit) {
    emit = false;
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    if (!out || (out->capacity && !out->prims)) return fail(c, SE_ERR_INVALID_ARG, "outline buffers are NULL");
    if ((reinterpret_cast<uintptr_t>(out->prims) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "prims must be 16-byte aligned");
    if (p->out_kind == SE_OUT_ARCS && out->capacity && !out->curvature)
        return fail(c, SE_ERR_INVALID_ARG, "arc output needs a curvature buffer");
    cudaSetDevice(c->device);
    se_scene_dev rs;
    const se_scene_dev* sx = s;
    c->last_dashed = has_dashes(s);
    c->last_input_tags = s->n_tags;
    if (c->last_dashed) {
        st = ensure_dash(c, s, 0, 0, 0);
        if (st == SE_OK) st = run_dash(c, s, &rs);
        if (st != SE_OK) return st;
        sx = &rs;
    }
    st = ensure_workspace(c, sx->n_tags, 0);
    if (st != SE_OK) return st;
    c->last_tags = sx->n_tags;
    st = front_half(c, sx, p, out->tag_offset, out->path_offset, out->capacity);
    if (st != SE_OK || sx->n_tags == 0) return st;
    a = make_args(c, sx, p);
    a.capacity = out->capacity;
    a.prims = reinterpret_cast<float4*>(out->prims);
    a.curvature = p->out_kind == SE_OUT_ARCS ? out->curvature : nullptr;
    a.path_id = out->path_id;
    emit = true;
    return SE_OK;
}

extern "C" se_status se_expand(se_ctx* c, const se_scene_dev* s, const se_params* p, const se_outline_dev* out) {
    if (!c) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    ExpandArgs a;
    bool emit = false;
    se_status st = expand_front(c, s, p, out, a, emit);
    if (st != SE_OK || !emit) return st;
    cudaError_t e = launch_emit(a, c->pb, c->tune, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "emit launch", e);
    if (c->profile) {
        cudaEventRecord(c->ev[5], c->stream);
        c->profiled = true;
    }
    return SE_OK;
}

extern "C" se_status se_count(se_ctx* c, const se_scene_dev* s, const se_params* p, uint64_t* n_prims) {
    if (!c || !n_prims) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    cudaSetDevice(c->device);
    uint64_t need = 0, need_t = 0, need_p = 0, need_c = 0;
    c->last_dashed = has_dashes(s);
    c->last_input_tags = s->n_tags;
    for (int attempt = 0; attempt < 3; attempt++) {
        se_scene_dev rs;
        const se_scene_dev* sx = s;
        if (c->last_dashed) {
            st = ensure_dash(c, s, need_t, need_p, need_c);
            if (st == SE_OK) st = run_dash(c, s, &rs);
            if (st != SE_OK) return st;
            sx = &rs;
        }
        st = ensure_workspace(c, sx->n_tags, need);
        if (st != SE_OK) return st;
        c->last_tags = sx->n_tags;
        st = front_half(c, sx, p, nullptr, nullptr, ~0ull);
        if (st != SE_OK) return st;
        st = read_back(c, n_prims, &need);
        if (st == SE_OK || st == SE_ERR_LIMIT) {
            c->counted = true;
            c->counted_scene = *s;
            c->counted_params = *p;
            c->counted_gen = c->ws_gen;
        }
        if (st != SE_ERR_WORKSPACE) return st;
        if (c->last_dashed && (c->h_dash[2] > c->dash.cap_tags || c->h_dash[3] > c->dash.cap_pts ||
                               c->h_dash[4] > c->dash.cap_cuts || c->h_dash[5] > c->dash.cap_slots)) {
            need_t = c->h_dash[2];
            need_p = c->h_dash[3];
            need_c = c->h_dash[4];
            c->dash_slots_need = c->h_dash[5];
            if (need_t >= (1ull << 31) || need_p >= (1ull << 32))
                return fail(c, SE_ERR_INVALID_INPUT, "the dashed scene has more than 2^31 tags or 2^32 points");
        }
    }
    return st;
}

static bool same_scene(const se_scene_dev& a, const se_scene_dev& b) {
    return a.tags == b.tags && a.n_tags == b.n_tags && a.words == b.words && a.n_words == b.n_words &&
           a.styles == b.styles && a.n_styles == b.n_styles && a.n_paths == b.n_paths && a.dashes == b.dashes &&
           a.n_dashes == b.n_dashes && a.transforms == b.transforms && a.n_transforms == b.n_transforms;
}

static bool same_params(const se_params& a, const se_params& b) {
    return a.tol == b.tol && a.fit_frac == b.fit_frac && a.flat_frac == b.flat_frac && a.out_kind == b.out_kind &&
           a.refine == b.refine;
}

extern "C" se_status se_expand_counted(se_ctx* c, const se_scene_dev* s, const se_params* p,
                                       const se_outline_dev* out) {
    if (!c) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    se_status st = check_scene(c, s);
    if (st == SE_OK) st = check_params(c, p);
    if (st != SE_OK) return st;
    if (!out || (out->capacity && !out->prims)) return fail(c, SE_ERR_INVALID_ARG, "outline buffers are NULL");
    if ((reinterpret_cast<uintptr_t>(out->prims) & 15u) != 0) return fail(c, SE_ERR_INVALID_ARG, "prims must be 16-byte aligned");
    if (p->out_kind == SE_OUT_ARCS && out->capacity && !out->curvature)
        return fail(c, SE_ERR_INVALID_ARG, "arc output needs a curvature buffer");
    if (!c->counted || c->counted_gen != c->ws_gen || !same_scene(c->counted_scene, *s) ||
        !same_params(c->counted_params, *p))
        return fail(c, SE_ERR_INVALID_ARG, "no se_count of this scene and params precedes the expansion");
    c->counted = false;  // once per count: the primitive scan below overwrites its offsets
    cudaSetDevice(c->device);
    se_scene_dev rs;
    const se_scene_dev* sx = s;
    if (c->last_dashed) {
        // the rewritten scene of the count's dash pass, still in the dash workspace
        rs = se_scene_dev{};
        rs.tags = c->dash.b.out_tags;
        rs.n_tags = c->dash.cap_tags;
        rs.words = reinterpret_cast<const uint32_t*>(c->dash.b.out_pts);
        rs.n_words = 2 * c->dash.cap_pts;
        rs.styles = c->dash.b.out_styles;
        rs.n_styles = s->n_styles;
        rs.n_paths = s->n_paths;
        rs.transforms = s->transforms;
        rs.n_transforms = s->n_transforms;
        sx = &rs;
    }
    if (sx->n_tags == 0) {
        cudaError_t e = cudaSuccess;
        if (out->path_offset) e = cudaMemsetAsync(out->path_offset, 0, 8ull * (s->n_paths + 1), c->stream);
        if (e == cudaSuccess && out->tag_offset) e = cudaMemsetAsync(out->tag_offset, 0, 8, c->stream);
        return e == cudaSuccess ? SE_OK : fail(c, SE_ERR_CUDA, "memset", e);
    }
    ExpandArgs a = make_args(c, sx, p);
    a.capacity = out->capacity;
    a.prims = reinterpret_cast<float4*>(out->prims);
    a.curvature = p->out_kind == SE_OUT_ARCS ? out->curvature : nullptr;
    a.path_id = out->path_id;
    // restart the primitive scan: its ticket and tile flags (the status word keeps the count's bits)
    const uint64_t tt = (c->cap_tags + kScanTile - 1) / kScanTile, ti = (c->item_cap + kScanTile - 1) / kScanTile;
    cudaError_t e = cudaMemsetAsync(c->scan_prims.ticket, 0, 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->scan_prims.flags, 0, ti * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->total, 0, 8, c->stream);
    (void)tt;
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "memset", e);
    rec(c, 0);
    rec(c, 1);
    rec(c, 2);
    rec(c, 3);
    e = launch_prim_scan(a, c->pb, out->tag_offset, out->path_offset, s->n_paths, c->scan_prims, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "primitive scan launch", e);
    rec(c, 4);
    e = launch_emit(a, c->pb, c->tune, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "emit launch", e);
    if (c->profile) {
        cudaEventRecord(c->ev[5], c->stream);
        if (!c->last_dashed) {
            cudaEventRecord(c->ev[6], c->stream);
            cudaEventRecord(c->ev[7], c->stream);
        }
        c->profiled = true;
    }
    return SE_OK;
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

extern "C" se_status se_expand_host(se_ctx* c, const uint8_t* tags, uint64_t n_tags, const uint32_t* words,
                                    uint64_t n_words, const se_style* styles, uint32_t n_styles, uint32_t n_paths,
                                    const float* dashes, uint32_t n_dashes, const float* transforms,
                                    uint32_t n_transforms, const se_params* p, float* host_prims,
                                    float* host_curvature, uint64_t capacity, uint64_t* n_prims) {
    if (!c || !n_prims || (n_tags && (!tags || !styles)) || (n_words && !words) || (capacity && !host_prims) ||
        (n_transforms && !transforms))
        return SE_ERR_INVALID_ARG;
    settle_pending(c);
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
    size_t o_tags = take(n_tags + 16), o_pts = take(n_words * 4 + 8), o_sty = take(size_t(n_styles) * sizeof(se_style) + 8);
    size_t o_xf = take(size_t(n_transforms) * 24 + 4), o_bounds = take(3 * 17 * 8);
    size_t o_dash = take(size_t(n_dashes) * 4 + 4), o_prims = take(capacity * 16 + 16), o_curv = take(arcs ? capacity * 4 + 4 : 4);
    if (off > c->io_bytes) {
        ctx_free(c, c->io);
        c->io = nullptr;
        c->io_bytes = 0;
        cudaError_t e = ctx_alloc(c, &c->io, off);
        if (e != cudaSuccess) {
            c->io = nullptr;
            return fail(c, SE_ERR_OOM, "host-path buffers", e);
        }
        c->io_bytes = off;
    }
    char* b = static_cast<char*>(c->io);
    cudaError_t e = cudaSuccess;
    if (n_tags) e = cudaMemcpyAsync(b + o_tags, tags, n_tags, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_words) e = cudaMemcpyAsync(b + o_pts, words, n_words * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_styles)
        e = cudaMemcpyAsync(b + o_sty, styles, size_t(n_styles) * sizeof(se_style), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_dashes) e = cudaMemcpyAsync(b + o_dash, dashes, size_t(n_dashes) * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_transforms)
        e = cudaMemcpyAsync(b + o_xf, transforms, size_t(n_transforms) * 24, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "upload", e);
    se_scene_dev s{};
    s.tags = reinterpret_cast<const uint8_t*>(b + o_tags);
    s.n_tags = n_tags;
    s.words = reinterpret_cast<const uint32_t*>(b + o_pts);
    s.n_words = n_words;
    s.styles = reinterpret_cast<const se_style*>(b + o_sty);
    s.n_styles = n_styles;
    s.n_paths = n_paths;
    s.dashes = n_dashes ? reinterpret_cast<const float*>(b + o_dash) : nullptr;
    s.n_dashes = n_dashes;
    s.transforms = n_transforms ? reinterpret_cast<const float*>(b + o_xf) : nullptr;
    s.n_transforms = n_transforms;
    se_outline_dev o{};
    o.prims = reinterpret_cast<float*>(b + o_prims);
    o.curvature = arcs ? reinterpret_cast<float*>(b + o_curv) : nullptr;
    o.capacity = capacity;
    // Large scenes download while they are emitted: the emit runs as kChunks tag
    // ranges, and a copy stream brings each range's primitives (a contiguous block
    // of the outline) to the host while the next range is emitted.  Six ranges
    // measured best on the map-like scene (end to end 5.26 ms; 4: 5.37, 8: 5.31,
    // 12: 5.50, 16: 5.68): fewer leave a longer last copy, more add emit tails.
    const uint32_t kChunks = n_tags >= 65536 ? 6u : 1u;
    ExpandArgs a;
    bool emit = false;
    st = expand_front(c, &s, p, &o, a, emit);
    if (st != SE_OK) return st;
    uint64_t* d_bounds = reinterpret_cast<uint64_t*>(b + o_bounds);
    if (emit) {
        e = launch_chunk_bounds(a, c->pb, kChunks, d_bounds, c->stream);
        if (e == cudaSuccess && !c->h_bounds) e = cudaMallocHost(&c->h_bounds, 3 * 17 * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_bounds, d_bounds, 3 * (kChunks + 1) * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "chunk bounds", e);
    }
    uint64_t n = 0;
    st = read_back(c, &n, nullptr);  // waits for the front half
    *n_prims = n;
    if (st != SE_OK && st != SE_ERR_LIMIT) return st;
    if (!emit || n == 0) return st;
    if (!c->copy_stream) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    for (uint32_t k = 0; e == cudaSuccess && k < kChunks; k++)
        if (!c->chunk_ev[k]) e = cudaEventCreateWithFlags(&c->chunk_ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "download stream", e);
    const uint64_t* hb = c->h_bounds;
    for (uint32_t k = 0; k < kChunks && e == cudaSuccess; k++) {
        ExpandArgs ak = a;
        ak.emit_tag_lo = hb[3 * k];
        ak.emit_tag_hi = hb[3 * k + 3];
        ak.emit_piece_lo = hb[3 * k + 1];
        ak.emit_piece_hi = hb[3 * k + 4];
        e = launch_emit(ak, c->pb, c->tune, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->chunk_ev[k], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->chunk_ev[k], 0);
        const uint64_t lo = hb[3 * k + 2], hi = hb[3 * k + 5] < n ? hb[3 * k + 5] : n;
        if (e == cudaSuccess && hi > lo) {
            e = cudaMemcpyAsync(host_prims + 4 * lo, b + o_prims + 16 * lo, (hi - lo) * 16, cudaMemcpyDeviceToHost,
                                c->copy_stream);
            if (e == cudaSuccess && arcs)
                e = cudaMemcpyAsync(host_curvature + lo, b + o_curv + 4 * lo, (hi - lo) * 4, cudaMemcpyDeviceToHost,
                                    c->copy_stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "download", e);
    return st;
}

namespace se {
cudaError_t launch_offsets_with_state(const uint32_t* counts, uint64_t n, uint64_t* offsets, ScanState st,
                                      uint32_t* status, cudaStream_t s);
cudaError_t launch_bulk_wait_probe(const void* src, uint32_t copy, uint32_t limit, uint32_t* status, cudaStream_t s);
}

extern "C" se_status se_debug_scan_timeout(se_ctx* c, uint64_t n, uint32_t spin_limit) {
    if (!c || n <= kScanTile || n >= (1ull << 32) || spin_limit == 0) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    cudaSetDevice(c->device);
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_cnt = take(n * 4), o_off = take((n + 1) * 8), o_ctl = take((4 + tiles) * 4);
    const size_t o_agg = take(tiles * 8), o_incl = take(tiles * 8);
    void* mem = nullptr;
    cudaError_t e = ctx_alloc(c, &mem, off);
    if (e != cudaSuccess) return fail(c, SE_ERR_OOM, "scratch allocation failed", e);
    char* b = static_cast<char*>(mem);
    uint32_t* ctl = reinterpret_cast<uint32_t*>(b + o_ctl);  // [status, ticket, pad, pad, flags...]
    static const uint32_t kFirstTicket = 1u;                  // tile 0 is never taken
    e = cudaMemsetAsync(b, 0, off, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl + 1, &kFirstTicket, 4, cudaMemcpyHostToDevice, c->stream);
    ScanState st;
    st.flags = ctl + 4;
    st.agg = b + o_agg;
    st.incl = b + o_incl;
    st.ticket = ctl + 1;
    st.spin_limit = spin_limit;
    if (e == cudaSuccess)
        e = launch_offsets_with_state(reinterpret_cast<const uint32_t*>(b + o_cnt), n,
                                      reinterpret_cast<uint64_t*>(b + o_off), st, ctl, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_status, ctl, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const uint32_t status = c->h_status[0];
    ctx_free(c, mem);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "timeout probe", e);
    if (status & kStatusTimeout) return fail(c, SE_ERR_TIMEOUT, "a bounded look-back wait gave up");
    return SE_OK;
}

extern "C" se_status se_debug_bulk_timeout(se_ctx* c, uint32_t spin_limit, int copy) {
    if (!c || spin_limit == 0) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    cudaSetDevice(c->device);
    void* mem = nullptr;
    cudaError_t e = ctx_alloc(c, &mem, 512);  // [0, 256): the copy's source; 256: the status word
    if (e != cudaSuccess) return fail(c, SE_ERR_OOM, "scratch allocation failed", e);
    char* b = static_cast<char*>(mem);
    uint32_t* status = reinterpret_cast<uint32_t*>(b + 256);
    e = cudaMemsetAsync(b, 0x5a, 256, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, c->stream);
    if (e == cudaSuccess) e = launch_bulk_wait_probe(b, copy ? 1u : 0u, spin_limit, status, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_status, status, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const uint32_t st = c->h_status[0];
    ctx_free(c, mem);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "bulk wait probe", e);
    if (st & kStatusTimeout) return fail(c, SE_ERR_TIMEOUT, "a bounded bulk-copy wait gave up");
    if (st & kStatusBadTag) return fail(c, SE_ERR_CUDA, "bulk copy delivered wrong bytes");
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
    cudaError_t e = cudaEventSynchronize(c->ev[5]);
    for (int k = 0; k < 5 && e == cudaSuccess; k++) e = cudaEventElapsedTime(&ms[k], c->ev[k], c->ev[k + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[5], c->ev[6], c->ev[7]);
    if (e != cudaSuccess) return fail(c, SE_ERR_CUDA, "event read", e);
    return SE_OK;
}

extern "C" se_status se_ctx_stats(se_ctx* c, se_stats* out) {
    if (!c || !out) return SE_ERR_INVALID_ARG;
    out->n_tags = c->last_tags;
    out->n_input_tags = c->last_input_tags;
    out->n_items = 0;
    out->n_prims = 0;
    out->piece_bytes = (uint32_t)sizeof(PieceRec);
    out->tail_bytes = (uint32_t)sizeof(TailRec);
    out->workspace_bytes = c->ws_bytes;
    if (!c->ws) return SE_OK;
    cudaSetDevice(c->device);
    se_status st = read_back(c, &out->n_prims, &out->n_items);
    if (c->last_dashed) out->n_tags = c->h_dash[0];
    return st == SE_ERR_CUDA ? st : SE_OK;
}
