// Library-owned scenes and outlines: the object form of the boundary.
//
// A scene is either built path by path (the SVG-style builder: path_begin
// with a style, move_to / line_to / cubic_to / close, path_end) or made from
// already encoded streams; se_scene_upload encodes a built scene on the host
// (Section 8.2) and copies it to the context's device.  se_scene_expand counts
// the scene (a synchronisation), allocates a library-owned outline of exactly
// that size and enqueues the expansion; se_outline_sync waits for it.  A batch
// of scenes expands as one scene (se_batch_*) into one buffer that the
// returned outlines share, each seeing its own document's range.
#include <cuda_runtime.h>

#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "ctx.h"

struct se_scene {
    se_ctx* ctx = nullptr;
    // builder (verbs) or encoded streams
    bool from_streams = false;
    bool in_path = false;
    std::vector<uint8_t> verbs;
    std::vector<float> pts;
    std::vector<uint32_t> path_verb_off{0};
    std::vector<se_style> path_styles;
    std::vector<float> path_xforms;  // 6 per path (builder)
    float cur_xform[6] = {1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
    bool any_xform = false;
    bool cur_coord16 = false;
    std::vector<uint8_t> path_coord16;  // per path: 16-bit coordinates asked for
    std::vector<float> dashes;
    std::vector<float> xforms;       // encoded transform stream (6 per entry)
    // encoded host streams
    std::vector<uint8_t> tags;
    std::vector<uint32_t> words;     // encoded path data stream
    std::vector<se_style> styles;
    uint32_t n_paths = 0;
    // device copy
    void* dmem = nullptr;
    se_scene_dev dev{};
    bool uploaded = false;
};

namespace {

// Device memory shared by the outlines of one expansion (one scene, or every
// document of a batch).
struct OutlineBuf {
    se_ctx* ctx = nullptr;
    void* mem = nullptr;
    float* prims = nullptr;
    float* curvature = nullptr;
    uint64_t* path_offset = nullptr;
    uint64_t capacity = 0;
    uint32_t n_paths = 0;
    bool synced = false;
    se_status status = SE_OK;
    uint64_t n_prims = 0;
    std::vector<uint64_t> h_path_offset;  // after sync: the whole path-offset array
    ~OutlineBuf() {
        if (mem) ctx_free(ctx, mem);
    }
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct se_outline {
    std::shared_ptr<OutlineBuf> buf;
    uint64_t path_first = 0, path_end = 0;  // this outline's paths of the shared buffer
    bool arcs = false;
};

namespace {

se_status builder_check(se_scene* s, bool need_path) {
    if (!s) return SE_ERR_INVALID_ARG;
    if (s->from_streams || s->uploaded) return se_fail(s->ctx, SE_ERR_INVALID_ARG, "the scene is no longer being built");
    if (need_path != s->in_path) return se_fail(s->ctx, SE_ERR_INVALID_ARG, need_path ? "no open path" : "a path is open");
    return SE_OK;
}

se_status push_verb(se_scene* s, uint8_t v, const float* p, int n) {
    se_status st = builder_check(s, true);
    if (st != SE_OK) return st;
    for (int k = 0; k < 2 * n; k++)
        if (!(p[k] == p[k]) || p[k] - p[k] != 0.0f) return se_fail(s->ctx, SE_ERR_INVALID_INPUT, "non-finite coordinate");
    if (v != SE_VERB_MOVE && s->verbs.size() == s->path_verb_off.back())
        return se_fail(s->ctx, SE_ERR_INVALID_INPUT, "a path starts with move_to");
    s->verbs.push_back(v);
    s->pts.insert(s->pts.end(), p, p + 2 * n);
    return SE_OK;
}

// one expansion of `s` into a fresh buffer (count, allocate, enqueue)
se_status expand_into(se_ctx* c, const se_scene_dev* scene, const se_params* p, uint64_t n_prims, uint32_t n_paths,
                      std::shared_ptr<OutlineBuf>& out, se_status (*launch)(void*, const se_params*, const se_outline_dev*),
                      void* arg) {
    auto b = std::make_shared<OutlineBuf>();
    b->ctx = c;
    b->capacity = n_prims;
    b->n_paths = n_paths;
    const bool arcs = p->out_kind == SE_OUT_ARCS;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = al256(o + bytes);
        return r;
    };
    size_t o_prims = take(n_prims * 16 + 16), o_curv = take(arcs ? n_prims * 4 + 4 : 0);
    size_t o_poff = take((n_paths + 1ull) * 8);
    cudaError_t e = ctx_alloc(c, &b->mem, o);
    if (e != cudaSuccess) {
        b->mem = nullptr;
        return se_fail(c, SE_ERR_OOM, "outline allocation failed", e);
    }
    char* m = static_cast<char*>(b->mem);
    b->prims = reinterpret_cast<float*>(m + o_prims);
    b->curvature = arcs ? reinterpret_cast<float*>(m + o_curv) : nullptr;
    b->path_offset = reinterpret_cast<uint64_t*>(m + o_poff);
    se_outline_dev od{};
    od.prims = b->prims;
    od.curvature = b->curvature;
    od.path_offset = b->path_offset;
    od.capacity = n_prims;
    se_status st = launch ? launch(arg, p, &od) : se_expand(c, scene, p, &od);
    if (st != SE_OK) return st;
    out = b;
    return SE_OK;
}

se_status sync_buf(OutlineBuf& b) {
    if (b.synced) return b.status;
    uint64_t n = 0;
    se_status st = se_sync(b.ctx, &n);
    b.n_prims = n;
    b.status = st;
    if (st == SE_OK || st == SE_ERR_LIMIT) {
        b.h_path_offset.resize(b.n_paths + 1ull);
        cudaError_t e = cudaMemcpy(b.h_path_offset.data(), b.path_offset, (b.n_paths + 1ull) * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) b.status = se_fail(b.ctx, SE_ERR_CUDA, "path offsets", e);
    }
    b.synced = true;
    return b.status;
}

// The context's read-back (count, status) describes `b` until `b` is
// synchronised: the next expansion on the context synchronises it first.
void hold_readback(se_ctx* c, const std::shared_ptr<OutlineBuf>& b) {
    std::weak_ptr<OutlineBuf> w = b;
    c->settle = [w] {
        if (std::shared_ptr<OutlineBuf> p = w.lock()) sync_buf(*p);
    };
}

se_status batch_launch(void* batch, const se_params* p, const se_outline_dev* od) {
    return se_batch_expand(static_cast<se_batch*>(batch), p, od);
}

}  // namespace

// --------------------------------------------------------------------------- scenes

extern "C" se_status se_scene_begin(se_ctx* ctx, se_scene** out) {
    if (!ctx || !out) return SE_ERR_INVALID_ARG;
    se_scene* s = new (std::nothrow) se_scene();
    if (!s) return SE_ERR_OOM;
    s->ctx = ctx;
    *out = s;
    return SE_OK;
}

extern "C" se_status se_path_begin(se_scene* s, const se_style* style) {
    se_status st = builder_check(s, false);
    if (st != SE_OK) return st;
    if (!style) return se_fail(s->ctx, SE_ERR_INVALID_ARG, "style is NULL");
    s->path_styles.push_back(*style);
    s->path_xforms.insert(s->path_xforms.end(), s->cur_xform, s->cur_xform + 6);
    s->path_coord16.push_back(s->cur_coord16 ? 1 : 0);
    s->in_path = true;
    return SE_OK;
}

extern "C" se_status se_set_transform(se_scene* s, const float* m) {
    se_status st = builder_check(s, false);
    if (st != SE_OK) return st;
    static const float id[6] = {1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f};
    const float* v = m ? m : id;
    for (int k = 0; k < 6; k++)
        if (!(v[k] == v[k]) || v[k] - v[k] != 0.0f) return se_fail(s->ctx, SE_ERR_INVALID_INPUT, "non-finite transform");
    for (int k = 0; k < 6; k++) s->cur_xform[k] = v[k];
    if (m) s->any_xform = true;
    return SE_OK;
}

extern "C" se_status se_move_to(se_scene* s, float x, float y) {
    const float p[2] = {x, y};
    return push_verb(s, SE_VERB_MOVE, p, 1);
}

extern "C" se_status se_line_to(se_scene* s, float x, float y) {
    const float p[2] = {x, y};
    return push_verb(s, SE_VERB_LINE, p, 1);
}

extern "C" se_status se_cubic_to(se_scene* s, float x1, float y1, float x2, float y2, float x3, float y3) {
    const float p[6] = {x1, y1, x2, y2, x3, y3};
    return push_verb(s, SE_VERB_CUBIC, p, 3);
}

extern "C" se_status se_set_coord16(se_scene* s, int enable) {
    se_status st = builder_check(s, false);
    if (st != SE_OK) return st;
    s->cur_coord16 = enable != 0;
    return SE_OK;
}

extern "C" se_status se_quad_to(se_scene* s, float x1, float y1, float x2, float y2) {
    const float p[4] = {x1, y1, x2, y2};
    return push_verb(s, SE_VERB_QUAD, p, 2);
}

extern "C" se_status se_close(se_scene* s) { return push_verb(s, SE_VERB_CLOSE, nullptr, 0); }

extern "C" se_status se_path_end(se_scene* s) {
    se_status st = builder_check(s, true);
    if (st != SE_OK) return st;
    s->path_verb_off.push_back((uint32_t)s->verbs.size());
    s->in_path = false;
    return SE_OK;
}

extern "C" se_status se_dash_pattern(se_scene* s, const float* lens, uint32_t n, uint32_t* first_out) {
    if (!s || (n && !lens) || !first_out) return SE_ERR_INVALID_ARG;
    if (s->from_streams || s->uploaded) return se_fail(s->ctx, SE_ERR_INVALID_ARG, "the scene is no longer being built");
    for (uint32_t k = 0; k < n; k++)
        if (!(lens[k] >= 0.0f) || lens[k] - lens[k] != 0.0f) return se_fail(s->ctx, SE_ERR_INVALID_INPUT, "bad dash length");
    *first_out = (uint32_t)s->dashes.size();
    s->dashes.insert(s->dashes.end(), lens, lens + n);
    return SE_OK;
}

extern "C" se_status se_scene_from_streams(se_ctx* ctx, const uint8_t* tags, size_t n_tags, const uint32_t* words,
                                           size_t n_words, const se_style* styles, size_t n_styles, uint32_t n_paths,
                                           const float* dashes, size_t n_dash, const float* transforms,
                                           size_t n_transforms, se_scene** out) {
    if (!ctx || !out || (n_tags && (!tags || !styles)) || (n_words && !words) || (n_dash && !dashes) ||
        (n_transforms && !transforms))
        return SE_ERR_INVALID_ARG;
    se_scene* s = new (std::nothrow) se_scene();
    if (!s) return SE_ERR_OOM;
    s->ctx = ctx;
    s->from_streams = true;
    s->tags.assign(tags, tags + n_tags);
    s->words.assign(words, words + n_words);
    s->styles.assign(styles, styles + n_styles);
    s->dashes.assign(dashes, dashes + n_dash);
    s->xforms.assign(transforms, transforms + 6 * n_transforms);
    s->n_paths = n_paths;
    *out = s;
    return SE_OK;
}

extern "C" se_status se_scene_upload(se_scene* s) {
    if (!s) return SE_ERR_INVALID_ARG;
    if (s->uploaded) return SE_OK;
    se_ctx* c = s->ctx;
    if (s->in_path) return se_fail(c, SE_ERR_INVALID_ARG, "a path is open");
    if (!s->from_streams) {
        uint32_t n_paths = (uint32_t)s->path_styles.size();
        uint64_t n_tags = 0, n_words = 0;
        se_status st = se_encode_size(s->verbs.data(), s->verbs.size(), s->pts.data(), s->pts.size() / 2,
                                      s->path_verb_off.data(), n_paths, s->path_styles.data(),
                                      s->path_coord16.data(), &n_tags, &n_words);
        if (st != SE_OK) return se_fail(c, st, "encoding failed");
        s->tags.resize(n_tags);
        s->words.resize(n_words);
        s->styles.resize(n_paths);
        uint32_t n_styles = 0, n_xf = 0;
        s->xforms.resize(s->any_xform ? 6ull * n_paths : 0);
        st = se_encode(s->verbs.data(), s->verbs.size(), s->pts.data(), s->pts.size() / 2, s->path_verb_off.data(),
                       n_paths, s->path_styles.data(), s->any_xform ? s->path_xforms.data() : nullptr,
                       s->path_coord16.data(), s->tags.data(), s->words.data(), s->styles.data(), &n_styles,
                       s->any_xform ? s->xforms.data() : nullptr, &n_xf);
        if (st != SE_OK) return se_fail(c, st, "encoding failed");
        s->xforms.resize(6ull * n_xf);
        s->styles.resize(n_styles);
        s->n_paths = n_paths;
    }
    cudaSetDevice(c->device);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = al256(o + bytes);
        return r;
    };
    size_t o_tags = take(s->tags.size() + 16), o_pts = take(s->words.size() * 4 + 8);
    size_t o_sty = take(s->styles.size() * sizeof(se_style) + 8), o_dash = take(s->dashes.size() * 4 + 4);
    size_t o_xf = take(s->xforms.size() * 4 + 4);
    cudaError_t e = ctx_alloc(c, &s->dmem, o);
    if (e != cudaSuccess) {
        s->dmem = nullptr;
        return se_fail(c, SE_ERR_OOM, "scene allocation failed", e);
    }
    char* m = static_cast<char*>(s->dmem);
    if (!s->tags.empty()) e = cudaMemcpyAsync(m + o_tags, s->tags.data(), s->tags.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !s->words.empty())
        e = cudaMemcpyAsync(m + o_pts, s->words.data(), s->words.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !s->styles.empty())
        e = cudaMemcpyAsync(m + o_sty, s->styles.data(), s->styles.size() * sizeof(se_style), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess && !s->dashes.empty())
        e = cudaMemcpyAsync(m + o_dash, s->dashes.data(), s->dashes.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !s->xforms.empty())
        e = cudaMemcpyAsync(m + o_xf, s->xforms.data(), s->xforms.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "scene upload", e);
    s->dev.tags = reinterpret_cast<const uint8_t*>(m + o_tags);
    s->dev.n_tags = s->tags.size();
    s->dev.words = reinterpret_cast<const uint32_t*>(m + o_pts);
    s->dev.n_words = s->words.size();
    s->dev.styles = reinterpret_cast<const se_style*>(m + o_sty);
    s->dev.n_styles = (uint32_t)s->styles.size();
    s->dev.n_paths = s->n_paths;
    s->dev.dashes = s->dashes.empty() ? nullptr : reinterpret_cast<const float*>(m + o_dash);
    s->dev.n_dashes = (uint32_t)s->dashes.size();
    s->dev.transforms = s->xforms.empty() ? nullptr : reinterpret_cast<const float*>(m + o_xf);
    s->dev.n_transforms = (uint32_t)(s->xforms.size() / 6);
    s->uploaded = true;
    return SE_OK;
}

extern "C" se_status se_scene_device(const se_scene* s, se_scene_dev* out) {
    if (!s || !out) return SE_ERR_INVALID_ARG;
    if (!s->uploaded) return se_fail(s->ctx, SE_ERR_INVALID_ARG, "the scene is not uploaded");
    *out = s->dev;
    return SE_OK;
}

extern "C" se_status se_scene_destroy(se_scene* s) {
    if (!s) return SE_ERR_INVALID_ARG;
    if (s->dmem) {
        cudaSetDevice(s->ctx->device);
        ctx_free(s->ctx, s->dmem);
    }
    delete s;
    return SE_OK;
}

// --------------------------------------------------------------------------- outlines

extern "C" se_status se_scene_expand(se_scene* s, float tol, uint32_t out_kind, se_outline** out) {
    if (!s || !out) return SE_ERR_INVALID_ARG;
    *out = nullptr;
    se_status st = se_scene_upload(s);
    if (st != SE_OK) return st;
    se_ctx* c = s->ctx;
    se_params p{};
    p.tol = tol;
    p.fit_frac = 0.2f;
    p.flat_frac = 1.0f;
    p.out_kind = out_kind;
    uint64_t n = 0;
    st = se_count(c, &s->dev, &p, &n);
    if (st != SE_OK && st != SE_ERR_LIMIT) return st;
    std::shared_ptr<OutlineBuf> b;
    st = expand_into(c, &s->dev, &p, n, s->n_paths, b, nullptr, nullptr);
    if (st != SE_OK) return st;
    hold_readback(c, b);
    se_outline* o = new (std::nothrow) se_outline();
    if (!o) return SE_ERR_OOM;
    o->buf = b;
    o->path_first = 0;
    o->path_end = s->n_paths;
    o->arcs = out_kind == SE_OUT_ARCS;
    *out = o;
    return SE_OK;
}

extern "C" se_status se_expand_batch(se_ctx* c, se_scene* const* scenes, uint32_t n, float tol, uint32_t out_kind,
                                     se_outline** outs) {
    if (!c || (n && (!scenes || !outs))) return SE_ERR_INVALID_ARG;
    std::vector<se_scene_dev> docs(n);
    for (uint32_t d = 0; d < n; d++) {
        outs[d] = nullptr;
        if (!scenes[d] || scenes[d]->ctx != c) return se_fail(c, SE_ERR_INVALID_ARG, "scene of another context");
        se_status st = se_scene_upload(scenes[d]);
        if (st != SE_OK) return st;
        docs[d] = scenes[d]->dev;
    }
    se_batch* batch = nullptr;
    se_status st = se_batch_create(c, docs.data(), n, &batch);
    if (st != SE_OK) return st;
    std::vector<uint64_t> first(n + 1);
    se_batch_doc_paths(batch, first.data());
    se_params p{};
    p.tol = tol;
    p.fit_frac = 0.2f;
    p.flat_frac = 1.0f;
    p.out_kind = out_kind;
    uint64_t total = 0;
    st = se_batch_count(batch, &p, &total);
    std::shared_ptr<OutlineBuf> b;
    if (st == SE_OK || st == SE_ERR_LIMIT) st = expand_into(c, nullptr, &p, total, (uint32_t)first[n], b, batch_launch, batch);
    if (st == SE_OK) st = sync_buf(*b);  // the batch's gathered scene is released below
    se_batch_destroy(batch);
    if (st != SE_OK && st != SE_ERR_LIMIT) return st;
    for (uint32_t d = 0; d < n; d++) {
        se_outline* o = new (std::nothrow) se_outline();
        if (!o) return SE_ERR_OOM;
        o->buf = b;
        o->path_first = first[d];
        o->path_end = first[d + 1];
        o->arcs = out_kind == SE_OUT_ARCS;
        outs[d] = o;
    }
    return SE_OK;
}

extern "C" se_status se_outline_sync(se_outline* o, uint64_t* n_prims, uint32_t* n_paths) {
    if (!o) return SE_ERR_INVALID_ARG;
    se_status st = sync_buf(*o->buf);
    const OutlineBuf& b = *o->buf;
    if (n_paths) *n_paths = (uint32_t)(o->path_end - o->path_first);
    if (n_prims) *n_prims = b.h_path_offset.empty() ? 0 : b.h_path_offset[o->path_end] - b.h_path_offset[o->path_first];
    return st;
}

extern "C" se_status se_outline_device(const se_outline* o, const float** prims, const float** curvature,
                                       const uint64_t** path_offset) {
    if (!o) return SE_ERR_INVALID_ARG;
    const OutlineBuf& b = *o->buf;
    if (!b.synced) return se_fail(b.ctx, SE_ERR_INVALID_ARG, "outline not synchronised");
    const uint64_t base = b.h_path_offset.empty() ? 0 : b.h_path_offset[o->path_first];
    if (prims) *prims = b.prims + 4 * base;
    if (curvature) *curvature = b.curvature ? b.curvature + base : nullptr;
    if (path_offset) *path_offset = b.path_offset + o->path_first;
    return SE_OK;
}

extern "C" se_status se_outline_copy(const se_outline* o, float* host_prims, float* host_curvature,
                                     uint64_t* host_path_offset) {
    if (!o) return SE_ERR_INVALID_ARG;
    const OutlineBuf& b = *o->buf;
    if (!b.synced) return se_fail(b.ctx, SE_ERR_INVALID_ARG, "outline not synchronised");
    cudaSetDevice(b.ctx->device);
    const uint64_t base = b.h_path_offset[o->path_first], n = b.h_path_offset[o->path_end] - base;
    cudaError_t e = cudaSuccess;
    if (host_prims && n) e = cudaMemcpy(host_prims, b.prims + 4 * base, n * 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_curvature && b.curvature && n)
        e = cudaMemcpy(host_curvature, b.curvature + base, n * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return se_fail(b.ctx, SE_ERR_CUDA, "outline copy", e);
    if (host_path_offset)
        for (uint64_t k = o->path_first; k <= o->path_end; k++) host_path_offset[k - o->path_first] = b.h_path_offset[k] - base;
    return SE_OK;
}

extern "C" se_status se_outline_destroy(se_outline* o) {
    if (!o) return SE_ERR_INVALID_ARG;
    if (o->buf) cudaSetDevice(o->buf->ctx->device);
    delete o;  // the shared buffer goes with its last outline
    return SE_OK;
}

// --------------------------------------------------------------------------- serving scenes

extern "C" se_status se_server_submit_scene(se_server* server, se_scene* s, float tol, uint32_t out_kind,
                                            uint64_t* req_id) {
    if (!server || !s || !req_id) return SE_ERR_INVALID_ARG;
    se_status st = se_scene_upload(s);
    if (st != SE_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s->ctx->stream);  // the server's streams read the upload
    if (e != cudaSuccess) return se_fail(s->ctx, SE_ERR_CUDA, "upload", e);
    se_params p{};
    p.tol = tol;
    p.fit_frac = 0.2f;
    p.flat_frac = 1.0f;
    p.out_kind = out_kind;
    return se_server_submit(server, &s->dev, &p, req_id);
}
