// Batched expansion and launch tuning.
//
// A batch gathers many device-resident documents (encoded scenes) into one
// scene and expands it with the ordinary launch sequence, so thousands of
// small documents cost one sequence of launches instead of one each; the
// sequence (gather included) can be captured once in a CUDA graph and replayed.
// Each document's primitives are a contiguous range of the batch outline
// (bounded by the path offsets of its first and last path), identical to
// what expanding the document alone produces: every step is per segment, and
// the only sums across segments are integer scans.
//
// The autotuner times the expansion of a scene under candidate launch shapes
// (threads per block of the per-tag, per-piece and emit kernels, and resident
// blocks per SM of the persistent emit kernels) and keeps the
// fastest; results do not depend on the launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ctx.h"

namespace se {

struct DocPtrs {
    const uint8_t* tags;
    const uint32_t* words;
    const se_style* styles;
    const float* dashes;
    const float* xforms;  // NULL: the document has none (it gets one identity entry when others have some)
};

struct DocOff {
    uint64_t tags, words, styles, dashes, xforms;  // xforms in entries of 6 floats
};

struct GatherBlock {
    uint32_t doc, chunk;
};

constexpr uint32_t kGatherChunk = 4096;
constexpr int kGatherThreads = 256;

// One block copies one chunk of every stream of one document; a document's
// style entries get their dash-pattern index moved past the dash entries of
// the documents before it.  When some documents carry transforms, a document
// without any gets one identity entry and the transform bit on its first tag
// (a document with transforms starts with that bit, as the encoder writes it).
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(const DocPtrs* docs, const DocOff* off,
                                                                const GatherBlock* blocks, uint8_t* tags, uint32_t* words,
                                                                se_style* styles, float* dashes, float* xforms) {
    const GatherBlock gb = blocks[blockIdx.x];
    const DocOff o0 = off[gb.doc], o1 = off[gb.doc + 1];
    const DocPtrs p = docs[gb.doc];
    const uint64_t lo = (uint64_t)gb.chunk * kGatherChunk, hi = lo + kGatherChunk;
    const bool ident = xforms && !p.xforms && o1.xforms > o0.xforms;
    uint64_t n = o1.tags - o0.tags;
    for (uint64_t i = lo + threadIdx.x; i < n && i < hi; i += kGatherThreads)
        tags[o0.tags + i] = (uint8_t)(p.tags[i] | ((ident && i == 0) ? SE_TAG_TRANSFORM : 0u));
    n = 6 * (o1.xforms - o0.xforms);
    for (uint64_t i = lo + threadIdx.x; xforms && i < n && i < hi; i += kGatherThreads)
        xforms[6 * o0.xforms + i] = ident ? ((i == 0 || i == 3) ? 1.0f : 0.0f) : p.xforms[i];
    n = o1.words - o0.words;
    for (uint64_t i = lo + threadIdx.x; i < n && i < hi; i += kGatherThreads) words[o0.words + i] = p.words[i];
    n = o1.styles - o0.styles;
    for (uint64_t i = lo + threadIdx.x; i < n && i < hi; i += kGatherThreads) {
        se_style st = p.styles[i];
        st.dash_first += (uint32_t)o0.dashes;
        styles[o0.styles + i] = st;
    }
    n = o1.dashes - o0.dashes;
    for (uint64_t i = lo + threadIdx.x; i < n && i < hi; i += kGatherThreads) dashes[o0.dashes + i] = p.dashes[i];
}

}  // namespace se

struct se_batch {
    se_ctx* ctx = nullptr;
    uint32_t n_docs = 0;
    std::vector<uint64_t> path_first;  // n_docs + 1
    void* mem = nullptr;
    se::DocPtrs* d_docs = nullptr;
    se::DocOff* d_off = nullptr;
    se::GatherBlock* d_blocks = nullptr;
    uint32_t n_blocks = 0;
    se_scene_dev scene{};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t ws_gen = 0;  // the context's workspace generation the graph was captured with
    size_t bytes = 0;     // device bytes the batch holds
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

se_status gather(se_batch* b) {
    if (b->n_blocks == 0) return SE_OK;
    se_ctx* c = b->ctx;
    se::gather_kernel<<<b->n_blocks, se::kGatherThreads, 0, c->stream>>>(
        b->d_docs, b->d_off, b->d_blocks, const_cast<uint8_t*>(b->scene.tags),
        const_cast<uint32_t*>(b->scene.words), const_cast<se_style*>(b->scene.styles),
        const_cast<float*>(b->scene.dashes), const_cast<float*>(b->scene.transforms));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SE_OK : se_fail(c, SE_ERR_CUDA, "gather launch", e);
}

void drop_graph(se_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" se_status se_batch_create(se_ctx* c, const se_scene_dev* docs, uint32_t n_docs, se_batch** out) {
    if (!c || !out || (n_docs && !docs)) return SE_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(c->device);
    std::vector<se::DocPtrs> ptrs(n_docs);
    std::vector<se::DocOff> off(n_docs + 1);
    std::vector<se::GatherBlock> blocks;
    std::vector<uint64_t> path_first(n_docs + 1, 0);
    se::DocOff acc{0, 0, 0, 0, 0};
    bool any_xf = false;
    for (uint32_t d = 0; d < n_docs; d++) any_xf = any_xf || docs[d].n_transforms > 0;
    for (uint32_t d = 0; d < n_docs; d++) {
        const se_scene_dev& s = docs[d];
        if (s.n_tags && (!s.tags || !s.styles)) return se_fail(c, SE_ERR_INVALID_ARG, "document pointer is NULL");
        if (s.n_words && !s.words) return se_fail(c, SE_ERR_INVALID_ARG, "document path data is NULL");
        if (s.n_dashes && !s.dashes) return se_fail(c, SE_ERR_INVALID_ARG, "document dash array is NULL");
        if (s.n_transforms && !s.transforms) return se_fail(c, SE_ERR_INVALID_ARG, "document transform array is NULL");
        ptrs[d] = se::DocPtrs{s.tags, s.words, s.styles, s.dashes,
                              s.n_transforms ? s.transforms : nullptr};
        off[d] = acc;
        path_first[d] = path_first[d > 0 ? d - 1 : 0] + (d > 0 ? docs[d - 1].n_paths : 0);
        const uint64_t nx = any_xf ? (s.n_transforms ? s.n_transforms : (s.n_tags ? 1u : 0u)) : 0u;
        uint64_t m = std::max(std::max(s.n_tags, s.n_words), std::max<uint64_t>(s.n_styles, s.n_dashes));
        m = std::max<uint64_t>(m, 6 * nx);
        for (uint64_t k = 0; k * se::kGatherChunk < m; k++) blocks.push_back(se::GatherBlock{d, (uint32_t)k});
        acc.tags += s.n_tags;
        acc.words += s.n_words;
        acc.styles += s.n_styles;
        acc.dashes += s.n_dashes;
        acc.xforms += nx;
    }
    off[n_docs] = acc;
    path_first[n_docs] = n_docs ? path_first[n_docs - 1] + docs[n_docs - 1].n_paths : 0;
    if (acc.tags >= (1ull << 31) || acc.words >= (1ull << 32) || acc.styles >= (1ull << 32) || acc.dashes >= (1ull << 32) || acc.xforms >= (1ull << 32) ||
        path_first[n_docs] >= (1ull << 32) || blocks.size() >= (1ull << 31))
        return se_fail(c, SE_ERR_INVALID_ARG, "the batch is larger than one scene may be");
    se_batch* b = new (std::nothrow) se_batch();
    if (!b) return SE_ERR_OOM;
    b->ctx = c;
    b->n_docs = n_docs;
    b->path_first = path_first;
    b->n_blocks = (uint32_t)blocks.size();
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = al256(o + bytes);
        return r;
    };
    size_t o_docs = take(sizeof(se::DocPtrs) * n_docs + 8), o_off = take(sizeof(se::DocOff) * (n_docs + 1));
    size_t o_blk = take(sizeof(se::GatherBlock) * blocks.size() + 8);
    size_t o_tags = take(acc.tags + 16), o_pts = take(acc.words * 4 + 8), o_sty = take(acc.styles * sizeof(se_style) + 8);
    size_t o_dash = take(acc.dashes * 4 + 4), o_xf = take(acc.xforms * 24 + 4);
    b->bytes = o;
    cudaError_t e = ctx_alloc(c, &b->mem, o);
    if (e != cudaSuccess) {
        delete b;
        return se_fail(c, SE_ERR_OOM, "batch allocation failed", e);
    }
    char* m = static_cast<char*>(b->mem);
    b->d_docs = reinterpret_cast<se::DocPtrs*>(m + o_docs);
    b->d_off = reinterpret_cast<se::DocOff*>(m + o_off);
    b->d_blocks = reinterpret_cast<se::GatherBlock*>(m + o_blk);
    e = cudaMemcpyAsync(b->d_docs, ptrs.data(), sizeof(se::DocPtrs) * n_docs, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_off, off.data(), sizeof(se::DocOff) * (n_docs + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !blocks.empty())
        e = cudaMemcpyAsync(b->d_blocks, blocks.data(), sizeof(se::GatherBlock) * blocks.size(), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the host vectors go out of scope
    if (e != cudaSuccess) {
        ctx_free(c, b->mem);
        delete b;
        return se_fail(c, SE_ERR_CUDA, "batch upload", e);
    }
    b->scene.tags = reinterpret_cast<const uint8_t*>(m + o_tags);
    b->scene.n_tags = acc.tags;
    b->scene.words = reinterpret_cast<const uint32_t*>(m + o_pts);
    b->scene.n_words = acc.words;
    b->scene.styles = reinterpret_cast<const se_style*>(m + o_sty);
    b->scene.n_styles = (uint32_t)acc.styles;
    b->scene.n_paths = (uint32_t)path_first[n_docs];
    b->scene.dashes = acc.dashes ? reinterpret_cast<const float*>(m + o_dash) : nullptr;
    b->scene.n_dashes = (uint32_t)acc.dashes;
    b->scene.transforms = acc.xforms ? reinterpret_cast<const float*>(m + o_xf) : nullptr;
    b->scene.n_transforms = (uint32_t)acc.xforms;
    *out = b;
    return SE_OK;
}

size_t se_batch_device_bytes(const se_batch* b) { return b ? b->bytes : 0; }

extern "C" se_status se_batch_destroy(se_batch* b) {
    if (!b) return SE_ERR_INVALID_ARG;
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->ctx->stream);
    if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    ctx_free(b->ctx, b->mem);
    delete b;
    return SE_OK;
}

extern "C" se_status se_batch_doc_paths(const se_batch* b, uint64_t* path_first) {
    if (!b || !path_first) return SE_ERR_INVALID_ARG;
    for (uint32_t d = 0; d <= b->n_docs; d++) path_first[d] = b->path_first[d];
    return SE_OK;
}

extern "C" se_status se_batch_scene(const se_batch* b, se_scene_dev* scene) {
    if (!b || !scene) return SE_ERR_INVALID_ARG;
    *scene = b->scene;
    return SE_OK;
}

extern "C" se_status se_batch_count(se_batch* b, const se_params* p, uint64_t* n_prims) {
    if (!b || !n_prims) return SE_ERR_INVALID_ARG;
    settle_pending(b->ctx);
    cudaSetDevice(b->ctx->device);
    se_status st = gather(b);
    if (st != SE_OK) return st;
    return se_count(b->ctx, &b->scene, p, n_prims);
}

extern "C" se_status se_batch_expand(se_batch* b, const se_params* p, const se_outline_dev* out) {
    if (!b) return SE_ERR_INVALID_ARG;
    settle_pending(b->ctx);
    cudaSetDevice(b->ctx->device);
    se_status st = gather(b);
    if (st != SE_OK) return st;
    return se_expand(b->ctx, &b->scene, p, out);
}

extern "C" se_status se_batch_expand_counted(se_batch* b, const se_params* p, const se_outline_dev* out) {
    if (!b) return SE_ERR_INVALID_ARG;
    cudaSetDevice(b->ctx->device);
    return se_expand_counted(b->ctx, &b->scene, p, out);
}

extern "C" se_status se_batch_capture(se_batch* b, const se_params* p, const se_outline_dev* out) {
    if (!b) return SE_ERR_INVALID_ARG;
    se_ctx* c = b->ctx;
    settle_pending(c);
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && !b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "capture stream", e);
    drop_graph(b);
    cudaStream_t saved = c->stream;
    bool prof = c->profile;
    c->stream = b->cap_stream;
    c->profile = false;
    c->capturing = true;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    se_status st = SE_OK;
    if (e == cudaSuccess) {
        st = gather(b);
        if (st == SE_OK) st = se_expand(c, &b->scene, p, out);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
        if (e2 == cudaSuccess && st == SE_OK) {
            b->graph = g;
            b->ws_gen = c->ws_gen;
            e = cudaGraphInstantiate(&b->exec, g, 0);
            if (e != cudaSuccess) b->exec = nullptr;
        } else {
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) e = e2;
        }
    }
    c->stream = saved;
    c->profile = prof;
    c->capturing = false;
    if (st != SE_OK) return st;
    if (e != cudaSuccess) {
        drop_graph(b);
        return se_fail(c, SE_ERR_CUDA, "graph capture", e);
    }
    return SE_OK;
}

extern "C" se_status se_batch_launch(se_batch* b) {
    if (!b) return SE_ERR_INVALID_ARG;
    if (!b->exec) return se_fail(b->ctx, SE_ERR_INVALID_ARG, "no captured graph");
    settle_pending(b->ctx);
    if (b->ws_gen != b->ctx->ws_gen)
        return se_fail(b->ctx, SE_ERR_INVALID_ARG, "the context's workspace was reallocated since the capture");
    cudaSetDevice(b->ctx->device);
    cudaError_t e = cudaGraphLaunch(b->exec, b->ctx->stream);
    return e == cudaSuccess ? SE_OK : se_fail(b->ctx, SE_ERR_CUDA, "graph launch", e);
}

// ---------------------------------------------------------------------------
// launch tuning
// ---------------------------------------------------------------------------
extern "C" se_status se_get_tuning(const se_ctx* c, se_tuning* t) {
    if (!c || !t) return SE_ERR_INVALID_ARG;
    t->plan_block = c->tune.plan_block;
    t->piece_block = c->tune.piece_block;
    t->emit_block = c->tune.emit_block;
    t->emit_blocks_per_sm = c->tune.emit_blocks_per_sm;
    return SE_OK;
}

extern "C" se_status se_set_tuning(se_ctx* c, const se_tuning* t) {
    if (!c || !t) return SE_ERR_INVALID_ARG;
    auto block_ok = [](uint32_t v) { return v == 64 || v == 128 || v == 256; };
    if (!block_ok(t->plan_block) || !block_ok(t->piece_block) ||
        !(t->emit_block == 64 || t->emit_block == 128) || t->emit_blocks_per_sm > 32)
        return se_fail(c, SE_ERR_INVALID_ARG, "tuning out of range");
    c->tune.plan_block = t->plan_block;
    c->tune.piece_block = t->piece_block;
    c->tune.emit_block = t->emit_block;
    c->tune.emit_blocks_per_sm = t->emit_blocks_per_sm;
    return SE_OK;
}

namespace {

// mean device time of `reps` expansions under the context's current tuning (ms)
se_status time_expand(se_ctx* c, const se_scene_dev* s, const se_params* p, const se_outline_dev* out, int reps,
                      cudaEvent_t e0, cudaEvent_t e1, float* ms) {
    se_status st = se_expand(c, s, p, out);  // warm-up (and the check that it runs)
    if (st != SE_OK) return st;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && st == SE_OK; r++) st = se_expand(c, s, p, out);
    cudaEventRecord(e1, c->stream);
    if (st != SE_OK) return st;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e != cudaSuccess) return se_fail(c, SE_ERR_CUDA, "tuning timer", e);
    uint64_t n = 0;
    st = se_sync(c, &n);
    if (st != SE_OK && st != SE_ERR_LIMIT) return st;
    *ms /= (float)reps;
    return SE_OK;
}

}  // namespace

extern "C" se_status se_autotune(se_ctx* c, const se_scene_dev* s, const se_params* p, const se_outline_dev* out,
                                 int reps, se_tuning* chosen) {
    if (!c || !s || !p || !out || reps < 1) return SE_ERR_INVALID_ARG;
    settle_pending(c);
    cudaSetDevice(c->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return se_fail(c, SE_ERR_CUDA, "event create");
    }
    bool prof = c->profile;
    c->profile = false;
    Tuning best = c->tune;
    float best_ms = 0.0f;
    se_status st = time_expand(c, s, p, out, reps, e0, e1, &best_ms);
    // coordinate descent: one knob at a time, the others at their best so far.  The
    // knobs are per work class: the emit (block size, resident blocks per SM), the
    // per-tag plan (block, which is also the tile its curves-first sort works on)
    // and the per-piece pass (records staged per block: its tile)
    const uint32_t blocks[3] = {64, 128, 256}, per_sm[5] = {1, 2, 3, 4, 0}, tiles[2] = {128, 256};
    for (int knob = 0; knob < 4 && st == SE_OK; knob++) {
        int n = knob == 1 ? 5 : knob == 3 ? 2 : 3;
        for (int k = 0; k < n && st == SE_OK; k++) {
            Tuning t = best;
            if (knob == 0) t.emit_block = blocks[k] > 128 ? 128 : blocks[k];
            else if (knob == 1) t.emit_blocks_per_sm = per_sm[k];
            else if (knob == 2) t.plan_block = blocks[k];
            else t.piece_block = tiles[k];
            c->tune = t;
            float ms = 0.0f;
            st = time_expand(c, s, p, out, reps, e0, e1, &ms);
            if (st == SE_OK && ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    c->tune = best;
    c->profile = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SE_OK) return st;
    if (chosen) se_get_tuning(c, chosen);
    return SE_OK;
}
