// Serving loop: continuous batching of expansion requests under an HBM budget.
//
// Not part of the paper's method (which expands one scene per dispatch): a
// runtime around the batched expansion.  Requests (a device-resident encoded
// document and expansion parameters) queue up as they arrive.  Each of the
// server's slots -- a worker thread with its own context, stream and
// workspace -- takes the queued requests that share the head request's
// parameters (up to a document and tag limit), counts them as one batch,
// waits until their outline fits the HBM budget, expands them and hands every
// request its range of the batch outline.  Requests that arrive while batches
// run are taken by the next free slot, so work from several batches overlaps
// on the device.  A request's outline stays in device memory until the client
// releases it; the budget covers the batches' gathered encodings and outline
// buffers.  Device memory comes from the caller's allocator, or by default from
// the stream-ordered allocator, so no slot's allocation or release waits for
// another slot's work.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.h"

namespace {

__global__ void boundary_kernel(const uint64_t* path_offset, const uint64_t* path_first, uint32_t n, uint64_t* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = path_offset[path_first[i]];
}

using Clock = std::chrono::steady_clock;

// One expanded batch's device memory, shared by its requests.
struct BatchOut {
    void* mem = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    se_free_fn free_fn = nullptr;  // the server's allocator (NULL: stream-ordered)
    void* alloc_user = nullptr;
    int refs = 0;
    float* prims = nullptr;
    float* curv = nullptr;
};

enum { kQueued = 0, kRunning = 1, kDone = 2 };

struct Request {
    se_scene_dev doc{};
    se_params params{};
    int state = kQueued;
    se_status status = SE_OK;
    uint32_t batch_docs = 0;
    int64_t t_submit = 0, t_start = 0, t_done = 0;
    std::shared_ptr<BatchOut> out;
    uint64_t lo = 0, hi = 0;
};

bool same_params(const se_params& a, const se_params& b) {
    return a.tol == b.tol && a.fit_frac == b.fit_frac && a.flat_frac == b.flat_frac && a.out_kind == b.out_kind &&
           a.refine == b.refine;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct se_server {
    int device = 0;
    se_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    uint64_t in_use = 0, peak = 0;
    bool stop = false;
    std::vector<se_ctx*> ctxs;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;
    Clock::time_point t0;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0;
    uint32_t busy = 0, max_busy = 0;
    std::string last_error;  // the most recent failed batch: its step and cause (under mu)

    int64_t now() const { return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count(); }

    // finish the requests of a batch (lock held)
    void finish(const std::vector<uint64_t>& ids, se_status st, const std::shared_ptr<BatchOut>& out,
                const std::vector<uint64_t>& bounds) {
        int64_t t = now();
        for (size_t d = 0; d < ids.size(); d++) {
            Request& r = reqs[ids[d]];
            r.state = kDone;
            r.status = st;
            r.batch_docs = (uint32_t)ids.size();
            r.t_done = t;
            if (st == SE_OK || st == SE_ERR_LIMIT) {
                r.out = out;
                r.lo = bounds[d];
                r.hi = bounds[d + 1];
                completed++;
            } else {
                failed++;
            }
        }
        cv_done.notify_all();
    }

    void run_batch(int k, std::vector<uint64_t> ids);
    void worker(int k);
};

void se_server::run_batch(int k, std::vector<uint64_t> ids) {
    se_ctx* c = ctxs[k];
    cudaStream_t s = streams[k];
    std::vector<se_scene_dev> docs;
    se_params params{};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (uint64_t id : ids) docs.push_back(reqs[id].doc);
        params = reqs[ids[0]].params;
    }
    const uint32_t n = (uint32_t)ids.size();
    const bool arcs = params.out_kind == SE_OUT_ARCS;
    se_batch* b = nullptr;
    uint64_t n_prims = 0;
    se_status st = se_batch_create(c, docs.data(), n, &b);
    if (st == SE_OK) st = se_batch_count(b, &params, &n_prims);
    if (st != SE_OK && st != SE_ERR_LIMIT) {
        if (b) se_batch_destroy(b);
        const std::string msg = std::string("batch count: ") + se_ctx_last_error(c);
        std::lock_guard<std::mutex> lk(mu);
        last_error = msg;
        finish(ids, st, nullptr, {});
        return;
    }
    se_scene_dev scene{};
    se_batch_scene(b, &scene);
    std::vector<uint64_t> path_first(n + 1), bounds(n + 1, 0);
    se_batch_doc_paths(b, path_first.data());
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = al256(o + bytes);
        return r;
    };
    size_t o_prims = take(n_prims * 16 + 16), o_curv = take(arcs ? n_prims * 4 + 4 : 0);
    size_t o_poff = take((scene.n_paths + 1ull) * 8), o_pf = take((n + 1ull) * 8), o_bd = take((n + 1ull) * 8);
    const size_t out_bytes = o;
    const size_t gather_bytes = se_batch_device_bytes(b);
    const size_t bytes = out_bytes + gather_bytes;
    {
        std::unique_lock<std::mutex> lk(mu);
        if (bytes > cfg.hbm_budget) {
            lk.unlock();
            se_batch_destroy(b);
            if (n > 1) {
                // too large together: send the second half back to the front of the queue
                std::vector<uint64_t> head(ids.begin(), ids.begin() + n / 2), tail(ids.begin() + n / 2, ids.end());
                {
                    std::lock_guard<std::mutex> lk2(mu);
                    for (auto it = tail.rbegin(); it != tail.rend(); ++it) {
                        reqs[*it].state = kQueued;
                        queue.push_front(*it);
                    }
                    cv_work.notify_all();
                }
                run_batch(k, head);
            } else {
                std::lock_guard<std::mutex> lk2(mu);
                last_error = "a request larger than the HBM budget";
                finish(ids, SE_ERR_BUDGET, nullptr, {});
            }
            return;
        }
        cv_mem.wait(lk, [&] { return stop || in_use + bytes <= cfg.hbm_budget; });
        in_use += bytes;
        peak = std::max(peak, in_use);
    }
    auto out = std::make_shared<BatchOut>();
    out->stream = s;
    out->bytes = out_bytes;
    out->free_fn = cfg.free_fn;
    out->alloc_user = cfg.alloc_user;
    cudaError_t e = dev_alloc(cfg.alloc_fn, cfg.alloc_user, &out->mem, out_bytes, s);
    if (e == cudaSuccess) {
        char* m = static_cast<char*>(out->mem);
        out->prims = reinterpret_cast<float*>(m + o_prims);
        out->curv = arcs ? reinterpret_cast<float*>(m + o_curv) : nullptr;
        uint64_t* poff = reinterpret_cast<uint64_t*>(m + o_poff);
        uint64_t* d_pf = reinterpret_cast<uint64_t*>(m + o_pf);
        uint64_t* d_bd = reinterpret_cast<uint64_t*>(m + o_bd);
        se_outline_dev od{};
        od.prims = out->prims;
        od.curvature = out->curv;
        od.path_offset = poff;
        od.capacity = n_prims;
        e = cudaMemcpyAsync(d_pf, path_first.data(), (n + 1ull) * 8, cudaMemcpyHostToDevice, s);
        // the count left the batch's front half in the slot's workspace: only the
        // primitive scan and the emit run now
        if (e == cudaSuccess) st = se_batch_expand_counted(b, &params, &od);
        if (e == cudaSuccess && st == SE_OK) {
            boundary_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(poff, d_pf, n, d_bd);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && st == SE_OK)
            e = cudaMemcpyAsync(bounds.data(), d_bd, (n + 1ull) * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && st == SE_OK) {
            uint64_t got = 0;
            st = se_sync(c, &got);  // waits for the stream (and so for the copies above)
        }
    }
    if (e != cudaSuccess && st == SE_OK) st = SE_ERR_CUDA;
    std::string msg;
    if (st != SE_OK && st != SE_ERR_LIMIT)
        msg = std::string("batch expand: ") + (e != cudaSuccess ? cudaGetErrorString(e) : se_ctx_last_error(c));
    se_batch_destroy(b);
    std::lock_guard<std::mutex> lk(mu);
    in_use -= gather_bytes;
    if (st != SE_OK && st != SE_ERR_LIMIT) {
        last_error = msg;
        dev_free(out->free_fn, out->alloc_user, out->mem, s);
        in_use -= out_bytes;
        cv_mem.notify_all();
        finish(ids, st, nullptr, {});
        return;
    }
    out->refs = (int)n;
    batches++;
    cv_mem.notify_all();
    finish(ids, st, out, bounds);
}

void se_server::worker(int k) {
    cudaSetDevice(device);
    for (;;) {
        std::vector<uint64_t> ids;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            if (stop) return;
            // the queued requests that share the head's parameters, in arrival order
            const se_params head = reqs[queue.front()].params;
            uint64_t tags = 0;
            for (auto it = queue.begin(); it != queue.end() && ids.size() < cfg.max_batch_docs;) {
                Request& r = reqs[*it];
                bool fits = ids.empty() || cfg.max_batch_tags == 0 || tags + r.doc.n_tags <= cfg.max_batch_tags;
                if (same_params(r.params, head) && fits) {
                    ids.push_back(*it);
                    tags += r.doc.n_tags;
                    r.state = kRunning;
                    r.t_start = now();
                    it = queue.erase(it);
                } else {
                    ++it;
                }
            }
            busy++;
            max_busy = std::max(max_busy, busy);
        }
        run_batch(k, ids);
        std::lock_guard<std::mutex> lk(mu);
        busy--;
    }
}

extern "C" se_status se_server_last_error(se_server* s, char* buf, size_t len) {
    if (!s || !buf || len == 0) return SE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t n = std::min(len - 1, s->last_error.size());
    memcpy(buf, s->last_error.data(), n);
    buf[n] = '\0';
    return SE_OK;
}

extern "C" se_status se_server_create(int device, const se_server_config* cfg, se_server** out) {
    if (!cfg || !out || cfg->slots < 1 || cfg->slots > 64 || cfg->max_batch_docs < 1 || cfg->hbm_budget == 0 ||
        (cfg->alloc_fn == nullptr) != (cfg->free_fn == nullptr))
        return SE_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SE_ERR_INVALID_ARG;
    cudaSetDevice(device);
    se_server* s = new (std::nothrow) se_server();
    if (!s) return SE_ERR_OOM;
    s->device = device;
    s->cfg = *cfg;
    s->t0 = Clock::now();
    // freed blocks stay in the device's stream-ordered pool for the next batch
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (uint32_t k = 0; k < cfg->slots; k++) {
        cudaStream_t st = nullptr;
        se_ctx* c = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            se_ctx_create(device, st, cfg->alloc_fn, cfg->free_fn, cfg->alloc_user, &c) != SE_OK) {
            if (st) cudaStreamDestroy(st);
            se_server_destroy(s);
            return SE_ERR_CUDA;
        }
        s->streams.push_back(st);
        s->ctxs.push_back(c);
    }
    for (uint32_t k = 0; k < cfg->slots; k++) s->workers.emplace_back([s, k] { s->worker((int)k); });
    *out = s;
    return SE_OK;
}

extern "C" se_status se_server_destroy(se_server* s) {
    if (!s) return SE_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
    for (auto& t : s->workers) t.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->reqs) {
        Request& r = kv.second;
        if (r.out && --r.out->refs == 0) dev_free(r.out->free_fn, r.out->alloc_user, r.out->mem, r.out->stream);
        r.out.reset();
    }
    for (size_t k = 0; k < s->ctxs.size(); k++) {
        cudaStreamSynchronize(s->streams[k]);
        se_ctx_destroy(s->ctxs[k]);
        cudaStreamDestroy(s->streams[k]);
    }
    delete s;
    return SE_OK;
}

extern "C" se_status se_server_submit(se_server* s, const se_scene_dev* doc, const se_params* params,
                                      uint64_t* req_id) {
    if (!s || !doc || !params || !req_id) return SE_ERR_INVALID_ARG;
    if (doc->n_tags && (!doc->tags || !doc->styles)) return SE_ERR_INVALID_ARG;
    if (doc->n_words && !doc->words) return SE_ERR_INVALID_ARG;
    if (!(params->tol > 0.0f) || !(params->fit_frac > 0.0f) || !(params->flat_frac > 0.0f) ||
        (params->out_kind != SE_OUT_LINES && params->out_kind != SE_OUT_ARCS))
        return SE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SE_ERR_INVALID_ARG;
    uint64_t id = s->next_id++;
    Request& r = s->reqs[id];
    r.doc = *doc;
    r.params = *params;
    r.t_submit = s->now();
    s->queue.push_back(id);
    s->submitted++;
    *req_id = id;
    s->cv_work.notify_one();
    return SE_OK;
}

extern "C" se_status se_server_poll(se_server* s, uint64_t req_id, int wait, se_request_result* out) {
    if (!s || !out) return SE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return SE_ERR_INVALID_ARG;
    if (wait) s->cv_done.wait(lk, [&] { return s->reqs[req_id].state == kDone; });
    const Request& r = s->reqs[req_id];
    std::memset(out, 0, sizeof(*out));
    out->done = r.state == kDone;
    out->status = r.state == kDone ? r.status : SE_OK;
    out->batch_docs = r.batch_docs;
    out->t_submit_ns = r.t_submit;
    out->t_start_ns = r.t_start;
    out->t_done_ns = r.t_done;
    if (r.out) {
        out->prims = r.out->prims + 4 * r.lo;
        out->curvature = r.out->curv ? r.out->curv + r.lo : nullptr;
        out->n_prims = r.hi - r.lo;
    }
    return SE_OK;
}

extern "C" se_status se_server_release(se_server* s, uint64_t req_id) {
    if (!s) return SE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || it->second.state != kDone) return SE_ERR_INVALID_ARG;
    Request& r = it->second;
    if (r.out && --r.out->refs == 0) {
        cudaSetDevice(s->device);
        dev_free(r.out->free_fn, r.out->alloc_user, r.out->mem, r.out->stream);
        s->in_use -= r.out->bytes;
        s->cv_mem.notify_all();
    }
    s->reqs.erase(it);
    return SE_OK;
}

extern "C" se_status se_server_get_stats(se_server* s, se_server_stats* out) {
    if (!s || !out) return SE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->batches = s->batches;
    out->queued = s->queue.size();
    out->max_concurrent = s->max_busy;
    out->bytes_in_use = s->in_use;
    out->bytes_peak = s->peak;
    out->hbm_budget = s->cfg.hbm_budget;
    return SE_OK;
}
