// Serving loop over device-resident prepared images (include/opta_serve.h).
//
// A queue of template requests and a fixed set of workers.  Each worker is
// a host thread with its own stream and search context; it takes the
// waiting requests of the oldest request's image (up to max_batch, in
// arrival order), searches them with optA_search_ctx and publishes one
// completion per request.  Requests that arrive while batches run wait in
// the queue and join the next worker that frees up, and the workers'
// batches overlap on the device.
//
// Admission by device memory: every worker's context holds search scratch
// (kept between batches).  Before a batch runs, the bytes its context will
// hold afterwards (optA_ctx_bytes_after) plus what the other workers hold
// must fit the budget.  Otherwise the batch is halved (the rest returns to
// the front of the queue); a single request first drops the worker's own
// scratch, then asks idle workers to drop theirs and waits for busy ones to
// finish; it fails with OPTA_ERR_OOM only when no other worker holds any.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "opta.h"
#include "opta_serve.h"

namespace {

struct Request {
    uint64_t id = 0;
    int image = 0;
    int m = 0, n = 0;
    std::vector<float> data;   // m x n, row-major
    double t_submit = 0.0;
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    opta_search_ctx *ctx = nullptr;
    size_t held = 0;   // device bytes of ctx as accounted in `used`
    bool idle = true;
};

}  // namespace

struct opta_server {
    opta_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;   // requests queued, scratch wanted, or stop
    std::condition_variable cv_done;   // completions published, or scratch released
    std::vector<opta_handle *> images;
    std::deque<Request> queue;
    std::deque<opta_completion> done;
    uint64_t next_id = 1;
    int64_t outstanding = 0;           // submitted and not yet returned by opta_server_wait
    size_t used = 0;                   // scratch bytes held by all workers
    int trim_waiters = 0;              // workers waiting for scratch: idle workers release theirs
    bool stop = false;
    std::vector<Worker> workers;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void release_ctx(opta_server *S, Worker &W) {
    if (W.ctx) optA_ctx_destroy(W.ctx);
    W.ctx = nullptr;
    S->used -= W.held;
    W.held = 0;
}

void complete(opta_server *S, const Request &r, const opta_result &res, int batch, int worker,
              double t_start, double t_done) {
    opta_completion c;
    std::memset(&c, 0, sizeof(c));
    c.request_id = r.id;
    c.image_id = r.image;
    c.batch_size = batch;
    c.worker = worker;
    c.status = res.status;
    c.t_submit = r.t_submit;
    c.t_start = t_start;
    c.t_done = t_done;
    c.result = res;
    S->done.push_back(c);
}

void fail(opta_server *S, const Request &r, opta_status st, int worker) {
    opta_result res;
    std::memset(&res, 0, sizeof(res));
    res.status = st;
    const double t = S->now();
    complete(S, r, res, 1, worker, t, t);
}

std::vector<opta_template> descriptors(const std::vector<Request> &batch) {
    std::vector<opta_template> d(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
        std::memset(&d[i], 0, sizeof(d[i]));
        d[i].rows = batch[i].m;
        d[i].cols = batch[i].n;
        d[i].stride_elems = batch[i].n;
        d[i].on_device = 0;
        d[i].data = batch[i].data.data();
    }
    return d;
}

void work(opta_server *S, int w) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    Worker &W = S->workers[w];
    for (;;) {
        S->cv_work.wait(lk, [&] {
            return S->stop || !S->queue.empty() || (S->trim_waiters > 0 && W.held > 0);
        });
        if (S->trim_waiters > 0 && W.held > 0) {
            release_ctx(S, W);
            S->cv_done.notify_all();
        }
        if (S->queue.empty()) {
            if (!S->stop) continue;
            release_ctx(S, W);   // a worker still waiting for scratch must not wait on this one
            S->cv_done.notify_all();
            break;
        }
        // the batch: waiting requests of the oldest request's image, in order
        const int img = S->queue.front().image;
        std::vector<Request> batch;
        for (auto it = S->queue.begin();
             it != S->queue.end() && (int)batch.size() < S->cfg.max_batch;) {
            if (it->image == img) {
                batch.push_back(std::move(*it));
                it = S->queue.erase(it);
            } else {
                ++it;
            }
        }
        opta_handle *h = S->images[img];
        if (!W.ctx && optA_ctx_create(h, &W.ctx) != OPTA_OK) {
            for (const Request &r : batch) fail(S, r, OPTA_ERR_OOM, w);
            S->cv_done.notify_all();
            continue;
        }
        // admission by device memory
        size_t need = 0;
        bool admitted = false;
        const size_t budget = (size_t)std::max<int64_t>(S->cfg.memory_budget, 0);
        for (;;) {
            std::vector<opta_template> d = descriptors(batch);
            const opta_status st = optA_ctx_bytes_after(h, W.ctx, d.data(), (int)d.size(), &need);
            if (st != OPTA_OK) {
                for (const Request &r : batch) fail(S, r, st, w);
                break;
            }
            if (budget == 0 || S->used - W.held + need <= budget) {
                admitted = true;
                break;
            }
            if (batch.size() > 1) {
                const size_t keep = batch.size() / 2;
                for (size_t i = batch.size(); i-- > keep;) S->queue.push_front(std::move(batch[i]));
                batch.resize(keep);
                continue;
            }
            if (W.held > 0) {   // start again from an empty context
                release_ctx(S, W);
                if (optA_ctx_create(h, &W.ctx) != OPTA_OK) {
                    fail(S, batch[0], OPTA_ERR_OOM, w);
                    break;
                }
                continue;
            }
            if (S->used > 0) {   // others hold scratch: idle ones release it, busy ones finish
                ++S->trim_waiters;
                S->cv_work.notify_all();
                S->cv_done.wait(lk);
                --S->trim_waiters;
                continue;
            }
            fail(S, batch[0], OPTA_ERR_OOM, w);
            break;
        }
        if (!admitted) {
            S->cv_done.notify_all();
            continue;
        }
        S->used += need - W.held;
        W.held = need;
        W.idle = false;
        lk.unlock();
        const double t_start = S->now();
        std::vector<opta_template> d = descriptors(batch);
        std::vector<opta_result> res(batch.size());
        optA_search_ctx(h, W.ctx, d.data(), (int)d.size(), res.data(), W.stream);
        const double t_done = S->now();
        size_t actual = need;
        optA_ctx_memory_bytes(W.ctx, &actual);
        lk.lock();
        S->used += actual;
        S->used -= W.held;
        W.held = actual;
        W.idle = true;
        for (size_t i = 0; i < batch.size(); ++i)
            complete(S, batch[i], res[i], (int)batch.size(), w, t_start, t_done);
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

void opta_server_config_default(opta_server_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->n_workers = 4;
    cfg->max_batch = 64;
    cfg->memory_budget = 0;
}

opta_status opta_server_create(const opta_server_config *cfg, opta_server **out) {
    if (!out) return OPTA_ERR_INVALID_ARG;
    *out = nullptr;
    opta_server_config c;
    if (cfg) c = *cfg; else opta_server_config_default(&c);
    if (c.n_workers < 1 || c.n_workers > 64 || c.max_batch < 1 || c.memory_budget < 0)
        return OPTA_ERR_INVALID_ARG;
    opta_server *S = new (std::nothrow) opta_server();
    if (!S) return OPTA_ERR_OOM;
    S->cfg = c;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return OPTA_ERR_CUDA;
    }
    S->workers.resize(c.n_workers);
    for (Worker &W : S->workers) {
        if (cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (Worker &V : S->workers)
                if (V.stream) cudaStreamDestroy(V.stream);
            delete S;
            return OPTA_ERR_CUDA;
        }
    }
    for (int w = 0; w < c.n_workers; ++w) S->workers[w].th = std::thread(work, S, w);
    *out = S;
    return OPTA_OK;
}

opta_status opta_server_add_image(opta_server *S, const opta_image *img, const opta_params *prm,
                                  const int32_t *sizes_mn, int32_t n_sizes, int32_t *image_id) {
    if (!S || !img || !image_id) return OPTA_ERR_INVALID_ARG;
    cudaSetDevice(S->device);
    opta_handle *h = nullptr;
    const opta_status st = optA_prepare(img, prm, sizes_mn, n_sizes, nullptr, &h);
    if (st != OPTA_OK) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    S->images.push_back(h);
    *image_id = (int32_t)S->images.size() - 1;
    return OPTA_OK;
}

opta_status opta_server_submit(opta_server *S, int32_t image_id, const opta_template *t,
                               uint64_t *request_id) {
    if (!S || !t || !t->data || t->on_device || t->rows < 1 || t->cols < 1 ||
        t->stride_elems < t->cols)
        return OPTA_ERR_INVALID_ARG;
    Request r;
    r.m = t->rows;
    r.n = t->cols;
    try {
        r.data.resize((size_t)r.m * r.n);
    } catch (...) {
        return OPTA_ERR_OOM;
    }
    for (int u = 0; u < r.m; ++u)
        std::memcpy(r.data.data() + (size_t)u * r.n, t->data + (size_t)u * t->stride_elems,
                    (size_t)r.n * sizeof(float));
    std::lock_guard<std::mutex> lk(S->mu);
    if (image_id < 0 || image_id >= (int32_t)S->images.size() || S->stop) return OPTA_ERR_INVALID_ARG;
    r.image = image_id;
    r.id = S->next_id++;
    r.t_submit = S->now();
    if (request_id) *request_id = r.id;
    try {
        S->queue.push_back(std::move(r));
    } catch (...) {
        return OPTA_ERR_OOM;
    }
    ++S->outstanding;
    S->cv_work.notify_one();
    return OPTA_OK;
}

opta_status opta_server_wait(opta_server *S, opta_completion *out, int32_t capacity,
                             int32_t min_count, int32_t timeout_ms, int32_t *n_out) {
    if (!S || !n_out || capacity < 0 || (capacity > 0 && !out)) return OPTA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const size_t want = (size_t)std::max(0, std::min(min_count, capacity));
    auto ready = [&] { return S->done.size() >= want; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    int32_t k = 0;
    while (k < capacity && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    S->outstanding -= k;
    *n_out = k;
    return OPTA_OK;
}

opta_status opta_server_pending(opta_server *S, int64_t *n) {
    if (!S || !n) return OPTA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *n = S->outstanding;
    return OPTA_OK;
}

opta_status opta_server_memory(opta_server *S, int32_t image_id, int64_t *image_bytes,
                               int64_t *scratch_bytes) {
    if (!S) return OPTA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (image_bytes) {
        if (image_id < 0 || image_id >= (int32_t)S->images.size()) return OPTA_ERR_INVALID_ARG;
        size_t b = 0;
        const opta_status st = optA_memory_bytes(S->images[image_id], &b);
        if (st != OPTA_OK) return st;
        *image_bytes = (int64_t)b;
    }
    if (scratch_bytes) *scratch_bytes = (int64_t)S->used;
    return OPTA_OK;
}

opta_status opta_server_destroy(opta_server *S) {
    if (!S) return OPTA_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (Worker &W : S->workers)
        if (W.th.joinable()) W.th.join();
    cudaSetDevice(S->device);
    for (Worker &W : S->workers) {
        release_ctx(S, W);
        if (W.stream) cudaStreamDestroy(W.stream);
    }
    for (opta_handle *h : S->images) optA_destroy(h);
    delete S;
    return OPTA_OK;
}

}  // extern "C"
