// Request loop over resident paths, index and Panther++ vectors (no
// counterpart in the paper).
//
// Requests (top-k or k-NN, 1..Qmax query vertices, their own k) are queued by
// any host thread. Each of `streams` workers owns a context (one CUDA stream)
// and device buffers sized from the memory budget; a free worker takes the
// oldest pending requests of one kind whose queries fit its buffers, runs
// them as ONE batched call with k = the largest k among them, and hands each
// request its rows. Ranking is a total order (count desc / distance asc, then
// id asc), so the first k entries of a k_max list are exactly the top-k: a
// result in the mix equals the result of the same request alone. Several
// workers run concurrently, so batches that arrive while others are on the
// GPU start as soon as a worker and its memory are free.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int kind;
    const int32_t* queries;
    int64_t q;
    int k;
    int32_t* out_ids;
    void* out_vals;
    clk::time_point t_submit;
    bool done = false;
    panther_status status = PANTHER_OK;
    double latency_ms = 0;
};

struct Worker {
    panther_ctx* ctx = nullptr;
    int32_t* d_q = nullptr;       // [qmax]
    int32_t* d_ids = nullptr;     // [qmax * 64]
    void* d_vals = nullptr;       // [qmax * 64] 8-byte values
    int32_t* h_q = nullptr;       // pinned staging
    int32_t* h_ids = nullptr;
    uint64_t* h_vals = nullptr;
    std::thread th;
};

constexpr int KMAX_TOPK = 64, KMAX_KNN = 32;

}  // namespace

struct panther_server {
    int device = 0;
    const panther_index* ix = nullptr;
    const panther_paths* paths = nullptr;
    const pantherpp_vecs* vecs = nullptr;
    int64_t qmax = 0;
    int max_inflight = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::map<int64_t, Request*> all;
    int64_t next_ticket = 1;
    bool stop = false;
    int busy = 0;
    int64_t st_submitted = 0, st_completed = 0, st_batches = 0, st_max_batch = 0, st_max_busy = 0, st_refused = 0;
    std::vector<Worker> workers;
};

panther_status topk_run(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, const int32_t* queries,
                        int64_t q, int k, int32_t* ids, uint32_t* cnt, bool plain);

static void worker_loop(panther_server* s, Worker* w) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Request*> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty(); });
            if (s->stop && s->pending.empty()) return;
            // oldest request decides the kind; take FIFO while the queries fit
            int kind = s->pending.front()->kind;
            int64_t used = 0;
            for (auto it = s->pending.begin(); it != s->pending.end();) {
                Request* r = *it;
                if (r->kind == kind && used + r->q <= s->qmax) {
                    used += r->q;
                    batch.push_back(r);
                    it = s->pending.erase(it);
                } else {
                    ++it;
                }
            }
            ++s->busy;
            ++s->st_batches;
            if ((int64_t)batch.size() > s->st_max_batch) s->st_max_batch = (int64_t)batch.size();
            if (s->busy > s->st_max_busy) s->st_max_busy = s->busy;
        }
        const int kind = batch[0]->kind;
        int kmax = 0;
        int64_t nq = 0;
        for (Request* r : batch) {
            memcpy(w->h_q + nq, r->queries, sizeof(int32_t) * r->q);
            nq += r->q;
            if (r->k > kmax) kmax = r->k;
        }
        panther_ctx* c = w->ctx;
        panther_status st = PANTHER_OK;
        cudaError_t e = cudaMemcpyAsync(w->d_q, w->h_q, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, c->stream);
        if (e) st = cuda_err(c, e, "serve upload");
        if (!st) {
            if (kind == 0)
                st = topk_run(c, s->ix, s->paths, w->d_q, nq, kmax, w->d_ids, (uint32_t*)w->d_vals, false);
            else
                st = pantherpp_knn(c, s->vecs, w->d_q, nq, kmax, w->d_ids, (uint64_t*)w->d_vals,
                                   PANTHER_KNN_BF16_SCREEN);
        }
        if (!st) {
            size_t vb = kind == 0 ? 4 : 8;
            if ((e = cudaMemcpyAsync(w->h_ids, w->d_ids, sizeof(int32_t) * nq * kmax, cudaMemcpyDeviceToHost,
                                     c->stream)) ||
                (e = cudaMemcpyAsync(w->h_vals, w->d_vals, vb * nq * kmax, cudaMemcpyDeviceToHost, c->stream)))
                st = cuda_err(c, e, "serve download");
        }
        if (!st) st = panther_sync(c);
        // hand out rows: request r gets its queries' first r->k entries
        int64_t off = 0;
        auto t_done = clk::now();
        for (Request* r : batch) {
            if (!st) {
                for (int64_t i = 0; i < r->q; ++i) {
                    memcpy(r->out_ids + i * r->k, w->h_ids + (off + i) * kmax, sizeof(int32_t) * r->k);
                    if (kind == 0)
                        memcpy((uint32_t*)r->out_vals + i * r->k, (uint32_t*)w->h_vals + (off + i) * kmax,
                               sizeof(uint32_t) * r->k);
                    else
                        memcpy((uint64_t*)r->out_vals + i * r->k, w->h_vals + (off + i) * kmax,
                               sizeof(uint64_t) * r->k);
                }
            }
            off += r->q;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (Request* r : batch) {
                r->status = st;
                r->latency_ms = std::chrono::duration<double, std::milli>(t_done - r->t_submit).count();
                r->done = true;
                ++s->st_completed;
            }
            --s->busy;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

extern "C" {

panther_status panther_serve_create(int device, const panther_index* ix, const panther_paths* p,
                                    const pantherpp_vecs* v, int64_t mem_budget_bytes, int max_inflight_requests,
                                    int streams, panther_server** out) {
    if (!out || !ix || !p) return PANTHER_EINVAL;
    *out = nullptr;
    if (ix->n != p->n || ix->R != p->R || (v && v->n != ix->n)) return PANTHER_EINVAL;
    if (streams < 1 || streams > 16 || max_inflight_requests < 1 || mem_budget_bytes < (1 << 20))
        return PANTHER_EINVAL;
    auto* s = new panther_server();
    s->device = device;
    s->ix = ix;
    s->paths = p;
    s->vecs = v;
    s->max_inflight = max_inflight_requests;
    // per query: id + 64 ids/values of 8 bytes, plus the top-k classification lists
    const int64_t per_q = 4 + KMAX_TOPK * (4 + 8) + 16;
    s->qmax = mem_budget_bytes / streams / per_q;
    if (s->qmax < 1) {
        delete s;
        return PANTHER_ENOMEM;
    }
    s->workers.resize(streams);
    for (Worker& w : s->workers) {
        panther_status st = panther_create(&w.ctx, device, nullptr);
        bool ok = st == PANTHER_OK;
        if (ok) {
            // k-NN needs its scratch inside the budget too: share it per worker
            panther_set_scratch_budget(w.ctx, std::max<int64_t>(mem_budget_bytes / streams / 2, 1 << 20));
            ok = cudaMalloc(&w.d_q, sizeof(int32_t) * s->qmax) == cudaSuccess &&
                 cudaMalloc(&w.d_ids, sizeof(int32_t) * s->qmax * KMAX_TOPK) == cudaSuccess &&
                 cudaMalloc(&w.d_vals, 8 * s->qmax * KMAX_TOPK) == cudaSuccess &&
                 cudaMallocHost(&w.h_q, sizeof(int32_t) * s->qmax) == cudaSuccess &&
                 cudaMallocHost(&w.h_ids, sizeof(int32_t) * s->qmax * KMAX_TOPK) == cudaSuccess &&
                 cudaMallocHost(&w.h_vals, 8 * s->qmax * KMAX_TOPK) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            panther_serve_destroy(s);
            return PANTHER_ENOMEM;
        }
    }
    for (Worker& w : s->workers) w.th = std::thread(worker_loop, s, &w);
    *out = s;
    return PANTHER_OK;
}

panther_status panther_serve_submit(panther_server* s, int kind, const int32_t* queries, int64_t q, int k,
                                    int32_t* out_ids, void* out_vals, int64_t* ticket) {
    if (!s || !queries || !out_ids || !out_vals || !ticket || q < 1) return PANTHER_EINVAL;
    if (kind != 0 && kind != 1) return PANTHER_EINVAL;
    if (kind == 1 && !s->vecs) return PANTHER_EINVAL;
    if (k < 1 || k > (kind == 0 ? KMAX_TOPK : KMAX_KNN)) return PANTHER_EINVAL;
    const int64_t n = s->ix->n;
    for (int64_t i = 0; i < q; ++i)
        if (queries[i] < 0 || queries[i] >= n) return PANTHER_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return PANTHER_EBUSY;
    int64_t open = (int64_t)s->all.size();
    if (q > s->qmax || open >= s->max_inflight) {
        ++s->st_refused;
        return PANTHER_EBUSY;
    }
    auto* r = new Request{s->next_ticket++, kind, queries, q, k, out_ids, out_vals, clk::now()};
    s->all[r->ticket] = r;
    s->pending.push_back(r);
    ++s->st_submitted;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return PANTHER_OK;
}

panther_status panther_serve_wait(panther_server* s, int64_t ticket, double timeout_s, double* latency_ms) {
    if (!s) return PANTHER_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return PANTHER_EINVAL;
    Request* r = it->second;
    bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9),
                                  [&] { return r->done; });
    if (!ok) return PANTHER_ETIMEOUT;
    if (latency_ms) *latency_ms = r->latency_ms;
    panther_status st = r->status;
    s->all.erase(it);
    delete r;
    return st;
}

panther_status panther_serve_stats(panther_server* s, int64_t stats[6]) {
    if (!s || !stats) return PANTHER_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    stats[0] = s->st_submitted;
    stats[1] = s->st_completed;
    stats[2] = s->st_batches;
    stats[3] = s->st_max_batch;
    stats[4] = s->st_max_busy;
    stats[5] = s->st_refused;
    return PANTHER_OK;
}

void panther_serve_destroy(panther_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (Worker& w : s->workers)
        if (w.th.joinable()) w.th.join();
    for (Worker& w : s->workers) {
        if (w.ctx) cudaSetDevice(w.ctx->device);
        cudaFree(w.d_q);
        cudaFree(w.d_ids);
        cudaFree(w.d_vals);
        cudaFreeHost(w.h_q);
        cudaFreeHost(w.h_ids);
        cudaFreeHost(w.h_vals);
        panther_destroy(w.ctx);
    }
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

}  // extern "C"
