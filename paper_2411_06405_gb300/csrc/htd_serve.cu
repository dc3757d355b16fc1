// htd_serve.cu -- served decomposition: a request loop with continuous batching.
//
// Requests (a graph as raw pairs on the host, and its hop threshold h) arrive at any time
// through htd_server_submit.  Each is admitted, in arrival order, once an estimate of its
// device footprint fits in the server's memory budget next to the requests already
// admitted; admitted requests are run by a pool of worker threads, each with its own
// stream and its own graph handle, so the rounds of different requests overlap on the
// device while each request's CSR and peel state stay resident until its result is copied
// back.  A request that still runs out of device memory goes back to the head of the queue
// and is retried once other requests have finished (alone, it fails with HTD_ENOMEM).
// Every request is an ordinary decomposition of its own graph (Def. 4; Sec. 3 peeling), so
// its result does not depend on what else runs.  Host code only: the device work is the
// library's own kernels, called through the entry points of htd_api.cu.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "htd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    int32_t n = 0, h = 0;
    std::vector<int32_t> src, dst;
    int64_t est = 0;
    // result
    std::vector<int32_t> eu, ev, truss;
    int64_t m = 0;
    htd_status status = HTD_OK;
    std::string error;
    htd_stats stats{};
    double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
    int32_t worker = -1;
    int32_t retries = 0;
    bool done = false;
};

using ReqPtr = std::shared_ptr<Request>;

}  // namespace

struct htd_server {
    int device = 0;
    int32_t nworkers = 0;
    int64_t budget = 0;
    uint32_t flags = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work;   // workers wait for admitted requests
    std::condition_variable cv_done;   // waiters wait for results
    std::deque<ReqPtr> pending;        // arrived, not yet admitted (arrival order)
    std::deque<ReqPtr> admitted;       // admitted, not yet taken by a worker
    std::unordered_map<int64_t, ReqPtr> live;  // every request not yet collected
    int64_t reserved = 0;              // estimates of the admitted and running requests
    int32_t running = 0;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> threads;
    int64_t peak_reserved = 0;
    int32_t peak_running = 0;
};

namespace {

double seconds_since(const htd_server *S) {
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

// Admits pending requests in arrival order while their estimates fit the budget; a
// request larger than the whole budget is admitted alone.  Called with the lock held.
void admit_locked(htd_server *S) {
    bool any = false;
    while (!S->pending.empty()) {
        ReqPtr r = S->pending.front();
        const bool fits = S->reserved + r->est <= S->budget;
        const bool alone = S->reserved == 0 && S->running == 0 && S->admitted.empty();
        if (!fits && !alone) break;
        S->pending.pop_front();
        S->reserved += r->est;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        r->t_admit = seconds_since(S);
        S->admitted.push_back(r);
        any = true;
    }
    if (any) S->cv_work.notify_all();
}

// Device buffers a worker keeps between requests (grown as needed).
struct WorkerBufs {
    int32_t *src = nullptr, *dst = nullptr, *truss = nullptr, *eu = nullptr, *ev = nullptr;
    int64_t cap_in = 0, cap_out = 0;
    int32_t *h_in = nullptr, *h_out = nullptr;  // pinned staging: 2 x cap_in, 3 x cap_out
    void release() {
        cudaFree(src);
        cudaFree(dst);
        cudaFree(truss);
        cudaFree(eu);
        cudaFree(ev);
        if (h_in) cudaFreeHost(h_in);
        if (h_out) cudaFreeHost(h_out);
        *this = WorkerBufs{};
    }
};

cudaError_t grow(WorkerBufs &b, int64_t m_in) {
    const int64_t need = std::max<int64_t>(m_in, 1);
    if (need > b.cap_in) {
        cudaFree(b.src);
        cudaFree(b.dst);
        cudaFree(b.truss);
        cudaFree(b.eu);
        cudaFree(b.ev);
        if (b.h_in) cudaFreeHost(b.h_in);
        if (b.h_out) cudaFreeHost(b.h_out);
        b = WorkerBufs{};
        cudaError_t e = cudaMalloc(&b.src, need * 4);
        if (e == cudaSuccess) e = cudaMalloc(&b.dst, need * 4);
        if (e == cudaSuccess) e = cudaMalloc(&b.truss, need * 4);
        if (e == cudaSuccess) e = cudaMalloc(&b.eu, need * 4);
        if (e == cudaSuccess) e = cudaMalloc(&b.ev, need * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&b.h_in, 2 * need * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&b.h_out, 3 * need * 4);
        if (e != cudaSuccess) {
            b.release();
            return e;
        }
        b.cap_in = b.cap_out = need;
    }
    return cudaSuccess;
}

// One request on a worker's stream: copy in, build the graph, decompose, copy out.
htd_status run_request(htd_server *S, Request &r, cudaStream_t s, WorkerBufs &b) {
    const int64_t m_in = (int64_t)r.src.size();
    cudaError_t e = grow(b, m_in);
    if (e != cudaSuccess) {
        r.error = std::string("server: staging buffers: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HTD_ENOMEM : HTD_ECUDA;
    }
    if (m_in > 0) {
        std::memcpy(b.h_in, r.src.data(), m_in * 4);
        std::memcpy(b.h_in + m_in, r.dst.data(), m_in * 4);
        e = cudaMemcpyAsync(b.src, b.h_in, m_in * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.dst, b.h_in + m_in, m_in * 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            r.error = std::string("server: input copy: ") + cudaGetErrorString(e);
            return HTD_ECUDA;
        }
    }
    htd_graph *g = nullptr;
    htd_status st = htd_build_csr(r.n, b.src, b.dst, m_in, 1, s, &g);
    if (st != HTD_OK) {
        r.error = htd_last_error();
        return st;
    }
    int32_t n = 0;
    int64_t m = 0;
    htd_graph_info(g, &n, &m);
    st = htd_truss_decompose_ex(g, r.h, S->flags, b.truss, nullptr, &r.stats, s);
    if (st == HTD_OK) st = htd_edges(g, b.eu, b.ev, s);
    if (st != HTD_OK) r.error = htd_last_error();
    if (st == HTD_OK && m > 0) {
        e = cudaMemcpyAsync(b.h_out, b.eu, m * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_out + m, b.ev, m * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_out + 2 * m, b.truss, m * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            r.error = std::string("server: result copy: ") + cudaGetErrorString(e);
            st = HTD_ECUDA;
        }
    }
    if (st == HTD_OK) {
        r.m = m;
        r.eu.assign(b.h_out, b.h_out + m);
        r.ev.assign(b.h_out + m, b.h_out + 2 * m);
        r.truss.assign(b.h_out + 2 * m, b.h_out + 3 * m);
    }
    htd_graph_free(g);
    return st;
}

void worker_main(htd_server *S, int wid) {
    cudaSetDevice(S->device);
    cudaStream_t s = nullptr;
    const cudaError_t se = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    WorkerBufs bufs;
    for (;;) {
        ReqPtr r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->admitted.empty(); });
            if (S->admitted.empty()) break;  // stopping and nothing left
            r = S->admitted.front();
            S->admitted.pop_front();
            S->running++;
            S->peak_running = std::max(S->peak_running, S->running);
            r->t_start = seconds_since(S);
            r->worker = wid;
        }
        htd_status st = HTD_ECUDA;
        if (se == cudaSuccess) st = run_request(S, *r, s, bufs);
        else r->error = "server: worker stream creation failed";
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->running--;
            S->reserved -= r->est;
            const bool others = S->running > 0 || !S->admitted.empty();
            if (st == HTD_ENOMEM && others && r->retries < 8) {
                // not enough room beside the others after all: retry when they are done
                r->retries++;
                r->stats = htd_stats{};
                S->pending.push_front(r);
            } else {
                r->status = st;
                r->t_done = seconds_since(S);
                r->done = true;
                S->cv_done.notify_all();
            }
            admit_locked(S);
        }
    }
    bufs.release();
    if (s) cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

int64_t htd_footprint_estimate(int32_t n, int64_t m_in, int32_t h, int64_t free_bytes) {
    if (n < 0 || m_in < 0) return -1;
    const double N = (double)n, M = (double)m_in;
    // CSR and per-edge peel state (each edge: 2 slots x (col, slot id, live mark) and 8 per-edge
    // int32 arrays), per-vertex arrays, work items and the staging buffers of the request
    double bytes = 4.0 * (6.0 * M + 8.0 * M) + 4.0 * 24.0 * N + 8.0 * (N + 2.0 * M / 64.0) + 5.0 * 4.0 * M;
    // balls: dense n-bit sets per vertex when they fit (radius h, plus radius 2 at h = 3,
    // plus the alive-adjacency sets), else about 16 words per vertex in the compact form
    const double W = (double)(((int64_t)n + 31) / 32 + 3) / 4.0 * 4.0;
    const double dense = 4.0 * N * W;
    const double fb = free_bytes > 0 ? (double)free_bytes : 0.0;
    if (h <= 3 && dense <= fb / 4.0) {
        bytes += dense * (h == 3 ? 2.0 : 1.0) + std::min(dense, std::min(fb / 4.0, 16.0 * (1 << 30)));
        // lost-pair tables and support-update items
        bytes += (h == 3 ? 256.0 : 64.0) * (1 << 20) + 16.0 * std::min(256.0 * M, (double)(1 << 30)) / 32.0;
    } else {
        bytes += 4.0 * N * std::min(W, 64.0);
    }
    // h >= 3: the ball builder's per-block BFS level lists (2n int32 for each of up to
    // about 8 resident blocks on each of 152 SMs)
    if (h >= 3) bytes += 8.0 * N * 152.0 * 8.0;
    // h = 3 incremental: radius-3 candidate items (up to 2^25 x 16 bytes)
    if (h == 3) bytes += 16.0 * std::min(8.0 * M, (double)(1 << 25));
    return (int64_t)bytes;
}

htd_status htd_server_create(int32_t workers, int64_t budget_bytes, uint32_t flags,
                             htd_server **out) {
    if (!out || workers < 1 || workers > 64 || budget_bytes < 0) {
        htd::set_last_error("htd_server_create: NULL out, workers outside [1, 64] or negative budget");
        return HTD_EINVAL;
    }
    *out = nullptr;
    htd_server *S = new htd_server();
    cudaError_t e = cudaGetDevice(&S->device);
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        htd::set_last_error(std::string("htd_server_create: ") + cudaGetErrorString(e));
        delete S;
        return HTD_ECUDA;
    }
    // default budget: 80% of the memory free now
    S->budget = budget_bytes > 0 ? budget_bytes : (int64_t)(0.8 * (double)free_b);
    S->nworkers = workers;
    S->flags = flags;
    S->t0 = Clock::now();
    for (int i = 0; i < workers; i++) S->threads.emplace_back(worker_main, S, i);
    *out = S;
    return HTD_OK;
}

htd_status htd_server_submit(htd_server *S, int32_t n, const int32_t *src_host,
                             const int32_t *dst_host, int64_t m_in, int32_t h, int64_t *id_out) {
    if (!S || !id_out || n < 0 || n > HTD_MAX_N || m_in < 0 || h < 1 || h > HTD_MAX_H ||
        (m_in > 0 && (!src_host || !dst_host))) {
        htd::set_last_error("htd_server_submit: NULL argument, bad n, m_in or h");
        return HTD_EINVAL;
    }
    if (2 * m_in >= (int64_t)INT32_MAX) {
        htd::set_last_error("htd_server_submit: 2*m_in >= 2^31");
        return HTD_EOVERFLOW;
    }
    auto r = std::make_shared<Request>();
    r->n = n;
    r->h = h;
    r->src.assign(src_host, src_host + m_in);
    r->dst.assign(dst_host, dst_host + m_in);
    r->est = htd_footprint_estimate(n, m_in, h, S->budget);
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = seconds_since(S);
    S->live[r->id] = r;
    S->pending.push_back(r);
    admit_locked(S);
    *id_out = r->id;
    return HTD_OK;
}

htd_status htd_server_poll(htd_server *S, int64_t id, int32_t *done) {
    if (!S || !done) {
        htd::set_last_error("htd_server_poll: NULL argument");
        return HTD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->live.find(id);
    if (it == S->live.end()) {
        htd::set_last_error("htd_server_poll: unknown or already collected request");
        return HTD_EINVAL;
    }
    *done = it->second->done ? 1 : 0;
    return HTD_OK;
}

htd_status htd_server_wait(htd_server *S, int64_t id, int32_t *eu_host, int32_t *ev_host,
                           int32_t *truss_host, int64_t capacity, htd_request_info *info) {
    if (!S) {
        htd::set_last_error("htd_server_wait: NULL server");
        return HTD_EINVAL;
    }
    ReqPtr r;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->live.find(id);
        if (it == S->live.end()) {
            htd::set_last_error("htd_server_wait: unknown or already collected request");
            return HTD_EINVAL;
        }
        r = it->second;
        S->cv_done.wait(lk, [&] { return r->done; });
        if (r->status == HTD_OK && r->m > capacity) {
            // the request stays collectable with larger buffers
            if (info) info->m = r->m;
            htd::set_last_error("htd_server_wait: result buffers hold fewer than m entries");
            return HTD_EINVAL;
        }
        if (r->status == HTD_OK && r->m > 0 && (!eu_host || !ev_host || !truss_host)) {
            htd::set_last_error("htd_server_wait: NULL result buffer");
            return HTD_EINVAL;
        }
        S->live.erase(it);
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->m = r->m;
        info->h = r->h;
        info->status = r->status;
        info->worker = r->worker;
        info->retries = r->retries;
        info->est_bytes = r->est;
        info->submit_s = r->t_submit;
        info->admit_s = r->t_admit;
        info->start_s = r->t_start;
        info->done_s = r->t_done;
        info->rounds = r->stats.rounds;
    }
    if (r->status != HTD_OK) {
        htd::set_last_error(r->error);
        return r->status;
    }
    if (r->m > 0) {
        std::memcpy(eu_host, r->eu.data(), r->m * 4);
        std::memcpy(ev_host, r->ev.data(), r->m * 4);
        std::memcpy(truss_host, r->truss.data(), r->m * 4);
    }
    return HTD_OK;
}

htd_status htd_server_info(htd_server *S, htd_server_stats *out) {
    if (!S || !out) {
        htd::set_last_error("htd_server_info: NULL argument");
        return HTD_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    out->budget_bytes = S->budget;
    out->reserved_bytes = S->reserved;
    out->peak_reserved_bytes = S->peak_reserved;
    out->workers = S->nworkers;
    out->running = S->running;
    out->peak_running = S->peak_running;
    out->pending = (int32_t)S->pending.size();
    out->admitted = (int32_t)S->admitted.size();
    return HTD_OK;
}

void htd_server_destroy(htd_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // requests never admitted are dropped; admitted ones finish
        for (auto &r : S->pending) {
            r->status = HTD_EINVAL;
            r->done = true;
        }
        S->pending.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    for (auto &t : S->threads) t.join();
    delete S;
}

}  // extern "C"
