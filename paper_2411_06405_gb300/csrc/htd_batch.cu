// htd_batch.cu -- many graphs in one call (htd_truss_decompose_batched).
//
// The (k,h)-truss of a disjoint union is the union of the members' (k,h)-trusses: the
// h-support of an edge counts only vertices of its own component (Def. 2, Def. 3), and the
// union of edge sets that each satisfy Def. 4 in different components satisfies it too, so
// t(e,h) in the union equals t(e,h) in e's own graph.  The batch is therefore decomposed as
// few large disjoint unions: the graphs of one hop threshold h are taken in input order
// and packed, with their vertex ids shifted, into unions of at most `max_union_vertices`
// vertices; each union is one peel on the device (every round of it serves all of its
// members at once).  Because ids are shifted by increasing offsets, the union's canonical
// (lexicographic) edge order is its members' canonical orders one after the other, so
// every member's result is a contiguous slice of the union's output.
#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "htd_internal.h"

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr int32_t kDefaultUnionVertices = 1 << 18;
constexpr int kBatchWorkers = 8;  // unions peeled at the same time (each on its own stream)
constexpr int64_t kMaxUnionPairs = ((int64_t)1 << 30) - 1;  // 2 m_in < 2^31

// One member graph of a union: its input pairs [pair_begin, pair_begin + count) land at
// union pairs [out_begin, out_begin + count), ids shifted by voff and checked against n.
struct Member {
    int64_t pair_begin;
    int64_t out_begin;
    int64_t count;
    int32_t voff;
    int32_t n;
};

// Copies the members' pairs into the union's arrays with shifted ids.  An id outside
// [0, n) of its own graph records the smallest such member index in *bad (and the pair
// becomes a loop, which normalisation drops).
__global__ void k_union_gather(const Member *__restrict__ mem, int nmem, int64_t total,
                               const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                               int32_t *__restrict__ usrc, int32_t *__restrict__ udst, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        // the member whose output range holds i (ranges are in increasing order)
        int lo = 0, hi = nmem - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mem[mid].out_begin <= i) lo = mid;
            else hi = mid - 1;
        }
        const Member M = mem[lo];
        const int64_t p = M.pair_begin + (i - M.out_begin);
        int32_t s = src[p], d = dst[p];
        if (s < 0 || s >= M.n || d < 0 || d >= M.n) {
            atomicMin(bad, lo);
            s = 0;
            d = 0;
        }
        usrc[i] = s + M.voff;
        udst[i] = d + M.voff;
    }
}

void add_stats(htd_stats *acc, const htd_stats &s) {
    acc->rounds += s.rounds;
    acc->levels += s.levels;
    acc->max_truss = std::max(acc->max_truss, s.max_truss);
    acc->h = std::max(acc->h, s.h);
    acc->hsup_evals += s.hsup_evals;
    acc->ball_builds += s.ball_builds;
    acc->balls_changed += s.balls_changed;
    acc->frontier_edges += s.frontier_edges;
    acc->pairs_tested += s.pairs_tested;
    acc->pairs_lost += s.pairs_lost;
    acc->member_tests += s.member_tests;
    acc->kernel_launches += s.kernel_launches;
    acc->ball_pool_bytes = std::max(acc->ball_pool_bytes, s.ball_pool_bytes);
    acc->timed_slots += s.timed_slots;
    acc->alg_bytes_ball += s.alg_bytes_ball;
    acc->alg_bytes_hsup += s.alg_bytes_hsup;
    acc->alg_bytes_hsup_initial += s.alg_bytes_hsup_initial;
    acc->alg_bytes_detect += s.alg_bytes_detect;
    acc->alg_bytes_update += s.alg_bytes_update;
    acc->ms_initial_ball += s.ms_initial_ball;
    acc->ms_initial_hsup += s.ms_initial_hsup;
    acc->ms_select += s.ms_select;
    acc->ms_find += s.ms_find;
    acc->ms_remove += s.ms_remove;
    acc->ms_ball += s.ms_ball;
    acc->ms_update += s.ms_update;
    acc->ms_minreduce += s.ms_minreduce;
    acc->ms_round_kernel += s.ms_round_kernel;
    acc->round_kernel_launches += s.round_kernel_launches;
    acc->slots += s.slots;
    acc->pairs3_tested += s.pairs3_tested;
    acc->pairs2_lost += s.pairs2_lost;
    acc->rounds_rebuilt += s.rounds_rebuilt;
}

// One union of the plan: its hop threshold and members (graph ids, in input order).
struct UnionPlan {
    int32_t h;
    std::vector<Member> mem;
    std::vector<int32_t> ids;
    int64_t n;      // vertices
    int64_t pairs;  // raw pairs
};

// Checks the batch description and packs it: graphs of each h in input order, a new
// union whenever the next graph would take it past cap_n vertices or 2^30 - 1 pairs (a
// graph larger than cap_n forms a union alone).
htd_status plan_unions(const char *who, int32_t num_graphs, const int32_t *n, const int32_t *h,
                       const int64_t *edge_offsets, int32_t max_union_vertices,
                       std::vector<UnionPlan> *plan, const std::vector<char> *include = nullptr) {
    if (num_graphs < 0 || (num_graphs > 0 && (!n || !h || !edge_offsets))) {
        set_last_error(std::string(who) + ": NULL argument or num_graphs < 0");
        return HTD_EINVAL;
    }
    if (num_graphs > 0 && edge_offsets[0] != 0) {
        set_last_error(std::string(who) + ": edge_offsets[0] must be 0");
        return HTD_EINVAL;
    }
    for (int32_t g = 0; g < num_graphs; g++) {
        if (n[g] < 0 || h[g] < 1 || h[g] > HTD_MAX_H || edge_offsets[g + 1] < edge_offsets[g]) {
            set_last_error(std::string(who) + ": graph " + std::to_string(g) +
                           ": n < 0, h outside [1, HTD_MAX_H] or decreasing edge_offsets");
            return HTD_EINVAL;
        }
        if (n[g] > HTD_MAX_N) {
            set_last_error(std::string(who) + ": graph " + std::to_string(g) + ": n exceeds HTD_MAX_N");
            return HTD_EUNSUPPORTED;
        }
        if (edge_offsets[g + 1] - edge_offsets[g] > kMaxUnionPairs) {
            set_last_error(std::string(who) + ": graph " + std::to_string(g) + ": 2*m_in >= 2^31");
            return HTD_EOVERFLOW;
        }
    }
    const int32_t cap_n = max_union_vertices > 0 ? std::min<int32_t>(max_union_vertices, HTD_MAX_N)
                                                 : kDefaultUnionVertices;
    plan->clear();
    for (int32_t hh = 1; hh <= HTD_MAX_H; hh++) {
        for (int32_t g = 0; g < num_graphs; g++) {
            if (h[g] != hh || (include && !(*include)[g])) continue;
            const int64_t cnt = edge_offsets[g + 1] - edge_offsets[g];
            if (plan->empty() || plan->back().h != hh || plan->back().n + n[g] > cap_n ||
                plan->back().pairs + cnt > kMaxUnionPairs) {
                plan->push_back(UnionPlan{hh, {}, {}, 0, 0});
            }
            UnionPlan &u = plan->back();
            u.mem.push_back(Member{edge_offsets[g], u.pairs, cnt, (int32_t)u.n, n[g]});
            u.ids.push_back(g);
            u.n += n[g];
            u.pairs += cnt;
        }
    }
    return HTD_OK;
}

// Frees the union's scratch on every exit path.
struct UnionScratch {
    Member *mem = nullptr;
    int32_t *usrc = nullptr, *udst = nullptr;
    int *bad = nullptr;
    htd_graph *g = nullptr;
    ~UnionScratch() {
        if (g) htd_graph_free(g);
        cudaFree(mem);
        cudaFree(usrc);
        cudaFree(udst);
        cudaFree(bad);
    }
};

// Gathers a union's pairs (ids shifted), builds its graph on U->g and finds each member's
// range [b[j], t[j]) of the union's canonical edges (the edges whose smaller endpoint lies
// in the member's id range).  *mu receives the union's edge count.  A union without any
// pair builds nothing (mu = 0, empty ranges).
htd_status build_union(const UnionPlan &up, const int32_t *src_dev, const int32_t *dst_dev,
                       void *stream, UnionScratch *U, int64_t *mu_out, std::vector<int64_t> *b,
                       std::vector<int64_t> *t, bool unused = false) {
    (void)unused;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::vector<Member> &mem = up.mem;
    const std::vector<int32_t> &ids = up.ids;
    const int64_t nu = up.n, pairs = up.pairs;
    b->assign(mem.size(), 0);
    t->assign(mem.size(), 0);
    *mu_out = 0;
    if (pairs == 0) return HTD_OK;
    cudaError_t e = cudaMalloc(&U->mem, mem.size() * sizeof(Member));
    if (e == cudaSuccess) e = cudaMalloc(&U->usrc, pairs * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&U->udst, pairs * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&U->bad, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(U->mem, mem.data(), mem.size() * sizeof(Member), cudaMemcpyHostToDevice, s);
    const int none = INT32_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(U->bad, &none, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>((pairs + kBlock - 1) / kBlock, 4096);
        k_union_gather<<<(unsigned)blocks, kBlock, 0, s>>>(U->mem, (int)mem.size(), pairs, src_dev, dst_dev,
                                                          U->usrc, U->udst, U->bad);
        add_launches(1);
        e = cudaGetLastError();
    }
    int bad = INT32_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, U->bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string("htd_truss_decompose_batched: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HTD_ENOMEM : HTD_ECUDA;
    }
    if (bad != INT32_MAX) {
        set_last_error("htd_truss_decompose_batched: graph " + std::to_string(ids[bad]) +
                       ": an endpoint outside [0, n)");
        return HTD_EINVAL;
    }
    htd_status st = htd_build_csr((int32_t)nu, U->usrc, U->udst, pairs, 1, stream, &U->g);
    if (st != HTD_OK) return st;
    int32_t nn = 0;
    int64_t mu = 0;
    htd_graph_info(U->g, &nn, &mu);
    std::vector<int32_t> eu(mu > 0 ? mu : 1);
    if (mu > 0) {
        e = cudaMemcpyAsync(eu.data(), graph_dev(U->g)->eu, mu * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_last_error(std::string("htd_truss_decompose_batched: ") + cudaGetErrorString(e));
            return HTD_ECUDA;
        }
    }
    for (size_t j = 0; j < mem.size(); j++) {
        const int32_t lo_id = mem[j].voff, hi_id = mem[j].voff + mem[j].n;
        (*b)[j] = std::lower_bound(eu.begin(), eu.begin() + mu, lo_id) - eu.begin();
        (*t)[j] = std::lower_bound(eu.begin(), eu.begin() + mu, hi_id) - eu.begin();
    }
    *mu_out = mu;
    return HTD_OK;
}

int num_sms_of_current() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

}  // namespace
}  // namespace htd

extern "C" htd_status htd_truss_decompose_batched(
    int32_t num_graphs, const int32_t *n, const int32_t *h, const int64_t *edge_offsets,
    const int32_t *src_dev, const int32_t *dst_dev, uint32_t flags, int32_t max_union_vertices,
    int32_t *truss_dev, int64_t *out_offsets, int64_t *out_m, int32_t *num_unions,
    htd_stats *stats, void *stream) {
    using namespace htd;
    std::vector<UnionPlan> plan;
    const htd_status ps = plan_unions("htd_truss_decompose_batched", num_graphs, n, h, edge_offsets,
                                      max_union_vertices, &plan);
    if (ps != HTD_OK) return ps;
    if (num_graphs > 0 && (!out_offsets || !out_m)) {
        set_last_error("htd_truss_decompose_batched: NULL output array");
        return HTD_EINVAL;
    }
    const int64_t total_in = num_graphs > 0 ? edge_offsets[num_graphs] : 0;
    if (total_in > 0 && (!src_dev || !dst_dev || !truss_dev)) {
        set_last_error("htd_truss_decompose_batched: NULL device buffer");
        return HTD_EINVAL;
    }
    htd_stats acc;
    std::memset(&acc, 0, sizeof(acc));
    acc.incremental = 1;
    int32_t unions = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t out_pos = 0;
    // block mode: graphs of at most kBlockMaxN vertices and h <= 3 are peeled one per block
    const bool blocks = (flags & HTD_OPT_BATCH_BLOCKS) != 0;
    std::vector<char> small(num_graphs > 0 ? num_graphs : 1, 0), large(num_graphs > 0 ? num_graphs : 1, 1);
    if (blocks) {
        for (int32_t g = 0; g < num_graphs; g++) {
            small[g] = (n[g] <= kBlockMaxN && h[g] <= 3) ? 1 : 0;
            large[g] = !small[g];
        }
        std::vector<UnionPlan> bplan;
        const htd_status ps2 = plan_unions("htd_truss_decompose_batched", num_graphs, n, h, edge_offsets,
                                           max_union_vertices, &bplan, &small);
        if (ps2 != HTD_OK) return ps2;
        std::vector<std::unique_ptr<UnionScratch>> held;
        std::vector<BlockGraphDescHost> descs;
        for (const UnionPlan &up : bplan) {
            auto U = std::make_unique<UnionScratch>();
            std::vector<int64_t> b, t;
            int64_t mu = 0;
            const htd_status us = build_union(up, src_dev, dst_dev, stream, U.get(), &mu, &b, &t);
            if (us != HTD_OK) return us;
            GraphDev *gdv = U->g ? graph_dev(U->g) : nullptr;
            for (size_t j = 0; j < up.mem.size(); j++) {
                out_offsets[up.ids[j]] = out_pos + b[j];
                out_m[up.ids[j]] = t[j] - b[j];
                if (t[j] > b[j])
                    descs.push_back(BlockGraphDescHost{gdv->row_ptr, gdv->col, gdv->slot_eid, gdv->eu, gdv->ev,
                                                       truss_dev + out_pos + b[j], b[j], t[j] - b[j],
                                                       up.mem[j].voff, up.mem[j].n, up.h});
            }
            out_pos += mu;
            if (mu > 0) unions++;
            held.push_back(std::move(U));
        }
        int64_t rounds = 0;
        const htd_status bs = batch_block_run(descs, s, num_sms_of_current(), &rounds);
        if (bs != HTD_OK) return bs;
        acc.rounds += rounds;
        acc.frontier_edges += 0;
    }

    std::vector<UnionPlan> lplan;
    if (blocks) {
        const htd_status ps3 = plan_unions("htd_truss_decompose_batched", num_graphs, n, h, edge_offsets,
                                           max_union_vertices, &lplan, &large);
        if (ps3 != HTD_OK) return ps3;
    }
    // unions are independent peels: build them all, then peel them concurrently on worker
    // threads with their own streams (each peel's rounds are latency-bound and leave most
    // of the GPU idle), as many at once as their footprint estimates fit the free memory
    const std::vector<UnionPlan> &uplan = blocks ? lplan : plan;
    struct Built {
        std::unique_ptr<UnionScratch> U;
        int64_t mu = 0, out = 0, est = 0;
        int32_t h = 0;
        htd_stats st{};
        htd_status rc = HTD_OK;
        std::string err;
    };
    std::vector<Built> built(uplan.size());
    for (size_t u = 0; u < uplan.size(); u++) {
        const UnionPlan &up = uplan[u];
        Built &B = built[u];
        B.U = std::make_unique<UnionScratch>();
        std::vector<int64_t> b, t;
        const htd_status st = build_union(up, src_dev, dst_dev, stream, B.U.get(), &B.mu, &b, &t, true);
        if (st != HTD_OK) return st;
        for (size_t j = 0; j < up.mem.size(); j++) {
            out_offsets[up.ids[j]] = out_pos + b[j];
            out_m[up.ids[j]] = t[j] - b[j];
        }
        B.out = out_pos;
        B.h = up.h;
        out_pos += B.mu;
    }
    bool any = false;
    for (const Built &B : built) any = any || B.mu > 0;
    if (!any) {
        if (num_unions) *num_unions = unions;
        if (stats) *stats = acc;
        return HTD_OK;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        set_last_error("htd_truss_decompose_batched: cudaMemGetInfo failed");
        return HTD_ECUDA;
    }
    const int64_t budget = (int64_t)(0.7 * (double)free_b);
    for (size_t u = 0; u < uplan.size(); u++)
        built[u].est = htd_footprint_estimate((int32_t)uplan[u].n, uplan[u].pairs, uplan[u].h, budget);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaEvent_t ev_start = nullptr;
    if (cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev_start, s) != cudaSuccess) {
        set_last_error("htd_truss_decompose_batched: event on the caller's stream failed");
        if (ev_start) cudaEventDestroy(ev_start);
        return HTD_ECUDA;
    }
    const int nworkers = (int)std::min<size_t>(kBatchWorkers, std::max<size_t>(1, uplan.size()));
    std::mutex mu;
    std::condition_variable cv;
    int64_t used = 0;
    int running = 0;
    size_t next = 0;
    auto worker = [&](int wid) {
        (void)wid;
        cudaSetDevice(dev);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) ws = nullptr;
        if (ws) cudaStreamWaitEvent(ws, ev_start, 0);
        for (;;) {
            size_t i;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (next >= built.size()) break;
                i = next++;
                Built &B = built[i];
                if (B.mu == 0) continue;
                // admission: wait until the estimate fits beside the running peels (a peel
                // larger than the whole budget runs alone)
                cv.wait(lk, [&] { return used + B.est <= budget || running == 0; });
                used += B.est;
                running++;
            }
            Built &B = built[i];
            if (!ws) {
                B.rc = HTD_ECUDA;
                B.err = "htd_truss_decompose_batched: worker stream creation failed";
            } else {
                B.rc = htd_truss_decompose_ex(B.U->g, B.h, flags & ~HTD_OPT_BATCH_BLOCKS, truss_dev + B.out,
                                              nullptr, &B.st, ws);
                if (B.rc != HTD_OK) B.err = htd_last_error();
                // the union's result is in place: its graph and peel scratch go now, so that
                // the memory serves the unions still to come
                else B.U.reset();
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                used -= B.est;
                running--;
            }
            cv.notify_all();
        }
        if (ws) {
            cudaStreamSynchronize(ws);
            cudaStreamDestroy(ws);
        }
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nworkers; w++) threads.emplace_back(worker, w);
    worker(0);
    for (auto &t : threads) t.join();
    cudaEventDestroy(ev_start);
    for (Built &B : built) {
        if (B.mu == 0) continue;
        if (B.rc == HTD_ENOMEM) {
            // out of memory beside the other peels: once more, alone, on the caller's stream
            std::memset(&B.st, 0, sizeof(B.st));
            B.rc = htd_truss_decompose_ex(B.U->g, B.h, flags & ~HTD_OPT_BATCH_BLOCKS, truss_dev + B.out,
                                          nullptr, &B.st, stream);
            if (B.rc != HTD_OK) B.err = htd_last_error();
        }
        if (B.rc != HTD_OK) {
            set_last_error(B.err);
            return B.rc;
        }
        add_stats(&acc, B.st);
        if (!B.st.incremental) acc.incremental = 0;
        unions++;
    }
    if (num_unions) *num_unions = unions;
    if (stats) *stats = acc;
    return HTD_OK;
}

extern "C" htd_status htd_batch_plan(int32_t num_graphs, const int32_t *n, const int32_t *h,
                                     const int64_t *edge_offsets, int32_t max_union_vertices,
                                     int32_t *union_of, int32_t *vertex_offset, int32_t *num_unions) {
    using namespace htd;
    std::vector<UnionPlan> plan;
    const htd_status ps = plan_unions("htd_batch_plan", num_graphs, n, h, edge_offsets,
                                      max_union_vertices, &plan);
    if (ps != HTD_OK) return ps;
    if (num_graphs > 0 && (!union_of || !vertex_offset)) {
        set_last_error("htd_batch_plan: NULL output array");
        return HTD_EINVAL;
    }
    for (size_t u = 0; u < plan.size(); u++) {
        for (size_t j = 0; j < plan[u].ids.size(); j++) {
            union_of[plan[u].ids[j]] = (int32_t)u;
            vertex_offset[plan[u].ids[j]] = plan[u].mem[j].voff;
        }
    }
    if (num_unions) *num_unions = (int32_t)plan.size();
    return HTD_OK;
}
