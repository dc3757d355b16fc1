// htd_api.cu -- the extern "C" entry points declared in include/htruss.h.
//
// Every call runs on a stream private to the handle (a CUDA graph can be captured on it)
// and is ordered against the caller's stream with two events: the private stream waits
// for the caller's prior work, and the caller's stream waits for the call's work.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "htd_internal.h"

struct htd_graph {
    htd::Handle H;
};

namespace htd {

namespace {
thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
constexpr int kRoundsPerGraph = 16;
}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

cudaError_t raise_smem_limit(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[{dev, func}];
    if (cur >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}
GraphDev *graph_dev(htd_graph *g) { return &g->H.g; }
void add_launches(int64_t k) { g_launches += k; }

}  // namespace htd

using htd::Handle;
using htd::set_last_error;

#define API_CHECK(...)                                                              \
    do {                                                                             \
        cudaError_t _e = (__VA_ARGS__);                                                     \
        if (_e != cudaSuccess) {                                                     \
            set_last_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e));      \
            return (_e == cudaErrorMemoryAllocation) ? HTD_ENOMEM : HTD_ECUDA;       \
        }                                                                            \
    } while (0)

#define API_TRY(expr)                        \
    do {                                     \
        htd_status _s = (expr);              \
        if (_s != HTD_OK) return _s;         \
    } while (0)

namespace {

htd_status begin_call(Handle *H, cudaStream_t user) {
    API_CHECK(cudaSetDevice(H->g.device));
    API_CHECK(cudaEventRecord(H->ev_in, user));
    API_CHECK(cudaStreamWaitEvent(H->pstream, H->ev_in, 0));
    return HTD_OK;
}

htd_status end_call(Handle *H, cudaStream_t user) {
    API_CHECK(cudaEventRecord(H->ev_out, H->pstream));
    API_CHECK(cudaStreamWaitEvent(user, H->ev_out, 0));
    API_CHECK(cudaStreamSynchronize(H->pstream));
    return HTD_OK;
}

void destroy_graph(Handle *H) {
    if (H->graph_exec) cudaGraphExecDestroy(H->graph_exec);
    if (H->graph_exec_timed) cudaGraphExecDestroy(H->graph_exec_timed);
    H->graph_exec = nullptr;
    H->graph_exec_timed = nullptr;
    H->graph_h = 0;
    H->graph_rounds = 0;
}

htd_status check_status_err(const htd::DevStatus *st) {
    if (st->err) {
        set_last_error("htd: device-side consistency check failed (code " +
                       std::to_string(st->err) + ")");
        return HTD_ECUDA;
    }
    return HTD_OK;
}

htd_status prepare_work(Handle *H, int32_t h, bool incremental, bool tiny = false) {
    if (H->w.status && (H->w.h != h || H->w.lost_tiny != tiny)) destroy_graph(H);
    return htd::ensure_work(H, h, incremental, tiny);
}

}  // namespace

extern "C" {

const char *htd_status_string(htd_status s) {
    switch (s) {
        case HTD_OK: return "ok";
        case HTD_EINVAL: return "invalid argument";
        case HTD_ENOMEM: return "device memory allocation failed";
        case HTD_ECUDA: return "CUDA error";
        case HTD_ETIMEOUT: return "peel exceeded its round cap";
        case HTD_EOVERFLOW: return "graph too large for 32-bit adjacency offsets";
        case HTD_EUNSUPPORTED: return "graph too large for shared-memory balls";
    }
    return "unknown status";
}

const char *htd_last_error(void) { return htd::g_last_error.c_str(); }

int64_t htd_kernel_launch_count(void) { return htd::g_launches; }

void htd_graph_free(htd_graph *g) {
    if (!g) return;
    Handle *H = &g->H;
    cudaSetDevice(H->g.device);
    if (H->pstream) cudaStreamSynchronize(H->pstream);
    destroy_graph(H);
    htd::free_work(&H->w);
    htd::free_graph_dev(&H->g);
    for (cudaEvent_t e : H->round_events) cudaEventDestroy(e);
    H->round_events.clear();
    if (H->ev_in) cudaEventDestroy(H->ev_in);
    if (H->ev_out) cudaEventDestroy(H->ev_out);
    if (H->pstream) cudaStreamDestroy(H->pstream);
    delete g;
}

htd_status htd_build_csr(int32_t n, const int32_t *src, const int32_t *dst, int64_t m_in,
                         int inputs_on_device, void *stream, htd_graph **out) {
    if (!out) {
        set_last_error("htd_build_csr: out is NULL");
        return HTD_EINVAL;
    }
    *out = nullptr;
    if (n < 0 || m_in < 0 || (m_in > 0 && (!src || !dst))) {
        set_last_error("htd_build_csr: bad n, m_in or NULL endpoint array");
        return HTD_EINVAL;
    }
    if (n > HTD_MAX_N) {
        set_last_error("htd_build_csr: n exceeds HTD_MAX_N");
        return HTD_EUNSUPPORTED;
    }
    if (2 * m_in >= (int64_t)INT32_MAX) {
        set_last_error("htd_build_csr: 2*m_in >= 2^31");
        return HTD_EOVERFLOW;
    }
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    htd_graph *G = new htd_graph();
    Handle *H = &G->H;
    htd_status st = HTD_OK;
    int32_t *dsrc = nullptr, *ddst = nullptr;
    int64_t launches = 0;
    auto fail = [&](htd_status s) {
        if (dsrc) cudaFree(dsrc);
        if (ddst) cudaFree(ddst);
        htd_graph_free(G);
        return s;
    };
    {
        cudaError_t e = cudaGetDevice(&H->g.device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount,
                                                         H->g.device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H->pstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&H->ev_out, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            set_last_error(std::string("htd_build_csr: ") + cudaGetErrorString(e));
            return fail(HTD_ECUDA);
        }
    }
    st = begin_call(H, user);
    if (st != HTD_OK) return fail(st);
    const int32_t *s_dev = src, *d_dev = dst;
    if (!inputs_on_device && m_in > 0) {
        cudaError_t e = cudaMalloc(&dsrc, m_in * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&ddst, m_in * sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dsrc, src, m_in * sizeof(int32_t), cudaMemcpyHostToDevice, H->pstream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ddst, dst, m_in * sizeof(int32_t), cudaMemcpyHostToDevice, H->pstream);
        if (e != cudaSuccess) {
            set_last_error(std::string("htd_build_csr: input copy: ") + cudaGetErrorString(e));
            return fail(e == cudaErrorMemoryAllocation ? HTD_ENOMEM : HTD_ECUDA);
        }
        s_dev = dsrc;
        d_dev = ddst;
    }
    st = htd::build_csr_device(n, s_dev, d_dev, m_in, H->pstream, &H->g, &launches);
    htd::g_launches += launches;
    if (st != HTD_OK) return fail(st);
    st = end_call(H, user);
    if (st != HTD_OK) return fail(st);
    if (dsrc) cudaFree(dsrc);
    if (ddst) cudaFree(ddst);
    *out = G;
    return HTD_OK;
}

htd_status htd_graph_info(const htd_graph *g, int32_t *n, int64_t *m) {
    if (!g) {
        set_last_error("htd_graph_info: NULL handle");
        return HTD_EINVAL;
    }
    if (n) *n = g->H.g.n;
    if (m) *m = g->H.g.m;
    return HTD_OK;
}

htd_status htd_edges(const htd_graph *g, int32_t *eu_dev, int32_t *ev_dev, void *stream) {
    if (!g || (g->H.g.m > 0 && (!eu_dev || !ev_dev))) {
        set_last_error("htd_edges: NULL argument");
        return HTD_EINVAL;
    }
    Handle *H = const_cast<Handle *>(&g->H);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    API_TRY(begin_call(H, user));
    if (H->g.m > 0) {
        API_CHECK(cudaMemcpyAsync(eu_dev, H->g.eu, H->g.m * 4, cudaMemcpyDeviceToDevice, H->pstream));
        API_CHECK(cudaMemcpyAsync(ev_dev, H->g.ev, H->g.m * 4, cudaMemcpyDeviceToDevice, H->pstream));
    }
    return end_call(H, user);
}

htd_status htd_csr(const htd_graph *g, int32_t *row_ptr_dev, int32_t *col_dev,
                   int32_t *slot_eid_dev, void *stream) {
    if (!g) {
        set_last_error("htd_csr: NULL handle");
        return HTD_EINVAL;
    }
    Handle *H = const_cast<Handle *>(&g->H);
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    API_TRY(begin_call(H, user));
    const int64_t n = H->g.n, m = H->g.m;
    if (row_ptr_dev)
        API_CHECK(cudaMemcpyAsync(row_ptr_dev, H->g.row_ptr, (n + 1) * 4, cudaMemcpyDeviceToDevice,
                                  H->pstream));
    if (col_dev && m > 0)
        API_CHECK(cudaMemcpyAsync(col_dev, H->g.col, 2 * m * 4, cudaMemcpyDeviceToDevice, H->pstream));
    if (slot_eid_dev && m > 0)
        API_CHECK(cudaMemcpyAsync(slot_eid_dev, H->g.slot_eid, 2 * m * 4, cudaMemcpyDeviceToDevice,
                                  H->pstream));
    return end_call(H, user);
}

htd_status htd_h_support(htd_graph *g, int32_t h, int32_t *sup_dev, void *stream) {
    if (!g || h < 1 || h > HTD_MAX_H || (g->H.g.m > 0 && !sup_dev)) {
        set_last_error("htd_h_support: NULL argument or h outside [1, HTD_MAX_H]");
        return HTD_EINVAL;
    }
    Handle *H = &g->H;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    API_TRY(begin_call(H, user));
    API_TRY(prepare_work(H, h, h <= 2));
    H->w.dense_balls = false;  // h-support alone streams the smaller form of each ball
    H->w.inc3 = false;
    int64_t launches = 0;
    htd_status ip = htd::initial_pass(H, h, H->pstream, &launches, nullptr);
    htd::g_launches += launches;
    API_TRY(ip);
    if (H->g.m > 0)
        API_CHECK(cudaMemcpyAsync(sup_dev, H->w.sup, H->g.m * 4, cudaMemcpyDeviceToDevice, H->pstream));
    API_CHECK(cudaMemcpyAsync(H->w.status_host, H->w.status, sizeof(htd::DevStatus),
                              cudaMemcpyDeviceToHost, H->pstream));
    API_TRY(end_call(H, user));
    return check_status_err(H->w.status_host);
}

htd_status htd_truss_decompose_ex(htd_graph *g, int32_t h, uint32_t flags, int32_t *truss_dev,
                                  int32_t *stamp_dev, htd_stats *stats, void *stream) {
    if (!g || h < 1 || h > HTD_MAX_H || (g->H.g.m > 0 && !truss_dev)) {
        set_last_error("htd_truss_decompose: NULL argument or h outside [1, HTD_MAX_H]");
        return HTD_EINVAL;
    }
    Handle *H = &g->H;
    htd::PeelWork &w = H->w;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    const bool timing = (flags & HTD_OPT_TIMING) != 0;
    const bool use_graph = (flags & HTD_OPT_NO_GRAPH) == 0;
    const int R = htd::kRoundsPerGraph;
    htd_stats local;
    std::memset(&local, 0, sizeof(local));
    local.h = h;
    int64_t launches = 0;
    int64_t launches_counted = 0;
    // adds the launches enqueued since the last call to the thread's counter
    auto count_launches = [&]() {
        htd::g_launches += launches - launches_counted;
        launches_counted = launches;
    };

    API_TRY(begin_call(H, user));
    bool incremental = (flags & HTD_OPT_REBUILD) == 0;
    {
        // the incremental peel's membership tests take one load on a dense ball, a binary
        // search on a compact one: keep every ball dense when the n x n bits fit comfortably.
        // At h = 3 the incremental rounds need two dense ball sets (radius 2 and 3).
        size_t free_b = 0, total_b = 0;
        API_CHECK(cudaMemGetInfo(&free_b, &total_b));
        const double Wp = (double)(((H->g.n + 31) / 32 + 3) & ~3);
        const double dense_bytes = 4.0 * (double)H->g.n * (Wp > 0 ? Wp : 4.0);
        const bool fits = dense_bytes <= (double)free_b / 4 && dense_bytes < 4.0 * (double)((int64_t)1 << 33);
        if (h == 3 && ((flags & HTD_OPT_COMPACT_BALLS) != 0 || !(2.0 * dense_bytes <= (double)free_b / 3) ||
                       dense_bytes >= 4.0 * (double)((int64_t)1 << 33)))
            incremental = false;
        API_TRY(prepare_work(H, h, incremental, (flags & HTD_OPT_TINY_LOSS_TABLE) != 0));
        incremental = w.incremental;
        w.dense_balls = incremental && (h == 3 || ((flags & HTD_OPT_COMPACT_BALLS) == 0 && fits));
    }
    {
        htd_status ip = htd::initial_pass(H, h, H->pstream, &launches, timing ? &local : nullptr);
        if (ip == HTD_OK) ip = htd::initial_pass_r2(H, H->pstream, &launches);
        htd::g_launches += launches;
        launches_counted = launches;
        API_TRY(ip);
    }
    API_CHECK(cudaMemcpyAsync(w.status_host, w.status, sizeof(htd::DevStatus), cudaMemcpyDeviceToHost,
                              H->pstream));
    API_CHECK(cudaStreamSynchronize(H->pstream));
    API_TRY(check_status_err(w.status_host));

    const int per_round = w.inc3 ? 5 : incremental ? 4 : h + 6;
    const bool persistent = incremental && h <= 2 && (flags & HTD_OPT_PERSISTENT_ROUNDS) != 0;
    if (persistent && w.status_host->alive > 0) {
        // one cooperative launch runs up to kPersistentSlots round slots; the host checks the
        // status block between launches
        constexpr int kPersistentSlots = 4096;
        const int64_t slot_cap = H->g.m + w.status_host->st_ball_total / 2 + 2;
        const int64_t launch_cap = slot_cap / kPersistentSlots + 3;
        cudaEvent_t p0 = nullptr, p1 = nullptr;
        API_CHECK(cudaEventCreate(&p0));
        API_CHECK(cudaEventCreate(&p1));
        int64_t nlaunch = 0;
        htd_status ps = HTD_OK;
        while (ps == HTD_OK && w.status_host->alive > 0) {
            if (++nlaunch > launch_cap) {
                set_last_error("htd_truss_decompose: no progress within the slot cap");
                ps = HTD_ETIMEOUT;
                break;
            }
            if (cudaEventRecord(p0, H->pstream) != cudaSuccess) ps = HTD_ECUDA;
            if (ps == HTD_OK) ps = htd::launch_persistent_rounds(H, H->pstream, kPersistentSlots, &launches);
            if (ps == HTD_OK && cudaEventRecord(p1, H->pstream) != cudaSuccess) ps = HTD_ECUDA;
            count_launches();
            if (ps != HTD_OK) break;
            if (cudaMemcpyAsync(w.status_host, w.status, sizeof(htd::DevStatus),
                                cudaMemcpyDeviceToHost, H->pstream) != cudaSuccess ||
                cudaStreamSynchronize(H->pstream) != cudaSuccess) {
                set_last_error(std::string("htd_truss_decompose: ") +
                               cudaGetErrorString(cudaGetLastError()));
                ps = HTD_ECUDA;
                break;
            }
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p0, p1) == cudaSuccess) {
                local.ms_round_kernel += ms;
                local.round_kernel_launches += 1;
            }
            if (w.status_host->err & htd::kErrBarrierTimeout) {
                set_last_error("htd_truss_decompose: a grid barrier of the round kernel timed out");
                ps = HTD_ETIMEOUT;
                break;
            }
            ps = check_status_err(w.status_host);
        }
        cudaEventDestroy(p0);
        cudaEventDestroy(p1);
        if (ps != HTD_OK) return ps;
        const htd::DevStatus *sh = w.status_host;
        local.ms_select = sh->st_phase_ns[0] * 1e-6f;
        local.ms_find = sh->st_phase_ns[1] * 1e-6f;
        local.ms_update = sh->st_phase_ns[2] * 1e-6f;
        local.ms_minreduce = sh->st_phase_ns[3] * 1e-6f;
        local.timed_slots = sh->st_slots;
    } else if (w.status_host->alive > 0) {
        // Graph path: R rounds per graph launch.  With HTD_OPT_TIMING a second graph with an
        // external event record at every phase boundary runs every kTimedEvery-th batch (the
        // events would otherwise slow every round); per-launch averages come from those.
        constexpr int kTimedEvery = 16;
        if (timing && H->round_events.empty()) {
            H->round_events.resize(htd::kRoundEvents * R, nullptr);
            for (auto &e : H->round_events) API_CHECK(cudaEventCreate(&e));
        }
        auto capture = [&](cudaGraphExec_t *exec, cudaEvent_t *ev) -> htd_status {
            cudaGraph_t graph = nullptr;
            API_CHECK(cudaStreamBeginCapture(H->pstream, cudaStreamCaptureModeThreadLocal));
            int64_t dummy = 0;
            htd_status cs = HTD_OK;
            for (int r = 0; r < R && cs == HTD_OK; r++)
                cs = htd::enqueue_round(H, H->pstream, &dummy, ev ? ev + htd::kRoundEvents * r : nullptr);
            cudaError_t ce = cudaStreamEndCapture(H->pstream, &graph);
            if (cs != HTD_OK) {
                if (graph) cudaGraphDestroy(graph);
                return cs;
            }
            if (ce != cudaSuccess) {
                set_last_error(std::string("htd: graph capture: ") + cudaGetErrorString(ce));
                return HTD_ECUDA;
            }
            ce = cudaGraphInstantiate(exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                *exec = nullptr;
                set_last_error(std::string("htd: graph instantiate: ") + cudaGetErrorString(ce));
                return HTD_ECUDA;
            }
            return HTD_OK;
        };
        // the captured kernel arguments fix h, the round variant and the ball layout
        if (use_graph && (!H->graph_exec || H->graph_h != h || H->graph_incremental != incremental ||
                          H->graph_dense != w.dense_balls)) {
            destroy_graph(H);
            API_TRY(capture(&H->graph_exec, nullptr));
            H->graph_h = h;
            H->graph_rounds = R;
            H->graph_incremental = incremental;
            H->graph_dense = w.dense_balls;
        }
        if (use_graph && timing && !H->graph_exec_timed)
            API_TRY(capture(&H->graph_exec_timed, H->round_events.data()));
        // every active round removes at least one edge, so m/R + 2 batches always suffice
        const int64_t round_cap = H->g.m + 2 * R + 2;
        // continued incremental rounds handle at least one new lost pair per slot, and a
        // pair is lost at most once (sum of ball sizes / 2 pairs in all)
        const int64_t batch_cap =
            (H->g.m + (incremental ? w.status_host->st_ball_total / 2 + 1 : 0)) / R + 3;
        int64_t batches = 0;
        bool timing_ok = timing;
        while (w.status_host->alive > 0) {
            if (++batches > batch_cap) {
                set_last_error("htd_truss_decompose: no progress within the batch cap");
                return HTD_ETIMEOUT;
            }
            const bool timed = timing_ok && (batches % kTimedEvery == 1);
            const int64_t slots_before = w.status_host->st_slots;
            if (use_graph) {
                API_CHECK(cudaGraphLaunch(timed ? H->graph_exec_timed : H->graph_exec, H->pstream));
                launches += (int64_t)R * per_round;
            } else {
                for (int r = 0; r < R; r++) {
                    API_TRY(htd::enqueue_round(H, H->pstream, &launches,
                                               timed ? &H->round_events[htd::kRoundEvents * r] : nullptr));
                }
            }
            count_launches();
            API_CHECK(cudaMemcpyAsync(w.status_host, w.status, sizeof(htd::DevStatus),
                                      cudaMemcpyDeviceToHost, H->pstream));
            API_CHECK(cudaStreamSynchronize(H->pstream));
            API_TRY(check_status_err(w.status_host));
            const bool halted = w.status_host->halt != 0;
            if (halted) {
                // an h = 3 round ran out of room: finish it by rebuilds, then go on (the
                // batch's sampled events then cover idle rounds and are not used)
                API_TRY(htd::recover_round_h3(H, H->pstream, &launches));
                count_launches();
                API_CHECK(cudaMemcpyAsync(w.status_host, w.status, sizeof(htd::DevStatus),
                                          cudaMemcpyDeviceToHost, H->pstream));
                API_CHECK(cudaStreamSynchronize(H->pstream));
                API_TRY(check_status_err(w.status_host));
            }
            if (timed && !halted) {
                // only the slots that ran a round (or a batch of one) count; those after the
                // last round are no-ops
                const int64_t active = std::min<int64_t>(R, w.status_host->st_slots - slots_before);
                for (int r = 0; r < active && timing_ok; r++) {
                    float t[htd::kRoundEvents - 1];
                    for (int q = 0; q + 1 < htd::kRoundEvents; q++) {
                        if (cudaEventElapsedTime(&t[q], H->round_events[htd::kRoundEvents * r + q],
                                                 H->round_events[htd::kRoundEvents * r + q + 1]) !=
                            cudaSuccess) {
                            (void)cudaGetLastError();  // not sticky: report "no timing" instead
                            timing_ok = false;
                            break;
                        }
                    }
                    if (!timing_ok) break;
                    local.ms_select += t[0];
                    if (incremental) {
                        local.ms_remove += t[1];
                        local.ms_find += t[2];
                        local.ms_update += t[3] + t[4];
                    } else {
                        local.ms_find += t[1];
                        local.ms_remove += t[2];
                        local.ms_ball += t[3];
                        local.ms_update += t[4];
                    }
                    local.ms_minreduce += t[5];
                    local.timed_slots += 1;
                }
                if (!timing_ok) local.timed_slots = -1;
            }
            if (w.status_host->round > round_cap) {
                set_last_error("htd_truss_decompose: round cap exceeded");
                return HTD_ETIMEOUT;
            }
        }
    }
    const int64_t m = H->g.m;
    if (m > 0) {
        API_CHECK(cudaMemcpyAsync(truss_dev, w.truss, m * 4, cudaMemcpyDeviceToDevice, H->pstream));
        if (stamp_dev)
            API_CHECK(cudaMemcpyAsync(stamp_dev, w.stamp, m * 4, cudaMemcpyDeviceToDevice, H->pstream));
    }
    API_TRY(end_call(H, user));
    if (stats) {
        const htd::DevStatus *s = w.status_host;
        local.rounds = s->round;
        local.levels = s->levels;
        local.max_truss = s->max_k;
        local.hsup_evals = m + s->st_recomputed;
        local.pairs_tested = s->st_pairs;
        local.pairs_lost = s->st_lost;
        local.member_tests = s->st_tests;
        local.incremental = incremental ? 1 : 0;
        local.slots = s->st_slots;
        local.levels = s->levels;
        local.ball_builds = H->g.n + s->st_candidates;
        local.balls_changed = s->st_changed;
        local.frontier_edges = s->st_frontier;
        local.alg_bytes_ball = (double)s->st_bytes_ball;
        local.alg_bytes_hsup = (double)s->st_bytes_hsup;
        local.alg_bytes_hsup_initial = (double)s->st_bytes_hsup_init;
        local.alg_bytes_detect = (double)s->st_bytes_detect;
        local.alg_bytes_update = (double)s->st_bytes_update;
        local.kernel_launches = launches;
        local.ball_pool_bytes = (w.pool_used + (w.inc3 ? (int64_t)H->g.n * w.Wpad : 0)) * 4;
        local.pairs3_tested = s->st_c3_pairs;
        local.pairs2_lost = s->st_lost2;
        local.rounds_rebuilt = s->st_recovered;
        *stats = local;
    }
    return HTD_OK;
}

htd_status htd_hindex_decompose_ex(htd_graph *g, int32_t h, int32_t sweeps, int32_t max_iter,
                                   uint32_t flags, int32_t *truss_dev, int32_t *hval_dev,
                                   htd_hindex_stats *stats, void *stream) {
    if (!g || h < 1 || h > HTD_MAX_H || sweeps < 1 || sweeps > 4096 || (flags & ~HTD_HX_PRUNE) != 0u ||
        ((flags & HTD_HX_PRUNE) && sweeps != 1)) {
        set_last_error("htd_hindex_decompose: NULL handle, h outside [1, HTD_MAX_H], sweeps outside "
                       "[1, 4096], unknown flags, or pruning with sweeps != 1");
        return HTD_EINVAL;
    }
    Handle *H = &g->H;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    API_TRY(begin_call(H, user));
    API_TRY(htd::hindex_run(g, H, h, sweeps, max_iter, (flags & HTD_HX_PRUNE) != 0u, truss_dev, hval_dev,
                            stats, H->pstream));
    return end_call(H, user);
}

htd_status htd_hindex_decompose(htd_graph *g, int32_t h, int32_t sweeps, int32_t max_iter,
                                int32_t *truss_dev, int32_t *hval_dev, htd_hindex_stats *stats,
                                void *stream) {
    return htd_hindex_decompose_ex(g, h, sweeps, max_iter, 0u, truss_dev, hval_dev, stats, stream);
}

htd_status htd_truss_decompose(htd_graph *g, int32_t h, int32_t *truss_dev, int32_t *stamp_dev,
                               htd_stats *stats, void *stream) {
    return htd_truss_decompose_ex(g, h, 0u, truss_dev, stamp_dev, stats, stream);
}

htd_status htd_truss_decompose_host(int32_t n, const int32_t *src_host, const int32_t *dst_host,
                                    int64_t m_in, int32_t h, int32_t *eu_host, int32_t *ev_host,
                                    int32_t *truss_host, int64_t *m_out, htd_stats *stats,
                                    void *stream) {
    if (!m_out || (m_in > 0 && (!src_host || !dst_host || !eu_host || !ev_host || !truss_host)) ||
        h < 1 || h > HTD_MAX_H) {
        set_last_error("htd_truss_decompose_host: NULL argument or bad h");
        return HTD_EINVAL;
    }
    htd_graph *g = nullptr;
    API_TRY(htd_build_csr(n, src_host, dst_host, m_in, 0, stream, &g));
    Handle *H = &g->H;
    const int64_t m = H->g.m;
    int32_t *truss_dev = nullptr;
    htd_status st = HTD_OK;
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    if (cudaMalloc(&truss_dev, (m > 0 ? m : 1) * 4) != cudaSuccess) {
        set_last_error("htd_truss_decompose_host: output allocation failed");
        htd_graph_free(g);
        return HTD_ENOMEM;
    }
    st = htd_truss_decompose(g, h, truss_dev, nullptr, stats, stream);
    if (st == HTD_OK && m > 0) {
        cudaError_t e = cudaMemcpyAsync(eu_host, H->g.eu, m * 4, cudaMemcpyDeviceToHost, user);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ev_host, H->g.ev, m * 4, cudaMemcpyDeviceToHost, user);
        if (e == cudaSuccess) e = cudaMemcpyAsync(truss_host, truss_dev, m * 4, cudaMemcpyDeviceToHost, user);
        if (e == cudaSuccess) e = cudaStreamSynchronize(user);
        if (e != cudaSuccess) {
            set_last_error(std::string("htd_truss_decompose_host: copy back: ") + cudaGetErrorString(e));
            st = HTD_ECUDA;
        }
    }
    if (st == HTD_OK) *m_out = m;
    cudaFree(truss_dev);
    htd_graph_free(g);
    return st;
}

}  // extern "C"
