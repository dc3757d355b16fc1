// htd_internal.h -- host-side structures shared by the translation units of libhtruss.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "htruss.h"
#include "htd_common.cuh"

namespace htd {

// Normalised graph on one device (Sec. 2 graph model, CSR form).
struct GraphDev {
    int device = 0;
    int32_t n = 0;
    int64_t m = 0;
    int32_t *row_ptr = nullptr;   // n+1
    int32_t *col = nullptr;       // 2m, sorted within each row
    int32_t *slot_eid = nullptr;  // 2m, edge id of each slot
    int32_t *eu = nullptr;        // m, eu < ev
    int32_t *ev = nullptr;        // m
    int32_t *slot_lo = nullptr;   // m, slot of ev[e] in row eu[e]
    int32_t *slot_hi = nullptr;   // m, slot of eu[e] in row ev[e]
};

// Device scratch of one h-support pass / peel, cached on the handle between calls.
struct PeelWork {
    int32_t h = 0;
    int32_t W = 0;                 // 32-bit words of an n-bit set
    int32_t Wpad = 0;              // W rounded up to a multiple of 4
    int64_t pool_words = 0;        // ball storage size (uint32 words)
    int64_t pool_used = 0;         // words the balls of the last initial pass took
    uint32_t *pool = nullptr;      // ball storage
    int64_t *ball_off = nullptr;   // n+1 offsets into pool (multiples of 4 words)
    int32_t *ball_need = nullptr;  // n storage words of the initial balls
    int32_t *ball_size = nullptr;  // n members of each ball (the vertex itself included)
    int32_t *ball_nw = nullptr;    // n: -1 = dense (W words), else (index,bits) pair count
    int2 *ball_meta = nullptr;     // n: (offset / 4, ball_nw) packed for one-load lookups
    int32_t *col_live = nullptr;   // 2m neighbour ids; -(round + 1) once removed in that round
    int32_t *deg_alive = nullptr;  // n alive degrees
    int32_t *sup = nullptr;        // m h-support (INT_MAX once removed)
    int32_t *truss = nullptr;      // m (points at the caller's output during a peel)
    int32_t *stamp = nullptr;      // m
    int32_t *frontier = nullptr;   // m
    int32_t *cand_list = nullptr;  // n
    int32_t *cand_stamp = nullptr; // n round of the last candidate mark
    int32_t *changed_list = nullptr;   // n
    int32_t *changed_stamp = nullptr;  // n round in which the ball last shrank
    int2 *items = nullptr;         // (vertex, first slot) h-support work items
    int64_t items_cap = 0;
    bool incremental = false;      // h <= 2: lost-pair support updates instead of rebuilds
    bool dense_balls = false;      // every ball stored dense (set per call before the initial pass)
    unsigned long long *lost_keys = nullptr;  // hash set of the round's lost pairs
    int64_t lost_cap = 0;          // hash slots (power of two)
    int64_t lost_max = 0;          // lost-pair records one batch may hold (half the slots)
    bool lost_tiny = false;        // table forced to 128 slots (test option)
    int4 *lost = nullptr;          // (min, max, hash slot, 0) per lost pair
    int32_t *edge_touch = nullptr; // n: last round in which the vertex's ball lost a member
    int32_t *hub_slot = nullptr;   // n: row of the vertex's alive-adjacency set, or -1
    int32_t *hub_list = nullptr;   // nhub vertices with such a set (degree >= hub_min_deg)
    uint32_t *hub_bits = nullptr;  // nhub x Wpad words: alive neighbours as n-bit sets
    int32_t nhub = 0;
    int32_t hub_min_deg = 0;
    int4 *pitems = nullptr;        // loss detection items (edge side, first slot, x, y), <= 32 pairs
    int64_t pitems_cap = 0;
    int4 *uitems = nullptr;        // support update items (first slot, v, w, row end), <= 32 slots
    int64_t uitems_cap = 0;
    int64_t upd_budget = 0;        // adjacency slots one batch of updates may visit
    // incremental h = 3: radius-2 balls (dense, x * Wpad) and their own metadata, used by
    // the loss tests and by the rebuild that finishes a round which ran out of room
    bool inc3 = false;
    uint32_t *pool2 = nullptr;
    int32_t *ball_size2 = nullptr;
    int32_t *ball_nw2 = nullptr;
    int2 *ball_meta2 = nullptr;
    int32_t *changed_list2 = nullptr;
    int32_t *changed_stamp2 = nullptr;
    unsigned long long *lost2_keys = nullptr;  // hash set of the round's radius-2 lost pairs
    int64_t lost2_cap = 0;
    int64_t lost2_max = 0;
    int4 *lost2 = nullptr;         // (min, max, hash slot, 0) per radius-2 lost pair
    int32_t *touch2 = nullptr;     // n: round in which the vertex last lost a radius-2 member
    int4 *c3items = nullptr;       // radius-3 candidate items of a round
    int64_t c3items_cap = 0;
    int32_t *bfs_lists = nullptr;  // per-block BFS level lists (h >= 3)
    int64_t bfs_list_len = 0;      // entries per list
    void *scan_tmp = nullptr;
    DevStatus *status = nullptr;
    DevStatus *status_host = nullptr;  // pinned mirror
    int grid_ball = 0;             // persistent grid sizes
    int grid_hsup = 0;
    int grid_edges = 0;
    size_t smem_ball = 0;
    size_t smem_hsup = 0;
};

struct Handle {
    GraphDev g;
    PeelWork w;
    cudaStream_t pstream = nullptr;       // private stream (graph capture needs one)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph_exec = nullptr;       // cached round graph
    cudaGraphExec_t graph_exec_timed = nullptr; // the same with an event at every phase
    std::vector<cudaEvent_t> round_events;      // events of the timed graph
    int graph_h = 0;
    int graph_rounds = 0;
    bool graph_incremental = false;
    bool graph_dense = false;      // ball layout the captured rounds address directly
    int num_sms = 0;
};

void set_last_error(const std::string &msg);
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// The limit is a process-wide property of the function: it is only ever raised (under a
// lock), so that a call for a small graph in one thread cannot lower it below what a
// launch for a large graph in another thread needs.
cudaError_t raise_smem_limit(const void *func, size_t bytes);
// Adds kernels launched outside the handle calls to the thread's launch counter.
void add_launches(int64_t k);

// CSR builder (htd_csr.cu).  src/dst are device pointers.
htd_status build_csr_device(int32_t n, const int32_t *src, const int32_t *dst, int64_t m_in,
                            cudaStream_t s, GraphDev *out, int64_t *launches);
void free_graph_dev(GraphDev *g);

// Ball builder, h-support and peel rounds (htd_peel.cu).
htd_status ensure_work(Handle *H, int32_t h, bool incremental, bool tiny_table = false);
void free_work(PeelWork *w);
htd_status initial_pass(Handle *H, int32_t h, cudaStream_t s, int64_t *launches,
                        htd_stats *timing);
// evs (nullable): kRoundEvents events marking the phase boundaries of the round.
constexpr int kRoundEvents = 7;
htd_status enqueue_round(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t *evs);

// Persistent kernel running up to max_slots incremental round slots (htd_loss.cu).
htd_status launch_persistent_rounds(Handle *H, cudaStream_t s, int max_slots, int64_t *launches);

// Finishes a round of the incremental h = 3 peel that ran out of room (status halt): its
// frontier is already removed; the balls of every vertex within distance 2 of a frontier
// endpoint are rebuilt and the supports of edges at changed balls recomputed (htd_peel.cu).
htd_status recover_round_h3(Handle *H, cudaStream_t s, int64_t *launches);
// Initial radius-2 balls of the incremental h = 3 peel (htd_peel.cu).
htd_status initial_pass_r2(Handle *H, cudaStream_t s, int64_t *launches);

// The normalised graph behind a public handle (htd_api.cu).
GraphDev *graph_dev(htd_graph *g);

// One small graph of a batch for the block-per-graph launch (htd_batch_block.cu): device
// pointers into its union's CSR, its vertices [v0, v0 + L) and edges [e0, e0 + m) there,
// and where its t(e,h) go.
struct BlockGraphDescHost {
    const int32_t *row_ptr, *col, *slot_eid, *eu, *ev;
    int32_t *out;
    int64_t e0, m;
    int32_t v0, L, h;
};
constexpr int32_t kBlockMaxN = 8192;  // largest graph a block peels alone
htd_status batch_block_run(const std::vector<BlockGraphDescHost> &graphs, cudaStream_t s,
                           int num_sms, int64_t *rounds_out);

// The H-index iteration of Sec. 4 on the device (htd_hindex.cu); G is H's public handle.
htd_status hindex_run(htd_graph *G, Handle *H, int32_t h, int32_t sweeps, int32_t max_iter, bool prune,
                      int32_t *truss_dev, int32_t *hval_dev, htd_hindex_stats *stats, cudaStream_t s);

// One incremental round (h <= 3) as four (h = 3: five) launches, the graph path (htd_loss.cu).
htd_status enqueue_incremental_round(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t *evs,
                                     unsigned record_flags);

}  // namespace htd
