/*
 * htruss.h -- C ABI of the GB300 (sm_103a) higher-order (k,h)-truss decomposition library.
 *
 * Method: Chen, Qian, Luo, Li, Wang, "Parallel Higher-order Truss Decomposition" (2024).
 *   - h-hop neighbourhood N_G(v,h): vertices within distance h of v (Sec. 2);
 *   - h-support sup_G(e,h) = |N_G(u,h) ∩ N_G(v,h)| for e = (u,v) (Def. 2, Def. 3);
 *   - (k,h)-truss and h-trussness t(e,h) (Def. 4), computed by peeling (Sec. 3, Lemma 1,
 *     Algorithm 1), here level-synchronously: every edge of the current level is removed
 *     in one round, and h-support is recomputed only for edges whose endpoints' h-hop
 *     balls shrank.
 * Readings fixed by this library where the paper is silent:
 *   - a subgraph is an edge set and distances inside it use only its edges;
 *   - paths through e itself count towards sup(e,h); u and v are not counted;
 *   - self-loops are dropped, duplicate and reverse pairs merged;
 *   - edge id = rank of (u,v), u < v, in lexicographic order; outputs are per edge id;
 *   - t(e,h) >= 2 for every edge (the 2-truss is the whole graph).
 *
 * Conventions for every call:
 *   - Pointers named *_dev are device pointers of the current CUDA device; *_host are host
 *     pointers (pinned memory makes the copies faster but is not required).
 *   - The caller owns every input and output buffer.  The library owns the graph handle
 *     and all scratch memory it allocates (stream-ordered, on the device of the call).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is ordered after
 *     prior work on `stream`; every call below except htd_h_support_static returns only
 *     after its results are complete and visible on `stream` (the calls synchronise
 *     internally).
 *   - On error nothing is written to the outputs; the handle stays valid unless stated.
 *   - Errors: HTD_EINVAL (bad argument: NULL pointer, h outside [1, HTD_MAX_H], n < 0,
 *     vertex id outside [0,n)), HTD_ENOMEM (device allocation failed), HTD_ECUDA (a CUDA
 *     call failed; htd_last_error() has the message), HTD_EOVERFLOW (2*m_in >= 2^31),
 *     HTD_EUNSUPPORTED (n > HTD_MAX_N), HTD_ETIMEOUT (the peel exceeded its round cap).
 *   - Functions are thread-safe for distinct handles; one handle must not be used by two
 *     threads at once.
 */
#ifndef HTRUSS_H
#define HTRUSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HTD_MAX_H 8          /* largest hop threshold h accepted */
#define HTD_MAX_N 1600000    /* largest vertex count: an h-hop ball must fit in shared memory as an n-bit set */

typedef enum htd_status {
    HTD_OK = 0,
    HTD_EINVAL = 1,
    HTD_ENOMEM = 2,
    HTD_ECUDA = 3,
    HTD_ETIMEOUT = 4,
    HTD_EOVERFLOW = 5,
    HTD_EUNSUPPORTED = 6
} htd_status;

/* Opaque handle: the normalised graph in CSR form on one device plus cached scratch. */
typedef struct htd_graph htd_graph;

/* Counters of one decomposition (all zero for calls that do not peel).  Times are device
 * time between CUDA events on the library's stream, filled only with HTD_OPT_TIMING. */
typedef struct htd_stats {
    int64_t rounds;          /* removal rounds (each removes every edge of the current level) */
    int64_t levels;          /* distinct k at which edges were removed */
    int32_t max_truss;       /* largest t(e,h) */
    int32_t h;
    int64_t hsup_evals;      /* h-support evaluations: m (initial) + supports brought up to date
                                in the rounds (edges with an endpoint whose ball shrank) */
    int64_t ball_builds;     /* h-hop balls built: n (initial) + rebuilt candidates */
    int64_t balls_changed;   /* rebuilt balls that had shrunk */
    int64_t frontier_edges;  /* edges removed (= m at the end) */
    int64_t pairs_tested;    /* incremental rounds: vertex pairs tested for loss */
    int64_t pairs_lost;      /* incremental rounds: pairs that left each other's balls */
    int64_t member_tests;    /* incremental rounds: ball-membership tests of support updates */
    int64_t kernel_launches; /* kernels this library launched for the call */
    int64_t ball_pool_bytes; /* device bytes the stored h-hop balls take */
    int64_t timed_slots;     /* round slots whose phases were timed (with HTD_OPT_TIMING the
                                graph path times every 16th batch of 16 slots) */
    double alg_bytes_ball;   /* algorithmic bytes: ball builds (initial and rebuilds) */
    double alg_bytes_hsup;   /* algorithmic bytes: full h-support intersections */
    double alg_bytes_detect; /* algorithmic bytes: loss detection (incremental rounds) */
    double alg_bytes_update; /* algorithmic bytes: support updates (incremental rounds) */
    float ms_initial_ball;   /* initial pass: ball builds (count + store) */
    float ms_initial_hsup;   /* initial pass: every edge's h-support */
    float ms_select;         /* rounds: frontier selection */
    float ms_find;           /* rounds: candidate search (rebuild) or loss detection */
    float ms_remove;         /* rounds: edge removal */
    float ms_ball;           /* rounds: ball rebuilds (rebuild variant) */
    float ms_update;         /* rounds: support recomputation or incremental updates */
    float ms_minreduce;      /* rounds: min alive support + alive count */
    float ms_round_kernel;   /* persistent round kernel: device time of all its launches
                                (always measured; the phase times above then come from the
                                GPU's global timer, as seen by one block) */
    int32_t round_kernel_launches;
    int32_t incremental;     /* 1 if the rounds used incremental support updates */
    int32_t reserved;
    int64_t slots;           /* round slots that ran (rounds plus continued batches) */
    int64_t pairs3_tested;   /* incremental h = 3 rounds: radius-3 candidate pairs tested */
    int64_t pairs2_lost;     /* incremental h = 3 rounds: pairs that left radius-2 balls */
    int64_t rounds_rebuilt;  /* incremental h = 3 rounds that ran out of room and were
                                finished by rebuilding the candidates' balls */
    double alg_bytes_hsup_initial; /* the part of alg_bytes_hsup taken by the initial pass */
} htd_stats;

/* Option flags for htd_truss_decompose_ex. */
#define HTD_OPT_TIMING 1u    /* time the initial ball-build and h-support launches and sample
                                the round phases (CUDA events; the graph path times every
                                16th batch of 16 rounds) into htd_stats */
#define HTD_OPT_NO_GRAPH 2u  /* launch each peel round directly instead of via a CUDA graph */
#define HTD_OPT_REBUILD 4u   /* h <= 3: rebuild shrunk balls and recompute their edges' support
                                instead of the incremental lost-pair updates (same results) */
#define HTD_OPT_PERSISTENT_ROUNDS 16u  /* h <= 2: all rounds in a persistent cooperative
                                          kernel (phases split by grid barriers) instead of
                                          a CUDA graph of 16 rounds (same results) */
#define HTD_OPT_TINY_LOSS_TABLE 8u  /* h <= 3: 128-slot lost-pair tables, so that h <= 2 rounds
                                       run in many batches and h = 3 rounds are finished by
                                       rebuilds (a test of those paths; slow) */
#define HTD_OPT_COMPACT_BALLS 32u   /* h <= 2: store each ball in its smaller form (sorted
                                       non-zero words when at most half the words are
                                       non-zero) even when every ball fits dense; by default
                                       the incremental peel keeps all balls dense (one load
                                       per membership test) when the n x n bits fit in a
                                       quarter of the free device memory (same results).
                                       h = 3: the incremental rounds need dense radius-2 and
                                       radius-3 balls (two n x n bit sets in a third of the
                                       free memory); with this flag, or when they do not
                                       fit, h = 3 peels by rebuilds */

#define HTD_OPT_BATCH_BLOCKS 64u    /* htd_truss_decompose_batched: every graph of at most
                                       8,192 vertices and h <= 3 is peeled by one block of a
                                       single persistent launch, all of its rounds inside the
                                       kernel (radius-1..h balls as bit rows, candidates'
                                       balls recomputed by ORs); larger graphs take the union
                                       path (same results) */

/* Normalise an undirected edge list and build the graph (Sec. 2 graph model).
 *   n            vertex count, ids in [0, n); 0 <= n <= HTD_MAX_N.
 *   src, dst     m_in int32 endpoints each (device pointers if inputs_on_device != 0,
 *                else host pointers); pairs may repeat, appear reversed or be loops.
 *   out          receives the new handle (set to NULL on error).
 * Builds: row offsets (n+1), sorted neighbour lists (2m), slot -> edge id (2m) and the
 * canonical edge list (eu < ev, m edges, lexicographic).  Errors: EINVAL for an id
 * outside [0,n), EOVERFLOW if 2*m_in >= 2^31, EUNSUPPORTED if n > HTD_MAX_N. */
htd_status htd_build_csr(int32_t n, const int32_t *src, const int32_t *dst, int64_t m_in,
                         int inputs_on_device, void *stream, htd_graph **out);

/* Vertex and edge counts of a handle. */
htd_status htd_graph_info(const htd_graph *g, int32_t *n, int64_t *m);

/* Canonical edges: eu_dev[e] < ev_dev[e], e in [0, m), lexicographic order (device
 * buffers of m int32 each). */
htd_status htd_edges(const htd_graph *g, int32_t *eu_dev, int32_t *ev_dev, void *stream);

/* CSR of the normalised graph: row_ptr_dev (n+1), col_dev (2m, neighbours sorted within
 * each row), slot_eid_dev (2m, edge id of each adjacency slot).  Any pointer may be NULL
 * to skip that array. */
htd_status htd_csr(const htd_graph *g, int32_t *row_ptr_dev, int32_t *col_dev,
                   int32_t *slot_eid_dev, void *stream);

/* h-support of every edge (Def. 2, Def. 3; the initial h-support loop of Algorithm 2):
 * sup_dev[e] = |N(u,h) ∩ N(v,h)| in the whole graph, u and v excluded.
 * sup_dev: device buffer of m int32.  1 <= h <= HTD_MAX_H. */
htd_status htd_h_support(htd_graph *g, int32_t h, int32_t *sup_dev, void *stream);

/* (k,h)-truss decomposition (Def. 4; Sec. 3 peeling): truss_dev[e] = t(e,h) for every
 * edge id (device buffer of m int32, values in [2, n]).
 *   stamp_dev  nullable device buffer of m int32: the 0-based round in which e was
 *              removed (rounds are level-synchronous; usable for a peeling certificate).
 *   stats      nullable host struct, filled on success. */
htd_status htd_truss_decompose(htd_graph *g, int32_t h, int32_t *truss_dev,
                               int32_t *stamp_dev, htd_stats *stats, void *stream);

/* Same as htd_truss_decompose with option flags (HTD_OPT_*). */
htd_status htd_truss_decompose_ex(htd_graph *g, int32_t h, uint32_t flags,
                                  int32_t *truss_dev, int32_t *stamp_dev,
                                  htd_stats *stats, void *stream);

/* End-to-end call on host buffers: copies src/dst (m_in each) to the device, builds the
 * graph, decomposes it at hop threshold h and copies the canonical edges and t(e,h) back.
 *   eu_host, ev_host, truss_host  host buffers with room for m_in int32 each; the first
 *                                 *m_out entries are written.
 *   m_out                         receives m, the number of distinct edges. */
htd_status htd_truss_decompose_host(int32_t n, const int32_t *src_host,
                                    const int32_t *dst_host, int64_t m_in, int32_t h,
                                    int32_t *eu_host, int32_t *ev_host, int32_t *truss_host,
                                    int64_t *m_out, htd_stats *stats, void *stream);

/* Many graphs in one call: every graph's (k,h)-truss decomposition (Def. 4; Sec. 3
 * peeling), each with its own hop threshold.  The paper decomposes one graph at a time;
 * the batch relies on the decomposition of a disjoint union being its members'
 * decompositions (h-support counts only vertices of the edge's own component), so the
 * graphs of each h are packed, in input order, into disjoint unions of at most
 * max_union_vertices vertices and each union is peeled once (htd_truss_decompose_ex with
 * `flags`).  The unions are independent and are peeled concurrently by up to 8 worker
 * threads, each on its own stream, as many at once as their footprint estimates fit 70% of
 * the free device memory (a union that still runs out of memory is retried alone).  With
 * HTD_OPT_BATCH_BLOCKS the graphs of at most 8,192 vertices and h <= 3 are instead peeled
 * one block per graph in a single persistent launch.  Results are identical to decomposing
 * each graph alone.
 *   num_graphs        number of graphs (>= 0).
 *   n, h              host arrays of num_graphs: vertex count (0 <= n <= HTD_MAX_N) and hop
 *                     threshold (1 <= h <= HTD_MAX_H) of each graph.
 *   edge_offsets      host array of num_graphs + 1, edge_offsets[0] = 0, non-decreasing:
 *                     graph g's raw pairs are src_dev/dst_dev[edge_offsets[g] ..
 *                     edge_offsets[g+1]), ids local to the graph, in [0, n[g]); pairs may
 *                     repeat, appear reversed or be loops (normalised as htd_build_csr does).
 *   src_dev, dst_dev  device arrays of edge_offsets[num_graphs] int32.
 *   max_union_vertices  vertices per union (<= 0: 262,144); a larger graph is a union alone.
 *   truss_dev         device output with room for edge_offsets[num_graphs] int32.
 *   out_offsets, out_m  host arrays of num_graphs, filled: graph g's t(e,h) for its
 *                     canonical edges (htd_edges order of the graph alone) are
 *                     truss_dev[out_offsets[g] .. out_offsets[g] + out_m[g]).
 *   num_unions        nullable: receives the number of unions peeled (a union without
 *                     any pair needs no peel and is not counted).
 *   stats             nullable: counters summed over the unions (max_truss, h and
 *                     ball_pool_bytes are maxima; incremental = 1 if every union was).
 * Synchronous on return.  Errors: EINVAL for a NULL argument, a bad n, h or offset, or an
 * endpoint outside [0, n[g]) (the message names the graph), EUNSUPPORTED for n > HTD_MAX_N,
 * EOVERFLOW for a graph with 2*m_in >= 2^31; any error of the underlying calls. */
htd_status htd_truss_decompose_batched(int32_t num_graphs, const int32_t *n, const int32_t *h,
                                       const int64_t *edge_offsets, const int32_t *src_dev,
                                       const int32_t *dst_dev, uint32_t flags,
                                       int32_t max_union_vertices, int32_t *truss_dev,
                                       int64_t *out_offsets, int64_t *out_m,
                                       int32_t *num_unions, htd_stats *stats, void *stream);

/* The union packing htd_truss_decompose_batched uses, computed on the host only (no
 * device call): graphs are taken by increasing h and, within one h, in input order; a
 * union is closed when the next graph would take it past max_union_vertices vertices (<=
 * 0: 262,144) or 2^30 - 1 raw pairs; a larger graph forms a union alone.
 *   union_of, vertex_offset  host arrays of num_graphs, filled: the union of graph g
 *                            (numbered in the order they are peeled, unions without any
 *                            pair included) and the shift added to its vertex ids there.
 *   num_unions               nullable: receives the number of unions.
 * Same argument checks and errors as htd_truss_decompose_batched (no device buffers). */
htd_status htd_batch_plan(int32_t num_graphs, const int32_t *n, const int32_t *h,
                          const int64_t *edge_offsets, int32_t max_union_vertices,
                          int32_t *union_of, int32_t *vertex_offset, int32_t *num_unions);

/* h-support of every edge without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory themselves
 * (code running inside an allocator or memory-pool callback, or under an external budget
 * that already owns all device memory).  The caller passes the normalised graph (the
 * arrays htd_csr and htd_edges return) and the output; the kernel's scratch is one
 * static device array of 32 MiB that every GPU loading this library keeps until the
 * process exits.
 *   n                        vertex count, n <= HTD_STATIC_MAX_N (two n-bit sets of a
 *                            block must fit in shared memory).
 *   row_ptr_dev, col_dev     CSR: n+1 offsets, 2m neighbours sorted within each row.
 *   eu_dev, ev_dev           the m canonical edges.
 *   sup_dev                  output, m int32: sup(e,h) as htd_h_support computes it.
 * Unlike the other calls this one only enqueues work on `stream` (NULL = legacy default
 * stream) and returns; the result is ready when the stream reaches that point.  The first
 * call on a device looks up the scratch array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is kept for the life of
 * the process: after cudaDeviceReset (which invalidates every device address) do not call
 * this entry point again in the same process.  Every call shares the one scratch
 * array and reuses what the previous call left there: calls that overlap on the GPU (two
 * streams, or two threads) race and must be serialised by the caller.  Errors: EINVAL for
 * a NULL pointer or h outside [1, HTD_MAX_H], EUNSUPPORTED for n > HTD_STATIC_MAX_N or, at
 * h >= 3, when one block's level lists (2n int32) exceed the scratch, or when the
 * device's per-block shared memory cannot hold two n-bit sets; ECUDA otherwise. */
#define HTD_STATIC_MAX_N 786432
htd_status htd_h_support_static(int32_t n, const int32_t *row_ptr_dev, const int32_t *col_dev,
                                int64_t m, const int32_t *eu_dev, const int32_t *ev_dev,
                                int32_t h, int32_t *sup_dev, void *stream);

/* ---- The paper's own parallel method: the higher-order H-index iteration (Sec. 4) -----
 *
 * H^(0)(e) = sup(e,h); order n sets, for every edge e = (u,v),
 *   H^(n)(e) = H({ min(P(u,w), P(v,w)) : w in N(u,h) ∩ N(v,h) }),
 * H(S) the largest y with at least y members of S >= y, and P(a,b) the h-hop reachable path
 * key: the largest, over paths from a to b of at most h edges, of the smallest H^(n-1) on
 * the path (Definition of the h-hop reachable path key; Algorithm 2).  Keys never increase
 * (Theorem 3) and stop at t(e,h) - 2 (Theorem 4).  Paths may use e itself; the common
 * h-neighbourhood is that of the whole graph. */
typedef struct htd_hindex_stats {
    int64_t ball_entries;    /* sum of the closed h-hop ball sizes (stored member lists) */
    int64_t kernel_launches;
    int32_t h;
    int32_t sweeps;          /* sub-sweeps per order (1 = synchronous) */
    int32_t iterations;      /* orders computed (the last one changed nothing if converged) */
    int32_t converged;
    float ms_total;          /* device time of the call (CUDA events) */
    int32_t pruned;          /* 1 if the orders used the Lemma 4 pruning */
    int64_t edge_evals;      /* H^(n)(e) computed, summed over the orders */
    int64_t vertex_evals;    /* vertices whose path keys were computed, summed over the orders */
} htd_hindex_stats;

/* Runs the H-index iteration from H^(0) = sup(e,h) until an order changes nothing (or for
 * max_iter orders, max_iter >= 0).  sweeps = 1: synchronous orders, each computed from the
 * previous order only (Algorithm 2).  sweeps = S > 1: asynchronous updating by blocks of
 * edges: each order is S sub-sweeps over consecutive edge-id ranges, each using the keys
 * already updated by the sub-sweeps before it.  Outputs (device, m int32 each, nullable):
 * truss_dev = H + 2 (the h-trussness once converged), hval_dev = the last H.  stats
 * (nullable host struct).  Synchronous on return.  Errors: EINVAL (NULL handle, h or sweeps
 * out of range), ENOMEM, EUNSUPPORTED (an n-bit set does not fit in shared memory). */
htd_status htd_hindex_decompose(htd_graph *g, int32_t h, int32_t sweeps, int32_t max_iter,
                                int32_t *truss_dev, int32_t *hval_dev, htd_hindex_stats *stats,
                                void *stream);

/* Options of htd_hindex_decompose_ex. */
#define HTD_HX_PRUNE 1u  /* redundant-computation pruning (Sec. 4, Lemma 4), synchronous orders
                            only: from the second order on, an edge keeps H^(n-1) without being
                            computed when no edge within h-1 hops of its endpoints fell across
                            its value in the previous order.  Same values after every order. */

/* htd_hindex_decompose with option flags (HTD_HX_*).  EINVAL also for unknown flags and for
 * HTD_HX_PRUNE with sweeps != 1. */
htd_status htd_hindex_decompose_ex(htd_graph *g, int32_t h, int32_t sweeps, int32_t max_iter,
                                   uint32_t flags, int32_t *truss_dev, int32_t *hval_dev,
                                   htd_hindex_stats *stats, void *stream);

/* ---- Served decomposition: a request loop with continuous batching -------------------
 *
 * The paper decomposes one graph per call; a server decomposes a stream of independent
 * requests, each an ordinary decomposition of its own graph (Def. 4; Sec. 3 peeling), so a
 * result does not depend on the other requests.  Requests are admitted in arrival order
 * while an estimate of their device footprint (htd_footprint_estimate) fits the server's
 * memory budget beside the requests already admitted; a pool of worker threads, each with
 * its own stream, runs the admitted requests concurrently (their rounds overlap on the
 * device), keeps each request's graph and peel state on the device until its result is
 * copied back, and releases its share of the budget when it finishes, admitting the next
 * requests.  A request larger than the whole budget is admitted alone.  A request that runs
 * out of device memory beside others is put back at the head of the queue and retried
 * after they finish.  All calls are thread-safe. */
typedef struct htd_server htd_server;

/* Timing and outcome of one request (seconds since the server was created). */
typedef struct htd_request_info {
    int64_t m;               /* distinct edges of the request's graph */
    int64_t est_bytes;       /* footprint estimate used for admission */
    int64_t rounds;          /* peel rounds */
    double submit_s;         /* htd_server_submit returned */
    double admit_s;          /* admitted (fits the budget) */
    double start_s;          /* a worker started it */
    double done_s;           /* result on the host */
    int32_t h;
    int32_t status;          /* htd_status of the decomposition */
    int32_t worker;          /* worker thread that ran it */
    int32_t retries;         /* times it was put back after running out of memory */
} htd_request_info;

/* Server state for monitoring. */
typedef struct htd_server_stats {
    int64_t budget_bytes;
    int64_t reserved_bytes;       /* estimates of the admitted and running requests */
    int64_t peak_reserved_bytes;
    int32_t workers;
    int32_t running;              /* requests a worker is running now */
    int32_t peak_running;         /* most requests run at the same time */
    int32_t pending;              /* arrived, waiting for room in the budget */
    int32_t admitted;             /* admitted, waiting for a worker */
    int32_t pad;
} htd_server_stats;

/* Upper estimate of the device bytes one decomposition of a graph with n vertices and m_in
 * raw pairs at hop threshold h takes (graph, peel state, balls; dense balls when they fit a
 * quarter of free_bytes, as the decomposition itself chooses).  Host only.  Returns -1 for
 * a negative n or m_in. */
int64_t htd_footprint_estimate(int32_t n, int64_t m_in, int32_t h, int64_t free_bytes);

/* Starts a server on the current device with `workers` threads (1..64).  budget_bytes: the
 * device memory the admitted requests may take together (0: 80% of the memory free now).
 * flags: HTD_OPT_* passed to every decomposition.  Errors: EINVAL, ECUDA. */
htd_status htd_server_create(int32_t workers, int64_t budget_bytes, uint32_t flags,
                             htd_server **out);

/* Queues a decomposition of the graph given by m_in raw pairs (host arrays, copied before
 * the call returns; normalised as htd_build_csr does) at hop threshold h.  *id_out receives
 * the request id.  Errors: EINVAL (bad n, h, NULL pointer), EOVERFLOW (2*m_in >= 2^31);
 * errors of the decomposition itself (a vertex id outside [0,n), ...) are returned by
 * htd_server_wait. */
htd_status htd_server_submit(htd_server *s, int32_t n, const int32_t *src_host,
                             const int32_t *dst_host, int64_t m_in, int32_t h, int64_t *id_out);

/* *done = 1 once the request's result is ready.  EINVAL for an unknown or collected id. */
htd_status htd_server_poll(htd_server *s, int64_t id, int32_t *done);

/* Waits for the request and collects it: canonical edges and t(e,h) into host buffers of
 * `capacity` entries each (eu_host[e] < ev_host[e], lexicographic, as htd_edges), and its
 * info (nullable).  Returns the decomposition's status; EINVAL (the request stays
 * collectable, info->m set) if capacity < m.  A collected id is forgotten. */
htd_status htd_server_wait(htd_server *s, int64_t id, int32_t *eu_host, int32_t *ev_host,
                           int32_t *truss_host, int64_t capacity, htd_request_info *info);

/* Budget, reservations and queue lengths now. */
htd_status htd_server_info(htd_server *s, htd_server_stats *out);

/* Lets the admitted requests finish, drops the ones still waiting for admission, stops the
 * workers and frees the server (uncollected results are lost).  NULL is ignored. */
void htd_server_destroy(htd_server *s);

/* Frees the handle and every device buffer it owns (NULL is ignored). */
void htd_graph_free(htd_graph *g);

/* Kernels this library has launched from the calling thread since it was loaded (a
 * diagnostic counter; graph launches count every kernel node they contain). */
int64_t htd_kernel_launch_count(void);

/* Static description of a status code. */
const char *htd_status_string(htd_status s);

/* Message of the last failing call on this thread ("" if none). */
const char *htd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HTRUSS_H */
