// htd_common.cuh -- device-side helpers and the per-decomposition status block shared by
// the CSR builder, the ball / h-support kernels and the peel-round kernels.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda_runtime.h>

namespace htd {

constexpr int kMaxH = 8;
constexpr int kWarp = 32;

// Device-resident state of one peel.  Written only by kernels (and zero-initialised by
// the host before the first pass); read by the host between CUDA-graph launches.
struct DevStatus {
    int32_t k;                 // current peeling level (Algorithm 1's k)
    int32_t round;             // removal rounds completed
    int64_t alive;             // edges not yet removed
    int32_t nF;                // frontier size of the current round
    int32_t cand_cnt[kMaxH];   // candidate vertices found at BFS depth 0..h-1
    int32_t nchanged;          // vertices whose ball shrank this round
    int32_t nitems;            // h-support work items this round
    int32_t q_ball;            // work-queue heads (reset at the end of every round)
    int32_t q_items;
    int32_t q_count;           // initial-pass queue heads (used once)
    int32_t q_store;
    uint32_t done_blocks;      // last-block detection of the min reduction
    int32_t min_acc;           // min-reduction accumulator (INT_MAX when idle)
    int64_t alive_acc;         // alive-count accumulator
    int32_t err;               // nonzero: a kernel detected an inconsistency
    int32_t levels;            // distinct k with removals
    int32_t last_k;            // k of the latest removal round
    int32_t max_k;
    int64_t st_frontier;       // edges removed so far
    int64_t st_candidates;     // candidate balls rebuilt
    int64_t st_changed;        // rebuilt balls that shrank
    int64_t st_recomputed;     // h-support recomputations (after the initial pass)
    unsigned long long st_bytes_ball;  // algorithmic bytes, ball builds
    unsigned long long st_bytes_hsup;  // algorithmic bytes, intersections
    unsigned long long st_bytes_hsup_init;  // the initial pass's share of st_bytes_hsup
    // incremental (h <= 2) rounds
    int32_t nlost;             // lost-pair records of the current batch (duplicates nulled)
    int32_t cont;              // 1: the current round continues (its frontier is removed)
    int32_t unit_begin;        // first frontier edge side the next loss detection tests
    int32_t overflow_unit;     // smallest edge side whose lost pairs did not fit (INT_MAX)
    int32_t npitems;           // loss detection items of the current batch
    int32_t nuitems;           // support update items of the current batch
    int32_t pad1;
    long long upd_work;        // adjacency slots reserved for the batch's updates
    unsigned bar_count;        // grid barrier of the persistent round kernel: groups arrived
    unsigned bar_gen;          // generation, advanced by the last arrival
    unsigned bar_group[64];    // blocks arrived, per group of 32 blocks
    long long st_slots;        // round slots run by the persistent kernel
    unsigned long long st_phase_ns[8];  // persistent kernel: time per phase (block 0's view)
    int64_t st_ball_total;     // sum of the initial ball sizes
    int64_t st_pairs;          // candidate pairs tested
    int64_t st_lost;           // lost pairs
    int64_t st_tests;          // ball-membership tests of the support updates
    unsigned long long st_bytes_detect;  // algorithmic bytes, loss detection
    unsigned long long st_bytes_update;  // algorithmic bytes, incremental support updates
    // incremental h = 3 rounds (radius-2 balls kept beside the radius-3 support balls)
    int32_t nlost2;            // radius-2 lost-pair records of the current round
    int32_t halt;              // 1: a round ran out of room; the host finishes it by rebuilds
    long long nc3items;        // stored radius-3 candidate items of the current round (64-bit: the
                               // reservations of a huge round may pass 2^31 before it halts)
    int64_t st_c3_pairs;       // radius-3 candidate pairs tested
    int64_t st_lost2;          // radius-2 lost pairs
    int64_t st_recovered;      // rounds finished by the rebuild recovery
};


enum : int32_t {
    kErrBallGrew = 1,        // a rebuilt ball was larger than before (cannot happen)
    kErrBallCapacity = 2,    // a ball did not fit its storage (cannot happen)
    kErrListOverflow = 4,    // a per-block BFS list overflowed (cannot happen)
    kErrBarrierTimeout = 16, // a grid barrier gave up waiting
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Exclusive prefix sum over the block; *total receives the block sum.  `scratch` needs
// BLOCK/32 ints of shared memory.  Every thread of the block must call it.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total, T *scratch) {
    static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "block size");
    constexpr int NW = BLOCK / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = (lane < NW) ? scratch[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) scratch[lane] = s;
    }
    __syncthreads();
    T before = (wid > 0) ? scratch[wid - 1] : T(0);
    *total = scratch[NW - 1];
    __syncthreads();
    return before + x - v;
}

template <int BLOCK, typename T>
__device__ __forceinline__ T block_sum(T v, T *scratch) {
    T total;
    (void)block_exclusive_scan<BLOCK, T>(v, &total, scratch);
    return total;
}

// Appends `item` to list[] through one atomic per warp (all active lanes with
// pred == true append).  Returns nothing; order within the list is unspecified.
__device__ __forceinline__ void warp_append(bool pred, int32_t item, int32_t *counter,
                                            int32_t *list) {
    const unsigned active = __activemask();
    const unsigned ballot = __ballot_sync(active, pred);
    if (ballot == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(ballot));
    base = __shfl_sync(active, base, leader);
    if (pred) list[base + __popc(ballot & lanemask_lt())] = item;
}

}  // namespace htd
