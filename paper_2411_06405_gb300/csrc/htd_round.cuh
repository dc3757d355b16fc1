// htd_round.cuh -- device pieces of a peel round shared by the per-phase kernels (one
// launch per phase inside a CUDA graph) and the persistent round kernel (all phases of
// many rounds in one cooperative launch, separated by grid barriers).
#pragma once

#include "htd_common.cuh"

namespace htd {

// Spins of a grid barrier before it gives up (after the first few thousand, each spin sleeps
// about 0.1 us): about 2 s, far longer than any phase; on expiry the barrier sets an error
// and the kernel returns.
constexpr unsigned kBarrierSpinLimit = 1u << 24;

// Removes edge e at level k in round `round` (the removal step of Algorithm 1): t(e) = k, its
// stamp, a support no selection matches, both adjacency slots marked dead with the round
// (-(round + 1), so a slot tells by itself whether it died in the current round), alive
// degrees and (when present) the endpoints' alive-adjacency sets updated.
__device__ __forceinline__ void remove_edge(int e, int k, int round, const int32_t *eu,
                                            const int32_t *ev, const int32_t *slot_lo,
                                            const int32_t *slot_hi, int32_t *sup, int32_t *truss,
                                            int32_t *stamp, int32_t *col_live, int32_t *deg_alive,
                                            const int32_t *hub_slot, uint32_t *hub_bits, int Wpad) {
    const int u = eu[e], v = ev[e];
    truss[e] = k;
    stamp[e] = round;
    sup[e] = INT_MAX;
    col_live[slot_lo[e]] = -(round + 1);
    col_live[slot_hi[e]] = -(round + 1);
    atomicSub(&deg_alive[u], 1);
    atomicSub(&deg_alive[v], 1);
    if (hub_slot) {
        const int hu = hub_slot[u], hv = hub_slot[v];
        if (hu >= 0) atomicAnd(hub_bits + (int64_t)hu * Wpad + (v >> 5), ~(1u << (v & 31)));
        if (hv >= 0) atomicAnd(hub_bits + (int64_t)hv * Wpad + (u >> 5), ~(1u << (u & 31)));
    }
}

// Closes a round (called by one thread once every block has added its minimum and alive
// count): round and level bookkeeping, the next level k = max(k, min + 2) (Algorithm 1's
// bins skip empty levels), continuation of an incremental round that ran out of room, and
// the reset of the per-round counters.
__device__ __forceinline__ void round_finalize(DevStatus *st, int initial) {
    __threadfence();
    const int mn = atomicAdd(&st->min_acc, 0);
    const long long al = (long long)atomicAdd((unsigned long long *)&st->alive_acc, 0ull);
    const int nF = st->nF;
    const bool unfinished = !initial && st->overflow_unit != INT_MAX && al > 0;
    st->cont = unfinished ? 1 : 0;
    st->unit_begin = unfinished ? st->overflow_unit : 0;
    st->overflow_unit = INT_MAX;
    if (!initial && nF > 0 && !unfinished) {
        if (st->k != st->last_k) {
            st->levels++;
            st->last_k = st->k;
        }
        st->max_k = max(st->max_k, st->k);
        st->round++;
        st->st_frontier += nF;
        int cands = 0;
        for (int j = 0; j < kMaxH; j++) cands += st->cand_cnt[j];
        st->st_candidates += cands;
        st->st_changed += st->nchanged;
    }
    if (!initial) st->st_slots++;
    st->alive = al;
    if (al > 0 && !unfinished) st->k = max(st->k, mn + 2);
    st->min_acc = INT_MAX;
    st->alive_acc = 0;
    st->done_blocks = 0u;
    if (!unfinished) st->nF = 0;
    for (int j = 0; j < kMaxH; j++) st->cand_cnt[j] = 0;
    st->nchanged = 0;
    st->nlost = 0;
    st->nlost2 = 0;
    st->nc3items = 0;
    st->npitems = 0;
    st->nuitems = 0;
    st->upd_work = 0;
    st->nitems = 0;
    st->q_ball = 0;
    st->q_items = 0;
    __threadfence();
}

// Minimum alive support and alive count over all edges; the last block to finish closes the
// round.  Every thread of every block calls it; `NW` = warps per block.
template <int NW>
__device__ __forceinline__ void minreduce_body(const int32_t *__restrict__ sup, int64_t m,
                                               DevStatus *st, int initial) {
    __shared__ int32_t s_min[NW];
    __shared__ long long s_cnt[NW];
    __shared__ bool s_last;
    int lmin = INT_MAX;
    long long lc = 0;
    // four coalesced loads per thread per step, issued before any of them is used
    const int64_t stride = 4 * (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = 4 * (blockIdx.x * (int64_t)blockDim.x) + threadIdx.x; e0 < m; e0 += stride) {
        int sv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t e = e0 + (int64_t)j * blockDim.x;
            sv[j] = (e < m) ? sup[e] : INT_MAX;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (sv[j] != INT_MAX) {
                lmin = min(lmin, sv[j]);
                lc++;
            }
        }
    }
    lmin = warp_min(lmin);
    lc = warp_sum_ll(lc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_min[wid] = lmin;
        s_cnt[wid] = lc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int bm = INT_MAX;
        long long bc = 0;
        for (int j = 0; j < NW; j++) {
            bm = min(bm, s_min[j]);
            bc += s_cnt[j];
        }
        if (bm != INT_MAX) atomicMin(&st->min_acc, bm);
        if (bc) atomicAdd((unsigned long long *)&st->alive_acc, (unsigned long long)bc);
        __threadfence();
        const unsigned ticket = atomicAdd(&st->done_blocks, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) round_finalize(st, initial);
    __syncthreads();
}

// Barrier across all blocks of a cooperative launch (all co-resident, at most 64 x 32
// blocks).  Arrivals are counted in two levels so that no counter takes more than 32
// atomics per barrier: blocks count in their group of 32, the last block of a group counts
// the group, and the last group advances the generation.  The others wait for the
// generation to move, at most kBarrierSpinLimit spins; a wait that gives up sets an error
// and returns false.  Memory written by any block before the barrier is visible to every
// thread after it: each block fences before it arrives (release), its first thread fences
// again once the generation has moved (acquire, which also drops stale lines from the SM's
// L1), and the block-wide barrier then orders the block's other threads after that fence.
__device__ __forceinline__ bool grid_barrier(DevStatus *st) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen_p = &st->bar_gen;
        const unsigned gen = *gen_p;
        __threadfence();
        const unsigned g = blockIdx.x >> 5, ngroups = (gridDim.x + 31) >> 5;
        const unsigned gsize = min(32u, gridDim.x - (g << 5));
        bool release = false;
        if (atomicAdd(&st->bar_group[g], 1u) == gsize - 1) {
            atomicExch(&st->bar_group[g], 0u);  // every block of the group is waiting now
            if (atomicAdd(&st->bar_count, 1u) == ngroups - 1) {
                atomicExch(&st->bar_count, 0u);
                release = true;
            }
        }
        int ok = 1;
        if (release) {
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            ok = 0;
            for (unsigned it = 0; it < kBarrierSpinLimit; it++) {
                if (*gen_p != gen) {
                    ok = 1;
                    break;
                }
                if (it >= 4096) __nanosleep(100);  // a long wait stops hammering the line
            }
            if (!ok) atomicOr(&st->err, kErrBarrierTimeout);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace htd
