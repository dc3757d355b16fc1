// htd_loss.cu -- exact incremental h-support updates for h <= 2.
//
// For h <= 2 the members a removal can take out of a ball are few and can be listed: an
// old path of length <= h that used a removed edge (a,b) is a-b itself, x-a-b with x in
// N(a), or a-b-w with w in N(b).  So after removing the frontier F of a round the only
// vertex pairs that can stop being within distance h of each other are
//     {a,b}, {a,z} for z in N_old(b) \ {a}, and {b,z} for z in N_old(a) \ {b}
// for every (a,b) in F (for h = 1 only {a,b}).  Each such pair is tested in the new graph
// (adjacent, or for h = 2 a common alive neighbour); a pair that fails is "lost": each
// endpoint leaves the other's ball (distance is symmetric).  Lost pairs are deduplicated
// in an open-addressing hash set.
//
// The h-support of an alive edge (x,y), x < y, then drops by exactly
//     |L(x) ∩ B_old(y)| + |L(y) ∩ B_new(x)|,
// where L(v) = B_old(v) \ B_new(v) (Def. 3: sup = |B(x) ∩ B(y)| - 2, and a member that
// leaves B(x) ∩ B(y) either leaves B(x), or stays in B(x) and leaves B(y)).  The first
// term is counted against the stored balls before the lost members are cleared, the
// second after.  Every step is exact integer arithmetic; no ball is rebuilt.
//
// A round whose lost pairs outgrow the table is processed in batches: the deltas of
// successive batches telescope (each is taken between the stored balls before and after
// that batch), and a pair whose stored bit is already clear was handled by an earlier
// batch of the same round, so it is skipped.  Detection records the first frontier edge
// side it could not finish; the next round slot resumes there without selecting anew.
#include <cstdint>

#include "htd_internal.h"
#include "htd_round.cuh"

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr unsigned long long kEmpty = ~0ull;

struct LossArgs {
    int64_t m;
    const int32_t *slot_lo;
    const int32_t *slot_hi;
    int32_t *truss;
    int32_t *stamp_w;
    int32_t *frontier_w;
    int32_t *col_live_w;
    int32_t *deg_alive_w;
    uint32_t *hub_bits_w;
    int32_t h;
    int32_t lost_max;
    unsigned long long cap_mask;
    const int32_t *row_ptr;
    const int32_t *col;
    const int32_t *col_live;
    const int32_t *slot_eid;
    const int32_t *eu;
    const int32_t *ev;
    const int32_t *frontier;
    const int32_t *stamp;
    uint32_t *pool;
    const int64_t *ball_off;
    const int32_t *ball_nw;
    const int2 *ball_meta;
    int32_t *ball_size;
    unsigned long long *keys;
    int4 *lost;
    int32_t *sup;
    int32_t *vtouch;
    const int32_t *deg_alive;
    const int32_t *hub_slot;
    const uint32_t *hub_bits;
    int32_t Wpad;
    int32_t pitems_cap;
    int2 *pitems;
    int32_t uitems_cap;
    int2 *uitems;
    long long upd_budget;
    DevStatus *st;
};

__device__ __forceinline__ unsigned long long pair_key(int p, int q) {
    const unsigned a = (unsigned)min(p, q), b = (unsigned)max(p, q);
    return ((unsigned long long)a << 32) | b;
}

// 64-bit finaliser of MurmurHash3 (public domain), used to spread pair keys.
__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Status fields are written by other blocks between the phases of the persistent kernel:
// read them through the memory system, never from a register copy.
template <typename T>
__device__ __forceinline__ T vload(const T &x) {
    return *(const volatile T *)&x;
}

// Alive-adjacency set of p if p has one (high degree), else null.
__device__ __forceinline__ const uint32_t *hub_set(const LossArgs &a, int p, unsigned &reads) {
    reads++;
    const int hs = a.hub_slot[p];
    return hs >= 0 ? a.hub_bits + (int64_t)hs * a.Wpad : nullptr;
}

// Is q an alive neighbour of p?  One bit of p's alive-adjacency set when p has one, else a
// binary search in p's sorted row and the alive mark.  `reads` counts the 4-byte words
// touched (algorithmic bytes = 4 x reads).
__device__ __forceinline__ bool alive_adjacent_set(const LossArgs &a, const uint32_t *pset, int p,
                                                   int q, unsigned &reads) {
    if (pset) {
        reads++;
        return (pset[q >> 5] >> (q & 31)) & 1u;
    }
    int lo = a.row_ptr[p], hi = a.row_ptr[p + 1] - 1;
    reads += 2;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = __ldg(a.col + mid);
        reads++;
        if (v == q) {
            reads++;
            return a.col_live[mid] >= 0;
        }
        if (v < q) lo = mid + 1;
        else hi = mid - 1;
    }
    return false;
}

__device__ __forceinline__ bool alive_adjacent(const LossArgs &a, int p, int q, unsigned &reads) {
    return alive_adjacent_set(a, hub_set(a, p, reads), p, q, reads);
}

// Short rows are scanned by one lane; pairs whose shorter row is longer go to the warp.
constexpr int kInlineScan = 4;

enum PairState { kKept = 0, kLost = 1, kHard = 2 };

// First test of the pair {p,q} (p != q) in the alive graph, by one lane: adjacency by
// binary search in the shorter row, then (h = 2) a common alive neighbour when the shorter
// row is at most kInlineScan long.  Longer scans are left to the warp (kHard).
__device__ __forceinline__ int pair_quick(const LossArgs &a, int &p, int &q, unsigned &reads) {
    const int dp = a.row_ptr[p + 1] - a.row_ptr[p];
    const int dq = a.row_ptr[q + 1] - a.row_ptr[q];
    reads += 4;
    if (dp > dq) {  // p: the shorter row
        const int t = p;
        p = q;
        q = t;
    }
    const uint32_t *qset = hub_set(a, q, reads);
    if (alive_adjacent_set(a, qset, q, p, reads)) return kKept;
    if (a.h < 2) return kLost;
    // with q's set every scanned neighbour costs one read; without it, a binary search
    if (min(dp, dq) > (qset ? 8 * kInlineScan : kInlineScan)) return kHard;
    const int re = a.row_ptr[p + 1];
    for (int s = a.row_ptr[p]; s < re; s++) {
        const int y = a.col_live[s];
        reads++;
        if (y >= 0 && alive_adjacent_set(a, qset, q, y, reads)) return kKept;
    }
    return kLost;
}

// Common alive neighbour of p (shorter row) and q, searched by the whole warp: lanes take
// p's slots 32 at a time and binary-search them in q's row; stops at the first hit.
__device__ __forceinline__ bool warp_common_neighbour(const LossArgs &a, int p, int q,
                                                      unsigned &reads) {
    const int lane = threadIdx.x & 31;
    const int rb = a.row_ptr[p], re = a.row_ptr[p + 1];
    const uint32_t *qset = hub_set(a, q, reads);
    for (int s0 = rb; s0 < re; s0 += 32) {
        const int s = s0 + lane;
        bool hit = false;
        if (s < re) {
            const int y = a.col_live[s];
            reads++;
            hit = (y >= 0) && alive_adjacent_set(a, qset, q, y, reads);
        }
        if (__any_sync(0xffffffffu, hit)) return true;
    }
    return false;
}

// Is w in the stored ball of z (dense words, or sorted (word index, word) pairs)?
// `bytes` counts the algorithmic bytes: 8 of metadata plus the words probed.
__device__ __forceinline__ bool ball_contains_meta(const LossArgs &a, int2 meta, int w,
                                                   unsigned &bytes) {
    const int nw = meta.y;
    const int64_t off = (int64_t)(unsigned)meta.x << 2;
    const uint32_t bit = 1u << (w & 31);
    const uint32_t wi = (uint32_t)(w >> 5);
    if (nw < 0) {
        bytes += 4;
        return (a.pool[off + wi] & bit) != 0u;
    }
    const uint2 *p = reinterpret_cast<const uint2 *>(a.pool + off);
    int lo = 0, hi = nw - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const uint2 v = p[mid];
        bytes += 8;
        if (v.x == wi) return (v.y & bit) != 0u;
        if (v.x < wi) lo = mid + 1;
        else hi = mid - 1;
    }
    return false;
}

__device__ __forceinline__ bool ball_contains(const LossArgs &a, int z, int w, unsigned &bytes) {
    bytes += 8;
    return ball_contains_meta(a, a.ball_meta[z], w, bytes);
}

// Records the lost pair {x,z} unless an earlier batch of this round handled it.  The
// record and the pair's update work (both rows are visited by the support updates) are
// reserved against the batch limits; a pair that does not fit marks its edge side u as
// the point where the next slot of this round resumes.
__device__ __forceinline__ void record_lost(const LossArgs &a, DevStatus *st, int x, int z, int u,
                                            unsigned &reads) {
    if (!ball_contains(a, x, z, reads)) return;  // stored bit already clear
    const long long work = (long long)(a.row_ptr[x + 1] - a.row_ptr[x]) +
                           (a.row_ptr[z + 1] - a.row_ptr[z]);
    const long long before =
        (long long)atomicAdd((unsigned long long *)&st->upd_work, (unsigned long long)work);
    const int idx = atomicAdd(&st->nlost, 1);
    if (idx >= a.lost_max || before + work > a.upd_budget) {
        atomicMin(&st->overflow_unit, u);
        if (idx < a.lost_max) a.lost[idx] = make_int4(-1, -1, -1, 0);
        return;
    }
    const unsigned long long key = pair_key(x, z);
    unsigned long long slot = mix64(key) & a.cap_mask;
    int4 rec = make_int4(-1, -1, -1, 0);  // null record: the pair is already held
    for (unsigned long long probe = 0; probe <= a.cap_mask; probe++) {
        const unsigned long long prev = atomicCAS(a.keys + slot, kEmpty, key);
        if (prev == kEmpty) {
            rec = make_int4(min(x, z), max(x, z), (int)slot, 0);
            break;
        }
        if (prev == key) break;
        slot = (slot + 1) & a.cap_mask;
    }
    a.lost[idx] = rec;
}

// Pair enumeration of edge side u = (edge F[u/2], side u%2): side 0 of (a,b) pairs a with
// {b} and with N_old(b) \ {a} (slots start-1 .. re-1 of b's row, start-1 standing for b);
// side 1 pairs b with N_old(a) \ {b}.  For h = 1 only {a,b}.
struct UnitInfo {
    int x, y, rb, start, stop;
};

__device__ __forceinline__ UnitInfo unit_info(const LossArgs &a, int u) {
    UnitInfo r;
    const int e = a.frontier[u >> 1];
    const int side = u & 1;
    r.x = side ? a.ev[e] : a.eu[e];
    r.y = side ? a.eu[e] : a.ev[e];
    r.rb = a.row_ptr[r.y];
    r.start = (side == 0) ? r.rb - 1 : r.rb;
    r.stop = (a.h < 2) ? ((side == 0) ? r.rb : r.rb) : a.row_ptr[r.y + 1];
    return r;
}

// Splits the frontier's edge sides into detection items of at most 32 pairs (one warp
// each), so a hub row is spread over many warps.  Sides that do not fit the item list are
// left to the next slot of the round (resume point).
__device__ void ph_pair_items(const LossArgs &a) {
    DevStatus *st = a.st;
    const int units = 2 * vload(st->nF), u0 = vload(st->unit_begin);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int b = u0 + blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < units; b += stride) {
        const int u = b + lane;
        int nch = 0, start = 0;
        if (u < units) {
            const UnitInfo r = unit_info(a, u);
            start = r.start;
            nch = (r.stop - r.start + 31) >> 5;
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && tot) base = atomicAdd(&st->npitems, tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        const int first = base + incl - nch;
        const bool fits = first + nch <= a.pitems_cap;
        if (!fits && nch) atomicMin(&st->overflow_unit, u);
        for (int c = 0; c < nch && first + c < a.pitems_cap; c++)
            a.pitems[first + c] = fits ? make_int2(u, start + 32 * c) : make_int2(-1, 0);
    }
}

// Loss detection, one warp per item: lane i tests the pair of slot item.y + i.  A pair is
// kept if its endpoints are adjacent or (h = 2) share an alive neighbour; lanes whose test
// needs a long row scan hand it to the whole warp, one pair after the other.
__device__ void ph_detect(const LossArgs &a) {
    __shared__ unsigned long long s_pairs, s_reads;
    DevStatus *st = a.st;
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_reads = 0ull;
    }
    __syncthreads();
    const int nitems = min(vload(st->npitems), a.pitems_cap), round = vload(st->round);
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned long long pairs = 0ull, reads_total = 0ull;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems; it += nwarps) {
        const int2 item = a.pitems[it];
        const int u = item.x;
        // sides past an overflow are redone by the next slot of the round: skip them now
        if (u < 0 || u > *(volatile int *)&st->overflow_unit) continue;
        const UnitInfo r = unit_info(a, u);
        const int sl = item.y + lane;
        int z = -1;
        unsigned reads = 0;
        if (sl < r.stop) {
            if (sl < r.rb) {
                z = r.y;
            } else {
                const int c = a.col[sl];
                reads += 2;
                if (c != r.x) {
                    if (a.col_live[sl] >= 0) {
                        z = c;
                    } else {
                        reads += 2;
                        if (a.stamp[a.slot_eid[sl]] == round) z = c;
                    }
                }
            }
        }
        int state = kKept, p = r.x, q = z;
        if (z >= 0) {
            pairs++;
            state = pair_quick(a, p, q, reads);
        }
        unsigned hard = __ballot_sync(0xffffffffu, state == kHard);
        while (hard) {
            const int leader = __ffs(hard) - 1;
            hard &= hard - 1;
            const int hp = __shfl_sync(0xffffffffu, p, leader);
            const int hq = __shfl_sync(0xffffffffu, q, leader);
            const bool kept = warp_common_neighbour(a, hp, hq, reads);
            if (lane == leader) state = kept ? kKept : kLost;
        }
        if (state == kLost) record_lost(a, st, r.x, z, u, reads);
        reads_total += reads;
    }
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        reads_total += __shfl_xor_sync(0xffffffffu, reads_total, o);
    }
    if (lane == 0 && pairs) {
        atomicAdd(&s_pairs, pairs);
        atomicAdd(&s_reads, reads_total);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_pairs) {
        atomicAdd((unsigned long long *)&st->st_pairs, s_pairs);
        atomicAdd(&st->st_bytes_detect, 4ull * s_reads);
    }
}

// Splits every directed loss (v loses w) into update items of at most 32 of v's slots.
// The detection reserved the work, so the item list always has room.  Also counts, once
// per round and vertex, the alive edges whose support the updates bring up to date.
__device__ void ph_loss_items(const LossArgs &a) {
    DevStatus *st = a.st;
    const int nd = 2 * min(vload(st->nlost), a.lost_max), round = vload(st->round);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    unsigned long long touched = 0ull;
    for (int b = blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < nd; b += stride) {
        const int d = b + lane;
        int nch = 0, rb = 0;
        if (d < nd) {
            const int4 L = a.lost[d >> 1];
            if (L.x >= 0) {
                const int v = (d & 1) ? L.y : L.x;
                rb = a.row_ptr[v];
                nch = (a.row_ptr[v + 1] - rb + 31) >> 5;
                if (atomicExch(a.vtouch + v, round) != round) touched += a.deg_alive[v];
            }
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && tot) base = atomicAdd(&st->nuitems, tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        const int first = base + incl - nch;
        for (int c = 0; c < nch && first + c < a.uitems_cap; c++)
            a.uitems[first + c] = make_int2(d, rb + 32 * c);
    }
    for (int o = 16; o > 0; o >>= 1) touched += __shfl_xor_sync(0xffffffffu, touched, o);
    if (lane == 0 && touched) atomicAdd((unsigned long long *)&st->st_recomputed, touched);
}

// Support updates, one warp per item (a directed loss v loses w, and 32 of v's slots).
// PASS 0 (stored balls still old) handles edges (v,z) with v < z and tests w in B_old(z);
// PASS 1 (after the clears) handles v > z and tests w in B_new(z).  Distance is symmetric,
// so w in B(z) is tested as z in B(w): all lanes read the same ball, at increasing z.
template <int PASS>
__device__ void ph_delta(const LossArgs &a) {
    __shared__ unsigned long long s_tests, s_bytes;
    DevStatus *st = a.st;
    if (threadIdx.x == 0) {
        s_tests = 0ull;
        s_bytes = 0ull;
    }
    __syncthreads();
    const int nitems = min(vload(st->nuitems), a.uitems_cap);
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned long long tests = 0ull, bytes_total = 0ull;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems; it += nwarps) {
        const int2 item = a.uitems[it];
        const int4 L = a.lost[item.x >> 1];
        const int v = (item.x & 1) ? L.y : L.x;
        const int w = (item.x & 1) ? L.x : L.y;
        const int2 wmeta = a.ball_meta[w];
        const int re = a.row_ptr[v + 1];
        const int sl = item.y + lane;
        unsigned bytes = (lane == 0) ? 32u : 0u;  // item, loss record, row end, ball metadata
        if (sl < re) {
            const int z = a.col_live[sl];
            bytes += 4;
            if (z >= 0 && (PASS == 0 ? (v < z) : (v > z))) {
                tests++;
                if (ball_contains_meta(a, wmeta, z, bytes)) {
                    atomicSub(a.sup + a.slot_eid[sl], 1);
                    bytes += 12;
                }
            }
        }
        bytes_total += bytes;
    }
    for (int o = 16; o > 0; o >>= 1) {
        tests += __shfl_xor_sync(0xffffffffu, tests, o);
        bytes_total += __shfl_xor_sync(0xffffffffu, bytes_total, o);
    }
    if (lane == 0 && (tests || bytes_total)) {
        atomicAdd(&s_tests, tests);
        atomicAdd(&s_bytes, bytes_total);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (s_tests || s_bytes)) {
        atomicAdd((unsigned long long *)&st->st_tests, s_tests);
        atomicAdd(&st->st_bytes_update, s_bytes);
    }
}

// Clears every lost member from the stored balls and empties the hash slots.
__device__ void ph_apply(const LossArgs &a) {
    DevStatus *st = a.st;
    const int nlost = min(vload(st->nlost), a.lost_max);
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < 2 * nlost; d += gridDim.x * blockDim.x) {
        const int4 L = a.lost[d >> 1];
        if (L.x < 0) continue;
        const int v = (d & 1) ? L.y : L.x;
        const int w = (d & 1) ? L.x : L.y;
        const int2 meta = a.ball_meta[v];
        const int nw = meta.y;
        const int64_t off = (int64_t)(unsigned)meta.x << 2;
        const uint32_t bit = 1u << (w & 31);
        const uint32_t wi = (uint32_t)(w >> 5);
        uint32_t *word = nullptr;
        if (nw < 0) {
            word = a.pool + off + wi;
        } else {
            const uint2 *p = reinterpret_cast<const uint2 *>(a.pool + off);
            int lo = 0, hi = nw - 1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const uint32_t idx = p[mid].x;
                if (idx == wi) {
                    word = a.pool + off + 2 * (int64_t)mid + 1;
                    break;
                }
                if (idx < wi) lo = mid + 1;
                else hi = mid - 1;
            }
        }
        if (word) {
            const uint32_t old = atomicAnd(word, ~bit);
            if (old & bit) atomicSub(a.ball_size + v, 1);
        }
        if ((d & 1) == 0) a.keys[L.z] = kEmpty;
    }
    // lost pairs of this batch (non-null records), one atomic per warp
    unsigned long long real = 0ull;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nlost; r += gridDim.x * blockDim.x)
        real += (a.lost[r].x >= 0);
    for (int o = 16; o > 0; o >>= 1) real += __shfl_xor_sync(0xffffffffu, real, o);
    if ((threadIdx.x & 31) == 0 && real) atomicAdd((unsigned long long *)&st->st_lost, real);
}

// Frontier selection and removal in one pass (incremental rounds): every alive edge with
// h-support <= k-2 joins F and is removed at once (Algorithm 1, lines 7-10).
__device__ void ph_select_remove(const LossArgs &a) {
    DevStatus *st = a.st;
    if (vload(st->cont)) return;  // a continued round keeps its (already removed) frontier
    const int k = vload(st->k), round = vload(st->round), thr = k - 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); e0 < a.m; e0 += stride) {
        const int64_t e = e0 + (threadIdx.x & 31);
        const bool p = e < a.m && a.sup[e] <= thr;
        warp_append(p, (int32_t)e, &st->nF, a.frontier_w);
        if (p)
            remove_edge((int)e, k, round, a.eu, a.ev, a.slot_lo, a.slot_hi, a.sup, a.truss,
                        a.stamp_w, a.col_live_w, a.deg_alive_w, a.hub_slot, a.hub_bits_w, a.Wpad);
    }
}

// One launch per phase (the rounds of a CUDA graph).
__global__ void __launch_bounds__(kBlock) k_pair_items(LossArgs a) {
    if (vload(a.st->alive) == 0) return;
    ph_pair_items(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_detect(LossArgs a) {
    if (vload(a.st->alive) == 0) return;
    ph_detect(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_items(LossArgs a) {
    if (vload(a.st->alive) == 0) return;
    ph_loss_items(a);
}
template <int PASS>
__global__ void __launch_bounds__(kBlock) k_loss_delta(LossArgs a) {
    if (vload(a.st->alive) == 0) return;
    ph_delta<PASS>(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_apply(LossArgs a) {
    if (vload(a.st->alive) == 0) return;
    ph_apply(a);
}

constexpr int kPBlock = 512;  // threads per block of the persistent kernel

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Persistent round kernel (cooperative launch, every block resident): runs up to
// `max_slots` round slots, each the eight phases of an incremental round separated by grid
// barriers, and stops early once no edge is alive or an error is flagged.  Block 0 adds
// the time of each phase to the status block.
__global__ void __launch_bounds__(kPBlock, 3) k_rounds_persistent(LossArgs a, int max_slots) {
    DevStatus *st = a.st;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_prev = timer ? global_ns() : 0ull;
    auto phase_done = [&](int p) -> bool {
        if (!grid_barrier(st)) return false;
        if (timer) {
            const unsigned long long t = global_ns();
            st->st_phase_ns[p] += t - t_prev;
            t_prev = t;
        }
        return true;
    };
    for (int slot = 0; slot < max_slots; slot++) {
        if (vload(st->alive) == 0 || vload(st->err) != 0) break;
        ph_select_remove(a);
        if (!phase_done(0)) return;
        ph_pair_items(a);
        if (!phase_done(1)) return;
        ph_detect(a);
        if (!phase_done(2)) return;
        ph_loss_items(a);
        if (!phase_done(3)) return;
        ph_delta<0>(a);
        if (!phase_done(4)) return;
        ph_apply(a);
        if (!phase_done(5)) return;
        ph_delta<1>(a);
        if (!phase_done(6)) return;
        minreduce_body<kPBlock / 32>(a.sup, a.m, st, 0);
        if (!phase_done(7)) return;
        if (timer) st->st_slots++;
    }
}

LossArgs loss_args(Handle *H) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    LossArgs a;
    a.h = w.h;
    a.lost_max = (int32_t)w.lost_max;
    a.cap_mask = (unsigned long long)(w.lost_cap - 1);
    a.row_ptr = g.row_ptr;
    a.col = g.col;
    a.col_live = w.col_live;
    a.slot_eid = g.slot_eid;
    a.eu = g.eu;
    a.ev = g.ev;
    a.frontier = w.frontier;
    a.stamp = w.stamp;
    a.pool = w.pool;
    a.ball_off = w.ball_off;
    a.ball_nw = w.ball_nw;
    a.ball_meta = w.ball_meta;
    a.ball_size = w.ball_size;
    a.keys = w.lost_keys;
    a.lost = w.lost;
    a.sup = w.sup;
    a.vtouch = w.edge_touch;
    a.deg_alive = w.deg_alive;
    a.pitems_cap = (int32_t)w.pitems_cap;
    a.pitems = w.pitems;
    a.uitems_cap = (int32_t)w.uitems_cap;
    a.uitems = w.uitems;
    a.upd_budget = w.upd_budget;
    a.hub_slot = w.hub_slot;
    a.hub_bits = w.hub_bits;
    a.Wpad = w.Wpad;
    a.m = g.m;
    a.slot_lo = g.slot_lo;
    a.slot_hi = g.slot_hi;
    a.truss = w.truss;
    a.stamp_w = w.stamp;
    a.frontier_w = w.frontier;
    a.col_live_w = w.col_live;
    a.deg_alive_w = w.deg_alive;
    a.hub_bits_w = w.hub_bits;
    a.st = w.status;
    return a;
}

}  // namespace

// Enqueues the loss detection and the support updates of one incremental round (after
// k_remove, before the min reduction).  ev_mid (nullable) is recorded between the two.
// Launches the persistent round kernel once (at most max_slots round slots).  The grid is
// every block that can be resident at once, as a cooperative launch requires.
htd_status launch_persistent_rounds(Handle *H, cudaStream_t s, int max_slots, int64_t *launches) {
    LossArgs a = loss_args(H);
    static thread_local int grid_cached = 0, dev_cached = -1;
    if (grid_cached == 0 || dev_cached != H->g.device) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rounds_persistent,
                                                                      kPBlock, 0);
        if (e != cudaSuccess || occ < 1) {
            set_last_error("persistent round kernel: no resident block fits");
            return HTD_ECUDA;
        }
        grid_cached = H->num_sms * occ;
        dev_cached = H->g.device;
    }
    void *args[] = {&a, &max_slots};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_rounds_persistent, dim3(grid_cached),
                                                dim3(kPBlock), args, 0, s);
    (*launches)++;
    if (e != cudaSuccess) {
        set_last_error(std::string("persistent round kernel: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    return HTD_OK;
}

htd_status enqueue_loss_kernels(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t ev_mid,
                                unsigned record_flags) {
    LossArgs a = loss_args(H);
    const int grid = H->num_sms * 8;
    k_pair_items<<<H->num_sms * 4, kBlock, 0, s>>>(a);
    k_loss_detect<<<grid, kBlock, 0, s>>>(a);
    if (ev_mid) cudaEventRecordWithFlags(ev_mid, s, record_flags);
    k_loss_items<<<H->num_sms * 4, kBlock, 0, s>>>(a);
    k_loss_delta<0><<<grid, kBlock, 0, s>>>(a);
    k_loss_apply<<<grid, kBlock, 0, s>>>(a);
    k_loss_delta<1><<<grid, kBlock, 0, s>>>(a);
    *launches += 6;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("enqueue_loss_kernels: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    return HTD_OK;
}

}  // namespace htd
