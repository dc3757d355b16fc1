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
#include <algorithm>
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
    int32_t dense_all;  // every ball dense at pool + x * Wpad (no metadata lookup)
    int32_t hub_all;    // every vertex has its alive-adjacency set, at row x
    int32_t pitems_cap;
    int4 *pitems;
    int32_t uitems_cap;
    int4 *uitems;
    long long upd_budget;
    DevStatus *st;
    // h = 3: radius-2 balls and the round's radius-2 losses
    int32_t h3;         // incremental h = 3 round: overflows halt the round (host rebuild)
    int32_t rec_r2;     // this launch records radius-2 losses (no support updates)
    uint32_t *pool2;    // dense radius-2 balls, row x at x * Wpad
    int32_t *ball_size2;
    unsigned long long *keys2;
    unsigned long long cap2_mask;
    int4 *lost2;
    int32_t lost2_max;
    int32_t c3items_cap;
    int4 *c3items;
    int32_t *touch2;    // h = 3: round in which the vertex last lost a radius-2 member
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

// A batch limit was reached at edge side u: h <= 2 resumes the round there in the next slot;
// an h = 3 round halts and the host finishes it by rebuilds.
__device__ __forceinline__ void overflow_at(const LossArgs &a, DevStatus *st, int u) {
    if (a.h3) atomicOr(&st->halt, 1);
    else atomicMin(&st->overflow_unit, u);
}

// Round kernels do nothing once the peel is over or a round halted.
__device__ __forceinline__ bool round_idle(const LossArgs &a) {
    return vload(a.st->alive) == 0 || vload(a.st->halt) != 0;
}

// Alive-adjacency set of p if p has one (high degree), else null.
__device__ __forceinline__ const uint32_t *hub_set(const LossArgs &a, int p, unsigned &reads) {
    if (a.hub_all) return a.hub_bits + (int64_t)p * a.Wpad;
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

// Short rows are scanned by one lane; pairs whose shorter row is longer go to the warp.
constexpr int kInlineScan = 8;

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
    if (min(dp, dq) > kInlineScan) return kHard;
    const int rb = a.row_ptr[p], re = a.row_ptr[p + 1];
    // four slots at a time: their loads (and their set lookups) are independent
    for (int s0 = rb; s0 < re; s0 += 4) {
        int y[4];
#pragma unroll
        for (int j = 0; j < 4; j++) y[j] = (s0 + j < re) ? a.col_live[s0 + j] : -1;
        bool hit = false;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (y[j] >= 0) hit |= alive_adjacent_set(a, qset, q, y[j], reads);
        reads += (unsigned)min(4, re - s0);
        if (hit) return kKept;
    }
    return kLost;
}

// Inclusive prefix sum over the warp.
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Slots of the concatenated rows each lane loads per step of a warp's common walk (their
// loads are independent, so a step costs two round trips whatever the count).
constexpr int kWalkUnroll = 4;

// Common alive neighbours for the warp's hard pairs (lanes with state == kHard; p the
// shorter row), all at once: the pairs' rows of p are laid end to end and the warp walks
// the concatenation 32 x kWalkUnroll slots per step, each lane finding the pair its slot belongs to by a
// binary search over the lanes' running row lengths.  A pair is kept at its first alive
// neighbour that q also has; the walk skips kept pairs and stops once none is pending.
// Called by whole warps.
__device__ __forceinline__ void warp_hard_pairs(const LossArgs &a, int &state, int p, int q,
                                                unsigned &reads) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool hard = state == kHard;
    int rb = 0, len = 0;
    const uint32_t *qset = nullptr;
    if (hard) {
        rb = a.row_ptr[p];
        len = a.row_ptr[p + 1] - rb;
        qset = hub_set(a, q, reads);
        reads += 2;
    }
    const int incl = warp_incl_scan(len);
    const int excl = incl - len;
    const int total = __shfl_sync(full, incl, 31);
    unsigned pending = __ballot_sync(full, hard);
    unsigned kept = 0u;
    for (int base = 0; base < total && pending; base += 32 * kWalkUnroll) {
        int y[kWalkUnroll], own[kWalkUnroll];
#pragma unroll
        for (int j = 0; j < kWalkUnroll; j++) {
            const int idx = base + 32 * j + lane;
            // owner lane: the number of lanes whose rows end at or before idx
            int o = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(full, incl, o + step - 1) <= idx) o += step;
            o = min(o, 31);
            const int ex = __shfl_sync(full, excl, o), rbo = __shfl_sync(full, rb, o);
            own[j] = o;
            y[j] = (idx < total && ((pending >> o) & 1u)) ? a.col_live[rbo + idx - ex] : -1;
        }
        unsigned hits = 0u;
#pragma unroll
        for (int j = 0; j < kWalkUnroll; j++) {
            const int qo = __shfl_sync(full, q, own[j]);
            const uint32_t *qs = reinterpret_cast<const uint32_t *>(
                __shfl_sync(full, reinterpret_cast<unsigned long long>(qset), own[j]));
            if (y[j] >= 0) {
                reads++;
                if (alive_adjacent_set(a, qs, qo, y[j], reads)) hits |= 1u << own[j];
            }
        }
        hits = __reduce_or_sync(full, hits);
        kept |= hits;
        pending &= ~hits;
    }
    if (hard) state = ((kept >> lane) & 1u) ? kKept : kLost;
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
    if (a.dense_all) {
        bytes += 4;
        return (a.pool[(int64_t)z * a.Wpad + (w >> 5)] >> (w & 31)) & 1u;
    }
    bytes += 8;
    return ball_contains_meta(a, a.ball_meta[z], w, bytes);
}

// Records the lost pair {x,z} unless an earlier batch of this round handled it.  The
// record and the pair's update work (both rows are visited by the support updates) are
// reserved against the batch limits; a pair that does not fit marks its edge side u as
// the point where the next slot of this round resumes.
// Is the pair {p,q} among this batch's lost pairs?
__device__ __forceinline__ bool lost_now(const LossArgs &a, int p, int q, unsigned &bytes) {
    const unsigned long long key = pair_key(p, q);
    unsigned long long slot = mix64(key) & a.cap_mask;
    for (unsigned long long probe = 0; probe <= a.cap_mask; probe++) {
        const unsigned long long k = a.keys[slot];
        bytes += 8;
        if (k == key) return true;
        if (k == kEmpty) return false;
        slot = (slot + 1) & a.cap_mask;
    }
    return false;
}

// Records the lost pairs {x, z} of a warp (lanes with lost == true; all lanes call it).
// A pair whose stored bit is already clear was handled by an earlier batch of this round
// and is skipped.  Each record and its update work (both rows are visited by the support
// updates) are reserved against the batch limits with one atomic per warp and counter; a
// pair that does not fit marks its edge side u as the point where the next slot of this
// round resumes.  New pairs go into the lost-pair set, and their update items (runs of 32
// slots of each endpoint's row) are written: by their own lane when few, else by the warp.
__device__ __forceinline__ void record_lost_warp(const LossArgs &a, DevStatus *st, bool lost, int x,
                                                 int z, int u, unsigned &reads) {
    constexpr int kOwnItems = 8;
    const int lane = threadIdx.x & 31;
    const bool r2 = a.rec_r2 != 0;  // radius-2 losses of an h = 3 round: record only
    bool want = false;
    if (lost) {
        if (r2) {
            reads++;
            want = (a.pool2[(int64_t)x * a.Wpad + (z >> 5)] >> (z & 31)) & 1u;
        } else {
            want = ball_contains(a, x, z, reads);
        }
    }
    int rbx = 0, rex = 0, rbz = 0, rez = 0;
    long long work = 0;
    if (want && !r2) {
        rbx = a.row_ptr[x];
        rex = a.row_ptr[x + 1];
        rbz = a.row_ptr[z];
        rez = a.row_ptr[z + 1];
        work = (long long)(rex - rbx) + (rez - rbz);
    }
    const unsigned wantb = __ballot_sync(0xffffffffu, want);
    if (wantb == 0u) return;
    const long long wincl = warp_incl_scan(work);
    const int rank = __popc(wantb & lanemask_lt());
    const long long wtot = __shfl_sync(0xffffffffu, wincl, 31);
    long long wbase = 0;
    int ibase = 0;
    if (lane == 0) {
        if (!r2)
            wbase = (long long)atomicAdd((unsigned long long *)&st->upd_work, (unsigned long long)wtot);
        ibase = atomicAdd(r2 ? &st->nlost2 : &st->nlost, __popc(wantb));
    }
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    ibase = __shfl_sync(0xffffffffu, ibase, 0);
    int4 *const lostv = r2 ? a.lost2 : a.lost;
    unsigned long long *const keys = r2 ? a.keys2 : a.keys;
    const unsigned long long cmask = r2 ? a.cap2_mask : a.cap_mask;
    const int lmax = r2 ? a.lost2_max : a.lost_max;
    int rec_idx = -1;
    if (want) {
        const int idx = ibase + rank;
        if (idx >= lmax || (!r2 && wbase + wincl > a.upd_budget)) {
            overflow_at(a, st, u);
            if (idx < lmax) lostv[idx] = make_int4(-1, -1, -1, 0);
        } else {
            const unsigned long long key = pair_key(x, z);
            unsigned long long slot = mix64(key) & cmask;
            int4 rec = make_int4(-1, -1, -1, 0);  // null record: the pair is already held
            for (unsigned long long probe = 0; probe <= cmask; probe++) {
                const unsigned long long prev = atomicCAS(keys + slot, kEmpty, key);
                if (prev == kEmpty) {
                    rec = make_int4(min(x, z), max(x, z), (int)slot, 0);
                    break;
                }
                if (prev == key) break;
                slot = (slot + 1) & cmask;
            }
            lostv[idx] = rec;
            if (rec.x >= 0) rec_idx = idx;
            if (r2) {
                // B2_new(v) differs from the stored B2(v) only at vertices marked here
                const int round = vload(st->round);
                a.touch2[x] = round;
                a.touch2[z] = round;
            }
        }
    }
    if (r2) return;  // radius-2 losses change no support directly
    // update items: direction 0 = v0 = min loses v1, direction 1 = v1 loses v0
    int v0 = 0, v1 = 0, rb0 = 0, re0 = 0, rb1 = 0, re1 = 0, n0 = 0, n1 = 0;
    if (rec_idx >= 0) {
        const bool xf = x < z;
        v0 = xf ? x : z;
        v1 = xf ? z : x;
        rb0 = xf ? rbx : rbz;
        re0 = xf ? rex : rez;
        rb1 = xf ? rbz : rbx;
        re1 = xf ? rez : rex;
        n0 = (re0 - rb0 + 31) >> 5;
        n1 = (re1 - rb1 + 31) >> 5;
    }
    const int nincl = warp_incl_scan(n0 + n1);
    int nbase = 0;
    if (lane == 31 && nincl) nbase = atomicAdd(&st->nuitems, nincl);
    nbase = __shfl_sync(0xffffffffu, nbase, 31);
    const int base = nbase + nincl - (n0 + n1);
    if (rec_idx >= 0 && n0 + n1 <= kOwnItems) {
        for (int c = 0; c < n0 + n1 && base + c < a.uitems_cap; c++)
            a.uitems[base + c] = (c < n0) ? make_int4(rb0 + 32 * c, v0, v1, re0)
                                          : make_int4(rb1 + 32 * (c - n0), v1, v0, re1);
    }
    unsigned big = __ballot_sync(0xffffffffu, rec_idx >= 0 && n0 + n1 > kOwnItems);
    while (big) {
        const int l = __ffs(big) - 1;
        big &= big - 1;
        const int b = __shfl_sync(0xffffffffu, base, l);
        const int c0 = __shfl_sync(0xffffffffu, n0, l), c1 = __shfl_sync(0xffffffffu, n1, l);
        const int w0 = __shfl_sync(0xffffffffu, v0, l), w1 = __shfl_sync(0xffffffffu, v1, l);
        const int b0 = __shfl_sync(0xffffffffu, rb0, l), e0 = __shfl_sync(0xffffffffu, re0, l);
        const int b1 = __shfl_sync(0xffffffffu, rb1, l), e1 = __shfl_sync(0xffffffffu, re1, l);
        for (int c = lane; c < c0 + c1 && b + c < a.uitems_cap; c += 32)
            a.uitems[b + c] = (c < c0) ? make_int4(b0 + 32 * c, w0, w1, e0)
                                       : make_int4(b1 + 32 * (c - c0), w1, w0, e1);
    }
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
        int nch = 0, start = 0, x = 0, y = 0;
        if (u < units) {
            const UnitInfo r = unit_info(a, u);
            start = r.start;
            x = r.x;
            y = r.y;
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
        if (!fits && nch) overflow_at(a, st, u);
        // the whole warp writes each lane's items in turn (a hub row has hundreds)
        unsigned todo = __ballot_sync(0xffffffffu, nch > 0);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const int f = __shfl_sync(0xffffffffu, first, l), c_n = __shfl_sync(0xffffffffu, nch, l);
            const int ul = __shfl_sync(0xffffffffu, u, l), sl = __shfl_sync(0xffffffffu, start, l);
            const int xl = __shfl_sync(0xffffffffu, x, l), yl = __shfl_sync(0xffffffffu, y, l);
            const bool fl = __shfl_sync(0xffffffffu, fits, l);
            for (int c = lane; c < c_n && f + c < a.pitems_cap; c += 32)
                a.pitems[f + c] = fl ? make_int4(ul, sl + 32 * c, xl, yl) : make_int4(-1, 0, 0, 0);
        }
    }
}

// Loss detection, one warp per item: lane i tests the pair of slot item.y + i.  A pair is
// kept if its endpoints are adjacent or (h = 2) share an alive neighbour; the pairs whose
// test needs a longer row scan are walked by the whole warp together.
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
    unsigned long long pairs = 0ull, reads_total = 0ull;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < nitems; it += nwarps) {
        const int4 item = a.pitems[it];
        const int u = item.x;
        // sides past an overflow are redone by the next slot of the round: skip them now
        if (u < 0 || u > *(volatile int *)&st->overflow_unit) continue;
        UnitInfo r;
        r.x = item.z;
        r.y = item.w;
        r.rb = a.row_ptr[r.y];
        r.stop = (a.h < 2) ? r.rb : a.row_ptr[r.y + 1];
        const int sl = item.y + lane;
        int z = -1;
        unsigned reads = 0;
        if (sl < r.stop) {
            if (sl < r.rb) {
                z = r.y;
            } else {
                // an old neighbour: alive, or removed in this round
                const int c = a.col[sl], cl = a.col_live[sl];
                reads += 2;
                if (c != r.x && (cl >= 0 || cl == -(round + 1))) z = c;
            }
        }
        int state = kKept, p = r.x, q = z;
        if (z >= 0) {
            pairs++;
            state = pair_quick(a, p, q, reads);
        }
        if (__any_sync(0xffffffffu, state == kHard)) warp_hard_pairs(a, state, p, q, reads);
        record_lost_warp(a, st, state == kLost, r.x, z, u, reads);
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

// Support updates, one warp per item (a directed loss v loses w, and <= 32 of v's slots),
// both orientations in one pass against the stored balls of before this batch: an edge
// (v,z) with v < z loses w from B(v) ∩ B(z) iff w in B_old(z); with v > z iff w in
// B_new(z) = B_old(z) minus this batch's losses.  Distance is symmetric, so w in B(z) is
// tested as z in B(w) (all lanes read one ball, at increasing z) and "w lost by z" as the
// pair {w,z} in the lost-pair set.
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
    unsigned long long tests = 0ull, bytes_total = 0ull;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    // four items per warp and step, their loads interleaved (one GB300, R-MAT 18 at h = 2:
    // 4.80 s per decomposition against 4.86 s with two)
    constexpr int U = 4;
    for (int it0 = U * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); it0 < nitems;
         it0 += U * nwarps) {
        int4 item[U];  // (first slot, v, w, end of v's row)
#pragma unroll
        for (int j = 0; j < U; j++)
            item[j] = (it0 + j < nitems) ? a.uitems[it0 + j] : make_int4(0, 0, 0, 0);
        int z[U], eid[U];
        bool in_w[U];
#pragma unroll
        for (int j = 0; j < U; j++) {
            const int sl = item[j].x + lane;
            const bool ok = sl < item[j].w;
            z[j] = ok ? a.col_live[sl] : -1;
            eid[j] = ok ? a.slot_eid[sl] : 0;
            if (lane == 0 && it0 + j < nitems) bytes_total += a.dense_all ? 16u : 24u;
            if (ok) bytes_total += 4;
        }
#pragma unroll
        for (int j = 0; j < U; j++) {
            in_w[j] = false;
            if (z[j] >= 0) {
                tests++;
                unsigned bytes = 0;
                if (a.dense_all) {
                    in_w[j] = (a.pool[(int64_t)item[j].z * a.Wpad + (z[j] >> 5)] >> (z[j] & 31)) & 1u;
                    bytes += 4;
                } else {
                    in_w[j] = ball_contains(a, item[j].z, z[j], bytes);
                }
                bytes_total += bytes;
            }
        }
#pragma unroll
        for (int j = 0; j < U; j++) {
            unsigned bytes = 0;
            if (in_w[j] && (item[j].y < z[j] || !lost_now(a, item[j].z, z[j], bytes))) {
                atomicSub(a.sup + eid[j], 1);
                bytes += 8;
            }
            bytes_total += bytes;
        }
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

// Clears every lost member from the stored balls and empties the hash slots.  Also counts,
// once per round and vertex, the alive edges whose support the round brings up to date
// (every alive edge at an endpoint of a lost pair).
__device__ void ph_apply(const LossArgs &a) {
    DevStatus *st = a.st;
    const int nlost = min(vload(st->nlost), a.lost_max), round = vload(st->round);
    unsigned long long touched = 0ull;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < 2 * nlost; d += gridDim.x * blockDim.x) {
        const int4 L = a.lost[d >> 1];
        if (L.x < 0) continue;
        const int v = (d & 1) ? L.y : L.x;
        const int w = (d & 1) ? L.x : L.y;
        const uint32_t bit = 1u << (w & 31);
        const uint32_t wi = (uint32_t)(w >> 5);
        uint32_t *word = nullptr;
        if (a.dense_all) {
            word = a.pool + (int64_t)v * a.Wpad + wi;
        } else {
            const int2 meta = a.ball_meta[v];
            const int nw = meta.y;
            const int64_t off = (int64_t)(unsigned)meta.x << 2;
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
        }
        if (word) {
            const uint32_t old = atomicAnd(word, ~bit);
            if (old & bit) atomicSub(a.ball_size + v, 1);
        }
        if ((d & 1) == 0) a.keys[L.z] = kEmpty;
        if (atomicExch(a.vtouch + v, round) != round) touched += (unsigned)a.deg_alive[v];
    }
    // lost pairs of this batch (non-null records), one atomic per warp
    unsigned long long real = 0ull;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nlost; r += gridDim.x * blockDim.x)
        real += (a.lost[r].x >= 0);
    for (int o = 16; o > 0; o >>= 1) {
        real += __shfl_xor_sync(0xffffffffu, real, o);
        touched += __shfl_xor_sync(0xffffffffu, touched, o);
    }
    if ((threadIdx.x & 31) == 0 && real) atomicAdd((unsigned long long *)&st->st_lost, real);
    if ((threadIdx.x & 31) == 0 && touched)
        atomicAdd((unsigned long long *)&st->st_recomputed, touched);
}

// ---- h = 3 -------------------------------------------------------------------------------
//
// At h = 3 the supports are taken on radius-3 balls B3 while radius-2 balls B2 are kept
// beside them.  Removing F can only separate pairs that had a path of at most 3 edges
// through a removed edge (a,b), i.e. pairs {p,q} with p in B(a,i), q in B(b,2-i) before the
// removal, i = 0, 1, 2:  {a} x B2_old(b),  N_old(a) x N_old(b),  B2_old(a) x {b}.  A
// candidate still in B3_old(p) stays within distance 3 iff q is in B2_new(z) for z = p or
// for some alive neighbour z of p (or, symmetrically, of q).  B2_new is the stored B2 minus
// this round's radius-2 losses, which the radius-2 detection (the h = 2 rule, recorded in
// their own pair set) has listed first.  Radius-3 losses then take the support deltas of
// the h = 2 rounds unchanged, on B3.

// Is the pair {p,q} among this round's radius-2 losses?
__device__ __forceinline__ bool lost2_now(const LossArgs &a, int p, int q, unsigned &bytes) {
    const unsigned long long key = pair_key(p, q);
    unsigned long long slot = mix64(key) & a.cap2_mask;
    for (unsigned long long probe = 0; probe <= a.cap2_mask; probe++) {
        const unsigned long long k = a.keys2[slot];
        bytes += 8;
        if (k == key) return true;
        if (k == kEmpty) return false;
        slot = (slot + 1) & a.cap2_mask;
    }
    return false;
}

// q in B2_new(z): the stored radius-2 bit, unless this round lost the pair (the pair set is
// probed only for vertices that lost a radius-2 member this round).
__device__ __forceinline__ bool in_b2_new(const LossArgs &a, int z, int q, int round, unsigned &bytes) {
    bytes += 4;
    if (!((a.pool2[(int64_t)z * a.Wpad + (q >> 5)] >> (q & 31)) & 1u)) return false;
    if (z == q) return true;
    bytes += 4;
    if (a.touch2[z] != round) return true;
    return !lost2_now(a, z, q, bytes);
}

// Position of the k-th (0-based) set bit of v (k < popc(v)).
__device__ __forceinline__ int nth_set_bit(uint32_t v, int k) {
    for (; k > 0; k--) v &= v - 1u;
    return __ffs(v) - 1;
}

// Words of a B2 row one radius-3 candidate item scans: at most 128 candidates, so that one
// item never holds up its launch (one GB300, DC-SBM n = 200,000 at h = 3: 3.7 s per
// decomposition with 4 words, 4.2 s with 16, 5.1 s with 32; 2 words made more rounds
// overflow the item list).
constexpr int kC3Words = 4;
// Range items one warp tests per step (kC3Words lanes each).
constexpr int kC3Groups = 32 / kC3Words;
static_assert(32 % kC3Words == 0, "range items must tile a warp");

// Radius-3 candidate items of the round's frontier.  For each frontier edge F[f] = (a,b):
//   (a, row b, word range) and (b, row a, word range): {a} x B2_old(b) and {b} x B2_old(a),
//     2 * nch items per edge, not stored: item index i < 2 * nch * |F| is frontier edge
//     i / (2 nch), side (i % (2 nch)) / nch, word chunk i % nch (c3_range_item);
//   (p, row b, 32 slots) for every old neighbour p != b of a: N_old(a) x N_old(b), written
//     by one warp per frontier edge into the item list.
// Item layout: (x, y, first word | first slot, -1 - end word | end slot).  A round whose
// items (both kinds) exceed the list's capacity halts.
__device__ __forceinline__ int c3_chunks(const LossArgs &a) { return (a.Wpad + kC3Words - 1) / kC3Words; }

__device__ __forceinline__ int4 c3_range_item(const LossArgs &a, int i, int nch) {
    const int f = i / (2 * nch), r = i - f * 2 * nch;
    const int side = r >= nch, ch = side ? r - nch : r;
    const int e = a.frontier[f];
    const int ea = a.eu[e], eb = a.ev[e];
    const int w0 = ch * kC3Words, w1 = min(a.Wpad, w0 + kC3Words);
    return side ? make_int4(eb, ea, w0, -1 - w1) : make_int4(ea, eb, w0, -1 - w1);
}

__device__ void ph_c3_items(const LossArgs &a) {
    DevStatus *st = a.st;
    const int nF = vload(st->nF), round = vload(st->round);
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const long long nA = 2ll * c3_chunks(a) * nF;
    if (nA > a.c3items_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&st->halt, 1);
        return;
    }
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nF; i += nwarps) {
        const int e = a.frontier[i];
        const int ea = a.eu[e], eb = a.ev[e];
        const int rba = a.row_ptr[ea], rea = a.row_ptr[ea + 1];
        const int rbb = a.row_ptr[eb], reb = a.row_ptr[eb + 1];
        const int nb = (reb - rbb + 31) >> 5;
        for (int s0 = rba; s0 < rea; s0 += 32) {
            const int sl = s0 + lane;
            int p = -1;
            if (sl < rea) {
                const int c = a.col[sl], cl = a.col_live[sl];
                if (c != eb && (cl >= 0 || cl == -(round + 1))) p = c;
            }
            const int cnt = p >= 0 ? nb : 0;
            const int incl = warp_incl_scan(cnt);
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            long long b2 = 0;
            if (lane == 31 && tot)
                b2 = (long long)atomicAdd((unsigned long long *)&st->nc3items, (unsigned long long)tot);
            b2 = __shfl_sync(0xffffffffu, b2, 31);
            if (nA + b2 + tot > a.c3items_cap) {
                if (lane == 0 && tot) atomicOr(&st->halt, 1);
                continue;
            }
            const int first = (int)b2 + incl - cnt;
            for (int c = 0; c < cnt; c++)
                a.c3items[first + c] = make_int4(p, eb, rbb + 32 * c, min(reb, rbb + 32 * (c + 1)));
        }
    }
}

// Common walk of the warp's hard radius-3 pairs (lanes with state == kHard): w is the
// endpoint whose alive row is walked, t the other one; the pair is kept at the first alive
// neighbour y of w with t in B2_new(y).  The rows are laid end to end and walked 128 slots
// per step as in warp_hard_pairs.  Called by whole warps.
__device__ __forceinline__ void warp_walk3(const LossArgs &a, int &state, int w, int t, int round,
                                           unsigned &reads) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool hard = state == kHard;
    int rb = 0, len = 0;
    if (hard) {
        rb = a.row_ptr[w];
        len = a.row_ptr[w + 1] - rb;
        reads += 2;
    }
    const int incl = warp_incl_scan(len);
    const int excl = incl - len;
    const int total = __shfl_sync(full, incl, 31);
    unsigned pending = __ballot_sync(full, hard);
    unsigned kept = 0u;
    for (int base = 0; base < total && pending; base += 128) {
        int y[4], own[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int idx = base + 32 * j + lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(full, incl, o + step - 1) <= idx) o += step;
            o = min(o, 31);
            const int ex = __shfl_sync(full, excl, o), rbo = __shfl_sync(full, rb, o);
            own[j] = o;
            y[j] = (idx < total && ((pending >> o) & 1u)) ? a.col_live[rbo + idx - ex] : -1;
        }
        unsigned hits = 0u;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int to = __shfl_sync(full, t, own[j]);
            if (y[j] >= 0) {
                reads++;
                if (in_b2_new(a, y[j], to, round, reads)) hits |= 1u << own[j];
            }
        }
        hits = __reduce_or_sync(full, hits);
        kept |= hits;
        pending &= ~hits;
    }
    if (hard) state = ((kept >> lane) & 1u) ? kKept : kLost;
}

// Tests the lanes' radius-3 candidate pairs {p,q} (q < 0: none; q is in B3_old(p)) in the
// new graph and records the lost ones with their support-update items.  Whole warps.
__device__ __forceinline__ void test_pairs3(const LossArgs &a, DevStatus *st, int p, int q, int round,
                                            unsigned &reads, unsigned long long &pairs) {
    int state = kKept, w = p, t = q;
    if (q >= 0) {
        pairs++;
        if (!in_b2_new(a, p, q, round, reads)) {
            state = kHard;
            reads += 2;
            if (a.deg_alive[q] < a.deg_alive[p]) {  // walk the shorter alive row
                w = q;
                t = p;
            }
        }
    }
    if (__any_sync(0xffffffffu, state == kHard)) warp_walk3(a, state, w, t, round, reads);
    record_lost_warp(a, st, state == kLost, p, q, 0, reads);
}

// Radius-3 loss tests, one warp per candidate item.
__device__ void ph_test3(const LossArgs &a) {
    __shared__ unsigned long long s_pairs, s_reads;
    DevStatus *st = a.st;
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_reads = 0ull;
    }
    __syncthreads();
    // a round whose items passed the capacity has halted (this kernel is then idle), so
    // both counts fit the list here
    const int nch = c3_chunks(a);
    const long long nA64 = 2ll * nch * vload(st->nF);
    if (nA64 > a.c3items_cap) return;
    const int nA = (int)nA64;
    const int nitems = nA + (int)min(vload(st->nc3items), (long long)a.c3items_cap - nA);
    const int round = vload(st->round);
    const int lane = threadIdx.x & 31;
    unsigned long long pairs = 0ull, reads_total = 0ull;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // {x} x B2_old(y) restricted to B3_old(x), kC3Groups range items per warp and step: the
    // lanes of group g hold the words of item (step * kC3Groups + g) * nwarps + warp (items
    // of one warp step lie far apart, so their candidate counts average out), and the
    // step's candidates are dealt out 32 at a time by a warp prefix sum
    for (int s0 = 0; s0 * kC3Groups * nwarps < nA; s0++) {
        const int it = (s0 * kC3Groups + lane / kC3Words) * nwarps + gw;
        int x = -1, wi = 0;
        uint32_t bits = 0u;
        unsigned reads = 0;
        if (it < nA) {
            const int4 item = c3_range_item(a, it, nch);
            x = item.x;
            wi = item.z + lane % kC3Words;
            if (wi < -1 - item.w) {
                bits = a.pool2[(int64_t)item.y * a.Wpad + wi] & a.pool[(int64_t)x * a.Wpad + wi];
                reads += 2;
                if (wi == (x >> 5)) bits &= ~(1u << (x & 31));
            }
        }
        const int cnt = __popc(bits);
        const int incl = warp_incl_scan(cnt);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int idx = t0 + lane;
            // owner lane: the number of lanes whose candidates end at or before idx
            int o = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(0xffffffffu, incl, o + step - 1) <= idx) o += step;
            o = min(o, 31);
            const uint32_t ob = __shfl_sync(0xffffffffu, bits, o);
            const int ex = __shfl_sync(0xffffffffu, incl - cnt, o);
            const int ow = __shfl_sync(0xffffffffu, wi, o), ox = __shfl_sync(0xffffffffu, x, o);
            int q = -1;
            if (idx < total) q = (ow << 5) + nth_set_bit(ob, idx - ex);
            test_pairs3(a, st, ox, q, round, reads, pairs);
        }
        reads_total += reads;
    }
    // {x} x N_old(y) for the 32 slots of a stored item, restricted to B3_old(x): one per warp
    for (int it = nA + gw; it < nitems; it += nwarps) {
        const int4 item = a.c3items[it - nA];
        const int x = item.x;
        unsigned reads = 0;
        const int sl = item.z + lane;
        int q = -1;
        if (sl < item.w) {
            const int c = a.col[sl], cl = a.col_live[sl];
            reads += 2;
            if (c != x && (cl >= 0 || cl == -(round + 1))) {
                reads++;
                if ((a.pool[(int64_t)x * a.Wpad + (c >> 5)] >> (c & 31)) & 1u) q = c;
            }
        }
        test_pairs3(a, st, x, q, round, reads, pairs);
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
        atomicAdd((unsigned long long *)&st->st_c3_pairs, s_pairs);
        atomicAdd(&st->st_bytes_detect, 4ull * s_reads);
    }
}

// Clears the round's radius-2 losses from the stored B2 (and their pair-set slots).
__device__ void ph_apply2(const LossArgs &a) {
    DevStatus *st = a.st;
    const int nlost = min(vload(st->nlost2), a.lost2_max);
    unsigned long long real = 0ull;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < 2 * nlost; d += gridDim.x * blockDim.x) {
        const int4 L = a.lost2[d >> 1];
        if (L.x < 0) continue;
        const int v = (d & 1) ? L.y : L.x;
        const int w = (d & 1) ? L.x : L.y;
        const uint32_t bit = 1u << (w & 31);
        const uint32_t old = atomicAnd(a.pool2 + (int64_t)v * a.Wpad + (w >> 5), ~bit);
        if (old & bit) atomicSub(a.ball_size2 + v, 1);
        if ((d & 1) == 0) {
            a.keys2[L.z] = kEmpty;
            real++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) real += __shfl_xor_sync(0xffffffffu, real, o);
    if ((threadIdx.x & 31) == 0 && real) atomicAdd((unsigned long long *)&st->st_lost2, real);
}

// One candidate edge per lane (p: it joins the frontier): warp-aggregated frontier slot,
// removal (the removal step of Algorithm 1) and the detection items of its two edge sides.  Whole
// warps call it.
__device__ __forceinline__ void select_one(const LossArgs &a, DevStatus *st, bool p, int e, int k,
                                           int round) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, p);
    if (bal == 0u) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&st->nF, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int pos = base + __popc(bal & lanemask_lt());
    int u_eu = 0, u_ev = 0, rb_u = 0, re_u = 0, rb_v = 0, re_v = 0, n0 = 0, n1 = 0;
    if (p) {
        a.frontier_w[pos] = e;
        remove_edge(e, k, round, a.eu, a.ev, a.slot_lo, a.slot_hi, a.sup, a.truss,
                    a.stamp_w, a.col_live_w, a.deg_alive_w, a.hub_slot, a.hub_bits_w, a.Wpad);
        u_eu = a.eu[e];
        u_ev = a.ev[e];
        rb_u = a.row_ptr[u_eu];
        re_u = a.row_ptr[u_eu + 1];
        rb_v = a.row_ptr[u_ev];
        re_v = a.row_ptr[u_ev + 1];
        // side 0: eu with {ev} and N_old(ev); side 1: ev with N_old(eu); h = 1: {eu,ev}
        n0 = (a.h < 2) ? 1 : (re_v - rb_v + 1 + 31) >> 5;
        n1 = (a.h < 2) ? 0 : (re_u - rb_u + 31) >> 5;
    }
    int incl = n0 + n1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    int ibase = 0;
    if (lane == 31 && tot) ibase = atomicAdd(&st->npitems, tot);
    ibase = __shfl_sync(0xffffffffu, ibase, 31);
    const int first = ibase + incl - (n0 + n1);
    if (p && first + n0 > a.pitems_cap) overflow_at(a, st, 2 * pos);
    if (p && n1 && first + n0 + n1 > a.pitems_cap) overflow_at(a, st, 2 * pos + 1);
    unsigned todo = __ballot_sync(0xffffffffu, p);
    while (todo) {
        const int l = __ffs(todo) - 1;
        todo &= todo - 1;
        const int f = __shfl_sync(0xffffffffu, first, l);
        const int c0 = __shfl_sync(0xffffffffu, n0, l), c1 = __shfl_sync(0xffffffffu, n1, l);
        const int pl = __shfl_sync(0xffffffffu, pos, l);
        const int xu = __shfl_sync(0xffffffffu, u_eu, l), xv = __shfl_sync(0xffffffffu, u_ev, l);
        const int su = __shfl_sync(0xffffffffu, rb_u, l), sv0 = __shfl_sync(0xffffffffu, rb_v, l);
        const bool fits0 = f + c0 <= a.pitems_cap, fits1 = f + c0 + c1 <= a.pitems_cap;
        for (int c = lane; c < c0 + c1 && f + c < a.pitems_cap; c += 32) {
            if (c < c0)
                a.pitems[f + c] = fits0 ? make_int4(2 * pl, sv0 - 1 + 32 * c, xu, xv)
                                        : make_int4(-1, 0, 0, 0);
            else
                a.pitems[f + c] = fits1 ? make_int4(2 * pl + 1, su + 32 * (c - c0), xv, xu)
                                        : make_int4(-1, 0, 0, 0);
        }
    }
}

// Phase 1 of an incremental round: every alive edge with h-support <= k-2 joins F and is
// removed at once (the selection and removal steps of Algorithm 1), and the loss detection items of its two edge
// sides are written.  A continued round only writes the items of its remaining sides.
__device__ void ph_select_items(const LossArgs &a) {
    DevStatus *st = a.st;
    if (vload(st->cont)) {
        ph_pair_items(a);
        return;
    }
    const int k = vload(st->k), round = vload(st->round), thr = k - 2;
    const int lane = threadIdx.x & 31;
    const int64_t stride = 4 * (int64_t)gridDim.x * blockDim.x;
    // four coalesced loads per thread per step, issued before any of them is used
    for (int64_t e0 = 4 * (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)); e0 < a.m;
         e0 += stride) {
        int sv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t e = e0 + 32 * j + lane;
            sv[j] = (e < a.m) ? a.sup[e] : INT_MAX;
        }
#pragma unroll
        for (int j = 0; j < 4; j++) select_one(a, st, sv[j] <= thr, (int)(e0 + 32 * j + lane), k, round);
    }
}

// Programmatic dependent launch: a phase kernel may be scheduled while the previous one
// still runs; it waits here until that grid has completed and its writes are visible, then
// lets the next phase be scheduled in turn.  (Without a programmatic launch the wait
// returns at once.)
__device__ __forceinline__ void phase_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One launch per phase (the rounds of a CUDA graph).
__global__ void __launch_bounds__(kBlock) k_inc_select(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_select_items(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_detect(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_detect(a);
}
// h = 3: the radius-2 detection (a.rec_r2) and the round's radius-3 candidate items
__global__ void __launch_bounds__(kBlock) k_loss_detect3(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_detect(a);
    ph_c3_items(a);
}
__global__ void __launch_bounds__(kBlock) k_loss3_test(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_test3(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_delta(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_delta(a);
}
__global__ void __launch_bounds__(kBlock) k_loss_apply_reduce(LossArgs a) {
    phase_entry();
    if (round_idle(a)) return;
    ph_apply(a);
    if (a.h3) ph_apply2(a);
    minreduce_body<kBlock / 32>(a.sup, a.m, a.st, 0);
}

constexpr int kPBlock = 512;  // threads per block of the persistent kernel

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Persistent round kernel (cooperative launch, every block resident): runs up to
// `max_slots` round slots, each the four phases of an incremental round separated by grid
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
        ph_select_items(a);
        if (!phase_done(0)) return;
        ph_detect(a);
        if (!phase_done(1)) return;
        ph_delta(a);
        if (!phase_done(2)) return;
        // clearing the lost members touches balls and hash slots only; the reduction reads
        // supports only, and its last block closes the round after every block did both
        ph_apply(a);
        minreduce_body<kPBlock / 32>(a.sup, a.m, st, 0);
        if (!phase_done(3)) return;
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
    a.dense_all = w.dense_balls ? 1 : 0;
    a.hub_all = (w.nhub == g.n && w.hub_min_deg == 1) ? 1 : 0;
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
    a.h3 = w.inc3 ? 1 : 0;
    a.rec_r2 = 0;
    a.pool2 = w.pool2;
    a.ball_size2 = w.ball_size2;
    a.keys2 = w.lost2_keys;
    a.cap2_mask = w.lost2_cap > 0 ? (unsigned long long)(w.lost2_cap - 1) : 0ull;
    a.lost2 = w.lost2;
    a.lost2_max = (int32_t)w.lost2_max;
    a.c3items_cap = (int32_t)w.c3items_cap;
    a.c3items = w.c3items;
    a.touch2 = w.touch2;
    return a;
}

}  // namespace

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
        grid_cached = std::min(H->num_sms * occ, 64 * 32);  // the grid barrier's limit
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

namespace {

// Blocks of one full wave of a phase kernel (every block resident at once), per device.
struct PhaseGrids {
    int device = -1;
    int detect = 0, detect3 = 0, delta = 0, test3 = 0;
};

htd_status phase_grids(Handle *H, PhaseGrids &pg) {
    if (pg.device == H->g.device) return HTD_OK;
    int od = 0, od3 = 0, ou = 0, ot = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&od, k_loss_detect, kBlock, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&od3, k_loss_detect3, kBlock, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ou, k_loss_delta, kBlock, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ot, k_loss3_test, kBlock, 0) != cudaSuccess ||
        od < 1 || od3 < 1 || ou < 1 || ot < 1) {
        set_last_error("incremental round: no resident block fits");
        return HTD_ECUDA;
    }
    pg.detect = H->num_sms * od;
    pg.detect3 = H->num_sms * od3;
    pg.delta = H->num_sms * ou;
    pg.test3 = H->num_sms * ot;
    pg.device = H->g.device;
    return HTD_OK;
}

// One phase launch; `pdl` lets it be scheduled before the previous kernel on the stream
// has finished (it waits in phase_entry).
cudaError_t launch_phase(void (*kernel)(LossArgs), int grid, cudaStream_t s, bool pdl,
                         const LossArgs &a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

}  // namespace

// Enqueues one incremental round as four launches (the graph path).  evs (nullable):
// kRoundEvents events; phases are marked as select | - | detect | update | - | reduce.
// Without events the launches are programmatic (each overlaps the previous one's tail).
htd_status enqueue_incremental_round(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t *evs,
                                     unsigned record_flags) {
    LossArgs a = loss_args(H);
    static thread_local PhaseGrids pg;
    const htd_status gs = phase_grids(H, pg);
    if (gs != HTD_OK) return gs;
    const bool pdl = evs == nullptr;
    auto mark = [&](int i) {
        if (evs) cudaEventRecordWithFlags(evs[i], s, record_flags);
    };
    // the two scans over all edges use fewer blocks: the reduction's per-block atomics all
    // hit the same few counters
    const int grid_scan = H->num_sms * 2;
    cudaError_t e = cudaSuccess;
    if (a.h3) {
        // select | radius-2 detection + radius-3 items | radius-3 tests | updates | - | reduce
        LossArgs a2 = a;
        a2.rec_r2 = 1;
        mark(0);
        if (e == cudaSuccess) e = launch_phase(k_inc_select, grid_scan, s, pdl, a);
        mark(1);
        if (e == cudaSuccess) e = launch_phase(k_loss_detect3, pg.detect3, s, pdl, a2);
        mark(2);
        if (e == cudaSuccess) e = launch_phase(k_loss3_test, pg.test3, s, pdl, a);
        mark(3);
        if (e == cudaSuccess) e = launch_phase(k_loss_delta, pg.delta, s, pdl, a);
        mark(4);
        mark(5);
        if (e == cudaSuccess) e = launch_phase(k_loss_apply_reduce, grid_scan, s, pdl, a);
        mark(6);
        *launches += 5;
    } else {
        mark(0);
        if (e == cudaSuccess) e = launch_phase(k_inc_select, grid_scan, s, pdl, a);
        mark(1);
        mark(2);
        if (e == cudaSuccess) e = launch_phase(k_loss_detect, pg.detect, s, pdl, a);
        mark(3);
        if (e == cudaSuccess) e = launch_phase(k_loss_delta, pg.delta, s, pdl, a);
        mark(4);
        mark(5);
        if (e == cudaSuccess) e = launch_phase(k_loss_apply_reduce, grid_scan, s, pdl, a);
        mark(6);
        *launches += 4;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("enqueue_incremental_round: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    return HTD_OK;
}

}  // namespace htd
