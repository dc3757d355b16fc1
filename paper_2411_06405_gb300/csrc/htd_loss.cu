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

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr unsigned long long kEmpty = ~0ull;

struct LossArgs {
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
    int32_t *ball_size;
    unsigned long long *keys;
    int4 *lost;
    int32_t *sup;
    int32_t *edge_touch;
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

// Is q an alive neighbour of p?  Binary search in p's sorted row, then the alive mark.
// `reads` counts the 4-byte words the search touches (algorithmic bytes = 4 x reads).
__device__ __forceinline__ bool alive_adjacent(const LossArgs &a, int p, int q, unsigned &reads) {
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

// dist(p,q) <= h in the alive graph, p != q, h in {1,2}.
__device__ bool within_h(const LossArgs &a, int p, int q, unsigned &reads) {
    const int dp = a.row_ptr[p + 1] - a.row_ptr[p];
    const int dq = a.row_ptr[q + 1] - a.row_ptr[q];
    reads += 4;
    if (dp > dq) {  // p: the shorter row
        const int t = p;
        p = q;
        q = t;
    }
    if (alive_adjacent(a, p, q, reads)) return true;
    if (a.h < 2) return false;
    const int re = a.row_ptr[p + 1];
    for (int s = a.row_ptr[p]; s < re; s++) {
        const int y = a.col_live[s];
        reads++;
        if (y >= 0 && alive_adjacent(a, q, y, reads)) return true;
    }
    return false;
}

// Is w in the stored ball of z (dense words, or sorted (word index, word) pairs)?
// `bytes` counts the algorithmic bytes: 12 of metadata plus the words probed.
__device__ __forceinline__ bool ball_contains(const LossArgs &a, int z, int w, unsigned &bytes) {
    const int nw = a.ball_nw[z];
    const int64_t off = a.ball_off[z];
    const uint32_t bit = 1u << (w & 31);
    const uint32_t wi = (uint32_t)(w >> 5);
    bytes += 12;
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

// Enumerates and tests the candidate pairs of every frontier edge (one warp per edge side):
// side 0 of (a,b) pairs a with {b} ∪ N_old(b) \ {a}; side 1 pairs b with N_old(a) \ {b}.
// "Old" adjacency = slots alive before this round: alive now, or removed in this round.
__global__ void __launch_bounds__(kBlock) k_loss_detect(LossArgs a) {
    __shared__ unsigned long long s_pairs, s_reads;
    DevStatus *st = a.st;
    if (st->alive == 0) return;
    if (threadIdx.x == 0) {
        s_pairs = 0ull;
        s_reads = 0ull;
    }
    __syncthreads();
    unsigned long long reads_total = 0ull;
    const int nF = st->nF, round = st->round, u0 = st->unit_begin;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned long long pairs = 0ull;
    for (int u = u0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); u < 2 * nF; u += nwarps) {
        const int e = a.frontier[u >> 1];
        const int side = u & 1;
        const int x = side ? a.ev[e] : a.eu[e];
        const int y = side ? a.eu[e] : a.ev[e];
        const int rb = a.row_ptr[y], re = a.row_ptr[y + 1];
        const int start = (side == 0) ? rb - 1 : rb;  // slot rb-1 stands for the pair {x,y}
        if (a.h < 2 && side == 1) continue;           // h = 1: only {a,b} can be lost
        const int stop = (a.h < 2) ? rb : re;
        for (int s0 = start; s0 < stop; s0 += 32) {
            const int s = s0 + lane;
            int z = -1;
            unsigned reads = 0;
            if (s < stop) {
                if (s < rb) {
                    z = y;
                } else {
                    const int c = a.col[s];
                    reads += 2;
                    if (c != x) {
                        if (a.col_live[s] >= 0) z = c;
                        else if (a.stamp[a.slot_eid[s]] == round) z = c;
                        reads += (a.col_live[s] >= 0) ? 0 : 2;
                    }
                }
            }
            bool lost = false;
            if (z >= 0) {
                pairs++;
                lost = !within_h(a, x, z, reads);
            }
            reads_total += reads;
            // a pair whose stored bit is clear was handled by an earlier batch of this round
            if (lost && ball_contains(a, x, z, reads)) {
                const int idx = atomicAdd(&st->nlost, 1);  // reserve the record first
                if (idx >= a.lost_max) {
                    atomicMin(&st->overflow_unit, u);       // resume here in the next slot
                } else {
                    const unsigned long long key = pair_key(x, z);
                    unsigned long long slot = mix64(key) & a.cap_mask;
                    int4 rec = make_int4(-1, -1, -1, 0);    // null record: pair already held
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
            }
        }
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

// Support updates for every directed loss (v loses w), one warp per loss, lanes over v's
// alive edges (v,z).  PASS 0 (stored balls still old) handles edges with v < z and tests
// w in B_old(z); PASS 1 (after the clears) handles v > z and tests w in B_new(z).
template <int PASS>
__global__ void __launch_bounds__(kBlock) k_loss_delta(LossArgs a) {
    __shared__ unsigned long long s_tests, s_bytes;
    DevStatus *st = a.st;
    if (st->alive == 0) return;
    if (threadIdx.x == 0) {
        s_tests = 0ull;
        s_bytes = 0ull;
    }
    __syncthreads();
    unsigned long long bytes_total = 0ull;
    const int nlost = min(st->nlost, a.lost_max), round = st->round;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    unsigned long long tests = 0ull;
    for (int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; d < 2 * nlost; d += nwarps) {
        const int4 L = a.lost[d >> 1];
        if (L.x < 0) continue;
        const int v = (d & 1) ? L.y : L.x;
        const int w = (d & 1) ? L.x : L.y;
        const int re = a.row_ptr[v + 1];
        unsigned bytes = (lane == 0) ? 24u : 0u;  // the loss record and v's row bounds
        for (int s = a.row_ptr[v] + lane; s < re; s += 32) {
            const int z = a.col_live[s];
            bytes += 4;
            if (z < 0) continue;
            const int e = a.slot_eid[s];
            bytes += 4;
            if (PASS == 0) a.edge_touch[e] = round;
            if (PASS == 0 ? (v < z) : (v > z)) {
                tests++;
                if (ball_contains(a, z, w, bytes)) {
                    atomicSub(a.sup + e, 1);
                    bytes += 8;
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
__global__ void k_loss_apply(LossArgs a) {
    DevStatus *st = a.st;
    if (st->alive == 0) return;
    const int nlost = min(st->nlost, a.lost_max);
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < 2 * nlost; d += gridDim.x * blockDim.x) {
        const int4 L = a.lost[d >> 1];
        if (L.x < 0) continue;
        const int v = (d & 1) ? L.y : L.x;
        const int w = (d & 1) ? L.x : L.y;
        const int nw = a.ball_nw[v];
        const int64_t off = a.ball_off[v];
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
    a.ball_size = w.ball_size;
    a.keys = w.lost_keys;
    a.lost = w.lost;
    a.sup = w.sup;
    a.edge_touch = w.edge_touch;
    a.st = w.status;
    return a;
}

}  // namespace

// Enqueues the loss detection and the support updates of one incremental round (after
// k_remove, before the min reduction).  ev_mid (nullable) is recorded between the two.
htd_status enqueue_loss_kernels(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t ev_mid,
                                unsigned record_flags) {
    LossArgs a = loss_args(H);
    const int grid = H->num_sms * 8;
    k_loss_detect<<<grid, kBlock, 0, s>>>(a);
    if (ev_mid) cudaEventRecordWithFlags(ev_mid, s, record_flags);
    k_loss_delta<0><<<grid, kBlock, 0, s>>>(a);
    k_loss_apply<<<grid, kBlock, 0, s>>>(a);
    k_loss_delta<1><<<grid, kBlock, 0, s>>>(a);
    *launches += 4;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("enqueue_loss_kernels: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    return HTD_OK;
}

}  // namespace htd
