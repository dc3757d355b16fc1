// htd_peel.cu -- h-hop balls, h-support and level-synchronous peeling on the device.
//
// Notation (Sec. 2): B(x,h) = x plus every vertex within distance h of x over the alive
// edges, so N(x,h) = B(x,h) \ {x} and, for an alive edge e = (u,v),
//     sup(e,h) = |N(u,h) ∩ N(v,h)| = |B(u,h) ∩ B(v,h)| - 2            (Def. 2, Def. 3)
// because u and v lie in both balls.
//
// Balls are materialised per vertex as n-bit sets, stored either dense (W words) or as a
// sorted list of (word index, word) pairs when that is at most W words; the choice is
// remade at every rebuild and always fits the storage reserved by the first build,
// because balls only shrink as edges are removed.
//
// One peel round (Sec. 3, Algorithm 1 with every edge of level k removed together):
//   select     F = alive edges with sup <= k-2 (k = max(k, min alive sup + 2));
//   candidates vertices within distance h-1 of an endpoint of F, before removal: only
//              their balls can lose members (a lost shortest path of length <= h runs
//              through a removed edge, so its start is within h-1 of that edge);
//   remove     t(e) = k, stamp(e) = round, the edge's two adjacency slots are marked dead;
//   rebuild    every candidate's ball; a ball that shrank marks its vertex "changed";
//   recompute  sup(e) for every alive edge with a changed endpoint (sup depends only on
//              the two balls), owned by one endpoint so each edge is computed once;
//   reduce     min alive sup and alive count; the host polls them between graph launches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "htd_internal.h"
#include "htd_round.cuh"
#include "htd_scan.cuh"

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr int kNWarps = kBlock / 32;
constexpr int kItemChunk = 64;  // adjacency slots per h-support work item

enum BallMode { kModeCount = 0, kModeStore = 1, kModeRebuild = 2 };

struct BallArgs {
    int32_t n, W, Wpad, h;
    int32_t count_bytes;
    int32_t force_dense;  // store every ball dense whatever its size
    const int32_t *row_ptr;
    const int32_t *col_live;
    const int32_t *deg_alive;
    uint32_t *pool;
    const int64_t *ball_off;
    int32_t *ball_need;
    int32_t *ball_size;
    int32_t *ball_nw;
    int2 *ball_meta;
    const int32_t *cand_list;
    int32_t *changed_list;
    int32_t *changed_stamp;
    int32_t *bfs_lists;
    int64_t bfs_list_len;
    DevStatus *st;
};

// Sets bit z of the block's n-bit set; returns true if this thread set it first.
__device__ __forceinline__ bool set_member(uint32_t *bits, int32_t z) {
    const uint32_t m = 1u << (z & 31);
    uint32_t *w = bits + (z >> 5);
    if (*(volatile uint32_t *)w & m) return false;
    return (atomicOr(w, m) & m) == 0u;
}

// Load-balanced expansion of up to kBlock frontier vertices (one per thread, -1 = none):
// every alive neighbour z of them is set in `bits`; if `next` is non-null, vertices set
// for the first time are appended to it.  Consecutive threads read consecutive slots.
__device__ __forceinline__ void expand_chunk(int32_t y, const int32_t *__restrict__ row_ptr,
                                             const int32_t *__restrict__ col_live,
                                             uint32_t *bits, int32_t *s_off, int32_t *s_beg,
                                             int32_t *s_scan, int32_t *next,
                                             int32_t *next_cnt) {
    int beg = 0, len = 0;
    if (y >= 0) {
        beg = row_ptr[y];
        len = row_ptr[y + 1] - beg;
    }
    int total;
    const int off = block_exclusive_scan<kBlock, int>(len, &total, s_scan);
    s_off[threadIdx.x] = off;
    s_beg[threadIdx.x] = beg;
    __syncthreads();
    for (int t = threadIdx.x; t < total; t += kBlock) {
        int lo = 0, hi = kBlock - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int z = col_live[s_beg[lo] + (t - s_off[lo])];
        bool fresh = false;
        if (z >= 0) fresh = set_member(bits, z);
        if (next) warp_append(fresh, z, next_cnt, next);
    }
    __syncthreads();
}

// Builds B(x,h) for a list of vertices, one vertex per block at a time (work queue).
//   kModeCount:   records the storage words the ball needs (first pass);
//   kModeStore:   stores the ball at its reserved offset (second pass);
//   kModeRebuild: rebuilds a peel candidate; stores it and marks x changed iff it shrank.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_ball(BallArgs a) {
    extern __shared__ __align__(16) uint32_t bits[];
    __shared__ int32_t s_scan[kNWarps];
    __shared__ int32_t s_off[kBlock], s_beg[kBlock];
    __shared__ int32_t s_item;
    __shared__ int32_t s_cnt[2];
    __shared__ int32_t s_wsz[kNWarps], s_wnz[kNWarps];
    __shared__ unsigned long long s_bytes;

    DevStatus *st = a.st;
    int count;
    int32_t *queue;
    if (MODE == kModeRebuild) {
        if (st->alive == 0) return;
        count = 0;
        for (int j = 0; j < a.h && j < kMaxH; j++) count += st->cand_cnt[j];
        queue = &st->q_ball;
    } else {
        count = a.n;
        queue = (MODE == kModeCount) ? &st->q_count : &st->q_store;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int W = a.W;
    const int seg = ((W + kNWarps - 1) / kNWarps + 31) & ~31;
    int32_t *lists[2] = {nullptr, nullptr};
    if (a.h >= 3) {
        lists[0] = a.bfs_lists + (int64_t)blockIdx.x * 2 * a.bfs_list_len;
        lists[1] = lists[0] + a.bfs_list_len;
    }
    if (threadIdx.x == 0) s_bytes = 0ull;
    unsigned long long bytes = 0ull;  // per-thread share of the algorithmic bytes

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= count) break;
        const int x = (MODE == kModeRebuild) ? a.cand_list[it] : it;

        uint4 *bits4 = reinterpret_cast<uint4 *>(bits);
        for (int i = threadIdx.x; i < (a.Wpad >> 2); i += kBlock) bits4[i] = make_uint4(0, 0, 0, 0);
        if (threadIdx.x == 0) {
            s_cnt[0] = 0;
            s_cnt[1] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicOr(&bits[x >> 5], 1u << (x & 31));
            if (a.count_bytes && a.h >= 2) bytes += 8ull + 4ull * (unsigned)a.deg_alive[x];
        }
        // depth 1 (x's alive neighbours) and depth 2 (their neighbours)
        const int rb = a.row_ptr[x], re = a.row_ptr[x + 1];
        for (int c = rb; c < re; c += kBlock) {
            const int s = c + threadIdx.x;
            int y = -1;
            if (s < re) {
                y = a.col_live[s];
                if (y < 0) y = -1;
            }
            if (y >= 0) {
                set_member(bits, y);
                if (a.count_bytes && a.h >= 2) bytes += 8ull + 4ull * (unsigned)a.deg_alive[y];
            }
            if (a.h >= 2) {
                expand_chunk(y, a.row_ptr, a.col_live, bits, s_off, s_beg, s_scan,
                             a.h >= 3 ? lists[0] : nullptr, &s_cnt[0]);
            }
        }
        // depth 3..h from the level lists
        for (int d = 3; d <= a.h; d++) {
            const int cur = (d - 3) & 1, nxt = cur ^ 1;
            __syncthreads();
            const int ncur = s_cnt[cur];
            __syncthreads();
            if (threadIdx.x == 0) s_cnt[nxt] = 0;
            __syncthreads();
            for (int c = 0; c < ncur; c += kBlock) {
                const int i = c + threadIdx.x;
                const int y = (i < ncur) ? lists[cur][i] : -1;
                if (a.count_bytes && y >= 0) bytes += 8ull + 4ull * (unsigned)a.deg_alive[y];
                expand_chunk(y, a.row_ptr, a.col_live, bits, s_off, s_beg, s_scan,
                             d < a.h ? lists[nxt] : nullptr, &s_cnt[nxt]);
            }
        }
        __syncthreads();

        // ball size and non-zero words, per warp segment of words
        const int w0 = wid * seg, w1 = min(W, w0 + seg);
        int sz = 0, nz = 0;
        for (int i = w0 + lane; i < w1; i += 32) {
            const uint32_t w = bits[i];
            sz += __popc(w);
            nz += (w != 0u);
        }
        sz = warp_sum(sz);
        nz = warp_sum(nz);
        if (lane == 0) {
            s_wsz[wid] = sz;
            s_wnz[wid] = nz;
        }
        __syncthreads();
        int size = 0, nzw = 0, wbase = 0;
#pragma unroll
        for (int j = 0; j < kNWarps; j++) {
            size += s_wsz[j];
            nzw += s_wnz[j];
            if (j < wid) wbase += s_wnz[j];
        }
        const bool dense = a.force_dense || 2 * nzw > W;
        const int stor = dense ? a.Wpad : ((2 * nzw + 3) & ~3);
        bool store = true;
        if (MODE == kModeCount) {
            if (threadIdx.x == 0) a.ball_need[x] = stor;
            store = false;
        } else if (MODE == kModeRebuild) {
            const int old = a.ball_size[x];
            if (size == old) store = false;
            else if (size > old) {
                if (threadIdx.x == 0) atomicOr(&st->err, kErrBallGrew);
                store = false;
            }
        }
        if (store) {
            const int64_t off = a.ball_off[x];
            const int64_t cap = a.ball_off[x + 1] - off;
            if (stor > cap) {
                if (threadIdx.x == 0) atomicOr(&st->err, kErrBallCapacity);
            } else if (dense) {
                uint4 *dst = reinterpret_cast<uint4 *>(a.pool + off);
                for (int i = threadIdx.x; i < (a.Wpad >> 2); i += kBlock) dst[i] = bits4[i];
            } else {
                uint2 *dst = reinterpret_cast<uint2 *>(a.pool + off);
                int run = wbase;
                for (int i0 = w0; i0 < w1; i0 += 32) {
                    const int i = i0 + lane;
                    const uint32_t w = (i < w1) ? bits[i] : 0u;
                    const unsigned bal = __ballot_sync(0xffffffffu, w != 0u);
                    if (w != 0u) dst[run + __popc(bal & lanemask_lt())] = make_uint2((uint32_t)i, w);
                    run += __popc(bal);
                }
            }
            if (threadIdx.x == 0 && stor <= cap) {
                if (MODE == kModeStore) atomicAdd((unsigned long long *)&st->st_ball_total,
                                                  (unsigned long long)size);
                a.ball_size[x] = size;
                a.ball_nw[x] = dense ? -1 : nzw;
                a.ball_meta[x] = make_int2((int)(off >> 2), dense ? -1 : nzw);
                if (MODE == kModeRebuild) {
                    a.changed_stamp[x] = st->round;
                    a.changed_list[atomicAdd(&st->nchanged, 1)] = x;
                }
            }
        }
        __syncthreads();
    }
    if (a.count_bytes) {
        unsigned long long b = bytes;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0 && b) atomicAdd(&s_bytes, b);
        __syncthreads();
        if (threadIdx.x == 0 && s_bytes) atomicAdd(&st->st_bytes_ball, s_bytes);
    }
}

struct HsupArgs {
    int32_t n, W, Wpad;
    int32_t initial;
    int32_t count_bytes;
    const int32_t *row_ptr;
    const int32_t *col_live;
    const int32_t *slot_eid;
    const uint32_t *pool;
    const int64_t *ball_off;
    const int32_t *ball_size;
    const int32_t *ball_nw;
    const int32_t *changed_stamp;
    const int2 *items;
    int32_t *sup;
    DevStatus *st;
};

// h-support of the edges of each work item (vertex x, run of x's adjacency slots).  The
// block loads B(x,h) into shared memory as a dense set; each warp takes one slot, and if
// x owns the edge it streams the other endpoint's stored ball against it:
//   sup(e) = popc(B(x) & B(y)) - 2.
// Ownership: x owns (x,y) if y's ball did not change this round, else the endpoint with
// the larger stored ball owns it (ties: smaller id).  In the initial pass every ball
// counts as changed, so each edge is computed exactly once.
__global__ void __launch_bounds__(kBlock) k_hsup(HsupArgs a) {
    extern __shared__ __align__(16) uint32_t bits[];
    __shared__ int32_t s_item;
    __shared__ unsigned long long s_bytes;
    __shared__ int32_t s_owned;
    DevStatus *st = a.st;
    if (!a.initial && st->alive == 0) return;
    const int nitems = st->nitems;
    const int round = st->round;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int W = a.W;
    uint4 *bits4 = reinterpret_cast<uint4 *>(bits);
    const uint4 *pool4 = reinterpret_cast<const uint4 *>(a.pool);
    const uint2 *pool2 = reinterpret_cast<const uint2 *>(a.pool);
    if (threadIdx.x == 0) {
        s_bytes = 0ull;
        s_owned = 0;
    }
    unsigned long long bytes = 0ull;
    int owned = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&st->q_items, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 item = a.items[it];
        const int x = item.x;
        const int nwx = a.ball_nw[x];
        const int64_t offx = a.ball_off[x];
        if (nwx < 0) {
            for (int i = threadIdx.x; i < (a.Wpad >> 2); i += kBlock) bits4[i] = pool4[(offx >> 2) + i];
        } else {
            for (int i = threadIdx.x; i < (a.Wpad >> 2); i += kBlock) bits4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            for (int j = threadIdx.x; j < nwx; j += kBlock) {
                const uint2 p = pool2[(offx >> 1) + j];
                bits[p.x] = p.y;
            }
        }
        __syncthreads();
        const int storx = nwx < 0 ? W : 2 * nwx;
        const int s1 = min(a.row_ptr[x + 1], item.y + kItemChunk);
        for (int s = item.y + wid; s < s1; s += kNWarps) {
            const int y = a.col_live[s];
            if (y < 0) continue;
            const bool ychanged = a.initial || a.changed_stamp[y] == round;
            const int nwy = a.ball_nw[y];
            const int story = nwy < 0 ? W : 2 * nwy;
            const bool own = !ychanged || storx > story || (storx == story && x < y);
            if (!own) continue;
            const int64_t offy = a.ball_off[y];
            int cnt = 0;
            if (nwy < 0) {
                const uint4 *p = pool4 + (offy >> 2);
                for (int i = lane; i < (a.Wpad >> 2); i += 32) {
                    const uint4 v = p[i];
                    const uint4 b = bits4[i];
                    cnt += __popc(v.x & b.x) + __popc(v.y & b.y) + __popc(v.z & b.z) +
                           __popc(v.w & b.w);
                }
            } else {
                const uint2 *p = pool2 + (offy >> 1);
                for (int j = lane; j < nwy; j += 32) {
                    const uint2 v = p[j];
                    cnt += __popc(bits[v.x] & v.y);
                }
            }
            cnt = warp_sum(cnt);
            if (lane == 0) {
                a.sup[a.slot_eid[s]] = cnt - 2;
                owned++;
                if (a.count_bytes)
                    bytes += 4ull * (unsigned)(story) + 12ull;
            }
        }
        if (a.count_bytes && threadIdx.x == 0) bytes += 4ull * (unsigned)storx;
        __syncthreads();
    }
    if (lane == 0 && owned) atomicAdd(&s_owned, owned);
    if (a.count_bytes) {
        unsigned long long b = bytes;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (lane == 0 && b) atomicAdd(&s_bytes, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.count_bytes && s_bytes) {
            atomicAdd(&st->st_bytes_hsup, s_bytes);
            if (a.initial) atomicAdd(&st->st_bytes_hsup_init, s_bytes);
        }
        if (!a.initial && s_owned) atomicAdd((unsigned long long *)&st->st_recomputed,
                                             (unsigned long long)s_owned);
    }
}

// Work items for k_hsup: every vertex of `list` (all vertices if list is null) gets one
// item per kItemChunk adjacency slots.  One atomic per warp.
__global__ void k_make_items(const int32_t *__restrict__ list, int32_t initial, int32_t n,
                             const int32_t *__restrict__ row_ptr, int2 *__restrict__ items,
                             DevStatus *st) {
    if (!initial && st->alive == 0) return;
    const int count = list ? st->nchanged : n;
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < count; i0 += stride) {
        const int i = i0 + lane;
        int x = -1, rb = 0, nch = 0;
        if (i < count) {
            x = list ? list[i] : i;
            rb = row_ptr[x];
            nch = (row_ptr[x + 1] - rb + kItemChunk - 1) / kItemChunk;
        }
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && tot) base = atomicAdd(&st->nitems, tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        const int first = base + incl - nch;
        for (int c = 0; c < nch; c++) items[first + c] = make_int2(x, rb + c * kItemChunk);
    }
}

__global__ void k_select(const int32_t *__restrict__ sup, int64_t m, DevStatus *st,
                         int32_t *__restrict__ frontier) {
    if (st->alive == 0 || st->cont) return;  // a continued round keeps its frontier
    const int thr = st->k - 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); e0 < m; e0 += stride) {
        const int64_t e = e0 + (threadIdx.x & 31);
        const bool p = e < m && sup[e] <= thr;
        warp_append(p, (int32_t)e, &st->nF, frontier);
    }
}

__device__ __forceinline__ void cand_mark(bool pred, int32_t w, int round, int level,
                                          int base, int32_t *cand_stamp, int32_t *cand_list,
                                          DevStatus *st) {
    bool fresh = pred && atomicExch(&cand_stamp[w], round) != round;
    warp_append(fresh, w, &st->cand_cnt[level], cand_list + base);
}

// Depth 0 of the candidate search: both endpoints of every frontier edge.
__global__ void k_cand_init(const int32_t *__restrict__ frontier, const int32_t *__restrict__ eu,
                            const int32_t *__restrict__ ev, DevStatus *st,
                            int32_t *__restrict__ cand_stamp, int32_t *__restrict__ cand_list) {
    if (st->alive == 0) return;
    const int nF = st->nF, round = st->round;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < nF; i0 += stride) {
        const int i = i0 + (threadIdx.x & 31);
        const bool p = i < nF;
        const int e = p ? frontier[i] : 0;
        cand_mark(p, p ? eu[e] : 0, round, 0, 0, cand_stamp, cand_list, st);
        cand_mark(p, p ? ev[e] : 0, round, 0, 0, cand_stamp, cand_list, st);
    }
}

// Depth d of the candidate search (alive edges, frontier still present): one warp per
// vertex found at depth d-1.
// with_removed: also follow the slots removed in the current round (the pre-removal graph
// after the round's frontier is already gone: the h = 3 recovery).
__global__ void k_cand_expand(int32_t d, const int32_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col, const int32_t *__restrict__ col_live,
                              int32_t with_removed, DevStatus *st,
                              int32_t *__restrict__ cand_stamp, int32_t *__restrict__ cand_list) {
    if (st->alive == 0) return;
    int start = 0;
    for (int j = 0; j < d - 1; j++) start += st->cand_cnt[j];
    const int len = st->cand_cnt[d - 1];
    const int out_base = start + len;
    const int round = st->round;
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < len; i += nwarps) {
        const int w = cand_list[start + i];
        const int rb = row_ptr[w], re = row_ptr[w + 1];
        for (int s0 = rb; s0 < re; s0 += 32) {
            const int s = s0 + lane;
            int z = (s < re) ? col_live[s] : -1;
            if (with_removed && s < re && z == -(round + 1)) z = col[s];
            cand_mark(z >= 0, z >= 0 ? z : 0, round, d, out_base, cand_stamp, cand_list, st);
        }
    }
}

__global__ void k_remove(const int32_t *__restrict__ frontier, DevStatus *st,
                         const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                         const int32_t *__restrict__ slot_lo, const int32_t *__restrict__ slot_hi,
                         int32_t *__restrict__ sup, int32_t *__restrict__ truss,
                         int32_t *__restrict__ stamp, int32_t *__restrict__ col_live,
                         int32_t *__restrict__ deg_alive, const int32_t *__restrict__ hub_slot,
                         uint32_t *__restrict__ hub_bits, int32_t Wpad) {
    if (st->alive == 0 || st->cont) return;  // a continued round removed its frontier already
    const int nF = st->nF, k = st->k, round = st->round;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nF; i += gridDim.x * blockDim.x)
        remove_edge(frontier[i], k, round, eu, ev, slot_lo, slot_hi, sup, truss, stamp, col_live,
                    deg_alive, hub_slot, hub_bits, Wpad);
}

// Alive-adjacency n-bit sets of the high-degree vertices (all edges alive), block per hub.
__global__ void __launch_bounds__(kBlock) k_hub_init(const int32_t *__restrict__ hub_list, int32_t nhub,
                                                    const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col,
                                                    uint32_t *__restrict__ hub_bits, int32_t Wpad) {
    for (int hb = blockIdx.x; hb < nhub; hb += gridDim.x) {
        uint32_t *bits = hub_bits + (int64_t)hb * Wpad;
        for (int i = threadIdx.x; i < Wpad; i += kBlock) bits[i] = 0u;
        __syncthreads();
        const int x = hub_list[hb];
        for (int s = row_ptr[x] + threadIdx.x; s < row_ptr[x + 1]; s += kBlock) {
            const int y = col[s];
            atomicOr(bits + (y >> 5), 1u << (y & 31));
        }
        __syncthreads();
    }
}

// Minimum alive h-support and alive count; the last block to finish closes the round.
__global__ void __launch_bounds__(kBlock) k_minreduce(const int32_t *__restrict__ sup, int64_t m,
                                                      DevStatus *st, int32_t initial) {
    if (!initial && st->alive == 0) return;
    minreduce_body<kNWarps>(sup, m, st, initial);
}

__global__ void k_init_deg(int32_t n, const int32_t *__restrict__ row_ptr,
                           int32_t *__restrict__ deg_alive) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        deg_alive[x] = row_ptr[x + 1] - row_ptr[x];
}

#define HTD_CHECK(...)                                                              \
    do {                                                                             \
        cudaError_t _e = (__VA_ARGS__);                                                     \
        if (_e != cudaSuccess) {                                                     \
            set_last_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e));      \
            return (_e == cudaErrorMemoryAllocation) ? HTD_ENOMEM : HTD_ECUDA;       \
        }                                                                            \
    } while (0)

template <typename T>
cudaError_t alloc_n(T **p, int64_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), (size_t)(count > 0 ? count : 1) * sizeof(T));
}

BallArgs ball_args(Handle *H) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    BallArgs a;
    a.n = g.n;
    a.W = w.W;
    a.Wpad = w.Wpad;
    a.h = w.h;
    a.count_bytes = 1;
    a.force_dense = w.dense_balls ? 1 : 0;
    a.row_ptr = g.row_ptr;
    a.col_live = w.col_live;
    a.deg_alive = w.deg_alive;
    a.pool = w.pool;
    a.ball_off = w.ball_off;
    a.ball_need = w.ball_need;
    a.ball_size = w.ball_size;
    a.ball_nw = w.ball_nw;
    a.ball_meta = w.ball_meta;
    a.cand_list = w.cand_list;
    a.changed_list = w.changed_list;
    a.changed_stamp = w.changed_stamp;
    a.bfs_lists = w.bfs_lists;
    a.bfs_list_len = w.bfs_list_len;
    a.st = w.status;
    return a;
}

HsupArgs hsup_args(Handle *H, int initial) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    HsupArgs a;
    a.n = g.n;
    a.W = w.W;
    a.Wpad = w.Wpad;
    a.initial = initial;
    a.count_bytes = 1;
    a.row_ptr = g.row_ptr;
    a.col_live = w.col_live;
    a.slot_eid = g.slot_eid;
    a.pool = w.pool;
    a.ball_off = w.ball_off;
    a.ball_size = w.ball_size;
    a.ball_nw = w.ball_nw;
    a.changed_stamp = w.changed_stamp;
    a.items = w.items;
    a.sup = w.sup;
    a.st = w.status;
    return a;
}

}  // namespace

void free_work(PeelWork *w) {
    cudaFree(w->pool);
    cudaFree(w->ball_off);
    cudaFree(w->ball_need);
    cudaFree(w->ball_size);
    cudaFree(w->ball_nw);
    cudaFree(w->ball_meta);
    cudaFree(w->col_live);
    cudaFree(w->deg_alive);
    cudaFree(w->sup);
    cudaFree(w->truss);
    cudaFree(w->stamp);
    cudaFree(w->frontier);
    cudaFree(w->cand_list);
    cudaFree(w->cand_stamp);
    cudaFree(w->changed_list);
    cudaFree(w->changed_stamp);
    cudaFree(w->items);
    cudaFree(w->bfs_lists);
    cudaFree(w->lost_keys);
    cudaFree(w->lost);
    cudaFree(w->edge_touch);
    cudaFree(w->hub_slot);
    cudaFree(w->hub_list);
    cudaFree(w->hub_bits);
    cudaFree(w->pitems);
    cudaFree(w->uitems);
    cudaFree(w->scan_tmp);
    cudaFree(w->pool2);
    cudaFree(w->ball_size2);
    cudaFree(w->ball_nw2);
    cudaFree(w->ball_meta2);
    cudaFree(w->changed_list2);
    cudaFree(w->changed_stamp2);
    cudaFree(w->lost2_keys);
    cudaFree(w->lost2);
    cudaFree(w->c3items);
    cudaFree(w->touch2);
    cudaFree(w->status);
    if (w->status_host) cudaFreeHost(w->status_host);
    *w = PeelWork{};
}

void drop_graphs(Handle *H);
namespace {
htd_status ensure_work_impl(Handle *H, int32_t h, bool incremental, bool tiny_table);
}  // namespace

// The captured round graphs hold the scratch pointers: dropped whenever the scratch goes.
void drop_graphs(Handle *H) {
    if (H->graph_exec) cudaGraphExecDestroy(H->graph_exec);
    if (H->graph_exec_timed) cudaGraphExecDestroy(H->graph_exec_timed);
    H->graph_exec = nullptr;
    H->graph_exec_timed = nullptr;
    H->graph_h = 0;
    H->graph_rounds = 0;
}

// Allocates (or reuses) the scratch of an h-support pass / peel; on failure nothing of it
// is kept (the handle stays usable for a later attempt).
htd_status ensure_work(Handle *H, int32_t h, bool incremental, bool tiny_table) {
    const htd_status st = ensure_work_impl(H, h, incremental, tiny_table);
    if (st != HTD_OK) {
        drop_graphs(H);
        free_work(&H->w);
    }
    return st;
}

namespace {
htd_status ensure_work_impl(Handle *H, int32_t h, bool incremental, bool tiny_table) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    incremental = incremental && h <= 3;
    if (w.status && w.h == h && (!incremental || (w.lost_keys && w.lost_tiny == tiny_table))) {
        w.incremental = incremental;
        w.inc3 = incremental && h == 3;
        return HTD_OK;
    }
    if (w.status) {
        // the per-block BFS lists and the ball storage depend on h: rebuild everything
        drop_graphs(H);
        free_work(&w);
    }
    const int64_t n = g.n, m = g.m;
    w.h = h;
    w.W = (int32_t)((n + 31) / 32);
    if (w.W < 1) w.W = 1;
    w.Wpad = (w.W + 3) & ~3;
    w.smem_ball = (size_t)w.Wpad * 4;
    w.smem_hsup = (size_t)w.Wpad * 4;
    HTD_CHECK(raise_smem_limit((const void *)k_ball<kModeCount>, w.smem_ball));
    HTD_CHECK(raise_smem_limit((const void *)k_ball<kModeStore>, w.smem_ball));
    HTD_CHECK(raise_smem_limit((const void *)k_ball<kModeRebuild>, w.smem_ball));
    HTD_CHECK(raise_smem_limit((const void *)k_hsup, w.smem_hsup));
    int occ_ball = 0, occ_hsup = 0;
    HTD_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ball, k_ball<kModeRebuild>,
                                                            kBlock, w.smem_ball));
    HTD_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_hsup, k_hsup, kBlock,
                                                            w.smem_hsup));
    if (occ_ball < 1 || occ_hsup < 1) {
        set_last_error("htd: an n-bit ball does not fit in shared memory");
        return HTD_EUNSUPPORTED;
    }
    w.grid_ball = H->num_sms * occ_ball;
    w.grid_hsup = H->num_sms * occ_hsup;
    w.grid_edges = H->num_sms * 4;
    HTD_CHECK(alloc_n(&w.ball_off, n + 1));
    HTD_CHECK(alloc_n(&w.ball_need, n));
    HTD_CHECK(alloc_n(&w.ball_size, n));
    HTD_CHECK(alloc_n(&w.ball_nw, n));
    HTD_CHECK(alloc_n(&w.ball_meta, n));
    HTD_CHECK(alloc_n(&w.col_live, 2 * m));
    HTD_CHECK(alloc_n(&w.deg_alive, n));
    HTD_CHECK(alloc_n(&w.sup, m));
    HTD_CHECK(alloc_n(&w.truss, m));
    HTD_CHECK(alloc_n(&w.stamp, m));
    HTD_CHECK(alloc_n(&w.frontier, m));
    HTD_CHECK(alloc_n(&w.cand_list, n));
    HTD_CHECK(alloc_n(&w.cand_stamp, n));
    HTD_CHECK(alloc_n(&w.changed_list, n));
    HTD_CHECK(alloc_n(&w.changed_stamp, n));
    w.items_cap = n + (2 * m + kItemChunk - 1) / kItemChunk + 1;
    HTD_CHECK(alloc_n(&w.items, w.items_cap));
    if (h >= 3) {
        w.bfs_list_len = n > 0 ? n : 1;
        HTD_CHECK(alloc_n(&w.bfs_lists, (int64_t)w.grid_ball * 2 * w.bfs_list_len));
    }
    if (incremental) {
        // a round's lost pairs: half of a power-of-two table of 8 x (2m) slots (>= 2^12)
        // sized to stay L2-resident (at most 2^22 slots, 32 MiB); larger rounds run in batches
        // h = 3 rounds lose many more radius-3 pairs: a table up to 2^24 slots
        const int64_t cap_max = (int64_t)1 << (h == 3 ? 24 : 22);
        int64_t cap = 4096;
        while (cap < 4 * m * (h == 3 ? 4 : 1) && cap < cap_max) cap <<= 1;
        if (tiny_table) cap = 128;  // forces rounds to run in many batches
        w.lost_tiny = tiny_table;
        w.lost_cap = cap;
        w.lost_max = cap / 2;
        HTD_CHECK(alloc_n(&w.lost_keys, cap));
        HTD_CHECK(alloc_n(&w.lost, w.lost_max));
        HTD_CHECK(alloc_n(&w.edge_touch, n));
        // work items of the loss detection and of the support updates (per batch)
        // (sized with the graph: 2m adjacency slots)
        w.pitems_cap = std::min<int64_t>((int64_t)1 << 22, std::max<int64_t>(4096, 2 * m));
        // adjacency slots the updates of one batch may visit
        w.upd_budget = std::min<int64_t>((int64_t)1 << 30, std::max<int64_t>(1 << 16, 256 * m));
        w.uitems_cap = 2 * w.lost_max + w.upd_budget / 32 + 1024;
        HTD_CHECK(alloc_n(&w.pitems, w.pitems_cap));
        HTD_CHECK(alloc_n(&w.uitems, w.uitems_cap));
        if (h == 3) {
            // radius-2 balls (dense) with their own metadata, the round's radius-2 losses and
            // the radius-3 candidate items
            HTD_CHECK(alloc_n(&w.pool2, n * (int64_t)w.Wpad));
            HTD_CHECK(alloc_n(&w.ball_size2, n));
            HTD_CHECK(alloc_n(&w.ball_nw2, n));
            HTD_CHECK(alloc_n(&w.ball_meta2, n));
            HTD_CHECK(alloc_n(&w.changed_list2, n));
            HTD_CHECK(alloc_n(&w.changed_stamp2, n));
            HTD_CHECK(alloc_n(&w.touch2, n));
            int64_t cap2 = 4096;
            while (cap2 < 4 * m && cap2 < ((int64_t)1 << 22)) cap2 <<= 1;
            if (tiny_table) cap2 = 128;
            w.lost2_cap = cap2;
            w.lost2_max = cap2 / 2;
            HTD_CHECK(alloc_n(&w.lost2_keys, cap2));
            HTD_CHECK(alloc_n(&w.lost2, w.lost2_max));
            w.c3items_cap = tiny_table ? 256
                                       : std::min<int64_t>((int64_t)1 << 25, std::max<int64_t>(1 << 16, 8 * m));
            HTD_CHECK(alloc_n(&w.c3items, w.c3items_cap));
        }
        // alive-adjacency n-bit sets: every vertex of degree >= T, the smallest power of two
        // for which they fit in min(16 GiB, a quarter of the free device memory)
        std::vector<int32_t> rp(n + 1);
        HTD_CHECK(cudaMemcpy(rp.data(), g.row_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        size_t free_b = 0, total_b = 0;
        HTD_CHECK(cudaMemGetInfo(&free_b, &total_b));
        const int64_t budget_words = std::min<int64_t>((int64_t)1 << 32, (int64_t)(free_b / 16));
        int32_t T = 1;
        int64_t cnt = 0;
        for (;; T *= 2) {
            cnt = 0;
            for (int64_t x = 0; x < n; x++) cnt += (rp[x + 1] - rp[x] >= T);
            if (cnt * w.Wpad <= budget_words || T > (1 << 24)) break;
        }
        std::vector<int32_t> slot(n > 0 ? n : 1, -1), list;
        // T = 1: every vertex gets a set (isolated ones too), so set x sits at row x
        for (int64_t x = 0; x < n; x++)
            if (T == 1 || rp[x + 1] - rp[x] >= T) {
                slot[x] = (int32_t)list.size();
                list.push_back((int32_t)x);
            }
        w.nhub = (int32_t)list.size();
        w.hub_min_deg = T;
        HTD_CHECK(alloc_n(&w.hub_slot, n));
        HTD_CHECK(cudaMemcpy(w.hub_slot, slot.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        if (w.nhub > 0) {
            HTD_CHECK(alloc_n(&w.hub_list, w.nhub));
            HTD_CHECK(cudaMemcpy(w.hub_list, list.data(), w.nhub * sizeof(int32_t),
                                 cudaMemcpyHostToDevice));
            HTD_CHECK(alloc_n(&w.hub_bits, (int64_t)w.nhub * w.Wpad));
        }
    }
    w.incremental = incremental;
    w.inc3 = incremental && h == 3;
    HTD_CHECK(cudaMalloc(&w.scan_tmp, scan_temp_bytes(n + 1)));
    HTD_CHECK(alloc_n(&w.status, 1));
    HTD_CHECK(cudaMallocHost(reinterpret_cast<void **>(&w.status_host), sizeof(DevStatus)));
    return HTD_OK;
}

}  // namespace

// Initial pass: every vertex's ball (count, reserve, store) and every edge's h-support,
// then the first min reduction.  Leaves the status ready for round 0.
htd_status initial_pass(Handle *H, int32_t h, cudaStream_t s, int64_t *launches,
                        htd_stats *timing) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    const int64_t n = g.n, m = g.m;
    (void)h;
    std::memset(w.status_host, 0, sizeof(DevStatus));
    w.status_host->k = 2;
    w.status_host->min_acc = INT_MAX;
    w.status_host->overflow_unit = INT_MAX;
    HTD_CHECK(cudaMemcpyAsync(w.status, w.status_host, sizeof(DevStatus), cudaMemcpyHostToDevice, s));
    if (m > 0)
        HTD_CHECK(cudaMemcpyAsync(w.col_live, g.col, 2 * m * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, s));
    HTD_CHECK(cudaMemsetAsync(w.cand_stamp, 0xff, (n > 0 ? n : 1) * sizeof(int32_t), s));
    HTD_CHECK(cudaMemsetAsync(w.changed_stamp, 0xff, (n > 0 ? n : 1) * sizeof(int32_t), s));
    HTD_CHECK(cudaMemsetAsync(w.stamp, 0xff, (m > 0 ? m : 1) * sizeof(int32_t), s));
    if (w.incremental) {
        HTD_CHECK(cudaMemsetAsync(w.edge_touch, 0xff, (n > 0 ? n : 1) * sizeof(int32_t), s));
        HTD_CHECK(cudaMemsetAsync(w.lost_keys, 0xff, w.lost_cap * sizeof(unsigned long long), s));
        if (w.inc3) {
            HTD_CHECK(cudaMemsetAsync(w.lost2_keys, 0xff, w.lost2_cap * sizeof(unsigned long long), s));
            HTD_CHECK(cudaMemsetAsync(w.changed_stamp2, 0xff, (n > 0 ? n : 1) * sizeof(int32_t), s));
            HTD_CHECK(cudaMemsetAsync(w.touch2, 0xff, (n > 0 ? n : 1) * sizeof(int32_t), s));
        }
        if (w.nhub > 0) {
            k_hub_init<<<std::min(w.nhub, H->num_sms * 8), kBlock, 0, s>>>(w.hub_list, w.nhub, g.row_ptr,
                                                                        g.col, w.hub_bits, w.Wpad);
            (*launches)++;
        }
    }
    if (n > 0) {
        k_init_deg<<<std::min<int64_t>((n + kBlock - 1) / kBlock, H->num_sms * 8), kBlock, 0, s>>>(
            (int32_t)n, g.row_ptr, w.deg_alive);
        (*launches)++;
    }
    BallArgs ba = ball_args(H);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
    if (timing) {
        HTD_CHECK(cudaEventCreate(&e0));
        HTD_CHECK(cudaEventCreate(&e1));
        HTD_CHECK(cudaEventCreate(&e2));
        HTD_CHECK(cudaEventCreate(&e3));
    }
    if (n > 0) {
        k_ball<kModeCount><<<w.grid_ball, kBlock, w.smem_ball, s>>>(ba);
        (*launches)++;
        HTD_CHECK(cudaGetLastError());
        HTD_CHECK(scan_exclusive<int32_t, int64_t>(w.ball_need, w.ball_off, n, w.scan_tmp, s, launches));
        int64_t total = 0;
        HTD_CHECK(cudaMemcpyAsync(&total, w.ball_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HTD_CHECK(cudaStreamSynchronize(s));
        if (total >= ((int64_t)1 << 33)) {
            set_last_error("htd: h-hop balls need more than 32 GiB of storage");
            return HTD_EUNSUPPORTED;
        }
        if (total > w.pool_words) {
            cudaFree(w.pool);
            w.pool = nullptr;
            w.pool_words = 0;
            HTD_CHECK(alloc_n(&w.pool, total));
            w.pool_words = total;
            if (H->graph_exec) {  // the captured rounds hold the old pool pointer
                cudaGraphExecDestroy(H->graph_exec);
                H->graph_exec = nullptr;
            }
            if (H->graph_exec_timed) {
                cudaGraphExecDestroy(H->graph_exec_timed);
                H->graph_exec_timed = nullptr;
            }
        }
        ba.pool = w.pool;
        w.pool_used = total;
        if (timing) HTD_CHECK(cudaEventRecord(e0, s));
        k_ball<kModeStore><<<w.grid_ball, kBlock, w.smem_ball, s>>>(ba);
        if (timing) HTD_CHECK(cudaEventRecord(e1, s));
        (*launches)++;
        HTD_CHECK(cudaGetLastError());
        k_make_items<<<std::min<int64_t>((n + kBlock - 1) / kBlock, H->num_sms * 8), kBlock, 0, s>>>(
            nullptr, 1, (int32_t)n, g.row_ptr, w.items, w.status);
        (*launches)++;
        HsupArgs ha = hsup_args(H, 1);
        if (timing) HTD_CHECK(cudaEventRecord(e2, s));
        k_hsup<<<w.grid_hsup, kBlock, w.smem_hsup, s>>>(ha);
        if (timing) HTD_CHECK(cudaEventRecord(e3, s));
        (*launches)++;
        HTD_CHECK(cudaGetLastError());
    }
    k_minreduce<<<w.grid_edges, kBlock, 0, s>>>(w.sup, m, w.status, 1);
    (*launches)++;
    HTD_CHECK(cudaGetLastError());
    if (timing) {
        HTD_CHECK(cudaStreamSynchronize(s));
        float a = 0.f, b = 0.f;
        if (n > 0) {
            HTD_CHECK(cudaEventElapsedTime(&a, e0, e1));
            HTD_CHECK(cudaEventElapsedTime(&b, e2, e3));
            timing->ms_initial_ball += a;
            timing->ms_initial_hsup += b;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        cudaEventDestroy(e3);
    }
    return HTD_OK;
}

// Enqueues one peel round.  evs (nullable) = kRoundEvents events at the phase boundaries:
//   rebuild:     | select | candidates | remove | ball rebuild | items + h-support | reduce |
//   incremental: | select | remove | loss detection | support updates | (empty) | reduce |
htd_status enqueue_round(Handle *H, cudaStream_t s, int64_t *launches, cudaEvent_t *evs) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    const int64_t m = g.m;
    const int gsmall = H->num_sms * 4;
    // inside a stream capture an ordinary record only orders nodes; an external record
    // node really records the event each time the graph runs, so it can be timed
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (evs) HTD_CHECK(cudaStreamIsCapturing(s, &cap));
    const unsigned rec_flags = (cap == cudaStreamCaptureStatusActive) ? cudaEventRecordExternal : 0u;
    auto mark = [&](int i) {
        if (evs) cudaEventRecordWithFlags(evs[i], s, rec_flags);
    };
    if (w.incremental) return enqueue_incremental_round(H, s, launches, evs, rec_flags);
    mark(0);
    k_select<<<w.grid_edges, kBlock, 0, s>>>(w.sup, m, w.status, w.frontier);
    mark(1);
    k_cand_init<<<gsmall, kBlock, 0, s>>>(w.frontier, g.eu, g.ev, w.status, w.cand_stamp, w.cand_list);
    *launches += 2;
    for (int d = 1; d < w.h; d++) {
        k_cand_expand<<<gsmall * 2, kBlock, 0, s>>>(d, g.row_ptr, g.col, w.col_live, 0, w.status,
                                                     w.cand_stamp, w.cand_list);
        (*launches)++;
    }
    mark(2);
    k_remove<<<gsmall, kBlock, 0, s>>>(w.frontier, w.status, g.eu, g.ev, g.slot_lo, g.slot_hi,
                                       w.sup, w.truss, w.stamp, w.col_live, w.deg_alive, nullptr,
                                       nullptr, 0);
    (*launches)++;
    mark(3);
    BallArgs ba = ball_args(H);
    k_ball<kModeRebuild><<<w.grid_ball, kBlock, w.smem_ball, s>>>(ba);
    mark(4);
    k_make_items<<<gsmall, kBlock, 0, s>>>(w.changed_list, 0, g.n, g.row_ptr, w.items, w.status);
    HsupArgs ha = hsup_args(H, 0);
    k_hsup<<<w.grid_hsup, kBlock, w.smem_hsup, s>>>(ha);
    mark(5);
    k_minreduce<<<w.grid_edges, kBlock, 0, s>>>(w.sup, m, w.status, 0);
    mark(6);
    *launches += 4;
    HTD_CHECK(cudaGetLastError());
    return HTD_OK;
}

// Radius-2 balls of every vertex for the incremental h = 3 peel, stored dense in pool2
// with their own sizes (the radius-3 balls and supports come from initial_pass).
htd_status initial_pass_r2(Handle *H, cudaStream_t s, int64_t *launches) {
    PeelWork &w = H->w;
    if (!w.inc3 || H->g.n == 0) return HTD_OK;
    BallArgs b2 = ball_args(H);
    b2.h = 2;
    b2.count_bytes = 0;
    b2.force_dense = 1;
    b2.pool = w.pool2;
    b2.ball_size = w.ball_size2;
    b2.ball_nw = w.ball_nw2;
    b2.ball_meta = w.ball_meta2;
    b2.changed_list = w.changed_list2;
    b2.changed_stamp = w.changed_stamp2;
    b2.bfs_lists = nullptr;
    HTD_CHECK(cudaMemsetAsync(&w.status->q_store, 0, sizeof(int32_t), s));
    k_ball<kModeStore><<<w.grid_ball, kBlock, w.smem_ball, s>>>(b2);
    (*launches)++;
    HTD_CHECK(cudaGetLastError());
    return HTD_OK;
}

namespace {

// Clears what a halted h = 3 round recorded (its pair sets are emptied by the caller) and
// the queue heads the rebuild kernels use.
__global__ void k_recover_reset(DevStatus *st) {
    st->halt = 0;
    st->nlost = 0;
    st->nlost2 = 0;
    st->npitems = 0;
    st->nuitems = 0;
    st->nc3items = 0;
    st->upd_work = 0;
    st->overflow_unit = INT_MAX;
    for (int j = 0; j < kMaxH; j++) st->cand_cnt[j] = 0;
    st->q_ball = 0;
    st->nchanged = 0;
    st->nitems = 0;
    st->q_items = 0;
    st->st_recovered++;
}

__global__ void k_reset_rebuild_queue(DevStatus *st) {
    st->q_ball = 0;
    st->nchanged = 0;
}

}  // namespace

// Finishes a halted round of the incremental h = 3 peel.  Its frontier is already removed
// (slots marked with the round) and nothing else of the round was applied: balls and
// supports are those of before the round.  Every vertex within distance 2 of a frontier
// endpoint in the pre-removal graph is a candidate: its radius-2 ball (if within distance
// 1) and its radius-3 ball are rebuilt, and the supports of the alive edges at vertices
// whose radius-3 ball shrank are recomputed; the min reduction then closes the round.
htd_status recover_round_h3(Handle *H, cudaStream_t s, int64_t *launches) {
    PeelWork &w = H->w;
    GraphDev &g = H->g;
    const int gsmall = H->num_sms * 4;
    HTD_CHECK(cudaMemsetAsync(w.lost_keys, 0xff, w.lost_cap * sizeof(unsigned long long), s));
    HTD_CHECK(cudaMemsetAsync(w.lost2_keys, 0xff, w.lost2_cap * sizeof(unsigned long long), s));
    k_recover_reset<<<1, 1, 0, s>>>(w.status);
    k_cand_init<<<gsmall, kBlock, 0, s>>>(w.frontier, g.eu, g.ev, w.status, w.cand_stamp, w.cand_list);
    *launches += 2;
    for (int d = 1; d < 3; d++) {
        k_cand_expand<<<gsmall * 2, kBlock, 0, s>>>(d, g.row_ptr, g.col, w.col_live, 1, w.status,
                                                     w.cand_stamp, w.cand_list);
        (*launches)++;
    }
    // radius 2: candidates of depth 0..1 (the rebuild counts the first h levels)
    BallArgs b2 = ball_args(H);
    b2.h = 2;
    b2.count_bytes = 0;
    b2.force_dense = 1;
    b2.pool = w.pool2;
    b2.ball_size = w.ball_size2;
    b2.ball_nw = w.ball_nw2;
    b2.ball_meta = w.ball_meta2;
    b2.changed_list = w.changed_list2;
    b2.changed_stamp = w.changed_stamp2;
    b2.bfs_lists = nullptr;
    k_ball<kModeRebuild><<<w.grid_ball, kBlock, w.smem_ball, s>>>(b2);
    k_reset_rebuild_queue<<<1, 1, 0, s>>>(w.status);
    // radius 3 and the supports it changes
    BallArgs b3 = ball_args(H);
    k_ball<kModeRebuild><<<w.grid_ball, kBlock, w.smem_ball, s>>>(b3);
    k_make_items<<<gsmall, kBlock, 0, s>>>(w.changed_list, 0, g.n, g.row_ptr, w.items, w.status);
    HsupArgs ha = hsup_args(H, 0);
    k_hsup<<<w.grid_hsup, kBlock, w.smem_hsup, s>>>(ha);
    k_minreduce<<<w.grid_edges, kBlock, 0, s>>>(w.sup, g.m, w.status, 0);
    *launches += 6;
    HTD_CHECK(cudaGetLastError());
    return HTD_OK;
}

}  // namespace htd
