// htd_batch_block.cu -- the batched decomposition of many small graphs in one persistent
// launch: one block owns one graph at a time and runs every peel round of it inside the
// kernel (Sec. 3 peeling, level-synchronous), then takes the next graph from a queue.
//
// For a graph of L <= kBlockMaxN vertices every closed ball is an L-bit row of W = L/32
// words, kept for every radius r = 1..h (B(x,1) = x plus its alive neighbours) in the
// block's scratch (L2-resident for these sizes).  Balls of radius r are ORs of balls of
// radius r-1:  B(x,r) = OR over z in {x} ∪ N(x) of B(z,r-1),  and
//     sup(e,h) = |B(u,h) ∩ B(v,h)| - 2                                   (Def. 2, Def. 3).
// A round takes the minimum alive support (k = max(k, min + 2)), removes every alive edge
// with sup <= k-2 (t(e) = k), and brings the rest up to date exactly:
//   * candidates C: the vertices within h-1 of a removed edge's endpoint before the round,
//     i.e. the OR of the endpoints' B(.,h-1) rows taken before any row changes (only their
//     balls can lose members: a lost path of at most h edges runs through a removed edge);
//   * the removed edges leave the radius-1 rows; then radius 2..h is recomputed for C, one
//     radius after the other (radius r only reads radius r-1, which is already final);
//   * every alive edge at a vertex whose radius-h ball shrank gets its support recomputed.
// Graphs are taken largest first so that the long ones start early.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kBB = 256;       // threads per block
constexpr int kBBWarps = kBB / 32;

// Reads of the union arrays a block needs for its graph (global ids; the graph's vertices are
// [v0, v0 + L) and its edges [e0, e0 + m) of the union).
struct BlockGraphDesc {
    const int32_t *row_ptr;
    const int32_t *col;
    const int32_t *slot_eid;
    const int32_t *eu;
    const int32_t *ev;
    int32_t *out;       // t(e,h) of the graph's edges, in the union's (canonical) order
    int64_t e0, m;
    int32_t v0, L, h, pad;
};

struct BlockScratch {
    uint32_t *rows;     // h_max x nmax x wmax words per block
    int32_t *sup;       // mmax per block
    int32_t *size;      // nmax per block
    int32_t *flist;     // mmax per block: the round's removed edges
    uint32_t *sets;     // 3 x wmax per block: endpoints E, candidates C, changed CH
    int64_t nmax, wmax, mmax;
    int32_t hmax;
};

__device__ __forceinline__ int bb_block_min(int v, int *s_red) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    int r = INT_MAX;
    for (int j = 0; j < kBBWarps; j++) r = min(r, s_red[j]);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBB) k_batch_block(const BlockGraphDesc *__restrict__ gd, int32_t count,
                                                     BlockScratch sc, int32_t *queue,
                                                     unsigned long long *rounds_total,
                                                     int32_t *err) {
    __shared__ int s_red[kBBWarps];
    __shared__ int s_g, s_k, s_nf;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *rows = sc.rows + (int64_t)blockIdx.x * sc.hmax * sc.nmax * sc.wmax;
    int32_t *sup = sc.sup + (int64_t)blockIdx.x * sc.mmax;
    int32_t *size = sc.size + (int64_t)blockIdx.x * sc.nmax;
    int32_t *flist = sc.flist + (int64_t)blockIdx.x * sc.mmax;
    uint32_t *E = sc.sets + (int64_t)blockIdx.x * 3 * sc.wmax;
    uint32_t *C = E + sc.wmax, *CH = C + sc.wmax;
    for (;;) {
        if (threadIdx.x == 0) s_g = atomicAdd(queue, 1);
        __syncthreads();
        const int gi = s_g;
        __syncthreads();
        if (gi >= count) break;
        const BlockGraphDesc G = gd[gi];
        const int L = G.L, h = G.h, W = (L + 31) >> 5;
        const int64_t m = G.m;
        if (L > sc.nmax || W > sc.wmax || m > sc.mmax || h > sc.hmax || h < 1) {
            if (threadIdx.x == 0) atomicOr(err, 1);
            continue;
        }
        const int32_t *rp = G.row_ptr + G.v0;
        auto row = [&](int r, int x) -> uint32_t * { return rows + ((int64_t)(r - 1) * sc.nmax + x) * sc.wmax; };
        // radius 1: x and its neighbours
        for (int x = wid; x < L; x += kBBWarps) {
            uint32_t *r1 = row(1, x);
            for (int w = lane; w < W; w += 32) r1[w] = 0u;
            __syncwarp();
            if (lane == 0) atomicOr(&r1[x >> 5], 1u << (x & 31));
            for (int s = rp[x] + lane; s < rp[x + 1]; s += 32) {
                const int z = G.col[s] - G.v0;
                atomicOr(&r1[z >> 5], 1u << (z & 31));
            }
        }
        for (int64_t e = threadIdx.x; e < m; e += kBB) sup[e] = 0;
        __syncthreads();
        // radius 2..h for every vertex
        for (int r = 2; r <= h; r++) {
            for (int x = wid; x < L; x += kBBWarps) {
                uint32_t *dst = row(r, x);
                const uint32_t *own = row(r - 1, x);
                for (int w = lane; w < W; w += 32) {
                    uint32_t acc = own[w];
                    for (int s = rp[x]; s < rp[x + 1]; s++) acc |= row(r - 1, G.col[s] - G.v0)[w];
                    dst[w] = acc;
                }
            }
            __syncthreads();
        }
        // sizes and every edge's h-support
        for (int x = wid; x < L; x += kBBWarps) {
            const uint32_t *bh = row(h, x);
            int c = 0;
            for (int w = lane; w < W; w += 32) c += __popc(bh[w]);
            c = warp_sum(c);
            if (lane == 0) size[x] = c;
        }
        for (int64_t e = wid; e < m; e += kBBWarps) {
            const int u = G.eu[G.e0 + e] - G.v0, v = G.ev[G.e0 + e] - G.v0;
            const uint32_t *bu = row(h, u), *bv = row(h, v);
            int c = 0;
            for (int w = lane; w < W; w += 32) c += __popc(bu[w] & bv[w]);
            c = warp_sum(c);
            if (lane == 0) sup[e] = c - 2;
        }
        if (threadIdx.x == 0) s_k = 2;
        __syncthreads();
        int64_t rounds = 0;
        for (int64_t guard = 0; guard <= m; guard++) {
            // level: k = max(k, min alive sup + 2)
            int lmin = INT_MAX;
            for (int64_t e = threadIdx.x; e < m; e += kBB) lmin = min(lmin, sup[e]);
            const int mn = bb_block_min(lmin, s_red);
            if (mn == INT_MAX) break;  // every edge removed
            const int k = max(s_k, mn + 2);
            for (int w = threadIdx.x; w < W; w += kBB) {
                E[w] = 0u;
                C[w] = 0u;
                CH[w] = 0u;
            }
            if (threadIdx.x == 0) s_nf = 0;
            __syncthreads();
            // remove the frontier: every alive edge with sup <= k - 2 (t = k)
            for (int64_t e = threadIdx.x; e < m; e += kBB) {
                if (sup[e] <= k - 2) {
                    const int u = G.eu[G.e0 + e] - G.v0, v = G.ev[G.e0 + e] - G.v0;
                    G.out[e] = k;
                    sup[e] = INT_MAX;
                    flist[atomicAdd(&s_nf, 1)] = (int)e;
                    atomicOr(&E[u >> 5], 1u << (u & 31));
                    atomicOr(&E[v >> 5], 1u << (v & 31));
                }
            }
            __syncthreads();
            const int nf = s_nf;
            // candidates: endpoints (h = 1) or the OR of their radius h-1 rows, before any
            // row changes
            if (h == 1) {
                for (int w = threadIdx.x; w < W; w += kBB) C[w] = E[w];
            } else {
                for (int x = wid; x < L; x += kBBWarps) {
                    if (!((E[x >> 5] >> (x & 31)) & 1u)) continue;
                    const uint32_t *src = row(h - 1, x);
                    for (int w = lane; w < W; w += 32)
                        if (src[w]) atomicOr(&C[w], src[w]);
                }
            }
            __syncthreads();
            // the removed edges leave the radius-1 rows
            for (int i = threadIdx.x; i < nf; i += kBB) {
                const int64_t e = flist[i];
                const int u = G.eu[G.e0 + e] - G.v0, v = G.ev[G.e0 + e] - G.v0;
                atomicAnd(&row(1, u)[v >> 5], ~(1u << (v & 31)));
                atomicAnd(&row(1, v)[u >> 5], ~(1u << (u & 31)));
            }
            __syncthreads();
            // radius 2..h of the candidates, from the already updated radius below
            for (int r = 2; r <= h; r++) {
                for (int x = wid; x < L; x += kBBWarps) {
                    if (!((C[x >> 5] >> (x & 31)) & 1u)) continue;
                    uint32_t *dst = row(r, x);
                    const uint32_t *own = row(r - 1, x);
                    for (int w = lane; w < W; w += 32) {
                        uint32_t acc = own[w];
                        for (int s = rp[x]; s < rp[x + 1]; s++) {
                            const int eid = G.slot_eid[s] - (int)G.e0;
                            if (sup[eid] == INT_MAX) continue;  // removed
                            acc |= row(r - 1, G.col[s] - G.v0)[w];
                        }
                        dst[w] = acc;
                    }
                }
                __syncthreads();
            }
            // vertices whose radius-h ball shrank
            for (int x = wid; x < L; x += kBBWarps) {
                if (!((C[x >> 5] >> (x & 31)) & 1u)) continue;
                const uint32_t *bh = row(h, x);
                int c = 0;
                for (int w = lane; w < W; w += 32) c += __popc(bh[w]);
                c = warp_sum(c);
                if (lane == 0 && c != size[x]) {
                    size[x] = c;
                    atomicOr(&CH[x >> 5], 1u << (x & 31));
                }
            }
            __syncthreads();
            // supports of the alive edges at a changed vertex (both ends may recompute an
            // edge: they write the same value)
            for (int x = wid; x < L; x += kBBWarps) {
                if (!((CH[x >> 5] >> (x & 31)) & 1u)) continue;
                const uint32_t *bx = row(h, x);
                for (int s = rp[x]; s < rp[x + 1]; s++) {
                    const int eid = G.slot_eid[s] - (int)G.e0;
                    if (sup[eid] == INT_MAX) continue;
                    const uint32_t *by = row(h, G.col[s] - G.v0);
                    int c = 0;
                    for (int w = lane; w < W; w += 32) c += __popc(bx[w] & by[w]);
                    c = warp_sum(c);
                    if (lane == 0) sup[eid] = c - 2;
                }
            }
            if (threadIdx.x == 0) s_k = k;
            __syncthreads();
            rounds++;
        }
        if (threadIdx.x == 0) atomicAdd(rounds_total, (unsigned long long)rounds);
        __syncthreads();
    }
}

}  // namespace

// Decomposes the graphs `gd` (host array of count descriptors, device pointers inside) with
// one block per graph in a single launch.  Scratch is sized from the largest graph.
htd_status batch_block_run(const std::vector<BlockGraphDescHost> &graphs, cudaStream_t s,
                           int num_sms, int64_t *rounds_out) {
    if (graphs.empty()) return HTD_OK;
    std::vector<BlockGraphDesc> gd(graphs.size());
    int64_t nmax = 1, mmax = 1;
    int32_t hmax = 1;
    for (size_t i = 0; i < graphs.size(); i++) {
        const BlockGraphDescHost &g = graphs[i];
        gd[i] = BlockGraphDesc{g.row_ptr, g.col, g.slot_eid, g.eu, g.ev, g.out, g.e0, g.m, g.v0, g.L, g.h, 0};
        nmax = std::max<int64_t>(nmax, g.L);
        mmax = std::max<int64_t>(mmax, g.m);
        hmax = std::max(hmax, g.h);
    }
    // largest graphs first
    std::sort(gd.begin(), gd.end(), [](const BlockGraphDesc &a, const BlockGraphDesc &b) {
        return a.m * (int64_t)a.h > b.m * (int64_t)b.h;
    });
    const int64_t wmax = (nmax + 31) / 32;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_block, kBB, 0) != cudaSuccess || occ < 1) {
        set_last_error("batched blocks: no resident block fits");
        return HTD_ECUDA;
    }
    // blocks: enough to keep every SM busy, bounded by the graphs and by the scratch
    const int64_t per_block = (int64_t)hmax * nmax * wmax * 4 + mmax * 8 + nmax * 4 + 3 * wmax * 4;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    int64_t grid = std::min<int64_t>((int64_t)num_sms * std::min(occ, 4), (int64_t)gd.size());
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, (int64_t)(free_b / 2) / std::max<int64_t>(per_block, 1)));
    BlockScratch sc;
    sc.nmax = nmax;
    sc.wmax = wmax;
    sc.mmax = mmax;
    sc.hmax = hmax;
    BlockGraphDesc *d_gd = nullptr;
    int32_t *d_q = nullptr, *d_err = nullptr;
    unsigned long long *d_rounds = nullptr;
    sc.rows = nullptr;
    sc.sup = sc.size = sc.flist = nullptr;
    sc.sets = nullptr;
    htd_status st = HTD_OK;
    cudaError_t e = cudaMalloc(&sc.rows, grid * hmax * nmax * wmax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sc.sup, grid * mmax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sc.flist, grid * mmax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sc.size, grid * nmax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sc.sets, grid * 3 * wmax * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_gd, gd.size() * sizeof(BlockGraphDesc));
    if (e == cudaSuccess) e = cudaMalloc(&d_q, 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_rounds, 8);
    if (e == cudaSuccess) d_err = d_q + 1;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_gd, gd.data(), gd.size() * sizeof(BlockGraphDesc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_q, 0, 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_rounds, 0, 8, s);
    if (e == cudaSuccess) {
        k_batch_block<<<(unsigned)grid, kBB, 0, s>>>(d_gd, (int32_t)gd.size(), sc, d_q, d_rounds, d_err);
        add_launches(1);
        e = cudaGetLastError();
    }
    int32_t herr = 0;
    unsigned long long hr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hr, d_rounds, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string("batched blocks: ") + cudaGetErrorString(e));
        st = e == cudaErrorMemoryAllocation ? HTD_ENOMEM : HTD_ECUDA;
    } else if (herr) {
        set_last_error("batched blocks: a graph exceeded the block scratch (cannot happen)");
        st = HTD_ECUDA;
    }
    if (rounds_out) *rounds_out = (int64_t)hr;
    cudaFree(sc.rows);
    cudaFree(sc.sup);
    cudaFree(sc.flist);
    cudaFree(sc.size);
    cudaFree(sc.sets);
    cudaFree(d_gd);
    cudaFree(d_q);
    cudaFree(d_rounds);
    return st;
}

}  // namespace htd
