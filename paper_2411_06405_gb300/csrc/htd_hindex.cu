// htd_hindex.cu -- the paper's own parallel method on the device: the higher-order H-index
// iteration of Sec. 4 (Definition of the h-hop reachable path key, Theorems 3 and 4,
// Algorithm 2, asynchronous updating).
//
// With H^(0)(e) = sup_G(e,h), order n computes for every edge e = (u,v)
//     H^(n)(e) = H({ min(P(u,w), P(v,w)) : w in N_G(u,h) ∩ N_G(v,h) }),
// where H(S) is the largest y such that at least y members of S are >= y, and P(a,b), the
// h-hop reachable path key, is the largest over paths from a to b of at most h edges of
// the smallest H^(n-1) on the path.  The iteration stops at the first order that changes
// nothing, and then t(e,h) = H(e) + 2 (Theorem 4).  Readings (as in the oracle): paths have
// at most h edges and may use e itself; the common h-neighbourhood is that of the whole
// graph G, which never changes.
//
// GPU form.  The graph is fixed, so every vertex's closed ball B(x,h) is built once, as a
// sorted member list.  An order is two kernels:
//   k_hx_pathkeys  one block per vertex x: P(x, .) over the members of B(x,h) by h rounds
//                  of hop-limited relaxation (round r extends paths of at most r-1 edges by
//                  one edge; a member is found in the sorted list by binary search);
//   k_hx_edges     one warp per edge: the common members of the two sorted lists (u and v
//                  excluded), their values min(P(u,w), P(v,w)) gathered in a per-warp
//                  buffer, and H(.) by a binary search on y of the monotone test
//                  "at least y values >= y".
// Synchronous orders (Algorithm 2) write the new keys to a second array.  With pruning
// (Lemma 4), from the second order on an edge keeps its key without being computed when no
// edge near it fell across that key in the previous order: per vertex, the range of the
// fallen edges' values (lowest new, highest old) is spread h-1 hops, and an edge whose two
// endpoints' ranges do not straddle its key is skipped (the range hull is a conservative
// form of the lemma's per-edge conditions, so the result is unchanged); path keys are then
// computed only at the endpoints of the edges still listed.  The asynchronous
// form splits every sweep into S sub-sweeps over consecutive edge-id ranges: a sub-sweep
// recomputes the path keys of the vertices its edges touch from the current keys and
// writes its edges' keys in place, so later sub-sweeps already use them (the paper's
// asynchronous updating, by blocks of edges).  Keys never increase, so both forms reach
// the same fixed point.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "htd_internal.h"
#include "htd_scan.cuh"

namespace htd {
namespace {

constexpr int kBlock = 256;

// BFS of one block from x to depth h over all edges into the block's n-bit set; lists are
// the block's two level lists (n entries each).
__device__ void hx_bfs(int32_t x, int32_t h, const int32_t *__restrict__ row_ptr,
                       const int32_t *__restrict__ col, uint32_t *bits, int32_t W, int32_t *l0,
                       int32_t *l1, int32_t *s_cnt) {
    for (int i = threadIdx.x; i < W; i += blockDim.x) bits[i] = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        bits[x >> 5] |= 1u << (x & 31);
        l0[0] = x;
        s_cnt[0] = 1;
        s_cnt[1] = 0;
    }
    __syncthreads();
    int32_t *cur = l0, *nxt = l1;
    for (int d = 1; d <= h; d++) {
        const int ncur = s_cnt[(d - 1) & 1];
        if (ncur == 0) break;
        for (int i = threadIdx.x; i < ncur; i += blockDim.x) {
            const int y = cur[i];
            for (int s = row_ptr[y]; s < row_ptr[y + 1]; s++) {
                const int z = col[s];
                const uint32_t m = 1u << (z & 31);
                if (*(volatile uint32_t *)&bits[z >> 5] & m) continue;
                if ((atomicOr(&bits[z >> 5], m) & m) == 0u && d < h) nxt[atomicAdd(&s_cnt[d & 1], 1)] = z;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cnt[(d + 1) & 1] = 0;
        __syncthreads();
        int32_t *t = cur;
        cur = nxt;
        nxt = t;
    }
}

// Ball sizes (MODE 0) or sorted member lists (MODE 1) of every vertex, block per vertex.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_hx_balls(int32_t n, int32_t h, const int32_t *__restrict__ row_ptr,
                                                    const int32_t *__restrict__ col, int32_t W,
                                                    int32_t *lists, int32_t *sizes,
                                                    const int64_t *__restrict__ off,
                                                    int32_t *__restrict__ members) {
    extern __shared__ __align__(16) uint32_t bits[];
    __shared__ int32_t s_cnt[2];
    __shared__ int32_t s_scan[kBlock / 32];
    int32_t *l0 = lists + (int64_t)blockIdx.x * 2 * n;
    int32_t *l1 = l0 + n;
    for (int x = blockIdx.x; x < n; x += gridDim.x) {
        hx_bfs(x, h, row_ptr, col, bits, W, l0, l1, s_cnt);
        if (MODE == 0) {
            int c = 0;
            for (int i = threadIdx.x; i < W; i += blockDim.x) c += __popc(bits[i]);
            const int tot = block_sum<kBlock, int>(c, s_scan);
            if (threadIdx.x == 0) sizes[x] = tot;
        } else {
            // members in increasing order: words in chunks of one per thread
            int64_t base = off[x];
            for (int w0 = 0; w0 < W; w0 += kBlock) {
                const int w = w0 + threadIdx.x;
                uint32_t v = w < W ? bits[w] : 0u;
                int tot;
                const int ex = block_exclusive_scan<kBlock, int>(__popc(v), &tot, s_scan);
                int k = 0;
                while (v) {
                    const int b = __ffs(v) - 1;
                    v &= v - 1u;
                    members[base + ex + k] = (w << 5) + b;
                    k++;
                }
                base += tot;
            }
        }
        __syncthreads();
    }
}

// Index of z in the sorted list m[0..len), or -1.
__device__ __forceinline__ int find_member(const int32_t *__restrict__ m, int len, int z) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int v = m[mid];
        if (v == z) return mid;
        if (v < z) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// P(x, .) for the vertices of `list` (all vertices if null), block per vertex.  `prev` is
// the block's scratch of maxb entries (the values of the previous round).
__global__ void __launch_bounds__(kBlock) k_hx_pathkeys(const int32_t *__restrict__ list, int32_t count,
                                                       int32_t h, const int32_t *__restrict__ row_ptr,
                                                       const int32_t *__restrict__ col,
                                                       const int32_t *__restrict__ slot_eid,
                                                       const int32_t *__restrict__ key,
                                                       const int64_t *__restrict__ off,
                                                       const int32_t *__restrict__ members,
                                                       int32_t *__restrict__ P, int32_t *prev_all,
                                                       int64_t maxb) {
    int32_t *prev = prev_all + (int64_t)blockIdx.x * maxb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = blockIdx.x; i < count; i += gridDim.x) {
        const int x = list ? list[i] : i;
        const int64_t o = off[x];
        const int len = (int)(off[x + 1] - o);
        const int32_t *m = members + o;
        int32_t *p = P + o;
        for (int j = threadIdx.x; j < len; j += blockDim.x) p[j] = (m[j] == x) ? INT_MAX : -1;
        __syncthreads();
        for (int r = 1; r <= h; r++) {
            for (int j = threadIdx.x; j < len; j += blockDim.x) prev[j] = p[j];
            __syncthreads();
            // one warp per member reached within r-1 edges; its lanes walk the row
            for (int j = wid; j < len; j += nw) {
                const int pv = prev[j];
                if (pv < 0) continue;
                const int y = m[j];
                for (int s = row_ptr[y] + lane; s < row_ptr[y + 1]; s += 32) {
                    const int z = col[s];
                    const int iz = find_member(m, len, z);
                    if (iz < 0) continue;
                    const int c = min(pv, key[slot_eid[s]]);
                    if (c > p[iz]) atomicMax(&p[iz], c);
                }
            }
            __syncthreads();
        }
    }
}

// New keys of the edges [e0, e1) (of elist[e0..e1) when elist is not null), one warp per
// edge.  vals: the warp's buffer of maxd.
__global__ void __launch_bounds__(kBlock) k_hx_edges(int64_t e0, int64_t e1, const int32_t *__restrict__ elist,
                                                    const int32_t *__restrict__ eu,
                                                    const int32_t *__restrict__ ev,
                                                    const int64_t *__restrict__ off,
                                                    const int32_t *__restrict__ members,
                                                    const int32_t *__restrict__ P,
                                                    const int32_t *key_in, int32_t *key_out,
                                                    int32_t *vals_all, int64_t maxd,
                                                    unsigned long long *changed) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t *vals = vals_all + gw * maxd;
    unsigned long long nchg = 0;
    for (int64_t i = e0 + gw; i < e1; i += nwarps) {
        const int64_t e = elist ? elist[i] : i;
        int u = eu[e], v = ev[e];
        int64_t ou = off[u], ov = off[v];
        int lu = (int)(off[u + 1] - ou), lv = (int)(off[v + 1] - ov);
        if (lu > lv) {  // walk the shorter list, search the longer one
            const int t = u; u = v; v = t;
            const int64_t to = ou; ou = ov; ov = to;
            const int tl = lu; lu = lv; lv = tl;
        }
        const int32_t *mu = members + ou, *mv = members + ov;
        int cnt = 0;
        for (int j0 = 0; j0 < lu; j0 += 32) {
            const int j = j0 + lane;
            int val = -1;
            if (j < lu) {
                const int w = mu[j];
                if (w != u && w != v) {
                    const int iv = find_member(mv, lv, w);
                    if (iv >= 0) val = min(P[ou + j], P[ov + iv]);
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, val >= 0);
            if (val >= 0) vals[cnt + __popc(b & ((1u << lane) - 1u))] = val;
            cnt += __popc(b);
        }
        __syncwarp();
        // H = largest y in [0, cnt] with at least y values >= y (the test is monotone in y)
        int lo = 0, hi = cnt + 1;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            int c = 0;
            for (int j = lane; j < cnt; j += 32) c += vals[j] >= mid;
            c = warp_sum(c);
            if (c >= mid) lo = mid;
            else hi = mid;
        }
        if (lane == 0) {
            if (lo != key_in[e]) nchg++;
            key_out[e] = lo;
        }
        __syncwarp();
    }
    if (lane == 0 && nchg) atomicAdd(changed, nchg);
}

// Vertices touched by the edges [e0, e1) (both endpoints), each listed once.
__global__ void k_hx_touch(int64_t e0, int64_t e1, const int32_t *__restrict__ eu,
                           const int32_t *__restrict__ ev, int32_t stamp, int32_t *mark,
                           int32_t *list, int32_t *count) {
    for (int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < e1 + 0; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = eu[i], b = ev[i];
        if (atomicExch(&mark[a], stamp) != stamp) list[atomicAdd(count, 1)] = a;
        if (atomicExch(&mark[b], stamp) != stamp) list[atomicAdd(count, 1)] = b;
    }
}

// Pruning, step 1: per vertex, the range of the values that fell at its edges in the
// previous order: hi = largest H^(n-2), lo = smallest H^(n-1) over its edges that changed.
__global__ void k_hx_fall(int64_t m, const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                          const int32_t *__restrict__ kold, const int32_t *__restrict__ kcur,
                          int32_t *hi, int32_t *lo) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = kold[e], b = kcur[e];
        if (a == b) continue;
        atomicMax(&hi[eu[e]], a);
        atomicMin(&lo[eu[e]], b);
        atomicMax(&hi[ev[e]], a);
        atomicMin(&lo[ev[e]], b);
    }
}

// Pruning, step 2 (h-1 times): one hop of spreading, warp per vertex: the range of x
// becomes the hull of the ranges of x and its neighbours.
__global__ void __launch_bounds__(kBlock) k_hx_spread(int32_t n, const int32_t *__restrict__ row_ptr,
                                                     const int32_t *__restrict__ col,
                                                     const int32_t *__restrict__ hi_in,
                                                     const int32_t *__restrict__ lo_in,
                                                     int32_t *__restrict__ hi_out, int32_t *__restrict__ lo_out) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = gw; x < n; x += nwarps) {
        int h = lane == 0 ? hi_in[x] : -1, l = lane == 0 ? lo_in[x] : INT_MAX;
        for (int s = row_ptr[x] + lane; s < row_ptr[x + 1]; s += 32) {
            const int y = col[s];
            h = max(h, hi_in[y]);
            l = min(l, lo_in[y]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
        }
        if (lane == 0) {
            hi_out[x] = h;
            lo_out[x] = l;
        }
    }
}

// Pruning, step 3: an edge e = (u,v) with T = H^(n-1)(e) is listed for computation when
// the hull [min(lo(u), lo(v)), max(hi(u), hi(v))] of the fallen values near it straddles
// T (some value went from >= T to < T); otherwise H^(n)(e) = T (Lemma 4).  The endpoints of
// listed edges are listed once each (mark holds the stamp of the order that listed them).
__global__ void k_hx_select(int64_t m, const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                            const int32_t *__restrict__ kcur, const int32_t *__restrict__ hi,
                            const int32_t *__restrict__ lo, int32_t *knew, int32_t *elist,
                            int32_t *ecount, int32_t stamp, int32_t *mark, int32_t *vlist,
                            int32_t *vcount) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int u = eu[e], v = ev[e], T = kcur[e];
        const int l = min(lo[u], lo[v]), hh = max(hi[u], hi[v]);
        if (l < T && T <= hh) {
            elist[atomicAdd(ecount, 1)] = (int32_t)e;
            if (atomicExch(&mark[u], stamp) != stamp) vlist[atomicAdd(vcount, 1)] = u;
            if (atomicExch(&mark[v], stamp) != stamp) vlist[atomicAdd(vcount, 1)] = v;
        } else {
            knew[e] = T;
        }
    }
}

// t(e,h) = H(e) + 2 at the fixed point (Theorem 4).
__global__ void k_hx_truss(int64_t m, const int32_t *__restrict__ hv, int32_t *__restrict__ t) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        t[e] = hv[e] + 2;
}

#define HX_CHECK(...)                                                               \
    do {                                                                             \
        cudaError_t _e = (__VA_ARGS__);                                              \
        if (_e != cudaSuccess) {                                                     \
            set_last_error(std::string("htd_hindex_decompose: ") + #__VA_ARGS__ + ": " + \
                           cudaGetErrorString(_e));                                   \
            st = (_e == cudaErrorMemoryAllocation) ? HTD_ENOMEM : HTD_ECUDA;         \
            goto done;                                                               \
        }                                                                            \
    } while (0)

}  // namespace

htd_status hindex_run(htd_graph *G, Handle *H, int32_t h, int32_t sweeps, int32_t max_iter, bool prune,
                      int32_t *truss_dev, int32_t *hval_dev, htd_hindex_stats *stats, cudaStream_t s) {
    GraphDev &g = H->g;
    const int64_t n = g.n, m = g.m;
    htd_status st = HTD_OK;
    int32_t *sizes = nullptr, *members = nullptr, *P = nullptr, *prev = nullptr, *vals = nullptr;
    int32_t *key = nullptr, *key2 = nullptr, *lists = nullptr, *mark = nullptr, *vlist = nullptr;
    int32_t *dcount = nullptr, *kold = nullptr, *hi = nullptr, *lo = nullptr, *hi2 = nullptr, *lo2 = nullptr;
    int32_t *elist = nullptr, *decount = nullptr, *hecount = nullptr;
    int64_t *off = nullptr;
    void *tmp = nullptr;
    unsigned long long *dchanged = nullptr, *hchanged = nullptr;
    int32_t *hcount = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    htd_hindex_stats loc;
    std::memset(&loc, 0, sizeof(loc));
    loc.h = h;
    loc.sweeps = sweeps;
    loc.pruned = prune ? 1 : 0;
    int64_t launches = 0;
    const int W = (int)std::max<int64_t>(1, (n + 31) / 32);
    const size_t smem = (size_t)W * 4;
    int occ = 0, grid_v = 0;
    int64_t total = 0, maxb = 0, maxd = 0;
    std::vector<int32_t> hsizes;
    if (m == 0) goto finish;
    HX_CHECK(cudaEventCreate(&t0));
    HX_CHECK(cudaEventCreate(&t1));
    HX_CHECK(cudaEventRecord(t0, s));
    HX_CHECK(raise_smem_limit((const void *)k_hx_balls<0>, smem));
    HX_CHECK(raise_smem_limit((const void *)k_hx_balls<1>, smem));
    HX_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hx_balls<1>, kBlock, smem));
    if (occ < 1) {
        set_last_error("htd_hindex_decompose: an n-bit set does not fit in shared memory");
        st = HTD_EUNSUPPORTED;
        goto done;
    }
    grid_v = (int)std::min<int64_t>(n, (int64_t)H->num_sms * occ);
    HX_CHECK(cudaMalloc(&sizes, n * 4));
    HX_CHECK(cudaMalloc(&off, (n + 1) * 8));
    HX_CHECK(cudaMalloc(&lists, (int64_t)grid_v * 2 * n * 4));
    HX_CHECK(cudaMalloc(&tmp, scan_temp_bytes(n + 1)));
    k_hx_balls<0><<<grid_v, kBlock, smem, s>>>((int32_t)n, h, g.row_ptr, g.col, W, lists, sizes, nullptr, nullptr);
    launches++;
    HX_CHECK(cudaGetLastError());
    HX_CHECK(scan_exclusive<int32_t, int64_t>(sizes, off, n, tmp, s, &launches));
    hsizes.resize(n);
    HX_CHECK(cudaMemcpyAsync(&total, off + n, 8, cudaMemcpyDeviceToHost, s));
    HX_CHECK(cudaMemcpyAsync(hsizes.data(), sizes, n * 4, cudaMemcpyDeviceToHost, s));
    HX_CHECK(cudaStreamSynchronize(s));
    for (int64_t x = 0; x < n; x++) maxb = std::max<int64_t>(maxb, hsizes[x]);
    maxd = maxb;
    loc.ball_entries = total;
    HX_CHECK(cudaMalloc(&members, std::max<int64_t>(total, 1) * 4));
    HX_CHECK(cudaMalloc(&P, std::max<int64_t>(total, 1) * 4));
    k_hx_balls<1><<<grid_v, kBlock, smem, s>>>((int32_t)n, h, g.row_ptr, g.col, W, lists, sizes, off, members);
    launches++;
    HX_CHECK(cudaGetLastError());
    cudaFree(lists);
    lists = nullptr;
    {
        // H^(0) = sup(e,h), the h-support of every edge (the initial step of Algorithm 2)
        HX_CHECK(cudaMalloc(&key, m * 4));
        HX_CHECK(cudaMalloc(&key2, m * 4));
        htd_status hs = htd_h_support(G, h, key, s);
        if (hs != HTD_OK) {
            st = hs;
            goto done;
        }
    }
    {
        const int grid_p = H->num_sms * 4;
        const int grid_e = H->num_sms * 8;
        HX_CHECK(cudaMalloc(&prev, (int64_t)grid_p * std::max<int64_t>(maxb, 1) * 4));
        HX_CHECK(cudaMalloc(&vals, (int64_t)grid_e * (kBlock / 32) * std::max<int64_t>(maxd, 1) * 4));
        HX_CHECK(cudaMalloc(&dchanged, 8));
        HX_CHECK(cudaMallocHost(&hchanged, 8));
        HX_CHECK(cudaMalloc(&mark, n * 4));
        HX_CHECK(cudaMalloc(&vlist, n * 4));
        HX_CHECK(cudaMalloc(&dcount, 4));
        HX_CHECK(cudaMallocHost(&hcount, 4));
        HX_CHECK(cudaMemsetAsync(mark, 0xff, n * 4, s));
        if (prune) {
            HX_CHECK(cudaMalloc(&kold, m * 4));
            HX_CHECK(cudaMalloc(&hi, n * 4));
            HX_CHECK(cudaMalloc(&lo, n * 4));
            HX_CHECK(cudaMalloc(&hi2, n * 4));
            HX_CHECK(cudaMalloc(&lo2, n * 4));
            HX_CHECK(cudaMalloc(&elist, m * 4));
            HX_CHECK(cudaMalloc(&decount, 4));
            HX_CHECK(cudaMallocHost(&hecount, 4));
        }
        // every order before the fixed point lowers at least one key (Theorem 3): the sum
        // of H^(0) plus one orders always suffice
        std::vector<int32_t> k0(m);
        HX_CHECK(cudaMemcpyAsync(k0.data(), key, m * 4, cudaMemcpyDeviceToHost, s));
        HX_CHECK(cudaStreamSynchronize(s));
        int64_t cap = 1;
        for (int64_t e = 0; e < m; e++) cap += k0[e];
        const int S = std::max(1, sweeps);
        int32_t stamp = 0;
        int32_t it = 0;
        bool converged = false;
        while (!converged && (max_iter < 0 || it < max_iter) && it < cap) {
            HX_CHECK(cudaMemsetAsync(dchanged, 0, 8, s));
            if (S == 1 && prune && it > 0) {
                // Lemma 4: list the edges that can still fall (key = H^(n-1), kold = H^(n-2))
                HX_CHECK(cudaMemsetAsync(hi, 0xff, n * 4, s));
                HX_CHECK(cudaMemsetAsync(lo, 0x7f, n * 4, s));
                HX_CHECK(cudaMemsetAsync(dcount, 0, 4, s));
                HX_CHECK(cudaMemsetAsync(decount, 0, 4, s));
                k_hx_fall<<<H->num_sms * 4, kBlock, 0, s>>>(m, g.eu, g.ev, kold, key, hi, lo);
                launches++;
                for (int r = 1; r < h; r++) {
                    k_hx_spread<<<H->num_sms * 8, kBlock, 0, s>>>((int32_t)n, g.row_ptr, g.col, hi, lo, hi2, lo2);
                    launches++;
                    std::swap(hi, hi2);
                    std::swap(lo, lo2);
                }
                k_hx_select<<<H->num_sms * 4, kBlock, 0, s>>>(m, g.eu, g.ev, key, hi, lo, key2, elist, decount,
                                                             stamp++, mark, vlist, dcount);
                launches++;
                HX_CHECK(cudaMemcpyAsync(hcount, dcount, 4, cudaMemcpyDeviceToHost, s));
                HX_CHECK(cudaMemcpyAsync(hecount, decount, 4, cudaMemcpyDeviceToHost, s));
                HX_CHECK(cudaStreamSynchronize(s));
                if (*hecount > 0) {
                    k_hx_pathkeys<<<grid_p, kBlock, 0, s>>>(vlist, *hcount, h, g.row_ptr, g.col, g.slot_eid, key,
                                                            off, members, P, prev, maxb);
                    k_hx_edges<<<grid_e, kBlock, 0, s>>>(0, *hecount, elist, g.eu, g.ev, off, members, P, key,
                                                         key2, vals, maxd, dchanged);
                    launches += 2;
                }
                loc.edge_evals += *hecount;
                loc.vertex_evals += *hcount;
                // H^(n-2) <- H^(n-1) <- H^(n)
                std::swap(kold, key);
                std::swap(key, key2);
            } else if (S == 1) {
                k_hx_pathkeys<<<grid_p, kBlock, 0, s>>>(nullptr, (int32_t)n, h, g.row_ptr, g.col, g.slot_eid,
                                                        key, off, members, P, prev, maxb);
                k_hx_edges<<<grid_e, kBlock, 0, s>>>(0, m, nullptr, g.eu, g.ev, off, members, P, key, key2, vals,
                                                     maxd, dchanged);
                launches += 2;
                loc.edge_evals += m;
                loc.vertex_evals += n;
                if (prune) std::swap(kold, key);  // with pruning: H^(n-2) <- H^(n-1) <- H^(n)
                std::swap(key, key2);
            } else {
                for (int j = 0; j < S; j++) {
                    const int64_t e0 = m * j / S, e1 = m * (j + 1) / S;
                    if (e1 <= e0) continue;
                    HX_CHECK(cudaMemsetAsync(dcount, 0, 4, s));
                    k_hx_touch<<<H->num_sms * 2, kBlock, 0, s>>>(e0, e1, g.eu, g.ev, stamp++, mark, vlist, dcount);
                    HX_CHECK(cudaMemcpyAsync(hcount, dcount, 4, cudaMemcpyDeviceToHost, s));
                    HX_CHECK(cudaStreamSynchronize(s));
                    k_hx_pathkeys<<<grid_p, kBlock, 0, s>>>(vlist, *hcount, h, g.row_ptr, g.col, g.slot_eid, key,
                                                            off, members, P, prev, maxb);
                    k_hx_edges<<<grid_e, kBlock, 0, s>>>(e0, e1, nullptr, g.eu, g.ev, off, members, P, key, key,
                                                         vals, maxd, dchanged);
                    launches += 3;
                    loc.edge_evals += e1 - e0;
                    loc.vertex_evals += *hcount;
                }
            }
            HX_CHECK(cudaGetLastError());
            HX_CHECK(cudaMemcpyAsync(hchanged, dchanged, 8, cudaMemcpyDeviceToHost, s));
            HX_CHECK(cudaStreamSynchronize(s));
            it++;
            if (*hchanged == 0) converged = true;
        }
        loc.iterations = it;
        loc.converged = converged ? 1 : 0;
    }
    if (hval_dev) HX_CHECK(cudaMemcpyAsync(hval_dev, key, m * 4, cudaMemcpyDeviceToDevice, s));
    if (truss_dev) {
        k_hx_truss<<<H->num_sms * 2, kBlock, 0, s>>>(m, key, truss_dev);
        launches++;
        HX_CHECK(cudaGetLastError());
    }
    HX_CHECK(cudaEventRecord(t1, s));
    HX_CHECK(cudaEventSynchronize(t1));
    {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        loc.ms_total = ms;
    }
finish:
    loc.kernel_launches = launches;
    if (stats) *stats = loc;
    add_launches(launches);
done:
    cudaFree(sizes);
    cudaFree(off);
    cudaFree(lists);
    cudaFree(tmp);
    cudaFree(members);
    cudaFree(P);
    cudaFree(prev);
    cudaFree(vals);
    cudaFree(key);
    cudaFree(key2);
    cudaFree(dchanged);
    cudaFree(mark);
    cudaFree(vlist);
    cudaFree(dcount);
    cudaFree(kold);
    cudaFree(hi);
    cudaFree(lo);
    cudaFree(hi2);
    cudaFree(lo2);
    cudaFree(elist);
    cudaFree(decount);
    if (hecount) cudaFreeHost(hecount);
    if (hchanged) cudaFreeHost(hchanged);
    if (hcount) cudaFreeHost(hcount);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    return st;
}

}  // namespace htd
