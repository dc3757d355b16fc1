// htd_csr.cu -- normalise an undirected edge list and build the CSR + edge ids.
//
// Graph model of Sec. 2 (simple undirected graph): self-loops are dropped, each pair is
// stored in both rows, every row is sorted and deduplicated (which merges duplicate and
// reversed pairs), and edge e is the e-th pair (u,v), u < v, in lexicographic order.
//
// Steps (all on the device; two host synchronisations, to size the outputs and to read
// the error flag and m):
//   1. count row lengths (ids checked against [0,n));     2. scan -> raw row offsets;
//   3. scatter both directions;                           4. sort + unique each row by size
//      class: <= 32 (one warp, register bitonic), <= 4096 (one block, shared-memory
//      bitonic), larger (one block, n-bit shared-memory set read back in order);
//   5. scan unique lengths -> row_ptr; compact rows and count neighbours above the row id;
//   6. scan those counts -> first edge id of each row; assign slot -> edge id.
#include <cstdio>

#include "htd_internal.h"
#include "htd_scan.cuh"

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr int kMedMax = 4096;

__global__ void k_csr_count(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            int64_t m_in, int32_t n, int32_t *__restrict__ deg,
                            int32_t *__restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_in;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicOr(err, 1);
            continue;
        }
        if (a == b) continue;
        atomicAdd(&deg[a], 1);
        atomicAdd(&deg[b], 1);
    }
}

__global__ void k_csr_scatter(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                              int64_t m_in, int32_t n, const int32_t *__restrict__ off,
                              int32_t *__restrict__ fill, int32_t *__restrict__ colraw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_in;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
        int pa = atomicAdd(&fill[a], 1);
        colraw[off[a] + pa] = b;
        int pb = atomicAdd(&fill[b], 1);
        colraw[off[b] + pb] = a;
    }
}

__device__ __forceinline__ int warp_bitonic_sort32(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            int p = __shfl_xor_sync(0xffffffffu, v, j);
            bool ascending = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            v = (lower == ascending) ? min(v, p) : max(v, p);
        }
    }
    return v;
}

// Rows of length <= 32: one warp each.  Longer rows are listed for the block kernels.
__global__ void k_row_sort_warp(int32_t n, const int32_t *__restrict__ off,
                                int32_t *__restrict__ colraw, int32_t *__restrict__ deg_new,
                                int32_t *__restrict__ med_list, int32_t *__restrict__ med_cnt,
                                int32_t *__restrict__ big_list, int32_t *__restrict__ big_cnt) {
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int b = off[x], len = off[x + 1] - b;
        if (len > 32) {
            if (lane == 0) {
                if (len <= kMedMax) med_list[atomicAdd(med_cnt, 1)] = x;
                else big_list[atomicAdd(big_cnt, 1)] = x;
            }
            continue;
        }
        int v = (lane < len) ? colraw[b + lane] : INT_MAX;
        v = warp_bitonic_sort32(v);
        int prev = __shfl_up_sync(0xffffffffu, v, 1);
        bool keep = lane < len && (lane == 0 || v != prev);
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) colraw[b + __popc(bal & lanemask_lt())] = v;
        if (lane == 0) deg_new[x] = __popc(bal);
    }
}

// Rows of length 33..4096: one block each, bitonic sort in shared memory.
__global__ void __launch_bounds__(kBlock)
k_row_sort_block(const int32_t *__restrict__ list, const int32_t *__restrict__ cnt,
                 const int32_t *__restrict__ off, int32_t *__restrict__ colraw,
                 int32_t *__restrict__ deg_new) {
    __shared__ int32_t buf[kMedMax];
    __shared__ int32_t scratch[kBlock / 32];
    const int rows = *cnt;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int x = list[r];
        const int b = off[x], len = off[x + 1] - b;
        int P = 64;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += kBlock) buf[i] = (i < len) ? colraw[b + i] : INT_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < (P >> 1); i += kBlock) {
                    int a = 2 * i - (i & (j - 1));
                    int c = a + j;
                    bool ascending = (a & k) == 0;
                    int va = buf[a], vc = buf[c];
                    if ((va > vc) == ascending) {
                        buf[a] = vc;
                        buf[c] = va;
                    }
                }
                __syncthreads();
            }
        }
        // unique + ordered compaction: thread t owns items [t*per, (t+1)*per)
        const int per = (len + kBlock - 1) / kBlock;
        const int lo = threadIdx.x * per, hi = min(len, lo + per);
        int keep = 0;
        for (int p = lo; p < hi; p++) keep += (p == 0 || buf[p] != buf[p - 1]);
        int total;
        int pos = block_exclusive_scan<kBlock, int>(keep, &total, scratch);
        for (int p = lo; p < hi; p++) {
            if (p == 0 || buf[p] != buf[p - 1]) colraw[b + pos++] = buf[p];
        }
        if (threadIdx.x == 0) deg_new[x] = total;
        __syncthreads();
    }
}

// Rows longer than 4096: one block each; the row is set into an n-bit shared-memory set
// and read back in increasing id order, which sorts and deduplicates it.
__global__ void __launch_bounds__(kBlock)
k_row_sort_bitset(const int32_t *__restrict__ list, const int32_t *__restrict__ cnt,
                  const int32_t *__restrict__ off, int32_t *__restrict__ colraw,
                  int32_t *__restrict__ deg_new, int32_t W) {
    extern __shared__ uint32_t bits[];
    __shared__ int32_t scratch[kBlock / 32];
    __shared__ int32_t warp_base[kBlock / 32];
    constexpr int NW = kBlock / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // word segment of each warp, a multiple of 32 words
    const int seg = ((W + NW - 1) / NW + 31) & ~31;
    const int rows = *cnt;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int x = list[r];
        const int b = off[x], len = off[x + 1] - b;
        for (int i = threadIdx.x; i < W; i += kBlock) bits[i] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += kBlock) {
            int v = colraw[b + i];
            atomicOr(&bits[v >> 5], 1u << (v & 31));
        }
        __syncthreads();
        const int w0 = wid * seg, w1 = min(W, w0 + seg);
        int c = 0;
        for (int i = w0 + lane; i < w1; i += 32) c += __popc(bits[i]);
        c = warp_sum(c);
        int total;
        int ex = block_exclusive_scan<kBlock, int>(lane == 0 ? c : 0, &total, scratch);
        if (lane == 0) warp_base[wid] = ex;
        __syncthreads();
        int run = warp_base[wid];
        for (int i0 = w0; i0 < w1; i0 += 32) {
            int i = i0 + lane;
            uint32_t word = (i < w1) ? bits[i] : 0u;
            int pc = __popc(word);
            int incl = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int pos = run + incl - pc;
            while (word) {
                int bit = __ffs(word) - 1;
                word &= word - 1;
                colraw[b + pos++] = i * 32 + bit;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (threadIdx.x == 0) deg_new[x] = total;
        __syncthreads();
    }
}

__global__ void k_compact_rows(int32_t n, const int32_t *__restrict__ off,
                               const int32_t *__restrict__ colraw,
                               const int32_t *__restrict__ len_new,
                               const int32_t *__restrict__ row_ptr, int32_t *__restrict__ col,
                               int32_t *__restrict__ fwd) {
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int b = off[x], len = len_new[x], d = row_ptr[x];
        int above = 0;
        for (int j = lane; j < len; j += 32) {
            int v = colraw[b + j];
            col[d + j] = v;
            above += (v > x);
        }
        above = warp_sum(above);
        if (lane == 0) fwd[x] = above;
    }
}

__global__ void k_assign_eids(int32_t n, const int32_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col, const int32_t *__restrict__ fwd,
                              const int32_t *__restrict__ fwd_off,
                              int32_t *__restrict__ slot_eid, int32_t *__restrict__ eu,
                              int32_t *__restrict__ ev, int32_t *__restrict__ slot_lo,
                              int32_t *__restrict__ slot_hi) {
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int rb = row_ptr[x], re = row_ptr[x + 1];
        const int first_fwd = re - fwd[x];
        for (int s = rb + lane; s < re; s += 32) {
            const int y = col[s];
            if (y > x) {
                const int e = fwd_off[x] + (s - first_fwd);
                eu[e] = x;
                ev[e] = y;
                slot_eid[s] = e;
                slot_lo[e] = s;
            } else {
                // position of x in the sorted row of y
                int lo = row_ptr[y], hi = row_ptr[y + 1] - 1;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (col[mid] < x) lo = mid + 1;
                    else hi = mid;
                }
                const int e = fwd_off[y] + (lo - (row_ptr[y + 1] - fwd[y]));
                slot_eid[s] = e;
                slot_hi[e] = s;
            }
        }
    }
}

int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

void free_graph_dev(GraphDev *g) {
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->slot_eid);
    cudaFree(g->eu);
    cudaFree(g->ev);
    cudaFree(g->slot_lo);
    cudaFree(g->slot_hi);
    *g = GraphDev{};
}

#define HTD_TRY(...)                                                                   \
    do {                                                                                \
        cudaError_t _e = (__VA_ARGS__);                                                        \
        if (_e != cudaSuccess) {                                                        \
            set_last_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e));         \
            st = (_e == cudaErrorMemoryAllocation) ? HTD_ENOMEM : HTD_ECUDA;            \
            goto done;                                                                  \
        }                                                                               \
    } while (0)

htd_status build_csr_device(int32_t n, const int32_t *src, const int32_t *dst, int64_t m_in,
                            cudaStream_t s, GraphDev *out, int64_t *launches) {
    htd_status st = HTD_OK;
    GraphDev g;
    int dev = 0;
    int nsm = 0;
    int32_t *deg = nullptr, *off = nullptr, *fill = nullptr, *colraw = nullptr;
    int32_t *deg_new = nullptr, *lists = nullptr, *counters = nullptr, *fwd = nullptr;
    int32_t *fwd_off = nullptr;
    void *tmp = nullptr;
    int32_t host_ctr[4] = {0, 0, 0, 0};
    int64_t nn = n > 0 ? n : 1;
    int64_t raw_slots = 2 * m_in;
    const int W = (n + 31) / 32;
    const size_t smem_big = (size_t)((W + 3) & ~3) * sizeof(uint32_t);
    int32_t two_m = 0;

    HTD_TRY(cudaGetDevice(&dev));
    HTD_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    g.device = dev;
    g.n = n;
    HTD_TRY(cudaMallocAsync(&deg, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&off, (nn + 1) * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&fill, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&colraw, (raw_slots > 0 ? raw_slots : 1) * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&deg_new, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&lists, 2 * nn * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&counters, 4 * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&fwd, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&fwd_off, (nn + 1) * sizeof(int32_t), s));
    HTD_TRY(cudaMallocAsync(&tmp, scan_temp_bytes(nn + raw_slots), s));
    HTD_TRY(cudaMallocAsync(&g.row_ptr, (nn + 1) * sizeof(int32_t), s));
    HTD_TRY(cudaMemsetAsync(deg, 0, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMemsetAsync(fill, 0, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMemsetAsync(deg_new, 0, nn * sizeof(int32_t), s));
    HTD_TRY(cudaMemsetAsync(counters, 0, 4 * sizeof(int32_t), s));

    if (m_in > 0) {
        int gb = grid_for(m_in, kBlock, nsm * 8);
        k_csr_count<<<gb, kBlock, 0, s>>>(src, dst, m_in, n, deg, counters + 2);
        (*launches)++;
    }
    HTD_TRY(scan_exclusive<int32_t, int32_t>(deg, off, n, tmp, s, launches));
    if (m_in > 0) {
        int gb = grid_for(m_in, kBlock, nsm * 8);
        k_csr_scatter<<<gb, kBlock, 0, s>>>(src, dst, m_in, n, off, fill, colraw);
        (*launches)++;
    }
    if (n > 0) {
        int gw = grid_for((int64_t)n * 32, kBlock, nsm * 16);
        k_row_sort_warp<<<gw, kBlock, 0, s>>>(n, off, colraw, deg_new, lists, counters, lists + nn,
                                              counters + 1);
        k_row_sort_block<<<nsm * 4, kBlock, 0, s>>>(lists, counters, off, colraw, deg_new);
        if (smem_big > 48 * 1024) {
            HTD_TRY(raise_smem_limit((const void *)k_row_sort_bitset, smem_big));
        }
        k_row_sort_bitset<<<nsm, kBlock, smem_big, s>>>(lists + nn, counters + 1, off, colraw,
                                                        deg_new, W);
        *launches += 3;
    }
    HTD_TRY(cudaGetLastError());
    HTD_TRY(scan_exclusive<int32_t, int32_t>(deg_new, g.row_ptr, n, tmp, s, launches));
    HTD_TRY(cudaMemcpyAsync(&two_m, g.row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HTD_TRY(cudaMemcpyAsync(host_ctr, counters, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HTD_TRY(cudaStreamSynchronize(s));
    if (host_ctr[2] != 0) {
        set_last_error("htd_build_csr: vertex id outside [0, n)");
        st = HTD_EINVAL;
        goto done;
    }
    g.m = two_m / 2;
    {
        int64_t mm = g.m > 0 ? g.m : 1;
        HTD_TRY(cudaMallocAsync(&g.col, 2 * mm * sizeof(int32_t), s));
        HTD_TRY(cudaMallocAsync(&g.slot_eid, 2 * mm * sizeof(int32_t), s));
        HTD_TRY(cudaMallocAsync(&g.eu, mm * sizeof(int32_t), s));
        HTD_TRY(cudaMallocAsync(&g.ev, mm * sizeof(int32_t), s));
        HTD_TRY(cudaMallocAsync(&g.slot_lo, mm * sizeof(int32_t), s));
        HTD_TRY(cudaMallocAsync(&g.slot_hi, mm * sizeof(int32_t), s));
    }
    if (n > 0) {
        int gw = grid_for((int64_t)n * 32, kBlock, nsm * 16);
        k_compact_rows<<<gw, kBlock, 0, s>>>(n, off, colraw, deg_new, g.row_ptr, g.col, fwd);
        (*launches)++;
        HTD_TRY(scan_exclusive<int32_t, int32_t>(fwd, fwd_off, n, tmp, s, launches));
        k_assign_eids<<<gw, kBlock, 0, s>>>(n, g.row_ptr, g.col, fwd, fwd_off, g.slot_eid, g.eu,
                                            g.ev, g.slot_lo, g.slot_hi);
        (*launches)++;
    }
    HTD_TRY(cudaGetLastError());
    HTD_TRY(cudaStreamSynchronize(s));

done:
    cudaFreeAsync(deg, s);
    cudaFreeAsync(off, s);
    cudaFreeAsync(fill, s);
    cudaFreeAsync(colraw, s);
    cudaFreeAsync(deg_new, s);
    cudaFreeAsync(lists, s);
    cudaFreeAsync(counters, s);
    cudaFreeAsync(fwd, s);
    cudaFreeAsync(fwd_off, s);
    cudaFreeAsync(tmp, s);
    if (st != HTD_OK) {
        cudaStreamSynchronize(s);
        free_graph_dev(&g);
        return st;
    }
    *out = g;
    return HTD_OK;
}

}  // namespace htd
