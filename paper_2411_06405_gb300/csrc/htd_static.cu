// htd_static.cu -- h-support without any device allocation (htd_h_support_static).
//
// For callers that cannot allocate device memory: the ones running where cudaMalloc is
// forbidden or unsafe (inside a custom allocator or memory-pool callback, under an
// external memory budget that owns every byte of the device, or in a process that must
// not grow its footprint after start-up).  The caller passes the graph's CSR and edge
// list and the output buffer; the kernel's scratch lives in one file-scope device array of
// fixed size (kStaticScratchInts int32 = 32 MiB), which every GPU that loads the library
// holds until the process exits.
//
// Each block takes edges from a work queue (its head lives in the scratch array) and builds
// both endpoints' h-hop balls as n-bit sets in shared memory, then counts the common
// members: sup(e,h) = |B(u,h) ∩ B(v,h)| - 2 (Def. 2, Def. 3).  For h >= 3 the vertices first
// reached at each depth are listed in per-block regions of the scratch array.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "htd_internal.h"

namespace htd {
namespace {

constexpr int kBlock = 256;
constexpr int64_t kStaticScratchInts = (int64_t)8 << 20;  // 32 MiB
constexpr int kCounterInts = 64;                          // queue head, padded to 256 bytes
constexpr int kMaxDevices = 64;

// Scratch of htd_h_support_static: [0] block work-queue head (cleared by each call), then
// per-block BFS level lists (h >= 3), 2 x n int32 per block.
static __device__ __align__(256) int32_t g_static_scratch[kStaticScratchInts];

// Sets bit z; returns true if this thread set it first.
__device__ __forceinline__ bool mark(uint32_t *bits, int32_t z) {
    const uint32_t m = 1u << (z & 31);
    return (atomicOr(bits + (z >> 5), m) & m) == 0u;
}

// B(x,h) into the shared n-bit set `bits` (cleared by the caller).  Depth 1 and 2 are
// expanded straight from the rows; deeper levels from the two block-private lists.
__device__ void build_ball(int32_t x, int32_t h, const int32_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col, uint32_t *bits, int32_t *list0,
                           int32_t *list1, int32_t *s_cnt) {
    if (threadIdx.x == 0) {
        mark(bits, x);
        s_cnt[0] = 0;
        s_cnt[1] = 0;
    }
    __syncthreads();
    const int rb = row_ptr[x], re = row_ptr[x + 1];
    for (int s = rb + threadIdx.x; s < re; s += kBlock) mark(bits, col[s]);
    __syncthreads();
    if (h >= 2) {
        // depth 2: a warp per neighbour of x, lanes over its row
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int s = rb + wid; s < re; s += kBlock / 32) {
            const int y = col[s];
            const int yb = row_ptr[y], ye = row_ptr[y + 1];
            for (int t = yb + lane; t < ye; t += 32) {
                const int z = col[t];
                const bool fresh = mark(bits, z);
                if (h >= 3 && fresh) list0[atomicAdd(&s_cnt[0], 1)] = z;
            }
        }
        __syncthreads();
    }
    for (int d = 3; d <= h; d++) {
        int32_t *cur = ((d - 3) & 1) ? list1 : list0;
        int32_t *nxt = ((d - 3) & 1) ? list0 : list1;
        const int ci = (d - 3) & 1;
        const int ncur = s_cnt[ci];
        __syncthreads();
        if (threadIdx.x == 0) s_cnt[ci ^ 1] = 0;
        __syncthreads();
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int i = wid; i < ncur; i += kBlock / 32) {
            const int y = cur[i];
            const int yb = row_ptr[y], ye = row_ptr[y + 1];
            for (int t = yb + lane; t < ye; t += 32) {
                const int z = col[t];
                const bool fresh = mark(bits, z);
                if (d < h && fresh) nxt[atomicAdd(&s_cnt[ci ^ 1], 1)] = z;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock)
k_hsup_static(int32_t n, int32_t W, const int32_t *__restrict__ row_ptr,
              const int32_t *__restrict__ col, int64_t m, const int32_t *__restrict__ eu,
              const int32_t *__restrict__ ev, int32_t h, int32_t *__restrict__ sup,
              int32_t *scratch) {
    extern __shared__ __align__(16) uint32_t sets[];  // two n-bit sets of W words
    __shared__ int32_t s_cnt[2];
    __shared__ int32_t s_red[kBlock / 32];
    __shared__ long long s_edge;
    uint32_t *A = sets, *B = sets + W;
    int32_t *list0 = nullptr, *list1 = nullptr;
    if (h >= 3) {
        list0 = scratch + kCounterInts + (int64_t)blockIdx.x * 2 * n;
        list1 = list0 + n;
    }
    for (;;) {
        if (threadIdx.x == 0) s_edge = (long long)atomicAdd(reinterpret_cast<unsigned int *>(scratch), 1u);
        __syncthreads();
        const long long e = s_edge;
        if (e >= m) break;
        for (int i = threadIdx.x; i < 2 * W; i += kBlock) sets[i] = 0u;
        __syncthreads();
        build_ball(eu[e], h, row_ptr, col, A, list0, list1, s_cnt);
        build_ball(ev[e], h, row_ptr, col, B, list0, list1, s_cnt);
        int c = 0;
        for (int i = threadIdx.x; i < W; i += kBlock) c += __popc(A[i] & B[i]);
        c = warp_sum(c);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int j = 0; j < kBlock / 32; j++) t += s_red[j];
            sup[e] = t - 2;
        }
        __syncthreads();
    }
}

std::mutex g_dev_mutex;
int32_t *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace htd

extern "C" htd_status htd_h_support_static(int32_t n, const int32_t *row_ptr_dev,
                                           const int32_t *col_dev, int64_t m,
                                           const int32_t *eu_dev, const int32_t *ev_dev,
                                           int32_t h, int32_t *sup_dev, void *stream) {
    using namespace htd;
    if (n < 0 || m < 0 || h < 1 || h > HTD_MAX_H || !row_ptr_dev ||
        (m > 0 && (!col_dev || !eu_dev || !ev_dev || !sup_dev))) {
        set_last_error("htd_h_support_static: NULL argument, negative size or h outside [1, HTD_MAX_H]");
        return HTD_EINVAL;
    }
    if (n > HTD_STATIC_MAX_N) {
        set_last_error("htd_h_support_static: n exceeds HTD_STATIC_MAX_N");
        return HTD_EUNSUPPORTED;
    }
    if (m >= ((int64_t)1 << 31)) {
        set_last_error("htd_h_support_static: m too large");
        return HTD_EOVERFLOW;
    }
    if (h >= 3 && kCounterInts + 2 * (int64_t)n > kStaticScratchInts) {
        set_last_error("htd_h_support_static: BFS lists of one block exceed the static scratch");
        return HTD_EUNSUPPORTED;
    }
    if (m == 0) return HTD_OK;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) e = cudaErrorInvalidDevice;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // once per device, with that device current: the device address of the scratch array
    // (its host-side name is only a stand-in and must never reach a kernel)
    int32_t *scratch = nullptr;
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_dev_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e == cudaSuccess) g_scratch_ptr[dev] = static_cast<int32_t *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    const int W = (n + 31) / 32 > 0 ? (n + 31) / 32 : 1;
    const size_t smem = (size_t)2 * W * sizeof(uint32_t);
    int occ = 0, optin = 0;
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_hsup_static);
    if (e == cudaSuccess && smem + fa.sharedSizeBytes > (size_t)optin) {
        // n is within HTD_STATIC_MAX_N but this device's blocks cannot hold two n-bit sets
        set_last_error("htd_h_support_static: two n-bit sets do not fit in this device's shared memory");
        return HTD_EUNSUPPORTED;
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_hsup_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hsup_static, kBlock, smem);
    if (e != cudaSuccess) {
        set_last_error(std::string("htd_h_support_static: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    if (occ < 1) {
        set_last_error("htd_h_support_static: two n-bit sets do not fit in shared memory");
        return HTD_EUNSUPPORTED;
    }
    int64_t grid = (int64_t)nsm * occ;
    if (h >= 3) grid = std::min<int64_t>(grid, (kStaticScratchInts - kCounterInts) / (2 * (int64_t)n));
    if (grid > m) grid = m;
    if (grid < 1) grid = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the queue head must start at zero; the lists need no clearing
    e = cudaMemsetAsync(scratch, 0, kCounterInts * sizeof(int32_t), s);
    if (e == cudaSuccess) {
        k_hsup_static<<<(unsigned)grid, kBlock, smem, s>>>(n, W, row_ptr_dev, col_dev, m, eu_dev, ev_dev,
                                                           h, sup_dev, scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_last_error(std::string("htd_h_support_static: ") + cudaGetErrorString(e));
        return HTD_ECUDA;
    }
    return HTD_OK;
}
