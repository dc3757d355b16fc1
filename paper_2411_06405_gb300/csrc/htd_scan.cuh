// htd_scan.cuh -- device-wide exclusive prefix sum (three launches: tile sums, scan of the
// tile sums in one block, per-tile scan with carry-in).  out[count] receives the total.
#pragma once

#include "htd_common.cuh"

namespace htd {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanBlock) k_scan_tile_sums(const Tin *__restrict__ in,
                                                               int64_t count,
                                                               Tout *__restrict__ partial) {
    __shared__ Tout scratch[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + (int64_t)i * kScanBlock + threadIdx.x;
        if (idx < count) s += (Tout)in[idx];
    }
    Tout tot = block_sum<kScanBlock, Tout>(s, scratch);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename Tout>
__global__ void __launch_bounds__(1024) k_scan_partials(Tout *__restrict__ partial, int64_t nt,
                                                        Tout *__restrict__ total_out) {
    __shared__ Tout scratch[32];
    Tout carry = 0;
    for (int64_t b = 0; b < nt; b += 1024) {
        int64_t i = b + threadIdx.x;
        Tout v = (i < nt) ? partial[i] : Tout(0);
        Tout tot;
        Tout ex = block_exclusive_scan<1024, Tout>(v, &tot, scratch);
        if (i < nt) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kScanBlock) k_scan_tiles(const Tin *__restrict__ in,
                                                           int64_t count,
                                                           const Tout *__restrict__ partial,
                                                           Tout *__restrict__ out) {
    __shared__ Tout scratch[kScanBlock / 32];
    // each thread owns kScanItems consecutive elements of the tile
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    Tout v[kScanItems];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        v[i] = (idx < count) ? (Tout)in[idx] : Tout(0);
        s += v[i];
    }
    Tout tot;
    Tout run = block_exclusive_scan<kScanBlock, Tout>(s, &tot, scratch) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + i;
        if (idx < count) out[idx] = run;
        run += v[i];
    }
}

// Bytes of temporary storage scan_exclusive needs for `count` elements.
inline size_t scan_temp_bytes(int64_t count) {
    int64_t nt = (count + kScanTile - 1) / kScanTile;
    return (size_t)(nt > 0 ? nt : 1) * 8;
}

// out[0..count] = exclusive prefix sums of in[0..count), out[count] = total.
// `tmp` must hold scan_temp_bytes(count) bytes.  Enqueues three kernels on `s`.
template <typename Tin, typename Tout>
inline cudaError_t scan_exclusive(const Tin *in, Tout *out, int64_t count, void *tmp,
                                  cudaStream_t s, int64_t *launches) {
    if (count <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(Tout), s);
    }
    int64_t nt = (count + kScanTile - 1) / kScanTile;
    Tout *partial = static_cast<Tout *>(tmp);
    k_scan_tile_sums<Tin, Tout><<<(unsigned)nt, kScanBlock, 0, s>>>(in, count, partial);
    k_scan_partials<Tout><<<1, 1024, 0, s>>>(partial, nt, out + count);
    k_scan_tiles<Tin, Tout><<<(unsigned)nt, kScanBlock, 0, s>>>(in, count, partial, out);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace htd
