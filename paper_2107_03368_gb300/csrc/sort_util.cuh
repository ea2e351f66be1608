// sort_util.cuh — stable LSD radix sort of (uint32 key, uint32 value) pairs
// on the device, 8 bits per pass.  A warp owns a tile of consecutive pairs
// (4,096 for large sorts, 512 below 2^21 pairs so that small sorts still
// spread over many warps); the per-(digit, tile) counts are scanned digit-major, so
// equal digits keep tile order, and inside a tile equal digits keep lane
// order within each 32-pair step.
#pragma once
#include <algorithm>
#include <utility>

#include "block_util.cuh"
#include "dt_internal.cuh"

namespace dtk {
namespace {

// Keys per warp in the radix passes.
inline int radix_tile(int64_t m) { return m > (1 << 21) ? 4096 : 512; }

__global__ void __launch_bounds__(128)
radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t m, int shift, int64_t n_tiles,
                  int tile_keys, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[4][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = lane; i < 256; i += 32) h[w][i] = 0;
    __syncwarp();
    const int64_t tile = (int64_t)blockIdx.x * 4 + w;
    if (tile >= n_tiles) return;
    const int64_t b = tile * tile_keys, e = std::min<int64_t>(b + tile_keys, m);
    for (int64_t i = b + lane; i < e; i += 32) atomicAdd(&h[w][(keys[i] >> shift) & 255u], 1u);
    __syncwarp();
    for (int d = lane; d < 256; d += 32) hist[(int64_t)d * n_tiles + tile] = h[w][d];
}

__global__ void __launch_bounds__(1024) excl_scan_kernel(uint32_t *a, int64_t len)
{
    __shared__ uint32_t tmp[33];
    uint32_t run = 0;
    for (int64_t c0 = 0; c0 < len; c0 += blockDim.x) {
        const int64_t c = c0 + threadIdx.x;
        uint32_t tot;
        const uint32_t before = block_excl_scan(c < len ? a[c] : 0u, tmp, &tot);
        if (c < len) a[c] = run + before;
        run += tot;
    }
}

__global__ void __launch_bounds__(128)
radix_scatter_kernel(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t m,
                     int shift, int64_t n_tiles, int tile_keys, const uint32_t *__restrict__ hist,
                     uint32_t *__restrict__ kout, uint32_t *__restrict__ vout)
{
    __shared__ uint32_t base[4][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t tile = (int64_t)blockIdx.x * 4 + w;
    if (tile >= n_tiles) return;
    for (int d = lane; d < 256; d += 32) base[w][d] = hist[(int64_t)d * n_tiles + tile];
    __syncwarp();
    const int64_t b = tile * tile_keys, e = std::min<int64_t>(b + tile_keys, m);
    const unsigned below = (1u << lane) - 1u;
    for (int64_t c = b; c < e; c += 32) {
        const int64_t i = c + lane;
        const bool valid = i < e;
        const uint32_t k = valid ? kin[i] : 0u;
        const uint32_t dg = valid ? ((k >> shift) & 255u) : 256u + (uint32_t)lane;   // unique if invalid
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = (uint32_t)__popc(peers & below);
        if (valid) {
            const uint32_t pos = base[w][dg] + rank;
            kout[pos] = k;
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (valid && rank == 0) base[w][dg] += (uint32_t)__popc(peers);
        __syncwarp();
    }
}

inline int64_t radix_tiles(int64_t m) { return (m + radix_tile(m) - 1) / radix_tile(m); }

// Sorts m pairs by the low `bits` bits of the keys.  *keys / *vals hold the
// input; on return they point at the sorted pairs (the buffers are swapped
// with *keys2 / *vals2 after each pass).  hist holds radix_tiles(m) * 256
// counters.
inline cudaError_t radix_sort_pairs(uint32_t **keys, uint32_t **vals, uint32_t **keys2,
                                    uint32_t **vals2, int64_t m, int bits, uint32_t *hist,
                                    cudaStream_t s)
{
    const int64_t n_tiles = radix_tiles(m);
    const int tile_keys = radix_tile(m);
    const unsigned blocks = (unsigned)((n_tiles + 3) / 4);
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<blocks, 128, 0, s>>>(*keys, m, shift, n_tiles, tile_keys, hist);
        excl_scan_kernel<<<1, 1024, 0, s>>>(hist, n_tiles * 256);
        radix_scatter_kernel<<<blocks, 128, 0, s>>>(*keys, *vals, m, shift, n_tiles, tile_keys, hist,
                                                    *keys2, *vals2);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        std::swap(*keys, *keys2);
        std::swap(*vals, *vals2);
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace dtk
