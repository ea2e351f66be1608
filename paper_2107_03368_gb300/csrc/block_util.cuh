// block_util.cuh — thread-block scan, reduction and bitonic sort helpers.
#pragma once

#include <cstdint>

namespace dtk {

// Exclusive prefix sum of one value per thread over the block.  `tmp` is
// shared scratch of at least 33 words.  Returns the thread's exclusive
// prefix; *total receives the block sum.  All threads must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *tmp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) tmp[lane] = s;          // inclusive warp totals
        if (lane == 31) tmp[32] = s;
    }
    __syncthreads();
    uint32_t before = wid > 0 ? tmp[wid - 1] : 0;
    uint32_t tot = tmp[32];
    __syncthreads();
    *total = tot;
    return before + x - v;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *tmp)
{
    uint32_t t;
    block_excl_scan(v, tmp, &t);
    return t;
}

// Ascending bitonic sort of a[0..p2) in shared memory; p2 a power of two.
__device__ __forceinline__ void block_bitonic_sort(uint64_t *a, int p2)
{
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t x = a[i], y = a[ixj];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[ixj] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace dtk
