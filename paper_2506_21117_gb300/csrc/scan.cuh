// Block-wide and device-wide exclusive prefix sums used for stream
// compaction (active set, active tiles) and for pair allocation.
#pragma once

#include "common.cuh"

namespace cls {

// Exclusive prefix sum over the block of `v` (BLOCK threads, a multiple of
// 32). `smem` needs BLOCK/32 + 1 slots. Returns the prefix; `total` gets the
// block sum. Contains __syncthreads(): every thread must call it.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* smem, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < BLOCK / 32 ? smem[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < BLOCK / 32) smem[lane] = w;  // inclusive warp totals
        if (lane == BLOCK / 32 - 1) smem[BLOCK / 32] = w;
    }
    __syncthreads();
    const T warp_prefix = warp > 0 ? smem[warp - 1] : T(0);
    total = smem[BLOCK / 32];
    const T excl = warp_prefix + x - v;
    __syncthreads();
    return excl;
}

// Single-block exclusive scan of `n` partial sums in place; the grand total
// goes to total64 and/or total32. If a capacity is given and the total
// exceeds it, CLS_ERR_CAPACITY is recorded in `status`.
__global__ void scan_partials_kernel(int64_t* partials, int64_t n, int64_t* total64,
                                     int32_t* total32, int64_t capacity, int32_t* status);

}  // namespace cls
