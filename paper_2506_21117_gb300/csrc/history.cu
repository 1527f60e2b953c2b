// History recovery and merging of scene updates (Supp. "History Recovery",
// its algorithm, and "Batched Updates"). Both reduce to a stable partition of
// rows by a changed-row mask I: before optimising update t, G^{t-1} is
// reordered so its unchanged rows come first in their order (then the changed
// ones), and G^{t-1} is recovered from G^t by sending G^t's first #static rows
// to the positions where I = 0 and the stored O^t to those where I = 1. Ranks
// come from one chunked exclusive scan of I; rows move by a gather whose map
// entry is a row of the first source, or ~row of the second.
#include "scan.cuh"

namespace cls {

constexpr int kHBlock = 256;
constexpr int kHItems = 8;
constexpr int kHChunk = kHBlock * kHItems;

__global__ void __launch_bounds__(kHBlock)
flag_count_kernel(const uint8_t* __restrict__ flags, int n, int64_t* __restrict__ partials) {
    __shared__ int64_t smem[kHBlock / 32 + 1];
    int64_t c = 0;
    for (int it = 0; it < kHItems; ++it) {
        const int i = blockIdx.x * kHChunk + it * kHBlock + threadIdx.x;
        if (i < n) c += flags[i] != 0;
    }
    int64_t tot;
    block_exclusive_sum<kHBlock>(c, smem, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// mode 0 (partition): map[dst] = i, dst = flagged ? n_static + ones_before(i)
//   : i - ones_before(i); mode 1 (recovery): map[i] = flagged ?
//   ~ones_before(i) (row of the second source, O) : i - ones_before(i).
__global__ void __launch_bounds__(kHBlock)
flag_map_kernel(const uint8_t* __restrict__ flags, int n, const int64_t* __restrict__ offsets,
                const int32_t* __restrict__ n_ones, int mode, int32_t* __restrict__ map) {
    __shared__ int64_t smem[kHBlock / 32 + 1];
    int64_t base = offsets[blockIdx.x];
    const int64_t n_static = (int64_t)n - *n_ones;
    for (int it = 0; it < kHItems; ++it) {
        const int i = blockIdx.x * kHChunk + it * kHBlock + threadIdx.x;
        const int64_t f = (i < n && flags[i]) ? 1 : 0;
        int64_t tot;
        const int64_t ones = base + block_exclusive_sum<kHBlock>(f, smem, tot);
        base += tot;
        if (i >= n) continue;
        if (mode == 0) map[f ? n_static + ones : i - ones] = i;
        else map[i] = f ? ~(int32_t)ones : (int32_t)(i - ones);
    }
}

// dst row i = map[i] >= 0 ? a[map[i]] : b[~map[i]] (stride floats, float4 units).
__global__ void __launch_bounds__(kHBlock)
gather_rows_kernel(const float4* __restrict__ a, const float4* __restrict__ b,
                   const int32_t* __restrict__ map, int n_out, int quads,
                   float4* __restrict__ dst) {
    const int64_t total = (int64_t)n_out * quads;
    for (int64_t e = (int64_t)blockIdx.x * kHBlock + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * kHBlock) {
        const int64_t i = e / quads;
        const int q = (int)(e - i * quads);
        const int32_t m = map[i];
        dst[e] = m >= 0 ? a[(int64_t)m * quads + q] : b[(int64_t)(~m) * quads + q];
    }
}

}  // namespace cls

using namespace cls;

extern "C" size_t cls_flag_map_workspace_size(int32_t n) {
    if (n < 0) return 0;
    const int64_t chunks = ((int64_t)n + kHChunk - 1) / kHChunk;
    return (size_t)((chunks + 1) * 8 + 255) / 256 * 256;
}

extern "C" int cls_flag_map(const uint8_t* flags, int32_t n, int32_t mode, int32_t* map,
                            int32_t* n_flagged_dev, void* workspace, size_t workspace_bytes,
                            cls_stream_t stream) {
    if (!flags || !map || !n_flagged_dev || !workspace || n < 0 || (mode != 0 && mode != 1) ||
        workspace_bytes < cls_flag_map_workspace_size(n))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        cudaMemsetAsync(n_flagged_dev, 0, 4, s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const int64_t chunks = ((int64_t)n + kHChunk - 1) / kHChunk;
    int64_t* partials = static_cast<int64_t*>(workspace);
    flag_count_kernel<<<(unsigned)chunks, kHBlock, 0, s>>>(flags, n, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, chunks, nullptr, n_flagged_dev, -1,
                                            nullptr);
    flag_map_kernel<<<(unsigned)chunks, kHBlock, 0, s>>>(flags, n, partials, n_flagged_dev, mode,
                                                         map);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_gather_rows(const float* a, const float* b, const int32_t* map, int32_t n_out,
                               int32_t stride, float* dst, cls_stream_t stream) {
    if (!a || !map || !dst || n_out < 0 || stride <= 0 || stride % 4 != 0)
        return CLS_ERR_INVALID_ARG;
    if (n_out > 0) {
        const int quads = stride / 4;
        const int64_t total = (int64_t)n_out * quads;
        const unsigned grid = (unsigned)hmin64((total + kHBlock - 1) / kHBlock, 8192);
        gather_rows_kernel<<<grid, kHBlock, 0, as_stream(stream)>>>(
            reinterpret_cast<const float4*>(a), reinterpret_cast<const float4*>(b ? b : a), map,
            n_out, quads, reinterpret_cast<float4*>(dst));
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
