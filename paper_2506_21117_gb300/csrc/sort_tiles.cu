// Per-tile depth sort of the bucketed layout. cls_project_and_bin has already
// done the most significant radix pass: every (Gaussian, tile) pair sits in
// the bucket of its (tile, depth bin), buckets in tile order and, inside a
// tile, in depth-bin order. What is left is sorting each bucket by its key
// (depth bits << 32 | record index). One block per tile walks the tile's
// depth bins, gathers consecutive bins into windows of at most kCap keys and
// sorts each window in shared memory with a stable LSD radix sort on the
// depth bits (8-bit digits, passes whose digit is shared by every key are
// skipped), then orders equal depths by record index. A single bin larger than
// kCap is sorted by the same block in chunks through global memory.
#include "common.cuh"

namespace cls {

constexpr int kTB = 512;
constexpr int kTW = kTB / 32;
constexpr int kTItems = 8;
constexpr int kCap = kTB * kTItems;  // 4096 keys per shared-memory window
constexpr int kRad = 256;
constexpr int kBinsPerTile = CLS_DEPTH_BINS;

struct TileSortSmem {
    uint64_t a[kCap];
    uint64_t b[kCap];
    uint16_t whist[kTW][kRad];
    uint32_t dtot[kRad];
    uint32_t dstart[kRad];
    int64_t gbase[kRad];
    uint32_t off[kBinsPerTile + 1];
    uint32_t scan_tmp[kRad / 32 + 1];
    int tile;
};

__device__ __forceinline__ uint32_t lane_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
    return (uint32_t)(k >> shift) & (kRad - 1);
}

// Rank `m` keys of `src` (m <= kCap) by digit, stably: per-warp match-any
// ranking, then warp prefixes per digit. Leaves per-key ranks in `rank`,
// digit totals in sm.dtot and warp prefixes in sm.whist. Block-wide.
__device__ __forceinline__ void rank_chunk(TileSortSmem& sm, const uint64_t* src, int m, int shift,
                                           uint64_t (&key)[kTItems], uint32_t (&rank)[kTItems]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lane_lt();
    for (int i = threadIdx.x; i < kTW * kRad; i += kTB) (&sm.whist[0][0])[i] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kTItems; ++r) {
        const int i = warp * (32 * kTItems) + r * 32 + lane;
        const bool ok = i < m;
        key[r] = ok ? src[i] : 0ull;
        const uint32_t d = ok ? digit_of(key[r], shift) : (uint32_t)kRad;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t base = 0;
        if (ok) base = sm.whist[warp][d];
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) sm.whist[warp][d] = (uint16_t)(base + __popc(peers));
        __syncwarp();
        rank[r] = ok ? base + __popc(peers & lt) : 0xffffffffu;
    }
    __syncthreads();
    if (threadIdx.x < kRad) {
        const int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kTW; ++w) {
            const uint32_t t = sm.whist[w][d];
            sm.whist[w][d] = (uint16_t)tot;
            tot += t;
        }
        sm.dtot[d] = tot;
    }
    __syncthreads();
}

// Exclusive scan of sm.dtot into sm.dstart (threads < kRad). Block-wide.
__device__ __forceinline__ void scan_digits(TileSortSmem& sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = 0, v = 0;
    if (threadIdx.x < kRad) {
        v = sm.dtot[threadIdx.x];
        x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm.scan_tmp[warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = threadIdx.x < kRad / 32 ? sm.scan_tmp[threadIdx.x] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (threadIdx.x < kRad / 32) sm.scan_tmp[threadIdx.x] = w;
    }
    __syncthreads();
    if (threadIdx.x < kRad) sm.dstart[threadIdx.x] = (warp > 0 ? sm.scan_tmp[warp - 1] : 0u) + x - v;
    __syncthreads();
}

// Equal depths: order by record index (the low word). Runs of equal depth are
// short; the first element of each run sorts it by insertion.
__device__ __forceinline__ void fix_ties(uint64_t* k, int n) {
    for (int i = threadIdx.x; i < n; i += kTB) {
        const uint32_t hi = (uint32_t)(k[i] >> 32);
        if (i > 0 && (uint32_t)(k[i - 1] >> 32) == hi) continue;
        int j = i + 1;
        while (j < n && (uint32_t)(k[j] >> 32) == hi) ++j;
        for (int p = i + 1; p < j; ++p) {
            const uint64_t x = k[p];
            int q = p - 1;
            while (q >= i && k[q] > x) {
                k[q + 1] = k[q];
                --q;
            }
            k[q + 1] = x;
        }
    }
}

// Sort keys[w0, w0 + n), n <= kCap, in shared memory.
__device__ void sort_window(TileSortSmem& sm, uint64_t* keys, int64_t w0, int n) {
    for (int i = threadIdx.x; i < n; i += kTB) sm.a[i] = keys[w0 + i];
    __syncthreads();
    uint64_t* src = sm.a;
    uint64_t* dst = sm.b;
    uint64_t key[kTItems];
    uint32_t rank[kTItems];
    const int warp = threadIdx.x >> 5;
    for (int p = 0; p < 4; ++p) {
        const int shift = 32 + 8 * p;
        rank_chunk(sm, src, n, shift, key, rank);
        const bool trivial = __syncthreads_or(threadIdx.x < kRad && sm.dtot[threadIdx.x] == (uint32_t)n);
        if (trivial) continue;
        scan_digits(sm);
#pragma unroll
        for (int r = 0; r < kTItems; ++r) {
            if (rank[r] != 0xffffffffu) {
                const uint32_t d = digit_of(key[r], shift);
                dst[sm.dstart[d] + sm.whist[warp][d] + rank[r]] = key[r];
            }
        }
        __syncthreads();
        uint64_t* t = src; src = dst; dst = t;
    }
    fix_ties(src, n);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kTB) keys[w0 + i] = src[i];
    __syncthreads();
}

// Sort keys[r0, r0 + n), n > kCap, in chunks through global memory; `alt` is a
// scratch buffer addressed with the same offsets.
__device__ void sort_big(TileSortSmem& sm, uint64_t* keys, uint64_t* alt, int64_t r0, int64_t n) {
    uint64_t* src = keys + r0;
    uint64_t* dst = alt + r0;
    uint64_t key[kTItems];
    uint32_t rank[kTItems];
    const int warp = threadIdx.x >> 5;
    for (int p = 0; p < 4; ++p) {
        const int shift = 32 + 8 * p;
        if (threadIdx.x < kRad) sm.dtot[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < n; i += kTB) atomicAdd(&sm.dtot[digit_of(src[i], shift)], 1u);
        __syncthreads();
        const bool trivial = __syncthreads_or(threadIdx.x < kRad && sm.dtot[threadIdx.x] == (uint32_t)n);
        if (trivial) continue;
        scan_digits(sm);
        if (threadIdx.x < kRad) sm.gbase[threadIdx.x] = sm.dstart[threadIdx.x];
        __syncthreads();
        for (int64_t c0 = 0; c0 < n; c0 += kCap) {
            const int m = (int)(n - c0 < kCap ? n - c0 : kCap);
            rank_chunk(sm, src + c0, m, shift, key, rank);
#pragma unroll
            for (int r = 0; r < kTItems; ++r) {
                if (rank[r] != 0xffffffffu) {
                    const uint32_t d = digit_of(key[r], shift);
                    dst[sm.gbase[d] + sm.whist[warp][d] + rank[r]] = key[r];
                }
            }
            __syncthreads();
            if (threadIdx.x < kRad) sm.gbase[threadIdx.x] += sm.dtot[threadIdx.x];
            __syncthreads();
        }
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != keys + r0) {
        for (int64_t i = threadIdx.x; i < n; i += kTB) keys[r0 + i] = src[i];
        __syncthreads();
    }
    fix_ties(keys + r0, (int)n);
    __syncthreads();
}

__global__ void __launch_bounds__(kTB)
sort_tiles_kernel(uint64_t* __restrict__ keys, uint64_t* __restrict__ alt,
                  const uint32_t* __restrict__ bin_offsets, const int32_t* __restrict__ n_active,
                  const int32_t* __restrict__ active_tiles,
                  const ClsTileCache* __restrict__ tile_cache, int* __restrict__ work_counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSortSmem& sm = *reinterpret_cast<TileSortSmem*>(smem_raw);
    const int n_tiles = *n_active;
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(work_counter, 1);
        __syncthreads();
        const int t = sm.tile;
        if (t >= n_tiles) break;
        if (threadIdx.x <= kBinsPerTile)
            sm.off[threadIdx.x] = bin_offsets[(int64_t)t * kBinsPerTile + threadIdx.x];
        __syncthreads();
        int b = 0;
        if (tile_cache) {  // bins that end inside a cached prefix are not emitted
            const uint32_t np = tile_cache[active_tiles[t]].n_prefix;
            if (np != CLS_PREFIX_UNKNOWN)
                while (b < kBinsPerTile && sm.off[b + 1] - sm.off[0] <= np) ++b;
        }
        while (b < kBinsPerTile) {  // uniform over the block
            const uint32_t w0 = sm.off[b];
            int e = b + 1;
            while (e < kBinsPerTile && sm.off[e + 1] - w0 <= (uint32_t)kCap) ++e;
            const uint32_t len = sm.off[e] - w0;
            if (len > (uint32_t)kCap) {  // one bin alone is too large
                sort_big(sm, keys, alt, w0, len);
            } else if (len > 1) {
                sort_window(sm, keys, w0, (int)len);
            }
            b = e;
        }
        __syncthreads();
    }
}

// Bins holding at least `min_bin` keys (the renderer sorts smaller ones): a
// warp per tile, eight consecutive bins per lane (the end of a lane's last bin
// is its right neighbour's first offset). With `cut`, bins beyond a tile's cut
// (not emitted yet) are skipped. With a list of completed tiles (`trunc`),
// only their bins beyond the old cut are taken. A bin that ends inside the
// tile's cached prefix is never read and is skipped too.
constexpr int kCollectBins = kBinsPerTile / 32;  // bins per lane

__global__ void __launch_bounds__(256)
collect_bins_kernel(const uint32_t* __restrict__ bin_offsets,
                    const int32_t* __restrict__ n_active,
                    const int32_t* __restrict__ active_tiles,
                    const uint8_t* __restrict__ cut,
                    const int32_t* __restrict__ trunc,
                    const int32_t* __restrict__ trunc_count, int64_t trunc_cap,
                    const ClsTileCache* __restrict__ tile_cache,
                    int min_bin, uint2* __restrict__ list,
                    int32_t* __restrict__ count, int64_t list_cap,
                    int32_t* __restrict__ sort_queue) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) *sort_queue = 0;  // the bin sort's tile queue
    const int64_t nt = trunc ? min((int64_t)*trunc_count, trunc_cap) : (int64_t)(*n_active);
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nt;
         t += n_warps) {
        int64_t rank = t;
        int b_lo = 0, b_hi = kBinsPerTile - 1;
        int64_t tile = -1;
        if (trunc) {
            tile = trunc[t];
            rank = trunc[trunc_cap + t];
            b_lo = trunc[2 * trunc_cap + t] + 1;
        } else if (active_tiles) {
            tile = active_tiles[t];
            if (cut) b_hi = cut[tile];
        }
        const uint32_t np = (tile_cache && tile >= 0) ? tile_cache[tile].n_prefix
                                                      : CLS_PREFIX_UNKNOWN;
        const uint32_t* off = bin_offsets + rank * kBinsPerTile;
        const int b0 = lane * kCollectBins;
        uint32_t o[kCollectBins + 1];
#pragma unroll
        for (int k = 0; k < kCollectBins; ++k) o[k] = off[b0 + k];
        const uint32_t next = __shfl_down_sync(0xffffffffu, o[0], 1);
        o[kCollectBins] = lane < 31 ? next : off[kBinsPerTile];
        const uint32_t first = __shfl_sync(0xffffffffu, o[0], 0);
#pragma unroll
        for (int k = 0; k < kCollectBins; ++k) {
            const int b = b0 + k;
            const uint32_t a = o[k], n = o[k + 1] - o[k];
            if (b < b_lo || b > b_hi || n < (uint32_t)min_bin) continue;
            if (np != CLS_PREFIX_UNKNOWN && a + n - first <= np) continue;
            const int slot = atomicAdd(count, 1);
            if (slot < list_cap) list[slot] = make_uint2(a, n);
        }
    }
}

__global__ void __launch_bounds__(kTB)
sort_bins_kernel(uint64_t* __restrict__ keys, uint64_t* __restrict__ alt,
                 const uint2* __restrict__ list, const int32_t* __restrict__ count,
                 int64_t list_cap, int* __restrict__ work_counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSortSmem& sm = *reinterpret_cast<TileSortSmem*>(smem_raw);
    const int64_t n_items = min((int64_t)*count, list_cap);
    if (n_items == 0) return;  // nothing to sort (the usual case): no queue traffic
    for (;;) {
        if (threadIdx.x == 0) sm.tile = atomicAdd(work_counter, 1);
        __syncthreads();
        const int t = sm.tile;
        if (t >= n_items) break;
        const uint2 it = list[t];
        if (it.y > (uint32_t)kCap) sort_big(sm, keys, alt, it.x, it.y);
        else sort_window(sm, keys, it.x, (int)it.y);
        __syncthreads();
    }
}

static PerDevice g_tiles_blocks;

}  // namespace cls

using namespace cls;

static int64_t list_cap_for(int64_t capacity, int32_t min_bin) {
    return min_bin <= 1 ? 0 : capacity / min_bin + 1;
}

extern "C" size_t cls_sort_tiles_workspace_size(int64_t capacity, int32_t min_bin) {
    return (size_t)(256 + list_cap_for(capacity, min_bin) * sizeof(uint2) + 255) / 256 * 256;
}

extern "C" int cls_sort_tiles(uint64_t* keys, uint64_t* keys_alt, const uint32_t* bin_offsets,
                              const int32_t* active_tiles, const int32_t* n_active_tiles_dev,
                              int64_t total_tiles, int64_t capacity, int32_t min_bin,
                              const uint8_t* cut, const int32_t* trunc,
                              const int32_t* trunc_count, int64_t trunc_cap,
                              const ClsTileCache* tile_cache, int32_t* work_counter,
                              void* workspace, size_t workspace_bytes, cls_stream_t stream) {
    if (!keys || !keys_alt || !bin_offsets || !n_active_tiles_dev || !work_counter ||
        total_tiles <= 0 || capacity < 0 || !workspace ||
        workspace_bytes < cls_sort_tiles_workspace_size(capacity, min_bin) ||
        ((cut || tile_cache) && !active_tiles) ||
        (trunc && (!trunc_count || trunc_cap < total_tiles)) ||
        ((cut || trunc) && min_bin <= 1))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int tiles_blocks = per_device(g_tiles_blocks, [](int dev) {
        cudaFuncSetAttribute(sort_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileSortSmem));
        cudaFuncSetAttribute(sort_bins_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TileSortSmem));
        return resident_blocks(dev, sort_tiles_kernel, kTB, sizeof(TileSortSmem));
    });
    if (min_bin <= 1) {
        cudaMemsetAsync(work_counter, 0, sizeof(int32_t), s);
        sort_tiles_kernel<<<(int)hmin64(total_tiles, tiles_blocks), kTB, sizeof(TileSortSmem),
                            s>>>(keys, keys_alt, bin_offsets, n_active_tiles_dev, active_tiles,
                                 tile_cache, work_counter);
    } else {
        int32_t* count = static_cast<int32_t*>(workspace);
        uint2* list = reinterpret_cast<uint2*>(static_cast<char*>(workspace) + 256);
        const int64_t cap = list_cap_for(capacity, min_bin);
        cudaMemsetAsync(count, 0, sizeof(int32_t), s);
        collect_bins_kernel<<<1024, 256, 0, s>>>(bin_offsets, n_active_tiles_dev, active_tiles,
                                                 cut, trunc, trunc_count, trunc_cap, tile_cache,
                                                 min_bin, list, count, cap, work_counter);
        sort_bins_kernel<<<tiles_blocks, kTB, sizeof(TileSortSmem), s>>>(keys, keys_alt, list,
                                                                          count, cap, work_counter);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
