// Stable LSD radix sort of 64-bit (tile, depth) keys carrying 32-bit values,
// in the single-pass style of Onesweep (Adinets & Merrill, 2022): one upfront
// pass builds the digit histograms of every pass, then each digit pass ranks
// a partition of keys in shared memory, learns the global offset of each of
// its digits by decoupled look-back over the preceding partitions, and
// scatters. Per-tile ranges of the sorted keys follow.
#include "common.cuh"

namespace cls {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;
constexpr int kSortItems = 15;
constexpr int kPartKeys = kSortBlock * kSortItems;  // 3840 keys per partition
constexpr int kWarpKeys = 32 * kSortItems;          // 480 keys per warp
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kMaxPasses = 8;

struct SortSmem {
    uint64_t keys[kPartKeys];
    uint32_t vals[kPartKeys];
    uint32_t whist[kSortWarps][kRadix];
    uint32_t dstart[kRadix];
    int64_t glob[kRadix];
    uint32_t scan_tmp[kSortWarps + 1];
    int part;
};

__device__ __forceinline__ int64_t sort_count(const int64_t* n_dev, int64_t capacity) {
    const int64_t n = *n_dev;
    return n < capacity ? (n < 0 ? 0 : n) : capacity;
}

__global__ void __launch_bounds__(256)
sort_hist_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ n_dev,
                 int64_t capacity, int passes, uint32_t* __restrict__ hist) {
    __shared__ uint32_t sh[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = sort_count(n_dev, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (p * kRadixBits)) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// Exclusive scan of each pass's histogram (one block of 256 per pass).
__global__ void __launch_bounds__(kRadix) sort_hist_scan_kernel(uint32_t* __restrict__ hist) {
    __shared__ uint32_t s[kRadix];
    uint32_t* h = hist + blockIdx.x * kRadix;
    s[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int d = 0; d < kRadix; ++d) {
            const uint32_t c = s[d];
            s[d] = run;
            run += c;
        }
    }
    __syncthreads();
    h[threadIdx.x] = s[threadIdx.x];
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t load_state(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ void store_state(uint32_t* p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// One digit pass. Persistent blocks take partitions in order from a counter.
__global__ void __launch_bounds__(kSortBlock, 2)
sort_pass_kernel(const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                 uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                 const int64_t* __restrict__ n_dev, int64_t capacity, int shift,
                 const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ state,
                 int* __restrict__ part_counter, int32_t* __restrict__ status,
                 int64_t spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
    const int64_t n = sort_count(n_dev, capacity);
    const int64_t n_parts = (n + kPartKeys - 1) / kPartKeys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    for (;;) {
        if (threadIdx.x == 0) sm.part = atomicAdd(part_counter, 1);
        for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortBlock)
            (&sm.whist[0][0])[i] = 0;
        __syncthreads();
        const int part = sm.part;
        if (part >= n_parts) break;
        const int64_t start = (int64_t)part * kPartKeys;

        // Load a warp-contiguous slice and rank keys within the warp.
        uint64_t k[kSortItems];
        uint32_t v[kSortItems];
        uint32_t rank[kSortItems];
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            const int64_t idx = start + warp * kWarpKeys + r * 32 + lane;
            const bool ok = idx < n;
            k[r] = ok ? keys_in[idx] : 0ull;
            v[r] = ok ? vals_in[idx] : 0u;
            const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & (kRadix - 1)) : (uint32_t)kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t base = 0;
            if (ok) base = sm.whist[warp][d];
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) sm.whist[warp][d] = base + __popc(peers);
            __syncwarp();
            rank[r] = ok ? base + __popc(peers & lt) : 0xffffffffu;
        }
        __syncthreads();

        // Per digit: warp prefixes and the partition's total.
        const int d = threadIdx.x;  // kSortBlock == kRadix
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t t = sm.whist[w][d];
            sm.whist[w][d] = total;
            total += t;
        }
        uint32_t* my_state = state + (int64_t)part * kRadix;
        store_state(my_state + d, (part == 0 ? kFlagInc : kFlagAgg) | total);

        // Local start of each digit inside the partition (block scan).
        {
            uint32_t x = total;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) sm.scan_tmp[warp] = x;
            __syncthreads();
            if (warp == 0) {
                uint32_t w = lane < kSortWarps ? sm.scan_tmp[lane] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += y;
                }
                if (lane < kSortWarps) sm.scan_tmp[lane] = w;
            }
            __syncthreads();
            sm.dstart[d] = (warp > 0 ? sm.scan_tmp[warp - 1] : 0u) + x - total;
        }

        // Decoupled look-back for this digit.
        uint32_t prefix = 0;
        if (part > 0) {
            int64_t j = part - 1;
            int64_t spins = 0;
            while (j >= 0) {
                const uint32_t st = load_state(state + j * kRadix + d);
                const uint32_t flag = st & ~kValueMask;
                if (flag == 0) {
                    if (++spins > spin_limit) {
                        set_status(status, CLS_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                prefix += st & kValueMask;
                if (flag == kFlagInc) break;
                --j;
            }
            store_state(my_state + d, kFlagInc | ((prefix + total) & kValueMask));
        }
        sm.glob[d] = (int64_t)digit_base[d] + prefix - sm.dstart[d];
        __syncthreads();

        // Stage the partition in digit order, then write out coalesced runs.
#pragma unroll
        for (int r = 0; r < kSortItems; ++r) {
            if (rank[r] != 0xffffffffu) {
                const uint32_t dg = (uint32_t)((k[r] >> shift) & (kRadix - 1));
                const uint32_t lp = sm.dstart[dg] + sm.whist[warp][dg] + rank[r];
                sm.keys[lp] = k[r];
                sm.vals[lp] = v[r];
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kPartKeys, n - start);
        for (int i = threadIdx.x; i < cnt; i += kSortBlock) {
            const uint64_t key = sm.keys[i];
            const uint32_t dg = (uint32_t)((key >> shift) & (kRadix - 1));
            const int64_t out = sm.glob[dg] + i;
            if (out >= 0 && out < n) {  // always true unless a look-back wait gave up
                keys_out[out] = key;
                vals_out[out] = sm.vals[i];
            }
        }
        __syncthreads();
    }
}

__global__ void sort_copy_kernel(const uint64_t* __restrict__ ka, const uint32_t* __restrict__ va,
                                 uint64_t* __restrict__ kb, uint32_t* __restrict__ vb,
                                 const int64_t* __restrict__ n_dev, int64_t capacity) {
    const int64_t n = sort_count(n_dev, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        kb[i] = ka[i];
        vb[i] = va[i];
    }
}

__global__ void tile_ranges_kernel(const uint64_t* __restrict__ keys,
                                   const int64_t* __restrict__ n_dev, int64_t capacity,
                                   int64_t n_tiles, uint32_t* __restrict__ ranges) {
    const int64_t n = sort_count(n_dev, capacity);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (int64_t)(keys[i] >> 32);
        const int64_t prev = i > 0 ? (int64_t)(keys[i - 1] >> 32) : -1;
        if (t >= n_tiles) continue;  // cannot happen for keys from cls_project_and_bin
        if (t != prev) {
            ranges[2 * t] = (uint32_t)i;
            if (prev >= 0 && prev < n_tiles) ranges[2 * prev + 1] = (uint32_t)i;
        }
        if (i == n - 1) ranges[2 * t + 1] = (uint32_t)n;
    }
}

static PerDevice g_sort_sms;
static PerDevice g_pass_blocks;

}  // namespace cls

using namespace cls;

static int64_t sort_parts(int64_t capacity) { return (capacity + kPartKeys - 1) / kPartKeys; }

static void sort_layout(int64_t capacity, int passes, size_t* off_hist, size_t* off_cnt,
                        size_t* off_state, size_t* total) {
    size_t o = 0;
    *off_hist = o;
    o += (size_t)kMaxPasses * kRadix * sizeof(uint32_t);
    *off_cnt = o;
    o += 64 * sizeof(int);
    *off_state = o;
    o += (size_t)passes * (size_t)sort_parts(capacity) * kRadix * sizeof(uint32_t);
    *total = (o + 255) / 256 * 256;
}

extern "C" size_t cls_sort_workspace_size(int64_t capacity, int32_t key_bits) {
    if (capacity < 0 || key_bits <= 0 || key_bits > 64) return 0;
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    size_t a, b, c, t;
    sort_layout(capacity, passes, &a, &b, &c, &t);
    return t;
}

extern "C" int cls_sort_keys_bounded(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                     uint32_t* vals_alt, const int64_t* n_pairs_dev,
                                     int64_t capacity, int32_t key_bits, uint32_t* ranges,
                                     int64_t n_tiles, int32_t* status_dev, void* workspace,
                                     size_t workspace_bytes, int64_t spin_limit,
                                     cls_stream_t stream) {
    if (capacity < 0 || capacity >= (int64_t)kValueMask || key_bits <= 0 || key_bits > 64 ||
        !n_pairs_dev || !status_dev || !workspace || spin_limit < 0 ||
        workspace_bytes < cls_sort_workspace_size(capacity, key_bits) ||
        (capacity > 0 && (!keys || !vals || !keys_alt || !vals_alt)) || (ranges && n_tiles <= 0))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (ranges) cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 2 * sizeof(uint32_t), s);
    if (capacity == 0) {
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const int sm_count = per_device(g_sort_sms, [](int dev) { return device_sms(dev); });
    const int pass_blocks_max = per_device(g_pass_blocks, [](int dev) {
        cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SortSmem));
        return resident_blocks(dev, sort_pass_kernel, kSortBlock, sizeof(SortSmem));
    });
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    size_t off_hist, off_cnt, off_state, total;
    sort_layout(capacity, passes, &off_hist, &off_cnt, &off_state, &total);
    char* ws = static_cast<char*>(workspace);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + off_hist);
    int* counters = reinterpret_cast<int*>(ws + off_cnt);
    uint32_t* state = reinterpret_cast<uint32_t*>(ws + off_state);
    cudaMemsetAsync(ws, 0, total, s);

    const int64_t parts = sort_parts(capacity);
    const int hist_blocks = (int)hmin64((capacity + 255) / 256, (int64_t)sm_count * 8);
    sort_hist_kernel<<<hist_blocks, 256, 0, s>>>(keys, n_pairs_dev, capacity, passes, hist);
    sort_hist_scan_kernel<<<passes, kRadix, 0, s>>>(hist);
    const int pass_blocks = (int)hmin64(parts, (int64_t)pass_blocks_max);
    uint64_t* kin = keys;
    uint32_t* vin = vals;
    uint64_t* kout = keys_alt;
    uint32_t* vout = vals_alt;
    for (int p = 0; p < passes; ++p) {
        sort_pass_kernel<<<pass_blocks, kSortBlock, sizeof(SortSmem), s>>>(
            kin, vin, kout, vout, n_pairs_dev, capacity, p * kRadixBits, hist + p * kRadix,
            state + (int64_t)p * parts * kRadix, counters + p, status_dev, spin_limit);
        uint64_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != keys) {
        sort_copy_kernel<<<sm_count * 4, 256, 0, s>>>(kin, vin, keys, vals, n_pairs_dev,
                                                        capacity);
    }
    if (ranges) {
        tile_ranges_kernel<<<sm_count * 4, 256, 0, s>>>(keys, n_pairs_dev, capacity, n_tiles,
                                                          ranges);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_sort_keys(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                             uint32_t* vals_alt, const int64_t* n_pairs_dev, int64_t capacity,
                             int32_t key_bits, uint32_t* ranges, int64_t n_tiles,
                             int32_t* status_dev, void* workspace, size_t workspace_bytes,
                             cls_stream_t stream) {
    return cls_sort_keys_bounded(keys, vals, keys_alt, vals_alt, n_pairs_dev, capacity,
                                 key_bits, ranges, n_tiles, status_dev, workspace,
                                 workspace_bytes, CLS_SORT_SPIN_LIMIT, stream);
}
