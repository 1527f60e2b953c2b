// Sphere region of the changed Gaussians and pruning outside it (Sec. 3.3
// "Sphere Pruning"; Supp. "Identifying Changed Gaussians": one sphere per
// cluster at the cluster mean with radius 1.1 x the 98th quantile of the
// members' distances; Supp. "3DGS Optimization in Changed Regions": every 15
// iterations each Gaussian of O^t outside every sphere is removed).
//
// Clusters come from K-Means (the paper's HDBSCAN is a serial third-party
// algorithm): farthest-point initial centres, then Lloyd iterations. Every
// distance is the float32 sequence ((dx*dx + dy*dy) + dz*dz) of rounded
// operations, and cluster sums are exact integers of 2^-24 units, so the
// clustering, the means and the radii do not depend on the order in which
// threads add, and are reproducible bit for bit.
#include "scan.cuh"

namespace cls {

constexpr int kSphBlock = 256;
constexpr int kSphItems = 8;
constexpr int kSphChunk = kSphBlock * kSphItems;
constexpr double kFixedScale = 16777216.0;  // 2^24 units per coordinate

__device__ __forceinline__ float3 point_of(const float* params, int row_stride, const int32_t* idx,
                                           int i) {
    const float4 m = *reinterpret_cast<const float4*>(params + (int64_t)idx[i] * row_stride);
    return make_float3(m.x, m.y, m.z);
}

__device__ __forceinline__ float sq_dist32(float3 p, float cx, float cy, float cz) {
    const float dx = __fsub_rn(p.x, cx), dy = __fsub_rn(p.y, cy), dz = __fsub_rn(p.z, cz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y > v ? y : v;
    }
    return v;
}

// Farthest-point initialisation, one step: nearest[i] = min(nearest[i],
// d2(p_i, centre j-1)) (the first step starts it), then the arg-max over i of
// nearest[i] (ties to the lowest i) as the 64-bit key (bits(d2) << 32) |
// ~i, reduced with atomicMax.
__global__ void __launch_bounds__(kSphBlock)
fpi_round_kernel(const float* __restrict__ params, int row_stride, const int32_t* __restrict__ idx,
                 int n, const float4* __restrict__ centers, int j, float* __restrict__ nearest,
                 unsigned long long* __restrict__ best) {
    const float4 c = centers[j - 1];
    unsigned long long key = 0ull;
    for (int i = blockIdx.x * kSphBlock + threadIdx.x; i < n; i += gridDim.x * kSphBlock) {
        const float d = sq_dist32(point_of(params, row_stride, idx, i), c.x, c.y, c.z);
        const float m = j == 1 ? d : fminf(nearest[i], d);
        nearest[i] = m;
        const unsigned long long k =
            ((unsigned long long)__float_as_uint(m) << 32) | (unsigned long long)(~(uint32_t)i);
        key = k > key ? k : key;
    }
    key = warp_max_u64(key);
    if ((threadIdx.x & 31) == 0 && key) atomicMax(best + j, key);
}

// Centre j = the point chosen by round j (centre 0 = the first point).
__global__ void fpi_pick_kernel(const float* __restrict__ params, int row_stride,
                                const int32_t* __restrict__ idx, float4* __restrict__ centers,
                                const unsigned long long* __restrict__ best, int j) {
    const int i = j == 0 ? 0 : (int)(~(uint32_t)(best[j] & 0xffffffffull));
    const float3 p = point_of(params, row_stride, idx, i);
    centers[j] = make_float4(p.x, p.y, p.z, 0.f);
}

// Lloyd assignment: nearest centre (ties to the lowest cluster), and the
// cluster's exact fixed-point coordinate sums and count, reduced per block in
// shared memory, then added with one 64-bit atomic per (cluster, component).
__global__ void __launch_bounds__(kSphBlock)
kmeans_assign_kernel(const float* __restrict__ params, int row_stride,
                     const int32_t* __restrict__ idx, int n, const float4* __restrict__ centers,
                     int k, int32_t* __restrict__ labels, unsigned long long* __restrict__ sums) {
    __shared__ float4 s_c[CLS_MAX_SPHERES];
    __shared__ unsigned long long s_sum[CLS_MAX_SPHERES][4];
    if (threadIdx.x < k) s_c[threadIdx.x] = centers[threadIdx.x];
    if (threadIdx.x < 4 * CLS_MAX_SPHERES) (&s_sum[0][0])[threadIdx.x] = 0ull;
    __syncthreads();
    for (int i = blockIdx.x * kSphBlock + threadIdx.x; i < n; i += gridDim.x * kSphBlock) {
        const float3 p = point_of(params, row_stride, idx, i);
        int best = 0;
        float bd = sq_dist32(p, s_c[0].x, s_c[0].y, s_c[0].z);
        for (int c = 1; c < k; ++c) {
            const float d = sq_dist32(p, s_c[c].x, s_c[c].y, s_c[c].z);
            if (d < bd) { bd = d; best = c; }
        }
        labels[i] = best;
        atomicAdd(&s_sum[best][0], (unsigned long long)__double2ll_rn((double)p.x * kFixedScale));
        atomicAdd(&s_sum[best][1], (unsigned long long)__double2ll_rn((double)p.y * kFixedScale));
        atomicAdd(&s_sum[best][2], (unsigned long long)__double2ll_rn((double)p.z * kFixedScale));
        atomicAdd(&s_sum[best][3], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 4 * k) {
        const unsigned long long v = (&s_sum[0][0])[threadIdx.x];
        if (v) atomicAdd(sums + threadIdx.x, v);
    }
}

// Lloyd update: each non-empty cluster's centre becomes its exact mean; the
// sums are cleared for the next assignment.
__global__ void kmeans_update_kernel(float4* __restrict__ centers,
                                     unsigned long long* __restrict__ sums, int k) {
    const int c = threadIdx.x;
    if (c >= k) return;
    const long long cnt = (long long)sums[4 * c + 3];
    if (cnt > 0) {
        float v[3];
        for (int a = 0; a < 3; ++a) {
            const double s = (double)(long long)sums[4 * c + a];
            v[a] = __double2float_rn(__ddiv_rn(__ddiv_rn(s, (double)cnt), kFixedScale));
        }
        centers[c] = make_float4(v[0], v[1], v[2], 0.f);
    }
    for (int a = 0; a < 4; ++a) sums[4 * c + a] = 0ull;
}

// Distance of every point to its centre as a sortable key (label << 32) |
// bits(distance), the distance being a non-negative float32.
__global__ void __launch_bounds__(kSphBlock)
sphere_dist_kernel(const float* __restrict__ params, int row_stride,
                   const int32_t* __restrict__ idx, int n, const float4* __restrict__ centers,
                   const int32_t* __restrict__ labels, uint64_t* __restrict__ keys,
                   uint32_t* __restrict__ vals, int32_t* __restrict__ counts,
                   int64_t* __restrict__ n_keys) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_keys = n;
    for (int i = blockIdx.x * kSphBlock + threadIdx.x; i < n; i += gridDim.x * kSphBlock) {
        const int c = labels[i];
        const float4 m = centers[c];
        const float d = __fsqrt_rn(sq_dist32(point_of(params, row_stride, idx, i), m.x, m.y, m.z));
        keys[i] = ((uint64_t)c << 32) | __float_as_uint(d);
        vals[i] = (uint32_t)i;
        atomicAdd(counts + c, 1);
    }
}

// Spheres from the sorted distances: NumPy's linear quantile at 0.98 in
// float64, radius float32(1.1 q); empty clusters get radius -1.
__global__ void sphere_radius_kernel(const uint64_t* __restrict__ keys,
                                     const int32_t* __restrict__ counts,
                                     const float4* __restrict__ centers, int k,
                                     ClsSphere* __restrict__ out, int32_t* __restrict__ counts_out) {
    const int c = threadIdx.x;
    if (c >= k) return;
    int64_t start = 0;
    for (int j = 0; j < c; ++j) start += counts[j];
    const int n = counts[c];
    const float4 m = centers[c];
    float r = -1.0f;
    if (n > 0) {
        const double h = __dmul_rn((double)(n - 1), 0.98);
        const double lo = floor(h);
        const int il = (int)lo, ih = min(il + 1, n - 1);
        const double dl = (double)__uint_as_float((uint32_t)(keys[start + il] & 0xffffffffull));
        const double dh = (double)__uint_as_float((uint32_t)(keys[start + ih] & 0xffffffffull));
        const double q = __dadd_rn(dl, __dmul_rn(__dsub_rn(h, lo), __dsub_rn(dh, dl)));
        r = __double2float_rn(__dmul_rn(1.1, q));
    }
    out[c] = ClsSphere{m.x, m.y, m.z, r};
    if (counts_out) counts_out[c] = n;
}

__device__ __forceinline__ bool inside_spheres(float3 p, const ClsSphere* s, int k) {
    for (int c = 0; c < k; ++c) {
        if (s[c].radius < 0.0f) continue;
        if (sq_dist32(p, s[c].cx, s[c].cy, s[c].cz) <= __fmul_rn(s[c].radius, s[c].radius))
            return true;
    }
    return false;
}

// Pruning, pass 1: for each Gaussian of O^t, inside the spheres or not; a
// removed one gets opacity logit -inf and leaves the active flags; per-chunk
// counts of the kept ones.
__global__ void __launch_bounds__(kSphBlock)
prune_flag_kernel(float* __restrict__ params, int row_stride, uint8_t* __restrict__ active,
                  const int32_t* __restrict__ active_idx, int n_active,
                  const ClsSphere* __restrict__ spheres, int k, uint8_t* __restrict__ keep,
                  int64_t* __restrict__ partials, int32_t* __restrict__ removed,
                  int32_t* __restrict__ n_removed) {
    __shared__ ClsSphere s_sp[CLS_MAX_SPHERES];
    __shared__ int64_t smem[kSphBlock / 32 + 1];
    if (threadIdx.x < k) s_sp[threadIdx.x] = spheres[threadIdx.x];
    __syncthreads();
    int64_t cnt = 0;
    for (int it = 0; it < kSphItems; ++it) {
        const int i = blockIdx.x * kSphChunk + it * kSphBlock + threadIdx.x;
        if (i >= n_active) break;
        const int g = active_idx[i];
        float* row = params + (int64_t)g * row_stride;
        const bool in = inside_spheres(make_float3(row[0], row[1], row[2]), s_sp, k);
        keep[i] = in ? 1 : 0;
        cnt += in;
        if (!in) {
            row[3] = -INFINITY;
            active[g] = 0;
            const int slot = atomicAdd(n_removed, 1);
            if (removed) removed[slot] = g;
        }
    }
    int64_t tot;
    block_exclusive_sum<kSphBlock>(cnt, smem, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Pruning, pass 2: the kept entries of the active list, in order.
__global__ void __launch_bounds__(kSphBlock)
prune_compact_kernel(const int32_t* __restrict__ active_idx, int n_active,
                     const uint8_t* __restrict__ keep, const int64_t* __restrict__ offsets,
                     int32_t* __restrict__ out) {
    __shared__ int64_t smem[kSphBlock / 32 + 1];
    int64_t base = offsets[blockIdx.x];
    for (int it = 0; it < kSphItems; ++it) {
        const int i = blockIdx.x * kSphChunk + it * kSphBlock + threadIdx.x;
        const int64_t f = (i < n_active && keep[i]) ? 1 : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_sum<kSphBlock>(f, smem, tot);
        if (f) out[base + ex] = active_idx[i];
        base += tot;
    }
}

}  // namespace cls

using namespace cls;

namespace {

struct SphLayout {
    size_t nearest, best, sums, centers, labels, keys, vals, keys_alt, vals_alt, counts, npairs,
        status, sort_ws, total;
};

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

SphLayout sph_layout(int32_t n) {
    SphLayout L;
    size_t o = 0;
    const size_t m = n > 0 ? (size_t)n : 1;
    L.nearest = o; o = a256(o + m * 4);
    L.best = o; o = a256(o + CLS_MAX_SPHERES * 8);
    L.sums = o; o = a256(o + CLS_MAX_SPHERES * 4 * 8);
    L.centers = o; o = a256(o + CLS_MAX_SPHERES * 16);
    L.labels = o; o = a256(o + m * 4);
    L.keys = o; o = a256(o + m * 8);
    L.vals = o; o = a256(o + m * 4);
    L.keys_alt = o; o = a256(o + m * 8);
    L.vals_alt = o; o = a256(o + m * 4);
    L.counts = o; o = a256(o + CLS_MAX_SPHERES * 4);
    L.npairs = o; o = a256(o + 8);
    L.status = o; o = a256(o + 4);
    L.sort_ws = o; o = a256(o + cls_sort_workspace_size((int64_t)m, 36));
    L.total = o;
    return L;
}

unsigned grid_for(int64_t n) {
    const int64_t g = hmin64((n + kSphBlock - 1) / kSphBlock, 1024);
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

extern "C" size_t cls_spheres_workspace_size(int32_t n_points) {
    return n_points < 0 ? 0 : sph_layout(n_points).total;
}

extern "C" int cls_fit_spheres(const float* params, int32_t row_stride, const int32_t* idx,
                               int32_t n_points, int32_t k, int32_t iters, ClsSphere* spheres,
                               int32_t* labels_out, int32_t* counts_out, void* workspace,
                               size_t workspace_bytes, cls_stream_t stream) {
    if (!params || !idx || !spheres || !workspace || n_points <= 0 || k < 1 ||
        k > CLS_MAX_SPHERES || k > n_points || iters < 1 || row_stride < 4 ||
        row_stride % 4 != 0 || workspace_bytes < cls_spheres_workspace_size(n_points))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const SphLayout L = sph_layout(n_points);
    char* ws = static_cast<char*>(workspace);
    float* nearest = reinterpret_cast<float*>(ws + L.nearest);
    unsigned long long* best = reinterpret_cast<unsigned long long*>(ws + L.best);
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(ws + L.sums);
    float4* centers = reinterpret_cast<float4*>(ws + L.centers);
    int32_t* labels = labels_out ? labels_out : reinterpret_cast<int32_t*>(ws + L.labels);
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + L.keys);
    uint32_t* vals = reinterpret_cast<uint32_t*>(ws + L.vals);
    int32_t* counts = reinterpret_cast<int32_t*>(ws + L.counts);
    int64_t* npairs = reinterpret_cast<int64_t*>(ws + L.npairs);
    int32_t* status = reinterpret_cast<int32_t*>(ws + L.status);
    const unsigned grid = grid_for(n_points);

    cudaMemsetAsync(best, 0, CLS_MAX_SPHERES * 8, s);
    cudaMemsetAsync(sums, 0, CLS_MAX_SPHERES * 4 * 8, s);
    cudaMemsetAsync(counts, 0, CLS_MAX_SPHERES * 4, s);
    cudaMemsetAsync(status, 0, 4, s);
    fpi_pick_kernel<<<1, 1, 0, s>>>(params, row_stride, idx, centers, best, 0);
    for (int j = 1; j < k; ++j) {
        fpi_round_kernel<<<grid, kSphBlock, 0, s>>>(params, row_stride, idx, n_points, centers, j,
                                                     nearest, best);
        fpi_pick_kernel<<<1, 1, 0, s>>>(params, row_stride, idx, centers, best, j);
    }
    for (int it = 0; it < iters; ++it) {
        kmeans_assign_kernel<<<grid, kSphBlock, 0, s>>>(params, row_stride, idx, n_points,
                                                         centers, k, labels, sums);
        kmeans_update_kernel<<<1, 32, 0, s>>>(centers, sums, k);
    }
    sphere_dist_kernel<<<grid, kSphBlock, 0, s>>>(params, row_stride, idx, n_points, centers,
                                                   labels, keys, vals, counts, npairs);
    CLS_CHECK_LAUNCH();
    const int rc = cls_sort_keys(keys, vals, reinterpret_cast<uint64_t*>(ws + L.keys_alt),
                                 reinterpret_cast<uint32_t*>(ws + L.vals_alt), npairs, n_points,
                                 36, nullptr, 0, status, ws + L.sort_ws,
                                 cls_sort_workspace_size(n_points, 36), stream);
    if (rc != CLS_OK) return rc;
    sphere_radius_kernel<<<1, 32, 0, s>>>(keys, counts, centers, k, spheres, counts_out);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" size_t cls_prune_workspace_size(int32_t n_active) {
    if (n_active < 0) return 0;
    const int64_t chunks = ((int64_t)n_active + kSphChunk - 1) / kSphChunk;
    return a256((size_t)(chunks + 1) * 8) + a256((size_t)n_active + 1) +
           a256((size_t)n_active * 4 + 4);
}

extern "C" int cls_prune_outside_spheres(float* params, int32_t row_stride, uint8_t* active,
                                         int32_t* active_idx, int32_t n_active,
                                         int32_t* n_active_dev, const ClsSphere* spheres,
                                         int32_t k, int32_t* removed, int32_t* n_removed_dev,
                                         void* workspace, size_t workspace_bytes,
                                         cls_stream_t stream) {
    if (!params || !active || !active_idx || !n_active_dev || !spheres || !n_removed_dev ||
        !workspace || n_active < 0 || k < 1 || k > CLS_MAX_SPHERES || row_stride < 4 ||
        row_stride % 4 != 0 || workspace_bytes < cls_prune_workspace_size(n_active))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    cudaMemsetAsync(n_removed_dev, 0, 4, s);
    if (n_active == 0) {
        cudaMemsetAsync(n_active_dev, 0, 4, s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const int64_t chunks = ((int64_t)n_active + kSphChunk - 1) / kSphChunk;
    char* ws = static_cast<char*>(workspace);
    int64_t* partials = reinterpret_cast<int64_t*>(ws);
    uint8_t* keep = reinterpret_cast<uint8_t*>(ws + a256((size_t)(chunks + 1) * 8));
    int32_t* tmp = reinterpret_cast<int32_t*>(ws + a256((size_t)(chunks + 1) * 8) +
                                              a256((size_t)n_active + 1));
    prune_flag_kernel<<<(unsigned)chunks, kSphBlock, 0, s>>>(
        params, row_stride, active, active_idx, n_active, spheres, k, keep, partials, removed,
        n_removed_dev);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, chunks, nullptr, n_active_dev, -1,
                                            nullptr);
    prune_compact_kernel<<<(unsigned)chunks, kSphBlock, 0, s>>>(active_idx, n_active, keep,
                                                                partials, tmp);
    cudaMemcpyAsync(active_idx, tmp, (size_t)n_active * 4, cudaMemcpyDeviceToDevice, s);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
