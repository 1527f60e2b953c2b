// New-point sampling for appearing objects (Sec. 3.2 "Gaussian Sampling for
// New Objects", New Point Sampling; Supp. Full-Scene and Region Point
// Sampling) and the base method's initialisation of a point cloud. The host
// drives the rounds (each needs the count of points the vote kept); every
// step of a round runs here or in the lifting and K-Means entry points.
// Points are rows of four floats (x, y, z, unused) so the vote and the
// clustering read them like parameter rows. All arithmetic that decides a
// kept point is a fixed float32 sequence of rounded operations on the given
// random inputs.
#include "scan.cuh"

namespace cls {

constexpr int kSmpBlock = 256;

// float <-> unsigned key, monotone in the float order
__device__ __forceinline__ uint32_t fkey(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fval(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void bbox_init_kernel(uint32_t* keys) {
    if (threadIdx.x < 3) keys[threadIdx.x] = 0xffffffffu;       // min
    else if (threadIdx.x < 6) keys[threadIdx.x] = 0u;           // max
}

__global__ void __launch_bounds__(kSmpBlock)
bbox_kernel(const float* __restrict__ params, int n, int row_stride, uint32_t* __restrict__ keys) {
    uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (int i = blockIdx.x * kSmpBlock + threadIdx.x; i < n; i += gridDim.x * kSmpBlock) {
        const float* r = params + (int64_t)i * row_stride;
        for (int a = 0; a < 3; ++a) {
            const uint32_t k = fkey(r[a]);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + a, lo[a]);
            atomicMax(keys + 3 + a, hi[a]);
        }
    }
}

__global__ void bbox_decode_kernel(const uint32_t* keys, float* lohi) {
    if (threadIdx.x < 6) lohi[threadIdx.x] = fval(keys[threadIdx.x]);
}

// p = min + u (max - min) per axis.
__global__ void __launch_bounds__(kSmpBlock)
box_sample_kernel(const float* __restrict__ lohi, const float* __restrict__ u, int n,
                  float* __restrict__ out) {
    const int i = blockIdx.x * kSmpBlock + threadIdx.x;
    if (i >= n) return;
    float p[3];
    for (int a = 0; a < 3; ++a)
        p[a] = __fadd_rn(lohi[a], __fmul_rn(u[3 * i + a], __fsub_rn(lohi[3 + a], lohi[a])));
    reinterpret_cast<float4*>(out)[i] = make_float4(p[0], p[1], p[2], 0.f);
}

// Rows idx[0 .. n) of `src` (stride `stride`, mean first) to packed points.
__global__ void __launch_bounds__(kSmpBlock)
gather_points_kernel(const float* __restrict__ src, int stride, const int32_t* __restrict__ idx,
                     const int32_t* __restrict__ n_dev, int n_max, float* __restrict__ out) {
    const int n = n_dev ? min(*n_dev, n_max) : n_max;
    for (int i = blockIdx.x * kSmpBlock + threadIdx.x; i < n; i += gridDim.x * kSmpBlock) {
        const float* r = src + (int64_t)(idx ? idx[i] : i) * stride;
        reinterpret_cast<float4*>(out)[i] = make_float4(r[0], r[1], r[2], 0.f);
    }
}

__device__ __forceinline__ float sq_dist3(float4 p, float cx, float cy, float cz) {
    const float dx = __fsub_rn(p.x, cx), dy = __fsub_rn(p.y, cy), dz = __fsub_rn(p.z, cz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Furthest member of each cluster (ties to the lowest position):
// key (bits(d2) << 32) | ~position, max-reduced per cluster.
__global__ void __launch_bounds__(kSmpBlock)
cluster_far_kernel(const float* __restrict__ points, int n, const int32_t* __restrict__ labels,
                   const ClsSphere* __restrict__ spheres, unsigned long long* __restrict__ far) {
    for (int i = blockIdx.x * kSmpBlock + threadIdx.x; i < n; i += gridDim.x * kSmpBlock) {
        const int c = labels[i];
        const float4 p = reinterpret_cast<const float4*>(points)[i];
        const float d = sq_dist3(p, spheres[c].cx, spheres[c].cy, spheres[c].cz);
        atomicMax(far + c,
                  ((unsigned long long)__float_as_uint(d) << 32) | (unsigned long long)(~(uint32_t)i));
    }
}

// |p_far - c| per cluster (zero for an empty one).
__global__ void cluster_absv_kernel(const float* __restrict__ points,
                                    const ClsSphere* __restrict__ spheres,
                                    const int32_t* __restrict__ counts,
                                    const unsigned long long* __restrict__ far, int k,
                                    float4* __restrict__ absv) {
    const int c = threadIdx.x;
    if (c >= k) return;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (counts[c] > 0) {
        const int i = (int)(~(uint32_t)(far[c] & 0xffffffffull));
        const float4 p = reinterpret_cast<const float4*>(points)[i];
        v = make_float4(fabsf(__fsub_rn(p.x, spheres[c].cx)), fabsf(__fsub_rn(p.y, spheres[c].cy)),
                        fabsf(__fsub_rn(p.z, spheres[c].cz)), 0.f);
    }
    absv[c] = v;
}

// Mixture draw: component = first j with floor(u |O|) < (members of 0..j),
// p = c_j + sqrt(|v_j|) z per axis.
__global__ void __launch_bounds__(kSmpBlock)
mixture_sample_kernel(const ClsSphere* __restrict__ spheres, const float4* __restrict__ absv,
                      const int32_t* __restrict__ counts, int k, const float* __restrict__ u,
                      const float* __restrict__ z, int m, float* __restrict__ out) {
    __shared__ int64_t s_cum[CLS_MAX_SPHERES];
    if (threadIdx.x == 0) {
        int64_t c = 0;
        for (int j = 0; j < k; ++j) { c += counts[j]; s_cum[j] = c; }
    }
    __syncthreads();
    const int i = blockIdx.x * kSmpBlock + threadIdx.x;
    if (i >= m) return;
    const int64_t total = s_cum[k - 1];
    const int64_t t = (int64_t)floor(__dmul_rn((double)u[i], (double)total));
    int j = 0;
    while (j < k - 1 && !(t < s_cum[j])) ++j;
    const float4 v = absv[j];
    const float px = __fadd_rn(spheres[j].cx, __fmul_rn(__fsqrt_rn(v.x), z[3 * i]));
    const float py = __fadd_rn(spheres[j].cy, __fmul_rn(__fsqrt_rn(v.y), z[3 * i + 1]));
    const float pz = __fadd_rn(spheres[j].cz, __fmul_rn(__fsqrt_rn(v.z), z[3 * i + 2]));
    reinterpret_cast<float4*>(out)[i] = make_float4(px, py, pz, 0.f);
}

// Mean squared distance to the three nearest other points (fewer if fewer
// exist), ((d1 + d2) + d3) / count in float32 with d ascending, at least 1e-7.
// Brute force over shared-memory tiles of the point set.
__global__ void __launch_bounds__(kSmpBlock)
knn3_kernel(const float* __restrict__ points, int n, float* __restrict__ mean_sq) {
    __shared__ float4 s_p[kSmpBlock];
    const int i = blockIdx.x * kSmpBlock + threadIdx.x;
    const float4 p = i < n ? reinterpret_cast<const float4*>(points)[i] : make_float4(0, 0, 0, 0);
    float d0 = INFINITY, d1 = INFINITY, d2 = INFINITY;
    for (int base = 0; base < n; base += kSmpBlock) {
        __syncthreads();
        if (base + threadIdx.x < n)
            s_p[threadIdx.x] = reinterpret_cast<const float4*>(points)[base + threadIdx.x];
        __syncthreads();
        const int cnt = min(kSmpBlock, n - base);
        for (int q = 0; q < cnt; ++q) {
            if (base + q == i) continue;
            const float d = sq_dist3(s_p[q], p.x, p.y, p.z);
            if (d < d2) {
                if (d < d1) {
                    d2 = d1;
                    if (d < d0) { d1 = d0; d0 = d; } else { d1 = d; }
                } else {
                    d2 = d;
                }
            }
        }
    }
    if (i >= n) return;
    const int cnt = min(3, n - 1);
    float r = 1e-7f;
    if (cnt >= 1) {
        float s = d0;
        if (cnt >= 2) s = __fadd_rn(s, d1);
        if (cnt >= 3) s = __fadd_rn(s, d2);
        r = fmaxf(__fdiv_rn(s, (float)cnt), 1e-7f);
    }
    mean_sq[i] = r;
}

// Parameter rows of new points: mean, opacity logit of 0.1, isotropic
// log-scale 0.5 log(mean squared distance), identity rotation, SH zero.
__global__ void __launch_bounds__(kSmpBlock)
init_rows_kernel(const float* __restrict__ points, const float* __restrict__ mean_sq, int n,
                 int row_stride, float* __restrict__ rows) {
    const int i = blockIdx.x * kSmpBlock + threadIdx.x;
    if (i >= n) return;
    const float4 p = reinterpret_cast<const float4*>(points)[i];
    float* r = rows + (int64_t)i * row_stride;
    const float ls = 0.5f * logf(mean_sq[i]);
    r[0] = p.x; r[1] = p.y; r[2] = p.z;
    r[3] = logf(0.1f / 0.9f);
    r[4] = ls; r[5] = ls; r[6] = ls; r[7] = 0.f;
    r[8] = 1.f; r[9] = 0.f; r[10] = 0.f; r[11] = 0.f;
    for (int k = 12; k < row_stride; ++k) r[k] = 0.f;
}

unsigned grid_of(int64_t n) {
    const int64_t g = (n + kSmpBlock - 1) / kSmpBlock;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace cls

using namespace cls;

extern "C" int cls_points_bbox(const float* params, int32_t n, int32_t row_stride, float* lohi,
                               uint32_t* scratch, cls_stream_t stream) {
    if (!params || !lohi || !scratch || n <= 0 || row_stride < 3) return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    bbox_init_kernel<<<1, 32, 0, s>>>(scratch);
    bbox_kernel<<<grid_of(n), kSmpBlock, 0, s>>>(params, n, row_stride, scratch);
    bbox_decode_kernel<<<1, 32, 0, s>>>(scratch, lohi);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_box_sample(const float* lohi, const float* u, int32_t n, float* points,
                              cls_stream_t stream) {
    if (!lohi || !u || !points || n < 0) return CLS_ERR_INVALID_ARG;
    if (n > 0)
        box_sample_kernel<<<(n + kSmpBlock - 1) / kSmpBlock, kSmpBlock, 0, as_stream(stream)>>>(
            lohi, u, n, points);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_gather_points(const float* src, int32_t stride, const int32_t* idx,
                                 const int32_t* n_dev, int32_t n_max, float* points,
                                 cls_stream_t stream) {
    if (!src || !points || stride < 3 || n_max < 0) return CLS_ERR_INVALID_ARG;
    if (n_max > 0)
        gather_points_kernel<<<grid_of(n_max), kSmpBlock, 0, as_stream(stream)>>>(
            src, stride, idx, n_dev, n_max, points);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_region_mixture(const float* points, int32_t n, const int32_t* labels,
                                  const ClsSphere* clusters, const int32_t* counts, int32_t k,
                                  unsigned long long* scratch, float* absv,
                                  cls_stream_t stream) {
    if (!points || !labels || !clusters || !counts || !scratch || !absv || n <= 0 || k < 1 ||
        k > CLS_MAX_SPHERES)
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    cudaMemsetAsync(scratch, 0, CLS_MAX_SPHERES * sizeof(unsigned long long), s);
    cluster_far_kernel<<<grid_of(n), kSmpBlock, 0, s>>>(points, n, labels, clusters, scratch);
    cluster_absv_kernel<<<1, 32, 0, s>>>(points, clusters, counts, scratch, k,
                                         reinterpret_cast<float4*>(absv));
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_mixture_sample(const ClsSphere* clusters, const float* absv,
                                  const int32_t* counts, int32_t k, const float* u,
                                  const float* z, int32_t m, float* points,
                                  cls_stream_t stream) {
    if (!clusters || !absv || !counts || !u || !z || !points || k < 1 || k > CLS_MAX_SPHERES ||
        m < 0)
        return CLS_ERR_INVALID_ARG;
    if (m > 0)
        mixture_sample_kernel<<<(m + kSmpBlock - 1) / kSmpBlock, kSmpBlock, 0,
                                as_stream(stream)>>>(
            clusters, reinterpret_cast<const float4*>(absv), counts, k, u, z, m, points);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_init_point_gaussians(const float* points, int32_t n, int32_t row_stride,
                                        float* mean_sq, float* rows, cls_stream_t stream) {
    if (!points || !mean_sq || !rows || n < 0 || row_stride < 16 || row_stride % 4 != 0)
        return CLS_ERR_INVALID_ARG;
    if (n > 0) {
        cudaStream_t s = as_stream(stream);
        knn3_kernel<<<(n + kSmpBlock - 1) / kSmpBlock, kSmpBlock, 0, s>>>(points, n, mean_sq);
        init_rows_kernel<<<(n + kSmpBlock - 1) / kSmpBlock, kSmpBlock, 0, s>>>(points, mean_sq, n,
                                                                              row_stride, rows);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
