// Densification restricted to O^t (Supp. "History Recovery": duplication and
// pruning only affect O^t; Supp. "Implementation Details": the base 3DGS
// optimiser's adaptive density control). Statistics per Gaussian row: the
// accumulated norm of the NDC-space gradient of the projected centre over
// the views where it is visible, the number of those observations, and the
// largest screen radius. A densification step classifies every Gaussian of
// O^t (clone, split into two, prune) with float32 comparisons against
// thresholds the caller rounds once from float64, writes the new rows in
// rank order (per Gaussian: its clone, then its children) and removes the
// split and pruned originals (opacity logit -inf, active flag 0).
#include "scan.cuh"

namespace cls {

constexpr int kDBlock = 256;
constexpr int kG2 = 12;

// One thread per Gaussian of O^t: its views in order.
__global__ void __launch_bounds__(kDBlock)
densify_accumulate_kernel(const ClsView* __restrict__ views, int first_view, int n_views,
                          const ClsProjected* __restrict__ records,
                          const float* __restrict__ grad2d, const int32_t* __restrict__ active_idx,
                          int n_active, float* __restrict__ accum, float* __restrict__ denom,
                          float* __restrict__ max_radius) {
    const float nv = (float)n_views;
    const int a = blockIdx.x * kDBlock + threadIdx.x;
    if (a >= n_active) return;
    const int g = active_idx[a];
    float acc = accum[g], den = denom[g], mr = max_radius[g];
    for (int j = first_view; j < first_view + n_views; ++j) {
        const ClsView& v = views[j];
        const int r = records[v.rec_base + g].radius;
        if (r <= 0) continue;
        const float* d = grad2d + (v.g2_base + a) * kG2;
        const float gx = __fmul_rn(d[0], 0.5f * (float)v.cam.width * nv);
        const float gy = __fmul_rn(d[1], 0.5f * (float)v.cam.height * nv);
        acc = __fadd_rn(acc, __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy))));
        den += 1.0f;
        mr = fmaxf(mr, (float)r);
    }
    accum[g] = acc;
    denom[g] = den;
    max_radius[g] = mr;
}

__device__ __forceinline__ float max3(float4 v) { return fmaxf(fmaxf(v.x, v.y), v.z); }

// kind bits: 1 clone kept, 2 child 0 kept, 4 child 1 kept, 8 original removed
__device__ __forceinline__ int classify(const float* row, float acc, float den, float maxr,
                                       const ClsDensifyRule& R) {
    const float4 ls = *reinterpret_cast<const float4*>(row + 4);
    const float avg = den > 0.f ? __fdiv_rn(acc, den) : 0.f;
    const float mls = max3(ls);
    const bool sel = avg >= R.grad_threshold;
    const bool clone = sel && mls <= R.clone_log_scale;
    const bool split = sel && mls > R.clone_log_scale;
    const float logit = row[3];
    const bool low = logit < R.min_logit || (R.big && (maxr > 20.0f || mls > R.big_log_scale));
    int kind = (split || low) ? 8 : 0;
    if (clone && !low) kind |= 1;
    if (split) {
        const float cmls =
            max3(make_float4(__fsub_rn(ls.x, R.log_shrink), __fsub_rn(ls.y, R.log_shrink),
                             __fsub_rn(ls.z, R.log_shrink), 0.f));
        const bool child_low = logit < R.min_logit || (R.big && cmls > R.big_log_scale);
        if (!child_low) kind |= 6;
    }
    return kind;
}

__device__ __forceinline__ int n_new_of(int k) {
    return (k & 1) + ((k >> 1) & 1) + ((k >> 2) & 1);
}

// partials[0][block]: new rows of the block; partials[1][block]: kept originals.
__global__ void __launch_bounds__(kDBlock)
densify_count_kernel(const float* __restrict__ params, int stride,
                     const int32_t* __restrict__ active_idx, int n_active,
                     const float* __restrict__ accum, const float* __restrict__ denom,
                     const float* __restrict__ max_radius, ClsDensifyRule R,
                     uint8_t* __restrict__ kind, int64_t* __restrict__ new_partials,
                     int64_t* __restrict__ keep_partials) {
    __shared__ int64_t smem[kDBlock / 32 + 1];
    const int a = blockIdx.x * kDBlock + threadIdx.x;
    int k = 8;
    if (a < n_active) {
        const int g = active_idx[a];
        k = classify(params + (int64_t)g * stride, accum[g], denom[g], max_radius[g], R);
        kind[a] = (uint8_t)k;
    }
    int64_t tot;
    block_exclusive_sum<kDBlock>((int64_t)(a < n_active ? n_new_of(k) : 0), smem, tot);
    if (threadIdx.x == 0) new_partials[blockIdx.x] = tot;
    block_exclusive_sum<kDBlock>((int64_t)((k & 8) ? 0 : 1), smem, tot);
    if (threadIdx.x == 0) keep_partials[blockIdx.x] = tot;
}

// New rows go to ids n + rank (rank order: per Gaussian its clone, then its
// children), with zero Adam moments. The next active list is the kept
// originals in order, then the new ids; counts[0] = new rows, counts[1] =
// kept originals, counts[2] = the new active count.
__global__ void __launch_bounds__(kDBlock)
densify_write_kernel(float* __restrict__ params, float* __restrict__ adam_m,
                     float* __restrict__ adam_v, int stride, int n, uint8_t* __restrict__ active,
                     const int32_t* __restrict__ active_idx, int n_active,
                     const uint8_t* __restrict__ kind, const int64_t* __restrict__ new_offsets,
                     const int64_t* __restrict__ keep_offsets, const float* __restrict__ z,
                     ClsDensifyRule R, int32_t* __restrict__ new_src,
                     int32_t* __restrict__ active_out, int32_t* __restrict__ counts,
                     uint8_t* __restrict__ removed) {
    __shared__ int64_t smem[kDBlock / 32 + 1];
    const int a = blockIdx.x * kDBlock + threadIdx.x;
    const int k = a < n_active ? kind[a] : 8;
    int64_t tot;
    int64_t o = new_offsets[blockIdx.x] +
                block_exclusive_sum<kDBlock>((int64_t)(a < n_active ? n_new_of(k) : 0), smem, tot);
    const int64_t keep = keep_offsets[blockIdx.x] +
                         block_exclusive_sum<kDBlock>((int64_t)((k & 8) ? 0 : 1), smem, tot);
    if (a == 0) counts[2] = counts[0] + counts[1];
    if (a >= n_active) return;
    const int n_keep = counts[1];
    const int g = active_idx[a];
    float* row = params + (int64_t)g * stride;
    auto start_row = [&](int64_t r) -> float* {
        float* dst = params + (n + r) * stride;
        float* dm = adam_m + (n + r) * stride;
        float* dv = adam_v + (n + r) * stride;
        for (int i = 0; i < stride; ++i) {
            dst[i] = row[i];
            dm[i] = 0.f;
            dv[i] = 0.f;
        }
        new_src[r] = g;
        active[n + r] = 1;
        active_out[n_keep + r] = (int32_t)(n + r);
        return dst;
    };
    if (k & 1) start_row(o++);
    if (k & 6) {
        const float4 m = *reinterpret_cast<const float4*>(row);
        const float4 ls = *reinterpret_cast<const float4*>(row + 4);
        const float4 q = *reinterpret_cast<const float4*>(row + 8);
        // rotation of the normalised quaternion (w, x, y, z) and scales
        const float n2 = radd(radd(radd(rmul(q.x, q.x), rmul(q.y, q.y)), rmul(q.z, q.z)),
                              rmul(q.w, q.w));
        const float nr = rsqrt_rn(n2);
        const float w = rdiv(q.x, nr), x = rdiv(q.y, nr), y = rdiv(q.z, nr), zq = rdiv(q.w, nr);
        const float xx = rmul(x, x), yy = rmul(y, y), zz2 = rmul(zq, zq);
        const float xy = rmul(x, y), xz = rmul(x, zq), yz = rmul(y, zq);
        const float wx = rmul(w, x), wy = rmul(w, y), wz = rmul(w, zq);
        const float Rm[9] = {rsub(1.0f, rmul(2.0f, radd(yy, zz2))), rmul(2.0f, rsub(xy, wz)),
                             rmul(2.0f, radd(xz, wy)),                rmul(2.0f, radd(xy, wz)),
                             rsub(1.0f, rmul(2.0f, radd(xx, zz2))), rmul(2.0f, rsub(yz, wx)),
                             rmul(2.0f, rsub(xz, wy)),                rmul(2.0f, radd(yz, wx)),
                             rsub(1.0f, rmul(2.0f, radd(xx, yy)))};
        const float s[3] = {exp_cw(ls.x), exp_cw(ls.y), exp_cw(ls.z)};
        for (int c2 = 0; c2 < 2; ++c2) {
            const float* zz = z + ((int64_t)a * 2 + c2) * 3;
            const float v[3] = {s[0] * zz[0], s[1] * zz[1], s[2] * zz[2]};
            float* dst = start_row(o++);
            dst[0] = m.x + (Rm[0] * v[0] + Rm[1] * v[1] + Rm[2] * v[2]);
            dst[1] = m.y + (Rm[3] * v[0] + Rm[4] * v[1] + Rm[5] * v[2]);
            dst[2] = m.z + (Rm[6] * v[0] + Rm[7] * v[1] + Rm[8] * v[2]);
            dst[4] = __fsub_rn(ls.x, R.log_shrink);
            dst[5] = __fsub_rn(ls.y, R.log_shrink);
            dst[6] = __fsub_rn(ls.z, R.log_shrink);
        }
    }
    if (removed) removed[a] = (k & 8) ? 1 : 0;
    if (k & 8) {
        row[3] = -INFINITY;
        active[g] = 0;
    } else {
        active_out[keep] = g;
    }
}

// Opacity reset of O^t (the base optimiser's periodic reset): logit =
// min(logit, limit); the Adam moments of the opacity entry restart at zero.
__global__ void __launch_bounds__(kDBlock)
opacity_reset_kernel(float* __restrict__ params, float* __restrict__ adam_m,
                     float* __restrict__ adam_v, int stride, const int32_t* __restrict__ active_idx,
                     int n_active, float limit) {
    const int a = blockIdx.x * kDBlock + threadIdx.x;
    if (a >= n_active) return;
    const int64_t i = (int64_t)active_idx[a] * stride + 3;
    params[i] = fminf(params[i], limit);
    adam_m[i] = 0.f;
    adam_v[i] = 0.f;
}

}  // namespace cls

using namespace cls;

extern "C" int cls_densify_accumulate(const ClsView* views_dev, int32_t first_view,
                                      int32_t n_views, const ClsProjected* records,
                                      const float* grad2d, const int32_t* active_idx,
                                      int32_t n_active, float* accum, float* denom,
                                      float* max_radius, cls_stream_t stream) {
    if (!views_dev || !records || !grad2d || !active_idx || !accum || !denom || !max_radius ||
        n_active < 0 || n_views <= 0 || first_view < 0)
        return CLS_ERR_INVALID_ARG;
    if (n_active > 0)
        densify_accumulate_kernel<<<(n_active + kDBlock - 1) / kDBlock, kDBlock, 0,
                                    as_stream(stream)>>>(views_dev, first_view, n_views, records,
                                                         grad2d, active_idx, n_active, accum,
                                                         denom, max_radius);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" size_t cls_densify_workspace_size(int32_t n_active) {
    if (n_active < 0) return 0;
    const size_t blocks = ((size_t)n_active + kDBlock - 1) / kDBlock;
    return 2 * (((blocks + 1) * 8 + 255) / 256 * 256) + ((size_t)n_active + 256) / 256 * 256;
}

extern "C" int cls_densify(float* params, float* adam_m, float* adam_v, int32_t row_stride,
                           int32_t n, int64_t capacity, uint8_t* active,
                           const int32_t* active_idx, int32_t n_active, const float* accum,
                           const float* denom, const float* max_radius,
                           const ClsDensifyRule* rule, const float* z, int32_t* new_src,
                           int32_t* active_idx_out, int32_t* counts_dev, uint8_t* removed,
                           void* workspace, size_t workspace_bytes, cls_stream_t stream) {
    if (!params || !adam_m || !adam_v || !active || !accum || !denom || !max_radius || !rule ||
        !active_idx_out || !counts_dev || !workspace ||
        (n_active > 0 && (!active_idx || !z || !new_src)) || n < 0 || n_active < 0 ||
        n_active > n || row_stride < 16 || row_stride % 4 != 0 ||
        capacity < (int64_t)n + 2 * (int64_t)n_active ||
        capacity > INT32_MAX || active_idx_out == active_idx ||
        workspace_bytes < cls_densify_workspace_size(n_active))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (n_active == 0) {
        cudaMemsetAsync(counts_dev, 0, 3 * sizeof(int32_t), s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const ClsDensifyRule R = *rule;
    const int64_t blocks = ((int64_t)n_active + kDBlock - 1) / kDBlock;
    const size_t part_bytes = (size_t)((blocks + 1) * 8 + 255) / 256 * 256;
    int64_t* new_partials = static_cast<int64_t*>(workspace);
    int64_t* keep_partials =
        reinterpret_cast<int64_t*>(static_cast<uint8_t*>(workspace) + part_bytes);
    uint8_t* kind = static_cast<uint8_t*>(workspace) + 2 * part_bytes;
    densify_count_kernel<<<(unsigned)blocks, kDBlock, 0, s>>>(
        params, row_stride, active_idx, n_active, accum, denom, max_radius, R, kind,
        new_partials, keep_partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(new_partials, blocks, nullptr, counts_dev, -1,
                                            nullptr);
    scan_partials_kernel<<<1, 1024, 0, s>>>(keep_partials, blocks, nullptr, counts_dev + 1, -1,
                                            nullptr);
    densify_write_kernel<<<(unsigned)blocks, kDBlock, 0, s>>>(
        params, adam_m, adam_v, row_stride, n, active, active_idx, n_active, kind, new_partials,
        keep_partials, z, R, new_src, active_idx_out, counts_dev, removed);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_opacity_reset(float* params, float* adam_m, float* adam_v, int32_t row_stride,
                                 const int32_t* active_idx, int32_t n_active, float limit,
                                 cls_stream_t stream) {
    if (!params || !adam_m || !adam_v || !active_idx || n_active < 0 || row_stride < 4)
        return CLS_ERR_INVALID_ARG;
    if (n_active > 0)
        opacity_reset_kernel<<<(n_active + kDBlock - 1) / kDBlock, kDBlock, 0,
                               as_stream(stream)>>>(params, adam_m, adam_v, row_stride,
                                                    active_idx, n_active, limit);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
