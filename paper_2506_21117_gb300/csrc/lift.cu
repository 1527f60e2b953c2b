// Change-mask lifting: per-Gaussian majority vote over the new views
// (Sec. 3.2 "Mask Majority Voting"; Supp. "Identifying Changed 3D Regions via
// Majority Voting", voting equation), then compaction of O^t into an
// ascending index list.
#include <mutex>

#include "scan.cuh"

namespace cls {

constexpr int kLiftBlock = 256;
constexpr int kLiftItems = 8;
constexpr int kLiftChunk = kLiftBlock * kLiftItems;

__global__ void scan_partials_kernel(int64_t* partials, int64_t n, int64_t* total64,
                                     int32_t* total32, int64_t capacity, int32_t* status) {
    __shared__ int64_t smem[1024 / 32 + 1];
    int64_t carry = 0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < n ? partials[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_sum<1024>(v, smem, tot);
        if (i < n) partials[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (total64) *total64 = carry;
        if (total32) *total32 = (int32_t)carry;
        if (capacity >= 0 && carry > capacity) set_status(status, CLS_ERR_CAPACITY);
    }
}

// One thread per Gaussian: votes over the scene's views, flag + counts, and a
// per-block count of active Gaussians.
__global__ void __launch_bounds__(kLiftBlock)
lift_vote_kernel(const float* __restrict__ params, int n, int row_stride,
                 const ClsView* __restrict__ views, int first_view, int n_views,
                 const uint8_t* __restrict__ masks, int vote_mode, uint8_t* __restrict__ active_out,
                 int32_t* __restrict__ votes_out, int64_t* __restrict__ partials) {
    __shared__ int64_t smem[kLiftBlock / 32 + 1];
    int64_t cnt = 0;
    for (int it = 0; it < kLiftItems; ++it) {
        const int64_t g = (int64_t)blockIdx.x * kLiftChunk + it * kLiftBlock + threadIdx.x;
        if (g >= n) break;
        const float4 mean = *reinterpret_cast<const float4*>(params + g * row_stride);
        int c = 0, o = 0;
        for (int j = first_view; j < first_view + n_views; ++j) {
            const ClsCamera& cam = views[j].cam;
            float px, py, pz;
            camera_point(cam, mean.x, mean.y, mean.z, px, py, pz);
            bool inside = pz > cam.znear;
            float u = 0.f, v = 0.f;
            if (inside) {
                u = radd(rmul(cam.fx, rdiv(px, pz)), cam.cx);
                v = radd(rmul(cam.fy, rdiv(py, pz)), cam.cy);
                inside = (u >= 0.0f) && (u < (float)cam.width) && (v >= 0.0f) &&
                         (v < (float)cam.height);
            }
            if (inside) {
                const int iu = (int)floorf(u), iv = (int)floorf(v);
                c += masks[views[j].pix_base + (int64_t)iv * cam.width + iu] != 0;
            } else {
                ++o;
            }
        }
        const bool act = vote_mode == 1 ? (c == n_views)
                                        : (4 * o < 3 * n_views) && (n_views < 2 * c);
        active_out[g] = act ? 1 : 0;
        if (votes_out) {
            votes_out[2 * g] = c;
            votes_out[2 * g + 1] = o;
        }
        cnt += act;
    }
    int64_t tot;
    block_exclusive_sum<kLiftBlock>(cnt, smem, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Ascending compaction of a uint8 flag array given per-chunk offsets.
__global__ void __launch_bounds__(kLiftBlock)
compact_flags_kernel(const uint8_t* __restrict__ flags, int64_t n,
                     const int64_t* __restrict__ offsets, int32_t* __restrict__ out) {
    __shared__ int64_t smem[kLiftBlock / 32 + 1];
    int64_t base = offsets[blockIdx.x];
    for (int it = 0; it < kLiftItems; ++it) {
        const int64_t g = (int64_t)blockIdx.x * kLiftChunk + it * kLiftBlock + threadIdx.x;
        const int64_t f = (g < n && flags[g]) ? 1 : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_sum<kLiftBlock>(f, smem, tot);
        if (f) out[base + ex] = (int32_t)g;
        base += tot;
    }
}

}  // namespace cls

using namespace cls;

extern "C" size_t cls_lift_workspace_size(int32_t n) {
    const int64_t chunks = (n + kLiftChunk - 1) / kLiftChunk;
    return (size_t)((chunks + 1) * sizeof(int64_t) + 255) / 256 * 256;
}

extern "C" int cls_lift_change_masks(const float* params, int32_t n, int32_t row_stride,
                                     const ClsView* views_dev, int32_t first_view,
                                     int32_t n_views, const uint8_t* masks, int32_t vote_mode,
                                     uint8_t* active_out, int32_t* active_idx_out,
                                     int32_t* n_active_out, int32_t* votes_out, void* workspace,
                                     size_t workspace_bytes, cls_stream_t stream) {
    if (n < 0 || n_views <= 0 || first_view < 0 || (vote_mode != 0 && vote_mode != 1) ||
        row_stride < 4 || row_stride % 4 != 0)
        return CLS_ERR_INVALID_ARG;
    if (!views_dev || !masks || !active_out || !active_idx_out || !n_active_out ||
        (n > 0 && !params) || !workspace || workspace_bytes < cls_lift_workspace_size(n))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        cudaMemsetAsync(n_active_out, 0, sizeof(int32_t), s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const int64_t chunks = (n + kLiftChunk - 1) / kLiftChunk;
    int64_t* partials = static_cast<int64_t*>(workspace);
    lift_vote_kernel<<<(unsigned)chunks, kLiftBlock, 0, s>>>(params, n, row_stride, views_dev,
                                                            first_view, n_views, masks, vote_mode,
                                                            active_out, votes_out, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, chunks, nullptr, n_active_out, -1, nullptr);
    compact_flags_kernel<<<(unsigned)chunks, kLiftBlock, 0, s>>>(active_out, n, partials,
                                                                active_idx_out);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant. Its only scratch, the per-chunk counts of active
// Gaussians, lives in this fixed device array instead of a caller workspace.
// Every slot a call reads is first written by the same call's vote kernel, so
// nothing has to be cleared between calls.
static __device__ __align__(256) int64_t g_lift_static_scratch[CLS_LIFT_STATIC_MAX_N / kLiftChunk + 1];

static std::mutex g_lift_static_mutex;
static void* g_lift_static_ptr[64] = {nullptr};

// Device address of the array on the current device, looked up once per device.
static int lift_static_scratch(int64_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CLS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_lift_static_mutex);
    if (!g_lift_static_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_lift_static_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return CLS_ERR_CUDA;
        }
        g_lift_static_ptr[dev] = p;
    }
    *out = static_cast<int64_t*>(g_lift_static_ptr[dev]);
    return CLS_OK;
}

extern "C" int cls_lift_change_masks_static(const float* params, int32_t n, int32_t row_stride,
                                            const ClsView* views_dev, int32_t first_view,
                                            int32_t n_views, const uint8_t* masks,
                                            int32_t vote_mode, uint8_t* active_out,
                                            int32_t* active_idx_out, int32_t* n_active_out,
                                            int32_t* votes_out, cls_stream_t stream) {
    if (n < 0 || n > CLS_LIFT_STATIC_MAX_N) return CLS_ERR_INVALID_ARG;
    if (n_views <= 0 || first_view < 0 || (vote_mode != 0 && vote_mode != 1) || row_stride < 4 ||
        row_stride % 4 != 0 || !views_dev || !masks || !active_out || !active_idx_out ||
        !n_active_out || (n > 0 && !params))
        return CLS_ERR_INVALID_ARG;
    int64_t* partials = nullptr;
    const int rc = lift_static_scratch(&partials);
    if (rc != CLS_OK) return rc;
    cudaStream_t s = as_stream(stream);
    if (n == 0) {
        cudaMemsetAsync(n_active_out, 0, sizeof(int32_t), s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const int64_t chunks = (n + kLiftChunk - 1) / kLiftChunk;
    lift_vote_kernel<<<(unsigned)chunks, kLiftBlock, 0, s>>>(params, n, row_stride, views_dev,
                                                            first_view, n_views, masks, vote_mode,
                                                            active_out, votes_out, partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(partials, chunks, nullptr, n_active_out, -1, nullptr);
    compact_flags_kernel<<<(unsigned)chunks, kLiftBlock, 0, s>>>(active_out, n, partials,
                                                                active_idx_out);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
