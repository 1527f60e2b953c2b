// Projection, dynamic render mask and (Gaussian, tile) pair emission
// (Supp. "Local Optimization Kernel", item 1; base 3DGS preprocessing).
#include "scan.cuh"

namespace cls {

constexpr int kProjBlock = 128;
constexpr int kBinBlock = 256;
constexpr int kBinItems = 8;
constexpr int kBinChunk = kBinBlock * kBinItems;

// ---------------------------------------------------------------------------
// Projection. mode 0: every Gaussian of the view's scene (slot -1); mode 1:
// the scene's active Gaussians (slot = view.g2_base + rank).
template <int MODE>
__global__ void __launch_bounds__(kProjBlock)
project_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
               ClsProjected* __restrict__ records) {
    const ClsView& view = views[blockIdx.y];
    const ClsScene& sc = scenes[view.scene];
    const int i = blockIdx.x * kProjBlock + threadIdx.x;
    int g, slot;
    if (MODE == 0) {
        if (i >= sc.n) return;
        g = i;
        slot = -1;
    } else {
        if (i >= sc.n_active) return;
        g = sc.active_idx[i];
        slot = (int)(view.g2_base + i);
    }
    const ClsCamera& cam = view.cam;
    const float* row = sc.params + (int64_t)g * sc.row_stride;
    const float4 m = *reinterpret_cast<const float4*>(row);
    const float4 ls = *reinterpret_cast<const float4*>(row + 4);
    const float4 q = *reinterpret_cast<const float4*>(row + 8);
    Proj P;
    project_gaussian(cam, m, ls, q, P);
    int x0, x1, y0, y1;
    bool valid = P.valid && tile_rect(P.u, P.v, P.radius, view.tiles_x, view.tiles_y, x0, x1, y0, y1);
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    int radius = 0;
    if (valid) {
        const float inv_det = 1.0f / P.det;
        // view-dependent colour
        float dx = m.x - cam.pos[0], dy = m.y - cam.pos[1], dz = m.z - cam.pos[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis(dx, dy, dz, sc.sh_degree, Y);
        const int K = (sc.sh_degree + 1) * (sc.sh_degree + 1);
        float col[3] = {0.5f, 0.5f, 0.5f};
        const float* sh = row + 12;
        for (int k = 0; k < K; ++k) {
            col[0] += Y[k] * sh[3 * k + 0];
            col[1] += Y[k] * sh[3 * k + 1];
            col[2] += Y[k] * sh[3 * k + 2];
        }
        const float opacity = 1.0f / (1.0f + __expf(-m.w));
        r0 = make_float4(P.u, P.v, P.c * inv_det, -P.b * inv_det);
        r1 = make_float4(P.a * inv_det, opacity, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
        r2 = make_float4(fmaxf(col[2], 0.f), __int_as_float(slot), P.z, 0.f);
        radius = (int)P.radius;
        if (radius < 1) radius = 1;  // cannot happen for a finite positive lambda
    } else {
        r2 = make_float4(0.f, __int_as_float(slot), 0.f, 0.f);
    }
    r2.w = __int_as_float(radius);
    float4* out = reinterpret_cast<float4*>(records + view.rec_base + g);
    out[0] = r0;
    out[1] = r1;
    out[2] = r2;
}

// Mark the tiles of every active Gaussian's rectangle.
__global__ void __launch_bounds__(256)
mark_tiles_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                  const ClsProjected* __restrict__ records, uint8_t* __restrict__ tile_active) {
    const ClsView& view = views[blockIdx.y];
    const ClsScene& sc = scenes[view.scene];
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= sc.n_active) return;
    const int g = sc.active_idx[i];
    const ClsProjected rec = records[view.rec_base + g];
    if (rec.radius <= 0) return;
    int x0, x1, y0, y1;
    if (!tile_rect(rec.u, rec.v, (float)rec.radius, view.tiles_x, view.tiles_y, x0, x1, y0, y1))
        return;
    for (int ty = y0; ty <= y1; ++ty) {
        uint8_t* row = tile_active + view.tile_base + (int64_t)ty * view.tiles_x;
        for (int tx = x0; tx <= x1; ++tx) row[tx] = 1;
    }
}

// Ascending list of active tiles (one block, 1024 threads).
__global__ void __launch_bounds__(1024)
compact_tiles_kernel(const uint8_t* __restrict__ tile_active, int64_t n_tiles,
                     int32_t* __restrict__ active_tiles, int32_t* __restrict__ n_active_tiles) {
    __shared__ int32_t smem[1024 / 32 + 1];
    int32_t carry = 0;
    for (int64_t base = 0; base < n_tiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const int32_t f = (t < n_tiles && tile_active[t]) ? 1 : 0;
        int32_t tot;
        const int32_t ex = block_exclusive_sum<1024>(f, smem, tot);
        if (f) active_tiles[carry + ex] = (int32_t)t;
        carry += tot;
    }
    if (threadIdx.x == 0) *n_active_tiles = carry;
}

// Summed-area table of the active-tile mask per view:
// S[y][x] = number of active tiles with ty < y and tx < x.
__global__ void __launch_bounds__(256)
tile_sat_kernel(const ClsView* __restrict__ views, const uint8_t* __restrict__ tile_active,
                int32_t* __restrict__ sat) {
    const ClsView& view = views[blockIdx.x];
    const int Tx = view.tiles_x, Ty = view.tiles_y, Wd = Tx + 1;
    int32_t* S = sat + view.sat_base;
    const uint8_t* act = tile_active + view.tile_base;
    for (int y = threadIdx.x; y <= Ty; y += blockDim.x) {
        int32_t run = 0;
        S[(int64_t)y * Wd] = 0;
        for (int x = 0; x < Tx; ++x) {
            if (y > 0) run += act[(int64_t)(y - 1) * Tx + x];
            S[(int64_t)y * Wd + x + 1] = run;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x <= Tx; x += blockDim.x) {
        int32_t run = 0;
        for (int y = 0; y <= Ty; ++y) {
            run += S[(int64_t)y * Wd + x];
            S[(int64_t)y * Wd + x] = run;
        }
    }
}

__device__ __forceinline__ int rect_count(const int32_t* S, int Wd, int x0, int x1, int y0,
                                          int y1) {
    return S[(int64_t)(y1 + 1) * Wd + x1 + 1] - S[(int64_t)y0 * Wd + x1 + 1] -
           S[(int64_t)(y1 + 1) * Wd + x0] + S[(int64_t)y0 * Wd + x0];
}

__device__ __forceinline__ int pair_count(const ClsView& view, const ClsProjected* records,
                                          const int32_t* sat, int g, int& x0, int& x1, int& y0,
                                          int& y1) {
    const float4 c0 = reinterpret_cast<const float4*>(records + view.rec_base + g)[0];
    const float4 c2 = reinterpret_cast<const float4*>(records + view.rec_base + g)[2];
    const int radius = __float_as_int(c2.w);
    if (radius <= 0) return 0;
    if (!tile_rect(c0.x, c0.y, (float)radius, view.tiles_x, view.tiles_y, x0, x1, y0, y1))
        return 0;
    return rect_count(sat + view.sat_base, view.tiles_x + 1, x0, x1, y0, y1);
}

__global__ void __launch_bounds__(kBinBlock)
count_pairs_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                   const ClsProjected* __restrict__ records, const int32_t* __restrict__ sat,
                   int chunks_per_view, int64_t* __restrict__ partials) {
    __shared__ int64_t smem[kBinBlock / 32 + 1];
    const ClsView& view = views[blockIdx.y];
    const int n = scenes[view.scene].n;
    int64_t cnt = 0;
    for (int it = 0; it < kBinItems; ++it) {
        const int g = blockIdx.x * kBinChunk + it * kBinBlock + threadIdx.x;
        if (g < n) {
            int x0, x1, y0, y1;
            cnt += pair_count(view, records, sat, g, x0, x1, y0, y1);
        }
    }
    int64_t tot;
    block_exclusive_sum<kBinBlock>(cnt, smem, tot);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * chunks_per_view + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBinBlock)
emit_pairs_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                  const ClsProjected* __restrict__ records, const int32_t* __restrict__ sat,
                  const uint8_t* __restrict__ tile_active, int chunks_per_view,
                  const int64_t* __restrict__ offsets, uint64_t* __restrict__ keys,
                  uint32_t* __restrict__ vals, int64_t capacity) {
    __shared__ int64_t smem[kBinBlock / 32 + 1];
    const ClsView& view = views[blockIdx.y];
    const int n = scenes[view.scene].n;
    int64_t base = offsets[(int64_t)blockIdx.y * chunks_per_view + blockIdx.x];
    for (int it = 0; it < kBinItems; ++it) {
        const int g = blockIdx.x * kBinChunk + it * kBinBlock + threadIdx.x;
        int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
        const int64_t cnt = g < n ? pair_count(view, records, sat, g, x0, x1, y0, y1) : 0;
        int64_t tot;
        int64_t pos = base + block_exclusive_sum<kBinBlock>(cnt, smem, tot);
        base += tot;
        if (cnt == 0) continue;
        const uint64_t zbits =
            (uint64_t)__float_as_uint(reinterpret_cast<const float4*>(records + view.rec_base + g)[2].z);
        const uint32_t val = (uint32_t)(view.rec_base + g);
        for (int ty = y0; ty <= y1; ++ty) {
            const int64_t row = (int64_t)view.tile_base + (int64_t)ty * view.tiles_x;
            for (int tx = x0; tx <= x1; ++tx) {
                if (!tile_active[row + tx]) continue;
                if (pos < capacity) {
                    keys[pos] = ((uint64_t)(row + tx) << 32) | zbits;
                    vals[pos] = val;
                }
                ++pos;
            }
        }
    }
}

}  // namespace cls

using namespace cls;

static int64_t bin_chunks_per_view(const ClsBatchInfo* info) {
    return (info->max_n + kBinChunk - 1) / kBinChunk;
}

extern "C" size_t cls_project_workspace_size(const ClsBatchInfo* info) {
    if (!info) return 0;
    const int64_t parts = bin_chunks_per_view(info) * info->n_views + 1;
    size_t bytes = (size_t)parts * sizeof(int64_t);
    bytes = (bytes + 255) / 256 * 256;
    bytes += (size_t)info->total_sat * sizeof(int32_t);
    return (bytes + 255) / 256 * 256;
}

extern "C" int cls_project_and_bin(const ClsScene* scenes_dev, const ClsView* views_dev,
                                   const ClsBatchInfo* info, int32_t project_mode,
                                   ClsProjected* records, uint8_t* tile_active,
                                   int32_t* active_tiles, int32_t* n_active_tiles_dev,
                                   uint64_t* keys, uint32_t* vals, int64_t capacity,
                                   int64_t* n_pairs_dev, int32_t* status_dev, void* workspace,
                                   size_t workspace_bytes, cls_stream_t stream) {
    if (!info || !scenes_dev || !views_dev || !records || !tile_active || !active_tiles ||
        !n_active_tiles_dev || !n_pairs_dev || !status_dev || !workspace ||
        (capacity > 0 && (!keys || !vals)) || capacity < 0 ||
        (project_mode != 0 && project_mode != 1))
        return CLS_ERR_INVALID_ARG;
    if (info->n_views <= 0 || info->n_views > 65535 || info->total_tiles <= 0 ||
        workspace_bytes < cls_project_workspace_size(info) || capacity >= ((int64_t)1 << 32))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const unsigned V = (unsigned)info->n_views;
    const int64_t cpv = bin_chunks_per_view(info);
    int64_t* partials = static_cast<int64_t*>(workspace);
    size_t off = ((size_t)(cpv * V + 1) * sizeof(int64_t) + 255) / 256 * 256;
    int32_t* sat = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + off);

    if (project_mode == 0) {
        if (info->max_n > 0)
            project_kernel<0><<<dim3((info->max_n + kProjBlock - 1) / kProjBlock, V), kProjBlock,
                                 0, s>>>(scenes_dev, views_dev, records);
    }
    if (info->max_active > 0)
        project_kernel<1><<<dim3((info->max_active + kProjBlock - 1) / kProjBlock, V), kProjBlock,
                             0, s>>>(scenes_dev, views_dev, records);
    cudaMemsetAsync(tile_active, 0, (size_t)info->total_tiles, s);
    if (info->max_active > 0)
        mark_tiles_kernel<<<dim3((info->max_active + 255) / 256, V), 256, 0, s>>>(
            scenes_dev, views_dev, records, tile_active);
    compact_tiles_kernel<<<1, 1024, 0, s>>>(tile_active, info->total_tiles, active_tiles,
                                            n_active_tiles_dev);
    tile_sat_kernel<<<V, 256, 0, s>>>(views_dev, tile_active, sat);
    if (cpv > 0) {
        count_pairs_kernel<<<dim3((unsigned)cpv, V), kBinBlock, 0, s>>>(
            scenes_dev, views_dev, records, sat, (int)cpv, partials);
        scan_partials_kernel<<<1, 1024, 0, s>>>(partials, cpv * V, n_pairs_dev, nullptr, capacity,
                                                status_dev);
        emit_pairs_kernel<<<dim3((unsigned)cpv, V), kBinBlock, 0, s>>>(
            scenes_dev, views_dev, records, sat, tile_active, (int)cpv, partials, keys, vals,
            capacity);
    } else {
        cudaMemsetAsync(n_pairs_dev, 0, sizeof(int64_t), s);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
