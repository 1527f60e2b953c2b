// D-SSIM term of the photometric loss over the rendered tiles (Supp.
// "Implementation Details": the base 3DGS optimiser's loss,
// (1 - lambda) L1 + lambda (1 - SSIM), SSIM with an 11 x 11 Gaussian window of
// standard deviation 1.5, C1 = 0.01^2, C2 = 0.03^2, zero padding at the image
// border).
//
// With mu = g * x, E[x^2] = g * x^2, E[xy] = g * (x y) per pixel p, the map
// S(p) depends on x only through those window sums, so
//   d/dx(q) sum_p S(p) = (g * a)(q) + 2 x(q) (g * b)(q) + y(q) (g * c)(q)
// with a = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy,
// b = dS/dsigma_x^2, c = dS/dsigma_xy. Pass 1 computes S, a, b, c at every
// pixel of every rendered tile (covered tiles and the ring around them, which
// holds every pixel within 10 of a covered one); pass 2 blurs a, b, c at the
// covered tiles' pixels and combines. A 128-thread block handles one 16 x 16
// tile, one channel at a time (small shared memory, many blocks per SM): it
// loads the channel's 26 x 26 region (5-pixel halo) of every plane it needs,
// then applies the separable 11-tap window with the taps in registers, one
// whole row (16 outputs from 26 inputs) or column (16 from 26) per work item,
// so each value is read from shared memory once per pass.
#include "common.cuh"

namespace cls {

constexpr int kSsimR = 5;                       // window radius
constexpr int kSsimW = 2 * kSsimR + 1;          // 11 taps
constexpr int kReg = kTile + 2 * kSsimR;        // 26 x 26 region
constexpr float kSsimSigma = 1.5f;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// Planar per-view images: channel c of pixel (x, y) of view v.
__device__ __forceinline__ int64_t plane_index(const ClsView& v, int c, int x, int y) {
    const int64_t plane = (int64_t)v.cam.width * v.cam.height;
    return 3 * v.pix_base + c * plane + (int64_t)y * v.cam.width + x;
}

// The normalised 11-tap Gaussian window, in registers.
__device__ __forceinline__ void ssim_taps(float* w) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kSsimW; ++k) {
        const float d = (float)(k - kSsimR);
        w[k] = expf(-(d * d) / (2.0f * kSsimSigma * kSsimSigma));
        s += w[k];
    }
#pragma unroll
    for (int k = 0; k < kSsimW; ++k) w[k] /= s;
}

constexpr int kSsimThreads = 128;

// One channel at a time: region planes x, y (pass 1) or a, b, c (pass 2) of
// the channel; after the horizontal sums, the vertical sums of the 16 x 16
// tile (5 planes in pass 1, 3 in pass 2) are written over them.
struct SsimSmem {
    float r[3][kReg][kReg];
    float h[5][kReg][kTile];      // horizontal sums: 5 (pass 1), 3 (pass 2)
    float red[kSsimThreads / 32];
};

// Vertical sums of the tile written over the region planes: plane q, row i, col j.
__device__ __forceinline__ float& vsum(SsimSmem& sm, int q, int i, int j) {
    return (&sm.r[0][0][0])[(q * kTile + i) * kTile + j];
}

// One row of 26 inputs to 16 window sums, in registers.
__device__ __forceinline__ void blur16(const float* in, const float* w, float* out) {
#pragma unroll
    for (int o = 0; o < kTile; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kSsimW; ++k) acc = __fmaf_rn(w[k], in[o + k], acc);
        out[o] = acc;
    }
}

// Horizontal pass: item (plane p of the kNP planes of h, region row), the
// 26 inputs of the row read once. Pass 1 (kNP = 5): p = x, y, x^2, y^2, x y
// of the channel from its region planes x (0) and y (1); pass 2 (kNP = 3):
// the a, b, c planes as loaded.
template <int kNP>
__device__ __forceinline__ void blur_rows(SsimSmem& sm, const float* w) {
    for (int e = threadIdx.x; e < kNP * kReg; e += blockDim.x) {
        const int p = e / kReg, row = e - p * kReg;
        float in[kReg];
        if (kNP == 5) {
            const float* xr = &sm.r[0][row][0];
            const float* yr = &sm.r[1][row][0];
            // one specialised loop per quantity (p is uniform over the item)
            switch (p) {
                case 0:
#pragma unroll
                    for (int k = 0; k < kReg; ++k) in[k] = xr[k];
                    break;
                case 1:
#pragma unroll
                    for (int k = 0; k < kReg; ++k) in[k] = yr[k];
                    break;
                case 2:
#pragma unroll
                    for (int k = 0; k < kReg; ++k) in[k] = xr[k] * xr[k];
                    break;
                case 3:
#pragma unroll
                    for (int k = 0; k < kReg; ++k) in[k] = yr[k] * yr[k];
                    break;
                default:
#pragma unroll
                    for (int k = 0; k < kReg; ++k) in[k] = xr[k] * yr[k];
            }
        } else {
            const float* vr = &sm.r[p][row][0];
#pragma unroll
            for (int k = 0; k < kReg; ++k) in[k] = vr[k];
        }
        float out[kTile];
        blur16(in, w, out);
#pragma unroll
        for (int o = 0; o < kTile; ++o) sm.h[p][row][o] = out[o];
    }
}

// Vertical pass: item (plane, column), the 26 horizontal sums of the column
// read once, the 16 results written to vsum (over the region planes).
template <int kNP>
__device__ __forceinline__ void blur_cols(SsimSmem& sm, const float* w) {
    for (int e = threadIdx.x; e < kNP * kTile; e += blockDim.x) {
        const int p = e / kTile, j = e - p * kTile;
        float in[kReg];
#pragma unroll
        for (int k = 0; k < kReg; ++k) in[k] = sm.h[p][k][j];
        float out[kTile];
        blur16(in, w, out);
#pragma unroll
        for (int i = 0; i < kTile; ++i) vsum(sm, p, i, j) = out[i];
    }
}

__device__ __forceinline__ float block_sum(SsimSmem& sm, float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm.red[k];
    __syncthreads();
    return t;
}

// Load `np` planes of the tile's 26 x 26 region (zero outside the image):
// plane q is value(q, flat index of the pixel in its view's plane).
template <typename Value>
__device__ __forceinline__ void load_region(SsimSmem& sm, int np, int x0, int y0, int W, int H,
                                            Value value) {
    for (int e = threadIdx.x; e < kReg * kReg; e += blockDim.x) {
        const int row = e / kReg, col = e - row * kReg;
        const int gx = x0 + col, gy = y0 + row;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const int64_t off = (int64_t)gy * W + gx;
        for (int q = 0; q < np; ++q) sm.r[q][row][col] = in ? value(q, off) : 0.f;
    }
}

// Pass 1: S, a, b, c at every pixel of every rendered tile; lambda (1 - S)
// summed into the loss over the covered tiles' pixels.
__global__ void __launch_bounds__(kSsimThreads)
ssim_maps_kernel(const ClsView* __restrict__ views, int n_views, const int32_t* __restrict__ tiles,
                 const int32_t* __restrict__ n_tiles, const uint8_t* __restrict__ tile_active,
                 const float* __restrict__ image, const float* __restrict__ target, float lambda,
                 float* __restrict__ abc, float* __restrict__ loss_per_scene) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SsimSmem& sm = *reinterpret_cast<SsimSmem*>(smem_raw);
    float w[kSsimW];
    ssim_taps(w);
    const int n = *n_tiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int tile = tiles[t];
        const ClsView& view = views[view_of_tile(views, n_views, tile)];
        const int local = tile - view.tile_base;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const int W = view.cam.width, H = view.cam.height;
        const int64_t plane = (int64_t)W * H;
        float lsum = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float* xi = image + 3 * view.pix_base + c * plane;
            const float* yi = target + 3 * view.pix_base + c * plane;
            __syncthreads();
            load_region(sm, 2, tx * kTile - kSsimR, ty * kTile - kSsimR, W, H,
                        [&](int q, int64_t off) { return (q ? yi : xi)[off]; });
            __syncthreads();
            blur_rows<5>(sm, w);
            __syncthreads();
            blur_cols<5>(sm, w);
            __syncthreads();
            for (int e = threadIdx.x; e < kTilePixels; e += blockDim.x) {
                const int i = e / kTile, j = e - i * kTile;
                const int px = tx * kTile + j, py = ty * kTile + i;
                if (!(px < W && py < H)) continue;
                const float mx = vsum(sm, 0, i, j), my = vsum(sm, 1, i, j);
                const float vx = vsum(sm, 2, i, j) - mx * mx;
                const float vy = vsum(sm, 3, i, j) - my * my;
                const float cxy = vsum(sm, 4, i, j) - mx * my;
                const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
                const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
                const float D = B1 * B2;
                const float S = A1 * A2 / D;
                const float dmu = 2.f * my * A2 / D - 2.f * mx * S / B1;
                const float dvx = -S / B2;
                const float dcxy = 2.f * A1 / D;
                const int64_t base = 9 * view.pix_base + (int64_t)(3 * c) * plane +
                                     (int64_t)py * W + px;
                abc[base] = dmu - 2.f * mx * dvx - my * dcxy;
                abc[base + plane] = dvx;
                abc[base + 2 * plane] = dcxy;
                lsum += 1.f - S;
            }
        }
        const bool covered = tile_active[tile] == 1;
        const float tot = block_sum(sm, covered ? lsum : 0.f);
        if (threadIdx.x == 0 && loss_per_scene && covered)
            atomicAdd(loss_per_scene + view.scene, lambda * view.loss_scale * tot);
    }
}

// Pass 2, covered tiles only: dL/dC = (1 - lambda) dL1/dC - lambda * scale *
// d(sum S)/dx, where dL1/dC = sign(C - C*) * scale was written by the forward
// pass; (1 - lambda) |C - C*| * scale is added to the loss.
__global__ void __launch_bounds__(kSsimThreads)
ssim_grad_kernel(const ClsView* __restrict__ views, int n_views, const int32_t* __restrict__ tiles,
                 const int32_t* __restrict__ n_tiles, const uint8_t* __restrict__ tile_active,
                 const float* __restrict__ image, const float* __restrict__ target, float lambda,
                 const float* __restrict__ abc, float* __restrict__ dL_dimage,
                 float* __restrict__ loss_per_scene) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SsimSmem& sm = *reinterpret_cast<SsimSmem*>(smem_raw);
    float w[kSsimW];
    ssim_taps(w);
    const int n = *n_tiles;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int tile = tiles[t];
        if (tile_active[tile] != 1) continue;  // uniform over the block
        const ClsView& view = views[view_of_tile(views, n_views, tile)];
        const int local = tile - view.tile_base;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const int W = view.cam.width, H = view.cam.height;
        const int64_t plane = (int64_t)W * H;
        float lsum = 0.f;
        for (int c = 0; c < 3; ++c) {
            const float* m = abc + 9 * view.pix_base + (int64_t)(3 * c) * plane;
            __syncthreads();
            load_region(sm, 3, tx * kTile - kSsimR, ty * kTile - kSsimR, W, H,
                        [&](int q, int64_t off) { return m[q * plane + off]; });
            __syncthreads();
            blur_rows<3>(sm, w);
            __syncthreads();
            blur_cols<3>(sm, w);
            __syncthreads();
            for (int e = threadIdx.x; e < kTilePixels; e += blockDim.x) {
                const int i = e / kTile, j = e - i * kTile;
                const int px = tx * kTile + j, py = ty * kTile + i;
                if (!(px < W && py < H)) continue;
                const int64_t idx = plane_index(view, c, px, py);
                const float xv = image[idx], yv = target[idx];
                const float gs = vsum(sm, 0, i, j) + 2.f * xv * vsum(sm, 1, i, j) +
                                 yv * vsum(sm, 2, i, j);
                dL_dimage[idx] = (1.f - lambda) * dL_dimage[idx] - lambda * view.loss_scale * gs;
                lsum += fabsf(xv - yv);
            }
        }
        const float tot = block_sum(sm, lsum);
        if (threadIdx.x == 0 && loss_per_scene)
            atomicAdd(loss_per_scene + view.scene, (1.f - lambda) * view.loss_scale * tot);
    }
}

static PerDevice g_ssim_blocks;

}  // namespace cls

using namespace cls;

extern "C" size_t cls_ssim_buffer_size(const ClsBatchInfo* info) {
    return info ? (size_t)info->total_pixels * 9 : 0;
}

extern "C" int cls_ssim_loss(const ClsView* views_dev, const ClsBatchInfo* info,
                             const int32_t* tiles, const int32_t* n_tiles_dev,
                             const uint8_t* tile_active, const float* image, const float* target,
                             float lambda, float* abc, float* dL_dimage, float* loss_per_scene,
                             cls_stream_t stream) {
    if (!views_dev || !info || !tiles || !n_tiles_dev || !tile_active || !image || !target ||
        !abc || !dL_dimage || info->n_views <= 0 || info->total_tiles <= 0 ||
        !(lambda >= 0.0f && lambda <= 1.0f))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int ssim_blocks = per_device(g_ssim_blocks, [](int dev) {
        cudaFuncSetAttribute(ssim_maps_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SsimSmem));
        cudaFuncSetAttribute(ssim_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SsimSmem));
        return resident_blocks(dev, ssim_maps_kernel, kSsimThreads, sizeof(SsimSmem));
    });
    const int blocks = (int)hmin64(info->total_tiles, ssim_blocks);
    ssim_maps_kernel<<<blocks, kSsimThreads, sizeof(SsimSmem), s>>>(
        views_dev, info->n_views, tiles, n_tiles_dev, tile_active, image, target, lambda, abc,
        loss_per_scene);
    ssim_grad_kernel<<<blocks, kSsimThreads, sizeof(SsimSmem), s>>>(
        views_dev, info->n_views, tiles, n_tiles_dev, tile_active, image, target, lambda, abc,
        dL_dimage, loss_per_scene);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
