// Projection, dynamic render mask and (Gaussian, tile) pair emission
// (Supp. "Local Optimization Kernel", item 1; base 3DGS preprocessing).
#include <algorithm>

#include "scan.cuh"

namespace cls {

constexpr int kProjBlock = 128;
constexpr int kBinBlock = 256;
constexpr int kBinItems = 8;
constexpr int kBinChunk = kBinBlock * kBinItems;
constexpr int kDepthBins = CLS_DEPTH_BINS;  // depth buckets per tile (bucketed layout)
constexpr int kBigArea = 128;               // rectangles above this many tiles: one warp each
constexpr uint32_t kPrefixMargin = 1u << 17; // float ulps between a prefix boundary and the
                                             // nearest active Gaussian (about 1.6% of depth)

// ---------------------------------------------------------------------------
// Projection. mode 0: every Gaussian of the view's scene (slot -1); mode 1:
// the scene's active Gaussians (slot = view.g2_base + rank).
// ---------------------------------------------------------------------------
// Dynamic render mask: every active Gaussian adds +1 over its tile rectangle
// in a per-view difference grid (four corner updates), whose 2D prefix sum is
// the number of active rectangles covering each tile.
__device__ __forceinline__ void stamp_rect(int32_t* grid, int Wd, int x0, int x1, int y0, int y1) {
    atomicAdd(grid + (int64_t)y0 * Wd + x0, 1);
    atomicAdd(grid + (int64_t)y0 * Wd + x1 + 1, -1);
    atomicAdd(grid + (int64_t)(y1 + 1) * Wd + x0, -1);
    atomicAdd(grid + (int64_t)(y1 + 1) * Wd + x1 + 1, 1);
}

// Depth bins of a view: its depth range [lo, hi] (float bits of the
// pair-producing Gaussians' depths) cut into kDepthBins equal parts. The bin
// of depth bits zb is floor((zb - lo) * scale), clamped; float rounding is
// monotone, so bins stay monotone in depth, and every kernel derives the same
// scale from the same lo and hi.
struct DepthBins {
    uint32_t lo;
    float scale;
};

__device__ __forceinline__ DepthBins depth_bins(uint32_t lo, uint32_t hi) {
    return DepthBins{lo, (float)kDepthBins / ((float)(hi - lo) + 1.0f)};
}

__device__ __forceinline__ int depth_bin(uint32_t zb, const DepthBins& d) {
    if (zb <= d.lo) return 0;
    return min((int)((float)(zb - d.lo) * d.scale), kDepthBins - 1);
}

// Smallest depth bits whose depth bin is at least b (0 for b <= 0, all ones
// for b >= kDepthBins): a binary search, exact because depth_bin is monotone.
__device__ __forceinline__ uint32_t bin_edge(int b, const DepthBins& d) {
    if (b <= 0) return 0u;
    if (b >= kDepthBins) return 0xffffffffu;
    uint64_t l = (uint64_t)d.lo + 1, h = 0xffffffffull;  // depth_bin(h) = kDepthBins - 1
    while (l < h) {
        const uint64_t m = (l + h) >> 1;
        if (depth_bin((uint32_t)m, d) >= b) h = m; else l = m + 1;
    }
    return (uint32_t)l;
}

// The same, at depth bin b of a bin-fastest grid (entry (cell, b) at cell * kDepthBins + b).
__device__ __forceinline__ void stamp_rect_bin(int32_t* G, int Wd, int b, int x0, int x1, int y0,
                                               int y1) {
    atomicAdd(G + ((int64_t)y0 * Wd + x0) * kDepthBins + b, 1);
    atomicAdd(G + ((int64_t)y0 * Wd + x1 + 1) * kDepthBins + b, -1);
    atomicAdd(G + ((int64_t)(y1 + 1) * Wd + x0) * kDepthBins + b, -1);
    atomicAdd(G + ((int64_t)(y1 + 1) * Wd + x1 + 1) * kDepthBins + b, 1);
}

// Tile rectangle and depth bits of every record, written by the projection
// (16 B: x0 | x1 << 16, y0 | y1 << 16, depth bits, and 1 for a visible static
// record, 2 for a visible active one, 0 if the record has no tiles), so
// binning reads 16 B per record instead of its 48.
__device__ __forceinline__ uint4 pack_rect(bool valid, int x0, int x1, int y0, int y1,
                                           uint32_t zbits, uint32_t flag) {
    return valid ? make_uint4((uint32_t)x0 | ((uint32_t)x1 << 16),
                              (uint32_t)y0 | ((uint32_t)y1 << 16), zbits, flag)
                 : make_uint4(0u, 0u, 0u, 0u);
}

__device__ __forceinline__ void unpack_rect(const uint4& r, int& x0, int& x1, int& y0, int& y1) {
    x0 = (int)(r.x & 0xffffu);
    x1 = (int)(r.x >> 16);
    y0 = (int)(r.y & 0xffffu);
    y1 = (int)(r.y >> 16);
}

__device__ __forceinline__ bool record_rect(const uint4* rects, int64_t rec, int& x0, int& x1,
                                            int& y0, int& y1, uint32_t& zbits) {
    const uint4 r = rects[rec];
    zbits = r.z;
    if (r.w == 0u) return false;
    unpack_rect(r, x0, x1, y0, y1);
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(kProjBlock)
project_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
               ClsProjected* __restrict__ records, uint4* __restrict__ rects,
               int32_t* __restrict__ diff, const uint32_t* __restrict__ zmin,
               const uint32_t* __restrict__ zmax, int32_t* __restrict__ abins,
               uint32_t* __restrict__ arange) {
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
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    bool valid = P.valid && tile_rect(P.u, P.v, P.radius, view.tiles_x, view.tiles_y, x0, x1, y0, y1);
    uint32_t b_lo = 0xffffffffu, b_hi = 0u;  // depth bin of a stamped active record
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
        if (K == 16) {  // degree 3: the 48 coefficients as twelve 16-byte loads, issued together
            float c[48];
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                const float4 v = reinterpret_cast<const float4*>(sh)[j];
                c[4 * j] = v.x; c[4 * j + 1] = v.y; c[4 * j + 2] = v.z; c[4 * j + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                col[0] += Y[k] * c[3 * k + 0];
                col[1] += Y[k] * c[3 * k + 1];
                col[2] += Y[k] * c[3 * k + 2];
            }
        } else {  // unrolled with a guard, so that Y stays in registers
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if (k < K) {
                    col[0] += Y[k] * sh[3 * k + 0];
                    col[1] += Y[k] * sh[3 * k + 1];
                    col[2] += Y[k] * sh[3 * k + 2];
                }
            }
        }
        const float opacity = 1.0f / (1.0f + __expf(-m.w));
        r0 = make_float4(P.u, P.v, P.c * inv_det, -P.b * inv_det);
        r1 = make_float4(P.a * inv_det, opacity, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
        r2 = make_float4(fmaxf(col[2], 0.f), __int_as_float(slot), P.z, 0.f);
        radius = (int)P.radius;
        if (radius < 1) radius = 1;  // cannot happen for a finite positive lambda
        // an active Gaussian stamps its tile rectangle into the render mask and,
        // with fixed depth bins (`abins`), into the active difference grid A at
        // its depth bin
        if (MODE == 1) {
            stamp_rect(diff + view.sat_base, view.tiles_x + 1, x0, x1, y0, y1);
            if (abins) {
                const int b = depth_bin(__float_as_uint(P.z),
                                        depth_bins(zmin[blockIdx.y], zmax[blockIdx.y]));
                stamp_rect_bin(abins + (int64_t)view.sat_base * kDepthBins, view.tiles_x + 1, b,
                               x0, x1, y0, y1);
                b_lo = b_hi = (uint32_t)b;
            }
        }
    } else {
        r2 = make_float4(0.f, __int_as_float(slot), 0.f, 0.f);
    }
    r2.w = __int_as_float(radius);
    rects[view.rec_base + g] =
        pack_rect(valid, x0, x1, y0, y1, __float_as_uint(r2.z), MODE == 1 ? 2u : 1u);
    float4* out = reinterpret_cast<float4*>(records + view.rec_base + g);
    out[0] = r0;
    out[1] = r1;
    out[2] = r2;
    if (MODE == 1 && abins) {
        // the range of occupied bins over the lanes here (lanes past the active
        // count have left; any subset of lanes gives a correct min and max)
        const unsigned m = __activemask();
        const uint32_t lo = __reduce_min_sync(m, b_lo), hi = __reduce_max_sync(m, b_hi);
        if ((int)(threadIdx.x & 31) == __ffs(m) - 1 && hi >= lo) {
            atomicMin(arange + blockIdx.y, lo);
            atomicMax(arange + gridDim.y + blockIdx.y, hi);
        }
    }
}



// In-place 2D inclusive prefix sum of a (rows x cols) grid with row pitch Wd.
__device__ __forceinline__ void prefix2d(int32_t* G, int rows, int cols, int Wd) {
    for (int y = threadIdx.x; y < rows; y += blockDim.x) {
        int32_t run = 0;
        for (int x = 0; x < cols; ++x) {
            run += G[(int64_t)y * Wd + x];
            G[(int64_t)y * Wd + x] = run;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < cols; x += blockDim.x) {
        int32_t run = 0;
        for (int y = 0; y < rows; ++y) {
            run += G[(int64_t)y * Wd + x];
            G[(int64_t)y * Wd + x] = run;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int32_t warp_inclusive_sum(int32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// The same in shared memory, by warp scans: rows, then columns. An odd pitch
// keeps the column pass free of bank conflicts.
__device__ __forceinline__ void prefix2d_smem(int32_t* S, int rows, int cols, int p) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int y = warp; y < rows; y += nw) {
        int32_t carry = 0;
        for (int x0 = 0; x0 < cols; x0 += 32) {
            const int x = x0 + lane;
            int32_t v = x < cols ? S[y * p + x] : 0;
            v = warp_inclusive_sum(v, lane) + carry;
            if (x < cols) S[y * p + x] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    for (int x = warp; x < cols; x += nw) {
        int32_t carry = 0;
        for (int y0 = 0; y0 < rows; y0 += 32) {
            const int y = y0 + lane;
            int32_t v = y < rows ? S[y * p + x] : 0;
            v = warp_inclusive_sum(v, lane) + carry;
            if (y < rows) S[y * p + x] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
}

// Odd shared-memory pitch for a grid of `cols` columns.
__host__ __device__ __forceinline__ int smem_pitch(int cols) { return cols | 1; }

// Ring around the covered tiles, with coverage in bit 0 of `cov` (other bits
// ignored): 2 for an uncovered tile with a covered one among its eight
// neighbours.
__device__ __forceinline__ uint8_t ring_value_bit(const int32_t* cov, int pitch, int Tx, int Ty,
                                                  int x, int y) {
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int xx = x + dx, yy = y + dy;
            if (xx >= 0 && xx < Tx && yy >= 0 && yy < Ty && (cov[yy * pitch + xx] & 1)) return 2;
        }
    return 0;
}

// Ring around the covered tiles: 2 for an uncovered tile with a covered one
// among its eight neighbours (cov: 1 covered, 0 not; row pitch `pitch`).
__device__ __forceinline__ uint8_t ring_value(const int32_t* cov, int pitch, int Tx, int Ty,
                                              int x, int y) {
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int xx = x + dx, yy = y + dy;
            if (xx >= 0 && xx < Tx && yy >= 0 && yy < Ty && cov[yy * pitch + xx] > 0) return 2;
        }
    return 0;
}

// Per view: coverage of the active stamps -> tile mask (1: covered by an
// active rectangle; with `ring`, 2: an uncovered tile next to a covered one,
// rendered too) -> summed-area table S[y][x] = number of rendered tiles with
// ty < y and tx < x. Also clears every tile's nearest-active depth for
// active_zmin_kernel. The grids go through shared memory when they fit in
// `smem_cap` bytes.
__global__ void __launch_bounds__(512)
tile_mask_kernel(const ClsView* __restrict__ views, int32_t* __restrict__ diff,
                 uint8_t* __restrict__ tile_active, int32_t* __restrict__ sat,
                 ClsTileCache* __restrict__ tile_cache, int smem_cap, int ring, int reset_zmin) {
    extern __shared__ int32_t s_grid[];
    const ClsView& view = views[blockIdx.x];
    const int Tx = view.tiles_x, Ty = view.tiles_y, Wd = Tx + 1;
    int32_t* D = diff + view.sat_base;
    uint8_t* act = tile_active + view.tile_base;
    int32_t* S = sat + view.sat_base;
    const int p = smem_pitch(Tx);
    if ((int64_t)Ty * p * 4 <= smem_cap) {
        // a warp per row, its lanes over the row's tiles
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int y = warp; y < Ty; y += nw)
#pragma unroll 4
            for (int x = lane; x < Tx; x += 32) s_grid[y * p + x] = D[(int64_t)y * Wd + x];
        __syncthreads();
        prefix2d_smem(s_grid, Ty, Tx, p);
        for (int y = warp; y < Ty; y += nw)
            for (int x = lane; x < Tx; x += 32) {
                s_grid[y * p + x] = s_grid[y * p + x] > 0 ? 1 : 0;
                if (reset_zmin) tile_cache[view.tile_base + y * Tx + x].zmin_active = 0xffffffffu;
            }
        __syncthreads();
        // rendered (covered, or in the ring) into bit 1 of the same entries
        for (int y = warp; y < Ty; y += nw)
            for (int x = lane; x < Tx; x += 32) {
                const uint8_t a = (s_grid[y * p + x] & 1)
                                      ? (uint8_t)1
                                      : (ring ? ring_value_bit(s_grid, p, Tx, Ty, x, y) : (uint8_t)0);
                act[y * Tx + x] = a;
                // only this thread writes the entry; its neighbours read bit 0
                if (a) s_grid[y * p + x] |= 2;
            }
        __syncthreads();
        for (int y = warp; y < Ty; y += nw)
            for (int x = lane; x < Tx; x += 32) s_grid[y * p + x] = s_grid[y * p + x] >> 1;
        __syncthreads();
        prefix2d_smem(s_grid, Ty, Tx, p);
        for (int y = warp; y <= Ty; y += nw)
            for (int x = lane; x <= Tx; x += 32)
                S[(int64_t)y * Wd + x] = (x == 0 || y == 0) ? 0 : s_grid[(y - 1) * p + x - 1];
        return;
    }
    prefix2d(D, Ty, Tx, Wd);
    for (int t = threadIdx.x; t < Tx * Ty; t += blockDim.x) {
        const int y = t / Tx, x = t - y * Tx;
        act[t] = D[(int64_t)y * Wd + x] > 0 ? 1 : 0;
        if (reset_zmin) tile_cache[view.tile_base + t].zmin_active = 0xffffffffu;
    }
    __syncthreads();
    if (ring) {  // the coverage counts in D stay > 0 exactly on covered tiles
        for (int t = threadIdx.x; t < Tx * Ty; t += blockDim.x) {
            const int y = t / Tx, x = t - y * Tx;
            if (!act[t]) act[t] = ring_value(D, Wd, Tx, Ty, x, y);
        }
        __syncthreads();
    }
    for (int y = threadIdx.x; y <= Ty; y += blockDim.x) {
        int32_t run = 0;
        S[(int64_t)y * Wd] = 0;
        for (int x = 0; x < Tx; ++x) {
            if (y > 0) run += act[(int64_t)(y - 1) * Tx + x] != 0;
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

// Nearest active Gaussian of every tile: the depth bits of each non-culled
// active record are min-reduced over the tiles of its rectangle. One warp per
// active Gaussian, its lanes over the rectangle's cells; each block reduces
// into a private copy of its view's tile grid in shared memory and merges it
// into the global grid once.
// q = k / w and rem = k - q w for 0 <= k < 2^22 and w >= 1: a float estimate
// of k / w, off by at most one, then corrected exactly (cheaper than an
// integer division).
__device__ __forceinline__ void divmod_small(int k, int w, int& q, int& rem) {
    q = (int)__fdividef((float)k + 0.5f, (float)w);
    rem = k - q * w;
    if (rem < 0) {
        --q;
        rem += w;
    } else if (rem >= w) {
        ++q;
        rem -= w;
    }
}

constexpr int kZminThreads = 1024;

__global__ void __launch_bounds__(kZminThreads)
active_zmin_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                   const ClsProjected* __restrict__ records,
                   ClsTileCache* __restrict__ tile_cache) {
    extern __shared__ uint32_t s_z[];
    const ClsView& view = views[blockIdx.y];
    const ClsScene& sc = scenes[view.scene];
    const int nt = view.tiles_x * view.tiles_y;
    if (sc.n_active == 0) return;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) s_z[i] = 0xffffffffu;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const int stride = gridDim.x * warps;
    int i = blockIdx.x * warps + (threadIdx.x >> 5);
    // the next Gaussian's record is requested before this one is processed
    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c2 = c0;
    if (i < sc.n_active) {
        const float4* r = reinterpret_cast<const float4*>(records + view.rec_base +
                                                          sc.active_idx[i]);
        c0 = r[0];
        c2 = r[2];
    }
    for (; i < sc.n_active; i += stride) {
        const float4 cur0 = c0, cur2 = c2;
        if (i + stride < sc.n_active) {
            const float4* r = reinterpret_cast<const float4*>(records + view.rec_base +
                                                              sc.active_idx[i + stride]);
            c0 = r[0];
            c2 = r[2];
        }
        const int radius = __float_as_int(cur2.w);
        const uint32_t zb = __float_as_uint(cur2.z);
        int x0, x1, y0, y1;
        if (radius <= 0 || !tile_rect(cur0.x, cur0.y, (float)radius, view.tiles_x, view.tiles_y,
                                      x0, x1, y0, y1))
            continue;  // uniform over the warp
        const int w = x1 - x0 + 1;
        const int area = w * (y1 - y0 + 1);
        for (int k = lane; k < area; k += 32) {
            int q, rem;
            divmod_small(k, w, q, rem);
            const int cell = (y0 + q) * view.tiles_x + x0 + rem;
            if (zb < s_z[cell]) atomicMin(&s_z[cell], zb);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const uint32_t z = s_z[i];
        if (z != 0xffffffffu) atomicMin(&tile_cache[view.tile_base + i].zmin_active, z);
    }
}

// Ascending list of active tiles and each tile's rank in it (-1 if inactive),
// and the static-prefix decision of every active tile: its cache holds while
// no active Gaussian of the tile lies in front of the boundary; otherwise the
// boundary moves a margin in front of the nearest active Gaussian and the
// prefix is rebuilt by the next forward pass (flat layout only, `decide` 1;
// the bucketed layout decides in col_counts_kernel). Two passes over chunks
// of kCompactChunk tiles around one scan of the chunk counts.
constexpr int kCompactPer = 4;  // consecutive tiles per thread
constexpr int kCompactChunk = 1024 * kCompactPer;

__global__ void __launch_bounds__(1024)
compact_count_kernel(const uint8_t* __restrict__ tile_active, int64_t n_tiles,
                     ClsTileCache* __restrict__ tile_cache, int prefix_mode, int decide,
                     int64_t* __restrict__ partials) {
    __shared__ int64_t smem[1024 / 32 + 1];
    const int64_t t0 = (int64_t)blockIdx.x * kCompactChunk + (int64_t)threadIdx.x * kCompactPer;
    int64_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kCompactPer; ++j) {
        const int64_t t = t0 + j;
        if (t < n_tiles && tile_active[t]) {
            ++cnt;
            if (!decide) continue;
            const ClsTileCache c = tile_cache[t];
            const bool keep = prefix_mode != 0 && c.n_prefix != CLS_PREFIX_UNKNOWN &&
                              c.zmin_active >= c.zb;
            if (!keep) {
                tile_cache[t].zb = c.zmin_active > kPrefixMargin ? c.zmin_active - kPrefixMargin
                                                                 : 0u;
                tile_cache[t].n_prefix = CLS_PREFIX_UNKNOWN;
            }
        }
    }
    int64_t tot;
    block_exclusive_sum<1024>(cnt, smem, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
compact_write_kernel(const uint8_t* __restrict__ tile_active, int64_t n_tiles,
                     const int64_t* __restrict__ offsets, int32_t* __restrict__ active_tiles,
                     int32_t* __restrict__ tile_rank) {
    __shared__ int64_t smem[1024 / 32 + 1];
    const int64_t t0 = (int64_t)blockIdx.x * kCompactChunk + (int64_t)threadIdx.x * kCompactPer;
    unsigned f = 0;
#pragma unroll
    for (int j = 0; j < kCompactPer; ++j)
        if (t0 + j < n_tiles && tile_active[t0 + j]) f |= 1u << j;
    int64_t tot;
    int64_t r = offsets[blockIdx.x] + block_exclusive_sum<1024>((int64_t)__popc(f), smem, tot);
#pragma unroll
    for (int j = 0; j < kCompactPer; ++j) {
        const int64_t t = t0 + j;
        if (t >= n_tiles) break;
        if (f & (1u << j)) {
            active_tiles[r] = (int32_t)t;
            tile_rank[t] = (int32_t)r++;
        } else {
            tile_rank[t] = -1;
        }
    }
}

__device__ __forceinline__ int rect_count(const int32_t* S, int Wd, int x0, int x1, int y0,
                                          int y1) {
    return S[(int64_t)(y1 + 1) * Wd + x1 + 1] - S[(int64_t)y0 * Wd + x1 + 1] -
           S[(int64_t)(y1 + 1) * Wd + x0] + S[(int64_t)y0 * Wd + x0];
}

// Pairs of one record (active tiles inside its rectangle), O(1) from the SAT.
__device__ __forceinline__ int pair_count(const ClsView& view, const uint4* rects,
                                          const int32_t* sat, int g, int& x0, int& x1, int& y0,
                                          int& y1, uint32_t& zbits) {
    if (!record_rect(rects, view.rec_base + g, x0, x1, y0, y1, zbits)) return 0;
    return rect_count(sat + view.sat_base, view.tiles_x + 1, x0, x1, y0, y1);
}

// The per-call resets of the bucketed binning, in one launch instead of a
// memset each: the render-mask difference grid, the flat layout's large-rect
// counter, the work-list, emission-group and block-ticket counters, the range
// of occupied active bins (lowest all ones, highest 0), the per-chunk pair
// totals and the tile ranges.
__global__ void reset_bucketed_kernel(int32_t* __restrict__ diff, int64_t n_diff,
                                      int32_t* __restrict__ big_count,
                                      int32_t* __restrict__ work_count, int n_work,
                                      uint32_t* __restrict__ arange, int n_views,
                                      int64_t* __restrict__ tile_partials, int64_t n_partials,
                                      uint32_t* __restrict__ ranges, int64_t n_ranges) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < n_diff; i += stride) diff[i] = 0;
    for (int64_t i = i0; i < n_ranges; i += stride) ranges[i] = 0u;
    for (int64_t i = i0; i < n_partials; i += stride) tile_partials[i] = 0;
    for (int64_t i = i0; i < n_work; i += stride) work_count[i] = 0;
    for (int64_t i = i0; i < 2 * (int64_t)n_views; i += stride)
        arange[i] = i < n_views ? 0xffffffffu : 0u;
    if (i0 == 0) *big_count = 0;
}

// Per-chunk pair totals (flat layout, `partials`), per view the depth range of
// the Gaussians that produce pairs and the list of pair-producing records
// (bucketed layout).
__global__ void __launch_bounds__(kBinBlock)
count_pairs_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                   const uint4* __restrict__ rects, const int32_t* __restrict__ sat,
                   int chunks_per_view, int64_t* __restrict__ partials,
                   uint32_t* __restrict__ zmin, uint32_t* __restrict__ zmax,
                   uint4* __restrict__ work_list, int32_t* __restrict__ work_count) {
    __shared__ int64_t smem[kBinBlock / 32 + 1];
    __shared__ int32_t smem32[kBinBlock / 32 + 1];
    __shared__ uint32_t s_lo, s_hi;
    __shared__ int32_t s_base;
    const ClsView& view = views[blockIdx.y];
    const int n = scenes[view.scene].n;
    if (threadIdx.x == 0) { s_lo = 0xffffffffu; s_hi = 0u; }
    __syncthreads();
    int64_t cnt = 0;
    uint32_t lo = 0xffffffffu, hi = 0u;
    unsigned produces = 0;  // bit `it`: item `it` of this thread has pairs
    uint4 rr[kBinItems];    // the items' packed rectangles, kept for the work list
#pragma unroll
    for (int it = 0; it < kBinItems; ++it) {
        const int g = blockIdx.x * kBinChunk + it * kBinBlock + threadIdx.x;
        rr[it] = g < n ? rects[view.rec_base + g] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int it = 0; it < kBinItems; ++it) {
        if (rr[it].w == 0u) continue;  // not visible (or past the scene)
        int x0, x1, y0, y1;
        unpack_rect(rr[it], x0, x1, y0, y1);
        const int c = rect_count(sat + view.sat_base, view.tiles_x + 1, x0, x1, y0, y1);
        if (c > 0) {
            cnt += c;
            lo = min(lo, rr[it].z);
            hi = max(hi, rr[it].z);
            produces |= 1u << it;
        }
    }
    if (partials) {  // chunk pair totals (flat layout)
        int64_t tot;
        block_exclusive_sum<kBinBlock>(cnt, smem, tot);
        if (threadIdx.x == 0) partials[(int64_t)blockIdx.y * chunks_per_view + blockIdx.x] = tot;
    }
    if (work_list) {  // compact the pair-producing records: one atomic per block
        int32_t nw;
        int32_t k = block_exclusive_sum<kBinBlock>((int32_t)__popc(produces), smem32, nw);
        if (threadIdx.x == 0) s_base = nw > 0 ? atomicAdd(work_count + blockIdx.y, nw) : 0;
        __syncthreads();
        k += s_base;
        // a work item is the record's packed rectangle with its record index
        // in place of the visible flag
#pragma unroll
        for (int it = 0; it < kBinItems; ++it)
            if (produces & (1u << it)) {
                const int64_t rec = view.rec_base + blockIdx.x * kBinChunk + it * kBinBlock +
                                    threadIdx.x;
                uint4 r = rr[it];
                r.w = (uint32_t)rec;
                work_list[view.rec_base + k++] = r;
            }
    }
    if (zmin) {
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if ((threadIdx.x & 31) == 0 && hi >= lo) {
            atomicMin(&s_lo, lo);
            atomicMax(&s_hi, hi);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_hi >= s_lo) {
            atomicMin(zmin + blockIdx.y, s_lo);
            atomicMax(zmax + blockIdx.y, s_hi);
        }
    }
}

// ---------------------------------------------------------------------------
// Bucketed layout: pairs per (tile, depth bin).
//
// A view's depth range (the depth bits of its pair-producing Gaussians) is
// fixed by the call that projects every Gaussian (project_mode 0) and kept by
// later calls, so a static Gaussian's depth bin does not change during an
// update and its pairs per (tile, bin) form a fixed 2D prefix sum S of
// difference-grid stamps, computed by that call. Every call stamps only the
// active Gaussians' rectangles into a second difference grid A (in their
// projection once the bins are fixed), prefix-sums
// the bins they occupy, and adds the two at the rendered tiles. Both grids are
// bin-fastest: entry (cell y * (Tx + 1) + x of the view, bin b) at
// (sat_base + cell) * kDepthBins + b, so a block of kDepthBins threads walks a
// row or a column with coalesced loads. The passes over A clear every entry
// they read, so A is zero between calls.
// ---------------------------------------------------------------------------

// S stamps: every visible static record of the view (rectangle flag 1).
__global__ void __launch_bounds__(kBinBlock)
stamp_static_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                    const uint4* __restrict__ rects, const uint32_t* __restrict__ zmin,
                    const uint32_t* __restrict__ zmax, int32_t* __restrict__ S) {
    const ClsView& view = views[blockIdx.y];
    const int n = scenes[view.scene].n;
    const DepthBins db = depth_bins(zmin[blockIdx.y], zmax[blockIdx.y]);
    int32_t* G = S + view.sat_base * kDepthBins;
    for (int g = blockIdx.x * kBinBlock + threadIdx.x; g < n; g += gridDim.x * kBinBlock) {
        const uint4 r = rects[view.rec_base + g];
        if (r.w != 1u) continue;
        int x0, x1, y0, y1;
        unpack_rect(r, x0, x1, y0, y1);
        stamp_rect_bin(G, view.tiles_x + 1, depth_bin(r.z, db), x0, x1, y0, y1);
    }
}

// A stamps: every visible active record of the view (rectangle flag 2), and
// the range of bins they occupy (arange[v] lowest, arange[V + v] highest). Used
// by a call that fixes the depth bins (project_mode 0); later calls make the
// same stamps in the projection of the active records (project_kernel<1>).
__global__ void __launch_bounds__(kBinBlock)
stamp_active_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                    const uint4* __restrict__ rects, const uint32_t* __restrict__ zmin,
                    const uint32_t* __restrict__ zmax, int32_t* __restrict__ A,
                    uint32_t* __restrict__ arange) {
    const ClsView& view = views[blockIdx.y];
    const ClsScene& sc = scenes[view.scene];
    const DepthBins db = depth_bins(zmin[blockIdx.y], zmax[blockIdx.y]);
    int32_t* G = A + view.sat_base * kDepthBins;
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int i = blockIdx.x * kBinBlock + threadIdx.x; i < sc.n_active;
         i += gridDim.x * kBinBlock) {
        const uint4 r = rects[view.rec_base + sc.active_idx[i]];
        if (r.w == 0u) continue;
        int x0, x1, y0, y1;
        unpack_rect(r, x0, x1, y0, y1);
        const int b = depth_bin(r.z, db);
        lo = min(lo, (uint32_t)b);
        hi = max(hi, (uint32_t)b);
        stamp_rect_bin(G, view.tiles_x + 1, b, x0, x1, y0, y1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0 && hi >= lo) {
        atomicMin(arange + blockIdx.y, lo);
        atomicMax(arange + gridDim.y + blockIdx.y, hi);
    }
}

// Prefix sums along x of every row of a grid (blocks of kDepthBins threads
// striding over the rows of view blockIdx.y, a thread per bin; with `arange`
// only the view's occupied bins). With `clear`, the column x = Tx and the row
// y = Ty, which no later pass reads, are cleared.
__device__ __forceinline__ void row_prefix(int32_t* p, int Tx, int clear) {
    int32_t run = 0;
    int x = 0;
    for (; x + 8 <= Tx; x += 8) {  // eight loads in flight
        int32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = p[(int64_t)(x + k) * kDepthBins];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            run += v[k];
            p[(int64_t)(x + k) * kDepthBins] = run;
        }
    }
    for (; x < Tx; ++x) {
        run += p[(int64_t)x * kDepthBins];
        p[(int64_t)x * kDepthBins] = run;
    }
    if (clear) p[(int64_t)Tx * kDepthBins] = 0;
}

__global__ void __launch_bounds__(kDepthBins)
row_prefix_kernel(const ClsView* __restrict__ views, int32_t* __restrict__ G,
                  const uint32_t* __restrict__ arange, int clear) {
    const ClsView& view = views[blockIdx.y];
    const int Tx = view.tiles_x, Ty = view.tiles_y, Wd = Tx + 1;
    const uint32_t b = threadIdx.x;
    if (arange && (b < arange[blockIdx.y] || b > arange[gridDim.y + blockIdx.y])) return;
    for (int y = blockIdx.x; y <= Ty; y += gridDim.x) {
        int32_t* p = G + (view.sat_base + (int64_t)y * Wd) * kDepthBins + b;
        if (y < Ty) {
            row_prefix(p, Tx, clear);
        } else if (clear) {
            for (int x = 0; x <= Tx; ++x) p[(int64_t)x * kDepthBins] = 0;
        }
    }
}

// Prefix sums along y of S (after row_prefix_kernel): S then holds, at every
// tile (y < Ty, x < Tx), its static pairs per bin. Blocks stride over the
// columns of view blockIdx.y.
__device__ __forceinline__ void col_prefix(int32_t* p, int Ty, int64_t step) {
    int32_t run = 0;
    int y = 0;
    for (; y + 8 <= Ty; y += 8) {
        int32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = p[(y + k) * step];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            run += v[k];
            p[(y + k) * step] = run;
        }
    }
    for (; y < Ty; ++y) {
        run += p[y * step];
        p[y * step] = run;
    }
}

__global__ void __launch_bounds__(kDepthBins)
col_prefix_kernel(const ClsView* __restrict__ views, int32_t* __restrict__ S) {
    const ClsView& view = views[blockIdx.y];
    const int Tx = view.tiles_x, Ty = view.tiles_y;
    const int64_t step = (int64_t)(Tx + 1) * kDepthBins;
    for (int x = blockIdx.x; x < Tx; x += gridDim.x)
        col_prefix(S + (view.sat_base + x) * kDepthBins + threadIdx.x, Ty, step);
}

// Per (column, view) block, a thread per bin: walks the column's tiles,
// completing A's prefix sums along y (and clearing A); at each rendered tile
// writes its pairs per bin, S + A, to counts[rank * kDepthBins + bin]. Per
// rendered tile also: its pair total (ttot[rank], and into its chunk's partial
// sum), the nearest active Gaussian's depth bin ba (the first bin where A is
// non-zero) and the static-prefix decision. A cached prefix holds while its
// boundary zb lies at or in front of edge(ba), the lowest depth of bin ba
// (then every active Gaussian of the tile has bits(z) >= zb); otherwise, or
// with prefix_mode 0, the boundary moves to edge(ba - 1), one bin in front,
// so that a nearest active Gaussian moving forward by less than a bin keeps
// the prefix, and the prefix is rebuilt by the next forward pass; the tile's
// depth cut (if any) is then raised to at least the old boundary's bin plus
// the margin. front[tile] = first bin to emit. Rows are processed eight at a time, their
// loads issued together.
constexpr int kTileChunk = 64;  // tiles per partial sum of the pair totals

// A tile whose cached prefix is dropped walks from the front again; its pixels
// that stopped inside the old prefix need no bin behind the old boundary's, so
// its cut covers that bin plus the margin. Kept out of line: the rare call
// would otherwise cost the column walk registers.
__device__ __noinline__ void raise_cut(uint8_t* cut, uint32_t old_zb, DepthBins db) {
    const int need = min(kDepthBins - 1, depth_bin(old_zb, db) + kCutMargin);
    if ((int)*cut < need) *cut = (uint8_t)need;
}

__global__ void __launch_bounds__(kDepthBins, 3)  // three blocks per SM: the grid in about one wave
col_counts_kernel(const ClsView* __restrict__ views, const int32_t* __restrict__ S,
                  int32_t* __restrict__ A, const uint32_t* __restrict__ arange,
                  const uint32_t* __restrict__ zmin, const uint32_t* __restrict__ zmax,
                  const int32_t* __restrict__ tile_rank, ClsTileCache* __restrict__ tile_cache,
                  int prefix_mode, int32_t* __restrict__ counts, uint8_t* __restrict__ front,
                  uint8_t* __restrict__ bin_cut, int32_t* __restrict__ ttot,
                  int64_t* __restrict__ tile_partials) {
    __shared__ int32_t s_tot[kDepthBins];
    __shared__ int32_t s_ba[kDepthBins];
    __shared__ int32_t s_rank[kDepthBins];
    const ClsView& view = views[blockIdx.y];
    const int Tx = view.tiles_x, Ty = view.tiles_y;
    const int b = threadIdx.x, lane = b & 31, warp = b >> 5;
    const bool occupied = (uint32_t)b >= arange[blockIdx.y] &&
                          (uint32_t)b <= arange[gridDim.y + blockIdx.y];
    const int64_t step = (int64_t)(Tx + 1) * kDepthBins;
    const int64_t tb = view.tile_base;
    const DepthBins db = depth_bins(zmin[blockIdx.y], zmax[blockIdx.y]);
    for (int x = blockIdx.x; x < Tx; x += gridDim.x) {
        const int32_t* sp = S + (view.sat_base + x) * kDepthBins + b;
        int32_t* ap = A + (view.sat_base + x) * kDepthBins + b;
        int32_t run = 0;
        for (int y0 = 0; y0 < Ty; y0 += kDepthBins) {
            const int ny = min(kDepthBins, Ty - y0);
            if (b < ny) {
                s_tot[b] = 0;
                s_ba[b] = kDepthBins;
                s_rank[b] = tile_rank[tb + (int64_t)(y0 + b) * Tx + x];
            }
            __syncthreads();
            for (int j0 = 0; j0 < ny; j0 += 8) {
                int32_t av[8], sv[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int j = j0 + k;
                    const int64_t at = (int64_t)(y0 + j) * step;
                    av[k] = occupied && j < ny ? ap[at] : 0;
                    sv[k] = j < ny && s_rank[j] >= 0 ? sp[at] : 0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int j = j0 + k;
                    if (j >= ny) break;  // uniform over the block
                    if (occupied) {
                        run += av[k];
                        ap[(int64_t)(y0 + j) * step] = 0;
                    }
                    const int r = s_rank[j];
                    if (r < 0) continue;
                    const int32_t c = sv[k] + run;
                    counts[(int64_t)r * kDepthBins + b] = c;
                    int32_t s = c;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                    const unsigned m = __ballot_sync(0xffffffffu, run > 0);
                    if (lane == 0) {
                        atomicAdd(&s_tot[j], s);
                        if (m) atomicMin(&s_ba[j], warp * 32 + __ffs(m) - 1);
                    }
                }
            }
            __syncthreads();
            if (b < ny) {
                const int64_t tile = tb + (int64_t)(y0 + b) * Tx + x;
                const int r = s_rank[b];
                if (r >= 0) {
                    ttot[r] = s_tot[b];
                    atomicAdd((unsigned long long*)(tile_partials + r / kTileChunk),
                              (unsigned long long)s_tot[b]);
                    const uint32_t edge = bin_edge(s_ba[b], db);
                    ClsTileCache c = tile_cache[tile];
                    const bool keep = prefix_mode != 0 && c.n_prefix != CLS_PREFIX_UNKNOWN &&
                                      c.zb <= edge;
                    if (!keep) {
                        if (bin_cut && c.n_prefix != CLS_PREFIX_UNKNOWN)
                            raise_cut(bin_cut + tile, c.zb, db);
                        c.zb = s_ba[b] >= kDepthBins ? edge : bin_edge(s_ba[b] - 1, db);
                        c.n_prefix = CLS_PREFIX_UNKNOWN;
                    }
                    c.zmin_active = edge;
                    tile_cache[tile] = c;
                    front[tile] = c.n_prefix != CLS_PREFIX_UNKNOWN ? (uint8_t)depth_bin(c.zb, db)
                                                                   : (uint8_t)0;
                }
            }
            __syncthreads();
        }
    }
}

// Offsets of every (tile, bin) bucket, in place of its count in `cursor`
// (the emission's slot cursors) and in bin_offsets, and the per-tile ranges,
// all clamped to the key capacity so every later access stays inside the key
// buffer; per view the rank of its first rendered tile. One block per chunk
// of kTileChunk rendered tiles (its base from the scanned partial sums), a
// warp per tile, eight bins per lane.
__global__ void __launch_bounds__(256)
tile_offsets_kernel(const ClsView* __restrict__ views, int n_views,
                    const int32_t* __restrict__ active_tiles, const int32_t* __restrict__ n_active,
                    const int32_t* __restrict__ ttot, const int64_t* __restrict__ tile_partials,
                    int64_t capacity, int32_t* __restrict__ cursor,
                    uint32_t* __restrict__ bin_offsets, uint32_t* __restrict__ ranges,
                    int32_t* __restrict__ rank0) {
    __shared__ int64_t smem[256 / 32 + 1];
    __shared__ int64_t s_base[kTileChunk];
    const int na = *n_active;
    const int t0 = blockIdx.x * kTileChunk;
    if (t0 >= na) return;
    const int i = threadIdx.x;
    const int64_t v = (i < kTileChunk && t0 + i < na) ? (int64_t)ttot[t0 + i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_sum<256>(v, smem, tot);
    if (i < kTileChunk) s_base[i] = tile_partials[blockIdx.x] + ex;
    __syncthreads();
    const int lane = i & 31, warp = i >> 5;
    auto clamp = [&](int64_t o) { return (uint32_t)(o < capacity ? o : capacity); };
    for (int k = warp; k < kTileChunk && t0 + k < na; k += 8) {
        const int t = t0 + k;
        int32_t* cp = cursor + (int64_t)t * kDepthBins + lane * 8;
        const int4 a = *reinterpret_cast<const int4*>(cp);
        const int4 c = *reinterpret_cast<const int4*>(cp + 4);
        const int32_t n8[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
        int32_t sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) sum += n8[j];
        int32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int64_t off = s_base[k] + (incl - sum);
        uint32_t o8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o8[j] = clamp(off);
            off += n8[j];
        }
        const uint4 lo = make_uint4(o8[0], o8[1], o8[2], o8[3]);
        const uint4 hi = make_uint4(o8[4], o8[5], o8[6], o8[7]);
        *reinterpret_cast<uint4*>(cp) = lo;
        *reinterpret_cast<uint4*>(cp + 4) = hi;
        uint32_t* bo = bin_offsets + (int64_t)t * kDepthBins + lane * 8;
        *reinterpret_cast<uint4*>(bo) = lo;
        *reinterpret_cast<uint4*>(bo + 4) = hi;
        if (lane == 31) {
            const int64_t tile = active_tiles[t];
            const uint32_t end = clamp(off);
            ranges[2 * tile] = clamp(s_base[k]);
            ranges[2 * tile + 1] = end;
            // the next tile's first offset, or the sentinel after the last tile
            if (t == na - 1) bin_offsets[(int64_t)na * kDepthBins] = end;
            const int vv = view_of_tile(views, n_views, (int)tile);
            if (t == 0 || active_tiles[t - 1] < views[vv].tile_base) rank0[vv] = t;
        }
    }
}

// Flat layout: pairs in view, Gaussian, row-major tile order at scanned
// offsets. Rectangles larger than kBigArea tiles go to a list that one warp per
// Gaussian emits (emit_big_kernel).
__global__ void __launch_bounds__(kBinBlock)
emit_pairs_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                  const uint4* __restrict__ rects, const int32_t* __restrict__ sat,
                  const uint8_t* __restrict__ tile_active, int chunks_per_view,
                  const int64_t* __restrict__ offsets, uint64_t* __restrict__ keys,
                  uint32_t* __restrict__ vals, int64_t capacity, uint4* __restrict__ big_list,
                  int32_t* __restrict__ big_count) {
    __shared__ int64_t smem[kBinBlock / 32 + 1];
    const ClsView& view = views[blockIdx.y];
    const int n = scenes[view.scene].n;
    int64_t base = offsets[(int64_t)blockIdx.y * chunks_per_view + blockIdx.x];
    for (int it = 0; it < kBinItems; ++it) {
        const int g = blockIdx.x * kBinChunk + it * kBinBlock + threadIdx.x;
        int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
        uint32_t zb = 0;
        const int64_t cnt = g < n ? pair_count(view, rects, sat, g, x0, x1, y0, y1, zb) : 0;
        int64_t tot;
        int64_t pos = base + block_exclusive_sum<kBinBlock>(cnt, smem, tot);
        base += tot;
        if (cnt == 0) continue;
        const uint32_t rec = (uint32_t)(view.rec_base + g);
        const int area = (x1 - x0 + 1) * (y1 - y0 + 1);
        if (area > kBigArea) {
            const int slot = atomicAdd(big_count, 1);
            big_list[slot] = make_uint4(rec, (uint32_t)blockIdx.y, (uint32_t)(pos & 0xffffffff),
                                        (uint32_t)(pos >> 32));
            continue;
        }
        for (int ty = y0; ty <= y1; ++ty) {
            const int64_t row = (int64_t)view.tile_base + (int64_t)ty * view.tiles_x;
            for (int tx = x0; tx <= x1; ++tx) {
                if (!tile_active[row + tx]) continue;
                if (pos < capacity) {
                    keys[pos] = ((uint64_t)(row + tx) << 32) | zb;
                    vals[pos] = rec;
                }
                ++pos;
            }
        }
    }
}

// Emission windows. Every rendered tile emits the depth bins from its first
// emitted bin (bins wholly in front of a cached prefix boundary are skipped)
// to its depth cut. Per tile the two are packed into 16 bits, first bin in the
// low byte and cut in the high byte; a tile that is not rendered holds the
// neutral 0x00ff, which admits no bin.
__device__ __forceinline__ uint32_t fc_pack(bool on, uint32_t first, uint32_t cut) {
    return on ? (first | (cut << 8)) : 0x00ffu;
}

// Window of the union of two runs of tiles: the smaller first bin, the larger cut.
__device__ __forceinline__ uint32_t fc_merge(uint32_t a, uint32_t b) {
    return min(a & 0xffu, b & 0xffu) | (max(a >> 8, b >> 8) << 8);
}

__device__ __forceinline__ bool fc_admits(uint32_t w, int bin) {
    return (int)(w & 0xffu) <= bin && bin <= (int)(w >> 8);
}

// Per tile row of every view: sparse tables of the packed windows over runs
// of 2^l tiles for l >= 1, level l at (l - 1) * total_tiles + tile (level 0 is
// the tiles' own windows).
constexpr int kRowLevels = 16;  // tiles per row < 2^16

__host__ __device__ __forceinline__ int row_levels(int Tx) {
    int levels = 0;
    while ((1 << levels) <= Tx) ++levels;  // 2^(levels - 1) <= Tx < 2^levels
    return levels;
}

// Shared memory of the emission: per tile a packed word (rank in the view's
// rendered tiles + 1 in the low half, 0 if not rendered; the window in the
// high half) and, when they fit, the row tables' levels 1 .. L-1. Views whose
// tables do not fit in `smem_bytes` use the global ones that
// bin_window_tables_kernel writes.
constexpr int kEmitThreads = 1024;

__host__ __device__ __forceinline__ bool emit_tables_fit(int64_t nt, int Tx, int64_t smem_bytes) {
    return nt * (4 + 2 * (int64_t)(row_levels(Tx) - 1)) <= smem_bytes;
}

// First lane of the warp whose inclusive cell prefix `incl` exceeds c (31 if
// none): a binary search by shuffles, every lane taking part.
__device__ __forceinline__ int owner_of(int incl, int c) {
    int lo = 0, hi = 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi) >> 1;
        const int pm = __shfl_sync(0xffffffffu, incl, mid);
        if (pm > c) hi = mid; else lo = mid + 1;
    }
    return lo;
}

__global__ void __launch_bounds__(1024)
bin_window_tables_kernel(const ClsView* __restrict__ views, const int32_t* __restrict__ tile_rank,
                         const uint8_t* __restrict__ front, const uint8_t* __restrict__ cut,
                         uint16_t* __restrict__ t_win, int64_t total_tiles, int emit_smem) {
    const ClsView& view = views[blockIdx.x];
    const int Tx = view.tiles_x, nt = Tx * view.tiles_y;
    const int64_t tb = view.tile_base;
    if (emit_tables_fit(nt, Tx, emit_smem)) return;  // the emission builds them itself
    auto win0 = [&](int i) {
        const bool on = tile_rank[tb + i] >= 0;
        return fc_pack(on, on ? front[tb + i] : 0u, cut ? cut[tb + i] : 255u);
    };
    for (int i = threadIdx.x; i < nt; i += blockDim.x)
        if (i % Tx + 2 <= Tx) t_win[tb + i] = (uint16_t)fc_merge(win0(i), win0(i + 1));
    for (int l = 2; l < kRowLevels && (1 << l) <= Tx; ++l) {
        __syncthreads();
        const int h = 1 << (l - 1);
        const int64_t prev = (int64_t)(l - 2) * total_tiles + tb, cur = prev + total_tiles;
        for (int i = threadIdx.x; i < nt; i += blockDim.x)
            if (i % Tx + 2 * h <= Tx)
                t_win[cur + i] = (uint16_t)fc_merge(t_win[prev + i], t_win[prev + i + h]);
    }
}

// Bucketed emission, load-balanced. A warp takes a group of 32 pair-producing
// records of one view, cuts each rectangle to the rows where its depth bin can
// be emitted and splits the cells of each cut rectangle into segments of
// kCells consecutive cells; per round each lane takes one segment, its record
// found by a binary search over the warp's segment prefix (the record's fields
// travel by shuffles, every lane taking part), and a cell whose tile admits
// the bin claims a slot in its (tile, depth bin) bucket. Persistent 1024-thread
// blocks, one wave; warps take groups from a per-view counter, the next group
// claimed and fetched while the current one is processed.
constexpr int kCells = 8;  // consecutive cells per lane and round

__global__ void __launch_bounds__(kEmitThreads)
emit_bucketed_kernel(const ClsView* __restrict__ views, const int32_t* __restrict__ tile_rank,
                     const int32_t* __restrict__ rank0, const uint32_t* __restrict__ zmin,
                     const uint32_t* __restrict__ zmax, int32_t* __restrict__ cursor,
                     uint64_t* __restrict__ keys, int64_t capacity,
                     const uint4* __restrict__ work_list, const int32_t* __restrict__ work_count,
                     int32_t* __restrict__ next_group, const uint8_t* __restrict__ cut,
                     const uint8_t* __restrict__ front, const uint16_t* __restrict__ t_win,
                     int64_t total_tiles, int smem_bytes, int n_views, int first_wave,
                     int32_t* __restrict__ ticket, int32_t* __restrict__ status) {
    extern __shared__ uint32_t s_tile[];
    __shared__ int s_view;
    // A block takes a view, builds its tables and works through the view's
    // groups beside the other blocks on it; when the view has none left it takes
    // the view with the most groups left, and leaves when no view has any, so
    // every group is processed whatever the grid. The first pick shares the
    // blocks out over the views in proportion to their groups. One thread
    // picks (other blocks advance the counters), so the whole block takes the
    // same view. A pick is of a view with groups left and every warp claims at
    // least one of its groups before the next pick, so a block's picks are
    // bounded; past the bound it reports CLS_ERR_INTERNAL and leaves.
    int64_t total_groups = 0;  // thread 0 only
    for (int round = 0;; ++round) {
        if (threadIdx.x == 0) {
            int pick = -1;
            if (round == 0) {
                for (int v = 0; v < n_views; ++v) total_groups += (work_count[v] + 31) / 32;
                const int t = atomicAdd(ticket, 1);
                if (t < first_wave) {
                    const int64_t target = ((int64_t)t * total_groups) / first_wave;  // its share
                    int64_t cum = 0;
                    for (int v = 0; v < n_views && pick < 0; ++v) {
                        cum += (work_count[v] + 31) / 32;
                        if (target < cum) pick = v;
                    }
                }
            }
            int best = 0;
            if (pick >= 0)
                best = (work_count[pick] + 31) / 32 - *(volatile int32_t*)(next_group + pick);
            if (best <= 0) {  // the share's view is done, or a later pick: the most left
                pick = -1;
                for (int v = 0; v < n_views; ++v) {
                    const int left =
                        (work_count[v] + 31) / 32 - *(volatile int32_t*)(next_group + v);
                    if (left > best) {
                        best = left;
                        pick = v;
                    }
                }
            }
            if (pick >= 0 && round > total_groups + n_views) {  // guard (never taken)
                set_status(status, CLS_ERR_INTERNAL);
                pick = -1;
            }
            s_view = pick;
        }
        __syncthreads();
        const int vi = s_view;
        if (vi < 0) return;
        const ClsView& view = views[vi];
        const int Tx = view.tiles_x;
        const int nt = Tx * view.tiles_y;
        const int n = work_count[vi];
        uint16_t* s_lv = reinterpret_cast<uint16_t*>(s_tile + nt);
        const int r0 = rank0[vi];  // rank of the view's first rendered tile
        const int64_t tb = view.tile_base;
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            const int r = tile_rank[tb + i];
            const bool on = r >= 0;
            const uint32_t win = fc_pack(on, on ? front[tb + i] : 0u, cut ? cut[tb + i] : 255u);
            s_tile[i] = (on ? (uint32_t)(r - r0 + 1) : 0u) | (win << 16);
        }
        const int levels = row_levels(Tx);
        const bool fits = emit_tables_fit(nt, Tx, smem_bytes);
        if (fits) {  // the row tables of the view, built here in shared memory (a warp per row)
            const int Ty = view.tiles_y, wy = threadIdx.x >> 5, lx = threadIdx.x & 31;
            __syncthreads();
            for (int y = wy; y < Ty; y += kEmitThreads / 32)
                for (int x = lx; x + 2 <= Tx; x += 32) {
                    const int i = y * Tx + x;
                    s_lv[i] = (uint16_t)fc_merge(s_tile[i] >> 16, s_tile[i + 1] >> 16);
                }
            for (int l = 2; l < levels; ++l) {
                __syncthreads();
                const int h = 1 << (l - 1);
                const int prev = (l - 2) * nt, cur = prev + nt;
                for (int y = wy; y < Ty; y += kEmitThreads / 32)
                    for (int x = lx; x + 2 * h <= Tx; x += 32) {
                        const int i = y * Tx + x;
                        s_lv[cur + i] = (uint16_t)fc_merge(s_lv[prev + i], s_lv[prev + i + h]);
                    }
            }
        }
        __syncthreads();
        const int lane = threadIdx.x & 31;
        const DepthBins db = depth_bins(zmin[vi], zmax[vi]);
        const uint4* wl = work_list + view.rec_base;
        int g_next = 0;
        if (lane == 0) g_next = atomicAdd(next_group + vi, 1);
        g_next = __shfl_sync(0xffffffffu, g_next, 0);
        uint4 it_next = make_uint4(0u, 0u, 0u, 0u);
        if (g_next * 32 + lane < n) it_next = wl[g_next * 32 + lane];
        for (;;) {
            const int g = g_next;
            const uint4 item = it_next;
            if (g * 32 >= n) break;
            {  // claim and fetch the next group now
                int gn = 0;
                if (lane == 0) gn = atomicAdd(next_group + vi, 1);
                g_next = __shfl_sync(0xffffffffu, gn, 0);
                if (g_next * 32 + lane < n) it_next = wl[g_next * 32 + lane];
            }
            int x0 = 0, x1 = -1, y0 = 0, y1 = -1, bin = 0, area = 0;
            const bool has = g * 32 + lane < n;
            const uint16_t* T = nullptr;
            int st = 1, d = 0;
            if (has) {
                unpack_rect(item, x0, x1, y0, y1);
                bin = depth_bin(item.z, db);
                const int l = 31 - __clz(x1 - x0 + 1);
                T = l == 0 ? reinterpret_cast<const uint16_t*>(s_tile) + 1
                    : fits ? s_lv + (l - 1) * nt
                           : t_win + (int64_t)(l - 1) * total_tiles + tb;
                st = l == 0 ? 2 : 1;
                d = (x1 - x0 + 1 - (1 << l)) * st;
            }
            // The rows of the rectangle where the bin can be emitted (a row
            // qualifies when some tile of it admits the bin; two overlapping runs
            // of 2^l tiles from the row tables cover its columns): the first and
            // the last such row. The loop runs to the warp's tallest rectangle
            // with every lane in it, so that the warp reaches the shuffles below
            // converged (lanes leaving per-lane loops at different trip counts
            // were seen to fall out of step with the rest of the warp).
            const int h = has ? y1 - y0 + 1 : 0;
            int hmax = h;
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
            int ra = -1, rb = -1;
            int64_t at = (int64_t)(y0 * Tx + x0) * st;
            for (int k = 0; k < hmax; ++k, at += Tx * st) {
                if (k < h && fc_admits(fc_merge(T[at], T[at + d]), bin)) {
                    if (ra < 0) ra = y0 + k;
                    rb = y0 + k;
                }
            }
            if (ra >= 0) {
                y0 = ra;
                y1 = rb;
                area = (x1 - x0 + 1) * (y1 - y0 + 1);
            }
            // The cells of each cut rectangle are split into segments of kCells
            // consecutive cells; lanes take whole segments (the segment prefix
            // over the warp gives each lane its record), so a lane's cells never
            // cross a record boundary.
            const int segs = (area + kCells - 1) / kCells;
            int incl = segs;
    #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);  // segments of the group
            const int first = incl - segs;
            const uint32_t xy = (uint32_t)x0 | ((uint32_t)y0 << 16);
            const uint32_t wb = (uint32_t)(x1 - x0 + 1) | ((uint32_t)bin << 16);
            for (int s0 = 0; s0 < total; s0 += 32) {
                const int sg = s0 + lane;
                const int own = owner_of(incl, sg);
                const int o_first = __shfl_sync(0xffffffffu, first, own);
                const int o_area = __shfl_sync(0xffffffffu, area, own);
                const uint32_t o_xy = __shfl_sync(0xffffffffu, xy, own);
                const uint32_t o_wb = __shfl_sync(0xffffffffu, wb, own);
                const uint64_t key = ((uint64_t)__shfl_sync(0xffffffffu, item.z, own) << 32) |
                                     __shfl_sync(0xffffffffu, item.w, own);
                const int w = max((int)(o_wb & 0xffffu), 1), ob = (int)(o_wb >> 16);
                const int k0 = (sg - o_first) * kCells;  // first cell of the segment in its record
                const int len = sg < total ? min(kCells, o_area - k0) : 0;
                int q, rem;
                divmod_small(max(k0, 0), w, q, rem);
                int cell = ((int)(o_xy >> 16) + q) * Tx + (int)(o_xy & 0xffffu) + rem;
                int32_t sub[kCells];
    #pragma unroll
                for (int u = 0; u < kCells; ++u) {
                    sub[u] = -1;
                    if (u < len) {
                        // guard (never taken): the cell is a tile of the view
                        const bool in_view = cell >= 0 && cell < nt;
                        const uint32_t word = in_view ? s_tile[cell] : 0x00ff0000u;
                        const int r = r0 + (int)(word & 0xffffu) - 1;
                        const bool admit = fc_admits(word >> 16, ob);
                        if (admit && r >= 0 && r < total_tiles) sub[u] = r * kDepthBins + ob;
                        else if (admit || !in_view) set_status(status, CLS_ERR_INTERNAL);
                        if (++rem == w) {
                            rem = 0;
                            cell += Tx - w + 1;
                        } else {
                            ++cell;
                        }
                    }
                }
                int32_t p[kCells];
    #pragma unroll
                for (int u = 0; u < kCells; ++u)
                    p[u] = sub[u] >= 0 ? atomicAdd(cursor + sub[u], 1) : -1;
    #pragma unroll
                for (int u = 0; u < kCells; ++u)
                    if (p[u] >= 0 && p[u] < capacity) keys[p[u]] = key;
            }
        }
        __syncthreads();  // every warp done with the view's tables
    }
}

// Completion of tiles whose depth cut was too shallow: every pair-producing
// Gaussian of the tile's view is tested against the tile and, if its depth bin
// lies beyond the old cut, claims a slot in its bucket. Work items are (tile,
// chunk of the view's list), taken from a counter.
constexpr int kCompleteChunks = 64;

__global__ void __launch_bounds__(256)
complete_tiles_kernel(const ClsView* __restrict__ views, int n_views,
                      const uint32_t* __restrict__ zmin,
                      const uint32_t* __restrict__ zmax, int32_t* __restrict__ cursor,
                      uint64_t* __restrict__ keys, int64_t capacity,
                      const uint4* __restrict__ work_list,
                      const int32_t* __restrict__ work_count, const int32_t* __restrict__ trunc,
                      const int32_t* __restrict__ trunc_count, int64_t trunc_cap,
                      const uint8_t* __restrict__ front, int* __restrict__ item_counter) {
    __shared__ int s_item;
    const int n_items = (int)min((int64_t)*trunc_count, trunc_cap) * kCompleteChunks;
    if (n_items <= 0) return;  // nothing truncated (the usual case): no queue traffic
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(item_counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const int e = item / kCompleteChunks, chunk = item - e * kCompleteChunks;
        const int tile = trunc[e], rank = trunc[trunc_cap + e], old_cut = trunc[2 * trunc_cap + e];
        const int v = view_of_tile(views, n_views, tile);
        const ClsView& view = views[v];
        const int local = tile - view.tile_base;
        const int ty = local / view.tiles_x, tx = local - ty * view.tiles_x;
        const int n = work_count[v];
        const int first_bin = front[tile];
        const DepthBins db = depth_bins(zmin[v], zmax[v]);
        const int per = (n + kCompleteChunks - 1) / kCompleteChunks;
        const int a = chunk * per, b = min(n, a + per);
        for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
            const uint4 r = work_list[view.rec_base + i];
            int x0, x1, y0, y1;
            unpack_rect(r, x0, x1, y0, y1);
            if (tx < x0 || tx > x1 || ty < y0 || ty > y1) continue;
            const int bin = depth_bin(r.z, db);
            if (bin <= old_cut || bin < first_bin) continue;
            const int64_t p = atomicAdd(cursor + (int64_t)rank * kDepthBins + bin, 1);
            if (p < capacity) keys[p] = ((uint64_t)r.z << 32) | r.w;
        }
    }
}

// One warp per large rectangle (flat layout); lanes walk its tiles in
// row-major order, kept with a ballot prefix.
__global__ void __launch_bounds__(256)
emit_big_kernel(const ClsView* __restrict__ views, const uint4* __restrict__ rects,
                const uint8_t* __restrict__ tile_active, uint64_t* __restrict__ keys,
                uint32_t* __restrict__ vals, int64_t capacity,
                const uint4* __restrict__ big_list, const int32_t* __restrict__ big_count) {
    const int lane = threadIdx.x & 31;
    const int nbig = *big_count;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nbig;
         w += (gridDim.x * blockDim.x) >> 5) {
        const uint4 item = big_list[w];
        const ClsView& view = views[item.y];
        int x0, x1, y0, y1;
        uint32_t zb;
        record_rect(rects, item.x, x0, x1, y0, y1, zb);
        const int wdt = x1 - x0 + 1;
        const int area = wdt * (y1 - y0 + 1);
        int64_t pos = ((int64_t)item.w << 32) | item.z;
        for (int k0 = 0; k0 < area; k0 += 32) {
            const int k = k0 + lane;
            int64_t tile = 0;
            bool on = false;
            if (k < area) {
                const int ty = y0 + k / wdt, tx = x0 + k % wdt;
                tile = (int64_t)view.tile_base + (int64_t)ty * view.tiles_x + tx;
                on = tile_active[tile] != 0;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, on);
            const int64_t p = pos + __popc(m & ((1u << lane) - 1u));
            if (on && p < capacity) {
                keys[p] = ((uint64_t)tile << 32) | zb;
                vals[p] = item.x;
            }
            pos += __popc(m);
        }
    }
}

}  // namespace cls

using namespace cls;

namespace {

__global__ void capacity_check_kernel(const int64_t* n_pairs, int64_t capacity,
                                      int32_t* status) {
    if (threadIdx.x == 0 && *n_pairs > capacity) set_status(status, CLS_ERR_CAPACITY);
}

struct ProjLayout {
    size_t partials, sat, diff, zmin, zmax, tile_rank, cursor, tile_partials, big_list,
        big_count, sbins, abins, arange, ttot, work_list, work_count, front, t_win, rank0, compact,
        rects, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int64_t bin_chunks_per_view(const ClsBatchInfo* info) {
    return (info->max_n + kBinChunk - 1) / kBinChunk;
}

ProjLayout proj_layout(const ClsBatchInfo* info) {
    ProjLayout L;
    const int64_t V = info->n_views;
    const int64_t subs = info->total_tiles * kDepthBins;
    size_t o = 0;
    L.partials = o; o = align256(o + (size_t)(bin_chunks_per_view(info) * V + 1) * 8);
    L.sat = o; o = align256(o + (size_t)info->total_sat * 4);
    L.diff = o; o = align256(o + (size_t)info->total_sat * 4);
    L.zmin = o; o = align256(o + (size_t)V * 4);
    L.zmax = o; o = align256(o + (size_t)V * 4);
    L.tile_rank = o; o = align256(o + (size_t)info->total_tiles * 4);
    L.cursor = o; o = align256(o + (size_t)subs * 4);
    L.tile_partials = o;
    o = align256(o + (size_t)((info->total_tiles + kTileChunk - 1) / kTileChunk + 1) * 8);
    L.big_list = o; o = align256(o + (size_t)info->total_records * 16);
    L.big_count = o; o = align256(o + 4);
    L.sbins = o; o = align256(o + (size_t)kDepthBins * info->total_sat * 4);
    L.abins = o; o = align256(o + (size_t)kDepthBins * info->total_sat * 4);
    L.arange = o; o = align256(o + (size_t)V * 8);
    L.ttot = o; o = align256(o + (size_t)info->total_tiles * 4);
    L.work_list = o; o = align256(o + (size_t)info->total_records * 16);
    L.work_count = o;  // + per-view emission counters + the emission's block ticket
    o = align256(o + (size_t)V * 8 + 4);
    L.front = o; o = align256(o + (size_t)info->total_tiles);
    L.t_win = o; o = align256(o + (size_t)info->total_tiles * (kRowLevels - 1) * 2);
    L.rank0 = o; o = align256(o + (size_t)V * 4);
    L.compact = o;
    o = align256(o + (size_t)((info->total_tiles + kCompactChunk - 1) / kCompactChunk + 1) * 8);
    L.rects = o; o = align256(o + (size_t)info->total_records * 16);
    L.total = o;
    return L;
}

}  // namespace

// SM count of the device; the kernels' raised shared-memory limits are set
// with it, once per device
static PerDevice g_proj_sms;

extern "C" size_t cls_project_workspace_size(const ClsBatchInfo* info) {
    return info ? proj_layout(info).total : 0;
}

extern "C" size_t cls_bin_offsets_size(const ClsBatchInfo* info) {
    return info ? (size_t)(info->total_tiles * kDepthBins + 1) : 0;
}

extern "C" int cls_project_and_bin(const ClsScene* scenes_dev, const ClsView* views_dev,
                                   const ClsBatchInfo* info, int32_t project_mode, int32_t layout,
                                   ClsProjected* records, uint8_t* tile_active,
                                   int32_t* active_tiles, int32_t* n_active_tiles_dev,
                                   uint64_t* keys, uint32_t* vals, int64_t capacity,
                                   int64_t* n_pairs_dev, uint32_t* ranges, uint32_t* bin_offsets,
                                   uint8_t* bin_cut, ClsTileCache* tile_cache,
                                   int32_t prefix_mode, int32_t tile_ring, int32_t* status_dev,
                                   void* workspace, size_t workspace_bytes, cls_stream_t stream) {
    if (!info || !scenes_dev || !views_dev || !records || !tile_active || !active_tiles ||
        !n_active_tiles_dev || !n_pairs_dev || !status_dev || !workspace || capacity < 0 ||
        !tile_cache || (prefix_mode != 0 && prefix_mode != 1) || (tile_ring != 0 && tile_ring != 1) ||
        project_mode < 0 || project_mode > 2 || (layout != 0 && layout != 1) ||
        (project_mode == 2 && (layout != 1 || keys == nullptr || capacity <= 0)) ||
        (capacity > 0 && !keys) || (layout == 0 && capacity > 0 && !vals) ||
        (layout == 1 && (!ranges || !bin_offsets)))
        return CLS_ERR_INVALID_ARG;
    if (info->n_views <= 0 || info->n_views > 65535 || info->total_tiles <= 0 ||
        workspace_bytes < cls_project_workspace_size(info) || capacity >= ((int64_t)1 << 32))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const unsigned V = (unsigned)info->n_views;
    const int64_t cpv = bin_chunks_per_view(info);
    const ProjLayout L = proj_layout(info);
    char* ws = static_cast<char*>(workspace);
    int64_t* partials = reinterpret_cast<int64_t*>(ws + L.partials);
    int32_t* sat = reinterpret_cast<int32_t*>(ws + L.sat);
    int32_t* diff = reinterpret_cast<int32_t*>(ws + L.diff);
    uint32_t* zmin = reinterpret_cast<uint32_t*>(ws + L.zmin);
    uint32_t* zmax = reinterpret_cast<uint32_t*>(ws + L.zmax);
    int32_t* tile_rank = reinterpret_cast<int32_t*>(ws + L.tile_rank);
    int32_t* cursor = reinterpret_cast<int32_t*>(ws + L.cursor);
    int64_t* tile_partials = reinterpret_cast<int64_t*>(ws + L.tile_partials);
    uint4* big_list = reinterpret_cast<uint4*>(ws + L.big_list);
    int32_t* big_count = reinterpret_cast<int32_t*>(ws + L.big_count);
    int32_t* sbins = reinterpret_cast<int32_t*>(ws + L.sbins);
    int32_t* abins = reinterpret_cast<int32_t*>(ws + L.abins);
    uint32_t* arange = reinterpret_cast<uint32_t*>(ws + L.arange);
    int32_t* ttot = reinterpret_cast<int32_t*>(ws + L.ttot);
    uint4* work_list = reinterpret_cast<uint4*>(ws + L.work_list);
    int32_t* work_count = reinterpret_cast<int32_t*>(ws + L.work_count);
    uint8_t* front = reinterpret_cast<uint8_t*>(ws + L.front);
    uint16_t* t_win = reinterpret_cast<uint16_t*>(ws + L.t_win);
    int32_t* rank0 = reinterpret_cast<int32_t*>(ws + L.rank0);
    uint4* rects = reinterpret_cast<uint4*>(ws + L.rects);  // kept from call to call
    const int64_t subs = info->total_tiles * kDepthBins;
    const int64_t max_view_tiles = info->max_view_tiles;
    if (layout == 1 && max_view_tiles * 6 > 200 * 1024) return CLS_ERR_INVALID_ARG;
    if (layout == 1 && subs >= INT32_MAX) return CLS_ERR_INVALID_ARG;  // int32 bucket ids
    if (max_view_tiles * 4 > 200 * 1024) return CLS_ERR_INVALID_ARG;  // nearest-active grid
    // shared-memory grids of the prefix sums (larger views use global memory)
    const int grid_cap = (int)hmin64(max_view_tiles * 4 + 16 * 1024, 200 * 1024);
    const int sms = per_device(g_proj_sms, [](int dev) {
        for (const void* k : {(const void*)emit_bucketed_kernel, (const void*)tile_mask_kernel,
                              (const void*)active_zmin_kernel})
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        return device_sms(dev);
    });
    const int64_t tchunks = (info->total_tiles + kTileChunk - 1) / kTileChunk;
    // bucketed layout, after the count: bucket offsets (clamped to the
    // capacity), the emission window tables and the emission
    auto emit_stage = [&]() {
        tile_offsets_kernel<<<(unsigned)tchunks, 256, 0, s>>>(
            views_dev, (int)V, active_tiles, n_active_tiles_dev, ttot, tile_partials, capacity,
            cursor, bin_offsets, ranges, rank0);
        // shared memory for the tables of views up to 2^8 tiles wide
        const int emit_smem =
            (int)hmin64(max_view_tiles * (4 + 2 * 7), 200 * 1024);
        bin_window_tables_kernel<<<V, 1024, 0, s>>>(views_dev, tile_rank, front, bin_cut, t_win,
                                                     info->total_tiles, emit_smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emit_bucketed_kernel,
                                                      kEmitThreads, (size_t)emit_smem);
        // one resident wave of persistent blocks; each picks a view when it
        // starts (in proportion to the views' work) and again when its view
        // has no work left
        const int resident = (int)hmin64((int64_t)sms * (per_sm > 0 ? per_sm : 1), 1 << 20);
        emit_bucketed_kernel<<<(unsigned)resident, kEmitThreads, (size_t)emit_smem, s>>>(
            views_dev, tile_rank, rank0, zmin, zmax, cursor, keys, capacity, work_list,
            work_count, work_count + V, bin_cut, front, t_win, info->total_tiles, emit_smem,
            (int)V, resident, work_count + 2 * V, status_dev);
    };
    if (project_mode == 2) {  // the previous call counted these pairs: emit them
        if (cpv > 0) {
            cudaMemsetAsync(work_count + V, 0, (size_t)V * 4 + 4, s);  // emission counters
            capacity_check_kernel<<<1, 32, 0, s>>>(n_pairs_dev, capacity, status_dev);
            emit_stage();
        }
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    if (layout == 1) {
        reset_bucketed_kernel<<<(unsigned)sms, 256, 0, s>>>(
            diff, info->total_sat, big_count, work_count, 2 * (int)V + 1, arange, (int)V,
            tile_partials, tchunks, ranges, info->total_tiles * 2);
    } else {
        cudaMemsetAsync(diff, 0, (size_t)info->total_sat * 4, s);
        cudaMemsetAsync(big_count, 0, 4, s);
    }
    if (project_mode == 0 && info->max_n > 0)
        project_kernel<0><<<dim3((info->max_n + kProjBlock - 1) / kProjBlock, V), kProjBlock, 0,
                             s>>>(scenes_dev, views_dev, records, rects, diff, nullptr, nullptr,
                                  nullptr, nullptr);
    // with the views' depth bins fixed (bucketed layout, mode 1) the projection
    // of the active records also makes their stamps in A
    const bool fused_stamps = layout == 1 && project_mode == 1;
    if (info->max_active > 0)  // active records, and their rectangles stamped into `diff`
        project_kernel<1><<<dim3((info->max_active + kProjBlock - 1) / kProjBlock, V), kProjBlock,
                             0, s>>>(scenes_dev, views_dev, records, rects, diff,
                                     fused_stamps ? zmin : nullptr, fused_stamps ? zmax : nullptr,
                                     fused_stamps ? abins : nullptr,
                                     fused_stamps ? arange : nullptr);
    tile_mask_kernel<<<V, 512, grid_cap, s>>>(views_dev, diff, tile_active, sat, tile_cache,
                                              grid_cap, tile_ring, layout == 0 ? 1 : 0);
    if (layout == 0 && info->max_active > 0)
        // one warp per active Gaussian; two 1024-thread blocks per SM
        active_zmin_kernel<<<dim3((unsigned)hmin64((info->max_active + kZminThreads / 32 - 1) /
                                                       (kZminThreads / 32),
                                                   (2 * sms + V - 1) / V), V),
                             kZminThreads, (size_t)max_view_tiles * 4, s>>>(
            scenes_dev, views_dev, records, tile_cache);
    {
        const int64_t chunks = (info->total_tiles + kCompactChunk - 1) / kCompactChunk;
        int64_t* cparts = reinterpret_cast<int64_t*>(ws + L.compact);
        compact_count_kernel<<<(unsigned)chunks, 1024, 0, s>>>(
            tile_active, info->total_tiles, tile_cache, prefix_mode, layout == 0 ? 1 : 0, cparts);
        scan_partials_kernel<<<1, 1024, 0, s>>>(cparts, chunks, nullptr, n_active_tiles_dev, -1,
                                                nullptr);
        compact_write_kernel<<<(unsigned)chunks, 1024, 0, s>>>(tile_active, info->total_tiles,
                                                               cparts, active_tiles, tile_rank);
    }
    if (cpv == 0) {
        cudaMemsetAsync(n_pairs_dev, 0, sizeof(int64_t), s);
        if (layout == 1) cudaMemsetAsync(ranges, 0, (size_t)info->total_tiles * 8, s);
        CLS_CHECK_LAUNCH();
        return CLS_OK;
    }
    const dim3 rec_grid((unsigned)cpv, V);
    if (layout == 1) {
        if (project_mode == 0) {  // the views' depth ranges, fixed until the next mode 0 call
            cudaMemsetAsync(zmin, 0xff, (size_t)V * 4, s);
            cudaMemsetAsync(zmax, 0, (size_t)V * 4, s);
        }
        // work_count, arange, tile_partials and ranges were reset above
    }
    const bool new_range = layout == 1 && project_mode == 0;
    count_pairs_kernel<<<rec_grid, kBinBlock, 0, s>>>(scenes_dev, views_dev, rects, sat,
                                                      (int)cpv, layout == 0 ? partials : nullptr,
                                                      new_range ? zmin : nullptr,
                                                      new_range ? zmax : nullptr,
                                                      layout == 1 ? work_list : nullptr,
                                                      work_count);
    if (layout == 0) {
        scan_partials_kernel<<<1, 1024, 0, s>>>(partials, cpv * V, n_pairs_dev, nullptr, capacity,
                                                status_dev);
        emit_pairs_kernel<<<rec_grid, kBinBlock, 0, s>>>(scenes_dev, views_dev, rects, sat,
                                                          tile_active, (int)cpv, partials, keys,
                                                          vals, capacity, big_list, big_count);
        emit_big_kernel<<<1024, 256, 0, s>>>(views_dev, rects, tile_active, keys, vals,
                                             capacity, big_list, big_count);
    } else {
        // grids of kDepthBins threads stride over the views' rows and columns
        constexpr unsigned kLines = 128;
        if (project_mode == 0) {  // the static Gaussians' pairs per (tile, bin)
            cudaMemsetAsync(sbins, 0, (size_t)kDepthBins * info->total_sat * 4, s);
            stamp_static_kernel<<<dim3((unsigned)hmin64((info->max_n + kBinBlock - 1) / kBinBlock,
                                                        2048), V), kBinBlock, 0, s>>>(
                scenes_dev, views_dev, rects, zmin, zmax, sbins);
            row_prefix_kernel<<<dim3(kLines, V), kDepthBins, 0, s>>>(views_dev, sbins, nullptr, 0);
            col_prefix_kernel<<<dim3(kLines, V), kDepthBins, 0, s>>>(views_dev, sbins);
        }
        if (info->max_active > 0) {  // the active Gaussians' stamps, prefix-summed along x
            if (!fused_stamps)
                stamp_active_kernel<<<dim3((unsigned)hmin64(
                                           (info->max_active + kBinBlock - 1) / kBinBlock, 2048),
                                       V), kBinBlock, 0, s>>>(scenes_dev, views_dev, rects, zmin,
                                                              zmax, abins, arange);
            row_prefix_kernel<<<dim3(kLines, V), kDepthBins, 0, s>>>(views_dev, abins, arange, 1);
        }
        // per (rank, bin) counts go to `cursor`, which tile_offsets_kernel
        // turns into the buckets' slot cursors
        col_counts_kernel<<<dim3(kLines, V), kDepthBins, 0, s>>>(
            views_dev, sbins, abins, arange, zmin, zmax, tile_rank, tile_cache, prefix_mode,
            cursor, front, bin_cut, ttot, tile_partials);
        scan_partials_kernel<<<1, 1024, 0, s>>>(tile_partials, tchunks, n_pairs_dev, nullptr,
                                                capacity, status_dev);
        // counting only (capacity planning): the per-bucket counts stay in
        // `cursor` for a following call in project_mode 2
        if (keys == nullptr || capacity == 0) {
            CLS_CHECK_LAUNCH();
            return CLS_OK;
        }
        emit_stage();
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}

extern "C" int cls_complete_truncated(const ClsView* views_dev, const ClsBatchInfo* info,
                                      const ClsProjected* records, uint64_t* keys,
                                      int64_t capacity, const int32_t* trunc,
                                      const int32_t* trunc_count, int64_t trunc_cap,
                                      int32_t* work_counter, void* workspace,
                                      size_t workspace_bytes, cls_stream_t stream) {
    if (!views_dev || !info || !records || !keys || !trunc || !trunc_count || !work_counter ||
        !workspace || workspace_bytes < cls_project_workspace_size(info) || trunc_cap <= 0)
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const ProjLayout L = proj_layout(info);
    char* ws = static_cast<char*>(workspace);
    cudaMemsetAsync(work_counter, 0, sizeof(int32_t), s);
    complete_tiles_kernel<<<1024, 256, 0, s>>>(
        views_dev, info->n_views, reinterpret_cast<uint32_t*>(ws + L.zmin),
        reinterpret_cast<uint32_t*>(ws + L.zmax), reinterpret_cast<int32_t*>(ws + L.cursor), keys,
        capacity, reinterpret_cast<const uint4*>(ws + L.work_list),
        reinterpret_cast<int32_t*>(ws + L.work_count), trunc, trunc_count, trunc_cap,
        reinterpret_cast<uint8_t*>(ws + L.front), work_counter);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
