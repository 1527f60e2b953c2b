// Forward rendering of the active tiles (Supp. "Local Optimization Kernel",
// item 2): a 128-thread block per 16x16 tile, two pixels per thread, the
// tile's depth-sorted list staged through shared memory in batches of 256
// records; blocks are persistent and take tiles from a queue. The photometric
// loss and its pixel gradient are fused into the epilogue.
//
// Static prefix: static Gaussians are frozen during an update, so the state of
// a pixel after the static entries in front of every active Gaussian of its
// tile repeats from one iteration to the next. A tile whose cache holds starts
// from that state at list position n_prefix; a tile to rebuild composites from
// the front and writes the state when it reaches the first entry at or behind
// the boundary depth. The same floating-point operations run on the same
// entries in the same order either way, so both give identical results.
#include "common.cuh"

namespace cls {

constexpr int kFwdThreads = kTilePixels / 2;  // two pixels per thread: rows 2 ly and 2 ly + 1
constexpr int kLazyWin = kTilePixels;  // keys per rank-sorted window
constexpr int kLazyMax = 1024;         // largest bin the renderer sorts itself
constexpr int kBins = CLS_DEPTH_BINS;

constexpr int kFwdWarps = kFwdThreads / 32;

struct FwdSmem {
    float4 a[kTilePixels];
    float4 b[kTilePixels];
    float c[kTilePixels];
    uint32_t pos[kTilePixels];  // list position of each staged entry
    uint64_t key[kLazyMax];
    uint64_t sorted[kLazyMax];
    uint32_t off[kBins + 1];
    float red[kFwdWarps];
    // per staging round and warp: entries kept, kept in front of the prefix
    // boundary, in front of the boundary
    int cnt[3][2][kFwdWarps];
    int tile;
    int last_bin;
    int first_bin;
    int last_active;  // last list position of a staged active entry
};

// Per-thread compositing state of one pixel.
struct PixelState {
    float T, c0, c1, c2;
    uint32_t last;
    bool done;
};

// Tile-uniform state of the static prefix while a tile is rendered.
struct PrefixWalk {
    uint32_t zb;        // boundary depth bits
    uint32_t skip_to;   // first list position to composite (cached prefix)
    bool rebuild;       // the state after the prefix is written this pass
    bool crossed;       // ... and has been
    uint32_t n_prefix;  // entries in front of the boundary (rebuild)
};

// Counts of one staged batch (uniform over the block).
struct Staged {
    int n;             // entries kept
    int n_below_kept;  // kept entries in front of the prefix boundary (a prefix of them)
    int n_below_all;   // batch entries in front of the boundary
};

// Stage batch entries i = 0 .. nb-1 (record rec_of(i), list position pos0 + i)
// into shared memory in list order, keeping those at or behind skip_to that
// tile_culled does not drop; counts the entries in front of the prefix
// boundary while a rebuild has not crossed it. Two entries per thread; an
// order-preserving compaction by ballots and per-warp counts.
template <typename RecOf>
__device__ __forceinline__ Staged stage_batch(FwdSmem& sm, int nb, uint32_t pos0, RecOf rec_of,
                                              const ClsProjected* records, uint32_t n_records,
                                              float tx0, float ty0, const PrefixWalk& pw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool count = pw.rebuild && !pw.crossed;
    uint32_t rec[2];
    unsigned mk[2];
    // pass 1: which entries stay (the records are read again in pass 2, from cache)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r * kFwdThreads + threadIdx.x;
        bool keep = false, below = false;
        rec[r] = 0;
        if (i < nb) rec[r] = rec_of(i);
        // guard (never taken): an index past the records is dropped unread
        if (i < nb && rec[r] < n_records) {
            const float4* p = reinterpret_cast<const float4*>(records + rec[r]);
            below = count && __float_as_uint(p[2].z) < pw.zb;
            keep = pos0 + (uint32_t)i >= pw.skip_to && !tile_culled(p[0], p[1], tx0, ty0);
        }
        mk[r] = __ballot_sync(0xffffffffu, keep);
        const unsigned mkb = __ballot_sync(0xffffffffu, keep && below);
        const unsigned mb = __ballot_sync(0xffffffffu, below);
        if (lane == 0) {
            sm.cnt[0][r][warp] = __popc(mk[r]);
            sm.cnt[1][r][warp] = __popc(mkb);
            sm.cnt[2][r][warp] = __popc(mb);
        }
    }
    __syncthreads();
    Staged st{0, 0, 0};
    int base[2] = {0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int w = 0; w < kFwdWarps; ++w) {
            if (w == warp) base[r] = st.n;
            st.n += sm.cnt[0][r][w];
            st.n_below_kept += sm.cnt[1][r][w];
            st.n_below_all += sm.cnt[2][r][w];
        }
    }
    // pass 2: the kept entries, compacted in list order
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (mk[r] & (1u << lane)) {
            const int k = base[r] + __popc(mk[r] & lt);
            const uint32_t pos = pos0 + (uint32_t)(r * kFwdThreads + threadIdx.x);
            const float4* p = reinterpret_cast<const float4*>(records + rec[r]);
            const float4 r2 = p[2];
            sm.a[k] = stage_conic_a(p[0]);
            sm.b[k] = stage_conic_b(p[1]);
            sm.c[k] = r2.x;
            sm.pos[k] = pos;
            if (__float_as_int(r2.y) >= 0) atomicMax(&sm.last_active, (int)pos);
        }
    }
    return st;
}

// One list entry at one pixel, without branches: every quantity is computed
// and the skip (power > 0, alpha < 1/255), stop (T (1 - alpha) < 1e-4) and done
// decisions select what is kept, so the two pixels of a thread form
// independent straight-line chains the compiler can interleave. A skipped or
// stopped entry adds exactly zero to the colour and leaves T and the last
// contributor as they were, so the result is the same as with branches.
__device__ __forceinline__ void composite_one(float P, float Q, float dy, const float4& bb,
                                              float cb, int k, PixelState& ps, int& lastk) {
    const float power2 = pair_power2(P, Q, dy, bb.x);  // with log2 o (bb.y) folded in
    const float alpha = fminf(kAlphaMax, ex2_approx(power2));
    const float wa = alpha * ps.T;       // the entry's weight if composited
    const float test_T = ps.T - wa;      // T (1 - alpha)
    const bool live = !ps.done && power2 <= bb.y && alpha >= kAlphaMin;
    const bool stop = live && test_T < kTMin;
    const bool take = live && !stop;
    const float w = take ? wa : 0.0f;
    ps.c0 = __fmaf_rn(bb.z, w, ps.c0);
    ps.c1 = __fmaf_rn(bb.w, w, ps.c1);
    ps.c2 = __fmaf_rn(cb, w, ps.c2);
    ps.T -= w;
    lastk = take ? k : lastk;
    ps.done = ps.done || stop;
}

// Composite staged records k0 .. k1 - 1 into two pixels of one column. The
// last contributor is tracked as a staged index and turned into its list
// position once at the end (one shared load per pixel instead of one per
// entry).
__device__ __forceinline__ void composite_batch(const FwdSmem& sm, int k0, int k1, float fx,
                                                float fy0, float fy1, PixelState& p0,
                                                PixelState& p1) {
    int l0 = -1, l1 = -1;
    auto entry = [&](int k) {
        const float4 a = sm.a[k];
        const float4 bb = sm.b[k];
        const float cb = sm.c[k];
        float P, Q;
        pair_column(fx - a.x, a.z, a.w, bb.y, P, Q);
        composite_one(P, Q, fy0 - a.y, bb, cb, k, p0, l0);
        composite_one(P, Q, fy1 - a.y, bb, cb, k, p1, l1);
    };
    // four entries per step (a pixel that stops at one of them leaves the
    // rest unchanged: a done pixel takes nothing)
    int k = k0;
    for (; k + 3 < k1 && !(p0.done && p1.done); k += 4) {
        entry(k);
        entry(k + 1);
        entry(k + 2);
        entry(k + 3);
    }
    for (; k < k1 && !(p0.done && p1.done); ++k) entry(k);
    if (l0 >= 0) p0.last = sm.pos[l0] + 1;
    if (l1 >= 0) p1.last = sm.pos[l1] + 1;
}

__device__ __forceinline__ void save_prefix(const PixelState& ps, const ClsView& view, int px,
                                            int py, float* prefix_state, int32_t* prefix_last) {
    if (!(px < view.cam.width && py < view.cam.height)) return;
    const int64_t pix = view.pix_base + (int64_t)py * view.cam.width + px;
    reinterpret_cast<float4*>(prefix_state)[pix] =
        make_float4(ps.done ? -ps.T : ps.T, ps.c0, ps.c1, ps.c2);
    prefix_last[pix] = (int32_t)ps.last;
}

__device__ __forceinline__ void load_prefix(PixelState& ps, const ClsView& view, int px, int py,
                                            const float* prefix_state,
                                            const int32_t* prefix_last) {
    if (ps.done) return;  // outside the image
    const int64_t pix = view.pix_base + (int64_t)py * view.cam.width + px;
    const float4 st = reinterpret_cast<const float4*>(prefix_state)[pix];
    ps.T = fabsf(st.x);
    ps.done = st.x < 0.0f;
    ps.c0 = st.y; ps.c1 = st.z; ps.c2 = st.w;
    ps.last = (uint32_t)prefix_last[pix];
}

// Composite one staged batch (nb list entries from position pos0, `st` as
// staged); when rebuilding, save the pixel state at the first entry at or
// behind the boundary. Uniform over the block.
__device__ __forceinline__ void composite_staged(const FwdSmem& sm, const Staged& st, int nb,
                                                 uint32_t pos0, PrefixWalk& pw,
                                                 const ClsView& view, int px, int py0, int py1,
                                                 float fx, float fy0, float fy1, PixelState& p0,
                                                 PixelState& p1, float* prefix_state,
                                                 int32_t* prefix_last) {
    if (pw.rebuild && !pw.crossed && st.n_below_all < nb) {
        composite_batch(sm, 0, st.n_below_kept, fx, fy0, fy1, p0, p1);
        save_prefix(p0, view, px, py0, prefix_state, prefix_last);
        save_prefix(p1, view, px, py1, prefix_state, prefix_last);
        pw.crossed = true;
        pw.n_prefix = pos0 + (uint32_t)st.n_below_all;
        composite_batch(sm, st.n_below_kept, st.n, fx, fy0, fy1, p0, p1);
        return;
    }
    composite_batch(sm, 0, st.n, fx, fy0, fy1, p0, p1);
}
__device__ __forceinline__ void finish_pixel(const PixelState& ps, const ClsView& view, int px,
                                             int py, float bg0, float bg1, float bg2,
                                             const float* target, int loss_mode, float* image,
                                             float* T_final, int32_t* n_contrib, float* dL_dimage,
                                             float& lsum) {
    const int W = view.cam.width, H = view.cam.height;
    if (!(px < W && py < H)) return;
    const float c0 = ps.c0 + ps.T * bg0, c1 = ps.c1 + ps.T * bg1, c2 = ps.c2 + ps.T * bg2;
    const int64_t pix = view.pix_base + (int64_t)py * W + px;
    const int64_t plane = (int64_t)W * H;
    const int64_t p3 = 3 * view.pix_base + (int64_t)py * W + px;
    T_final[pix] = ps.T;
    n_contrib[pix] = (int32_t)ps.last;
    if (image) {
        image[p3] = c0;
        image[p3 + plane] = c1;
        image[p3 + 2 * plane] = c2;
    }
    if (loss_mode != 0) {
        const float d0 = c0 - target[p3], d1 = c1 - target[p3 + plane],
                    d2 = c2 - target[p3 + 2 * plane];
        const float sc = view.loss_scale;
        float g0, g1, g2, l;
        if (loss_mode == 1) {
            g0 = (d0 > 0.f) - (d0 < 0.f);
            g1 = (d1 > 0.f) - (d1 < 0.f);
            g2 = (d2 > 0.f) - (d2 < 0.f);
            l = fabsf(d0) + fabsf(d1) + fabsf(d2);
        } else {
            g0 = 2.f * d0; g1 = 2.f * d1; g2 = 2.f * d2;
            l = d0 * d0 + d1 * d1 + d2 * d2;
        }
        dL_dimage[p3] = g0 * sc;
        dL_dimage[p3 + plane] = g1 * sc;
        dL_dimage[p3 + 2 * plane] = g2 * sc;
        lsum += l * sc;
    }
}

__global__ void __launch_bounds__(kFwdThreads, 8)
render_fwd_kernel(const ClsView* __restrict__ views, int n_views,
                  const ClsProjected* __restrict__ records, uint32_t n_records,
                  const uint32_t* __restrict__ vals,
                  int vals_stride, const uint32_t* __restrict__ ranges,
                  const int32_t* __restrict__ active_tiles,
                  const int32_t* __restrict__ n_active_tiles, uint64_t* __restrict__ lazy_keys,
                  const uint32_t* __restrict__ bin_offsets, const int32_t* __restrict__ list_ranks,
                  const uint8_t* __restrict__ cut_in, uint8_t* __restrict__ cut_out,
                  int32_t* __restrict__ trunc, int32_t* __restrict__ trunc_count,
                  int64_t trunc_cap, ClsTileCache* __restrict__ tile_cache,
                  float* __restrict__ prefix_state, int32_t* __restrict__ prefix_last, float bg0,
                  float bg1, float bg2, const float* __restrict__ target, int loss_mode,
                  float* __restrict__ image, float* __restrict__ T_final,
                  int32_t* __restrict__ n_contrib, float* __restrict__ dL_dimage,
                  float* __restrict__ loss_per_scene, int* __restrict__ work_counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem& sm = *reinterpret_cast<FwdSmem*>(smem_raw);
    const int n_tiles = *n_active_tiles;
    if (n_tiles <= 0) return;  // an empty list (the usual rerun): no queue traffic
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;  // ly in [0, 8)
    const bool lazy = bin_offsets != nullptr;
    for (;;) {
        if (threadIdx.x == 0) {
            sm.tile = atomicAdd(work_counter, 1);
            sm.last_active = -1;
        }
        __syncthreads();
        const int t = sm.tile;
        if (t >= n_tiles) break;
        const int tile = active_tiles[t];
        const int vi = view_of_tile(views, n_views, tile);
        const ClsView& view = views[vi];
        const int local = tile - view.tile_base;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const int W = view.cam.width, H = view.cam.height;
        // a warp covers a 16 x 4 strip of the tile (its pixels saturate at
        // similar depths, so the warp leaves the list walk sooner)
        const int px = tx * kTile + lx, py0 = ty * kTile + 2 * ly, py1 = py0 + 1;
        const float fx = (float)px + 0.5f, fy0 = (float)py0 + 0.5f, fy1 = (float)py1 + 0.5f;
        const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
        const uint32_t start = ranges[2 * (int64_t)tile], end = ranges[2 * (int64_t)tile + 1];

        PixelState p0{1.0f, 0.f, 0.f, 0.f, 0u, !(px < W && py0 < H)};
        PixelState p1{1.0f, 0.f, 0.f, 0.f, 0u, !(px < W && py1 < H)};
        PrefixWalk pw;
        {
            const ClsTileCache c = tile_cache[tile];
            pw.zb = c.zb;
            pw.rebuild = c.n_prefix == CLS_PREFIX_UNKNOWN;
            pw.crossed = false;
            pw.skip_to = pw.rebuild ? 0u : c.n_prefix;
            pw.n_prefix = 0u;
        }
        if (!pw.rebuild) {
            load_prefix(p0, view, px, py0, prefix_state, prefix_last);
            load_prefix(p1, view, px, py1, prefix_state, prefix_last);
        }
        bool truncated = false;
        if (!lazy) {
            for (uint32_t b = start + min(pw.skip_to, end - start); b < end; b += kTilePixels) {
                if (__syncthreads_count(p0.done && p1.done) == kFwdThreads) break;
                const int nb = (int)min((uint32_t)kTilePixels, end - b);
                const Staged st = stage_batch(
                    sm, nb, b - start,
                    [&](int i) { return vals[(int64_t)(b + i) * vals_stride]; }, records,
                    n_records, tx0, ty0, pw);
                __syncthreads();
                composite_staged(sm, st, nb, b - start, pw, view, px, py0, py1, fx, fy0, fy1, p0,
                                 p1, prefix_state, prefix_last);
                __syncthreads();
            }
        } else {
            // Walk the tile's depth bins front to back. Consecutive bins up to
            // kLazyWin keys (or one bin up to kLazyMax) are sorted here by rank
            // counting on the unique (depth, index) keys, written back for the
            // backward pass, and composited; bins behind the point where every
            // pixel saturated are never sorted. Larger bins were sorted before.
            // Only bins up to cut_in[tile] were emitted; if the tile needs more,
            // it is queued for completion and its outputs are left to the rerun.
            // A cached prefix starts the walk at the bin holding its end.
            const int rank = list_ranks ? list_ranks[t] : t;
            const int limit = cut_in ? (int)cut_in[tile] : kBins - 1;
            for (int i = threadIdx.x; i <= kBins; i += kFwdThreads)
                sm.off[i] = bin_offsets[(int64_t)rank * kBins + i];
            __syncthreads();
            if (threadIdx.x == 0) {
                sm.last_bin = -1;
                int lo = 0;  // last bin starting at or before skip_to
                if (!pw.rebuild) {
                    int hi = kBins - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sm.off[mid] - sm.off[0] <= pw.skip_to) lo = mid; else hi = mid - 1;
                    }
                }
                sm.first_bin = lo;
            }
            __syncthreads();
            int bin = sm.first_bin;
            while (bin <= limit) {
                if (__syncthreads_count(p0.done && p1.done) == kFwdThreads) break;
                const uint32_t w0 = sm.off[bin];
                const int b0 = bin;
                // the window: bins b0 .. e - 1, e the first bin past the cut or
                // whose inclusion would take the window above kLazyWin keys
                // (at least one bin); a binary search over the monotone offsets
                int e = bin + 1, e_hi = limit + 1;
                while (e < e_hi) {
                    const int mid = (e + e_hi) >> 1;
                    if (sm.off[mid + 1] - w0 > (uint32_t)kLazyWin) e_hi = mid; else e = mid + 1;
                }
                const int n = (int)(sm.off[e] - w0);
                bin = e;
                if (n == 0) continue;
                if (threadIdx.x == 0) sm.last_bin = e - 1;
                const bool here = n <= kLazyMax;
                if (here) {
                    for (int i = threadIdx.x; i < n; i += kFwdThreads) sm.key[i] = lazy_keys[w0 + i];
                    __syncthreads();
                    // the bins are already in depth order: rank each key inside its own bin
                    for (int i = threadIdx.x; i < n; i += kFwdThreads) {
                        const uint32_t p = w0 + (uint32_t)i;
                        int lo = b0, hi = e - 1;  // last bin starting at or before p (non-empty)
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (sm.off[mid] <= p) lo = mid; else hi = mid - 1;
                        }
                        const int s0 = (int)(sm.off[lo] - w0), s1 = (int)(sm.off[lo + 1] - w0);
                        const uint64_t k = sm.key[i];
                        int r = s0;
                        for (int j = s0; j < s1; ++j) r += sm.key[j] < k;
                        sm.sorted[r] = k;
                    }
                    __syncthreads();
                    for (int i = threadIdx.x; i < n; i += kFwdThreads) lazy_keys[w0 + i] = sm.sorted[i];
                }
                for (int c0 = 0; c0 < n; c0 += kTilePixels) {
                    const uint32_t pos0 = w0 - start + c0;
                    const int nb = min(kTilePixels, n - c0);
                    if (pos0 + nb <= pw.skip_to) continue;  // inside the cached prefix
                    if (c0 > 0 && __syncthreads_count(p0.done && p1.done) == kFwdThreads) break;
                    const Staged st = stage_batch(
                        sm, nb, pos0,
                        [&](int i) {
                            return (uint32_t)(here ? sm.sorted[c0 + i] : lazy_keys[w0 + c0 + i]);
                        },
                        records, n_records, tx0, ty0, pw);
                    __syncthreads();
                    composite_staged(sm, st, nb, pos0, pw, view, px, py0, py1, fx, fy0, fy1, p0,
                                     p1, prefix_state, prefix_last);
                    __syncthreads();
                }
            }
            const bool all_done = __syncthreads_count(p0.done && p1.done) == kFwdThreads;
            // entries the tile may still need: behind the cut and behind the cached prefix
            const uint32_t needed_from = max(sm.off[limit + 1], start + pw.skip_to);
            truncated = !all_done && limit < kBins - 1 && needed_from < sm.off[kBins];
            if (threadIdx.x == 0) {
                if (truncated) {
                    const int slot = atomicAdd(trunc_count, 1);
                    if (slot < trunc_cap) {
                        trunc[slot] = tile;
                        trunc[trunc_cap + slot] = rank;
                        trunc[2 * trunc_cap + slot] = limit;
                    }
                } else if (cut_out) {
                    cut_out[tile] =
                        sm.last_bin < 0 ? (uint8_t)0
                                        : (uint8_t)min(kBins - 1, sm.last_bin + kCutMargin);
                }
            }
        }
        if (truncated) {  // uniform over the block; the completion rerun writes this tile
            __syncthreads();
            continue;
        }
        if (pw.rebuild) {
            if (!pw.crossed) {  // every pixel stopped (or the list ended) in front of it
                save_prefix(p0, view, px, py0, prefix_state, prefix_last);
                save_prefix(p1, view, px, py1, prefix_state, prefix_last);
                pw.n_prefix = end - start;
            }
            if (threadIdx.x == 0) tile_cache[tile].n_prefix = pw.n_prefix;
        }
        if (threadIdx.x == 0) tile_cache[tile].last_active = sm.last_active;

        float lsum = 0.0f;
        finish_pixel(p0, view, px, py0, bg0, bg1, bg2, target, loss_mode, image, T_final,
                     n_contrib, dL_dimage, lsum);
        finish_pixel(p1, view, px, py1, bg0, bg1, bg2, target, loss_mode, image, T_final,
                     n_contrib, dL_dimage, lsum);
        if (loss_mode != 0 && loss_per_scene) {
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = lsum;
            __syncthreads();
            if (threadIdx.x == 0) {
                float tot = 0.f;
                for (int w = 0; w < kFwdThreads / 32; ++w) tot += sm.red[w];
                atomicAdd(loss_per_scene + view.scene, tot);
            }
        }
        __syncthreads();
    }
}

static PerDevice g_fwd_blocks;

}  // namespace cls

using namespace cls;

extern "C" int cls_render_forward(const ClsView* views_dev, const ClsBatchInfo* info,
                                  const ClsProjected* records, const uint32_t* vals,
                                  int32_t vals_stride, const uint32_t* ranges, const int32_t* active_tiles,
                                  const int32_t* n_active_tiles_dev, uint64_t* lazy_keys,
                                  const uint32_t* bin_offsets, const int32_t* list_ranks,
                                  const uint8_t* cut_in, uint8_t* cut_out, int32_t* trunc,
                                  int32_t* trunc_count, int64_t trunc_cap,
                                  ClsTileCache* tile_cache, float* prefix_state,
                                  int32_t* prefix_last, const float* bg,
                                  const float* target, int32_t loss_mode, float* image,
                                  float* T_final, int32_t* n_contrib, float* dL_dimage,
                                  float* loss_per_scene, int32_t* work_counter,
                                  cls_stream_t stream) {
    if (!views_dev || !info || !records ||
        (bin_offsets ? !lazy_keys : (!vals || (vals_stride != 1 && vals_stride != 2))) ||
        (cut_in && (!bin_offsets || !trunc || !trunc_count || trunc_cap < info->total_tiles)) ||
        !ranges || !active_tiles || !n_active_tiles_dev || !tile_cache || !prefix_state ||
        !prefix_last || !image ||
        !bg || !T_final || !n_contrib || !work_counter || loss_mode < 0 || loss_mode > 2 ||
        (loss_mode != 0 && (!target || !dL_dimage)) || info->n_views <= 0 ||
        info->total_tiles <= 0)
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int fwd_blocks = per_device(g_fwd_blocks, [](int dev) {
        cudaFuncSetAttribute(render_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(FwdSmem));
        return resident_blocks(dev, render_fwd_kernel, kFwdThreads, sizeof(FwdSmem));
    });
    const int blocks = (int)hmin64(info->total_tiles, fwd_blocks);
    cudaMemsetAsync(work_counter, 0, sizeof(int32_t), s);
    render_fwd_kernel<<<blocks, kFwdThreads, sizeof(FwdSmem), s>>>(
        views_dev, info->n_views, records, (uint32_t)hmin64(info->total_records, 0xffffffffll),
        vals, vals_stride, ranges, active_tiles, n_active_tiles_dev, lazy_keys, bin_offsets,
        list_ranks, cut_in, cut_out, trunc, trunc_count, trunc_cap, tile_cache, prefix_state,
        prefix_last, bg[0], bg[1], bg[2], target, loss_mode, image, T_final, n_contrib, dL_dimage,
        loss_per_scene, work_counter);
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
