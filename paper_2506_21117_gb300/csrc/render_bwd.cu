// Backward pass of the local optimisation (Supp. "Local Optimization Kernel",
// items 2 and 3).
//
// Pixel part: one 64-thread block per active tile (persistent, queue of
// tiles), four pixels of one column per thread. Each pixel starts from the state the forward
// pass kept after the tile's static prefix (nothing in front of it depends on
// an active Gaussian) and walks its list front to back, up to the earlier of
// its last contributor and the tile's last active entry (nothing behind both
// reaches an active gradient). T in front of each Gaussian is recomputed with
// the forward pass's own operations; the colour behind a Gaussian is the final
// colour minus what has been composited up to and including it, so nothing
// per (pixel, Gaussian) is stored. Static Gaussians update T and that colour
// but skip all gradient work. The 2D gradients of an active Gaussian are
// reduced over the tile with warp shuffles and a shared-memory sum over warps,
// then added to global memory with one atomic per component per tile.
//
// Gaussian part: one thread per active Gaussian; the chain rule from the 2D
// gradients of every view of its scene to every float of its parameter row.
#include "common.cuh"

namespace cls {

constexpr int kSub = 32;      // list entries reduced per shared-memory flush
constexpr int kGradComps = 9; // du dv dA dB dC dopacity dr dg db
constexpr int kG2Stride = 12;
constexpr int kPPT = 4;  // pixels per thread: one column, rows ly, ly + 4, ly + 8, ly + 12
constexpr int kRowStep = kTile / kPPT;
constexpr int kBwdThreads = kTilePixels / kPPT;
constexpr int kBwdWarps = kBwdThreads / 32;
constexpr int kStage = kTilePixels / kBwdThreads;  // list entries staged per thread

// Walk state of one pixel: T in front of the next entry, R = colour not yet
// composited (final colour minus everything in front, background included).
struct BwdPixel {
    float fx, fy;
    float T, g0, g1, g2, R0, R1, R2;
    int end;  // list positions before `end` are walked
};

// One list entry at one pixel: the forward pass's alpha and T, the colour
// behind, and (for an active Gaussian) the entry's colour gradient added to
// gr[6..8] and dL/dpower (0 unless the entry contributes with alpha below the
// clamp) returned in `dpow` with the pixel's dy; the caller turns those into
// the per-thread sums of the centre, conic and opacity gradients.
// a = (u, v, a2, b2), bb = (c2, log2 opacity, r, g) as staged (base-2 conic,
// the opacity folded into the exponent).
// Written without branches: the walk-end and skip decisions select what is
// kept (a skipped entry has weight exactly zero and leaves T as it was), so
// the pixels of a thread form independent straight-line chains.
template <bool ACTIVE>
__device__ __forceinline__ bool bwd_entry(BwdPixel& p, int pos, float P, float Q,
                                          const float4& a, const float4& bb, float cb, float* gr,
                                          float& dpow, float& dy) {
    dy = p.fy - a.y;
    const float power2 = pair_power2(P, Q, dy, bb.x);
    const float G = ex2_approx(power2);  // opacity times the Gaussian
    const float alpha = fminf(kAlphaMax, G);
    const bool live = pos < p.end && power2 <= bb.y && alpha >= kAlphaMin;
    const float w = live ? alpha * p.T : 0.0f;
    p.R0 = __fmaf_rn(-bb.z, w, p.R0);
    p.R1 = __fmaf_rn(-bb.w, w, p.R1);
    p.R2 = __fmaf_rn(-cb, w, p.R2);
    if (ACTIVE) {
        const float inv_om = __fdividef(1.0f, 1.0f - alpha);
        const float cg = bb.z * p.g0 + bb.w * p.g1 + cb * p.g2;
        const float gR = p.g0 * p.R0 + p.g1 * p.R1 + p.g2 * p.R2;
        const float dLda = p.T * cg - gR * inv_om;
        dpow = (live && !(G > kAlphaMax)) ? dLda * alpha : 0.f;
        gr[6] += w * p.g0;
        gr[7] += w * p.g1;
        gr[8] += w * p.g2;
    }
    p.T -= w;  // T (1 - alpha) as the forward pass forms it: T - alpha T
    return live;
}

// Warp reduce-scatter of eight values: after it, lane L holds the warp sum of
// value (L >> 2) & 7 (butterfly halving: 4 + 2 + 1 exchanges, then two more to
// finish the sum), 9 shuffles instead of 40.
__device__ __forceinline__ float reduce8_scatter(const float* v, int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4];
        const float keep = b4 ? v[i + 4] : v[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? w[i] : w[i + 2];
        const float keep = b3 ? w[i + 2] : w[i];
        x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    return y;
}

// Pixel start state: after the tile's prefix (n_prefix entries), walking to
// min(n_contrib, last active + 1). A pixel that stopped inside the prefix, or
// lies outside the image, walks nothing.
__device__ __forceinline__ void bwd_load_pixel(BwdPixel& p, const ClsView& view, int px, int py,
                                               int n_prefix, int end_active,
                                               const float* prefix_state, const float* image,
                                               const int32_t* n_contrib,
                                               const float* dL_dimage) {
    const int W = view.cam.width, H = view.cam.height;
    p.fx = (float)px + 0.5f;
    p.fy = (float)py + 0.5f;
    p.T = 1.0f; p.g0 = p.g1 = p.g2 = 0.f; p.R0 = p.R1 = p.R2 = 0.f;
    p.end = 0;
    if (!(px < W && py < H)) return;
    const int64_t pix = view.pix_base + (int64_t)py * W + px;
    const float4 st = reinterpret_cast<const float4*>(prefix_state)[pix];
    if (st.x < 0.0f) return;
    const int end = min(n_contrib[pix], end_active);
    if (end <= n_prefix) return;
    const int64_t plane = (int64_t)W * H;
    const int64_t p3 = 3 * view.pix_base + (int64_t)py * W + px;
    p.end = end;
    p.T = st.x;
    p.g0 = dL_dimage[p3];
    p.g1 = dL_dimage[p3 + plane];
    p.g2 = dL_dimage[p3 + 2 * plane];
    p.R0 = image[p3] - st.y;
    p.R1 = image[p3 + plane] - st.z;
    p.R2 = image[p3 + 2 * plane] - st.w;
}

__global__ void __launch_bounds__(kBwdThreads, 14)
render_bwd_kernel(const ClsView* __restrict__ views, int n_views,
                  const ClsProjected* __restrict__ records, uint32_t n_records,
                  const uint32_t* __restrict__ vals,
                  int vals_stride, const uint32_t* __restrict__ ranges,
                  const int32_t* __restrict__ active_tiles,
                  const int32_t* __restrict__ n_active_tiles,
                  const ClsTileCache* __restrict__ tile_cache,
                  const float* __restrict__ prefix_state, const float* __restrict__ image,
                  const int32_t* __restrict__ n_contrib, const float* __restrict__ dL_dimage,
                  float* __restrict__ grad2d, int* __restrict__ work_counter) {
    __shared__ float4 s_a[kTilePixels];
    __shared__ float4 s_b[kTilePixels];
    // per staged entry: the bits of its blue colour, its active slot (-1 for a
    // static Gaussian) and its list position, read with one shared load
    __shared__ int4 s_e[kTilePixels];
    __shared__ float s_g[kSub][kBwdWarps][kGradComps + 1];
    __shared__ int s_cnt[kStage][kBwdWarps];
    __shared__ int s_tile;
    __shared__ int s_maxend;
    const int n_tiles = *n_active_tiles;
    if (n_tiles <= 0) return;  // nothing rendered: no queue traffic
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;  // ly in [0, kRowStep)
    for (;;) {
        if (threadIdx.x == 0) {
            s_tile = atomicAdd(work_counter, 1);
            s_maxend = 0;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= n_tiles) break;
        const int tile = active_tiles[t];
        const ClsTileCache c = tile_cache[tile];
        const int n_prefix = (int)c.n_prefix;
        // no active entry behind the prefix: no gradient (an unrendered tile
        // has no prefix and is skipped too)
        if (c.n_prefix == CLS_PREFIX_UNKNOWN || c.last_active < n_prefix) {
            __syncthreads();
            continue;
        }
        const ClsView& view = views[view_of_tile(views, n_views, tile)];
        const int local = tile - view.tile_base;
        const int tx = local % view.tiles_x, ty = local / view.tiles_x;
        const uint32_t start = ranges[2 * (int64_t)tile];
        const float tx0 = (float)(tx * kTile), ty0 = (float)(ty * kTile);
        BwdPixel p[kPPT];
        int my_end = 0;
#pragma unroll
        for (int j = 0; j < kPPT; ++j) {
            bwd_load_pixel(p[j], view, tx * kTile + lx, ty * kTile + ly + j * kRowStep, n_prefix,
                           c.last_active + 1, prefix_state, image, n_contrib, dL_dimage);
            my_end = max(my_end, p[j].end);
        }
        if (my_end > n_prefix) atomicMax(&s_maxend, my_end);
        __syncthreads();
        const int max_end = s_maxend;

        for (int lo = n_prefix; lo < max_end; lo += kTilePixels) {
            const int nb = min(kTilePixels, max_end - lo);
            // stage the batch, dropping entries the forward pass's tile cull
            // drops (no pixel of the tile reaches alpha >= 1/255), in order
            uint32_t rec[kStage];
            unsigned mk[kStage];
#pragma unroll
            for (int r = 0; r < kStage; ++r) {
                const int i = r * kBwdThreads + threadIdx.x;
                bool keep = false;
                rec[r] = 0;
                if (i < nb) rec[r] = vals[(int64_t)(start + lo + i) * vals_stride];
                // guard (never taken): an index past the records is dropped unread
                if (i < nb && rec[r] < n_records) {
                    const float4* q = reinterpret_cast<const float4*>(records + rec[r]);
                    keep = !tile_culled(q[0], q[1], tx0, ty0);
                }
                mk[r] = __ballot_sync(0xffffffffu, keep);
                if (lane == 0) s_cnt[r][warp] = __popc(mk[r]);
            }
            __syncthreads();
            int nk = 0, base[kStage];
#pragma unroll
            for (int r = 0; r < kStage; ++r) {
                base[r] = 0;
#pragma unroll
                for (int w = 0; w < kBwdWarps; ++w) {
                    if (w == warp) base[r] = nk;
                    nk += s_cnt[r][w];
                }
            }
#pragma unroll
            for (int r = 0; r < kStage; ++r) {
                if (mk[r] & (1u << lane)) {
                    const int k = base[r] + __popc(mk[r] & ((1u << lane) - 1u));
                    const float4* q = reinterpret_cast<const float4*>(records + rec[r]);
                    s_a[k] = stage_conic_a(q[0]);
                    s_b[k] = stage_conic_b(q[1]);
                    const float4 cc = q[2];
                    s_e[k] = make_int4(__float_as_int(cc.x), __float_as_int(cc.y),
                                       lo + r * kBwdThreads + threadIdx.x, 0);
                }
            }
            __syncthreads();
            for (int k0 = 0; k0 < nk; k0 += kSub) {
                const int k1 = min(nk, k0 + kSub);
                bool any_active = false;
                for (int k = k0; k < k1; ++k) {
                    const float4 a = s_a[k];
                    const float4 bb = s_b[k];
                    const int4 e = s_e[k];
                    const float cb = __int_as_float(e.x);
                    const bool active = e.y >= 0;  // uniform over the block
                    const int pos = e.z;
                    const float dx = p[0].fx - a.x;  // one column: shared by the pixels
                    float cP, cQ;  // the exponent's terms of this column
                    pair_column(dx, a.z, a.w, bb.y, cP, cQ);
                    float P[kPPT], dy[kPPT];
#pragma unroll
                    for (int j = 0; j < kPPT; ++j) P[j] = dy[j] = 0.f;
                    if (!active) {
#pragma unroll
                        for (int j = 0; j < kPPT; ++j)
                            bwd_entry<false>(p[j], pos, cP, cQ, a, bb, cb, nullptr, P[j], dy[j]);
                        continue;
                    }
                    any_active = true;
                    // per-thread sums over its pixels of dpow x (dx, dy, dx^2,
                    // dx dy, dy^2, 1) and of w g; the conic's coefficients and
                    // the opacity are applied per tile
                    float gr[kGradComps];
                    gr[6] = gr[7] = gr[8] = 0.f;
                    bool contrib = false;
#pragma unroll
                    for (int j = 0; j < kPPT; ++j)
                        contrib |= bwd_entry<true>(p[j], pos, cP, cQ, a, bb, cb, gr, P[j], dy[j]);
                    {
                        float D = 0.f, Sy = 0.f, Syy = 0.f;
#pragma unroll
                        for (int j = 0; j < kPPT; ++j) {
                            const float q = P[j] * dy[j];
                            D += P[j];
                            Sy += q;
                            Syy = __fmaf_rn(q, dy[j], Syy);
                        }
                        gr[0] = dx * D;
                        gr[1] = Sy;
                        gr[2] = dx * gr[0];
                        gr[3] = dx * Sy;
                        gr[4] = Syy;
                        gr[5] = D;
                    }
                    float* dst = &s_g[k - k0][warp][0];
                    if (__any_sync(0xffffffffu, contrib)) {
                        const float y = reduce8_scatter(gr, lane);
                        float z = gr[8];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
                        if ((lane & 3) == 0) dst[lane >> 2] = y;
                        if (lane == 0) dst[8] = z;
                    } else {
                        if ((lane & 3) == 0) dst[lane >> 2] = 0.f;
                        if (lane == 0) dst[8] = 0.f;
                    }
                }
                if (any_active) {  // uniform over the block
                    __syncthreads();
                    const int cnt = k1 - k0;
                    for (int e = threadIdx.x; e < cnt * kGradComps; e += kBwdThreads) {
                        const int ent = e / kGradComps, comp = e - ent * kGradComps;
                        const int slot = s_e[k0 + ent].y;
                        if (slot < 0) continue;
                        float S = 0.f, S2 = 0.f;  // this component's sums; S2 the other of du/dv
#pragma unroll
                        for (int w = 0; w < kBwdWarps; ++w) {
                            S += s_g[ent][w][comp];
                            if (comp < 2) S2 += s_g[ent][w][comp ^ 1];
                        }
                        // conic (A, B, C) and opacity of the entry, from its staged form
                        const float4 a = s_a[k0 + ent];
                        const float4 bb = s_b[k0 + ent];
                        const float A = -2.0f * kLn2 * a.z, B = -kLn2 * a.w,
                                    C = -2.0f * kLn2 * bb.x;
                        float g;
                        switch (comp) {
                            case 0: g = A * S + B * S2; break;   // du
                            case 1: g = C * S + B * S2; break;   // dv
                            case 2: g = -0.5f * S; break;        // dA
                            case 3: g = -S; break;               // dB
                            case 4: g = -0.5f * S; break;        // dC
                            case 5: g = S / ex2_approx(bb.y); break;  // dopacity
                            default: g = S;                      // colour
                        }
                        if (g != 0.f) atomicAdd(grad2d + (int64_t)slot * kG2Stride + comp, g);
                    }
                    __syncthreads();
                }
            }
            __syncthreads();
        }
        __syncthreads();  // s_tile / s_maxend are rewritten for the next tile
    }
}

// Zeroes the 2D gradient sums (float4 at a time) and the tile queue's counter.
__global__ void bwd_prologue_kernel(float4* __restrict__ grad2d, int64_t n4,
                                    int32_t* __restrict__ work_counter) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        grad2d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x == 0) *work_counter = 0;
}

// d Y_k / d(x, y, z) contracted with coefficients dY[k], accumulated in g.
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, int degree,
                                             const float* dY, float& gx, float& gy, float& gz) {
    const float C1 = 0.4886025119029199f;
    if (degree < 1) return;
    gy += -C1 * dY[1];
    gz += C1 * dY[2];
    gx += -C1 * dY[3];
    if (degree < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float a0 = 1.0925484305920792f, a1 = -1.0925484305920792f, a2 = 0.31539156525252005f,
                a3 = -1.0925484305920792f, a4 = 0.5462742152960396f;
    gx += a0 * y * dY[4];              gy += a0 * x * dY[4];
    gy += a1 * z * dY[5];              gz += a1 * y * dY[5];
    gx += -2.f * a2 * x * dY[6];       gy += -2.f * a2 * y * dY[6];   gz += 4.f * a2 * z * dY[6];
    gx += a3 * z * dY[7];              gz += a3 * x * dY[7];
    gx += 2.f * a4 * x * dY[8];        gy += -2.f * a4 * y * dY[8];
    if (degree < 3) return;
    const float b0 = -0.5900435899266435f, b1 = 2.890611442640554f, b2 = -0.4570457994644658f,
                b3 = 0.3731763325901154f, b4 = -0.4570457994644658f, b5 = 1.445305721320277f,
                b6 = -0.5900435899266435f;
    gx += 6.f * b0 * x * y * dY[9];    gy += b0 * (3.f * xx - 3.f * yy) * dY[9];
    gx += b1 * y * z * dY[10];         gy += b1 * x * z * dY[10];    gz += b1 * x * y * dY[10];
    gx += -2.f * b2 * x * y * dY[11];  gy += b2 * (4.f * zz - xx - 3.f * yy) * dY[11];
    gz += 8.f * b2 * y * z * dY[11];
    gx += -6.f * b3 * x * z * dY[12];  gy += -6.f * b3 * y * z * dY[12];
    gz += b3 * (6.f * zz - 3.f * xx - 3.f * yy) * dY[12];
    gx += b4 * (4.f * zz - 3.f * xx - yy) * dY[13];  gy += -2.f * b4 * x * y * dY[13];
    gz += 8.f * b4 * x * z * dY[13];
    gx += 2.f * b5 * x * z * dY[14];   gy += -2.f * b5 * y * z * dY[14];
    gz += b5 * (xx - yy) * dY[14];
    gx += b6 * (3.f * xx - 3.f * yy) * dY[15];  gy += -6.f * b6 * x * y * dY[15];
}

__global__ void __launch_bounds__(128)
backward_gaussian_kernel(const ClsScene* __restrict__ scenes, const ClsView* __restrict__ views,
                         const float* __restrict__ grad2d, float* __restrict__ grads) {
    const ClsScene& sc = scenes[blockIdx.y];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= sc.n_active) return;
    const int g = sc.active_idx[a];
    const float* row = sc.params + (int64_t)g * sc.row_stride;
    const float4 m = *reinterpret_cast<const float4*>(row);
    const float4 ls = *reinterpret_cast<const float4*>(row + 4);
    const float4 q = *reinterpret_cast<const float4*>(row + 8);
    const int deg = sc.sh_degree;
    const int K = (deg + 1) * (deg + 1);
    const float* sh = row + 12;

    float dmean[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
    float dlogit = 0.f;
    float dsh[48];
#pragma unroll
    for (int i = 0; i < 48; ++i) dsh[i] = 0.f;

    for (int j = sc.first_view; j < sc.first_view + sc.n_views; ++j) {
        const ClsView& view = views[j];
        const float4* g2p = reinterpret_cast<const float4*>(grad2d + (view.g2_base + a) * kG2Stride);
        const float4 e0 = g2p[0], e1 = g2p[1], e2 = g2p[2];
        const float du = e0.x, dv = e0.y, dA = e0.z, dB = e0.w, dC = e1.x, dop = e1.y;
        const float dcol[3] = {e1.z, e1.w, e2.x};
        if (du == 0.f && dv == 0.f && dA == 0.f && dB == 0.f && dC == 0.f && dop == 0.f &&
            dcol[0] == 0.f && dcol[1] == 0.f && dcol[2] == 0.f)
            continue;
        const ClsCamera& cam = view.cam;
        Proj P;
        project_gaussian(cam, m, ls, q, P);

        // colour
        float ddx = m.x - cam.pos[0], ddy = m.y - cam.pos[1], ddz = m.z - cam.pos[2];
        const float len = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
        const float il = 1.0f / len;
        const float dxn = ddx * il, dyn = ddy * il, dzn = ddz * il;
        float Y[16];
        sh_basis(dxn, dyn, dzn, deg, Y);
        // the loops run to 16 with a guard so that every index is a constant and
        // the arrays stay in registers
        float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < K) {
                raw[0] += Y[k] * sh[3 * k];
                raw[1] += Y[k] * sh[3 * k + 1];
                raw[2] += Y[k] * sh[3 * k + 2];
            }
        }
        float draw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) draw[c] = raw[c] >= 0.f ? dcol[c] : 0.f;
        float dY[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            dY[k] = 0.f;
            if (k < K) {
                dsh[3 * k] += Y[k] * draw[0];
                dsh[3 * k + 1] += Y[k] * draw[1];
                dsh[3 * k + 2] += Y[k] * draw[2];
                dY[k] = sh[3 * k] * draw[0] + sh[3 * k + 1] * draw[1] + sh[3 * k + 2] * draw[2];
            }
        }
        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
        sh_basis_vjp(dxn, dyn, dzn, deg, dY, gdx, gdy, gdz);
        const float dotd = gdx * dxn + gdy * dyn + gdz * dzn;
        dmean[0] += (gdx - dxn * dotd) * il;
        dmean[1] += (gdy - dyn * dotd) * il;
        dmean[2] += (gdz - dzn * dotd) * il;

        // opacity
        const float sig = 1.0f / (1.0f + __expf(-m.w));
        dlogit += dop * sig * (1.0f - sig);

        // conic -> 2D covariance (a, b, c)
        const float ca = P.a, cb = P.b, cc = P.c;
        const float det = P.det;
        const float id2 = 1.0f / (det * det);
        const float da = (-cc * cc * dA + cb * cc * dB - cb * cb * dC) * id2;
        const float dc = (-cb * cb * dA + ca * cb * dB - ca * ca * dC) * id2;
        const float db = (2.f * cb * cc * dA - (ca * cc + cb * cb) * dB + 2.f * ca * cb * dC) * id2;

        // 2D covariance -> 3D covariance and T = J W
        const float* T = P.T;
        const float* S = P.Sig;
        // Sigma T0^T and Sigma T1^T
        const float ST0[3] = {S[0] * T[0] + S[1] * T[1] + S[2] * T[2],
                              S[1] * T[0] + S[3] * T[1] + S[4] * T[2],
                              S[2] * T[0] + S[4] * T[1] + S[5] * T[2]};
        const float ST1[3] = {S[0] * T[3] + S[1] * T[4] + S[2] * T[5],
                              S[1] * T[3] + S[3] * T[4] + S[4] * T[5],
                              S[2] * T[3] + S[4] * T[4] + S[5] * T[5]};
        float dT0[3], dT1[3];
        for (int i = 0; i < 3; ++i) {
            dT0[i] = 2.f * da * ST0[i] + db * ST1[i];
            dT1[i] = 2.f * dc * ST1[i] + db * ST0[i];
        }
        // symmetric gradient of Sigma: G = da T0'T0 + db sym(T0'T1) + dc T1'T1
        float Gs[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k)
                Gs[i][k] = da * T[i] * T[k] + 0.5f * db * (T[i] * T[3 + k] + T[3 + i] * T[k]) +
                           dc * T[3 + i] * T[3 + k];
        // M = Rq diag(s); dL/dM = 2 G M
        float Mx[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) Mx[i][k] = P.Rq[i * 3 + k] * P.s[k];
        float dRq[9];
        float ds[3] = {0.f, 0.f, 0.f};
        for (int i = 0; i < 3; ++i) {
            for (int k = 0; k < 3; ++k) {
                const float dM = 2.f * (Gs[i][0] * Mx[0][k] + Gs[i][1] * Mx[1][k] + Gs[i][2] * Mx[2][k]);
                dRq[i * 3 + k] = dM * P.s[k];
                ds[k] += dM * P.Rq[i * 3 + k];
            }
        }
        for (int k = 0; k < 3; ++k) dls[k] += ds[k] * P.s[k];
        // rotation matrix -> normalised quaternion -> raw quaternion
        {
            const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
            const float* Gq = dRq;
            const float dw = 2.f * (-z * Gq[1] + y * Gq[2] + z * Gq[3] - x * Gq[5] - y * Gq[6] +
                                    x * Gq[7]);
            const float dx_ = 2.f * (y * Gq[1] + z * Gq[2] + y * Gq[3] - 2.f * x * Gq[4] - w * Gq[5] +
                                     z * Gq[6] + w * Gq[7] - 2.f * x * Gq[8]);
            const float dy_ = 2.f * (-2.f * y * Gq[0] + x * Gq[1] + w * Gq[2] + x * Gq[3] + z * Gq[5] -
                                     w * Gq[6] + z * Gq[7] - 2.f * y * Gq[8]);
            const float dz_ = 2.f * (-2.f * z * Gq[0] - w * Gq[1] + x * Gq[2] + w * Gq[3] -
                                     2.f * z * Gq[4] + y * Gq[5] + x * Gq[6] + y * Gq[7]);
            const float dot = w * dw + x * dx_ + y * dy_ + z * dz_;
            const float inv = 1.0f / P.qnorm;
            dq[0] += (dw - w * dot) * inv;
            dq[1] += (dx_ - x * dot) * inv;
            dq[2] += (dy_ - y * dot) * inv;
            dq[3] += (dz_ - z * dot) * inv;
        }
        // T = J W -> J entries -> camera-space point
        const float* Wr = cam.R;
        const float dJ00 = dT0[0] * Wr[0] + dT0[1] * Wr[1] + dT0[2] * Wr[2];
        const float dJ02 = dT0[0] * Wr[6] + dT0[1] * Wr[7] + dT0[2] * Wr[8];
        const float dJ11 = dT1[0] * Wr[3] + dT1[1] * Wr[4] + dT1[2] * Wr[5];
        const float dJ12 = dT1[0] * Wr[6] + dT1[1] * Wr[7] + dT1[2] * Wr[8];
        const float pz = P.pz;
        const float iz = 1.0f / pz, iz2 = iz * iz, iz3 = iz2 * iz;
        const float limx = 1.3f * (0.5f * (float)cam.width / cam.fx);
        const float limy = 1.3f * (0.5f * (float)cam.height / cam.fy);
        const float txz = fminf(fmaxf(P.xz, -limx), limx);
        const float tyz = fminf(fmaxf(P.yz, -limy), limy);
        const float tx = txz * pz, ty = tyz * pz;
        const float dtx = -cam.fx * iz2 * dJ02;
        const float dty = -cam.fy * iz2 * dJ12;
        float dpx = 0.f, dpy = 0.f;
        float dpz = -cam.fx * iz2 * dJ00 + 2.f * cam.fx * tx * iz3 * dJ02 - cam.fy * iz2 * dJ11 +
                    2.f * cam.fy * ty * iz3 * dJ12;
        if (P.clamp_x) dpz += dtx * txz; else dpx += dtx;
        if (P.clamp_y) dpz += dty * tyz; else dpy += dty;
        // image position
        dpx += du * cam.fx * iz;
        dpy += dv * cam.fy * iz;
        dpz += -(du * cam.fx * P.px + dv * cam.fy * P.py) * iz2;
        dmean[0] += Wr[0] * dpx + Wr[3] * dpy + Wr[6] * dpz;
        dmean[1] += Wr[1] * dpx + Wr[4] * dpy + Wr[7] * dpz;
        dmean[2] += Wr[2] * dpx + Wr[5] * dpy + Wr[8] * dpz;
    }

    float* out = grads + (sc.grad_base + a) * sc.row_stride;
    reinterpret_cast<float4*>(out)[0] = make_float4(dmean[0], dmean[1], dmean[2], dlogit);
    reinterpret_cast<float4*>(out)[1] = make_float4(dls[0], dls[1], dls[2], 0.f);
    reinterpret_cast<float4*>(out)[2] = make_float4(dq[0], dq[1], dq[2], dq[3]);
    // the colour coefficients (constant indices, so dsh stays in registers),
    // then zeros up to the row's stride
#pragma unroll
    for (int i = 0; i < 48; i += 4) {
        if (i < sc.row_stride - 12) {
            float4 v;
            v.x = i < 3 * K ? dsh[i] : 0.f;
            v.y = i + 1 < 3 * K ? dsh[i + 1] : 0.f;
            v.z = i + 2 < 3 * K ? dsh[i + 2] : 0.f;
            v.w = i + 3 < 3 * K ? dsh[i + 3] : 0.f;
            reinterpret_cast<float4*>(out + 12)[i / 4] = v;
        }
    }
    for (int i = 48; i < sc.row_stride - 12; i += 4)
        reinterpret_cast<float4*>(out + 12)[i / 4] = make_float4(0.f, 0.f, 0.f, 0.f);
}

static PerDevice g_bwd_blocks;

}  // namespace cls

using namespace cls;

extern "C" int cls_render_backward(const ClsScene* scenes_dev, const ClsView* views_dev,
                                   const ClsBatchInfo* info, const ClsProjected* records,
                                   const uint32_t* vals, int32_t vals_stride,
                                   const uint32_t* ranges,
                                   const int32_t* active_tiles, const int32_t* n_active_tiles_dev,
                                   const ClsTileCache* tile_cache, const float* prefix_state,
                                   const float* image, const int32_t* n_contrib,
                                   const float* dL_dimage, float* grad2d, float* grads,
                                   int32_t* work_counter, cls_stream_t stream) {
    if (!scenes_dev || !views_dev || !info || !records || !vals ||
        (vals_stride != 1 && vals_stride != 2) || !ranges || !active_tiles ||
        !n_active_tiles_dev || !tile_cache || !prefix_state || !image || !n_contrib ||
        !dL_dimage || !work_counter ||
        info->n_views <= 0 || info->total_tiles <= 0 || info->n_scenes > 65535 ||
        (info->total_g2 > 0 && !grad2d) || (info->total_grad_rows > 0 && !grads))
        return CLS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int bwd_blocks = per_device(g_bwd_blocks, [](int dev) {
        return resident_blocks(dev, render_bwd_kernel, kBwdThreads, 0);
    });
    const int blocks = (int)hmin64(info->total_tiles, bwd_blocks);
    if (info->total_g2 > 0 && ((uintptr_t)grad2d & 15) == 0) {
        // the 2D gradient sums and the tile queue zeroed in one launch
        const int64_t n4 = info->total_g2 * (kG2Stride / 4);
        bwd_prologue_kernel<<<(unsigned)hmin64((n4 + 255) / 256, 1024), 256, 0, s>>>(
            reinterpret_cast<float4*>(grad2d), n4, work_counter);
    } else {
        if (info->total_g2 > 0)
            cudaMemsetAsync(grad2d, 0, (size_t)info->total_g2 * kG2Stride * sizeof(float), s);
        cudaMemsetAsync(work_counter, 0, sizeof(int32_t), s);
    }
    render_bwd_kernel<<<blocks, kBwdThreads, 0, s>>>(
        views_dev, info->n_views, records, (uint32_t)hmin64(info->total_records, 0xffffffffll),
        vals, vals_stride, ranges, active_tiles, n_active_tiles_dev, tile_cache, prefix_state,
        image, n_contrib, dL_dimage, grad2d, work_counter);
    if (info->max_active > 0 && info->total_grad_rows > 0) {
        backward_gaussian_kernel<<<dim3((info->max_active + 127) / 128, info->n_scenes), 128, 0,
                                   s>>>(scenes_dev, views_dev, grad2d, grads);
    }
    CLS_CHECK_LAUNCH();
    return CLS_OK;
}
