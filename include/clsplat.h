/*
 * clsplat.h - C ABI of the GB300 (sm_103a) active-set Gaussian-splatting
 * library: the local-optimisation hot path of CL-Splats (arXiv 2506.21117).
 *
 * The paper updates an existing 3D Gaussian Splatting scene after a local
 * change: Gaussians whose centres project into the 2D change masks of enough
 * new views form the active set O^t (Sec. 3.2, Supp. majority-voting
 * equation); only O^t is optimised, while every other Gaussian is still
 * rendered as a frozen occluder (Table 4 (a)); rendering and back-propagation
 * run only on the 16x16 tiles that O^t touches, and the gradients of O^t are
 * the full-scene gradients (Sec. 3.3 and Supp. "Local Optimization Kernel").
 * The rasterizer itself is the base 3DGS method's (Supp. "Implementation
 * Details"): EWA projection with SH colour, 3-sigma tile binning, a
 * (tile, depth) sort and front-to-back alpha compositing.
 *
 * Conventions shared by every call
 *  - All pointers named *_dev, and every array argument unless stated
 *    otherwise, are DEVICE pointers owned by the caller. The library never
 *    allocates, frees or synchronises; it only enqueues work on `stream`.
 *  - Work buffers come from the caller; their sizes come from the matching
 *    *_workspace_size query. Workspaces must be 256-byte aligned.
 *  - Every call returns CLS_OK or an error code. Argument errors are detected
 *    on the host before anything is launched. Errors found on the device
 *    (pair capacity exceeded, a wait that gave up) are written to the caller's
 *    device status word `status_dev` (CLS_OK is never written there, so the
 *    caller zeroes it once and reads it after a synchronisation); the kernels
 *    stay within every buffer whatever the status.
 *  - float32 throughout; row-major; no ownership is transferred.
 *
 * Gaussian parameter rows (one row of `row_stride` floats per Gaussian):
 *   [0..2] mean xyz   [3] opacity logit   [4..6] log scale xyz   [7] unused
 *   [8..11] rotation quaternion (w, x, y, z), any non-zero norm
 *   [12 ..] SH coefficients, coefficient-major: sh[k*3 + channel], k < (deg+1)^2
 *   row_stride = cls_row_stride(sh_degree): 16, 24, 40, 64 for degree 0..3.
 */
#ifndef CLSPLAT_H
#define CLSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cls_stream_t; /* the same handle as cudaStream_t */

enum {
    CLS_OK = 0,
    CLS_ERR_INVALID_ARG = 1, /* bad size, NULL pointer or unsupported option */
    CLS_ERR_CAPACITY = 2,    /* more (Gaussian, tile) pairs than key capacity */
    CLS_ERR_CUDA = 3,        /* a launch failed (cudaGetLastError) */
    CLS_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    CLS_ERR_INTERNAL = 5     /* a device-side consistency guard skipped an access
                                (the call's outputs are not valid) */
};

#define CLS_TILE 16
#define CLS_MAX_SH_DEGREE 3

/* Pinhole camera (Supp. "Camera Pose Estimation": poses are inputs).
 * p_cam = R * p_world + t; x right, y down, z forward; pixel (i, j) covers
 * [i, i+1) x [j, j+1); u = fx * x / z + cx. `pos` is the camera centre in
 * world space (origin of the SH view direction). Points with z <= znear are
 * culled. */
typedef struct ClsCamera {
    float R[9];
    float t[3];
    float pos[3];
    float fx, fy, cx, cy;
    float znear;
    int32_t width, height;
} ClsCamera;

/* One scene of a batch. `params`, `adam_m`, `adam_v` are [n][row_stride].
 * `active_idx` lists O^t in ascending order (n_active entries). `adam_step`
 * is one device int per scene (the shared Adam step counter t). Fields marked
 * "derived" are filled by cls_batch_prepare. */
typedef struct ClsScene {
    float* params;
    float* adam_m;
    float* adam_v;
    const int32_t* active_idx;
    int32_t* adam_step;
    int32_t n;
    int32_t row_stride;
    int32_t sh_degree;
    int32_t n_active;
    int32_t first_view; /* views of a scene are contiguous in the view table */
    int32_t n_views;
    int64_t grad_base;  /* derived: first row of this scene in `grads` */
} ClsScene;

/* One rendered view of a batch. Every view belongs to one scene. */
typedef struct ClsView {
    ClsCamera cam;
    int32_t scene;
    int32_t tiles_x, tiles_y; /* derived: ceil(W/16), ceil(H/16) */
    int32_t tile_base;        /* derived: first global tile id */
    int32_t sat_base;         /* derived: first entry of its tile-count table */
    int32_t pad0;
    int64_t rec_base;         /* derived: first projected record (= sum of n of earlier views) */
    int64_t pix_base;         /* derived: first pixel in per-pixel buffers */
    int64_t g2_base;          /* derived: first 2D-gradient slot (sum of n_active of earlier views) */
    float loss_scale;         /* derived: 1 / (3 W H n_views(scene)) */
    int32_t pad1;
} ClsView;

/* Totals of a batch, filled by cls_batch_prepare (host struct). */
typedef struct ClsBatchInfo {
    int32_t n_scenes, n_views;
    int32_t max_n, max_active;
    int32_t max_row_stride;
    int32_t key_bits;      /* 32 + bits of the largest global tile id */
    int64_t total_tiles;   /* sum of tiles_x * tiles_y */
    int64_t total_sat;     /* sum of (tiles_x + 1) * (tiles_y + 1) */
    int64_t total_records; /* sum over views of n(scene) */
    int64_t total_pixels;  /* sum over views of W * H */
    int64_t total_g2;      /* sum over views of n_active(scene) */
    int64_t total_grad_rows; /* sum over scenes of n_active */
    int64_t max_view_tiles;  /* largest tiles_x * tiles_y of a view */
} ClsBatchInfo;

/* Projected 2D record of one Gaussian in one view (48 bytes), written by
 * cls_project_and_bin at record index view.rec_base + gaussian index.
 * radius == 0 marks a culled Gaussian. `g2_slot` is the 2D-gradient slot of an
 * active Gaussian (view.g2_base + rank in active_idx) or -1 (static). */
typedef struct ClsProjected {
    float u, v, conic_a, conic_b;
    float conic_c, opacity, r, g;
    float b;
    int32_t g2_slot;
    float z;
    int32_t radius;
} ClsProjected;

/* Static-prefix cache of one tile (16 bytes), kept by the caller across the
 * iterations of one update (ClsTileCache [total_tiles], every byte 0xff at the
 * start of an update, i.e. no tile cached). Static Gaussians are frozen during
 * an update, so the compositing state of a pixel after the static Gaussians in
 * front of every active Gaussian of its tile does not change between
 * iterations. The prefix of a tile is the entries of its sorted list with
 * bits(z) < zb; the pixel state after the prefix is kept in prefix_state /
 * prefix_last (see cls_render_forward). cls_project_and_bin decides per active
 * tile whether the cache still holds (every active Gaussian of the tile has
 * bits(z) >= zb) or must be rebuilt (n_prefix is then set to
 * CLS_PREFIX_UNKNOWN and zb moved in front of the tile's nearest active
 * Gaussian: in the flat layout a margin of 2^17 float ulps, about 1.6%, in
 * front of its depth; in the bucketed layout to the lowest depth of the depth
 * bin in front of the one that holds it); the forward pass writes the state and n_prefix of
 * rebuilt tiles and last_active of every tile it renders. */
typedef struct ClsTileCache {
    uint32_t zb;          /* prefix boundary, bits of a positive float depth */
    uint32_t n_prefix;    /* list entries in the prefix, or CLS_PREFIX_UNKNOWN */
    uint32_t zmin_active; /* flat layout: smallest bits(z) of the tile's active
                             Gaussians; bucketed: the lowest bits(z) of the depth
                             bin of the nearest one (a lower bound of it) */
    int32_t last_active;  /* last list position of an active entry, -1 if none */
} ClsTileCache;
#define CLS_PREFIX_UNKNOWN 0xffffffffu

/* Floats per parameter row for an SH degree (0..3); -1 if out of range. */
int32_t cls_row_stride(int32_t sh_degree);

/* Fill the derived fields of `scenes` and `views` (host arrays) and the batch
 * totals. Views must be grouped by scene (scene s owns views
 * [first_view, first_view + n_views)). Pure host code; copy both tables to
 * the device afterwards. Returns CLS_ERR_INVALID_ARG on inconsistent tables. */
int cls_batch_prepare(ClsScene* scenes, int32_t n_scenes, ClsView* views, int32_t n_views,
                      ClsBatchInfo* info);

/* ------------------------------------------------------------------------
 * Change-mask lifting (Sec. 3.2 "Mask Majority Voting"; Supp. "Identifying
 * Changed 3D Regions via Majority Voting", voting equation).
 * For every Gaussian of one scene and every one of its views: project the
 * centre, c = views whose binary mask is non-zero at the centre's pixel,
 * o = views where the centre is outside the image or behind znear.
 * vote_mode 0: active iff 4 o < 3 V and V < 2 c  ((4/3) o < |I^t| < 2 c).
 * vote_mode 1 ("All Vote", Table 4 (b)): active iff c == V.
 *   params      [n][row_stride] of the scene (only the mean is read)
 *   views_dev   the batch view table; this scene's views are
 *               [first_view, first_view + n_views)
 *   masks       uint8, view j's H x W mask at offset views[j].pix_base
 *   active_out  uint8 [n] (1 = in O^t)
 *   active_idx_out int32 [n] capacity; ascending indices of O^t
 *   n_active_out   device int32 (count)
 *   votes_out   optional int32 [n][2] = (c, o), may be NULL
 * The float32 projection uses one fixed sequence of correctly rounded
 * operations, so the votes are bit-reproducible. */
size_t cls_lift_workspace_size(int32_t n);
int cls_lift_change_masks(const float* params, int32_t n, int32_t row_stride,
                          const ClsView* views_dev, int32_t first_view, int32_t n_views,
                          const uint8_t* masks, int32_t vote_mode, uint8_t* active_out,
                          int32_t* active_idx_out, int32_t* n_active_out, int32_t* votes_out,
                          void* workspace, size_t workspace_bytes, cls_stream_t stream);

/* Allocation-free change-mask lifting. The paper has no counterpart: this
 * entry exists for callers that cannot allocate device memory at all, for
 * example a plug-in that runs inside a host application owning every device
 * allocation, or a latency-critical loop where an allocation call could
 * synchronise the device. It computes exactly what cls_lift_change_masks
 * computes, with the same arguments minus the workspace: its scratch (one
 * count per 2048 Gaussians) sits in a fixed device array inside the library,
 * sized for at most CLS_LIFT_STATIC_MAX_N Gaussians (64 KiB, held on every
 * device that loads the library until the process exits).
 *  - n above CLS_LIFT_STATIC_MAX_N returns CLS_ERR_INVALID_ARG, nothing runs.
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current and keeps it for later
 *    calls; make that first call before any stream capture. It allocates
 *    nothing (no cudaMalloc/cudaFree, no allocating library routine).
 *  - The kept address belongs to the device's current context: after
 *    cudaDeviceReset on that device it is stale, so do not call this entry
 *    again in a process that has reset the device.
 *  - All calls share the one array. Each call writes every slot it reads
 *    before reading it, so no clearing is needed, but two calls that overlap
 *    on the GPU (different streams, no ordering between them) race on it and
 *    give wrong results: order them. */
#define CLS_LIFT_STATIC_MAX_N (1 << 24)
int cls_lift_change_masks_static(const float* params, int32_t n, int32_t row_stride,
                                 const ClsView* views_dev, int32_t first_view, int32_t n_views,
                                 const uint8_t* masks, int32_t vote_mode, uint8_t* active_out,
                                 int32_t* active_idx_out, int32_t* n_active_out,
                                 int32_t* votes_out, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Projection, dynamic render mask and binning (Supp. "Local Optimization
 * Kernel", item 1; base 3DGS preprocessing).
 * project_mode 0 projects every Gaussian of every view (the frozen occluders;
 * do this once per camera set), mode 1 re-projects only the active Gaussians
 * (every iteration, after the parameters change); the records and the
 * workspace (which keeps every record's tile rectangle) of earlier calls
 * supply the rest, so both must be kept between calls. In the bucketed layout
 * the mode 0 call also fixes each view's depth bins (from the depths of its
 * pair-producing Gaussians) and counts the static Gaussians' pairs per (tile,
 * depth bin) once; mode 1 calls keep both, so between a mode 0 call and the
 * mode 1 calls that follow it the active set and the static Gaussians must
 * not change (the workspace must be zero-filled before its first use).
 * Mode 2 (bucketed layout, keys and a capacity > 0 required) only writes the
 * bucket offsets and emits the pairs that the immediately preceding call
 * counted with capacity 0, with the same arguments otherwise and the same
 * workspace: nothing it reads may change in between. Then:
 *   tile_active[total_tiles]  uint8: 1 iff a non-culled active Gaussian's
 *                             tile rectangle holds the tile
 *   active_tiles[total_tiles] int32: ascending global ids of active tiles,
 *                             n_active_tiles_dev = their count
 *   one pair per (Gaussian, active tile), static and active Gaussians alike,
 *   in one of two layouts:
 *   layout 0 (flat, for cls_sort_keys): keys[i] = (global tile id << 32) |
 *     bits(depth z), vals[i] = record index, emitted in view order, then
 *     Gaussian order, then row-major tile order.
 *   layout 1 (bucketed, for cls_sort_tiles): keys[i] = (bits(z) << 32) |
 *     record index; `vals` is unused. Pairs are grouped by tile (tiles in
 *     active-tile order) and, inside a tile, by CLS_DEPTH_BINS depth bins
 *     that split the view's depth range of pair-producing Gaussians evenly in
 *     float-bit space (up to float rounding; monotone in depth); the order
 *     inside a bin is unspecified until cls_sort_tiles. ranges[tile] =
 *     (start, end) of each tile ((0, 0) if inactive) and
 *     bin_offsets[r * CLS_DEPTH_BINS + b] the start of bin b of the r-th
 *     active tile (cls_bin_offsets_size entries).
 *   n_pairs_dev               device int64: number of pairs needed; if it
 *                             exceeds `capacity`, CLS_ERR_CAPACITY is written
 *                             to status_dev and only `capacity` pairs are kept
 *                             (offsets and ranges are clamped to capacity).
 *                             With capacity 0 (keys may then be NULL) the
 *                             bucketed layout only counts: n_pairs, the
 *                             tile mask and list (ranges stay zero); the
 *                             per-bucket counts stay in the workspace for
 *                             project_mode 2.
 * Tile rectangle: radius r = ceil(3 sqrt(lambda_max(Sigma'))), tiles
 * floor((u - r)/16) .. floor((u + r)/16) clamped to the grid (same for v).
 * records [total_records] ClsProjected.
 * tile_cache [total_tiles] (required): the static-prefix decision of every
 * active tile (see ClsTileCache). prefix_mode 0 rebuilds every active tile's
 * prefix (for callers whose static Gaussians may change between calls);
 * prefix_mode 1 keeps a tile's cached prefix while it holds, and the bucketed
 * layout then does not write the pairs of depth bins that lie entirely in
 * front of the tile's boundary (their slots stay in bin_offsets).
 * tile_ring 1 also renders the ring of tiles around the covered ones
 * (tile_active 2: uncovered, one of its eight neighbours covered), which the
 * D-SSIM window needs (cls_ssim_loss); tile_active is 1 on covered tiles in
 * both modes, and every tile with tile_active != 0 is in active_tiles. */
#define CLS_DEPTH_BINS 256
size_t cls_project_workspace_size(const ClsBatchInfo* info);
size_t cls_bin_offsets_size(const ClsBatchInfo* info); /* uint32 entries */
int cls_project_and_bin(const ClsScene* scenes_dev, const ClsView* views_dev,
                        const ClsBatchInfo* info, int32_t project_mode, int32_t layout,
                        ClsProjected* records, uint8_t* tile_active, int32_t* active_tiles,
                        int32_t* n_active_tiles_dev, uint64_t* keys, uint32_t* vals,
                        int64_t capacity, int64_t* n_pairs_dev, uint32_t* ranges,
                        uint32_t* bin_offsets, uint8_t* bin_cut,
                        ClsTileCache* tile_cache, int32_t prefix_mode, int32_t tile_ring,
                        int32_t* status_dev, void* workspace, size_t workspace_bytes,
                        cls_stream_t stream);

/* Speculative depth cut (bucketed layout). With bin_cut != NULL (uint8
 * [total_tiles], the last depth bin to emit per global tile id), pairs of
 * deeper bins are counted and given their slots in bin_offsets but not
 * written. cls_render_forward with cut_in = bin_cut stops each tile at its
 * cut, records in cut_out the last bin the tile needed plus a margin (the cut
 * of the next iteration), and lists in `trunc` every tile that ran out of
 * emitted bins before all its pixels saturated (its outputs are not written).
 * cls_complete_truncated then writes the missing pairs of those tiles (same
 * workspace as the preceding cls_project_and_bin call, unchanged), and a
 * second cls_render_forward over the listed tiles (active_tiles = trunc,
 * n_active_tiles_dev = trunc_count, list_ranks = trunc + trunc_cap, cut_in =
 * NULL) renders them completely. The result equals rendering without a cut.
 *   trunc  int32 [3 * trunc_cap]: tile ids, their active-tile ranks, old cuts
 *   trunc_cap >= total_tiles; trunc_count device int32 (caller zeroes it)
 * Bins in front of a cached prefix boundary stay unwritten here too.
 * cls_project_and_bin writes bin_cut in one case: a tile whose cached prefix
 * it drops (the tile is rebuilt from the front) gets a cut of at least the
 * depth bin of its old boundary plus the margin, since its pixels that stopped
 * inside the old prefix need no deeper bin. */
int cls_complete_truncated(const ClsView* views_dev, const ClsBatchInfo* info,
                           const ClsProjected* records, uint64_t* keys, int64_t capacity,
                           const int32_t* trunc, const int32_t* trunc_count, int64_t trunc_cap,
                           int32_t* work_counter, void* workspace, size_t workspace_bytes,
                           cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Per-tile depth sort of the bucketed layout (Supp. "Local Optimization
 * Kernel", item 1: per-tile depth order). Binning already did the most
 * significant radix pass (tile, then depth bin); this sorts every bucket with
 * at least `min_bin` keys by its key, i.e. by depth, equal depths by record
 * index, in shared memory. min_bin <= 1 sorts every bucket, so each tile's
 * pairs end in (depth, index) order. A larger min_bin leaves the small buckets
 * to cls_render_forward, which sorts them lazily (pass CLS_LAZY_MAX_BIN + 1).
 *   keys        [capacity] in/out, layout 1 of cls_project_and_bin
 *   keys_alt    [capacity] scratch (used only for buckets above 4096 pairs)
 *   bin_offsets as written by cls_project_and_bin
 *   work_counter device int32 scratch (reset by the call)
 *   workspace   cls_sort_tiles_workspace_size(capacity, min_bin) bytes
 * With the speculative depth cut (min_bin > 1 only): `cut` (with
 * active_tiles) skips bins beyond each tile's cut, which are not emitted yet;
 * `trunc` (see cls_complete_truncated) restricts the call to the completed
 * tiles' bins beyond their old cut, to be run after cls_complete_truncated.
 * `tile_cache` (optional) skips bins that lie entirely in a tile's cached
 * prefix, which are not emitted. */
#define CLS_LAZY_MAX_BIN 1024
size_t cls_sort_tiles_workspace_size(int64_t capacity, int32_t min_bin);
int cls_sort_tiles(uint64_t* keys, uint64_t* keys_alt, const uint32_t* bin_offsets,
                   const int32_t* active_tiles, const int32_t* n_active_tiles_dev,
                   int64_t total_tiles, int64_t capacity, int32_t min_bin, const uint8_t* cut,
                   const int32_t* trunc, const int32_t* trunc_count, int64_t trunc_cap,
                   const ClsTileCache* tile_cache, int32_t* work_counter, void* workspace,
                   size_t workspace_bytes, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Stable LSD radix sort of the flat layout's (tile, depth) keys with their
 * values (Supp. "Local Optimization Kernel", item 1: per-tile depth order),
 * one 8-bit digit per pass, single-pass digit scattering with decoupled
 * look-back, then the per-tile [start, end) ranges.
 *   keys, vals        [capacity] in/out; sorted result ends here
 *   keys_alt, vals_alt [capacity] ping-pong buffers
 *   n_pairs_dev       device int64 count (values above capacity are clamped)
 *   key_bits          significant key bits (<= 64); passes = ceil(bits / 8)
 *   ranges            optional uint32 [n_tiles][2] (start, end); tiles with
 *                     no pair get (0, 0); may be NULL
 * A look-back wait (a partition polling the state of the one before it)
 * that exceeds CLS_SORT_SPIN_LIMIT polls writes CLS_ERR_TIMEOUT to status_dev;
 * the pass then goes on with the prefix summed so far, so every write stays
 * inside the buffers but the order is unspecified. The call never hangs. */
#define CLS_SORT_SPIN_LIMIT (1 << 22)
size_t cls_sort_workspace_size(int64_t capacity, int32_t key_bits);
int cls_sort_keys(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                  const int64_t* n_pairs_dev, int64_t capacity, int32_t key_bits,
                  uint32_t* ranges, int64_t n_tiles, int32_t* status_dev, void* workspace,
                  size_t workspace_bytes, cls_stream_t stream);
/* cls_sort_keys with the look-back bound given: at most `spin_limit` polls
 * (>= 0; CLS_ERR_INVALID_ARG otherwise) per wait before CLS_ERR_TIMEOUT. A
 * small bound makes the timeout path reachable on purpose (0: give up at the
 * first partition that has not published yet); cls_sort_keys passes
 * CLS_SORT_SPIN_LIMIT. */
int cls_sort_keys_bounded(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                          uint32_t* vals_alt, const int64_t* n_pairs_dev, int64_t capacity,
                          int32_t key_bits, uint32_t* ranges, int64_t n_tiles,
                          int32_t* status_dev, void* workspace, size_t workspace_bytes,
                          int64_t spin_limit, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Forward render of the active tiles only (Supp. "Local Optimization
 * Kernel", item 2). Per pixel of an active tile, over its tile's sorted list:
 * alpha = min(0.99, opacity * exp(-1/2 (A dx^2 + C dy^2) - B dx dy)), skipped
 * if the exponent is > 0 or alpha < 1/255; stop before a Gaussian when
 * T (1 - alpha) < 1e-4; C += colour alpha T; T *= 1 - alpha; C += T bg.
 * The record index of sorted pair i is vals[i * vals_stride]: vals_stride 1
 * with the flat layout's vals, 2 with the bucketed layout's keys (low words).
 * Lazy sorting (bucketed layout, bin_offsets != NULL): the tile's depth bins
 * are walked front to back; bins of at most CLS_LAZY_MAX_BIN keys are sorted
 * here in shared memory (consecutive bins gathered up to 256 keys) and written
 * back to lazy_keys, larger bins must already be sorted (cls_sort_tiles with
 * min_bin = CLS_LAZY_MAX_BIN + 1); bins behind the depth at which every pixel
 * of the tile stopped are left unsorted (the backward pass never reads them).
 * vals/vals_stride are ignored in that mode. list_ranks (optional) gives the
 * active-tile rank of each listed tile (default: its position in the list);
 * cut_in/cut_out/trunc: see cls_complete_truncated (all may be NULL).
 * Static prefix (tile_cache, as decided by cls_project_and_bin): a tile whose
 * cache holds starts from the kept pixel state at list position n_prefix; a
 * tile to rebuild is composited from the front, and the state of each pixel on
 * reaching the first entry with bits(z) >= zb (or at the end, if every pixel
 * saturated before it) is written to
 *   prefix_state [total_pixels][4] float: (T, C_r, C_g, C_b) after the
 *                prefix, T negated if the pixel stopped inside the prefix
 *   prefix_last  [total_pixels] int32: n_contrib after the prefix
 * and n_prefix to the tile's cache. Both paths give the same result.
 * Outputs at the view's pix_base (pixels of inactive tiles are not written):
 *   image      [3][H][W] per view (planar; required, read by the backward)
 *   T_final    [H][W], n_contrib [H][W] (one past the last list position
 *              composited, counted from the tile's range start)
 *   loss_mode  0 none, 1 L1, 2 L2 against `target` ([3][H][W] per view):
 *              dL_dimage = l'(C - C*) * loss_scale and loss_per_scene[scene]
 *              += sum l(C - C*) * loss_scale over the rendered pixels.
 *              dL_dimage and loss_per_scene may be NULL when loss_mode is 0;
 *              loss_per_scene is accumulated, the caller zeroes it.
 *   work_counter device int32 scratch (reset by the call).
 * bg is a host array of 3 floats. */
int cls_render_forward(const ClsView* views_dev, const ClsBatchInfo* info,
                       const ClsProjected* records, const uint32_t* vals, int32_t vals_stride,
                       const uint32_t* ranges, const int32_t* active_tiles,
                       const int32_t* n_active_tiles_dev, uint64_t* lazy_keys,
                       const uint32_t* bin_offsets, const int32_t* list_ranks,
                       const uint8_t* cut_in, uint8_t* cut_out, int32_t* trunc,
                       int32_t* trunc_count, int64_t trunc_cap, ClsTileCache* tile_cache,
                       float* prefix_state, int32_t* prefix_last, const float* bg,
                       const float* target,
                       int32_t loss_mode, float* image, float* T_final, int32_t* n_contrib,
                       float* dL_dimage, float* loss_per_scene, int32_t* work_counter,
                       cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Backward pass (Supp. "Local Optimization Kernel", items 2 and 3). Pixel
 * part: per active-tile pixel, start from the state the forward pass kept
 * after the tile's static prefix (tile_cache, prefix_state) and walk the list
 * front to back up to the earlier of the pixel's last contributor and the
 * tile's last active entry, recomputing T before each Gaussian exactly as the
 * forward pass did; the colour behind a Gaussian is the final colour (image)
 * minus the colour composited up to and including it, so no
 * per-Gaussian-per-pixel state is stored. Static Gaussians update T and that
 * colour but produce no gradient; the 2D gradients of each active
 * Gaussian are reduced over the tile's pixels and added into
 *   grad2d [total_g2][12]: du, dv, dA, dB, dC, d opacity, d r, d g, d b, 0, 0, 0
 * (zeroed by the call). Gaussian part (active Gaussians only): chain rule to
 * every parameter of the row, summed over the scene's views, written to
 *   grads [total_grad_rows][row_stride] at row scene.grad_base + rank
 * (every float of the row is written). dL_dimage as written by the forward
 * call or supplied by the caller ([3][H][W] per view); image, prefix_state
 * and n_contrib as the forward call left them. */
int cls_render_backward(const ClsScene* scenes_dev, const ClsView* views_dev,
                        const ClsBatchInfo* info, const ClsProjected* records,
                        const uint32_t* vals, int32_t vals_stride, const uint32_t* ranges,
                        const int32_t* active_tiles,
                        const int32_t* n_active_tiles_dev, const ClsTileCache* tile_cache,
                        const float* prefix_state, const float* image,
                        const int32_t* n_contrib, const float* dL_dimage, float* grad2d,
                        float* grads, int32_t* work_counter, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * D-SSIM term of the photometric loss (Supp. "Implementation Details": the
 * base 3DGS optimiser's (1 - lambda) L1 + lambda (1 - SSIM), SSIM with an
 * 11 x 11 Gaussian window of standard deviation 1.5, C1 = 0.01^2,
 * C2 = 0.03^2, zero padding at the image border, mean over 3 H W per view).
 * Call after cls_render_forward with loss_mode 1 (L1) and loss_per_scene NULL,
 * on a batch binned with tile_ring 1: `tiles`/`n_tiles_dev` the rendered tile
 * list (active_tiles), tile_active as cls_project_and_bin wrote it. On the
 * pixels of covered tiles (tile_active 1) it replaces dL_dimage (the forward
 * pass's L1 gradient sign(C - C*) * loss_scale) by the gradient of the
 * combined loss with respect to the image — the D-SSIM part is that of the
 * whole image: the ring supplies every pixel within 10 of a covered one — and
 * adds to loss_per_scene the combined loss summed over the covered tiles'
 * pixels (times loss_scale). abc: float [cls_ssim_buffer_size(info)] scratch
 * (nine planes per view). */
size_t cls_ssim_buffer_size(const ClsBatchInfo* info); /* float entries */
int cls_ssim_loss(const ClsView* views_dev, const ClsBatchInfo* info, const int32_t* tiles,
                  const int32_t* n_tiles_dev, const uint8_t* tile_active, const float* image,
                  const float* target, float lambda, float* abc, float* dL_dimage,
                  float* loss_per_scene, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Sphere region and pruning (Sec. 3.3 "Sphere Pruning"; Supp. "Identifying
 * Changed Gaussians": a sphere per cluster of O^t's centres, at the cluster
 * mean, radius 1.1 x the 98th quantile of the members' distances to it; Supp.
 * "3DGS Optimization in Changed Regions": every 15 iterations each Gaussian of
 * O^t whose centre is in no sphere is removed).
 * The clusters are K-Means ones (the paper uses HDBSCAN): farthest-point
 * initial centres (first point of the list, then repeatedly the point
 * farthest from its nearest chosen centre, ties to the lowest position), then
 * `iters` Lloyd iterations (nearest centre, ties to the lowest cluster; an
 * empty cluster keeps its centre). Distances are the float32 sequence
 * ((dx*dx + dy*dy) + dz*dz) of rounded operations; cluster means are exact
 * (coordinates summed as int64 multiples of 2^-24, rounded half to even; mean
 * = float32(sum / count / 2^24) in float64), so the result does not depend on
 * thread order. The quantile is NumPy's linear estimator in float64 over the
 * members' float32 distances; radius = float32(1.1 q), -1 for an empty cluster.
 *   params, row_stride  parameter rows (mean at floats 0..2)
 *   idx [n_points]      device rows of the points (O^t's active_idx)
 *   spheres [k]         device output; labels [n_points], counts [k] optional
 *   workspace           cls_spheres_workspace_size(n_points) bytes
 * Pruning: for each of the n_active Gaussians of active_idx, inside iff its
 * float32 squared distance to some sphere's centre is <= radius * radius
 * (float32); an outside one gets opacity logit -inf (it never contributes to
 * a pixel again), active[g] = 0, its id in `removed` (optional, any order) and
 * n_removed_dev; active_idx is compacted in order and n_active_dev written.
 *   workspace  cls_prune_workspace_size(n_active) bytes */
#define CLS_MAX_SPHERES 10
typedef struct ClsSphere {
    float cx, cy, cz, radius;
} ClsSphere;
size_t cls_spheres_workspace_size(int32_t n_points);
int cls_fit_spheres(const float* params, int32_t row_stride, const int32_t* idx,
                    int32_t n_points, int32_t k, int32_t iters, ClsSphere* spheres,
                    int32_t* labels, int32_t* counts, void* workspace, size_t workspace_bytes,
                    cls_stream_t stream);
size_t cls_prune_workspace_size(int32_t n_active);
int cls_prune_outside_spheres(float* params, int32_t row_stride, uint8_t* active,
                              int32_t* active_idx, int32_t n_active, int32_t* n_active_dev,
                              const ClsSphere* spheres, int32_t k, int32_t* removed,
                              int32_t* n_removed_dev, void* workspace, size_t workspace_bytes,
                              cls_stream_t stream);

/* ------------------------------------------------------------------------
 * New-point sampling for appearing objects (Sec. 3.2 "Gaussian Sampling for
 * New Objects", New Point Sampling; Supp. Full-Scene and Region Point
 * Sampling). The caller runs the rounds: an empty point set O is replaced by
 * the vote-kept part of a uniform box sample (cls_points_bbox,
 * cls_box_sample, cls_lift_change_masks on the samples, cls_gather_points);
 * a non-empty one grows by the vote-kept part of n/5 mixture draws
 * (cls_fit_spheres for the K-Means clusters of O, cls_region_mixture,
 * cls_mixture_sample, vote, gather). Points are rows of 4 floats (x, y, z,
 * unused). Random numbers are inputs: u in [0, 1), z standard normal.
 *   cls_points_bbox: per-axis min and max of n parameter rows -> lohi[6]
 *     (min xyz, max xyz; device); scratch: 6 uint32 (device)
 *   cls_box_sample: points[i] = lo + u[i] (hi - lo) per axis (float32 ops)
 *   cls_gather_points: points[i] = src row idx[i] (or row i if idx is NULL),
 *     i < min(*n_dev, n_max) (or n_max if n_dev is NULL)
 *   cls_region_mixture: per cluster (labels/clusters/counts from
 *     cls_fit_spheres on the same points), |p_far - c| of the member of
 *     largest float32 squared distance (ties to the lowest position) ->
 *     absv [k][4]; scratch: CLS_MAX_SPHERES uint64 (device)
 *   cls_mixture_sample: per draw i, component j = first with
 *     floor(u[i] * n_points) < (members of clusters 0..j) (float64), point =
 *     c_j + sqrt(|v_j|) z[i] per axis (float32 ops)
 *   cls_init_point_gaussians: the base method's initialisation of a point
 *     cloud without colours: parameter rows (stride >= 16) with the point as
 *     mean, opacity 0.1, identity rotation, SH zero (grey), isotropic
 *     log-scale 0.5 log(d), d = ((d1 + d2) + d3) / 3 over the squared
 *     distances to the three nearest other points (fewer if fewer; float32),
 *     at least 1e-7 (written to mean_sq[n]). Brute force, O(n^2). */
int cls_points_bbox(const float* params, int32_t n, int32_t row_stride, float* lohi,
                    uint32_t* scratch, cls_stream_t stream);
int cls_box_sample(const float* lohi, const float* u, int32_t n, float* points,
                   cls_stream_t stream);
int cls_gather_points(const float* src, int32_t stride, const int32_t* idx,
                      const int32_t* n_dev, int32_t n_max, float* points, cls_stream_t stream);
int cls_region_mixture(const float* points, int32_t n, const int32_t* labels,
                       const ClsSphere* clusters, const int32_t* counts, int32_t k,
                       unsigned long long* scratch, float* absv, cls_stream_t stream);
int cls_mixture_sample(const ClsSphere* clusters, const float* absv, const int32_t* counts,
                       int32_t k, const float* u, const float* z, int32_t m, float* points,
                       cls_stream_t stream);
int cls_init_point_gaussians(const float* points, int32_t n, int32_t row_stride,
                             float* mean_sq, float* rows, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * History recovery and merging of updates (Supp. "History Recovery" and its
 * algorithm; "Batched Updates"): stable partitions of rows by a mask.
 *   cls_flag_map mode 0: map[dst] = the source row of dst when the rows with
 *     flags = 0 come first in order, then those with flags = 1 (the reorder of
 *     G^{t-1} before update t); mode 1: map[i] = i - ones_before(i) if
 *     flags[i] = 0, else ~ones_before(i) (recovery of G^{t-1}: unchanged rows
 *     from G^t's first #static rows, changed rows from the stored O^t).
 *     n_flagged_dev: device int32 count of set flags. workspace:
 *     cls_flag_map_workspace_size(n) bytes.
 *   cls_gather_rows: dst row i = a[map[i]] if map[i] >= 0 else b[~map[i]];
 *     rows of `stride` floats (a multiple of 4). */
size_t cls_flag_map_workspace_size(int32_t n);
int cls_flag_map(const uint8_t* flags, int32_t n, int32_t mode, int32_t* map,
                 int32_t* n_flagged_dev, void* workspace, size_t workspace_bytes,
                 cls_stream_t stream);
int cls_gather_rows(const float* a, const float* b, const int32_t* map, int32_t n_out,
                    int32_t stride, float* dst, cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Densification restricted to O^t (Supp. "History Recovery": duplication and
 * pruning only affect O^t; Supp. "Implementation Details": the base 3DGS
 * optimiser's adaptive density control with its defaults).
 *
 * cls_densify_accumulate: statistics of one scene's iteration. For every
 * active Gaussian g (rank a in active_idx) and every view j of
 * [first_view, first_view + n_views) with records[view.rec_base + g].radius
 * > 0: gx = grad2d[view.g2_base + a][0] * (W/2 * n_views), gy = [1] * (H/2 *
 * n_views) (the gradient of that view's own loss in NDC units; the batch loss
 * is the mean over the views), accum[g] += sqrt(gx^2 + gy^2), denom[g] += 1,
 * max_radius[g] = max(max_radius[g], radius); all float32, round to nearest,
 * views in order. accum, denom, max_radius: [n] device floats, caller-zeroed
 * at the start of a densification interval.
 *
 * cls_densify: one densification step of one scene. Per active Gaussian
 * (float32 comparisons with the rule's thresholds): avg = accum / denom (0 if
 * denom = 0); selected if avg >= grad_threshold; a selected Gaussian whose
 * largest log-scale is <= clone_log_scale is cloned, otherwise split into two
 * children mu + R(q) (exp(log-scale) * z) with log-scales reduced by
 * log_shrink; a Gaussian is pruned if its opacity logit < min_logit or, with
 * `big`, its max_radius > 20 or its largest log-scale > big_log_scale (a
 * clone inherits the test; a child takes it on its own log-scales with
 * max_radius 0). Split and pruned originals are removed: opacity logit -inf,
 * active flag 0. New rows take ids n, n+1, ... in rank order (per Gaussian:
 * its clone, then its children), copy the source row except the changed
 * entries, get zero Adam moments and active flag 1.
 *   params, adam_m, adam_v: [capacity][row_stride]; capacity >= n + 2 n_active
 *   active: [capacity] uint8 flags; active_idx: O^t ascending (n_active)
 *   z: [n_active][2][3] standard normals (input; row a for rank a)
 *   new_src: [2 n_active] source id per new row
 *   active_idx_out: the next O^t (kept originals in order, then the new ids),
 *     capacity entries; must not alias active_idx
 *   counts_dev: device int32[3] = new rows, kept originals, next n_active
 *   removed: optional [n_active] uint8, 1 where the original was removed
 *   (active_idx, z and new_src may be NULL when n_active = 0)
 *   workspace: cls_densify_workspace_size(n_active) bytes
 * The accumulated statistics are read only (the caller resets them).
 *
 * cls_opacity_reset: the base optimiser's periodic opacity reset on O^t:
 * logit = min(logit, limit); Adam moments of that entry set to 0. */
typedef struct ClsDensifyRule {
    float grad_threshold;   /* mean NDC-gradient norm that selects a Gaussian */
    float clone_log_scale;  /* log(percent_dense * extent) */
    float min_logit;        /* logit(min opacity) */
    float big_log_scale;    /* log(0.1 * extent) */
    float log_shrink;       /* log(0.8 * 2) */
    int32_t big;            /* apply the size rules (after the first opacity reset) */
} ClsDensifyRule;

int cls_densify_accumulate(const ClsView* views_dev, int32_t first_view, int32_t n_views,
                           const ClsProjected* records, const float* grad2d,
                           const int32_t* active_idx, int32_t n_active, float* accum,
                           float* denom, float* max_radius, cls_stream_t stream);
size_t cls_densify_workspace_size(int32_t n_active);
int cls_densify(float* params, float* adam_m, float* adam_v, int32_t row_stride, int32_t n,
                int64_t capacity, uint8_t* active, const int32_t* active_idx, int32_t n_active,
                const float* accum, const float* denom, const float* max_radius,
                const ClsDensifyRule* rule, const float* z, int32_t* new_src,
                int32_t* active_idx_out, int32_t* counts_dev, uint8_t* removed, void* workspace,
                size_t workspace_bytes, cls_stream_t stream);
int cls_opacity_reset(float* params, float* adam_m, float* adam_v, int32_t row_stride,
                      const int32_t* active_idx, int32_t n_active, float limit,
                      cls_stream_t stream);

/* ------------------------------------------------------------------------
 * Masked Adam on the active set (Supp. "3DGS Optimization in Changed
 * Regions"): increments the adam_step t of each scene with active Gaussians
 * (a scene with none is left untouched), then for every active row
 * and every float of it: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). Rows of
 * Gaussians outside O^t (params, adam_m, adam_v) are never touched.
 *   grads   [total_grad_rows][row_stride] as written by cls_render_backward
 *   workspace: cls_adam_workspace_size(n_scenes) bytes */
size_t cls_adam_workspace_size(int32_t n_scenes);
int cls_adam_step_active(const ClsScene* scenes_dev, const ClsBatchInfo* info, const float* grads,
                         float lr, float beta1, float beta2, float eps, void* workspace,
                         size_t workspace_bytes, cls_stream_t stream);

/* Library version string. */
const char* cls_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CLSPLAT_H */
