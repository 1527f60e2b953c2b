// Host-side batch planning of libclsplat: row strides, derived view/scene
// offsets and batch totals. Pure host code (no CUDA calls).
#include <string.h>

#include "common.cuh"

extern "C" int32_t cls_row_stride(int32_t sh_degree) {
    switch (sh_degree) {
        case 0: return 16;
        case 1: return 24;
        case 2: return 40;
        case 3: return 64;
        default: return -1;
    }
}

extern "C" const char* cls_version(void) { return "clsplat 1.0 (sm_103a)"; }

extern "C" int cls_batch_prepare(ClsScene* scenes, int32_t n_scenes, ClsView* views,
                                 int32_t n_views, ClsBatchInfo* info) {
    if (!scenes || !views || !info || n_scenes <= 0 || n_views <= 0) return CLS_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->n_scenes = n_scenes;
    info->n_views = n_views;
    int64_t grad_rows = 0;
    for (int s = 0; s < n_scenes; ++s) {
        ClsScene& sc = scenes[s];
        if (sc.n < 0 || sc.n_active < 0 || sc.n_active > sc.n) return CLS_ERR_INVALID_ARG;
        if (cls_row_stride(sc.sh_degree) < 0 || sc.row_stride < cls_row_stride(sc.sh_degree) ||
            sc.row_stride % 4 != 0)
            return CLS_ERR_INVALID_ARG;
        if (sc.n_views <= 0 || sc.first_view < 0 || sc.first_view + sc.n_views > n_views)
            return CLS_ERR_INVALID_ARG;
        sc.grad_base = grad_rows;
        grad_rows += sc.n_active;
        if (sc.n > info->max_n) info->max_n = sc.n;
        if (sc.n_active > info->max_active) info->max_active = sc.n_active;
        if (sc.row_stride > info->max_row_stride) info->max_row_stride = sc.row_stride;
    }
    int64_t tiles = 0, sat = 0, recs = 0, pix = 0, g2 = 0;
    for (int j = 0; j < n_views; ++j) {
        ClsView& v = views[j];
        if (v.scene < 0 || v.scene >= n_scenes) return CLS_ERR_INVALID_ARG;
        const ClsScene& sc = scenes[v.scene];
        if (j < sc.first_view || j >= sc.first_view + sc.n_views) return CLS_ERR_INVALID_ARG;
        if (v.cam.width <= 0 || v.cam.height <= 0 || !(v.cam.fx > 0.0f) || !(v.cam.fy > 0.0f))
            return CLS_ERR_INVALID_ARG;
        v.tiles_x = (v.cam.width + CLS_TILE - 1) / CLS_TILE;
        v.tiles_y = (v.cam.height + CLS_TILE - 1) / CLS_TILE;
        if (tiles > INT32_MAX - (int64_t)v.tiles_x * v.tiles_y) return CLS_ERR_INVALID_ARG;
        v.tile_base = (int32_t)tiles;
        v.sat_base = (int32_t)sat;
        v.rec_base = recs;
        v.pix_base = pix;
        v.g2_base = g2;
        v.loss_scale = (float)(1.0 / (3.0 * (double)v.cam.width * (double)v.cam.height *
                                      (double)sc.n_views));
        tiles += (int64_t)v.tiles_x * v.tiles_y;
        if ((int64_t)v.tiles_x * v.tiles_y > info->max_view_tiles)
            info->max_view_tiles = (int64_t)v.tiles_x * v.tiles_y;
        sat += (int64_t)(v.tiles_x + 1) * (v.tiles_y + 1);
        recs += sc.n;
        pix += (int64_t)v.cam.width * v.cam.height;
        g2 += sc.n_active;
    }
    if (recs > INT32_MAX || tiles >= (int64_t)1 << 31) return CLS_ERR_INVALID_ARG;
    info->total_tiles = tiles;
    info->total_sat = sat;
    info->total_records = recs;
    info->total_pixels = pix;
    info->total_g2 = g2;
    info->total_grad_rows = grad_rows;
    int bits = 1;
    while (((int64_t)1 << bits) < tiles) ++bits;
    info->key_bits = 32 + bits;
    return CLS_OK;
}
