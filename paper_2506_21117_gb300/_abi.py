"""ctypes binding of libclsplat's C ABI (include/clsplat.h).

Argument marshalling only: every function here forwards to the CUDA library
with the same name. Device buffers are passed as integer addresses (for
example `tensor.data_ptr()`), streams as CUDA stream handles. Loading fails
loudly if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libclsplat.so")

CLS_OK, CLS_ERR_INVALID_ARG, CLS_ERR_CAPACITY, CLS_ERR_CUDA, CLS_ERR_TIMEOUT, \
    CLS_ERR_INTERNAL = range(6)
STATUS_NAMES = {0: "CLS_OK", 1: "CLS_ERR_INVALID_ARG", 2: "CLS_ERR_CAPACITY",
                3: "CLS_ERR_CUDA", 4: "CLS_ERR_TIMEOUT", 5: "CLS_ERR_INTERNAL"}
TILE = 16
G2_STRIDE = 12
CLS_SORT_SPIN_LIMIT = 1 << 22


class ClsCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("pos", C.c_float * 3),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("znear", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class ClsScene(C.Structure):
    _fields_ = [("params", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p),
                ("active_idx", C.c_void_p), ("adam_step", C.c_void_p),
                ("n", C.c_int32), ("row_stride", C.c_int32), ("sh_degree", C.c_int32),
                ("n_active", C.c_int32), ("first_view", C.c_int32), ("n_views", C.c_int32),
                ("grad_base", C.c_int64)]


class ClsView(C.Structure):
    _fields_ = [("cam", ClsCamera), ("scene", C.c_int32), ("tiles_x", C.c_int32),
                ("tiles_y", C.c_int32), ("tile_base", C.c_int32), ("sat_base", C.c_int32),
                ("pad0", C.c_int32), ("rec_base", C.c_int64), ("pix_base", C.c_int64),
                ("g2_base", C.c_int64), ("loss_scale", C.c_float), ("pad1", C.c_int32)]


class ClsBatchInfo(C.Structure):
    _fields_ = [("n_scenes", C.c_int32), ("n_views", C.c_int32), ("max_n", C.c_int32),
                ("max_active", C.c_int32), ("max_row_stride", C.c_int32),
                ("key_bits", C.c_int32), ("total_tiles", C.c_int64), ("total_sat", C.c_int64),
                ("total_records", C.c_int64), ("total_pixels", C.c_int64),
                ("total_g2", C.c_int64), ("total_grad_rows", C.c_int64),
                ("max_view_tiles", C.c_int64)]


class ClsProjected(C.Structure):
    _fields_ = [("u", C.c_float), ("v", C.c_float), ("conic_a", C.c_float),
                ("conic_b", C.c_float), ("conic_c", C.c_float), ("opacity", C.c_float),
                ("r", C.c_float), ("g", C.c_float), ("b", C.c_float), ("g2_slot", C.c_int32),
                ("z", C.c_float), ("radius", C.c_int32)]


class ClsTileCache(C.Structure):
    _fields_ = [("zb", C.c_uint32), ("n_prefix", C.c_uint32), ("zmin_active", C.c_uint32),
                ("last_active", C.c_int32)]


PREFIX_UNKNOWN = 0xFFFFFFFF
MAX_SPHERES = 10


class ClsSphere(C.Structure):
    _fields_ = [("cx", C.c_float), ("cy", C.c_float), ("cz", C.c_float), ("radius", C.c_float)]


class ClsDensifyRule(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("clone_log_scale", C.c_float),
                ("min_logit", C.c_float), ("big_log_scale", C.c_float),
                ("log_shrink", C.c_float), ("big", C.c_int32)]


TILE_CACHE_BYTES = 16

assert C.sizeof(ClsCamera) == 88 and C.sizeof(ClsScene) == 72
assert C.sizeof(ClsTileCache) == TILE_CACHE_BYTES and C.sizeof(ClsSphere) == 16
assert C.sizeof(ClsView) == 144 and C.sizeof(ClsProjected) == 48

P = C.c_void_p
I32, I64, SZ, F32 = C.c_int32, C.c_int64, C.c_size_t, C.c_float

# name -> (restype, argtypes); the same order as include/clsplat.h
SIGNATURES = {
    "cls_row_stride": (I32, [I32]),
    "cls_version": (C.c_char_p, []),
    "cls_batch_prepare": (C.c_int, [P, I32, P, I32, P]),
    "cls_lift_workspace_size": (SZ, [I32]),
    "cls_lift_change_masks": (C.c_int, [P, I32, I32, P, I32, I32, P, I32, P, P, P, P, P, SZ, P]),
    "cls_lift_change_masks_static": (C.c_int, [P, I32, I32, P, I32, I32, P, I32, P, P, P, P, P]),
    "cls_project_workspace_size": (SZ, [P]),
    "cls_bin_offsets_size": (SZ, [P]),
    "cls_project_and_bin": (C.c_int, [P, P, P, I32, I32, P, P, P, P, P, P, I64, P, P, P, P, P,
                                      I32, I32, P, P, SZ, P]),
    "cls_complete_truncated": (C.c_int, [P, P, P, P, I64, P, P, I64, P, P, SZ, P]),
    "cls_sort_tiles_workspace_size": (SZ, [I64, I32]),
    "cls_sort_tiles": (C.c_int, [P, P, P, P, P, I64, I64, I32, P, P, P, I64, P, P, P, SZ, P]),
    "cls_sort_workspace_size": (SZ, [I64, I32]),
    "cls_sort_keys": (C.c_int, [P, P, P, P, P, I64, I32, P, I64, P, P, SZ, P]),
    "cls_sort_keys_bounded": (C.c_int, [P, P, P, P, P, I64, I32, P, I64, P, P, SZ, I64, P]),
    "cls_render_forward": (C.c_int, [P, P, P, P, I32, P, P, P, P, P, P, P, P, P, P, I64, P, P,
                                     P, P, P, I32, P, P, P, P, P, P, P]),
    "cls_render_backward": (C.c_int, [P, P, P, P, P, I32, P, P, P, P, P, P, P, P, P, P, P, P]),
    "cls_adam_workspace_size": (SZ, [I32]),
    "cls_adam_step_active": (C.c_int, [P, P, P, F32, F32, F32, F32, P, SZ, P]),
    "cls_ssim_buffer_size": (SZ, [P]),
    "cls_ssim_loss": (C.c_int, [P, P, P, P, P, P, P, F32, P, P, P, P]),
    "cls_flag_map_workspace_size": (SZ, [I32]),
    "cls_flag_map": (C.c_int, [P, I32, I32, P, P, P, SZ, P]),
    "cls_gather_rows": (C.c_int, [P, P, P, I32, I32, P, P]),
    "cls_points_bbox": (C.c_int, [P, I32, I32, P, P, P]),
    "cls_box_sample": (C.c_int, [P, P, I32, P, P]),
    "cls_gather_points": (C.c_int, [P, I32, P, P, I32, P, P]),
    "cls_region_mixture": (C.c_int, [P, I32, P, P, P, I32, P, P, P]),
    "cls_mixture_sample": (C.c_int, [P, P, P, I32, P, P, I32, P, P]),
    "cls_init_point_gaussians": (C.c_int, [P, I32, I32, P, P, P]),
    "cls_spheres_workspace_size": (SZ, [I32]),
    "cls_fit_spheres": (C.c_int, [P, I32, P, I32, I32, I32, P, P, P, P, SZ, P]),
    "cls_prune_workspace_size": (SZ, [I32]),
    "cls_prune_outside_spheres": (C.c_int, [P, I32, P, P, I32, P, P, I32, P, P, P, SZ, P]),
    "cls_densify_accumulate": (C.c_int, [P, I32, I32, P, P, P, I32, P, P, P, P]),
    "cls_densify_workspace_size": (SZ, [I32]),
    "cls_densify": (C.c_int, [P, P, P, I32, I32, I64, P, P, I32, P, P, P, P, P, P, P, P, P, P,
                              SZ, P]),
    "cls_opacity_reset": (C.c_int, [P, P, P, I32, P, I32, F32, P]),
}

_lib = None


def library_path() -> str:
    return LIB_PATH


def load() -> C.CDLL:
    """Load libclsplat.so (build it first with paper_2506_21117_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libclsplat.so is not built ({LIB_PATH}); run "
                "`python -m paper_2506_21117_gb300.build` (needs nvcc)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class ClsError(RuntimeError):
    pass


def check(code: int, what: str) -> None:
    if code != CLS_OK:
        raise ClsError(f"{what} returned {STATUS_NAMES.get(code, code)}")


def _ref(x):
    return None if x is None else C.byref(x)


def cls_row_stride(sh_degree: int) -> int:
    return load().cls_row_stride(sh_degree)


def cls_version() -> str:
    return load().cls_version().decode()


def cls_batch_prepare(scenes, views, info) -> int:
    return load().cls_batch_prepare(C.cast(scenes, P), len(scenes), C.cast(views, P),
                                    len(views), C.byref(info))


def cls_lift_workspace_size(n: int) -> int:
    return load().cls_lift_workspace_size(n)


def cls_lift_change_masks(params, n, row_stride, views_dev, first_view, n_views, masks,
                          vote_mode, active_out, active_idx_out, n_active_out, votes_out,
                          workspace, workspace_bytes, stream) -> int:
    return load().cls_lift_change_masks(params, n, row_stride, views_dev, first_view, n_views,
                                        masks, vote_mode, active_out, active_idx_out,
                                        n_active_out, votes_out, workspace, workspace_bytes,
                                        stream)


LIFT_STATIC_MAX_N = 1 << 24


def cls_lift_change_masks_static(params, n, row_stride, views_dev, first_view, n_views, masks,
                                 vote_mode, active_out, active_idx_out, n_active_out, votes_out,
                                 stream) -> int:
    """Same as cls_lift_change_masks, with the library's fixed scratch array
    instead of a caller workspace (for callers that cannot allocate)."""
    return load().cls_lift_change_masks_static(params, n, row_stride, views_dev, first_view,
                                               n_views, masks, vote_mode, active_out,
                                               active_idx_out, n_active_out, votes_out, stream)


def cls_project_workspace_size(info) -> int:
    return load().cls_project_workspace_size(C.byref(info))


def cls_bin_offsets_size(info) -> int:
    return load().cls_bin_offsets_size(C.byref(info))


def cls_project_and_bin(scenes_dev, views_dev, info, project_mode, layout, records, tile_active,
                        active_tiles, n_active_tiles_dev, keys, vals, capacity, n_pairs_dev,
                        ranges, bin_offsets, bin_cut, tile_cache, prefix_mode, tile_ring,
                        status_dev, workspace, workspace_bytes, stream) -> int:
    return load().cls_project_and_bin(scenes_dev, views_dev, C.byref(info), project_mode, layout,
                                      records, tile_active, active_tiles, n_active_tiles_dev,
                                      keys, vals, capacity, n_pairs_dev, ranges, bin_offsets,
                                      bin_cut, tile_cache, prefix_mode, tile_ring, status_dev,
                                      workspace, workspace_bytes, stream)


def cls_complete_truncated(views_dev, info, records, keys, capacity, trunc, trunc_count,
                           trunc_cap, work_counter, workspace, workspace_bytes, stream) -> int:
    return load().cls_complete_truncated(views_dev, C.byref(info), records, keys, capacity, trunc,
                                         trunc_count, trunc_cap, work_counter, workspace,
                                         workspace_bytes, stream)


LAZY_MAX_BIN = 1024


def cls_sort_tiles_workspace_size(capacity, min_bin) -> int:
    return load().cls_sort_tiles_workspace_size(capacity, min_bin)


def cls_sort_tiles(keys, keys_alt, bin_offsets, active_tiles, n_active_tiles_dev, total_tiles,
                   capacity, min_bin, cut, trunc, trunc_count, trunc_cap, tile_cache,
                   work_counter, workspace, workspace_bytes, stream) -> int:
    return load().cls_sort_tiles(keys, keys_alt, bin_offsets, active_tiles, n_active_tiles_dev,
                                 total_tiles, capacity, min_bin, cut, trunc, trunc_count,
                                 trunc_cap, tile_cache, work_counter, workspace, workspace_bytes,
                                 stream)


def cls_sort_workspace_size(capacity, key_bits) -> int:
    return load().cls_sort_workspace_size(capacity, key_bits)


def cls_sort_keys(keys, vals, keys_alt, vals_alt, n_pairs_dev, capacity, key_bits, ranges,
                  n_tiles, status_dev, workspace, workspace_bytes, stream) -> int:
    return load().cls_sort_keys(keys, vals, keys_alt, vals_alt, n_pairs_dev, capacity, key_bits,
                                ranges, n_tiles, status_dev, workspace, workspace_bytes, stream)


def cls_sort_keys_bounded(keys, vals, keys_alt, vals_alt, n_pairs_dev, capacity, key_bits,
                          ranges, n_tiles, status_dev, workspace, workspace_bytes, spin_limit,
                          stream) -> int:
    return load().cls_sort_keys_bounded(keys, vals, keys_alt, vals_alt, n_pairs_dev, capacity,
                                        key_bits, ranges, n_tiles, status_dev, workspace,
                                        workspace_bytes, spin_limit, stream)


def cls_render_forward(views_dev, info, records, vals, vals_stride, ranges, active_tiles,
                       n_active_tiles_dev, lazy_keys, bin_offsets, list_ranks, cut_in, cut_out,
                       trunc, trunc_count, trunc_cap, tile_cache, prefix_state, prefix_last, bg,
                       target, loss_mode, image, T_final, n_contrib, dL_dimage, loss_per_scene,
                       work_counter, stream) -> int:
    bg3 = (C.c_float * 3)(*bg)
    return load().cls_render_forward(views_dev, C.byref(info), records, vals, vals_stride, ranges,
                                     active_tiles, n_active_tiles_dev, lazy_keys, bin_offsets,
                                     list_ranks, cut_in, cut_out, trunc, trunc_count, trunc_cap,
                                     tile_cache, prefix_state, prefix_last, bg3, target, loss_mode,
                                     image, T_final, n_contrib, dL_dimage, loss_per_scene,
                                     work_counter, stream)


def cls_render_backward(scenes_dev, views_dev, info, records, vals, vals_stride, ranges,
                        active_tiles, n_active_tiles_dev, tile_cache, prefix_state, image,
                        n_contrib, dL_dimage, grad2d, grads, work_counter, stream) -> int:
    return load().cls_render_backward(scenes_dev, views_dev, C.byref(info), records, vals,
                                      vals_stride, ranges, active_tiles, n_active_tiles_dev,
                                      tile_cache, prefix_state, image, n_contrib, dL_dimage,
                                      grad2d, grads, work_counter, stream)


def cls_adam_workspace_size(n_scenes) -> int:
    return load().cls_adam_workspace_size(n_scenes)


def cls_adam_step_active(scenes_dev, info, grads, lr, beta1, beta2, eps, workspace,
                         workspace_bytes, stream) -> int:
    return load().cls_adam_step_active(scenes_dev, C.byref(info), grads, lr, beta1, beta2, eps,
                                       workspace, workspace_bytes, stream)


def exported_symbols():
    """Names the header declares (for the export check)."""
    return list(SIGNATURES)


def cls_spheres_workspace_size(n_points) -> int:
    return load().cls_spheres_workspace_size(n_points)


def cls_fit_spheres(params, row_stride, idx, n_points, k, iters, spheres, labels, counts,
                    workspace, workspace_bytes, stream) -> int:
    return load().cls_fit_spheres(params, row_stride, idx, n_points, k, iters, spheres, labels,
                                  counts, workspace, workspace_bytes, stream)


def cls_prune_workspace_size(n_active) -> int:
    return load().cls_prune_workspace_size(n_active)


def cls_prune_outside_spheres(params, row_stride, active, active_idx, n_active, n_active_dev,
                              spheres, k, removed, n_removed_dev, workspace, workspace_bytes,
                              stream) -> int:
    return load().cls_prune_outside_spheres(params, row_stride, active, active_idx, n_active,
                                            n_active_dev, spheres, k, removed, n_removed_dev,
                                            workspace, workspace_bytes, stream)


def cls_ssim_buffer_size(info) -> int:
    return load().cls_ssim_buffer_size(C.byref(info))


def cls_ssim_loss(views_dev, info, tiles, n_tiles_dev, tile_active, image, target, lam, abc,
                  dL_dimage, loss_per_scene, stream) -> int:
    return load().cls_ssim_loss(views_dev, C.byref(info), tiles, n_tiles_dev, tile_active, image,
                                target, lam, abc, dL_dimage, loss_per_scene, stream)


def cls_points_bbox(params, n, row_stride, lohi, scratch, stream) -> int:
    return load().cls_points_bbox(params, n, row_stride, lohi, scratch, stream)


def cls_box_sample(lohi, u, n, points, stream) -> int:
    return load().cls_box_sample(lohi, u, n, points, stream)


def cls_gather_points(src, stride, idx, n_dev, n_max, points, stream) -> int:
    return load().cls_gather_points(src, stride, idx, n_dev, n_max, points, stream)


def cls_region_mixture(points, n, labels, clusters, counts, k, scratch, absv, stream) -> int:
    return load().cls_region_mixture(points, n, labels, clusters, counts, k, scratch, absv, stream)


def cls_mixture_sample(clusters, absv, counts, k, u, z, m, points, stream) -> int:
    return load().cls_mixture_sample(clusters, absv, counts, k, u, z, m, points, stream)


def cls_init_point_gaussians(points, n, row_stride, mean_sq, rows, stream) -> int:
    return load().cls_init_point_gaussians(points, n, row_stride, mean_sq, rows, stream)


def cls_flag_map_workspace_size(n) -> int:
    return load().cls_flag_map_workspace_size(n)


def cls_flag_map(flags, n, mode, map_, n_flagged_dev, workspace, workspace_bytes, stream) -> int:
    return load().cls_flag_map(flags, n, mode, map_, n_flagged_dev, workspace, workspace_bytes,
                               stream)


def cls_gather_rows(a, b, map_, n_out, stride, dst, stream) -> int:
    return load().cls_gather_rows(a, b, map_, n_out, stride, dst, stream)


def cls_densify_accumulate(views_dev, first_view, n_views, records, grad2d, active_idx,
                           n_active, accum, denom, max_radius, stream) -> int:
    return load().cls_densify_accumulate(views_dev, first_view, n_views, records, grad2d,
                                         active_idx, n_active, accum, denom, max_radius, stream)


def cls_densify_workspace_size(n_active) -> int:
    return load().cls_densify_workspace_size(n_active)


def cls_densify(params, adam_m, adam_v, row_stride, n, capacity, active, active_idx, n_active,
                accum, denom, max_radius, rule, z, new_src, active_idx_out, counts_dev, removed,
                workspace, workspace_bytes, stream) -> int:
    return load().cls_densify(params, adam_m, adam_v, row_stride, n, capacity, active,
                              active_idx, n_active, accum, denom, max_radius, _ref(rule), z,
                              new_src, active_idx_out, counts_dev, removed, workspace,
                              workspace_bytes, stream)


def cls_opacity_reset(params, adam_m, adam_v, row_stride, active_idx, n_active, limit,
                      stream) -> int:
    return load().cls_opacity_reset(params, adam_m, adam_v, row_stride, active_idx, n_active,
                                    limit, stream)
