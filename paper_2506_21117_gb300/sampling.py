"""New-point sampling for appearing objects (Sec. 3.2 "Gaussian Sampling for
New Objects", New Point Sampling; Supp. Full-Scene and Region Point
Sampling), and adding the sampled points to a resident scene as Gaussians of
O^t with the base method's point-cloud initialisation.

The rounds run on the host, as the algorithm is written (each needs to know
how many points the vote kept); every step of a round is a libclsplat kernel:
box sample or K-Means mixture draw, majority vote, compaction. The random
numbers are inputs: `draws(round, kind, shape)` returns float32 arrays (kind
"box": uniform n x 3; "comp": uniform n/5; "normal": standard normal
n/5 x 3), e.g. `synthetic.sampling_draws(seed)`.
"""
from __future__ import annotations

from typing import Callable, Dict

import numpy as np
import torch

from . import _abi as abi
from .update import SceneState, _bytes, _ptr, _views_for

MAX_ROUNDS = 64
REGION_K = 10
KMEANS_ITERS = 16


def _stream():
    return torch.cuda.current_stream().cuda_stream


def sample_points(state: SceneState, cams, masks, n: int, draws: Callable,
                  device="cuda") -> Dict[str, object]:
    """The New Point Sampling loop on O = the centres of the scene's active
    Gaussians. Returns {"points": [m][4] device tensor (the final O),
    "new": the sampled rows of it, "rounds": int}."""
    views, pix = _views_for(cams)
    views_dev = _bytes(views).to(device)
    if isinstance(masks, torch.Tensor):
        masks_dev = masks.to(device)
    else:
        masks_dev = torch.from_numpy(np.concatenate(
            [np.ascontiguousarray(m, np.uint8).reshape(-1) for m in masks])).to(device)
    if masks_dev.numel() != pix:
        raise ValueError("mask size does not match the cameras")
    A = state.n_active
    cap = max(A, n) + n // 5 + 1
    O = torch.zeros((cap, 4), dtype=torch.float32, device=device)
    s = _stream()
    abi.check(abi.cls_gather_points(_ptr(state.params), state.stride, _ptr(state.active_idx),
                                    None, A, _ptr(O), s), "cls_gather_points")
    lohi = torch.empty(6, dtype=torch.float32, device=device)
    scratch = torch.empty(64, dtype=torch.int64, device=device)
    abi.check(abi.cls_points_bbox(_ptr(state.params), state.n, state.stride, _ptr(lohi),
                                  _ptr(scratch), s), "cls_points_bbox")
    size, fresh, rounds = A, False, 0

    def vote_into(S: torch.Tensor, m: int, at: int) -> int:
        flags = torch.empty(max(m, 1), dtype=torch.uint8, device=device)
        idx = torch.empty(max(m, 1), dtype=torch.int32, device=device)
        n_keep = torch.zeros(1, dtype=torch.int32, device=device)
        ws = torch.empty(max(abi.cls_lift_workspace_size(m), 256), dtype=torch.uint8,
                         device=device)
        abi.check(abi.cls_lift_change_masks(
            _ptr(S), m, 4, _ptr(views_dev), 0, len(cams), _ptr(masks_dev), 0, _ptr(flags),
            _ptr(idx), _ptr(n_keep), None, _ptr(ws), ws.numel(), s), "cls_lift_change_masks")
        kept = int(n_keep.item())
        abi.check(abi.cls_gather_points(_ptr(S), 4, _ptr(idx), None, kept, _ptr(O[at:]), s),
                  "cls_gather_points")
        return kept

    while size < n and rounds < MAX_ROUNDS:
        if size == 0:
            u = torch.from_numpy(np.ascontiguousarray(draws(rounds, "box", (n, 3)))).to(device)
            S = torch.empty((n, 4), dtype=torch.float32, device=device)
            abi.check(abi.cls_box_sample(_ptr(lohi), _ptr(u), n, _ptr(S), s), "cls_box_sample")
            size = vote_into(S, n, 0)
            fresh = True
        else:
            m = n // 5
            k = min(REGION_K, size)
            idx = torch.arange(size, dtype=torch.int32, device=device)
            clusters = torch.empty(k * 4, dtype=torch.float32, device=device)
            labels = torch.empty(size, dtype=torch.int32, device=device)
            counts = torch.empty(k, dtype=torch.int32, device=device)
            ws = torch.empty(abi.cls_spheres_workspace_size(size), dtype=torch.uint8,
                             device=device)
            abi.check(abi.cls_fit_spheres(_ptr(O), 4, _ptr(idx), size, k, KMEANS_ITERS,
                                          _ptr(clusters), _ptr(labels), _ptr(counts), _ptr(ws),
                                          ws.numel(), s), "cls_fit_spheres")
            absv = torch.empty(k * 4, dtype=torch.float32, device=device)
            abi.check(abi.cls_region_mixture(_ptr(O), size, _ptr(labels), _ptr(clusters),
                                             _ptr(counts), k, _ptr(scratch), _ptr(absv), s),
                      "cls_region_mixture")
            u = torch.from_numpy(np.ascontiguousarray(draws(rounds, "comp", (m,)))).to(device)
            z = torch.from_numpy(np.ascontiguousarray(draws(rounds, "normal", (m, 3)))).to(device)
            S = torch.empty((max(m, 1), 4), dtype=torch.float32, device=device)
            abi.check(abi.cls_mixture_sample(_ptr(clusters), _ptr(absv), _ptr(counts), k,
                                             _ptr(u), _ptr(z), m, _ptr(S), s),
                      "cls_mixture_sample")
            size += vote_into(S, m, size) if m > 0 else 0
        rounds += 1
    points = O[:size]
    return {"points": points, "new": points if fresh else O[A:size], "rounds": rounds}


def init_gaussians(points: torch.Tensor, sh_degree: int) -> torch.Tensor:
    """Parameter rows [m][row_stride] of new points (rows of 4 floats, as
    `sample_points` returns them): the base method's initialisation of a
    point cloud without colours."""
    if points.dim() != 2 or points.shape[1] != 4:
        raise ValueError("points are rows of 4 floats (x, y, z, unused)")
    m = int(points.shape[0])
    stride = abi.cls_row_stride(sh_degree)
    rows = torch.empty((max(m, 1), stride), dtype=torch.float32, device=points.device)
    mean_sq = torch.empty(max(m, 1), dtype=torch.float32, device=points.device)
    abi.check(abi.cls_init_point_gaussians(_ptr(points.contiguous()), m, stride, _ptr(mean_sq),
                                           _ptr(rows), _stream()), "cls_init_point_gaussians")
    return rows[:m]


def add_to_scene(state: SceneState, rows: torch.Tensor) -> None:
    """Append new Gaussians (parameter rows) to a resident scene as members of
    O^t with fresh Adam moments; the active list keeps ascending order."""
    m = int(rows.shape[0])
    if m == 0:
        return
    dev = state.params.device
    n0, A = state.n, state.n_active
    state.params = torch.cat([state.params, rows.to(dev)])
    state.adam_m = torch.cat([state.adam_m, torch.zeros_like(rows)])
    state.adam_v = torch.cat([state.adam_v, torch.zeros_like(rows)])
    state.active = torch.cat([state.active, torch.ones(m, dtype=torch.uint8, device=dev)])
    state.active_idx = torch.cat([state.active_idx[:A],
                                  torch.arange(n0, n0 + m, dtype=torch.int32, device=dev)])
    state.n = n0 + m
    state.n_active = A + m
    state.epoch += 1
