"""Densification restricted to O^t (Supp. "History Recovery": duplication and
pruning only affect O^t; Supp. "Implementation Details": the base 3DGS
optimiser's adaptive density control with its defaults).

Per iteration (before `until`): the statistics of every active Gaussian are
accumulated from the renderer's 2D gradients (cls_densify_accumulate). Every
`interval` iterations after `start`: one densification step (clone, split,
prune; cls_densify) grows the scene in place, the statistics restart at zero
and the optimiser skips that iteration (the base optimiser's new parameters
have no gradient yet). Every `reset_every` iterations: the opacity reset of
O^t (cls_opacity_reset). The split draws its standard normals from
`draws(step, n_active)` (e.g. `synthetic.densify_draws(seed)`).
"""
from __future__ import annotations

import math
from typing import Callable, Optional, Sequence

import numpy as np
import torch

from . import _abi as abi
from .update import SceneState, _ptr

GRAD_THRESHOLD = 0.0002
PERCENT_DENSE = 0.01
MIN_OPACITY = 0.005
SPLIT_SHRINK = 0.8 * 2
BIG_WORLD = 0.1
RESET_OPACITY = 0.01


def camera_extent(cams: Sequence) -> float:
    """The base optimiser's scene extent: 1.1 x the largest distance of a
    camera centre from their mean."""
    pos = np.array([np.asarray(c["pos"], np.float64) for c in cams])
    centre = pos.mean(axis=0)
    return 1.1 * float(np.linalg.norm(pos - centre, axis=1).max())


def rule(extent: float, big: bool, grad_threshold: float = GRAD_THRESHOLD
         ) -> abi.ClsDensifyRule:
    """Thresholds computed once in float64 and rounded to float32 (the kernel
    compares float32 quantities with them)."""
    f = lambda x: float(np.float32(x))
    return abi.ClsDensifyRule(
        f(grad_threshold), f(math.log(PERCENT_DENSE * extent)),
        f(math.log(MIN_OPACITY / (1.0 - MIN_OPACITY))), f(math.log(BIG_WORLD * extent)),
        f(math.log(SPLIT_SHRINK)), 1 if big else 0)


def reset_limit() -> float:
    return float(np.float32(math.log(RESET_OPACITY / (1.0 - RESET_OPACITY))))


def _stream():
    return torch.cuda.current_stream().cuda_stream


def reserve_rows(state: SceneState, rows: int) -> None:
    """Make the storage behind the scene's rows (params, moments, active
    flags) hold at least `rows` rows; the logical tensors stay views of the
    first n. Grows by at least a quarter so repeated growth stays cheap."""
    def cap_of(t, width):
        return t.untyped_storage().nbytes() // (t.element_size() * width)
    st = state
    if (st.params.storage_offset() == 0 and cap_of(st.params, st.stride) >= rows
            and cap_of(st.adam_m, st.stride) >= rows and cap_of(st.adam_v, st.stride) >= rows
            and st.active.storage_offset() == 0 and cap_of(st.active, 1) >= rows):
        return
    cap = max(rows, st.n + st.n // 4 + 1024)
    dev = st.params.device

    def grow(t, shape, dtype):
        buf = torch.zeros(shape, dtype=dtype, device=dev)
        buf[: st.n].copy_(t[: st.n])
        return buf
    st.params = grow(st.params, (cap, st.stride), torch.float32)[: st.n]
    st.adam_m = grow(st.adam_m, (cap, st.stride), torch.float32)[: st.n]
    st.adam_v = grow(st.adam_v, (cap, st.stride), torch.float32)[: st.n]
    st.active = grow(st.active, (cap,), torch.uint8)[: st.n]


class Densifier:
    """Adaptive density control of one resident scene's O^t."""

    def __init__(self, state: SceneState, cams: Sequence, draws: Callable,
                 interval: int = 100, start: int = 500, until: int = 15000,
                 reset_every: int = 3000, extent: Optional[float] = None,
                 grad_threshold: float = GRAD_THRESHOLD):
        self.state = state
        self.n_views = len(cams)
        self.extent = float(extent) if extent is not None else camera_extent(cams)
        self.draws = draws
        self.interval, self.start, self.until = int(interval), int(start), int(until)
        self.reset_every = int(reset_every)
        self.grad_threshold = float(grad_threshold)
        self.steps = 0
        self.added = self.removed = 0
        self._alloc_stats(state.n)

    def _alloc_stats(self, n: int):
        dev = self.state.params.device
        self.accum = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)
        self.denom = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)
        self.max_radius = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)

    def accumulate(self, batch, scene: int = 0) -> None:
        """Add this iteration's statistics (after the backward pass, with the
        active list the pass used)."""
        st = self.state
        sc = batch.scene_tab[scene]
        if sc.n_active <= 0:
            return
        if self.accum.numel() < st.n:  # the scene grew outside densification
            self._alloc_stats(st.n)
        abi.check(abi.cls_densify_accumulate(
            _ptr(batch.views_dev), sc.first_view, sc.n_views, _ptr(batch.records),
            _ptr(batch.grad2d), _ptr(st.active_idx), sc.n_active, _ptr(self.accum),
            _ptr(self.denom), _ptr(self.max_radius), _stream()), "cls_densify_accumulate")

    def due(self, iteration: int) -> bool:
        return (iteration < self.until and iteration > self.start
                and iteration % self.interval == 0)

    def reset_due(self, iteration: int) -> bool:
        return iteration < self.until and iteration % self.reset_every == 0

    def densify(self, iteration: int, want: bool = False):
        """One densification step; returns (new rows, removed originals) and,
        with `want`, the source ids of the new rows and the removed flags per
        rank of the old active list."""
        st = self.state
        A, n = st.n_active, st.n
        dev = st.params.device
        big = iteration > self.reset_every
        reserve_rows(st, n + 2 * A)
        cap = st.params.untyped_storage().nbytes() // (4 * st.stride)
        z = torch.from_numpy(np.ascontiguousarray(self.draws(self.steps, A), np.float32))
        z = z.pin_memory().to(dev, non_blocking=True) if A else torch.zeros(1, device=dev)
        new_src = torch.empty(max(2 * A, 1), dtype=torch.int32, device=dev)
        active_out = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        counts = torch.zeros(3, dtype=torch.int32, device=dev)
        removed = torch.empty(max(A, 1), dtype=torch.uint8, device=dev) if want else None
        ws = torch.empty(max(abi.cls_densify_workspace_size(A), 256), dtype=torch.uint8,
                         device=dev)
        r = rule(self.extent, big, self.grad_threshold)
        abi.check(abi.cls_densify(
            _ptr(st.params), _ptr(st.adam_m), _ptr(st.adam_v), st.stride, n, cap,
            _ptr(st.active), _ptr(st.active_idx), A, _ptr(self.accum), _ptr(self.denom),
            _ptr(self.max_radius), r, _ptr(z), _ptr(new_src), _ptr(active_out), _ptr(counts),
            _ptr(removed), _ptr(ws), ws.numel(), _stream()), "cls_densify")
        n_new, n_keep, n_act = (int(x) for x in counts.cpu().tolist())
        self.steps += 1
        full = lambda t, rows: t.as_strided((rows,) + tuple(t.shape[1:]), t.stride())
        st.params = full(st.params, n + n_new)
        st.adam_m = full(st.adam_m, n + n_new)
        st.adam_v = full(st.adam_v, n + n_new)
        st.active = full(st.active, n + n_new)
        st.active_idx = active_out
        st.n, st.n_active = n + n_new, n_act
        st.epoch += 1
        self.added += n_new
        self.removed += A - n_keep
        self._alloc_stats(st.n)
        if want:
            return n_new, A - n_keep, new_src[:n_new].cpu().numpy(), removed[:A].cpu().numpy()
        return n_new, A - n_keep

    def reset_opacity(self) -> None:
        st = self.state
        abi.check(abi.cls_opacity_reset(
            _ptr(st.params), _ptr(st.adam_m), _ptr(st.adam_v), st.stride, _ptr(st.active_idx),
            st.n_active, reset_limit(), _stream()), "cls_opacity_reset")
