"""Local scene update on the GPU: the CL-Splats local optimisation loop.

Sec. 3 of the paper: lift the 2D change masks of the new views to the active
set O^t (Sec. 3.2), then optimise only O^t with a rasterizer restricted to the
tiles O^t touches, static Gaussians rendered as frozen occluders (Sec. 3.3,
Supp. "Local Optimization Kernel", Supp. "3DGS Optimization in Changed
Regions"). Every step runs in libclsplat's CUDA kernels; this module owns the
device buffers (PyTorch tensors, used for memory and streams only) and the
order of the calls.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _abi as abi

LOSS_MODES = {"none": 0, "l1": 1, "l2": 2, "l1+ssim": 1}
SSIM_LAMBDA = 0.2  # weight of D-SSIM in the base 3DGS optimiser's loss


def sh_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


def pack_params(scene: Dict[str, np.ndarray], sh_degree: int) -> np.ndarray:
    """Scene dict -> float32 rows [n][row_stride] in the library's layout."""
    n = scene["means"].shape[0]
    stride = abi.cls_row_stride(sh_degree)
    k = sh_coeffs(sh_degree)
    rows = np.zeros((n, stride), np.float32)
    rows[:, 0:3] = scene["means"]
    rows[:, 3] = scene["opacity_logits"]
    rows[:, 4:7] = scene["log_scales"]
    rows[:, 8:12] = scene["quats"]
    rows[:, 12:12 + 3 * k] = np.asarray(scene["sh"], np.float32)[:, :k, :].reshape(n, 3 * k)
    return rows


def unpack_rows(rows: np.ndarray, sh_degree: int) -> Dict[str, np.ndarray]:
    """Rows (parameters or gradients) -> dict shaped like a scene."""
    k = sh_coeffs(sh_degree)
    n = rows.shape[0]
    return {"means": rows[:, 0:3], "opacity_logits": rows[:, 3], "log_scales": rows[:, 4:7],
            "quats": rows[:, 8:12], "sh": rows[:, 12:12 + 3 * k].reshape(n, k, 3)}


def make_camera(cam) -> abi.ClsCamera:
    c = abi.ClsCamera()
    R = np.asarray(cam["R"], np.float64).reshape(9)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(cam["t"][i])
        c.pos[i] = float(cam["pos"][i])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.znear = float(cam["znear"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _bytes(ctypes_array) -> torch.Tensor:
    raw = bytes(memoryview(ctypes_array).cast("B"))
    return torch.frombuffer(bytearray(raw), dtype=torch.uint8)


_COPY_STREAMS: Dict[object, object] = {}


def _copy_stream(device):
    """One side stream per device for host-to-device uploads."""
    key = torch.device(device)
    if key not in _COPY_STREAMS:
        _COPY_STREAMS[key] = torch.cuda.Stream(device=key)
    return _COPY_STREAMS[key]


def _upload(ctypes_array, device) -> torch.Tensor:
    """A host table on the device without waiting for the stream: through
    pinned memory, asynchronously on the current stream."""
    if torch.device(device).type != "cuda":
        return _bytes(ctypes_array).to(device)
    return _bytes(ctypes_array).pin_memory().to(device, non_blocking=True)


class SceneState:
    """One scene resident on the device: parameter rows, Adam moments and step."""

    def __init__(self, scene: Dict[str, np.ndarray], sh_degree: int, device="cuda"):
        self.sh_degree = sh_degree
        self.stride = abi.cls_row_stride(sh_degree)
        rows = pack_params(scene, sh_degree)
        self.n = rows.shape[0]
        self.params = torch.from_numpy(rows).to(device)
        self.adam_m = torch.zeros_like(self.params)
        self.adam_v = torch.zeros_like(self.params)
        self.adam_step = torch.zeros(1, dtype=torch.int32, device=device)
        self.active = torch.zeros(self.n, dtype=torch.uint8, device=device)
        self.active_idx = torch.zeros(max(self.n, 1), dtype=torch.int32, device=device)
        self.n_active = 0
        self.epoch = 0  # bumped whenever the active set changes

    def set_active(self, active: np.ndarray):
        a = np.asarray(active, bool)
        idx = np.flatnonzero(a).astype(np.int32)
        self.active.copy_(torch.from_numpy(a.astype(np.uint8)))
        self.active_idx[: idx.size].copy_(torch.from_numpy(idx))
        self.n_active = int(idx.size)
        self.epoch += 1

    def bytes_resident(self) -> int:
        return 3 * self.params.numel() * 4 + self.active.numel() * 5


class Batch:
    """Scene/view tables of one launch batch and every buffer the hot path uses."""

    def __init__(self, scenes: Sequence[SceneState], cams_per_scene: Sequence[Sequence],
                 device="cuda", layout: int = 1, lazy: bool = True, prefix_cache: bool = True,
                 ssim: bool = False):
        """layout 1: pairs bucketed by (tile, depth bin); with `lazy` the
        renderer sorts the depth bins it reaches (cls_sort_tiles only pre-sorts
        bins above CLS_LAZY_MAX_BIN keys), otherwise cls_sort_tiles sorts every
        bin. layout 0: flat (tile, depth) keys sorted by the global onesweep
        radix sort (cls_sort_keys). `prefix_cache` keeps each tile's static
        prefix across iterations (valid while the static rows of the scenes do
        not change, which masked Adam guarantees); off, every iteration
        rebuilds it. `ssim` adds the D-SSIM term to an L1 loss (the base
        optimiser's (1 - 0.2) L1 + 0.2 D-SSIM); the ring of tiles around the
        covered ones is then rendered too (the window needs it)."""
        self.device = device
        self.ssim = bool(ssim)
        self.layout = layout
        self.lazy = lazy and layout == 1
        self.prefix_mode = 1 if prefix_cache else 0
        self.scenes = list(scenes)
        S = len(scenes)
        views = []
        for s, cams in enumerate(cams_per_scene):
            for cam in cams:
                v = abi.ClsView()
                v.cam = make_camera(cam)
                v.scene = s
                views.append(v)
        self.n_views = len(views)
        self.scene_tab = (abi.ClsScene * S)()
        first = 0
        for s, st in enumerate(scenes):
            sc = self.scene_tab[s]
            sc.params, sc.adam_m, sc.adam_v = _ptr(st.params), _ptr(st.adam_m), _ptr(st.adam_v)
            sc.active_idx, sc.adam_step = _ptr(st.active_idx), _ptr(st.adam_step)
            sc.n, sc.row_stride, sc.sh_degree = st.n, st.stride, st.sh_degree
            sc.n_active = st.n_active
            sc.first_view, sc.n_views = first, len(cams_per_scene[s])
            first += len(cams_per_scene[s])
        self.view_tab = (abi.ClsView * self.n_views)(*views)
        self.info = abi.ClsBatchInfo()
        abi.check(abi.cls_batch_prepare(self.scene_tab, self.view_tab, self.info),
                  "cls_batch_prepare")
        self.scenes_dev = _upload(self.scene_tab, device)
        self.views_dev = _upload(self.view_tab, device)
        info = self.info
        dev = device
        # records: the first binning projects every Gaussian (reproject below)
        self.records = torch.empty(info.total_records * 12, dtype=torch.float32, device=dev)
        self.tile_active = torch.zeros(info.total_tiles, dtype=torch.uint8, device=dev)
        self.active_tiles = torch.zeros(info.total_tiles, dtype=torch.int32, device=dev)
        self.n_active_tiles = torch.zeros(1, dtype=torch.int32, device=dev)
        self.n_pairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.ranges = torch.zeros(info.total_tiles * 2, dtype=torch.int32, device=dev)
        self.T_final = torch.zeros(info.total_pixels, dtype=torch.float32, device=dev)
        self.n_contrib = torch.zeros(info.total_pixels, dtype=torch.int32, device=dev)
        self.image = torch.zeros(info.total_pixels * 3, dtype=torch.float32, device=dev)
        self.dL_dimage = torch.zeros(info.total_pixels * 3, dtype=torch.float32, device=dev)
        # the per-scene loss and the truncated-tile count share one buffer, so
        # one fill clears both before a forward pass
        self._fwd_acc = torch.zeros(S + 1, dtype=torch.int32, device=dev)
        self.loss = self._fwd_acc[:S].view(torch.float32)
        # grad2d: zeroed by the backward pass; grads: written for every active row
        self.grad2d = torch.empty(max(info.total_g2, 1) * abi.G2_STRIDE, dtype=torch.float32,
                                  device=dev)
        self.grads = torch.empty(max(info.total_grad_rows, 1) * info.max_row_stride,
                                 dtype=torch.float32, device=dev)
        self.counter = torch.zeros(4, dtype=torch.int32, device=dev)
        self.bin_offsets = torch.zeros(abi.cls_bin_offsets_size(info), dtype=torch.int32,
                                       device=dev)
        # speculative depth cut per tile (bucketed + lazy): every bin at first
        self.use_cut = self.lazy
        self.cut = torch.full((info.total_tiles,), 255, dtype=torch.uint8, device=dev)
        self.trunc = torch.zeros(3 * info.total_tiles, dtype=torch.int32, device=dev)
        self.trunc_count = self._fwd_acc[S:]
        # static-prefix cache: per tile (ClsTileCache), per pixel state after the prefix
        self.tile_cache = torch.empty(info.total_tiles * abi.TILE_CACHE_BYTES // 4,
                                      dtype=torch.int32, device=dev)
        # read only for tiles whose prefix a forward pass has written
        self.prefix_state = torch.empty(info.total_pixels * 4, dtype=torch.float32, device=dev)
        self.prefix_last = torch.empty(info.total_pixels, dtype=torch.int32, device=dev)
        self._epochs = [st.epoch for st in self.scenes]
        self.reset_prefix()
        self.reproject = True  # project every Gaussian on the next call (first, after pruning)
        self.abc = (torch.empty(abi.cls_ssim_buffer_size(info), dtype=torch.float32, device=dev)
                    if self.ssim else None)
        self.proj_ws = torch.zeros(abi.cls_project_workspace_size(info), dtype=torch.uint8,
                                   device=dev)
        self.adam_ws = torch.zeros(max(abi.cls_adam_workspace_size(S), 256), dtype=torch.uint8,
                                   device=dev)
        self.capacity = 0
        self.keys = self.vals = self.keys_alt = self.vals_alt = self.sort_ws = None
        self.target = None
        self.target_ready = None  # event of an asynchronous target upload
        self.counted = False  # the last binning only counted (capacity planning)

    # -- geometry of per-pixel buffers ---------------------------------------
    def view_slices(self):
        out = []
        for j in range(self.n_views):
            v = self.view_tab[j]
            out.append((int(v.pix_base), int(v.cam.height), int(v.cam.width)))
        return out

    def set_targets(self, targets: Sequence[np.ndarray]):
        t = torch.zeros(self.info.total_pixels * 3, dtype=torch.float32)
        for (base, H, W), img in zip(self.view_slices(), targets):
            t[3 * base: 3 * base + 3 * H * W] = torch.from_numpy(
                np.ascontiguousarray(img, np.float32).reshape(-1))
        self.target = t.to(self.device)

    def per_view(self, flat: torch.Tensor, channels: int) -> List[torch.Tensor]:
        out = []
        for base, H, W in self.view_slices():
            out.append(flat[channels * base: channels * (base + H * W)].view(channels, H, W)
                       if channels > 1 else flat[base: base + H * W].view(H, W))
        return out

    # -- the hot path -----------------------------------------------------------
    def stream(self):
        return torch.cuda.current_stream().cuda_stream

    def refresh_active(self):
        """Take the scenes' current active sets (after pruning shrank them):
        rebuild the batch tables; the next projection covers every Gaussian so
        no record keeps a gradient slot of a removed Gaussian."""
        for s, st in enumerate(self.scenes):
            self.scene_tab[s].n_active = st.n_active
        abi.check(abi.cls_batch_prepare(self.scene_tab, self.view_tab, self.info),
                  "cls_batch_prepare")
        self.scenes_dev.copy_(_bytes(self.scene_tab).pin_memory(), non_blocking=True)
        self.views_dev.copy_(_bytes(self.view_tab).pin_memory(), non_blocking=True)
        self.reproject = True
        self.counted = False

    def matches(self, scenes: Sequence[SceneState], cams_per_scene: Sequence[Sequence]) -> bool:
        """Whether this batch was built for these scenes (the same resident
        states, unchanged sizes) and these cameras (the same poses, intrinsics
        and sizes), so a new update of them can reuse its tables and buffers."""
        if len(scenes) != len(self.scenes) or any(a is not b for a, b in zip(scenes, self.scenes)):
            return False
        if any(int(self.scene_tab[s].n) != st.n for s, st in enumerate(scenes)):
            return False
        j = 0
        for cams in cams_per_scene:
            for cam in cams:
                if j >= self.n_views:
                    return False
                if bytes(memoryview(make_camera(cam)).cast("B")) != \
                        bytes(memoryview(self.view_tab[j].cam).cast("B")):
                    return False
                j += 1
        return j == self.n_views

    def reuse_for_update(self) -> None:
        """Prepare the batch for a new update of the same scenes and views
        after lifting changed the active sets: tables refreshed for the new
        active counts, gradient buffers grown if needed, every record projected
        again and every static prefix rebuilt; the depth cuts learnt by the
        previous update are kept as the first guess (a tile that needs more is
        completed as usual)."""
        self.refresh_active()
        info = self.info
        dev = self.device
        if self.grad2d.numel() < max(info.total_g2, 1) * abi.G2_STRIDE:
            self.grad2d = torch.empty(max(info.total_g2, 1) * abi.G2_STRIDE,
                                      dtype=torch.float32, device=dev)
        if self.grads.numel() < max(info.total_grad_rows, 1) * info.max_row_stride:
            self.grads = torch.empty(max(info.total_grad_rows, 1) * info.max_row_stride,
                                     dtype=torch.float32, device=dev)
        self._epochs = [st.epoch for st in self.scenes]
        self.reset_prefix()
        self.status.zero_()

    def deactivate(self, scene_indices) -> None:
        """Drop scenes from the work of later iterations without rebuilding:
        their active count becomes 0 in the device table (no active tiles, no
        gradient, no optimiser step), which captured graphs also read."""
        for s in scene_indices:
            self.scene_tab[s].n_active = 0
        self.scenes_dev.copy_(_bytes(self.scene_tab).pin_memory(), non_blocking=True)
        self.counted = False

    def record_stream(self, stream) -> None:
        """Mark every device buffer as used on `stream` (for a batch built on
        another stream), so the allocator does not reuse its memory early."""
        for t in vars(self).values():
            if isinstance(t, torch.Tensor) and t.is_cuda:
                t.record_stream(stream)

    def reset_prefix(self):
        """Forget every tile's static prefix (the next iteration rebuilds it)."""
        self.tile_cache.fill_(-1)
        self.counted = False

    def project_and_bin(self, mode: int):
        b = self
        if b.reproject:
            mode, b.reproject = 0, False
        epochs = [st.epoch for st in b.scenes]
        if epochs != b._epochs:  # an active set changed: the frozen rows did too
            b._epochs = epochs
            b.reset_prefix()
            b.counted = False
            mode = 0  # project them again (and recount their pairs)
        if b.counted and mode == 1:  # the planning pass counted this binning already
            mode = 2
        b.counted = False
        abi.check(abi.cls_project_and_bin(
            _ptr(b.scenes_dev), _ptr(b.views_dev), b.info, mode, b.layout, _ptr(b.records),
            _ptr(b.tile_active), _ptr(b.active_tiles), _ptr(b.n_active_tiles),
            _ptr(b.keys), _ptr(b.vals), b.capacity, _ptr(b.n_pairs), _ptr(b.ranges),
            _ptr(b.bin_offsets), _ptr(b.cut) if b.use_cut else None, _ptr(b.tile_cache),
            b.prefix_mode, 1 if b.ssim else 0, _ptr(b.status), _ptr(b.proj_ws),
            b.proj_ws.numel(), b.stream()),
            "cls_project_and_bin")

    def plan_capacity(self, slack: float = 1.5, extra: int = 1 << 16):
        """Count the pairs once (mode 0 projection, no keys) and size the key
        buffers; the only host synchronisation of an update besides lifting."""
        cap_before = self.capacity
        self.capacity = 0
        self.project_and_bin(0)
        need = int(self.n_pairs.item())
        self.status.zero_()
        cap = max(int(need * slack) + extra, cap_before)
        self.allocate_keys(cap)
        # the next binning (nothing changes before the first iteration) only
        # emits what this one counted
        self.counted = self.layout == 1
        return need

    def allocate_keys(self, capacity: int):
        dev = self.device
        self.capacity = capacity
        self.keys = torch.empty(capacity, dtype=torch.int64, device=dev)
        self.keys_alt = torch.empty(capacity, dtype=torch.int64, device=dev)
        self.tiles_ws = torch.empty(
            max(abi.cls_sort_tiles_workspace_size(capacity, self.min_bin()), 256),
            dtype=torch.uint8, device=dev)
        if self.layout == 0:
            self.vals = torch.empty(capacity, dtype=torch.int32, device=dev)
            self.vals_alt = torch.empty(capacity, dtype=torch.int32, device=dev)
            self.sort_ws = torch.empty(abi.cls_sort_workspace_size(capacity, self.info.key_bits),
                                       dtype=torch.uint8, device=dev)

    def _sort_tiles(self, cut=False, after_completion=False):
        b = self
        cap = b.info.total_tiles
        abi.check(abi.cls_sort_tiles(
            _ptr(b.keys), _ptr(b.keys_alt), _ptr(b.bin_offsets), _ptr(b.active_tiles),
            _ptr(b.n_active_tiles), cap, b.capacity, b.min_bin(),
            _ptr(b.cut) if cut and not after_completion else None,
            _ptr(b.trunc) if after_completion else None,
            _ptr(b.trunc_count) if after_completion else None, cap, _ptr(b.tile_cache),
            _ptr(b.counter) + 8,
            _ptr(b.tiles_ws), b.tiles_ws.numel(), b.stream()), "cls_sort_tiles")

    def min_bin(self) -> int:
        return abi.LAZY_MAX_BIN + 1 if self.lazy else 1

    def sort(self):
        b = self
        if b.layout == 1:
            b._sort_tiles(cut=b.use_cut)
            return
        abi.check(abi.cls_sort_keys(
            _ptr(b.keys), _ptr(b.vals), _ptr(b.keys_alt), _ptr(b.vals_alt), _ptr(b.n_pairs),
            b.capacity, b.info.key_bits, _ptr(b.ranges), b.info.total_tiles, _ptr(b.status),
            _ptr(b.sort_ws), b.sort_ws.numel(), b.stream()), "cls_sort_keys")

    def forward(self, loss_mode: int, bg=(0.0, 0.0, 0.0)):
        """Render the active tiles into `image` (the backward pass reads it),
        with the fused loss when loss_mode is 1 (L1) or 2 (L2), then the D-SSIM
        term if the batch has it."""
        self.render(loss_mode, bg)
        if self.ssim and loss_mode:
            self.apply_ssim(loss_mode)

    def render(self, loss_mode: int, bg=(0.0, 0.0, 0.0)):
        b = self
        if b.target_ready is not None:  # targets still on their way
            torch.cuda.current_stream().wait_event(b.target_ready)
            b.target_ready = None
        cut = b.use_cut
        if loss_mode or cut:
            b._fwd_acc.zero_()  # the loss and the truncated-tile count
        b._forward_call(loss_mode, bg, _ptr(b.active_tiles), _ptr(b.n_active_tiles),
                        None, _ptr(b.cut) if cut else None, _ptr(b.cut) if cut else None)
        if cut:
            # tiles whose cut was too shallow: write their missing pairs, render again
            cap = b.info.total_tiles
            abi.check(abi.cls_complete_truncated(
                _ptr(b.views_dev), b.info, _ptr(b.records), _ptr(b.keys), b.capacity,
                _ptr(b.trunc), _ptr(b.trunc_count), cap, _ptr(b.counter) + 12, _ptr(b.proj_ws),
                b.proj_ws.numel(), b.stream()), "cls_complete_truncated")
            b._sort_tiles(after_completion=True)  # large bins the completion filled
            b._forward_call(loss_mode, bg, _ptr(b.trunc), _ptr(b.trunc_count),
                            _ptr(b.trunc) + 4 * cap, None, _ptr(b.cut), rerun=True)

    def apply_ssim(self, loss_mode: int = 1):
        """Combine the forward pass's L1 gradient with the D-SSIM term."""
        b = self
        if loss_mode != 1:
            raise ValueError("the D-SSIM term combines with the L1 loss")
        abi.check(abi.cls_ssim_loss(
            _ptr(b.views_dev), b.info, _ptr(b.active_tiles), _ptr(b.n_active_tiles),
            _ptr(b.tile_active), _ptr(b.image), _ptr(b.target), SSIM_LAMBDA, _ptr(b.abc),
            _ptr(b.dL_dimage), _ptr(b.loss), b.stream()), "cls_ssim_loss")

    def _forward_call(self, loss_mode, bg, tiles, n_tiles, list_ranks, cut_in, cut_out,
                      rerun=False):
        b = self
        cap = b.info.total_tiles
        abi.check(abi.cls_render_forward(
            _ptr(b.views_dev), b.info, _ptr(b.records), *b._sorted_vals(), _ptr(b.ranges),
            tiles, n_tiles, _ptr(b.keys) if b.lazy else None,
            _ptr(b.bin_offsets) if b.lazy else None, list_ranks, cut_in, cut_out,
            None if rerun or cut_in is None else _ptr(b.trunc),
            None if rerun or cut_in is None else _ptr(b.trunc_count), cap, _ptr(b.tile_cache),
            _ptr(b.prefix_state), _ptr(b.prefix_last), bg,
            _ptr(b.target) if loss_mode else None, loss_mode,
            _ptr(b.image), _ptr(b.T_final), _ptr(b.n_contrib),
            _ptr(b.dL_dimage) if loss_mode else None,
            _ptr(b.loss) if loss_mode and not b.ssim else None,
            _ptr(b.counter), b.stream()), "cls_render_forward")

    def _sorted_vals(self):
        """Record index of sorted pair i: vals[i] (flat) or the low word of
        keys[i] (bucketed)."""
        if self.layout == 1:
            return _ptr(self.keys), 2
        return _ptr(self.vals), 1

    def sorted_records(self) -> np.ndarray:
        """Record index of every sorted pair (host copy, for checks)."""
        n = min(int(self.n_pairs.item()), self.capacity)
        if self.layout == 1:
            return self.keys[:n].cpu().numpy().view(np.uint32)[0::2].copy()
        return self.vals[:n].cpu().numpy().view(np.uint32).copy()

    def backward(self):
        """Gradients of the active rows from dL_dimage (the background is in
        the image the forward pass wrote)."""
        b = self
        abi.check(abi.cls_render_backward(
            _ptr(b.scenes_dev), _ptr(b.views_dev), b.info, _ptr(b.records), *b._sorted_vals(),
            _ptr(b.ranges), _ptr(b.active_tiles), _ptr(b.n_active_tiles), _ptr(b.tile_cache),
            _ptr(b.prefix_state), _ptr(b.image), _ptr(b.n_contrib), _ptr(b.dL_dimage),
            _ptr(b.grad2d), _ptr(b.grads), _ptr(b.counter) + 4, b.stream()),
            "cls_render_backward")

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-15):
        b = self
        abi.check(abi.cls_adam_step_active(
            _ptr(b.scenes_dev), b.info, _ptr(b.grads), lr, beta1, beta2, eps,
            _ptr(b.adam_ws), b.adam_ws.numel(), b.stream()), "cls_adam_step_active")

    def launches_per_step(self) -> int:
        """Kernels of one iteration. project_and_bin (mode 1): project (with
        the render-mask stamps) and nearest-active depth (2 if any Gaussian
        is active), tile mask, compaction (count, scan, write), pair count,
        then flat: scan, emit, emit-big (3) or bucketed: bin stamps, bin
        prefix, bucket counts, scan, offsets, emission window tables, emit (7). Sort: flat
        hist + scan + passes (+ copy if odd) + ranges; bucketed 1 or 2.
        Forward 1, or 5 with the depth cut (forward, completion, large-bin
        collection and sort, rerun);
        backward 2, Adam 2."""
        active = 2 if self.info.max_active > 0 else 0
        proj = (2 if active else 0) + 5 + (7 if self.layout == 1 else 3)
        if self.layout == 1:
            sort = 2 if self.lazy else 1
        else:
            passes = -(-self.info.key_bits // 8)
            sort = 3 + passes + passes % 2
        fwd = 5 if self.use_cut else 1
        return proj + sort + fwd + (1 + active // 2) + (1 + active // 2)

    def check_status(self):
        code = int(self.status.item())
        if code != abi.CLS_OK:
            raise abi.ClsError(f"device status {abi.STATUS_NAMES.get(code, code)}")


def _views_for(cams):
    views = (abi.ClsView * len(cams))()
    pix = 0
    for j, cam in enumerate(cams):
        views[j].cam = make_camera(cam)
        views[j].pix_base = pix
        pix += int(cam["width"]) * int(cam["height"])
    return views, pix


def lift(state: SceneState, cams: Sequence, masks, vote_mode: int = 0, device="cuda",
         want_votes: bool = False):
    """Change-mask lifting on the GPU; sets the scene's active set. `masks` is a
    list of H x W uint8 arrays or one flat uint8 tensor (views concatenated).
    Returns (active uint8 numpy, votes [n, 2] numpy or None)."""
    views, pix = _views_for(cams)
    views_dev = _bytes(views).to(device)
    if isinstance(masks, torch.Tensor):
        masks_dev = masks.to(device, non_blocking=True)
    else:
        masks_dev = torch.from_numpy(np.concatenate(
            [np.ascontiguousarray(m, np.uint8).reshape(-1) for m in masks])).to(device)
    if masks_dev.numel() != pix:
        raise ValueError("mask size does not match the cameras")
    n = state.n
    ws = torch.zeros(max(abi.cls_lift_workspace_size(n), 256), dtype=torch.uint8, device=device)
    n_act = torch.zeros(1, dtype=torch.int32, device=device)
    votes = torch.zeros(2 * max(n, 1), dtype=torch.int32, device=device) if want_votes else None
    stream = torch.cuda.current_stream().cuda_stream
    abi.check(abi.cls_lift_change_masks(
        _ptr(state.params), n, state.stride, _ptr(views_dev), 0, len(cams), _ptr(masks_dev),
        vote_mode, _ptr(state.active), _ptr(state.active_idx), _ptr(n_act), _ptr(votes),
        _ptr(ws), ws.numel(), stream), "cls_lift_change_masks")
    state.n_active = int(n_act.item())
    state.epoch += 1
    if not want_votes:
        return None, None
    return state.active.cpu().numpy(), votes.view(-1, 2)[:n].cpu().numpy()


class SphereRegion:
    """The spheres bounding O^t (Sec. 3.3 "Sphere Pruning"; Supp. "Identifying
    Changed Gaussians"): K-Means clusters of the active Gaussians' centres, a
    sphere per cluster at its mean with radius 1.1 x the 98th quantile of the
    members' distances. K defaults to min(10, max(1, A // 1000))."""

    def __init__(self, state: "SceneState", k: Optional[int] = None, iters: int = 16):
        A = state.n_active
        if A <= 0:
            raise ValueError("the sphere region needs a non-empty active set")
        dev = state.params.device
        self.k = int(k) if k is not None else int(min(abi.MAX_SPHERES, max(1, A // 1000)))
        self.k = min(self.k, A)
        self.spheres = torch.empty(self.k * 4, dtype=torch.float32, device=dev)
        self.labels = torch.empty(A, dtype=torch.int32, device=dev)
        self.counts = torch.empty(self.k, dtype=torch.int32, device=dev)
        ws = torch.empty(abi.cls_spheres_workspace_size(A), dtype=torch.uint8, device=dev)
        abi.check(abi.cls_fit_spheres(
            _ptr(state.params), state.stride, _ptr(state.active_idx), A, self.k, iters,
            _ptr(self.spheres), _ptr(self.labels), _ptr(self.counts), _ptr(ws), ws.numel(),
            torch.cuda.current_stream().cuda_stream), "cls_fit_spheres")

    def host(self) -> Dict[str, np.ndarray]:
        s = self.spheres.view(self.k, 4).cpu().numpy()
        return {"centers": s[:, :3].copy(), "radii": s[:, 3].copy(),
                "counts": self.counts.cpu().numpy().astype(np.int64),
                "labels": self.labels.cpu().numpy()}


def prune_outside(state: "SceneState", region: SphereRegion, want_removed: bool = False):
    """Supp. "3DGS Optimization in Changed Regions": remove every Gaussian of
    O^t whose centre lies in no sphere (opacity logit -inf, out of the active
    set). Returns the number removed (and their ids if asked)."""
    dev = state.params.device
    A = state.n_active
    ws = torch.empty(max(abi.cls_prune_workspace_size(A), 256), dtype=torch.uint8, device=dev)
    n_active = torch.zeros(1, dtype=torch.int32, device=dev)
    n_removed = torch.zeros(1, dtype=torch.int32, device=dev)
    removed = torch.empty(max(A, 1), dtype=torch.int32, device=dev) if want_removed else None
    abi.check(abi.cls_prune_outside_spheres(
        _ptr(state.params), state.stride, _ptr(state.active), _ptr(state.active_idx), A,
        _ptr(n_active), _ptr(region.spheres), region.k, _ptr(removed), _ptr(n_removed),
        _ptr(ws), ws.numel(), torch.cuda.current_stream().cuda_stream),
        "cls_prune_outside_spheres")
    k = int(n_removed.item())
    if k:
        state.n_active = int(n_active.item())
        state.epoch += 1
    if want_removed:
        return k, np.sort(removed[:k].cpu().numpy())
    return k


class LocalUpdate:
    """One scene, a handful of posed views and their change masks: lift, then
    iterate project/bin -> sort -> render forward (+loss) -> render backward ->
    masked Adam, all on the device."""

    def __init__(self, scene, cams, sh_degree: int, targets=None, masks=None, active=None,
                 vote_mode: int = 0, loss: str = "l1", lr: float = 1e-3,
                 bg=(0.0, 0.0, 0.0), device="cuda", capacity_slack: float = 1.5,
                 layout: int = 1, lazy: bool = True, prune_every: int = 0,
                 sphere_k: Optional[int] = None, densify: Optional[dict] = None):
        """prune_every > 0 fits the sphere region of the lifted O^t and removes
        the Gaussians that leave it every `prune_every` iterations (the paper
        uses 15). `densify` (a dict of Densifier options with at least
        `draws`) turns on adaptive density control of O^t."""
        self.cams = list(cams)
        self.loss_mode = LOSS_MODES[loss]
        self.lr = lr
        self.bg = tuple(float(x) for x in bg)
        self.state = SceneState(scene, sh_degree, device)
        if active is not None:
            self.state.set_active(active)
        elif masks is not None:
            lift(self.state, self.cams, masks, vote_mode, device)
        else:
            raise ValueError("give either an active set or change masks")
        self.batch = Batch([self.state], [self.cams], device, layout, lazy,
                           ssim=loss == "l1+ssim")
        if targets is not None:
            self.batch.set_targets(targets)
        self.capacity_slack = capacity_slack
        self.pairs_planned = self.batch.plan_capacity(capacity_slack)
        self._init_region(prune_every, sphere_k, densify)
        torch.cuda.synchronize()

    def _init_region(self, prune_every: int, sphere_k: Optional[int],
                     densify: Optional[dict] = None):
        self.prune_every = int(prune_every)
        self.iteration = 0
        self.removed = 0
        self.region = SphereRegion(self.state, sphere_k) if self.prune_every > 0 else None
        self.densifier = None
        if densify:
            from .densify import Densifier
            self.densifier = Densifier(self.state, self.cams, **densify)

    def _rebuild_batch(self):
        """New batch tables and buffers after the scene grew."""
        old = self.batch
        b = Batch([self.state], [self.cams], old.device, old.layout, old.lazy,
                  prefix_cache=old.prefix_mode == 1, ssim=old.ssim)
        b.target = old.target
        self.batch = b
        self.pairs_planned = b.plan_capacity(self.capacity_slack)

    @classmethod
    def from_resident(cls, state: SceneState, cams, targets, masks, vote_mode: int = 0,
                      loss: str = "l1", lr: float = 1e-3, bg=(0.0, 0.0, 0.0),
                      capacity_slack: float = 1.5, layout: int = 1, lazy: bool = True,
                      reuse: Optional["LocalUpdate"] = None):
        """A new update of a scene already resident on the device. `targets`
        (float32, [3][H][W] per view, concatenated) and `masks` (uint8, [H][W]
        per view, concatenated) are flat tensors, typically pinned host memory;
        they are copied to the device here. `reuse`: a finished earlier update
        of the same scene with the same cameras, whose batch (tables, buffers,
        learnt depth cuts) this update takes over instead of building new
        ones; otherwise, or if it does not match, a new batch is built."""
        self = cls.__new__(cls)
        self.cams = list(cams)
        self.loss_mode = LOSS_MODES[loss]
        self.lr = lr
        self.bg = tuple(float(x) for x in bg)
        self.state = state
        dev = state.params.device
        lift(state, self.cams, masks, vote_mode, dev)
        ssim = loss == "l1+ssim"
        old = reuse.batch if reuse is not None else None
        if (old is not None and old.layout == layout and old.lazy == (lazy and layout == 1)
                and old.ssim == ssim and old.matches([state], [self.cams])):
            self.batch = old
            reuse.batch = None  # the earlier update no longer owns it
            self.batch.reuse_for_update()
        else:
            self.batch = Batch([state], [self.cams], dev, layout, lazy, ssim=ssim)
        # the targets travel on a copy stream while lifting and planning run;
        # the first forward pass waits for them
        main = torch.cuda.current_stream()
        copy = _copy_stream(dev)
        copy.wait_stream(main)
        with torch.cuda.stream(copy):
            tgt = targets.to(dev, non_blocking=True)
        tgt.record_stream(main)
        self.batch.target = tgt
        self.batch.target_ready = copy.record_event()
        self.capacity_slack = capacity_slack
        self.pairs_planned = self.batch.plan_capacity(capacity_slack)
        self._init_region(0, None)
        return self

    def render_pass(self, with_backward: bool = True, with_adam: bool = True):
        b = self.batch
        b.project_and_bin(1)
        b.sort()
        b.forward(self.loss_mode if b.target is not None else 0, self.bg)
        if with_backward:
            b.backward()
            if with_adam:
                b.adam(self.lr)

    def capture(self):
        """One iteration (project/bin, sort, forward + loss, backward, masked
        Adam) recorded as a CUDA graph, to replay with `.replay()`: valid while
        the batch, its targets and the active set stay as they are (no
        pruning or densification in between)."""
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            g.capture_begin()
            self.render_pass(True, True)
            g.capture_end()
        torch.cuda.current_stream().wait_stream(side)
        return g

    def step(self):
        d = self.densifier
        if d is None:
            self.render_pass(True, True)
            self.iteration += 1
        else:
            # the base optimiser's order: statistics, densification (no
            # optimiser step on that iteration), then the opacity reset
            it = self.iteration + 1
            self.render_pass(True, False)
            grew = False
            if it < d.until:
                d.accumulate(self.batch)
                if d.due(it):
                    d.densify(it)
                    grew = True
            if not grew:
                self.batch.adam(self.lr)
            if d.reset_due(it):
                d.reset_opacity()
            if grew:
                self._rebuild_batch()
            self.iteration = it
        if self.region is not None and self.iteration % self.prune_every == 0:
            k = prune_outside(self.state, self.region)
            if k:
                self.removed += k
                self.batch.refresh_active()

    def run(self, iters: int):
        for _ in range(iters):
            self.step()
        self.batch.check_status()
