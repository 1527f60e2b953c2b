"""History recovery and merging of scene updates (Supp. "History Recovery",
its algorithm, and "Batched Updates").

Before update t optimises, `begin_update` stores O^t (the changed rows, in
G^{t-1}'s order) and the mask I^t, and reorders the resident scene so that its
first #static rows are G^{t-1}'s unchanged Gaussians in order (then O^t). The
optimiser only ever changes, appends or removes rows of O^t, so `recover`
rebuilds G^{t-1} from G^t exactly, and `recover_state` walks back any number
of updates. `merge` combines two updates of the same scene. Row moves are
libclsplat kernels (a stable partition map from one scan, then a row gather).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import torch

from . import _abi as abi
from .update import SceneState, _ptr


@dataclasses.dataclass
class HistoryEntry:
    O: torch.Tensor   # [|O^t|][row_stride] changed rows before optimisation
    I: torch.Tensor   # [n_{t-1}] uint8 mask of the changed rows in G^{t-1}


def _stream():
    return torch.cuda.current_stream().cuda_stream


def flag_map(flags: torch.Tensor, mode: int):
    n = int(flags.numel())
    dev = flags.device
    m = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(max(abi.cls_flag_map_workspace_size(n), 256), dtype=torch.uint8, device=dev)
    abi.check(abi.cls_flag_map(_ptr(flags), n, mode, _ptr(m), _ptr(cnt), _ptr(ws), ws.numel(),
                               _stream()), "cls_flag_map")
    return m[:n], cnt


def gather_rows(a: torch.Tensor, b, m: torch.Tensor, n_out: int) -> torch.Tensor:
    stride = int(a.shape[1])
    out = torch.empty((max(n_out, 1), stride), dtype=a.dtype, device=a.device)
    abi.check(abi.cls_gather_rows(_ptr(a), _ptr(b), _ptr(m), n_out, stride, _ptr(out), _stream()),
              "cls_gather_rows")
    return out[:n_out]


def begin_update(state: SceneState) -> HistoryEntry:
    """Store (O^t, I^t) of the scene's current active set and reorder the
    scene: unchanged rows first in order, then O^t, which stays the active
    set. Adam moments move with their rows."""
    n, A = state.n, state.n_active
    idx = state.active_idx[:A]
    entry = HistoryEntry(O=gather_rows(state.params, None, idx, A), I=state.active.clone())
    m, _ = flag_map(state.active, 0)
    state.params = gather_rows(state.params, None, m, n)
    state.adam_m = gather_rows(state.adam_m, None, m, n)
    state.adam_v = gather_rows(state.adam_v, None, m, n)
    dev = state.params.device
    state.active = torch.cat([torch.zeros(n - A, dtype=torch.uint8, device=dev),
                              torch.ones(A, dtype=torch.uint8, device=dev)])
    state.active_idx = torch.arange(n - A, max(n, 1), dtype=torch.int32, device=dev)
    state.epoch += 1
    return entry


def recover(rows_t: torch.Tensor, entry: HistoryEntry) -> torch.Tensor:
    """G^{t-1} from G^t (rows) and the stored entry of update t."""
    n_prev = int(entry.I.numel())
    n_static = n_prev - int(entry.O.shape[0])
    if rows_t.shape[0] < n_static:
        raise ValueError("G^t has fewer rows than the unchanged part of G^{t-1}")
    m, _ = flag_map(entry.I, 1)
    return gather_rows(rows_t, entry.O, m, n_prev)


def recover_state(rows_T: torch.Tensor, entries: Sequence[HistoryEntry], steps: int):
    """History Recovery: `entries` newest first, `steps` states back."""
    rows = rows_T
    for e in entries[:steps]:
        rows = recover(rows, e)
    return rows


def merge(rows_prev: torch.Tensor, updates: List[Tuple[torch.Tensor, torch.Tensor]]):
    """Batched Updates: rows of G^{t-1} in no update's mask, in order, then
    each update's optimised Gaussians. `updates`: (I uint8 mask, O rows)."""
    touched = torch.zeros_like(updates[0][0]) if updates else None
    for I, _ in updates:
        touched = touched | I
    m, cnt = flag_map(touched, 0)
    n_keep = int(rows_prev.shape[0]) - int(cnt.item())
    parts = [gather_rows(rows_prev, None, m, n_keep)] + [O for _, O in updates]
    return torch.cat(parts)
