"""History recovery and merging of scene updates. TEST INFRASTRUCTURE ONLY
(see the package docstring).

Supp. "History Recovery": at each update t the changed Gaussians O^t and their
index mask I^t over G^{t-1} are stored before optimisation, and G^t is ordered
so that its first #static = |G^{t-1} \\ O^t| rows are G^{t-1}'s static
Gaussians in their order (an invariant optimisation keeps, since duplication
and pruning only touch O^t). Then G^{t-1} is recovered from G^t by placing
G^t's first #static rows where I^t = 0 and the stored O^t where I^t = 1; the
History Recovery algorithm repeats this down to any past state.

Supp. "Batched Updates": two updates of the same G^{t-1} with index masks I_1,
I_2 and optimised Gaussians O_1, O_2 merge into G^t = O_1 u O_2 u (the
Gaussians of G^{t-1} in neither mask) (the printed set expression removes
G^{t-1} at the complement of both masks, which would drop the static part; the
reading here removes the rows in either mask).

Readings: rows are parameter rows; "first #static rows" keeps G^{t-1}'s order;
O^t is stored in G^{t-1}'s order; the merged scene is the kept static rows in
order, then O_1, then O_2 (the updates are taken as disjoint).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def begin_update(rows: np.ndarray, changed: np.ndarray) -> Tuple[np.ndarray, Dict[str, np.ndarray]]:
    """(G^t before optimisation: static rows first, then O^t; the stored
    entry {"O": O^t rows, "I": mask})."""
    I = np.asarray(changed, bool)
    entry = {"O": np.array(rows[I], copy=True), "I": I.copy()}
    return np.concatenate([rows[~I], rows[I]]), entry


def recover(rows_t: np.ndarray, entry: Dict[str, np.ndarray]) -> np.ndarray:
    """G^{t-1} from G^t and the stored (O^t, I^t)."""
    I = entry["I"]
    n_static = int((~I).sum())
    out = np.empty((I.size,) + rows_t.shape[1:], rows_t.dtype)
    out[~I] = rows_t[:n_static]
    out[I] = entry["O"]
    return out


def recover_state(rows_T: np.ndarray, entries: Sequence[Dict[str, np.ndarray]], steps: int
                  ) -> np.ndarray:
    """History Recovery: `entries` newest first; `steps` states back."""
    rows = rows_T
    for e in entries[:steps]:
        rows = recover(rows, e)
    return rows


def merge(rows_prev: np.ndarray, updates: List[Tuple[np.ndarray, np.ndarray]]) -> np.ndarray:
    """Batched Updates: (I_j, optimised O_j) pairs over the same G^{t-1}."""
    touched = np.zeros(rows_prev.shape[0], bool)
    for I, _ in updates:
        touched |= np.asarray(I, bool)
    return np.concatenate([rows_prev[~touched]] + [np.asarray(O) for _, O in updates])
