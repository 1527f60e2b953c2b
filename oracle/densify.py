"""Densification restricted to O^t. TEST INFRASTRUCTURE ONLY (see the
package docstring).

Supp. "History Recovery" notes that duplication and pruning only affect O^t;
Supp. "Implementation Details" adopts the base 3DGS optimiser's defaults,
whose adaptive density control is, every 100 iterations: accumulate per
Gaussian the norm of the view-space (NDC) gradient of its projected centre
over the views where it is visible; a Gaussian whose mean accumulated norm is
at least 0.0002 is cloned if its largest scale is at most 0.01 x the scene
extent, else split into 2 Gaussians sampled from it with scales divided by
1.6 (the original removed); then Gaussians with opacity below 0.005 are
removed, and (after the first opacity reset) those larger than 20 pixels on
screen or 0.1 x the extent in the world. Here all of it applies to O^t only.

Readings of points the paper leaves open: the accumulation takes each view of
an iteration as one observation, with the gradient of that view's own loss
(the iteration's loss is the mean over its n views, so n x its gradient);
the opacity reset (every 3000 iterations) caps the logit of O^t at
logit(0.01) and restarts the Adam moments of that entry; the decisions compare float32 quantities
with thresholds computed once in float64 and rounded to float32: mean norm
(float32 accum / denom) >= 0.0002, largest log-scale <= log(0.01 extent),
opacity logit < logit(0.005), largest log-scale > log(0.1 extent); the split
children are mu + R(q) (s * z) for input standard normals z (two per
Gaussian) with log-scales log s - log(1.6); new rows are appended in rank
order (per Gaussian: its clone, then its children) and start with zero
statistics; a removed Gaussian leaves O^t with opacity logit -inf.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

F = np.float32
GRAD_THRESHOLD = 0.0002
PERCENT_DENSE = 0.01
MIN_OPACITY = 0.005
N_SPLIT = 2
SPLIT_SHRINK = 0.8 * N_SPLIT
MAX_SCREEN = 20.0
BIG_WORLD = 0.1
RESET_OPACITY = 0.01


def thresholds(extent: float) -> Dict[str, np.float32]:
    return {"grad": F(GRAD_THRESHOLD),
            "clone_ls": F(np.log(PERCENT_DENSE * extent)),
            "logit": F(np.log(MIN_OPACITY / (1.0 - MIN_OPACITY))),
            "big_ls": F(np.log(BIG_WORLD * extent)),
            "shrink": F(np.log(SPLIT_SHRINK))}


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(means, log_scales, quats, logits, active_idx, accum, denom, max_radius, extent,
            z, big: bool) -> Dict[str, np.ndarray]:
    """One densification step over O^t. z: [len(active_idx)][2][3] normals.
    Returns removed original ids, and for the new rows their source id and
    means/log-scales (other parameters copy the source)."""
    th = thresholds(extent)
    removed, src, new_means, new_ls = [], [], [], []
    for a, g in enumerate(np.asarray(active_idx)):
        d = F(denom[g])
        avg = F(F(accum[g]) / d) if d > 0 else F(0)
        ls = np.asarray(log_scales[g], F)
        mls = F(ls.max())
        sel = avg >= th["grad"]
        clone = sel and mls <= th["clone_ls"]
        split = sel and mls > th["clone_ls"]

        def pruned(logit, mls_, maxr):
            return logit < th["logit"] or (big and (maxr > MAX_SCREEN or mls_ > th["big_ls"]))

        low = pruned(F(logits[g]), mls, max_radius[g])
        if split or low:
            removed.append(int(g))
        if clone and not low:
            src.append(int(g))
            new_means.append(np.asarray(means[g], np.float64))
            new_ls.append(ls.copy())
        if split:
            R = quat_to_rot(quats[g])
            s = np.exp(ls.astype(np.float64))
            cls = (ls - th["shrink"]).astype(F)
            for k in range(N_SPLIT):
                if pruned(F(logits[g]), F(cls.max()), 0.0):
                    continue
                src.append(int(g))
                new_means.append(np.asarray(means[g], np.float64) +
                                 R @ (s * np.asarray(z[a][k], np.float64)))
                new_ls.append(cls)
    return {"removed": np.array(removed, np.int64), "src": np.array(src, np.int64),
            "means": np.array(new_means).reshape(-1, 3), "log_scales": np.array(new_ls, F).reshape(-1, 3)}


def accumulate(accum, denom, max_radius, gids, du, dv, radius, W, H, n_views=1):
    """One view's statistics: for each visible Gaussian (radius > 0), the
    norm of its NDC-space positional gradient (pixel gradient x W/2, H/2)
    for the view's own loss (x n_views when du, dv are gradients of the mean
    over n_views views)."""
    for g, a, b, r in zip(gids, du, dv, radius):
        if r <= 0:
            continue
        gx, gy = F(F(a) * F(0.5 * W * n_views)), F(F(b) * F(0.5 * H * n_views))
        accum[g] = F(accum[g] + F(np.sqrt(F(gx * gx + gy * gy))))
        denom[g] += 1
        max_radius[g] = max(max_radius[g], float(r))


def reset_limit() -> np.float32:
    return F(np.log(RESET_OPACITY / (1.0 - RESET_OPACITY)))


def reset_opacity(logits, active_idx):
    """Opacity reset of O^t: sigmoid(logit) becomes min(sigmoid(logit), 0.01)
    (in the logit domain, min(logit, logit(0.01)))."""
    out = np.array(logits, F)
    idx = np.asarray(active_idx, np.int64)
    out[idx] = np.minimum(out[idx], reset_limit())
    return out
