"""New-point sampling for appearing objects. TEST INFRASTRUCTURE ONLY (see
the package docstring).

Sec. 3.2 "Gaussian Sampling for New Objects" and its algorithm New Point
Sampling: while the point set O has fewer than n points, an empty O is replaced
by a uniform sample of n points in the bounding box of the scene's centres
(Supp. Full-Scene Point Sampling), a non-empty one is extended by n/5 points
drawn from a Gaussian mixture fitted to K-Means (K = 10) clusters of O (Supp.
Region Point Sampling: component mean = cluster centre, covariance = the
diagonal matrix holding the vector from the centre to the cluster's furthest
point); every drawn point is kept only if it passes the majority vote of
Sec. 3.2. The new points are then initialised as the base 3DGS method
initialises a point cloud.

Readings of points the paper leaves open:
  * the draws are inputs: per round, uniform numbers in [0, 1) (n x 3 for the
    box, n/5 for the component choice) and standard normals (n/5 x 3), made
    by the seeded input generator, so both implementations consume the same
    numbers;
  * box sample: p = min + u (max - min) per axis, float32 operations;
  * clusters: the K-Means of the sphere region (farthest-point start, 16 Lloyd
    iterations, exact fixed-point means) with K = min(10, |O|); the furthest
    point of a cluster is its member of largest float32 squared distance to
    the centre, ties to the lowest position in O;
  * mixture: component weights proportional to the cluster sizes; a draw
    takes component j, the first with t < (members of clusters 0..j), where
    t = floor(u * |O|) in float64; the covariance diagonal holds |v|, so the
    standard deviation per axis is sqrt(|v|) (float32), p = c + sqrt(|v|) z;
  * at most 64 rounds;
  * initialisation of the new points (the base method's defaults for a
    point cloud without colours): isotropic log-scale 0.5 log(d), d the float32
    mean ((d1 + d2) + d3) / 3 of the squared distances to the three nearest
    other new points (fewer if there are fewer), at least 1e-7; identity
    rotation; opacity 0.1; colour 0.5 grey (all SH coefficients 0).
"""
from __future__ import annotations

from typing import Callable, Dict

import numpy as np

from . import fp32_index as fx
from . import spheres as osp

F = np.float32
REGION_K = 10
MAX_ROUNDS = 64
INIT_OPACITY = 0.1


def bbox(means: np.ndarray):
    m = np.asarray(means, F)
    return m.min(axis=0), m.max(axis=0)


def box_sample(lo: np.ndarray, hi: np.ndarray, u: np.ndarray) -> np.ndarray:
    lo, hi, u = np.asarray(lo, F), np.asarray(hi, F), np.asarray(u, F)
    return lo + u * (hi - lo)


def vote_keep(points: np.ndarray, cams, masks) -> np.ndarray:
    c, o = fx.votes(points, cams, masks)
    return np.asarray(points, F)[fx.vote_rule(c, o, len(cams))]


def region_mixture(points: np.ndarray):
    """(centres [k][3], |v| [k][3], counts [k]) of the K-Means clusters."""
    points = np.asarray(points, F)
    k = min(REGION_K, points.shape[0])
    labels, centres = osp.kmeans(points, k)
    absv = np.zeros((k, 3), F)
    counts = np.zeros(k, np.int64)
    for j in range(k):
        m = np.flatnonzero(labels == j)
        counts[j] = m.size
        if m.size:
            d = osp.sq_dist32(points[m], centres[j])
            far = m[int(np.argmax(d))]  # first maximum: lowest position
            absv[j] = np.abs(points[far] - centres[j])
    return centres, absv, counts


def mixture_sample(centres, absv, counts, u_comp: np.ndarray, z: np.ndarray) -> np.ndarray:
    total = int(counts.sum())
    cum = np.cumsum(counts)
    t = np.floor(np.asarray(u_comp, F).astype(np.float64) * total).astype(np.int64)
    comp = np.searchsorted(cum, t, side="right")  # first j with t < cum[j]
    std = np.sqrt(np.asarray(absv, F))
    return np.asarray(centres, F)[comp] + std[comp] * np.asarray(z, F)


def sample_points(active_means: np.ndarray, scene_means: np.ndarray, cams, masks, n: int,
                  draws: Callable) -> Dict[str, np.ndarray]:
    """The New Point Sampling loop. `draws(round, kind, shape)` returns the
    round's input numbers (kind "box": uniform n x 3; "comp": uniform n/5;
    "normal": standard normal n/5 x 3). Returns the final point set and the
    new points (those not in the initial O)."""
    O = np.asarray(active_means, F).reshape(-1, 3)
    start = O.shape[0]
    lo, hi = bbox(scene_means)
    rounds = 0
    fresh = False  # O holds only sampled points (after a box round)
    while O.shape[0] < n and rounds < MAX_ROUNDS:
        if O.shape[0] == 0:
            S = box_sample(lo, hi, draws(rounds, "box", (n, 3)))
            O = vote_keep(S, cams, masks)
            fresh = True
        else:
            m = n // 5
            c, v, k = region_mixture(O)
            S = mixture_sample(c, v, k, draws(rounds, "comp", (m,)), draws(rounds, "normal", (m, 3)))
            O = np.concatenate([O, vote_keep(S, cams, masks)])
        rounds += 1
    new = O if fresh else O[start:]
    return {"points": O, "new": new, "rounds": rounds}


def knn_mean_sq(points: np.ndarray) -> np.ndarray:
    p = np.asarray(points, F)
    n = p.shape[0]
    out = np.full(n, F(1e-7), F)
    if n < 2:
        return out
    for i in range(n):
        d = osp.sq_dist32(p, p[i])
        d = np.delete(d, i)
        d = np.sort(d)[: min(3, n - 1)]
        s = d[0]
        for x in d[1:]:
            s = F(s + x)
        out[i] = max(F(s / F(d.size)), F(1e-7))
    return out


def init_gaussians(points: np.ndarray, sh_degree: int) -> Dict[str, np.ndarray]:
    """Scene arrays of the new points (the base method's point-cloud defaults)."""
    p = np.asarray(points, F)
    n = p.shape[0]
    K = (sh_degree + 1) ** 2
    ls = 0.5 * np.log(knn_mean_sq(p).astype(np.float64))
    return {"means": p.copy(),
            "log_scales": np.repeat(ls[:, None], 3, axis=1).astype(F),
            "quats": np.tile(np.array([1, 0, 0, 0], F), (n, 1)),
            "opacity_logits": np.full(n, np.log(INIT_OPACITY / (1 - INIT_OPACITY)), F),
            "sh": np.zeros((n, K, 3), F)}
