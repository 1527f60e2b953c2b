"""Sphere region of the changed Gaussians and pruning outside it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.3 ("Sphere Pruning") bounds the optimisation region by a union of
spheres, one per cluster of the changed Gaussians' centres; Supp.
("Identifying Changed Gaussians") fits each sphere at the cluster mean m_i
with radius 1.1 x the 98th quantile of the members' distances to m_i; Supp.
("3DGS Optimization in Changed Regions") removes, every 15 iterations, each
Gaussian of O^t whose centre lies in no sphere.

Readings of points the paper leaves open:
  * clusters: the paper's HDBSCAN (minimum cluster size 1000) is a third-party
    serial algorithm and out of scope; K-Means (Lloyd) stands in, with
    K = min(10, max(1, A // 1000)) for A changed Gaussians (at most one cluster
    per 1000 points, capped at the K = 10 the paper uses for its own K-Means),
    farthest-point initial centres (Gonzalez: the first point of the list,
    then repeatedly the point whose float32 squared distance to its nearest
    chosen centre is largest, ties to the lowest list position), 16 Lloyd
    iterations, an empty cluster keeping its centre;
  * every distance is float32 with the operation order
    ((dx*dx + dy*dy) + dz*dz), each operation rounded; a point goes to its
    nearest centre, ties to the lowest cluster index;
  * cluster means are exact: coordinates are summed as integers of 2^-24 units
    (each float32 coordinate times 2^24, rounded half to even, in int64), and
    the mean is the float64 quotient sum / count / 2^24 rounded to float32, so
    no summation order changes it;
  * the quantile is NumPy's default ("linear") estimator over the members'
    float32 distances in float64: h = (n - 1) 0.98, q = d[lo] + (h - lo)
    (d[lo + 1] - d[lo]) with lo = floor(h); the radius is float32(1.1 q);
  * a centre is inside a sphere iff its float32 squared distance is <= r * r
    (float32); clusters without members have no sphere;
  * a pruned Gaussian leaves O^t and its opacity logit becomes -inf (opacity 0:
    it can no longer contribute to any pixel), which renders exactly as if its
    row were removed.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

F = np.float32
SCALE = 2.0 ** 24
PRUNE_EVERY = 15
QUANTILE = 0.98
RADIUS_FACTOR = 1.1
KMEANS_ITERS = 16


def n_clusters(n_points: int) -> int:
    return int(min(10, max(1, n_points // 1000)))


def sq_dist32(p: np.ndarray, c: np.ndarray) -> np.ndarray:
    """float32 ((dx*dx + dy*dy) + dz*dz) of every row of p to centre c."""
    p = np.asarray(p, F)
    c = np.asarray(c, F)
    dx, dy, dz = p[:, 0] - c[0], p[:, 1] - c[1], p[:, 2] - c[2]
    return (dx * dx + dy * dy) + dz * dz


def assign(points: np.ndarray, centers: np.ndarray) -> np.ndarray:
    D = np.stack([sq_dist32(points, c) for c in centers], axis=1)
    return np.argmin(D, axis=1).astype(np.int32)  # first minimum: lowest index on ties


def fixed_point(x: np.ndarray) -> np.ndarray:
    return np.rint(np.asarray(x, F).astype(np.float64) * SCALE).astype(np.int64)


def cluster_means(points: np.ndarray, labels: np.ndarray, centers: np.ndarray) -> np.ndarray:
    q = fixed_point(points)
    out = np.array(centers, F, copy=True)
    for k in range(len(centers)):
        m = labels == k
        cnt = int(m.sum())
        if cnt:
            s = q[m].sum(axis=0)  # exact in int64
            out[k] = ((s.astype(np.float64) / cnt) / SCALE).astype(F)
    return out


def farthest_point_init(points: np.ndarray, k: int) -> np.ndarray:
    points = np.asarray(points, F)
    chosen = [0]
    nearest = sq_dist32(points, points[0])
    for _ in range(1, k):
        j = int(np.argmax(nearest))  # first maximum: lowest position on ties
        chosen.append(j)
        nearest = np.minimum(nearest, sq_dist32(points, points[j]))
    return points[chosen].copy()


def kmeans(points: np.ndarray, k: int, iters: int = KMEANS_ITERS):
    """Lloyd's algorithm: (labels of the last assignment, means of it)."""
    points = np.asarray(points, F)
    n = points.shape[0]
    centers = farthest_point_init(points, k)
    labels = np.zeros(n, np.int32)
    for _ in range(iters):
        labels = assign(points, centers)
        centers = cluster_means(points, labels, centers)
    return labels, centers


def quantile_linear(d: np.ndarray, q: float) -> float:
    d = np.sort(np.asarray(d, np.float64))
    n = d.size
    h = (n - 1) * q
    lo = int(np.floor(h))
    hi = min(lo + 1, n - 1)
    return float(d[lo] + (h - lo) * (d[hi] - d[lo]))


def fit_spheres(points: np.ndarray, k: int = None) -> Dict[str, np.ndarray]:
    """Spheres of the clusters of `points` (the changed Gaussians' centres):
    centres [k][3] float32, radii [k] float32 (-1: empty cluster), counts,
    labels."""
    points = np.asarray(points, F)
    if k is None:
        k = n_clusters(points.shape[0])
    labels, centers = kmeans(points, k)
    radii = np.full(k, -1.0, F)
    counts = np.zeros(k, np.int64)
    for i in range(k):
        m = labels == i
        counts[i] = int(m.sum())
        if counts[i]:
            d = np.sqrt(sq_dist32(points[m], centers[i]))  # float32, correctly rounded
            radii[i] = F(RADIUS_FACTOR * quantile_linear(d, QUANTILE))
    return {"centers": centers, "radii": radii, "counts": counts, "labels": labels}


def inside(points: np.ndarray, spheres: Dict[str, np.ndarray]) -> np.ndarray:
    points = np.asarray(points, F)
    out = np.zeros(points.shape[0], bool)
    for c, r in zip(spheres["centers"], spheres["radii"]):
        if r < 0:
            continue
        out |= sq_dist32(points, c) <= F(r) * F(r)
    return out


def prune(means: np.ndarray, opacity_logit: np.ndarray, active: np.ndarray,
          spheres: Dict[str, np.ndarray]):
    """Pruning step: (new active mask, new opacity logits, removed indices)."""
    active = np.asarray(active, bool)
    idx = np.flatnonzero(active)
    out = ~inside(np.asarray(means, F)[idx], spheres)
    removed = idx[out]
    new_active = active.copy()
    new_active[removed] = False
    logit = np.array(opacity_logit, F, copy=True)
    logit[removed] = -np.inf
    return new_active, logit, removed
