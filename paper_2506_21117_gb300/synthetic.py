"""Seeded synthetic inputs shaped like the paper's local-update workloads.

This module draws scenes, cameras, change boxes and binary change masks. It is
shared by the tests, the benchmark and the oracle harness, and it holds none of
the method's arithmetic: no projection of Gaussians, no compositing, no voting,
no optimizer. Everything is drawn with NumPy's PCG64 (`default_rng(seed)`) in
float64 and cast once to float32.

Scene shapes follow the workloads the paper describes: 3DGS scenes with
spherical-harmonics colour (Sec. 3, Supp. "Implementation Details": the base
3DGS parameterisation of mean, log-scale, rotation quaternion, opacity logit and
SH coefficients), a handful of new posed views (Sec. 3, "Detecting Changes in
2D"), and a local change that covers a small fraction of the scene (Supp.
"Dataset": changes of 10-20%, 1-2% and under 1% of the scene).

A scene is a dict of float32 arrays:
  means   [n, 3]        log_scales [n, 3]     quats [n, 4] (w, x, y, z)
  opacity_logits [n]    sh [n, K, 3] with K = (degree + 1)^2
A camera is a dict with R (3x3 world-to-camera), t (3), pos (3), fx, fy, cx,
cy, znear, width, height (float64 / int).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

Scene = Dict[str, np.ndarray]
Camera = Dict[str, object]

ZNEAR = 0.2


def sh_coeff_count(degree: int) -> int:
    return (degree + 1) * (degree + 1)


def _dc_from_colour(colour: np.ndarray) -> np.ndarray:
    # A DC coefficient d shows as colour d / (2 sqrt(pi)) + 0.5 under the base
    # method's degree-0 convention; draw colours U(0,1) and store that d.
    return (colour - 0.5) * (2.0 * math.sqrt(math.pi))


def _random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _finish(rng, means, sh_degree, higher_sigma=0.1) -> Scene:
    n = means.shape[0]
    log_scales = rng.normal(-3.0, 0.3, size=(n, 3))
    quats = _random_quats(rng, n)
    opacity_logits = rng.standard_normal(n)
    k = sh_coeff_count(sh_degree)
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = _dc_from_colour(rng.uniform(0.0, 1.0, size=(n, 3)))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_sigma, size=(n, k - 1, 3))
    return {
        "means": means.astype(np.float32),
        "log_scales": log_scales.astype(np.float32),
        "quats": quats.astype(np.float32),
        "opacity_logits": opacity_logits.astype(np.float32),
        "sh": sh.astype(np.float32),
    }


def uniform_scene(n: int, sh_degree: int = 0, seed: int = 0) -> Scene:
    """Means U[-1,1]^3, log-scales N(-3,0.3), random unit quaternions,
    opacity logits N(0,1), DC colours U(0,1), higher SH N(0,0.1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    return _finish(rng, means, sh_degree)


def cluster_scene(n: int, n_clusters: int = 20, sigma: float = 0.3,
                  centre_extent: float = 4.0, room: float = 5.0,
                  sh_degree: int = 3, seed: int = 0) -> Tuple[Scene, np.ndarray]:
    """Means from a mixture of isotropic clusters (centres U[-4,4]^3,
    std `sigma`) clipped to a [-room, room]^3 room. Returns (scene, centres)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-centre_extent, centre_extent, size=(n_clusters, 3))
    which = rng.integers(0, n_clusters, size=n)
    means = centres[which] + rng.normal(0.0, sigma, size=(n, 3))
    means = np.clip(means, -room, room)
    return _finish(rng, means, sh_degree), centres


def look_at_camera(pos: Sequence[float], target: Sequence[float], width: int,
                   height: int, fov_x_deg: float = 60.0,
                   znear: float = ZNEAR) -> Camera:
    """Pinhole camera at `pos` looking at `target`, world up +y.

    Camera axes: x right, y down, z forward. Focal lengths are equal and set by
    the horizontal field of view; the principal point is the image centre, so
    pixel (i, j) covers [i, i+1) x [j, j+1) in image coordinates."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return {
        "R": R, "t": t, "pos": pos, "fx": fx, "fy": fx,
        "cx": width / 2.0, "cy": height / 2.0, "znear": znear,
        "width": int(width), "height": int(height),
    }


def ring_cameras(n_views: int, radius: float, width: int, height: int,
                 fov_x_deg: float = 60.0, angles: Sequence[float] | None = None
                 ) -> List[Camera]:
    """Cameras on the y = 0 ring of `radius`, looking at the origin. Angle 0 is
    the position (0, 0, -radius)."""
    if angles is None:
        angles = [2.0 * math.pi * k / n_views for k in range(n_views)]
    cams = []
    for a in angles:
        pos = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        cams.append(look_at_camera(pos, (0.0, 0.0, 0.0), width, height, fov_x_deg))
    return cams


def cube_box(centre: Sequence[float], edge: float) -> Tuple[np.ndarray, np.ndarray]:
    c = np.asarray(centre, dtype=np.float64)
    return c - edge / 2.0, c + edge / 2.0


def random_box_in_unit_cube(fraction: float = 0.05, seed: int = 0
                            ) -> Tuple[np.ndarray, np.ndarray]:
    """Axis-aligned cube holding `fraction` of the volume of [-1,1]^3, centre
    uniform so the cube stays inside [-1,1]^3."""
    rng = np.random.default_rng(seed + 1)
    edge = 2.0 * fraction ** (1.0 / 3.0)
    half = 1.0 - edge / 2.0
    centre = rng.uniform(-half, half, size=3)
    return cube_box(centre, edge)


def box_holding_fraction(means: np.ndarray, centre: Sequence[float],
                         fraction: float) -> Tuple[np.ndarray, np.ndarray]:
    """Cube around `centre` whose edge is bisected so it holds `fraction` of
    the means."""
    m = means.astype(np.float64)
    c = np.asarray(centre, dtype=np.float64)
    cheb = np.max(np.abs(m - c), axis=1)
    k = max(1, int(round(fraction * m.shape[0])))
    half = float(np.partition(cheb, k - 1)[k - 1]) * (1.0 + 1e-9)
    return c - half, c + half


def change_cluster(centres: np.ndarray, cams: Sequence[Camera]) -> np.ndarray:
    """The cluster centre seen by the most views (in front by more than 1 unit
    and inside the image), ties broken by the smallest angle to the first
    camera's optical axis."""
    best, best_key = None, None
    for c in centres:
        seen = 0
        for cam in cams:
            R = np.asarray(cam["R"])
            p = R @ c + np.asarray(cam["t"])
            if p[2] > 1.0:
                u = cam["fx"] * p[0] / p[2] + cam["cx"]
                v = cam["fy"] * p[1] / p[2] + cam["cy"]
                seen += int(0 < u < cam["width"] and 0 < v < cam["height"])
        p0 = np.asarray(cams[0]["R"]) @ c + np.asarray(cams[0]["t"])
        ang = math.hypot(p0[0], p0[1]) / p0[2] if p0[2] > 1e-9 else math.inf
        key = (-seen, ang)
        if best_key is None or key < best_key:
            best, best_key = c, key
    return np.asarray(best)


def inside_box(means: np.ndarray, box: Tuple[np.ndarray, np.ndarray]) -> np.ndarray:
    lo, hi = box
    m = means.astype(np.float64)
    return np.all((m >= lo) & (m <= hi), axis=1)


def box_change_mask(cam: Camera, box: Tuple[np.ndarray, np.ndarray]) -> np.ndarray:
    """uint8 [H, W]: 1 where the ray through the pixel centre hits the box
    (slab test in float64)."""
    W, H = int(cam["width"]), int(cam["height"])
    R = np.asarray(cam["R"], dtype=np.float64)
    pos = np.asarray(cam["pos"], dtype=np.float64)
    i = (np.arange(W) + 0.5 - cam["cx"]) / cam["fx"]
    j = (np.arange(H) + 0.5 - cam["cy"]) / cam["fy"]
    dc = np.stack(np.broadcast_arrays(i[None, :], j[:, None], np.ones((H, W))), axis=-1)
    d = dc @ R  # camera-to-world: R^T applied to row vectors
    lo, hi = box
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (lo - pos) * inv
        t1 = (hi - pos) * inv
    tmin = np.nanmax(np.minimum(t0, t1), axis=-1)
    tmax = np.nanmin(np.maximum(t0, t1), axis=-1)
    hit = (tmax >= np.maximum(tmin, 0.0))
    return hit.astype(np.uint8)


def perturb_scene(scene: Scene, which: np.ndarray, sigma: float = 0.05,
                  seed: int = 0) -> Scene:
    """Copy of `scene` where every parameter of the Gaussians in `which` gets
    N(0, sigma) noise (the changed target scene)."""
    rng = np.random.default_rng(seed + 2)
    out = {k: v.copy() for k, v in scene.items()}
    idx = np.flatnonzero(which)
    for k, v in out.items():
        noise = rng.normal(0.0, sigma, size=(idx.size,) + v.shape[1:])
        v[idx] = (v[idx].astype(np.float64) + noise).astype(np.float32)
    return out


def random_image(cam: Camera, seed: int = 0) -> np.ndarray:
    """float32 [3, H, W] uniform in [0, 1)."""
    rng = np.random.default_rng(seed + 3)
    return rng.uniform(0.0, 1.0, size=(3, int(cam["height"]), int(cam["width"]))
                       ).astype(np.float32)


def random_adam_state(n: int, width: int, seed: int = 0):
    """Seeded parameter, moment and gradient arrays for optimizer unit tests."""
    rng = np.random.default_rng(seed + 4)
    theta = rng.standard_normal((n, width)).astype(np.float32)
    m = (rng.standard_normal((n, width)) * 1e-2).astype(np.float32)
    v = (rng.uniform(0.0, 1e-3, size=(n, width))).astype(np.float32)
    g = (rng.standard_normal((n, width)) * 1e-2).astype(np.float32)
    return theta, m, v, g


# --- the workloads the tests and the benchmark use --------------------------

def workload_plain(seed: int = 0):
    """2,000 Gaussians, SH degree 0, one 64x64 view at distance 4, random
    target, every Gaussian active."""
    scene = uniform_scene(2000, 0, seed)
    cams = ring_cameras(1, 4.0, 64, 64, angles=[0.0])
    target = [random_image(cams[0], seed)]
    return scene, cams, target


def workload_local(n: int = 100_000, n_views: int = 8, size: int = 800,
                   fraction: float = 0.05, sh_degree: int = 3, seed: int = 0):
    """Uniform scene, ring views, a random box holding about `fraction` of the
    unit cube; returns (scene, target_scene, cams, masks, box)."""
    scene = uniform_scene(n, sh_degree, seed)
    cams = ring_cameras(n_views, 4.0, size, size)
    box = random_box_in_unit_cube(fraction, seed)
    changed = inside_box(scene["means"], box)
    target_scene = perturb_scene(scene, changed, 0.05, seed)
    masks = [box_change_mask(c, box) for c in cams]
    return scene, target_scene, cams, masks, box


def workload_large(n: int = 1_000_000, n_views: int = 4, width: int = 1920,
                   height: int = 1080, fraction: float = 0.05,
                   sh_degree: int = 3, seed: int = 0):
    """Clustered room scene, views at 0, pi/2, pi, 3pi/2, a change box around
    the cluster seen by the most views (nearest view 0's image centre among
    those) holding `fraction` of the Gaussians; returns (scene, target_scene,
    cams, masks, box)."""
    scene, centres = cluster_scene(n, 20, 0.3, 4.0, 5.0, sh_degree, seed)
    angles = [0.5 * math.pi * k for k in range(n_views)]
    cams = ring_cameras(n_views, 4.0, width, height, angles=angles)
    centre = change_cluster(centres, cams)
    box = box_holding_fraction(scene["means"], centre, fraction)
    changed = inside_box(scene["means"], box)
    target_scene = perturb_scene(scene, changed, 0.05, seed)
    masks = [box_change_mask(c, box) for c in cams]
    return scene, target_scene, cams, masks, box


def workload_fd(seed: int = 0):
    """500 Gaussians, SH degree 1, two 32x32 views at angles 0 and pi/2,
    random targets."""
    scene = uniform_scene(500, 1, seed)
    cams = ring_cameras(2, 4.0, 32, 32, angles=[0.0, 0.5 * math.pi])
    targets = [random_image(c, seed + i) for i, c in enumerate(cams)]
    return scene, cams, targets


def workload_addition(n: int = 100_000, n_views: int = 8, size: int = 800,
                      fraction: float = 0.05, sh_degree: int = 3, seed: int = 0):
    """An object appears: the uniform scene with every Gaussian inside a random
    box removed (so lifting finds almost nothing there), ring views whose change
    masks are the box's projection. Returns (scene, cams, masks, box)."""
    scene = uniform_scene(n, sh_degree, seed)
    box = random_box_in_unit_cube(fraction, seed)
    keep = ~inside_box(scene["means"], box)
    scene = {k: v[keep] for k, v in scene.items()}
    cams = ring_cameras(n_views, 4.0, size, size)
    masks = [box_change_mask(c, box) for c in cams]
    return scene, cams, masks, box


def sampling_draws(seed: int = 0):
    """The random numbers new-point sampling consumes, as a function
    (round, kind, shape) -> float32 array: kind "box" and "comp" uniform in
    [0, 1), "normal" standard normal; each (round, kind) has its own stream."""
    codes = {"box": 1, "comp": 2, "normal": 3}
    below_one = np.nextafter(np.float32(1.0), np.float32(0.0))

    def draws(round_: int, kind: str, shape):
        rng = np.random.default_rng([seed, round_, codes[kind]])
        if kind == "normal":
            return rng.standard_normal(shape).astype(np.float32)
        return np.minimum(rng.random(shape).astype(np.float32), below_one)
    return draws


def densify_draws(seed: int = 0):
    """The standard normals the split of densification consumes, as a
    function (step, n_active) -> float32 [n_active][2][3]; each densification
    step has its own stream."""
    def draws(step: int, n_active: int):
        rng = np.random.default_rng([seed, step, 4])
        return rng.standard_normal((n_active, 2, 3)).astype(np.float32)
    return draws


def serving_scenes(n_scenes: int = 64, n_lo: int = 50_000, n_hi: int = 500_000,
                   sh_degree: int = 3, seed: int = 0):
    """Resident scenes of the serving workload: Gaussian counts log-uniform in
    [n_lo, n_hi], each a clustered room like the large workload with the
    cluster count scaled to its size. Returns (scenes, centres)."""
    rng = np.random.default_rng(seed + 10)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_scenes)).astype(int)
    scenes, centres = [], []
    for i, n in enumerate(ns):
        k = max(2, int(round(20 * n / 1_000_000)))
        sc, c = cluster_scene(int(n), k, 0.3, 4.0, 5.0, sh_degree, seed + 100 + i)
        scenes.append(sc)
        centres.append(c)
    return scenes, centres


SERVING_RESOLUTIONS = [(640, 480), (800, 800), (1280, 720)]


def serving_templates(scenes, centres, n_templates: int = 32, seed: int = 0):
    """Update requests of the serving workload: a scene drawn uniformly, one of
    its clusters as the changed region, 2-8 views of it on a ring of radius 3
    around the cluster centre (random phase, every view looking at the
    centre, as new photos of a changed spot would), one of three resolutions,
    and a change box around the centre holding 1-10% of the scene's
    Gaussians, seen by every view so that lifting finds it. Returns dicts with
    scene, cams, masks (list of H x W uint8)."""
    rng = np.random.default_rng(seed + 20)
    out = []
    for _ in range(n_templates):
        s = int(rng.integers(0, len(scenes)))
        V = int(rng.integers(2, 9))
        W, H = SERVING_RESOLUTIONS[int(rng.integers(0, len(SERVING_RESOLUTIONS)))]
        centre = np.asarray(centres[s][int(rng.integers(0, len(centres[s])))], np.float64)
        phase = float(rng.uniform(0, 2 * math.pi))
        cams = []
        for k in range(V):
            a = phase + 2 * math.pi * k / V
            pos = centre + 3.0 * np.array([math.sin(a), 0.0, -math.cos(a)])
            cams.append(look_at_camera(pos, centre, W, H))
        frac = float(rng.uniform(0.01, 0.10))
        box = box_holding_fraction(scenes[s]["means"], centre, frac)
        masks = [box_change_mask(c, box) for c in cams]
        out.append({"scene": s, "cams": cams, "masks": masks, "fraction": frac})
    return out


def poisson_arrivals(rate: float, duration: float, n_templates: int, seed: int = 0):
    """Arrival offsets (seconds) of a Poisson stream and the template of each."""
    rng = np.random.default_rng(seed + 30)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration:
            return out
        out.append((t, int(rng.integers(0, n_templates))))
