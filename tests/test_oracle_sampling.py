"""Pins of the new-point sampling oracle (Sec. 3.2 "Gaussian Sampling for New
Objects", its New Point Sampling algorithm and Supp. Full-Scene / Region Point
Sampling) against closed forms and brute force."""
import numpy as np
import pytest

from oracle import fp32_index as fx
from oracle import sampling as osa
from oracle import spheres as osp
from paper_2506_21117_gb300 import synthetic as S


def test_box_sample_spans_the_bounding_box():
    rng = np.random.default_rng(0)
    means = rng.uniform(-2, 3, (500, 3)).astype(np.float32)
    lo, hi = osa.bbox(means)
    assert np.array_equal(lo, means.min(0)) and np.array_equal(hi, means.max(0))
    u = np.array([[0, 0, 0], [0.5, 0.5, 0.5]], np.float32)
    p = osa.box_sample(lo, hi, u)
    assert np.array_equal(p[0], lo)
    np.testing.assert_allclose(p[1], (lo.astype(np.float64) + hi) / 2, atol=1e-6)
    q = osa.box_sample(lo, hi, S.sampling_draws(1)(0, "box", (1000, 3)))
    assert np.all(q >= lo) and np.all(q <= hi)


def test_mixture_component_rule_brute_force():
    counts = np.array([3, 0, 5, 2])
    centres = np.arange(12, dtype=np.float32).reshape(4, 3)
    absv = np.zeros((4, 3), np.float32)
    u = np.linspace(0, 0.999, 200).astype(np.float32)
    p = osa.mixture_sample(centres, absv, counts, u, np.zeros((200, 3), np.float32))
    for ui, pi in zip(u, p):
        t = int(np.floor(float(ui) * 10))
        j = next(k for k in range(4) if t < counts[:k + 1].sum())
        assert np.array_equal(pi, centres[j])  # z = 0: the component's centre
    assert not any(np.array_equal(pi, centres[1]) for pi in p)  # empty cluster never drawn


def test_mixture_standard_deviation_is_sqrt_abs_v():
    centres = np.zeros((1, 3), np.float32)
    absv = np.array([[0.25, 4.0, 1.0]], np.float32)
    z = np.array([[1, 1, 1], [-2, 0.5, 3]], np.float32)
    p = osa.mixture_sample(centres, absv, np.array([7]), np.array([0.1, 0.9], np.float32), z)
    np.testing.assert_allclose(p, z * np.array([0.5, 2.0, 1.0], np.float32), rtol=1e-7)


def test_region_mixture_furthest_points_brute_force():
    rng = np.random.default_rng(2)
    pts = np.concatenate([rng.normal(c, 0.1, (300, 3)) for c in ([0, 0, 0], [2, 0, 0], [0, 2, 0])]
                         ).astype(np.float32)
    c, v, k = osa.region_mixture(pts)
    labels, centres = osp.kmeans(pts, min(10, pts.shape[0]))
    assert np.array_equal(c, centres) and k.sum() == pts.shape[0]
    for j in range(c.shape[0]):
        m = np.flatnonzero(labels == j)
        if m.size == 0:
            continue
        d = [float(np.sum((pts[i].astype(np.float64) - centres[j]) ** 2)) for i in m]
        far = m[int(np.argmax(d))]
        np.testing.assert_allclose(v[j], np.abs(pts[far] - centres[j]), atol=1e-6)


def _addition():
    scene, cams, masks, box = S.workload_addition(n=20000, n_views=6, size=96, seed=3)
    return scene, cams, masks, box


def test_sampling_from_nothing_fills_the_changed_region():
    scene, cams, masks, box = _addition()
    out = osa.sample_points(np.zeros((0, 3), np.float32), scene["means"], cams, masks, 400,
                            S.sampling_draws(0))
    pts = out["points"]
    assert pts.shape[0] >= 400 and 2 <= out["rounds"] <= osa.MAX_ROUNDS
    assert out["new"].shape[0] == pts.shape[0]
    # every kept point passes the vote
    c2, o2 = fx.votes(pts, cams, masks)
    assert fx.vote_rule(c2, o2, len(cams)).all()
    # the vote keeps points near the box: most lie inside it (grown by its half edge)
    lo, hi = box
    pad = 0.5 * (hi - lo)
    inside = np.all((pts >= lo - pad) & (pts <= hi + pad), axis=1)
    assert inside.mean() > 0.9


def test_sampling_extends_a_small_active_set():
    scene, cams, masks, box = _addition()
    lo, hi = box
    rng = np.random.default_rng(4)
    seeds = rng.uniform(lo, hi, (30, 3)).astype(np.float32)
    out = osa.sample_points(seeds, scene["means"], cams, masks, 300, S.sampling_draws(1))
    assert np.array_equal(out["points"][:30], seeds)
    assert out["new"].shape[0] == out["points"].shape[0] - 30 >= 270


def test_knn_mean_sq_brute_force_and_small_sets():
    rng = np.random.default_rng(5)
    p = rng.uniform(0, 1, (60, 3)).astype(np.float32)
    got = osa.knn_mean_sq(p)
    d2 = ((p[:, None].astype(np.float64) - p[None]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    ref = np.sort(d2, axis=1)[:, :3].mean(1)
    np.testing.assert_allclose(got, ref, rtol=1e-5)
    assert osa.knn_mean_sq(p[:1])[0] == np.float32(1e-7)
    two = osa.knn_mean_sq(np.array([[0, 0, 0], [3, 4, 0]], np.float32))
    assert np.allclose(two, 25.0)


def test_init_gaussians_base_defaults():
    p = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0], [0, 0, 3]], np.float32)
    g = osa.init_gaussians(p, 3)
    assert np.allclose(1 / (1 + np.exp(-g["opacity_logits"])), 0.1)
    assert np.all(g["quats"] == np.array([1, 0, 0, 0], np.float32))
    assert g["sh"].shape == (4, 16, 3) and not g["sh"].any()
    d = osa.knn_mean_sq(p)
    np.testing.assert_allclose(g["log_scales"][:, 0], 0.5 * np.log(d), rtol=1e-6)
    assert np.all(g["log_scales"] == g["log_scales"][:, :1])
