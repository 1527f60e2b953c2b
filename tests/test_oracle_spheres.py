"""Pins of the sphere-region oracle (Sec. 3.3 "Sphere Pruning"; Supp.
"Identifying Changed Gaussians", "3DGS Optimization in Changed Regions")
against closed forms, library special cases and brute force."""
import numpy as np
import pytest

from oracle import spheres as sp


def _blobs(seed=0, n=(1500, 1200, 900), centres=((-3, 0, 0), (2, 2, 0), (0, -2, 3)), s=0.2):
    rng = np.random.default_rng(seed)
    pts, lab = [], []
    for i, (c, m) in enumerate(zip(centres, n)):
        pts.append(np.asarray(c) + s * rng.standard_normal((m, 3)))
        lab.append(np.full(m, i))
    perm = rng.permutation(sum(n))
    return (np.concatenate(pts)[perm].astype(np.float32), np.concatenate(lab)[perm])


def test_kmeans_recovers_separated_blobs_and_their_means():
    pts, truth = _blobs()
    labels, centers = sp.kmeans(pts, 3)
    # one-to-one between clusters and blobs
    pairs = {(int(a), int(b)) for a, b in zip(labels, truth)}
    assert len(pairs) == 3 and len({a for a, _ in pairs}) == 3
    for k in range(3):
        m = labels == k
        np.testing.assert_allclose(centers[k], pts[m].astype(np.float64).mean(0), atol=1e-6)


def test_cluster_means_do_not_depend_on_point_order():
    pts, truth = _blobs(seed=1)
    labels = truth.astype(np.int32)
    c0 = np.zeros((3, 3), np.float32)
    a = sp.cluster_means(pts, labels, c0)
    perm = np.random.default_rng(2).permutation(pts.shape[0])
    b = sp.cluster_means(pts[perm], labels[perm], c0)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_assignment_ties_go_to_the_lowest_cluster():
    centers = np.array([[1, 0, 0], [-1, 0, 0], [0, 5, 0]], np.float32)
    pts = np.array([[0, 0, 0], [0.5, 0, 0], [-0.5, 0, 0]], np.float32)
    assert sp.assign(pts, centers).tolist() == [0, 0, 1]


def test_empty_cluster_keeps_its_centre():
    pts = np.array([[0, 0, 0], [0.1, 0, 0]], np.float32)
    c = np.array([[0, 0, 0], [9, 9, 9]], np.float32)
    out = sp.cluster_means(pts, np.array([0, 0], np.int32), c)
    assert np.array_equal(out[1], c[1])


@pytest.mark.parametrize("n", [1, 2, 3, 50, 1001, 4097])
def test_quantile_is_numpys_linear_estimator(n):
    d = np.random.default_rng(n).exponential(size=n).astype(np.float32)
    ref = float(np.quantile(d.astype(np.float64), 0.98))
    assert sp.quantile_linear(d, 0.98) == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_sphere_of_a_shell_has_radius_1p1_R():
    """Points on a sphere shell of radius R around c: mean c (symmetric
    antipodal pairs), every distance R, so the radius is 1.1 R."""
    rng = np.random.default_rng(3)
    v = rng.standard_normal((1000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    R, c = 0.75, np.array([1.0, -2.0, 0.5])
    pts = np.concatenate([c + R * v, c - R * v]).astype(np.float32)
    s = sp.fit_spheres(pts, 1)
    np.testing.assert_allclose(s["centers"][0], c, atol=1e-6)
    assert s["radii"][0] == pytest.approx(1.1 * R, rel=1e-5)
    assert s["counts"][0] == 2000


def test_inside_matches_brute_force_and_boundary():
    spheres = {"centers": np.array([[0, 0, 0], [5, 0, 0], [9, 9, 9]], np.float32),
               "radii": np.array([1.0, 2.0, -1.0], np.float32)}
    pts = np.array([[0.999, 0, 0], [1.001, 0, 0], [5, 1.999, 0], [5, 2.001, 0], [9, 9, 9],
                    [0, 0, 1.0]], np.float32)
    assert sp.inside(pts, spheres).tolist() == [True, False, True, False, False, True]
    rng = np.random.default_rng(4)
    q = rng.uniform(-3, 8, (500, 3)).astype(np.float32)
    brute = (np.linalg.norm(q[:, None, :2 * 0 + 3] - spheres["centers"][None, :2], axis=2)
             <= spheres["radii"][None, :2]).any(1)
    far = np.abs(np.linalg.norm(q[:, None] - spheres["centers"][None, :2], axis=2) -
                 spheres["radii"][None, :2]).min(1) > 1e-5
    assert np.array_equal(sp.inside(q, spheres)[far], brute[far])


def test_n_clusters_reading():
    assert [sp.n_clusters(a) for a in (0, 1, 999, 1000, 2500, 9999, 10000, 10**6)] == \
        [1, 1, 1, 1, 2, 9, 10, 10]


def test_prune_removes_only_active_gaussians_outside():
    means = np.array([[0, 0, 0], [3, 0, 0], [0.5, 0, 0], [7, 7, 7]], np.float32)
    logit = np.array([0.1, 0.2, 0.3, 0.4], np.float32)
    active = np.array([True, True, False, False])
    spheres = {"centers": np.array([[0, 0, 0]], np.float32), "radii": np.array([1.0], np.float32)}
    new_active, new_logit, removed = sp.prune(means, logit, active, spheres)
    assert removed.tolist() == [1]
    assert new_active.tolist() == [True, False, False, False]
    assert new_logit[1] == -np.inf and np.array_equal(new_logit[[0, 2, 3]], logit[[0, 2, 3]])


def test_farthest_point_init_brute_force():
    rng = np.random.default_rng(5)
    pts = rng.uniform(-1, 1, (40, 3)).astype(np.float32)
    got = sp.farthest_point_init(pts, 4)
    chosen = [0]
    for _ in range(3):
        best, arg = -1.0, -1
        for j in range(40):
            d = min(float(np.sum((pts[j].astype(np.float64) - pts[c]) ** 2)) for c in chosen)
            if d > best + 1e-9:
                best, arg = d, j
        chosen.append(arg)
    assert np.array_equal(got, pts[chosen])
