"""Pins of the densification oracle (base 3DGS adaptive density control
restricted to O^t; Supp. "History Recovery", "Implementation Details")."""
import numpy as np

from oracle import densify as od


def _scene(n=6):
    means = np.zeros((n, 3), np.float32)
    ls = np.full((n, 3), np.log(0.005), np.float32)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    logits = np.zeros(n, np.float32)
    return means, ls, quats, logits


def test_clone_split_prune_rules():
    means, ls, quats, logits = _scene()
    extent = 1.0  # clone if largest scale <= 0.01
    ls[1] = np.log(0.05)          # big enough to split
    ls[2] = np.log(0.05)          # large but low gradient: untouched
    logits[3] = -10.0             # low opacity: pruned
    ls[4] = np.log(0.005)         # clone candidate with low opacity: pruned, no clone
    logits[4] = -10.0
    active = np.array([0, 1, 2, 3, 4])
    accum = np.array([1e-3, 1e-3, 1e-5, 1e-3, 1e-3, 0], np.float32)
    denom = np.array([2, 2, 2, 2, 2, 0], np.float32)
    z = np.zeros((5, 2, 3), np.float32)
    out = od.densify(means, ls, quats, logits, active, accum, denom, np.zeros(6), extent, z,
                     big=False)
    assert sorted(out["removed"].tolist()) == [1, 3, 4]
    assert out["src"].tolist() == [0, 1, 1]           # clone of 0, two children of 1
    np.testing.assert_allclose(out["log_scales"][1:], np.log(0.05 / 1.6), rtol=1e-6)
    assert np.all(out["means"] == 0)                   # z = 0: children at the centre


def test_split_children_are_samples_of_the_gaussian():
    means, ls, quats, logits = _scene(1)
    means[0] = [1, 2, 3]
    ls[0] = np.log([0.2, 0.1, 0.05])
    quats[0] = [np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)]  # 90 degrees about z
    z = np.array([[[1, 0, 0], [0, 1, 0]]], np.float32)
    out = od.densify(means, ls, quats, logits, np.array([0]), np.array([1.0], np.float32),
                     np.array([1.0], np.float32), np.zeros(1), 1.0, z, big=False)
    # R maps x to y and y to -x
    np.testing.assert_allclose(out["means"][0], [1, 2.2, 3], atol=1e-6)
    np.testing.assert_allclose(out["means"][1], [0.9, 2, 3], atol=1e-6)


def test_big_rule_only_after_reset():
    means, ls, quats, logits = _scene(2)
    maxr = np.array([30.0, 5.0])
    acc = np.zeros(2, np.float32)
    den = np.zeros(2, np.float32)
    z = np.zeros((2, 2, 3), np.float32)
    a = od.densify(means, ls, quats, logits, np.array([0, 1]), acc, den, maxr, 1.0, z, big=False)
    b = od.densify(means, ls, quats, logits, np.array([0, 1]), acc, den, maxr, 1.0, z, big=True)
    assert a["removed"].size == 0 and b["removed"].tolist() == [0]


def test_accumulate_ndc_norm():
    acc = np.zeros(3, np.float32)
    den = np.zeros(3, np.float32)
    mr = np.zeros(3)
    od.accumulate(acc, den, mr, [0, 1, 2], [1e-3, 2e-3, 5.0], [0.0, 1e-3, 5.0], [3, 4, 0], 200, 100)
    np.testing.assert_allclose(acc, [0.1, np.hypot(0.2, 0.05), 0.0], rtol=1e-6)
    assert den.tolist() == [1, 1, 0] and mr.tolist() == [3, 4, 0]


def test_accumulate_per_view_loss_scaling():
    """With the batch loss the mean over 4 views, one view's own gradient is
    4 x the batch gradient."""
    acc = np.zeros(1, np.float32)
    den = np.zeros(1, np.float32)
    mr = np.zeros(1)
    od.accumulate(acc, den, mr, [0], [1e-3], [0.0], [1], 200, 100, n_views=4)
    np.testing.assert_allclose(acc, [0.4], rtol=1e-6)


def test_opacity_reset_caps_sigmoid():
    logits = np.array([-8.0, -4.0, 0.0, 3.0, 5.0], np.float32)
    out = od.reset_opacity(logits, [1, 2, 3])
    sig = lambda x: 1 / (1 + np.exp(-np.asarray(x, np.float64)))
    np.testing.assert_allclose(sig(out[1:4]), np.minimum(sig(logits[1:4]), 0.01), rtol=1e-6)
    assert out[0] == logits[0] and out[4] == logits[4]


def test_history_recovers_after_densification():
    """Densification only appends rows after the static ones and tombstones rows
    of O^t, so History Recovery still rebuilds G^{t-1} exactly (Supp. "History
    Recovery": duplication and pruning only affect O^t)."""
    from oracle import history as oh
    rng = np.random.default_rng(7)
    n = 300
    means = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    ls = rng.uniform(-6, -1, (n, 3)).astype(np.float32)
    quats = rng.standard_normal((n, 4)).astype(np.float32)
    logits = rng.uniform(-7, 3, n).astype(np.float32)
    rows = np.concatenate([means, logits[:, None], ls, np.zeros((n, 1), np.float32), quats],
                          axis=1)
    I = rng.uniform(size=n) < 0.3
    g_t, entry = oh.begin_update(rows, I)
    k = int((~I).sum())
    A = np.arange(k, n)                                   # O^t is the tail
    accum = (rng.uniform(0, 1e-3, n) * 4).astype(np.float32)
    denom = np.full(n, 4, np.float32)
    z = rng.standard_normal((A.size, 2, 3)).astype(np.float32)
    out = od.densify(g_t[:, 0:3], g_t[:, 4:7], g_t[:, 8:12], g_t[:, 3], A, accum, denom,
                     np.zeros(n), 2.0, z, big=False)
    assert out["src"].size > 0 and out["removed"].size > 0
    new = g_t[out["src"]].copy()
    new[:, 0:3] = out["means"]
    new[:, 4:7] = out["log_scales"]
    g_after = np.concatenate([g_t, new])
    g_after[out["removed"], 3] = -np.inf                  # tombstones inside O^t
    assert np.all(out["removed"] >= k)                    # static rows untouched
    back = oh.recover(g_after, entry)
    assert np.array_equal(back.view(np.uint32), rows.view(np.uint32))
