"""Pins of the oracle's compositing, tile lists, sort, votes and gradients
(no GPU)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import fp32_index as fx
from oracle import step
from oracle.composite import composite
from paper_2506_21117_gb300 import synthetic as S

T64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(x):
    return torch.tensor(np.asarray(x, np.float64), dtype=T64)


def test_single_opaque_gaussian_on_pixel():
    """An opaque Gaussian centred on a pixel centre: C = 0.99 c + 0.01 bg."""
    c = np.array([0.2, 0.5, 0.9])
    bg = np.array([0.3, 0.1, 0.7])
    r = composite(_t([10.5]), _t([7.5]), _t([[0.5, 0.0, 0.5]]), _t([0.9999]), _t([c]),
                  torch.tensor([10]), torch.tensor([7]), _t(bg))
    np.testing.assert_allclose(r["colour"].numpy()[0], 0.99 * c + 0.01 * bg, atol=1e-15)
    assert r["T_final"].item() == pytest.approx(0.01, abs=1e-15)
    assert r["n_contrib"].item() == 1


def test_transmittance_telescopes_to_one():
    """sum_i alpha_i T_i + T_final = 1: white Gaussians on a white background
    composite to exactly 1."""
    rng = np.random.default_rng(0)
    L = 300
    u = rng.uniform(0, 16, L); v = rng.uniform(0, 16, L)
    conic = np.stack([rng.uniform(0.05, 0.5, L), rng.uniform(-0.02, 0.02, L),
                      rng.uniform(0.05, 0.5, L)], 1)
    op = rng.uniform(0.05, 0.6, L)
    xs, ys = np.meshgrid(np.arange(16), np.arange(16))
    r = composite(_t(u), _t(v), _t(conic), _t(op), _t(np.ones((L, 3))),
                  torch.tensor(xs.ravel()), torch.tensor(ys.ravel()), _t([1.0, 1.0, 1.0]))
    np.testing.assert_allclose(r["colour"].numpy(), 1.0, atol=1e-12)
    assert (r["T_final"].numpy() < 1).all()


def test_front_to_back_order_and_swap():
    """Two Gaussians on one pixel: C = a1 c1 + (1 - a1) a2 c2 + T bg; swapping
    their order swaps the roles."""
    c1, c2, bg = np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, 0, 1.0])
    a1, a2 = 0.6, 0.3
    args = dict(px=torch.tensor([3]), py=torch.tensor([4]), bg=_t(bg))
    conic = _t([[0.5, 0, 0.5], [0.5, 0, 0.5]])
    r = composite(_t([3.5, 3.5]), _t([4.5, 4.5]), conic, _t([a1, a2]), _t([c1, c2]), **args)
    ref = a1 * c1 + (1 - a1) * a2 * c2 + (1 - a1) * (1 - a2) * bg
    np.testing.assert_allclose(r["colour"].numpy()[0], ref, atol=1e-15)
    r2 = composite(_t([3.5, 3.5]), _t([4.5, 4.5]), conic, _t([a2, a1]), _t([c2, c1]), **args)
    ref2 = a2 * c2 + (1 - a2) * a1 * c1 + (1 - a1) * (1 - a2) * bg
    np.testing.assert_allclose(r2["colour"].numpy()[0], ref2, atol=1e-15)
    assert not np.allclose(ref, ref2)


def test_early_stop_rule():
    """alpha = 0.98 repeated: T goes 1 -> 0.02 -> 4e-4; the third test
    4e-4 * 0.02 < 1e-4 stops before the third Gaussian."""
    L = 10
    r = composite(_t([2.5] * L), _t([2.5] * L), _t([[0.5, 0, 0.5]] * L), _t([0.98] * L),
                  _t(np.ones((L, 3))), torch.tensor([2]), torch.tensor([2]), _t([0, 0, 0]))
    assert r["n_contrib"].item() == 2
    assert r["T_final"].item() == pytest.approx(4e-4, rel=1e-12)
    assert r["colour"].numpy()[0] == pytest.approx([1 - 4e-4] * 3, abs=1e-15)


def test_low_alpha_skipped():
    r = composite(_t([0.5]), _t([0.5]), _t([[0.5, 0, 0.5]]), _t([0.5 / 255]),
                  _t([[1.0, 1.0, 1.0]]), torch.tensor([0]), torch.tensor([0]), _t([0, 0, 0]))
    assert r["n_contrib"].item() == 0 and r["T_final"].item() == 1.0


def _brute_force_image(scene, cam, sh_degree):
    """Pure-Python per-pixel compositing over all Gaussians (no tile lists):
    a Gaussian is in a pixel's list iff its float32 tile rectangle holds the
    pixel's tile; order by (depth bits, index)."""
    from oracle.projection import project, scene64
    P = project(scene64(scene), cam, sh_degree)
    pidx = fx.project_index(scene, cam)
    u, v = P["u"].numpy(), P["v"].numpy()
    A, B, C = P["conic"].numpy().T
    op, rgb = P["opacity"].numpy(), P["rgb"].numpy()
    W, H = int(cam["width"]), int(cam["height"])
    img = np.zeros((3, H, W))
    n = scene["means"].shape[0]
    for y in range(H):
        for x in range(W):
            tx, ty = x // 16, y // 16
            lst = [g for g in range(n) if pidx["valid"][g] and pidx["tx0"][g] <= tx <= pidx["tx1"][g]
                   and pidx["ty0"][g] <= ty <= pidx["ty1"][g]]
            lst.sort(key=lambda g: (int(pidx["zbits"][g]), g))
            T = 1.0
            col = [0.0, 0.0, 0.0]
            for g in lst:
                dx, dy = x + 0.5 - u[g], y + 0.5 - v[g]
                power = -0.5 * (A[g] * dx * dx + C[g] * dy * dy) - B[g] * dx * dy
                if power > 0:
                    continue
                a = min(0.99, op[g] * math.exp(power))
                if a < 1.0 / 255.0:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                for ch in range(3):
                    col[ch] += rgb[g, ch] * a * T
                T *= 1 - a
            img[:, y, x] = col
    return img


def test_tile_oracle_equals_brute_force_per_pixel():
    scene = S.uniform_scene(60, 1, seed=11)
    scene["log_scales"] += np.float32(1.0)  # bigger splats, several tiles each
    cam = S.ring_cameras(1, 4.0, 40, 24, angles=[0.4])[0]
    ref = _brute_force_image(scene, cam, 1)
    got = step.render(scene, [cam], 1)["image"][0]
    np.testing.assert_allclose(got, ref, atol=1e-12)


def test_untruncated_difference_is_reported_not_gated():
    """Truncation at the 3-sigma tile rectangle: compositing every Gaussian at
    every pixel differs slightly from the truncated image; the size is printed,
    not gated."""
    from oracle.projection import project, scene64
    scene = S.uniform_scene(300, 0, seed=12)
    cam = S.ring_cameras(1, 4.0, 32, 32)[0]
    r = step.render(scene, [cam], 0)
    pidx = r["pidx"][0]
    P = project(scene64(scene), cam, 0)
    ids = np.flatnonzero(pidx["valid"])
    ids = ids[np.lexsort((ids, pidx["zbits"][ids]))]
    xs, ys = np.meshgrid(np.arange(32), np.arange(32))
    t = torch.tensor(ids)
    full = composite(P["u"][t], P["v"][t], P["conic"][t], P["opacity"][t], P["rgb"][t],
                     torch.tensor(xs.ravel()), torch.tensor(ys.ravel()), _t([0, 0, 0]))
    img = full["colour"].detach().numpy().T.reshape(3, 32, 32)
    diff = np.abs(img - r["image"][0]).max()
    print(f"max |untruncated - truncated| = {diff:.3e}")
    assert np.isfinite(diff)


# ---------------------------------------------------------------- votes ---

def _read_vote_golden():
    rows = []
    with open(os.path.join(GOLDEN, "vote_rule.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(tuple(int(x) for x in line.split()))
    return rows


def test_vote_rule_golden_table():
    rows = _read_vote_golden()
    assert len(rows) > 40
    for V, c, o, act in rows:
        assert bool(fx.vote_rule(np.array([c]), np.array([o]), V)[0]) == bool(act), (V, c, o)


def test_all_vote_mode():
    c = np.arange(5)
    assert list(fx.vote_rule(c, np.zeros(5, int), 4, mode=1)) == [False] * 4 + [True]


def test_votes_brute_force():
    """float64 brute-force counting with centres kept away from pixel borders so
    the float32 decision cannot differ."""
    rng = np.random.default_rng(13)
    cams = S.ring_cameras(3, 4.0, 24, 20, angles=[0.0, 1.0, 2.5])
    masks = [(rng.uniform(size=(20, 24)) < 0.4).astype(np.uint8) for _ in cams]
    means = rng.uniform(-2.0, 2.0, (400, 3)).astype(np.float32)
    means[:5] = np.array([0, 0, -10], np.float32)  # behind view 0
    c, o = fx.votes(means, cams, masks)
    keep = np.ones(len(means), bool)
    cb = np.zeros(len(means), int); ob = np.zeros(len(means), int)
    for cam, mask in zip(cams, masks):
        R = np.asarray(cam["R"], np.float32).astype(np.float64)
        t = np.asarray(cam["t"], np.float32).astype(np.float64)
        fxx, fy = float(np.float32(cam["fx"])), float(np.float32(cam["fy"]))
        cx, cy = float(np.float32(cam["cx"])), float(np.float32(cam["cy"]))
        for i, mu in enumerate(means.astype(np.float64)):
            p = R @ mu + t
            if not p[2] > 0.2:
                ob[i] += 1
                continue
            uu, vv = fxx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy
            if min(abs(uu - round(uu)), abs(vv - round(vv))) < 1e-3 or abs(p[2] - 0.2) < 1e-4:
                keep[i] = False
            if 0 <= uu < cam["width"] and 0 <= vv < cam["height"]:
                cb[i] += int(mask[int(math.floor(vv)), int(math.floor(uu))] != 0)
            else:
                ob[i] += 1
    assert keep.sum() > 300
    assert np.array_equal(c[keep], cb[keep]) and np.array_equal(o[keep], ob[keep])
    assert (o[:5] >= 1).all()


# ---------------------------------------------------------- tile lists ---

def _brute_pairs(projs, masks, cams, n):
    keys, vals = [], []
    tile_base, rec_base, _ = fx.batch_layout(cams, n)
    for j, (p, m, cam) in enumerate(zip(projs, masks, cams)):
        Tx, _ = fx.tiles_of(cam)
        for g in range(n):
            if not p["valid"][g]:
                continue
            for ty in range(p["ty0"][g], p["ty1"][g] + 1):
                for tx in range(p["tx0"][g], p["tx1"][g] + 1):
                    if m[ty, tx]:
                        keys.append(((tile_base[j] + ty * Tx + tx) << 32) | int(p["zbits"][g]))
                        vals.append(rec_base[j] + g)
    return keys, vals


def test_pairs_sort_and_ranges_brute_force():
    scene = S.uniform_scene(300, 0, seed=14)
    scene["log_scales"] += np.float32(0.7)
    cams = S.ring_cameras(2, 4.0, 72, 40, angles=[0.0, 2.0])
    active = np.random.default_rng(15).uniform(size=300) < 0.1
    projs = [fx.project_index(scene, c) for c in cams]
    masks = [fx.tile_mask(p, active, c) for p, c in zip(projs, cams)]
    # tile mask brute force
    for p, m, cam in zip(projs, masks, cams):
        Tx, Ty = fx.tiles_of(cam)
        for ty in range(Ty):
            for tx in range(Tx):
                hit = any(p["valid"][g] and active[g] and p["tx0"][g] <= tx <= p["tx1"][g]
                          and p["ty0"][g] <= ty <= p["ty1"][g] for g in range(300))
                assert bool(m[ty, tx]) == hit
    keys, vals, n_tiles = fx.pairs(projs, masks, cams, 300)
    bk, bv = _brute_pairs(projs, masks, cams, 300)
    assert keys.tolist() == bk and vals.tolist() == bv
    assert len(bk) > 100
    sk, sv = fx.sort_pairs(keys, vals)
    order = sorted(range(len(bk)), key=lambda i: bk[i])  # Python's sort is stable
    assert sk.tolist() == [bk[i] for i in order] and sv.tolist() == [bv[i] for i in order]
    rng = fx.tile_ranges(sk, n_tiles)
    for t in range(n_tiles):
        idx = [i for i, k in enumerate(sk.tolist()) if (k >> 32) == t]
        if idx:
            assert rng[t].tolist() == [idx[0], idx[-1] + 1]
        else:
            assert rng[t].tolist() == [0, 0]
    assert fx.key_bits(n_tiles) == 32 + (n_tiles - 1).bit_length()


# ----------------------------------------------------------- gradients ---

def _signature(scene, cams, sh_degree, g):
    r = step.render(scene, cams, sh_degree)
    sig = [(int(p["tx0"][g]), int(p["tx1"][g]), int(p["ty0"][g]), int(p["ty1"][g]),
            bool(p["valid"][g])) for p in r["pidx"]]
    order = [np.argsort(p["zbits"], kind="stable").tobytes() for p in r["pidx"]]
    return sig, order, [a.tobytes() for a in r["n_contrib"]], [a.tobytes() for a in r["n_incl"]]


def test_gradients_match_central_differences():
    """Central differences (h = 1e-5, float64) of the L2 loss on the 500-Gaussian
    two-view workload, for every parameter of the Gaussians with the largest
    gradients; probes whose discrete structure changes between +h and -h are
    excluded and counted."""
    scene, cams, targets = S.workload_fd()
    deg = 1
    ref = step.render(scene, cams, deg, targets=targets, loss="l2", need_grad=True)
    G = ref["grads"]
    mag = np.abs(G["means"]).sum(1) + np.abs(G["opacity_logits"])
    picks = np.argsort(-mag)[:4].tolist() + [int(np.argsort(-mag)[40])]
    h = 1e-5
    checked = excluded = 0
    for g in picks:
        for key in step.PARAM_KEYS:
            arr = scene[key]
            for flat in range(int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1):
                sp = {k: v.astype(np.float64) for k, v in scene.items()}
                sm = {k: v.astype(np.float64) for k, v in scene.items()}
                idx = (g,) + np.unravel_index(flat, arr.shape[1:]) if arr.ndim > 1 else (g,)
                sp[key][idx] += h
                sm[key][idx] -= h
                if _signature(sp, cams, deg, g) != _signature(sm, cams, deg, g):
                    excluded += 1
                    continue
                fd = (step.loss_value(sp, cams, deg, targets, "l2") -
                      step.loss_value(sm, cams, deg, targets, "l2")) / (2 * h)
                ad = G[key][idx]
                assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-10, (key, idx, fd, ad)
                checked += 1
    print(f"finite differences: {checked} checked, {excluded} excluded")
    assert checked >= 100 and excluded <= 0.1 * (checked + excluded)


def test_local_gradient_equals_full_image_gradient():
    """Exactness property: rendering only the tiles touched by O^t gives O^t the
    same gradient as the full image."""
    scene = S.uniform_scene(500, 1, seed=16)
    cams = S.ring_cameras(2, 4.0, 96, 64, angles=[0.0, 0.5 * math.pi])
    targets = [S.random_image(c, 16 + i) for i, c in enumerate(cams)]
    rng = np.random.default_rng(16)
    active = rng.uniform(size=500) < 0.03
    full = step.local_step_reference(scene, cams, 1, targets, active, "l2")
    tiles = step.active_tiles(scene, cams, active)
    loc = step.render(scene, cams, 1, targets=targets, loss="l2", need_grad=True, tiles=tiles)
    for k in step.PARAM_KEYS:
        np.testing.assert_allclose(loc["grads"][k][active], full["grads"][k][active],
                                   rtol=1e-12, atol=1e-18)
    assert sum(len(t) for t in tiles) < sum(fx.tiles_of(c)[0] * fx.tiles_of(c)[1] for c in cams)


def _fd_case():
    scene, cams, targets = S.workload_fd()
    return scene, cams, targets, np.ones(scene["means"].shape[0], bool)


def test_held_pixels_split_the_gradient():
    """Holding pixel colours constant removes exactly their share of the
    gradient: the L2 loss is a sum over pixels, so the gradient with a set H
    held plus the gradient with its complement held is the plain gradient;
    holding nothing changes nothing; holding every pixel gives zero."""
    scene, cams, targets, active = _fd_case()
    plain = step.local_step_reference(scene, cams, 1, targets, active, "l2")
    rng = np.random.default_rng(3)
    H = [rng.uniform(size=(int(c["height"]), int(c["width"]))) < 0.3 for c in cams]
    a = step.local_step_reference(scene, cams, 1, targets, active, "l2", held=H)
    b = step.local_step_reference(scene, cams, 1, targets, active, "l2",
                                  held=[~h for h in H])
    none = step.local_step_reference(scene, cams, 1, targets, active, "l2",
                                     held=[np.zeros_like(h) for h in H])
    every = step.local_step_reference(scene, cams, 1, targets, active, "l2",
                                      held=[np.ones_like(h) for h in H])
    for k in step.PARAM_KEYS:
        g = plain["grads"][k]
        scale = np.abs(g).max()
        np.testing.assert_allclose(a["grads"][k] + b["grads"][k], g, rtol=0, atol=1e-12 * scale)
        assert np.array_equal(none["grads"][k], g)
        assert np.abs(every["grads"][k]).max() == 0.0
        assert np.abs(a["grads"][k] - g).max() > 1e-6 * scale  # the held share is not nothing
    assert a["loss"] == pytest.approx(plain["loss"], rel=1e-15)
    assert all(np.array_equal(x, y) for x, y in zip(a["held"], H))


def test_ambiguous_pixels_are_those_near_a_threshold():
    """A pixel is ambiguous exactly when a reached decision sits within the
    relative margin of its threshold: one Gaussian whose alpha at the pixel is
    (1/255)(1 + d) is ambiguous for |d| below the margin and not above it."""
    for d, want in ((1e-5, True), (-2e-4, True), (1e-3, False), (-5e-3, False)):
        op = 0.5
        power = math.log((1.0 + d) / 255.0 / op)
        dx = math.sqrt(-2.0 * power)  # conic A = 1 along x
        r = composite(_t([5.5 - dx]), _t([5.5]), _t([[1.0, 0.0, 1.0]]), _t([op]),
                      _t([[0.5, 0.5, 0.5]]), torch.tensor([5]), torch.tensor([5]),
                      _t([0.0, 0.0, 0.0]), grad_margin=3e-4)
        assert bool(r["ambiguous"][0]) is want, d


def test_truncated_lists_give_the_same_result():
    """Compositing each tile over the prefix that holds every composited entry
    gives the same gradients and images as the whole list."""
    scene, cams, masks, targets = (lambda s: (s[0], s[2], s[3], None))(
        S.workload_local(n=20000, n_views=2, size=96))
    targets = [S.random_image(c, 9 + j) for j, c in enumerate(cams)]
    active = np.zeros(20000, bool)
    active[::50] = True
    full = step.local_step_reference(scene, cams, 3, targets, active, "l1")
    cut = step.render(scene, cams, 3, targets=targets, loss="l1", need_grad=True,
                      truncate=True)
    for k in step.PARAM_KEYS:
        g = full["grads"][k][active]
        np.testing.assert_allclose(cut["grads"][k][active], g, rtol=0,
                                   atol=1e-13 * np.abs(g).max())
    for x, y in zip(full["image"], cut["image"]):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-13)
    assert all(np.array_equal(x, y) for x, y in zip(full["n_contrib"], cut["n_contrib"]))


def test_float32_evaluation_stays_within_float32_rounding():
    """The oracle's arithmetic in float32 gives pixels within 1e-5 of float64
    and gradients whose largest gap is a small multiple of float32 rounding of
    the group's size (and far from float64 agreement), which is what the
    parity floor is measured with."""
    scene, cams, targets, active = _fd_case()
    r64 = step.local_step_reference(scene, cams, 1, targets, active, "l2")
    r32 = step.local_step_reference(scene, cams, 1, targets, active, "l2",
                                    dtype=torch.float32)
    for a, b, n in zip(r64["image"], r32["image"], r64["near"]):
        assert np.abs(a - b)[:, ~n].max() <= 1e-5
    for k in step.PARAM_KEYS:
        g64, g32 = r64["grads"][k], r32["grads"][k]
        rms = math.sqrt(float(np.mean(g64 * g64)))
        gap = np.abs(g32 - g64).max() / rms
        assert 1e-8 < gap < 1e-3, (k, gap)


def _branch_scene():
    """60 background Gaussians and three that sit on a branch of the image
    formation: A far off-axis (its tangent x/z beyond 1.3 tan(fov/2), so the
    EWA Jacobian uses the clamped tangent) but wide enough to reach the image;
    B with a negative raw red channel (clamped to 0); C nearly opaque in front
    (alpha clamped at 0.99 on its central pixels)."""
    scene = S.uniform_scene(63, 1, seed=91)
    for k in scene:
        scene[k] = np.asarray(scene[k], np.float64).copy()
    A, B, C = 60, 61, 62
    scene["means"][A] = [3.4, 0.1, 0.0]
    scene["log_scales"][A] = [0.05, -0.4, -0.2]
    scene["opacity_logits"][A] = 1.0
    scene["means"][B] = [0.1, -0.05, 0.3]
    scene["log_scales"][B] = [-1.6, -1.7, -1.5]
    scene["sh"][B, 0] = [-2.0, 0.8, 0.4]
    scene["opacity_logits"][B] = 2.0
    scene["means"][C] = [-0.2, 0.15, -1.5]
    scene["log_scales"][C] = [-1.8, -1.7, -1.9]
    scene["opacity_logits"][C] = 8.0
    cams = [S.look_at_camera((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 40)]
    targets = [S.random_image(cams[0], 92)]
    return scene, cams, targets, (A, B, C)


def test_branch_gradients_match_central_differences():
    """Central differences of the L2 loss for every parameter of three
    Gaussians that each sit on one branch (clamped tangent, clamped colour,
    clamped alpha), with the branch checked to be taken; probes whose discrete
    structure changes are excluded and counted."""
    from oracle.projection import project, scene64
    scene, cams, targets, (A, B, C) = _branch_scene()
    P = project(scene64(scene), cams[0], 1)
    pz = (scene["means"] @ np.asarray(cams[0]["R"]).T + cams[0]["t"])[:, 2]
    px = (scene["means"] @ np.asarray(cams[0]["R"]).T + cams[0]["t"])[:, 0]
    lim = 1.3 * 0.5 * cams[0]["width"] / cams[0]["fx"]
    assert abs(px[A] / pz[A]) > lim                              # tangent clamped
    assert float(P["rgb_raw"][B, 0]) < 0 < float(P["rgb_raw"][B, 1])  # red clamped
    u, v = float(P["u"][C]), float(P["v"][C])
    Ac, Bc, Cc = (float(x) for x in P["conic"][C])
    peak = max(float(P["opacity"][C]) * math.exp(
        -0.5 * (Ac * (x + 0.5 - u) ** 2 + Cc * (y + 0.5 - v) ** 2) - Bc * (x + 0.5 - u) * (y + 0.5 - v))
        for x in range(int(u) - 2, int(u) + 3) for y in range(int(v) - 2, int(v) + 3))
    assert peak > 0.99                                           # alpha clamped on a pixel
    ref = step.render(scene, cams, 1, targets=targets, loss="l2", need_grad=True)
    assert ref["n_incl"][0].max() > 0
    p = ref["pidx"][0]
    assert p["valid"][A] and p["tx1"][A] >= 0 and p["tx0"][A] <= 2   # A reaches the image
    G = ref["grads"]
    h = 1e-5
    checked = excluded = 0
    per = {A: 0, B: 0, C: 0}
    for g in (A, B, C):
        for key in step.PARAM_KEYS:
            arr = scene[key]
            for flat in range(int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1):
                sp = {k: v.copy() for k, v in scene.items()}
                sm = {k: v.copy() for k, v in scene.items()}
                idx = (g,) + np.unravel_index(flat, arr.shape[1:]) if arr.ndim > 1 else (g,)
                sp[key][idx] += h
                sm[key][idx] -= h
                if _signature(sp, cams, 1, g) != _signature(sm, cams, 1, g):
                    excluded += 1
                    continue
                fd = (step.loss_value(sp, cams, 1, targets, "l2") -
                      step.loss_value(sm, cams, 1, targets, "l2")) / (2 * h)
                ad = G[key][idx]
                assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-10, (g, key, idx, fd, ad)
                checked += 1
                per[g] += 1
    assert np.abs(G["means"][A]).max() > 1e-4                   # A reaches pixels
    # the clamped red channel takes no gradient through any SH coefficient of B
    assert np.all(G["sh"][B, :, 0] == 0.0)
    assert np.any(G["sh"][B, :, 1] != 0.0)
    print(f"branch finite differences: {checked} checked, {excluded} excluded, per Gaussian {per}")
    assert min(per.values()) >= 15 and excluded <= 0.15 * (checked + excluded)
