"""Host-side accounting of the benchmark (no GPU): the walked-evaluation
counts behind the render roofline equal a per-pixel brute force."""
import os
import types

import numpy as np
import pytest
import torch

import bench
from paper_2506_21117_gb300 import _abi as abi


def _fake_batch(seed=0, sizes=((40, 20), (33, 17))):
    rng = np.random.default_rng(seed)
    views = (abi.ClsView * len(sizes))()
    pix = tiles = 0
    for j, (W, H) in enumerate(sizes):
        v = views[j]
        v.cam.width, v.cam.height = W, H
        v.tiles_x, v.tiles_y = -(-W // 16), -(-H // 16)
        v.pix_base, v.tile_base = pix, tiles
        pix += W * H
        tiles += v.tiles_x * v.tiles_y
    tc = np.zeros((tiles, 4), np.int64)
    tc[:, 1] = rng.integers(0, 30, tiles)
    tc[rng.uniform(size=tiles) < 0.2, 1] = -1          # unknown prefix
    tc[:, 3] = rng.integers(-1, 60, tiles)             # last active position
    active = np.flatnonzero(rng.uniform(size=tiles) < 0.6).astype(np.int32)
    state = rng.standard_normal((pix, 4)).astype(np.float32)
    bt = types.SimpleNamespace(
        n_contrib=torch.from_numpy(rng.integers(0, 80, pix).astype(np.int32)),
        info=types.SimpleNamespace(total_tiles=tiles, total_pixels=pix),
        n_views=len(sizes), view_tab=views,
        n_active_tiles=torch.tensor([active.size], dtype=torch.int32),
        active_tiles=torch.from_numpy(np.concatenate([active, np.zeros(tiles - active.size,
                                                                       np.int32)])),
        tile_cache=torch.from_numpy(tc.astype(np.int32).reshape(-1)),
        prefix_mode=1, prefix_state=torch.from_numpy(state.reshape(-1)))
    return bt, tc, set(active.tolist()), state


def test_walked_evaluations_brute_force():
    bt, tc, active, state = _fake_batch()
    nc = bt.n_contrib.numpy()
    fwd = bwd = full = 0
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        for y in range(v.cam.height):
            for x in range(v.cam.width):
                p = v.pix_base + y * v.cam.width + x
                t = v.tile_base + (y // 16) * v.tiles_x + x // 16
                if t not in active:
                    continue
                full += nc[p]
                if state[p, 0] < 0:        # stopped inside the cached prefix
                    continue
                start = 0 if tc[t, 1] == -1 else tc[t, 1]
                fwd += max(0, nc[p] - start)
                bwd += max(0, min(nc[p], tc[t, 3] + 1) - start)
    got = bench.walked_evaluations(bt)
    assert got == {"forward": fwd, "backward": bwd, "full_list": full}


def _bucketed_fake(seed=1):
    """A fake bucketed pass: per rendered tile a contiguous key range split in
    256 depth bins of random sizes, cached prefixes, last contributors."""
    bt, tc, active, state = _fake_batch(seed)
    rng = np.random.default_rng(seed + 10)
    T = bt.info.total_tiles
    act = bt.active_tiles[: int(bt.n_active_tiles.item())].numpy()
    sizes = rng.integers(0, 3, (act.size, 256)) * rng.integers(0, 2, (act.size, 256))
    sizes[rng.uniform(size=sizes.shape) < 0.01] = 1500   # a few bins above the sort limit
    off = np.concatenate([[0], np.cumsum(sizes.ravel())]).astype(np.int64)
    ranges = np.zeros((T, 2), np.int64)
    for r, t in enumerate(act):
        ranges[t] = off[r * 256], off[(r + 1) * 256]
    bt.layout = 1
    bt.bin_offsets = torch.from_numpy(off[:-1].astype(np.int32))
    bt.ranges = torch.from_numpy(ranges.reshape(-1).astype(np.int32))
    return bt, tc, active, state, sizes, off


def test_walk_counts_brute_force():
    bt, tc, active, state, sizes, off = _bucketed_fake()
    nc = bt.n_contrib.numpy().astype(np.int64)
    act = bt.active_tiles[: int(bt.n_active_tiles.item())].numpy()
    rank = {int(t): r for r, t in enumerate(act)}
    fmax, bmax = {}, {}
    F = Bn = Pr = Pf = Pb = 0
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        for y in range(v.cam.height):
            for x in range(v.cam.width):
                p = v.pix_base + y * v.cam.width + x
                t = v.tile_base + (y // 16) * v.tiles_x + x // 16
                if t not in active:
                    continue
                Pr += 1
                if state[p, 0] < 0:
                    continue
                start = 0 if tc[t, 1] == -1 else tc[t, 1]
                e_b = min(nc[p], tc[t, 3] + 1)
                fmax[t] = max(fmax.get(t, 0), nc[p])
                bmax[t] = max(bmax.get(t, 0), e_b)
                Pf += nc[p] > start
                Pb += e_b > start
    S = big = 0
    for t in act:
        t = int(t)
        start = 0 if tc[t, 1] == -1 else tc[t, 1]
        F += max(0, fmax.get(t, 0) - start)
        Bn += max(0, bmax.get(t, 0) - start)
        if fmax.get(t, 0) <= start:
            continue
        r = rank[t]
        starts = off[r * 256: r * 256 + 256]
        pos_first = off[r * 256] + start
        pos_last = off[r * 256] + fmax[t] - 1
        # the bin holding a position: the last bin that starts at or before it
        b_lo = max(b for b in range(256) if starts[b] <= pos_first)
        b_hi = max(b_lo, max(b for b in range(256) if starts[b] <= pos_last))
        S += int(off[r * 256 + b_hi + 1] - off[r * 256 + b_lo])
        big += int(sum(sizes[r, b] for b in range(b_lo, b_hi + 1) if sizes[r, b] > 1024))
    got = bench.walk_counts(bt)
    assert got == {"rendered_tiles": len(act), "rendered_pixels": Pr, "forward_entries": F,
                   "backward_entries": Bn, "forward_pixels": Pf, "backward_pixels": Pb,
                   "keys_sorted_by_forward": S, "keys_in_large_bins": big}
    assert S > 0 and F > 0


def _with_records(bt, seed, far):
    """Keys and records for the fake pass: every list entry its own record, a
    Gaussian centred in its tile (far=False: reaches every pixel) or far away
    (far=True: culled for its tile)."""
    rng = np.random.default_rng(seed)
    T = bt.info.total_tiles
    ranges = bt.ranges.view(T, 2).numpy().astype(np.int64)
    n = int(ranges[:, 1].max())
    rec = np.zeros((max(n, 1), 12), np.float32)
    tile_xy = np.zeros((T, 2), np.float32)
    for j in range(bt.n_views):
        v = bt.view_tab[j]
        for t in range(v.tiles_x * v.tiles_y):
            tile_xy[v.tile_base + t] = (16 * (t % v.tiles_x), 16 * (t // v.tiles_x))
    for t in range(T):
        a, e = ranges[t]
        if e <= a:
            continue
        c = tile_xy[t] + 8.0 + (1e4 if far else 0.0)
        rec[a:e, 0], rec[a:e, 1] = c[0], c[1]
        rec[a:e, 2] = rng.uniform(0.01, 0.05, e - a)   # conic A
        rec[a:e, 3] = 0.0                              # B
        rec[a:e, 4] = rng.uniform(0.01, 0.05, e - a)   # C
        rec[a:e, 5] = 0.9                              # opacity
    bt.records = torch.from_numpy(rec.reshape(-1))
    bt.keys = torch.arange(max(n, 1), dtype=torch.int64)   # record index in the low word
    return bt


def test_executed_evaluations_bounds():
    """Entries that reach every pixel of their tile are all executed (the count
    equals the walked count); entries far from their tile are all culled."""
    bt, tc, active, state, sizes, off = _bucketed_fake(seed=4)
    walked = bench.walked_evaluations(_with_records(bt, 4, far=False))
    got = bench.executed_evaluations(bt)
    assert got["forward"] == walked["forward"] > 0
    assert got["backward"] == walked["backward"]
    assert got["kept_share"] == 1.0
    got = bench.executed_evaluations(_with_records(bt, 4, far=True))
    assert got["forward"] == 0 and got["backward"] == 0 and got["kept_share"] == 0.0


def test_projection_workspace_layout_matches_the_library():
    """The benchmark's copy of the projection workspace layout (it reads the
    active depth-bin ranges from it) totals the library's own size."""
    if not os.path.exists(abi.library_path()):
        pytest.skip("libclsplat.so not built")
    for nv, tx, ty, n, act in [(4, 120, 68, 1_000_000, 37_948), (2, 8, 6, 500, 17), (1, 240, 135, 3, 3)]:
        info = abi.ClsBatchInfo()
        info.n_scenes, info.n_views, info.max_n, info.max_active = 1, nv, n, act
        info.total_tiles = nv * tx * ty
        info.total_sat = nv * (tx + 1) * (ty + 1)
        info.total_records = nv * n
        info.max_view_tiles = tx * ty
        assert bench.proj_workspace_offsets(info)["total"] == abi.cls_project_workspace_size(info)
