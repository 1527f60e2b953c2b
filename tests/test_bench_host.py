"""Host-side accounting of the benchmark (no GPU): the walked-evaluation
counts behind the render roofline equal a per-pixel brute force."""
import types

import numpy as np
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
