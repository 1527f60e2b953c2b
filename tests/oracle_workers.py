"""Worker processes for oracle work at the benchmark's full size (test
infrastructure). Each worker renders one view's sampled tiles with the float64
oracle and differentiates its share of the loss; the parent sums the views.
Workers are started with the `spawn` method, so they are safe to start after
CUDA has been initialised in the parent."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def reaching(pidx, tiles, cam):
    """Gaussians (ids) whose tile rectangle holds at least one of `tiles`
    ((tx, ty) pairs) in the view of `pidx`: a summed-area table of the marked
    tiles, read at every rectangle's corners."""
    from oracle import fp32_index as fx
    Tx, Ty = fx.tiles_of(cam)
    mark = np.zeros((Ty, Tx), np.int64)
    for (tx, ty) in tiles:
        mark[ty, tx] = 1
    sat = np.zeros((Ty + 1, Tx + 1), np.int64)
    sat[1:, 1:] = mark.cumsum(0).cumsum(1)
    v = pidx["valid"]
    x0 = np.clip(pidx["tx0"], 0, Tx - 1).astype(np.int64)
    x1 = np.clip(pidx["tx1"], 0, Tx - 1).astype(np.int64)
    y0 = np.clip(pidx["ty0"], 0, Ty - 1).astype(np.int64)
    y1 = np.clip(pidx["ty1"], 0, Ty - 1).astype(np.int64)
    cnt = sat[y1 + 1, x1 + 1] - sat[y0, x1 + 1] - sat[y1 + 1, x0] + sat[y0, x0]
    return np.flatnonzero(v & (x0 <= x1) & (y0 <= y1) & (cnt > 0))


def _view_task(task):
    import torch
    torch.set_num_threads(task["threads"])
    from oracle import step as ostep
    r = ostep.render(task["scene"], [task["cam"]], task["sh_degree"], targets=[task["target"]],
                     loss=task["loss"], need_grad=True, tiles=[task["tiles"]], truncate=True,
                     hold_ambiguous=True)
    want = task["want"]
    scale = 1.0 / task["n_views"]  # the view's loss was normalised as if alone
    grads = {k: r["grads"][k][want] * scale for k in ostep.PARAM_KEYS}
    return {"grads": grads, "held": r["held"][0], "loss": r["loss"] * scale,
            "near_ids": sorted(int(task["ids"][i]) for i in r["near_ids"])}


def sampled_gradients(scene, cams, sh_degree, targets, pidx, pick, loss="l1", workers=None):
    """Float64 oracle gradients of the Gaussians `pick` (ids into `scene`):
    per view, every tile their rectangles reach is rendered over the Gaussians
    reaching it and differentiated (loss normalised over the whole image and
    all views). Returns (grads dict of [len(pick)] arrays, held pixels per view)."""
    from oracle import step as ostep
    tasks = []
    V = len(cams)
    threads = max(1, (os.cpu_count() or 4) // V)
    for j, (cam, p) in enumerate(zip(cams, pidx)):
        tl = set()
        for g in pick:
            if p["valid"][g]:
                tl |= {(x, y) for x in range(int(p["tx0"][g]), int(p["tx1"][g]) + 1)
                       for y in range(int(p["ty0"][g]), int(p["ty1"][g]) + 1)}
        ids = reaching(p, sorted(tl), cam)
        pos = np.searchsorted(ids, pick)
        inside = (pos < ids.size) & (ids[np.minimum(pos, ids.size - 1)] == pick)
        tasks.append({"scene": {k: v[ids] for k, v in scene.items()}, "cam": cam,
                      "sh_degree": sh_degree, "target": targets[j], "loss": loss,
                      "tiles": sorted(tl), "want": np.where(inside, pos, 0), "inside": inside,
                      "ids": ids, "n_views": V, "threads": threads})
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers or V, mp_context=ctx) as ex:
        outs = list(ex.map(_view_task, [{k: v for k, v in t.items() if k != "inside"}
                                        for t in tasks]))
    grads = {k: 0.0 for k in ostep.PARAM_KEYS}
    for t, o in zip(tasks, outs):
        for k in ostep.PARAM_KEYS:
            g = o["grads"][k].copy()
            g[~t["inside"]] = 0.0
            grads[k] = grads[k] + g
    return grads, [o["held"] for o in outs], [len(t["tiles"]) for t in tasks]
