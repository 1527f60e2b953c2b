"""The float32 OpenMP CPU baseline (oracle/cpu_fp32.cpp) against the float64
oracle (no GPU): pixels within 1e-4, the loss over the rendered tiles, and the
gradients of every active Gaussian within the parity tolerance (pixels with an
ambiguous threshold decision held constant on both sides), on the plain, the
two-view and a local SH-3 workload; masked Adam against the oracle's."""
import math

import numpy as np
import pytest

from oracle import adam as oadam
from oracle import cpu_baseline as cb
from oracle import fp32_index as fx
from oracle import step as ostep
from paper_2506_21117_gb300 import synthetic as S

FLOOR = 3.5e-2  # the GPU parity floor; this float32 code measures below 1.5e-2


def _local():
    scene = S.uniform_scene(6000, 3, 5)
    cams = S.ring_cameras(3, 4.0, 100, 75)
    box = S.random_box_in_unit_cube(0.05, 5)
    masks = [S.box_change_mask(c, box) for c in cams]
    targets = [S.random_image(c, 5 + j) for j, c in enumerate(cams)]
    active = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    return scene, cams, targets, active


def _unpack(g, deg):
    k = (deg + 1) ** 2
    return {"means": g[:, 0:3], "opacity_logits": g[:, 3], "log_scales": g[:, 4:7],
            "quats": g[:, 8:12], "sh": g[:, 12:12 + 3 * k].reshape(-1, k, 3)}


@pytest.mark.parametrize("case", ["plain", "two_view", "local"])
def test_cpu_baseline_matches_oracle(case):
    if case == "plain":
        scene, cams, targets = S.workload_plain()
        deg, active, loss = 0, np.ones(2000, bool), "l1"
    elif case == "two_view":
        scene, cams, targets = S.workload_fd()
        deg, active, loss = 1, np.ones(500, bool), "l2"
    else:
        scene, cams, targets, active = _local()
        deg, loss = 3, "l1"
    ref = ostep.local_step_reference(scene, cams, deg, targets, active, loss,
                                     hold_ambiguous=True)
    b = cb.Baseline(scene, cams, deg, targets, active, loss)
    out = b.gradients(held=ref["held"], want_image=True)
    # pixels of the rendered tiles
    tiles = ostep.active_tiles(scene, cams, active)
    part = ostep.render(scene, cams, deg, targets=targets, loss=loss, tiles=tiles)
    for im, r, near in zip(out["image"], part["image"], part["near"]):
        done = np.isfinite(r[0])
        assert np.array_equal(np.isfinite(im[0]), done)
        assert np.abs(im - r)[:, done & ~near].max() <= 1e-4
    assert out["loss"] == pytest.approx(part["loss"], rel=1e-5)
    got = _unpack(out["grads"].astype(np.float64), deg)
    idx = np.flatnonzero(active)
    for k in ostep.PARAM_KEYS:
        r = ref["grads"][k][idx].reshape(idx.size, -1)
        g = got[k][idx].reshape(idx.size, -1)
        rms = math.sqrt(float(np.mean(r * r)))
        bound = 1e-3 * np.maximum(np.abs(r), FLOOR * rms)
        assert (np.abs(g - r) <= bound).all(), (case, k)
        assert np.all(got[k][~active] == 0)


def test_cpu_adam_matches_oracle():
    scene, cams, targets, active = _local()
    b = cb.Baseline(scene, cams, 3, targets, active, "l1")
    theta0 = b.rows.copy()
    b.iteration(lr=1e-3, eps=1e-8)
    grads = b.grads.astype(np.float64)
    th, _, _ = oadam.masked_adam_step(theta0.astype(np.float64), np.zeros_like(grads),
                                      np.zeros_like(grads), grads, active, 1, 1e-3, eps=1e-8)
    np.testing.assert_allclose(b.rows[active], th[active], rtol=1e-5, atol=1e-7)
    assert np.array_equal(b.rows[~active], theta0[~active])
