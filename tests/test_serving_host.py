"""Host-side policy of the serving loop (no GPU): FIFO admission, slots,
HBM-footprint budget, one in-flight update per scene, admissions held while a
composition is young, completion, and the
rejection of malformed requests (non-finite poses, empty or mismatched change
masks) before they reach the device."""
import numpy as np

from paper_2506_21117_gb300 import synthetic as S
from paper_2506_21117_gb300.serving import (Request, Scheduler, estimate_footprint,
                                            latency_stats, validate_request)

CAMS = S.ring_cameras(2, 4.0, 24, 16)


def _inputs(cams=CAMS):
    pix = sum(int(c["width"]) * int(c["height"]) for c in cams)
    masks = np.zeros(pix, np.uint8)
    masks[pix // 3: pix // 2] = 1
    return masks, np.full(3 * pix, 0.5, np.float32)


def _req(rid, scene, fp, iters=3, arrival=0.0, cams=CAMS, masks=None, targets=None):
    m, t = _inputs(cams)
    return Request(rid=rid, scene=scene, cams=cams, masks=m if masks is None else masks,
                   targets=t if targets is None else targets, iters=iters, arrival=arrival,
                   footprint=fp)


def test_fifo_slots_and_budget():
    s = Scheduler(max_slots=2, budget=100)
    for i, (sc, fp) in enumerate([(0, 40), (1, 40), (2, 10), (3, 10)]):
        s.submit(_req(i, sc, fp))
    a = s.admit(0.0)
    assert [r.rid for r in a] == [0, 1]           # slot limit
    assert s.used == 80 and len(s.queue) == 2
    s3 = Scheduler(max_slots=8, budget=100)
    for i, fp in enumerate([60, 50, 30]):
        s3.submit(_req(i, i, fp))
    assert [r.rid for r in s3.admit(0.0)] == [0, 2]  # 50 does not fit, 30 does (no reorder of 1)
    assert [r.rid for r in s3.queue] == [1]


def test_busy_scene_waits_and_completion_frees():
    s = Scheduler(max_slots=4, budget=1000)
    s.submit(_req(0, 7, 10, iters=2))
    s.submit(_req(1, 7, 10, iters=1))
    s.submit(_req(2, 8, 10, iters=1))
    assert [r.rid for r in s.admit(0.0)] == [0, 2]
    assert [r.rid for r in s.advance(1.0)] == [2]
    assert s.admit(1.0) == []                      # scene 7 still busy
    assert [r.rid for r in s.advance(2.0)] == [0]
    assert s.used == 0
    assert [r.rid for r in s.admit(2.0)] == [1]
    assert [r.rid for r in s.advance(3.0)] == [1]
    assert s.idle()
    st = latency_stats(s.finished, 3.0)
    assert st["completed"] == 3 and st["p99_ms"] >= st["p50_ms"] > 0


def test_admissions_held_while_a_composition_is_young():
    s = Scheduler(max_slots=4, budget=1000)
    assert not s.holds(0, 3)                       # nothing in flight: admit at once
    s.submit(_req(0, 0, 10))
    s.admit(0.0)
    s.submit(_req(1, 1, 10))
    assert s.holds(0, 3) and s.holds(2, 3)         # one waiting, three slots free
    assert not s.holds(3, 3)                       # the composition has run 3 steps
    # interval 1 admits every step: the loop checks after each step, so the
    # composition has always run at least one step there
    assert not s.holds(1, 1)
    for i in (2, 3):
        s.submit(_req(i, i, 10))
    assert not s.holds(0, 3)                       # enough waiting to fill every free slot
    assert [r.rid for r in s.admit(0.0)] == [1, 2, 3]


def test_oversized_request_rejected():
    s = Scheduler(max_slots=4, budget=100)
    s.submit(_req(0, 0, 101))
    assert s.rejected and not s.queue


def test_footprint_grows_with_views_and_resolution():
    c1 = [{"width": 640, "height": 480}]
    c2 = c1 * 2
    c3 = [{"width": 1280, "height": 720}]
    assert estimate_footprint(1000, c2) > estimate_footprint(1000, c1)
    assert estimate_footprint(1000, c3) > estimate_footprint(1000, c1)
    assert estimate_footprint(2000, c1) > estimate_footprint(1000, c1)


def test_malformed_requests_are_rejected_with_a_reason():
    s = Scheduler(max_slots=4, budget=10**9)
    nan_pose = [dict(c) for c in CAMS]
    nan_pose[1]["t"] = np.array([0.0, float("nan"), 4.0])
    bad_focal = [dict(c) for c in CAMS]
    bad_focal[0]["fx"] = 0.0
    m, t = _inputs()
    cases = {
        "pose": _req(0, 0, 10, cams=nan_pose),
        "focal": _req(1, 1, 10, cams=bad_focal),
        "empty": _req(2, 2, 10, masks=np.zeros_like(m)),
        "masks": _req(3, 3, 10, masks=m[:-1]),
        "targets": _req(4, 4, 10, targets=t[:-3]),
        "views": Request(rid=5, scene=5, cams=[], masks=m, targets=t, footprint=10),
        "iters": _req(6, 6, 10, iters=0),
    }
    for r in cases.values():
        s.submit(r)
    good = _req(7, 7, 10)
    s.submit(good)
    assert [r.rid for r in s.queue] == [7] and good.status == "queued"
    assert len(s.rejected) == len(cases)
    assert all(r.status.startswith("rejected: ") for r in s.rejected)
    assert "not finite" in cases["pose"].status
    assert "focal" in cases["focal"].status
    assert "empty change mask" in cases["empty"].status
    assert "masks do not match" in cases["masks"].status
    assert "target images do not match" in cases["targets"].status
    assert "no views" in cases["views"].status and "iterations" in cases["iters"].status
    assert validate_request(good) is None
    assert [r.rid for r in s.admit(0.0)] == [7]


def test_request_with_nothing_lifted_leaves_without_iterations():
    s = Scheduler(max_slots=2, budget=100)
    a, b = _req(0, 0, 40), _req(1, 0, 40)
    s.submit(a)
    s.submit(b)
    assert [r.rid for r in s.admit(0.0)] == [0]    # scene 0 busy
    s.retire_empty(a, 0.5, "no Gaussian lifted")
    assert a.status.startswith("empty: ") and a.done == 0.5 and s.used == 0
    assert [r.rid for r in s.admit(0.5)] == [1]    # the scene is free again
    assert s.advance(1.0) == [] and s.advance(2.0) == []
    assert [r.rid for r in s.advance(3.0)] == [1] and b.status == "ok"
    assert s.empty == [a] and a not in s.finished


def test_serving_templates_lift_a_change():
    """Every update request of the serving workload lifts a non-empty active
    set: its views surround the changed cluster, so the change box is inside
    every change mask and the majority vote keeps its Gaussians."""
    from oracle import fp32_index as fx
    scenes, centres = S.serving_scenes(6, n_lo=20_000, n_hi=60_000, seed=3)
    for tp in S.serving_templates(scenes, centres, 8, seed=3):
        sc = scenes[tp["scene"]]
        c, o = fx.votes(sc["means"], tp["cams"], tp["masks"])
        active = fx.vote_rule(c, o, len(tp["cams"]))
        assert active.sum() >= 0.005 * sc["means"].shape[0]
        assert all(m.any() for m in tp["masks"])
