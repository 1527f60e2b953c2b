"""Host-side policy of the serving loop (no GPU): FIFO admission, slots,
HBM-footprint budget, one in-flight update per scene, completion."""
from paper_2506_21117_gb300.serving import Request, Scheduler, estimate_footprint, latency_stats


def _req(rid, scene, fp, iters=3, arrival=0.0):
    return Request(rid=rid, scene=scene, cams=[], masks=None, targets=None, iters=iters,
                   arrival=arrival, footprint=fp)


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
