"""Host-side densification logic (no GPU): the float32 thresholds handed to
the kernel equal the oracle's, the scene extent follows the base optimiser's
camera rule, and the schedule fires where the base optimiser does."""
import math

import numpy as np
import pytest

from oracle import densify as od


def test_rule_matches_oracle_thresholds():
    from paper_2506_21117_gb300.densify import reset_limit, rule
    for extent in (0.37, 2.0, 11.5):
        th = od.thresholds(extent)
        for big in (False, True):
            r = rule(extent, big)
            assert np.float32(r.grad_threshold) == th["grad"]
            assert np.float32(r.clone_log_scale) == th["clone_ls"]
            assert np.float32(r.min_logit) == th["logit"]
            assert np.float32(r.big_log_scale) == th["big_ls"]
            assert np.float32(r.log_shrink) == th["shrink"]
            assert r.big == (1 if big else 0)
    assert np.float32(reset_limit()) == od.reset_limit()


def test_camera_extent():
    from paper_2506_21117_gb300.densify import camera_extent
    cams = [{"pos": p} for p in ([1.0, 0, 0], [-1.0, 0, 0], [0, 3.0, 0], [0, -3.0, 0])]
    # centre at the origin; the farthest camera is 3 away
    assert camera_extent(cams) == pytest.approx(3.3)


def test_schedule():
    from paper_2506_21117_gb300.densify import Densifier
    d = Densifier.__new__(Densifier)
    d.interval, d.start, d.until, d.reset_every = 100, 500, 15000, 3000
    due = [i for i in range(1, 16001) if d.due(i)]
    assert due[0] == 600 and due[-1] == 14900 and all(b - a == 100 for a, b in zip(due, due[1:]))
    resets = [i for i in range(1, 16001) if d.reset_due(i)]
    assert resets == [3000, 6000, 9000, 12000]
