"""Pins of the history-recovery and merge oracle (Supp. "History Recovery",
its algorithm, and "Batched Updates")."""
import numpy as np

from oracle import history as oh


def _rows(n, seed, w=8):
    return np.random.default_rng(seed).standard_normal((n, w)).astype(np.float32)


def test_reorder_puts_static_rows_first_in_order():
    rows = _rows(50, 0)
    I = np.random.default_rng(1).uniform(size=50) < 0.3
    g, e = oh.begin_update(rows, I)
    k = int((~I).sum())
    assert np.array_equal(g[:k], rows[~I]) and np.array_equal(g[k:], rows[I])
    assert np.array_equal(e["O"], rows[I])


def test_recovery_inverts_any_optimisation_of_the_changed_rows():
    """Whatever happens to the tail (changed values, duplication, pruning), the
    previous state comes back exactly."""
    rows = _rows(60, 2)
    I = np.random.default_rng(3).uniform(size=60) < 0.25
    g, e = oh.begin_update(rows, I)
    k = int((~I).sum())
    tail = _rows(int(I.sum()) + 7, 4)  # optimised, densified
    g_t = np.concatenate([g[:k], tail])
    assert np.array_equal(oh.recover(g_t, e), rows)


def test_multi_step_history_recovery():
    states = [_rows(40, 5)]
    entries = []
    rng = np.random.default_rng(6)
    for step in range(4):
        I = rng.uniform(size=states[-1].shape[0]) < 0.2
        g, e = oh.begin_update(states[-1], I)
        k = int((~I).sum())
        grown = _rows(int(I.sum()) + step, 10 + step)
        states.append(np.concatenate([g[:k], grown]))
        entries.insert(0, e)  # newest first
    for back in range(5):
        assert np.array_equal(oh.recover_state(states[-1], entries, back), states[-1 - back])


def test_merge_of_two_disjoint_updates():
    rows = _rows(30, 7)
    I1 = np.zeros(30, bool); I1[3:8] = True
    I2 = np.zeros(30, bool); I2[20:23] = True
    O1, O2 = _rows(6, 8), _rows(2, 9)
    m = oh.merge(rows, [(I1, O1), (I2, O2)])
    keep = ~(I1 | I2)
    assert m.shape[0] == keep.sum() + 6 + 2
    assert np.array_equal(m[:keep.sum()], rows[keep])
    assert np.array_equal(m[keep.sum():keep.sum() + 6], O1) and np.array_equal(m[-2:], O2)
