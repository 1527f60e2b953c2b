"""History recovery and merging on the GPU against the oracle (Supp. "History
Recovery", its algorithm, "Batched Updates"): every row move is bit-exact, and
after a real local update (optimised, pruned) the previous scene comes back
exactly."""
import numpy as np
import pytest
import torch

from oracle import fp32_index as fx
from oracle import history as oh
from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def test_reorder_and_recover_bit_exact():
    from paper_2506_21117_gb300 import history as H
    rng = np.random.default_rng(0)
    rows = rng.standard_normal((70_001, 16)).astype(np.float32)
    I = rng.uniform(size=70_001) < 0.07
    d = torch.from_numpy(rows).cuda()
    flags = torch.from_numpy(I.astype(np.uint8)).cuda()
    m, cnt = H.flag_map(flags, 0)
    g = H.gather_rows(d, None, m, rows.shape[0]).cpu().numpy()
    ref, e = oh.begin_update(rows, I)
    assert int(cnt.item()) == int(I.sum())
    assert np.array_equal(g.view(np.uint32), ref.view(np.uint32))
    # recovery after the tail changed size and values
    k = int((~I).sum())
    tail = rng.standard_normal((int(I.sum()) + 123, 16)).astype(np.float32)
    g_t = np.concatenate([ref[:k], tail])
    entry = H.HistoryEntry(O=torch.from_numpy(e["O"]).cuda(), I=flags)
    back = H.recover(torch.from_numpy(g_t).cuda(), entry).cpu().numpy()
    assert np.array_equal(back.view(np.uint32), rows.view(np.uint32))
    assert np.array_equal(back.view(np.uint32), oh.recover(g_t, e).view(np.uint32))


def test_merge_bit_exact():
    from paper_2506_21117_gb300 import history as H
    rng = np.random.default_rng(1)
    rows = rng.standard_normal((5000, 24)).astype(np.float32)
    I1 = np.zeros(5000, bool); I1[100:400] = True
    I2 = np.zeros(5000, bool); I2[3000:3050] = True
    O1 = rng.standard_normal((320, 24)).astype(np.float32)
    O2 = rng.standard_normal((41, 24)).astype(np.float32)
    got = H.merge(torch.from_numpy(rows).cuda(),
                  [(torch.from_numpy(I1.astype(np.uint8)).cuda(), torch.from_numpy(O1).cuda()),
                   (torch.from_numpy(I2.astype(np.uint8)).cuda(), torch.from_numpy(O2).cuda())])
    ref = oh.merge(rows, [(I1, O1), (I2, O2)])
    assert np.array_equal(got.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_history_across_two_real_updates():
    """Two successive local updates (with pruning) of one resident scene: the
    scene before each update is recovered exactly from the final one."""
    from paper_2506_21117_gb300 import history as H
    from paper_2506_21117_gb300.update import LocalUpdate, SceneState, pack_params
    scene, _, cams, masks, _ = S.workload_local(n=20000, n_views=4, size=128, seed=2)
    st = SceneState(scene, 3)
    states = [st.params.clone()]
    entries = []
    for u, (box_seed, tseed) in enumerate([(2, 120), (9, 130)]):
        box = S.random_box_in_unit_cube(0.05, box_seed)
        m = [S.box_change_mask(c, box) for c in cams]
        t = [S.random_image(c, tseed + j) for j, c in enumerate(cams)]
        flat_m = torch.from_numpy(np.concatenate([x.reshape(-1) for x in m]))
        flat_t = torch.from_numpy(np.concatenate([x.reshape(-1) for x in t]))
        from paper_2506_21117_gb300.update import lift
        lift(st, cams, flat_m)
        entries.insert(0, H.begin_update(st))
        lu = LocalUpdate.from_resident(st, cams, flat_t, flat_m, lr=0.02)
        # the lift inside from_resident must find the same set, now the tail
        assert st.n_active == int(entries[0].O.shape[0])
        assert np.array_equal(st.active_idx[:st.n_active].cpu().numpy(),
                              np.arange(st.n - st.n_active, st.n))
        lu.run(8)
        torch.cuda.synchronize()
        states.append(st.params.clone())
    for back in range(3):
        got = H.recover_state(states[-1], entries, back).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), states[-1 - back].cpu().numpy().view(np.uint32))
    assert np.array_equal(states[0].cpu().numpy(), pack_params(scene, 3))
