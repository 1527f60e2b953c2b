"""The allocation-free lifting entry point agrees with the regular one.

cls_lift_change_masks_static serves callers that cannot allocate device
memory (for example a plug-in living inside a host application that owns all
device allocations): it takes no workspace and keeps its scratch in a fixed
array inside the library. This file is collected last so a stop-at-first-
failure run has executed every other test before it; it also passes alone in a
fresh process, since it sets up everything it uses.
"""
import numpy as np
import pytest
import torch

from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _lift_both(scene, cams, masks, vote_mode):
    from paper_2506_21117_gb300 import _abi
    from paper_2506_21117_gb300.update import SceneState, _bytes, _views_for
    st = SceneState(scene, 3)
    views, _ = _views_for(cams)
    views_dev = _bytes(views).to("cuda")
    masks_dev = torch.from_numpy(np.concatenate([m.reshape(-1) for m in masks])).to("cuda")
    n = st.n
    stream = torch.cuda.current_stream().cuda_stream
    out = []
    for static in (False, True):
        act = torch.zeros(n, dtype=torch.uint8, device="cuda")
        idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        votes = torch.zeros(2 * n, dtype=torch.int32, device="cuda")
        if static:
            code = _abi.cls_lift_change_masks_static(
                st.params.data_ptr(), n, st.stride, views_dev.data_ptr(), 0, len(cams),
                masks_dev.data_ptr(), vote_mode, act.data_ptr(), idx.data_ptr(), cnt.data_ptr(),
                votes.data_ptr(), stream)
        else:
            ws = torch.zeros(_abi.cls_lift_workspace_size(n), dtype=torch.uint8, device="cuda")
            code = _abi.cls_lift_change_masks(
                st.params.data_ptr(), n, st.stride, views_dev.data_ptr(), 0, len(cams),
                masks_dev.data_ptr(), vote_mode, act.data_ptr(), idx.data_ptr(), cnt.data_ptr(),
                votes.data_ptr(), ws.data_ptr(), ws.numel(), stream)
        assert code == _abi.CLS_OK
        torch.cuda.synchronize()
        k = int(cnt.item())
        out.append((act.cpu().numpy(), idx[:k].cpu().numpy(), k, votes.cpu().numpy()))
    return out


def test_static_scratch_lift_matches_workspace_lift_twice():
    # two calls in a row, the second smaller, so stale scratch from the first
    # call would show up
    cases = [S.workload_local(n=60_000, n_views=8, size=160, seed=1),
             S.workload_local(n=5_000, n_views=4, size=96, seed=2)]
    for (scene, _, cams, masks, _), mode in zip(cases, (0, 0)):
        (a0, i0, k0, v0), (a1, i1, k1, v1) = _lift_both(scene, cams, masks, mode)
        # votes and the active set are integers: the tolerance is exact equality
        assert k0 == k1 > 0
        assert np.array_equal(a0, a1) and np.array_equal(i0, i1) and np.array_equal(v0, v1)


def test_static_scratch_lift_rejects_oversized_input():
    from paper_2506_21117_gb300 import _abi
    code = _abi.cls_lift_change_masks_static(
        1, _abi.LIFT_STATIC_MAX_N + 1, 16, 1, 0, 1, 1, 0, 1, 1, 1, None,
        torch.cuda.current_stream().cuda_stream)
    assert code == _abi.CLS_ERR_INVALID_ARG
