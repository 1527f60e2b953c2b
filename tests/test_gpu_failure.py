"""Failure detection without faulting the GPU: a bounded wait that runs out
reports CLS_ERR_TIMEOUT and returns (the context stays usable); malformed or
empty serving requests come back with a status instead of running."""
import numpy as np
import pytest
import torch

from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def _sort(abi, keys_np, bits, spin_limit, n_tiles):
    n = keys_np.size
    kd = torch.from_numpy(keys_np.view(np.int64)).cuda()
    vd = torch.arange(n, dtype=torch.int32, device="cuda")
    ka, va = torch.empty_like(kd), torch.empty_like(vd)
    nd = torch.tensor([n], dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.zeros(abi.cls_sort_workspace_size(n, bits), dtype=torch.uint8, device="cuda")
    ranges = torch.zeros(2 * n_tiles, dtype=torch.int32, device="cuda")
    code = abi.cls_sort_keys_bounded(kd.data_ptr(), vd.data_ptr(), ka.data_ptr(), va.data_ptr(),
                                     nd.data_ptr(), n, bits, ranges.data_ptr(), n_tiles,
                                     st.data_ptr(), ws.data_ptr(), ws.numel(), spin_limit,
                                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()  # the call returns: no wait is unbounded
    return code, int(st.item()), kd.cpu().numpy().view(np.uint64), vd.cpu().numpy()


def test_sort_lookback_timeout_is_reported_and_context_survives():
    """With a spin bound of 0 a digit pass gives up at the first preceding
    partition that has not published its count yet (thousands of partitions
    run at once, so some do): CLS_ERR_TIMEOUT comes back, the call returns, and
    a sort with the default bound on the same context is exact again."""
    from paper_2506_21117_gb300 import _abi
    rng = np.random.default_rng(5)
    n, bits, n_tiles = 4_000_000, 44, 4096
    keys = (rng.integers(0, n_tiles, n).astype(np.uint64) << np.uint64(32)) | \
        rng.integers(0x3F000000, 0x3F800000, n).astype(np.uint64)
    seen = 0
    for _ in range(6):
        code, status, _, _ = _sort(_abi, keys, bits, 0, n_tiles)
        assert code == _abi.CLS_OK
        assert status in (_abi.CLS_OK, _abi.CLS_ERR_TIMEOUT)
        seen += status == _abi.CLS_ERR_TIMEOUT
        if seen:
            break
    assert seen, "no look-back wait ran out with a spin bound of 0"
    code, status, k, v = _sort(_abi, keys, bits, _abi.CLS_SORT_SPIN_LIMIT, n_tiles)
    assert code == _abi.CLS_OK and status == _abi.CLS_OK
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[order]) and np.array_equal(v, order.astype(np.int32))


def test_negative_spin_bound_is_rejected():
    from paper_2506_21117_gb300 import _abi
    code, _, _, _ = _sort(_abi, np.arange(10, dtype=np.uint64), 8, -1, 1)
    assert code == _abi.CLS_ERR_INVALID_ARG


def _serving_set():
    from paper_2506_21117_gb300.serving import Request
    from paper_2506_21117_gb300.update import SceneState
    scene = S.uniform_scene(8000, 3, seed=61)
    cams = S.ring_cameras(2, 4.0, 64, 48)
    box = S.random_box_in_unit_cube(0.08, seed=61)
    masks = np.concatenate([S.box_change_mask(c, box).reshape(-1) for c in cams])
    tg = np.concatenate([S.random_image(c, 62 + j).reshape(-1) for j, c in enumerate(cams)])
    m = torch.from_numpy(masks).pin_memory()
    t = torch.from_numpy(tg).pin_memory()
    # a mask with set pixels that no Gaussian centre projects into: one
    # corner pixel of each view, far outside the scene's footprint
    corner = np.zeros_like(masks)
    corner[0] = 1
    nan_cams = [dict(c) for c in cams]
    nan_cams[0]["R"] = np.full((3, 3), np.nan)
    reqs = [Request(rid=0, scene=0, cams=cams, masks=m, targets=t, iters=3),
            Request(rid=1, scene=0, cams=nan_cams, masks=m, targets=t, iters=3),
            Request(rid=2, scene=0, cams=cams, masks=torch.zeros_like(m), targets=t, iters=3),
            Request(rid=3, scene=0, cams=cams, masks=torch.from_numpy(corner).pin_memory(),
                    targets=t, iters=3),
            Request(rid=4, scene=1, cams=cams, masks=m, targets=t, iters=3)]
    return [SceneState(scene, 3)], reqs


def test_serving_rejects_malformed_and_retires_empty_requests():
    """A non-finite pose and an all-zero change mask are rejected before they
    reach the device; a request whose lifting finds no Gaussian leaves without
    an iteration; a request for an unknown scene is rejected; the good request
    completes with a finite loss."""
    from paper_2506_21117_gb300.serving import Server
    states, reqs = _serving_set()
    srv = Server(states, max_slots=4)
    st = srv.serve(reqs, realtime=False)
    status = {r.rid: r.status for r in reqs}
    assert status[0] == "ok" and np.isfinite(reqs[0].loss)
    assert status[1].startswith("rejected: camera pose")
    assert status[2].startswith("rejected: empty change mask")
    assert status[3].startswith("empty: ")
    assert status[4] == "rejected: unknown scene"
    assert st["completed"] == 1 and st["rejected"] == 3 and st["empty"] == 1
    assert st["errors"] == 0
