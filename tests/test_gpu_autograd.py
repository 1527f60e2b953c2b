"""The torch.autograd.Function over the local rasterizer: a forward whose
pairs outgrow the planned key capacity re-plans instead of dropping pairs, and
a backward run against buffers that a later forward overwrote, or after the
parameters changed in place, raises instead of returning another call's
gradient."""
import numpy as np
import pytest
import torch

from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def _setup():
    from paper_2506_21117_gb300.autograd import ActiveRasterizer
    from paper_2506_21117_gb300.update import SceneState
    scene, cams, targets = S.workload_fd()
    st = SceneState(scene, 1)
    st.set_active(np.ones(500, bool))
    return st, cams, targets, ActiveRasterizer(st, cams)


def _loss(imgs, targets):
    tg = [torch.from_numpy(t).cuda() for t in targets]
    return sum(((im - t) ** 2).mean() for im, t in zip(imgs, tg)) / len(imgs)


def test_capacity_overflow_replans_and_matches():
    st, cams, targets, rast = _setup()
    params = st.params.requires_grad_(True)
    loss = _loss(rast(params), targets)
    loss.backward()
    want_img = rast.batch.image.clone()
    want_grad = params.grad.clone()
    planned = rast.batch.capacity
    # shrink the key buffers below what this scene needs
    rast.batch.allocate_keys(max(int(rast.batch.n_pairs.item()) // 4, 16))
    params.grad = None
    loss2 = _loss(rast(params), targets)
    loss2.backward()
    assert rast.batch.capacity >= int(rast.batch.n_pairs.item())
    assert torch.equal(rast.batch.image, want_img)
    torch.testing.assert_close(params.grad, want_grad, rtol=1e-4, atol=1e-9)
    assert float(loss2.detach()) == pytest.approx(float(loss.detach()), rel=1e-6)
    print(f"capacity {planned} -> shrunk -> re-planned {rast.batch.capacity}")


def test_backward_of_an_older_forward_raises():
    st, cams, targets, rast = _setup()
    params = st.params.requires_grad_(True)
    first = _loss(rast(params), targets)
    _loss(rast(params), targets)  # overwrites the shared buffers
    with pytest.raises(RuntimeError, match="later forward"):
        first.backward()


def test_in_place_parameter_change_before_backward_raises():
    st, cams, targets, rast = _setup()
    params = st.params.requires_grad_(True)
    loss = _loss(rast(params), targets)
    with torch.no_grad():
        params[0, 0] += 0.01
    with pytest.raises(RuntimeError):
        loss.backward()
