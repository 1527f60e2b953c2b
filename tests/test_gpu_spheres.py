"""Sphere region and pruning on the GPU against the oracle (Sec. 3.3 "Sphere
Pruning"; Supp. "Identifying Changed Gaussians", "3DGS Optimization in Changed
Regions"): cluster labels, sphere centres and radii and the pruned set are
bit-exact; pixels rendered after pruning match the oracle's render of the
pruned scene within 1e-4."""
import numpy as np
import pytest
import torch

from oracle import fp32_index as fx
from oracle import spheres as osp
from oracle import step as ostep
from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def _state(scene, active, deg):
    from paper_2506_21117_gb300.update import SceneState
    st = SceneState(scene, deg)
    st.set_active(active)
    return st


def _blob_scene(seed=0):
    rng = np.random.default_rng(seed)
    sc = S.uniform_scene(6000, 0, seed)
    centres = np.array([[-0.6, 0.1, 0.2], [0.5, 0.5, -0.3], [0.2, -0.6, 0.5]])
    lab = rng.integers(0, 3, 4000)
    sc["means"][:4000] = (centres[lab] + 0.08 * rng.standard_normal((4000, 3))).astype(np.float32)
    active = np.zeros(6000, bool)
    active[:4000] = True
    return sc, active


def _cases():
    sc, act = _blob_scene()
    yield "blobs", sc, act, 0, 3
    scene, _, cams, masks, _ = S.workload_local(n=30000, n_views=8, size=160)
    act = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    yield "local", scene, act, 3, None
    scene, _, cams, masks, _ = S.workload_large(n=1_000_000, fraction=0.05)
    act = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    yield "large", scene, act, 3, None


@pytest.mark.parametrize("case", ["blobs", "local", "large"])
def test_fit_spheres_bit_exact(case):
    from paper_2506_21117_gb300.update import SphereRegion
    name, scene, active, deg, k = next(c for c in _cases() if c[0] == case)
    st = _state(scene, active, deg)
    region = SphereRegion(st, k)
    torch.cuda.synchronize()
    got = region.host()
    pts = scene["means"][np.flatnonzero(active)]
    ref = osp.fit_spheres(pts, region.k)
    assert region.k == (k if k else osp.n_clusters(pts.shape[0]))
    assert np.array_equal(got["labels"], ref["labels"])
    assert np.array_equal(got["counts"], ref["counts"])
    assert np.array_equal(got["centers"].view(np.uint32), ref["centers"].view(np.uint32))
    assert np.array_equal(got["radii"].view(np.uint32), ref["radii"].view(np.uint32))
    print(f"{case}: {pts.shape[0]} points, {region.k} spheres, radii {np.round(ref['radii'], 3)}")


def test_prune_bit_exact_and_render_after_pruning():
    from paper_2506_21117_gb300.update import (LocalUpdate, SphereRegion, pack_params,
                                               prune_outside)
    scene, _, cams, masks, _ = S.workload_local(n=20000, n_views=4, size=128, seed=4)
    targets = [S.random_image(c, 90 + j) for j, c in enumerate(cams)]
    active = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    lu = LocalUpdate(scene, cams, 3, targets=targets, active=active, loss="l1", prune_every=15)
    st = lu.state
    ref_sp = osp.fit_spheres(scene["means"][np.flatnonzero(active)], lu.region.k)
    got_sp = lu.region.host()
    assert np.array_equal(got_sp["radii"].view(np.uint32), ref_sp["radii"].view(np.uint32))
    # the active Gaussians move (generator-side), some out of the spheres
    moved = S.perturb_scene(scene, active, 0.12, seed=9)
    idx = np.flatnonzero(active)
    rows = pack_params(moved, 3)
    st.params[torch.from_numpy(idx).long().cuda()] = torch.from_numpy(rows[idx]).cuda()
    k, removed = prune_outside(st, lu.region, want_removed=True)
    torch.cuda.synchronize()
    new_active, new_logit, ref_removed = osp.prune(moved["means"], moved["opacity_logits"],
                                                  active, ref_sp)
    assert k == ref_removed.size > 0
    assert np.array_equal(removed, ref_removed)
    assert np.array_equal(st.active.cpu().numpy().astype(bool), new_active)
    assert st.n_active == int(new_active.sum())
    assert np.array_equal(st.active_idx[: st.n_active].cpu().numpy(), np.flatnonzero(new_active))
    logit = st.params.view(st.n, st.stride)[:, 3].cpu().numpy()
    assert np.array_equal(logit[ref_removed], new_logit[ref_removed])
    print(f"pruned {k} of {idx.size} active Gaussians")
    # render after pruning: the removed Gaussians contribute nothing
    lu.batch.refresh_active()
    lu.render_pass(with_backward=True, with_adam=False)
    torch.cuda.synchronize()
    lu.batch.check_status()
    pruned = {kk: v.copy() for kk, v in moved.items()}
    pruned["opacity_logits"] = new_logit
    tiles = ostep.active_tiles(pruned, cams, new_active)
    ref = ostep.render(pruned, cams, 3, targets=targets, tiles=tiles)
    imgs = lu.batch.per_view(lu.batch.image, 3)
    tm = lu.batch.tile_active.cpu().numpy()
    base = 0
    checked = 0
    for j, cam in enumerate(cams):
        Tx, Ty = fx.tiles_of(cam)
        m = tm[base:base + Tx * Ty].reshape(Ty, Tx)
        base += Tx * Ty
        pix = np.kron(m, np.ones((16, 16), np.uint8))[:cam["height"], :cam["width"]].astype(bool)
        ok = pix & ~ref["near"][j]
        err = np.abs(imgs[j].cpu().numpy() - ref["image"][j])[:, ok]
        assert err.max() <= 1e-4
        checked += int(ok.sum())
    assert checked > 1000


def test_local_update_prunes_every_15_iterations():
    """A run with pruning: the static rows never change, removed Gaussians
    leave O^t with opacity logit -inf, and the update keeps running."""
    from paper_2506_21117_gb300.update import LocalUpdate, pack_params
    scene, _, cams, masks, _ = S.workload_local(n=20000, n_views=4, size=128, seed=6)
    targets = [S.random_image(c, 95 + j) for j, c in enumerate(cams)]
    lu = LocalUpdate(scene, cams, 3, targets=targets, masks=masks, loss="l1", lr=0.05,
                     prune_every=15)
    A0 = lu.state.n_active
    lu.run(30)
    torch.cuda.synchronize()
    act0 = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    rows0 = pack_params(scene, 3)
    p = lu.state.params.view(lu.state.n, lu.state.stride).cpu().numpy()
    assert np.array_equal(p[~act0], rows0[~act0])
    act = lu.state.active.cpu().numpy().astype(bool)
    gone = act0 & ~act
    assert lu.state.n_active == A0 - lu.removed == int(act.sum())
    assert np.all(p[gone, 3] == -np.inf)
    print(f"pruning run: {lu.removed} of {A0} active Gaussians removed in 30 iterations")
