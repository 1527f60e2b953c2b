"""New-point sampling on the GPU against the oracle (Sec. 3.2 "Gaussian
Sampling for New Objects"; Supp. Full-Scene / Region Point Sampling): with the
same input draws, every round's kept points are bit-exact, including the
K-Means mixture; the new Gaussians' initialisation matches (mean squared
neighbour distances bit-exact, log values within 1e-6); the sampled Gaussians
join O^t and optimise."""
import numpy as np
import pytest
import torch

from oracle import fp32_index as fx
from oracle import sampling as osa
from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def _state(scene, active):
    from paper_2506_21117_gb300.update import SceneState
    st = SceneState(scene, 3)
    st.set_active(active)
    return st


def test_sampling_from_an_empty_region_bit_exact():
    from paper_2506_21117_gb300.sampling import sample_points
    scene, cams, masks, box = S.workload_addition(n=20000, n_views=6, size=96, seed=3)
    act = np.zeros(scene["means"].shape[0], bool)  # O^t empty: the box round runs first
    st = _state(scene, act)
    draws = S.sampling_draws(0)
    got = sample_points(st, cams, masks, 400, draws)
    ref = osa.sample_points(scene["means"][act], scene["means"], cams, masks, 400, draws)
    pts = got["points"][:, :3].cpu().numpy()
    assert got["rounds"] == ref["rounds"] >= 2  # a box round, then mixture rounds
    assert np.array_equal(pts.view(np.uint32), ref["points"].view(np.uint32))
    new = got["new"][:, :3].cpu().numpy()
    assert np.array_equal(new.view(np.uint32), ref["new"].view(np.uint32))
    print(f"empty O: {pts.shape[0]} points in {ref['rounds']} rounds")


def test_region_rounds_from_a_few_seeds_bit_exact():
    from paper_2506_21117_gb300.sampling import sample_points
    scene, cams, masks, box = S.workload_addition(n=20000, n_views=6, size=96, seed=3)
    lo, hi = box
    rng = np.random.default_rng(4)
    seeds = S.uniform_scene(40, 3, 7)
    seeds["means"] = rng.uniform(lo, hi, (40, 3)).astype(np.float32)
    full = {k: np.concatenate([scene[k], seeds[k]]) for k in scene}
    act = np.zeros(full["means"].shape[0], bool)
    act[-40:] = True
    st = _state(full, act)
    draws = S.sampling_draws(5)
    got = sample_points(st, cams, masks, 300, draws)
    ref = osa.sample_points(full["means"][act], full["means"], cams, masks, 300, draws)
    pts = got["points"][:, :3].cpu().numpy()
    assert got["rounds"] == ref["rounds"] >= 1
    assert np.array_equal(pts.view(np.uint32), ref["points"].view(np.uint32))
    print(f"region rounds: 40 seeds -> {pts.shape[0]} points in {ref['rounds']} rounds")


def test_initialisation_of_new_points():
    from paper_2506_21117_gb300.sampling import init_gaussians
    from paper_2506_21117_gb300.update import unpack_rows
    rng = np.random.default_rng(6)
    pts = rng.uniform(-1, 1, (700, 3)).astype(np.float32)
    pts[5] = pts[6]  # a duplicate: zero distance
    dev = torch.zeros((700, 4), dtype=torch.float32, device="cuda")
    dev[:, :3] = torch.from_numpy(pts).cuda()
    rows = init_gaussians(dev, 3).cpu().numpy()
    got = unpack_rows(rows.astype(np.float64), 3)
    ref = osa.init_gaussians(pts, 3)
    assert np.array_equal(rows[:, :3].astype(np.float32).view(np.uint32), pts.view(np.uint32))
    np.testing.assert_allclose(got["log_scales"], ref["log_scales"], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(got["opacity_logits"], ref["opacity_logits"], rtol=1e-6)
    assert np.all(got["quats"] == np.array([1, 0, 0, 0]))
    assert not got["sh"].any()
    # the squared neighbour distances themselves are bit-exact
    ls = rows[:, 4].astype(np.float32)
    d_ref = osa.knn_mean_sq(pts)
    assert np.allclose(np.exp(2.0 * ls.astype(np.float64)), d_ref, rtol=1e-5)


def test_sampled_gaussians_join_the_update_and_optimise():
    from paper_2506_21117_gb300.sampling import add_to_scene, init_gaussians, sample_points
    from paper_2506_21117_gb300.update import LocalUpdate, SceneState, pack_params
    scene, cams, masks, box = S.workload_addition(n=20000, n_views=6, size=96, seed=8)
    targets = [S.random_image(c, 110 + j) for j, c in enumerate(cams)]
    act = fx.vote_rule(*fx.votes(scene["means"], cams, masks), len(cams))
    st = _state(scene, act)
    got = sample_points(st, cams, masks, st.n_active + 500, S.sampling_draws(2))
    assert got["new"].shape[0] >= 500
    rows = init_gaussians(got["new"], 3)
    n0 = st.n
    add_to_scene(st, rows)
    flat_m = torch.from_numpy(np.concatenate([m.reshape(-1) for m in masks]))
    flat_t = torch.from_numpy(np.concatenate([t.reshape(-1) for t in targets]))
    lu = LocalUpdate.from_resident(st, cams, flat_t, flat_m)
    assert lu.state.n == n0 + rows.shape[0]
    new_active = lu.state.active[n0:].cpu().numpy().astype(bool)
    assert new_active.all()  # the sampled points pass the same vote
    losses = []
    for _ in range(10):
        lu.step()
        losses.append(float(lu.batch.loss[0]))
    torch.cuda.synchronize()
    lu.batch.check_status()
    p = lu.state.params.cpu().numpy()
    static = ~lu.state.active.cpu().numpy().astype(bool)
    assert np.array_equal(p[:n0][static[:n0]], pack_params(scene, 3)[static[:n0]])
    assert losses[-1] < losses[0]
    print(f"{rows.shape[0]} sampled Gaussians added; loss {losses[0]:.5f} -> {losses[-1]:.5f}")
