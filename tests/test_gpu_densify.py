"""Densification of O^t on the GPU against the oracle (Supp. "History
Recovery", "Implementation Details"; the base 3DGS adaptive density control):
accumulated statistics, the clone/split/prune decisions, source ids, moved
rows and the next active list are bit-exact; split children's means agree
within 1e-5; the opacity reset is bit-exact; a local update with
densification keeps every static row unchanged."""
import numpy as np
import pytest
import torch

from oracle import densify as od
from paper_2506_21117_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_21117_gb300 import build
    build.build()


def _ptr(t):
    return None if t is None else t.data_ptr()


def _rows(n, seed, deg=1):
    """Scene rows whose log-scales, logits and statistics straddle every
    threshold of the rule (extent 2: clone below log 0.02, world-size rule
    above log 0.2; opacity logit(0.005) = -5.29; mean gradient 2e-4)."""
    from paper_2506_21117_gb300.update import pack_params
    rng = np.random.default_rng(seed)
    scene = S.uniform_scene(n, deg, seed)
    scene["log_scales"] = rng.uniform(-6.0, -1.0, (n, 3)).astype(np.float32)
    scene["opacity_logits"] = rng.uniform(-7.0, 3.0, n).astype(np.float32)
    rows = pack_params(scene, deg)
    denom = rng.integers(0, 9, n).astype(np.float32)
    accum = (denom * np.exp(rng.uniform(np.log(1e-5), np.log(1e-3), n))).astype(np.float32)
    maxr = rng.integers(0, 41, n).astype(np.float32)
    return scene, rows, accum, denom, maxr


def _run_densify(rows, A_idx, accum, denom, maxr, z, extent, big):
    from paper_2506_21117_gb300 import _abi as abi
    from paper_2506_21117_gb300.densify import rule
    n, stride = rows.shape
    A = A_idx.size
    cap = n + 2 * A + 7
    dev = "cuda"
    params = torch.zeros((cap, stride), device=dev)
    params[:n] = torch.from_numpy(rows).to(dev)
    m = torch.full((cap, stride), 0.5, device=dev)
    v = torch.full((cap, stride), 0.25, device=dev)
    active = torch.zeros(cap, dtype=torch.uint8, device=dev)
    active[torch.from_numpy(A_idx).long().to(dev)] = 1
    idx = torch.from_numpy(A_idx.astype(np.int32)).to(dev)
    out = torch.full((cap,), -7, dtype=torch.int32, device=dev)
    src = torch.empty(max(2 * A, 1), dtype=torch.int32, device=dev)
    counts = torch.zeros(3, dtype=torch.int32, device=dev)
    removed = torch.empty(max(A, 1), dtype=torch.uint8, device=dev)
    ws = torch.empty(max(abi.cls_densify_workspace_size(A), 256), dtype=torch.uint8, device=dev)
    zt = torch.from_numpy(np.ascontiguousarray(z)).to(dev) if A else torch.zeros(1, device=dev)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
    acc_t, den_t, mr_t = t(accum), t(denom), t(maxr)
    abi.check(abi.cls_densify(
        _ptr(params), _ptr(m), _ptr(v), stride, n, cap, _ptr(active), _ptr(idx), A,
        _ptr(acc_t), _ptr(den_t), _ptr(mr_t), rule(extent, big), _ptr(zt), _ptr(src), _ptr(out),
        _ptr(counts), _ptr(removed), _ptr(ws), ws.numel(),
        torch.cuda.current_stream().cuda_stream), "cls_densify")
    c = counts.cpu().numpy()
    return dict(params=params.cpu().numpy(), m=m.cpu().numpy(), v=v.cpu().numpy(),
                active=active.cpu().numpy(), out=out.cpu().numpy(), src=src.cpu().numpy(),
                counts=c, removed=removed.cpu().numpy()[:A])


@pytest.mark.parametrize("big", [False, True])
@pytest.mark.parametrize("n,frac", [(20_011, 0.3), (1000, 1.0), (513, 0.0)])
def test_densify_bit_exact(n, frac, big):
    scene, rows, accum, denom, maxr = _rows(n, 5 + n)
    rng = np.random.default_rng(n)
    A_idx = np.flatnonzero(rng.uniform(size=n) < frac).astype(np.int64)
    A = A_idx.size
    z = rng.standard_normal((A, 2, 3)).astype(np.float32)
    extent = 2.0
    got = _run_densify(rows, A_idx, accum, denom, maxr, z, extent, big)
    ref = od.densify(scene["means"], scene["log_scales"], scene["quats"],
                     scene["opacity_logits"], A_idx, accum, denom, maxr, extent, z, big)
    n_new, n_keep, n_act = (int(x) for x in got["counts"])
    assert n_new == ref["src"].size
    assert n_keep == A - ref["removed"].size and n_act == n_keep + n_new
    if A:
        # every branch is exercised on the large case
        if n > 10_000:
            assert ref["removed"].size > 0 and n_new > 0
        assert np.array_equal(np.flatnonzero(got["removed"]), np.searchsorted(A_idx, ref["removed"]))
    assert np.array_equal(got["src"][:n_new], ref["src"])
    new = got["params"][n:n + n_new]
    np.testing.assert_allclose(new[:, 0:3], ref["means"], rtol=0, atol=1e-5)
    assert np.array_equal(new[:, 4:7].view(np.uint32), ref["log_scales"].view(np.uint32))
    keep_cols = [3, 7] + list(range(8, rows.shape[1]))
    assert np.array_equal(new[:, keep_cols].view(np.uint32),
                          rows[ref["src"]][:, keep_cols].view(np.uint32))
    assert np.all(got["m"][n:n + n_new] == 0) and np.all(got["v"][n:n + n_new] == 0)
    # removed originals: logit -inf, inactive; everything else unchanged
    after = got["params"][:n]
    rem = ref["removed"]
    assert np.all(np.isneginf(after[rem, 3]))
    untouched = np.setdiff1d(np.arange(n), rem)
    assert np.array_equal(after[untouched].view(np.uint32), rows[untouched].view(np.uint32))
    expect_active = np.zeros(n + n_new, np.uint8)
    expect_active[np.setdiff1d(A_idx, rem)] = 1
    expect_active[n:] = 1
    assert np.array_equal(got["active"][:n + n_new], expect_active)
    assert np.array_equal(got["out"][:n_act], np.flatnonzero(expect_active))


def _views(n_views, W, H, n, A):
    from paper_2506_21117_gb300 import _abi as abi
    from paper_2506_21117_gb300.update import _bytes
    views = (abi.ClsView * n_views)()
    for j in range(n_views):
        views[j].cam.width, views[j].cam.height = W + 16 * j, H
        views[j].rec_base = j * n
        views[j].g2_base = j * A
    return _bytes(views).cuda(), [W + 16 * j for j in range(n_views)]


def test_accumulate_bit_exact():
    from paper_2506_21117_gb300 import _abi as abi
    rng = np.random.default_rng(3)
    n, n_views, H = 30_001, 3, 90
    A_idx = np.flatnonzero(rng.uniform(size=n) < 0.4).astype(np.int32)
    A = A_idx.size
    views, widths = _views(n_views, 160, H, n, A)
    acc = np.zeros(n, np.float32)
    den = np.zeros(n, np.float32)
    mr = np.zeros(n, np.float64)
    acc_t = torch.zeros(n, device="cuda")
    den_t = torch.zeros(n, device="cuda")
    mr_t = torch.zeros(n, device="cuda")
    idx = torch.from_numpy(A_idx).cuda()
    for it in range(2):
        rec = rng.standard_normal((n_views * n, 12)).astype(np.float32)
        radius = rng.integers(-2, 30, n_views * n).astype(np.int32)
        rec[:, 11] = radius.view(np.float32)
        g2 = (rng.standard_normal((n_views * A, 12)) * 1e-5).astype(np.float32)
        rec_t, g2_t = torch.from_numpy(rec).cuda(), torch.from_numpy(g2).cuda()
        abi.check(abi.cls_densify_accumulate(
            _ptr(views), 0, n_views, _ptr(rec_t), _ptr(g2_t), _ptr(idx), A, _ptr(acc_t), _ptr(den_t),
            _ptr(mr_t), torch.cuda.current_stream().cuda_stream), "cls_densify_accumulate")
        torch.cuda.synchronize()
        for j in range(n_views):
            od.accumulate(acc, den, mr, A_idx, g2[j * A:(j + 1) * A, 0], g2[j * A:(j + 1) * A, 1],
                          radius[j * n + A_idx], widths[j], H, n_views)
    assert np.array_equal(acc_t.cpu().numpy().view(np.uint32), acc.view(np.uint32))
    assert np.array_equal(den_t.cpu().numpy(), den)
    assert np.array_equal(mr_t.cpu().numpy(), mr.astype(np.float32))


def test_opacity_reset_bit_exact():
    from paper_2506_21117_gb300 import _abi as abi
    from paper_2506_21117_gb300.densify import reset_limit
    rng = np.random.default_rng(4)
    n, stride = 5000, 16
    rows = rng.uniform(-8, 4, (n, stride)).astype(np.float32)
    A_idx = np.flatnonzero(rng.uniform(size=n) < 0.5).astype(np.int32)
    p = torch.from_numpy(rows).cuda()
    m = torch.ones_like(p)
    v = torch.ones_like(p)
    idx = torch.from_numpy(A_idx).cuda()
    abi.check(abi.cls_opacity_reset(_ptr(p), _ptr(m), _ptr(v), stride, _ptr(idx), A_idx.size,
                                    reset_limit(), torch.cuda.current_stream().cuda_stream),
              "cls_opacity_reset")
    got = p.cpu().numpy()
    assert reset_limit() == float(od.reset_limit())
    ref = od.reset_opacity(rows[:, 3], A_idx)
    assert np.array_equal(got[:, 3].view(np.uint32), ref.view(np.uint32))
    other = np.ones(stride, bool)
    other[3] = False
    assert np.array_equal(got[:, other], rows[:, other])
    mh = m.cpu().numpy()
    assert np.all(mh[A_idx, 3] == 0) and np.all(np.delete(mh, A_idx, axis=0)[:, 3] == 1)


def test_local_update_with_densification():
    """A local update whose O^t densifies: the scene grows, removed originals
    leave O^t, the active list stays ascending and equal to the flags, and the
    static rows never change."""
    from paper_2506_21117_gb300.update import LocalUpdate, pack_params
    scene, _, cams, masks, _ = S.workload_local(n=20000, n_views=4, size=128, seed=6)
    targets = [S.random_image(c, 200 + j) for j, c in enumerate(cams)]
    lu = LocalUpdate(scene, cams, 3, targets=targets, masks=masks, lr=0.01,
                     densify=dict(draws=S.densify_draws(1), interval=5, start=4, until=40,
                                  reset_every=12, grad_threshold=1e-6))
    st = lu.state
    rows0 = pack_params(scene, 3)
    static0 = np.flatnonzero(st.active.cpu().numpy() == 0)
    d = lu.densifier
    lu.run(30)
    torch.cuda.synchronize()
    assert d.steps == 6  # iterations 5, 10, ..., 30 (after start 4)
    assert d.added > 0 and d.removed > 0
    n0 = rows0.shape[0]
    assert st.n == n0 + d.added
    p = st.params.cpu().numpy()
    assert np.array_equal(p[static0].view(np.uint32), rows0[static0].view(np.uint32))
    act = st.active.cpu().numpy()
    idx = st.active_idx[:st.n_active].cpu().numpy()
    assert np.array_equal(idx, np.flatnonzero(act))
    removed = np.setdiff1d(np.flatnonzero(act[:n0] == 0), static0)
    assert removed.size > 0 and np.all(np.isneginf(p[removed, 3]))
