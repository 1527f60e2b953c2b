"""Pins of the oracle's projection maths against closed forms, library routines
and finite differences (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import fp32_index as fx
from oracle import projection as pj
from oracle import sh as shb
from paper_2506_21117_gb300 import synthetic as S


def ulp_err(approx32, exact64):
    approx32 = np.asarray(approx32, np.float32)
    ref32 = np.asarray(exact64, np.float64).astype(np.float32)
    spacing = np.spacing(np.abs(ref32)).astype(np.float64)
    return np.abs(approx32.astype(np.float64) - np.asarray(exact64)) / spacing


def test_exp32_within_two_ulp():
    rng = np.random.default_rng(1)
    x = np.concatenate([np.linspace(-87.0, 88.0, 400001), rng.normal(-3, 1, 200000),
                        np.array([0.0, -0.0, 1.0, -1.0, 0.5 * math.log(2)])]).astype(np.float32)
    err = ulp_err(fx.exp32(x), np.exp(x.astype(np.float64)))
    assert err.max() <= 2.0, err.max()
    assert fx.exp32(np.float32(0.0)) == np.float32(1.0)


def test_exp32_clamps_domain():
    assert np.isfinite(fx.exp32(np.float32(1000.0)))
    assert fx.exp32(np.float32(-1000.0)) > 0


def _real_sh_scipy(l, m, theta, phi):
    from scipy.special import sph_harm_y
    if m < 0:
        return math.sqrt(2.0) * np.imag(sph_harm_y(l, -m, theta, phi))
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    return math.sqrt(2.0) * np.real(sph_harm_y(l, m, theta, phi))


def test_sh_basis_equals_scipy_real_harmonics():
    """Library special case: the basis equals the real harmonics built from
    scipy's complex Y_l^m (Condon-Shortley phase) as sqrt(2) Im / Re."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(2)
    theta = np.arccos(rng.uniform(-1, 1, 500))
    phi = rng.uniform(0, 2 * np.pi, 500)
    x, y, z = np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)
    Y = shb.basis(x, y, z, 3)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, theta, phi)
            np.testing.assert_allclose(Y[k], ref, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_basis_orthonormal():
    """Gauss-Legendre x uniform-phi quadrature integrates degree <= 6 exactly."""
    ct, wt = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * (2 * np.pi / 24)
    CT, PH = np.meshgrid(ct, phi, indexing="ij")
    Wq = wt[:, None] * (2 * np.pi / 24) * np.ones_like(PH)
    st = np.sqrt(1 - CT ** 2)
    Y = np.stack(shb.basis(st * np.cos(PH), st * np.sin(PH), CT, 3))
    G = np.einsum("aij,bij,ij->ab", Y, Y, Wq)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_quat_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    q = rng.standard_normal((50, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = pj.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    np.testing.assert_allclose(R, ref, atol=1e-12)


def test_covariance3d_eigen_structure():
    rng = np.random.default_rng(4)
    ls = rng.normal(-2, 0.5, (20, 3))
    q = rng.standard_normal((20, 4))
    Sig = pj.covariance3d(torch.tensor(ls), torch.tensor(q)).numpy()
    Rq = pj.quat_to_rotmat(torch.tensor(q / np.linalg.norm(q, axis=1, keepdims=True))).numpy()
    for i in range(20):
        for k in range(3):
            col = Rq[i][:, k]
            np.testing.assert_allclose(Sig[i] @ col, np.exp(2 * ls[i, k]) * col, atol=1e-12)


def _uv_of_world(mu, cam):
    c = pj.cam64(cam)
    p = c["R"].numpy() @ mu + c["t"].numpy()
    return np.array([c["fx"] * p[0] / p[2] + c["cx"], c["fy"] * p[1] / p[2] + c["cy"]])


def test_ewa_jacobian_is_derivative_of_projection():
    """J R equals the finite-difference Jacobian of mu -> (u, v) for points
    inside the clamp window (so the clamp is inactive)."""
    cam = S.ring_cameras(1, 4.0, 64, 48, angles=[0.7])[0]
    c = pj.cam64(cam)
    rng = np.random.default_rng(5)
    mus = rng.uniform(-0.8, 0.8, (10, 3))
    for mu in mus:
        p = c["R"].numpy() @ mu + c["t"].numpy()
        J = pj.ewa_jacobian(torch.tensor(p[None]), c)[0].numpy()
        T = J @ c["R"].numpy()
        h = 1e-6
        fd = np.stack([(_uv_of_world(mu + h * e, cam) - _uv_of_world(mu - h * e, cam)) / (2 * h)
                       for e in np.eye(3)], axis=1)
        np.testing.assert_allclose(T, fd, rtol=1e-7, atol=1e-6)


def test_ewa_jacobian_clamps_tangent():
    cam = S.ring_cameras(1, 4.0, 64, 64, angles=[0.0])[0]
    c = pj.cam64(cam)
    limx = 1.3 * 0.5 * 64 / c["fx"]
    p = np.array([[3.0 * limx * 2.0, 0.1, 2.0]])  # x/z = 3 limx
    J = pj.ewa_jacobian(torch.tensor(p), c)[0].numpy()
    pc = p.copy()
    pc[0, 0] = limx * 2.0
    Jc = pj.ewa_jacobian(torch.tensor(pc), c)[0].numpy()
    np.testing.assert_allclose(J, Jc, atol=1e-12)
    assert J[0, 2] == pytest.approx(-c["fx"] * limx * 2.0 / 4.0)


def _iso_scene(mu, s, n=1):
    return {
        "means": np.asarray(mu, np.float32).reshape(n, 3),
        "log_scales": np.full((n, 3), np.log(s), np.float32),
        "quats": np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
        "opacity_logits": np.zeros(n, np.float32),
        "sh": np.zeros((n, 1, 3), np.float32),
    }


def test_isotropic_projection_closed_form():
    """Sigma = s^2 I gives Sigma' = s^2 T T^T + 0.3 I; on the optical axis
    Sigma' = ((f s / z)^2 + 0.3) I and r = ceil(3 sqrt((f s / z)^2 + 0.3))."""
    cam = S.ring_cameras(1, 4.0, 64, 64, angles=[0.0])[0]
    s = 0.037
    scene = _iso_scene([0.0, 0.0, 0.0], s)
    P = pj.project(pj.scene64(scene), cam, 0)
    c = pj.cam64(cam)
    z = 4.0
    s64 = float(np.exp(np.float64(np.float32(np.log(s)))))
    ref = (c["fx"] * s64 / z) ** 2 + 0.3
    np.testing.assert_allclose(P["cov2d"].numpy()[0], [ref, 0.0, ref], atol=1e-9)
    r_ref = math.ceil(3.0 * math.sqrt(ref))
    pidx = fx.project_index(scene, cam)
    assert pidx["radius"][0] == r_ref
    assert pidx["u"][0] == np.float32(32.0) and pidx["v"][0] == np.float32(32.0)
    # off axis: s^2 T T^T + 0.3 I
    scene2 = _iso_scene([0.3, -0.2, 0.5], s)
    P2 = pj.project(pj.scene64(scene2), cam, 0)
    p = c["R"].numpy() @ np.array([0.3, -0.2, 0.5], np.float32).astype(np.float64) + c["t"].numpy()
    T = pj.ewa_jacobian(torch.tensor(p[None]), c)[0].numpy() @ c["R"].numpy()
    M = s64 ** 2 * T @ T.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(P2["cov2d"].numpy()[0], [M[0, 0], M[0, 1], M[1, 1]], rtol=1e-12)


def test_conic_inverts_cov2d():
    scene = S.uniform_scene(200, 0, seed=6)
    cam = S.ring_cameras(1, 4.0, 64, 64)[0]
    P = pj.project(pj.scene64(scene), cam, 0)
    a, b, c = P["cov2d"].numpy().T
    A, B, C = P["conic"].numpy().T
    np.testing.assert_allclose(a * A + b * B, 1.0, atol=1e-9)
    np.testing.assert_allclose(a * B + b * C, 0.0, atol=1e-9)
    np.testing.assert_allclose(b * B + c * C, 1.0, atol=1e-9)


def test_index_mode_agrees_with_float64_values():
    scene = S.uniform_scene(3000, 0, seed=7)
    cam = S.ring_cameras(1, 4.0, 100, 75, angles=[0.3])[0]
    pidx = fx.project_index(scene, cam)
    P = pj.project(pj.scene64(scene), cam, 0)
    ok = pidx["valid"]
    assert ok.sum() > 2500
    np.testing.assert_allclose(pidx["u"][ok], P["u"].numpy()[ok], rtol=2e-6, atol=1e-4)
    np.testing.assert_allclose(pidx["v"][ok], P["v"].numpy()[ok], rtol=2e-6, atol=1e-4)
    np.testing.assert_allclose(pidx["z"][ok], P["z"].numpy()[ok], rtol=1e-6)
    a, b, c = P["cov2d"].numpy().T
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (a * c - b * b)))
    r64 = 3.0 * np.sqrt(lam)
    clear = ok & (np.abs(r64 - np.round(r64)) > 1e-3)
    assert np.array_equal(pidx["radius"][clear], np.ceil(r64[clear]))
    # rectangles follow the stated reading
    Tx, Ty = fx.tiles_of(cam)
    g = np.flatnonzero(clear)
    x0 = np.clip(np.floor((P["u"].numpy()[g] - np.ceil(r64[g])) / 16), 0, Tx - 1)
    agree = np.mean(x0 == pidx["tx0"][g])
    assert agree > 0.999


def test_degree0_colour_is_drawn_colour():
    """Degree-0 colour = C0 * dc + 1/2 recovers the generator's U(0,1) colour."""
    rng = np.random.default_rng(0)
    n = 50
    _ = rng.uniform(-1.0, 1.0, size=(n, 3))
    _ = rng.normal(-3.0, 0.3, size=(n, 3))
    _ = rng.standard_normal((n, 4))
    _ = rng.standard_normal(n)
    colour = rng.uniform(0.0, 1.0, size=(n, 3))
    scene = S.uniform_scene(n, 0, seed=0)
    cam = S.ring_cameras(1, 4.0, 32, 32)[0]
    P = pj.project(pj.scene64(scene), cam, 0)
    np.testing.assert_allclose(P["rgb"].numpy(), colour, atol=1e-6)
