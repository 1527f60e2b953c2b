"""Pins of the D-SSIM oracle (the base 3DGS optimiser's loss that Supp.
"Implementation Details" adopts) against closed forms, brute-force window sums
and central finite differences through the whole render."""
import numpy as np
import pytest
import torch

from oracle import ssim as osim
from oracle import step
from paper_2506_21117_gb300 import synthetic as S


def test_window_is_normalised_gaussian():
    w = osim.window_1d()
    assert w.shape == (11,) and w.sum() == pytest.approx(1.0, abs=1e-15)
    assert w[5] / w[6] == pytest.approx(np.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-12)


def test_identical_images_have_ssim_one():
    x = torch.rand(3, 17, 23, dtype=torch.float64, generator=torch.Generator().manual_seed(0))
    s = osim.ssim_map(x, x)
    assert torch.allclose(s, torch.ones_like(s), atol=1e-12)
    assert float(osim.dssim(x, x)) == pytest.approx(0.0, abs=1e-12)


def test_constant_images_closed_form():
    """Away from the border, constant a and b give mu = a, b and zero
    variances, so S = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x = torch.full((3, 30, 30), a, dtype=torch.float64)
    y = torch.full((3, 30, 30), b, dtype=torch.float64)
    s = osim.ssim_map(x, y)[:, 5:-5, 5:-5]
    ref = (2 * a * b + osim.C1) / (a * a + b * b + osim.C1)
    assert torch.allclose(s, torch.full_like(s, ref), rtol=1e-12)


def test_convolution_matches_brute_force_window_sums():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, 13, 12))
    y = rng.uniform(0, 1, (3, 13, 12))
    got = osim.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    np.testing.assert_allclose(got, osim.ssim_map_brute(x, y), rtol=1e-11, atol=1e-12)


def _signature(scene, cams, sh_degree, g):
    r = step.render(scene, cams, sh_degree)
    sig = [(int(p["tx0"][g]), int(p["tx1"][g]), int(p["ty0"][g]), int(p["ty1"][g]),
            bool(p["valid"][g])) for p in r["pidx"]]
    return sig, [a.tobytes() for a in r["n_contrib"]], [a.tobytes() for a in r["n_incl"]]


def test_dssim_gradient_matches_central_differences():
    """h = 1e-5 central differences of the D-SSIM loss of the 500-Gaussian
    two-view workload for every parameter of the three Gaussians with the
    largest gradients; probes that change the discrete structure are
    excluded and counted."""
    scene, cams, targets = S.workload_fd()
    deg = 1
    ref = step.render(scene, cams, deg, targets=targets, loss="ssim", need_grad=True)
    G = ref["grads"]
    mag = np.abs(G["means"]).sum(1) + np.abs(G["opacity_logits"])
    picks = np.argsort(-mag)[:3].tolist()
    h = 1e-5
    checked = excluded = 0
    for g in picks:
        for key in step.PARAM_KEYS:
            arr = scene[key]
            for flat in range(int(np.prod(arr.shape[1:])) if arr.ndim > 1 else 1):
                sp = {k: v.astype(np.float64) for k, v in scene.items()}
                sm = {k: v.astype(np.float64) for k, v in scene.items()}
                idx = (g,) + np.unravel_index(flat, arr.shape[1:]) if arr.ndim > 1 else (g,)
                sp[key][idx] += h
                sm[key][idx] -= h
                if _signature(sp, cams, deg, g) != _signature(sm, cams, deg, g):
                    excluded += 1
                    continue
                fd = (step.loss_value(sp, cams, deg, targets, "ssim") -
                      step.loss_value(sm, cams, deg, targets, "ssim")) / (2 * h)
                ad = G[key][idx]
                assert abs(fd - ad) <= 1e-5 * abs(ad) + 1e-10, (key, idx, fd, ad)
                checked += 1
    print(f"D-SSIM finite differences: {checked} checked, {excluded} excluded")
    assert checked >= 50 and excluded <= 0.1 * (checked + excluded)


def test_combined_loss_is_the_weighted_sum():
    """(1 - lambda) L1 + lambda D-SSIM: image gradients add up linearly."""
    scene, cams, targets = S.workload_fd()
    a = step.render(scene, cams, 1, targets=targets, loss="l1+ssim", need_grad=True)
    b = step.render(scene, cams, 1, targets=targets, loss="ssim", need_grad=True)
    for j, t in enumerate(targets):
        img = a["image"][j]
        l1_grad = np.sign(img - t) / (3 * img[0].size * len(cams))
        np.testing.assert_allclose(a["dL_dimage"][j],
                                   (1 - osim.LAMBDA) * l1_grad + osim.LAMBDA * b["dL_dimage"][j],
                                   rtol=1e-10, atol=1e-15)
