"""Pins of the oracle's masked Adam (no GPU)."""
import numpy as np
import torch

from oracle import adam
from paper_2506_21117_gb300 import synthetic as S


def test_first_step_closed_form():
    """At t = 1 from zero moments, m_hat = g and v_hat = g^2, so the step is
    -lr g / (|g| + eps)."""
    theta, _, _, g = S.random_adam_state(64, 7)
    z = np.zeros_like(theta)
    th, m, v = adam.adam_step(theta, z, z, g, 1, 1e-3, eps=1e-15)
    g64 = g.astype(np.float64)
    np.testing.assert_allclose(th, theta - 1e-3 * g64 / (np.abs(g64) + 1e-15), rtol=0, atol=1e-15)


def test_matches_torch_adam_float64():
    """Library special case: several steps equal torch.optim.Adam in float64."""
    theta, _, _, _ = S.random_adam_state(32, 5)
    rng = np.random.default_rng(9)
    p = torch.tensor(theta.astype(np.float64), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta.astype(np.float64), np.zeros_like(theta, np.float64), np.zeros_like(theta, np.float64)
    for t in range(1, 6):
        g = rng.standard_normal(theta.shape)
        p.grad = torch.tensor(g)
        opt.step()
        th, m, v = adam.adam_step(th, m, v, g, t, 1e-3, 0.9, 0.999, 1e-8)
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=0, atol=1e-13)


def test_masked_rows_untouched():
    theta, m, v, g = S.random_adam_state(100, 9)
    active = np.zeros(100, bool)
    active[::7] = True
    th, mo, vo = adam.masked_adam_step(theta, m, v, g, active, 3, 1e-3)
    assert np.array_equal(th[~active], theta[~active].astype(np.float64))
    assert np.array_equal(mo[~active], m[~active].astype(np.float64))
    assert np.array_equal(vo[~active], v[~active].astype(np.float64))
    assert not np.allclose(th[active], theta[active])
