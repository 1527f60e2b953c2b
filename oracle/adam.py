"""Masked Adam in float64 (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Supp. "3DGS Optimization in Changed Regions": gradients of Gaussians outside
O^t are masked and the optimizer steps only the Gaussians in O^t, so that
Adam's first and second moments cannot move the frozen part of the scene.
The step itself is textbook Adam (Kingma & Ba, Algorithm 1) at step t:
  m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
  m_hat = m / (1 - b1^t),   v_hat = v / (1 - b2^t),
  theta <- theta - lr m_hat / (sqrt(v_hat) + eps).
"""
from __future__ import annotations

import numpy as np


def adam_step(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-15):
    theta = np.asarray(theta, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * np.asarray(g, np.float64)
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * np.asarray(g, np.float64) ** 2
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def masked_adam_step(theta, m, v, g, active: np.ndarray, t: int, lr: float,
                     b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15):
    """Rows of `active` take an Adam step; every other row of theta, m and v is
    returned unchanged (bit for bit)."""
    theta_o = np.array(theta, np.float64, copy=True)
    m_o = np.array(m, np.float64, copy=True)
    v_o = np.array(v, np.float64, copy=True)
    idx = np.flatnonzero(active)
    th, mm, vv = adam_step(theta_o[idx], m_o[idx], v_o[idx], np.asarray(g)[idx], t, lr,
                           b1, b2, eps)
    theta_o[idx], m_o[idx], v_o[idx] = th, mm, vv
    return theta_o, m_o, v_o
