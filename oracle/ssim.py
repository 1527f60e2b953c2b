"""D-SSIM term of the photometric loss. TEST INFRASTRUCTURE ONLY (see the
package docstring).

Supp. "Implementation Details": the method adopts every default of the base
3DGS optimiser, whose photometric loss is (1 - lambda) L1 + lambda D-SSIM with
lambda = 0.2 and D-SSIM = 1 - SSIM, SSIM being the mean over pixels and
channels of the structural-similarity map of Wang et al. with an 11 x 11
Gaussian window of standard deviation 1.5, constants C1 = (0.01)^2 and
C2 = (0.03)^2 for intensities in [0, 1], and the window applied with zero
padding of 5 at the image borders (a convolution with "same" output size).
Written here as that definition, in float64:

  mu_x = g * x,  sigma_x^2 = g * x^2 - mu_x^2,  sigma_xy = g * (x y) - mu_x mu_y,
  S = ((2 mu_x mu_y + C1)(2 sigma_xy + C2)) /
      ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).
"""
from __future__ import annotations

import numpy as np
import torch

LAMBDA = 0.2
WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window_1d() -> np.ndarray:
    i = np.arange(WINDOW, dtype=np.float64) - WINDOW // 2
    w = np.exp(-(i * i) / (2.0 * SIGMA * SIGMA))
    return w / w.sum()


def _blur(z: torch.Tensor) -> torch.Tensor:
    """Per-channel 2D window over [C, H, W] with zero padding."""
    w = torch.tensor(window_1d(), dtype=z.dtype)
    k = torch.outer(w, w)[None, None].repeat(z.shape[0], 1, 1, 1)
    return torch.nn.functional.conv2d(z[None], k, padding=WINDOW // 2, groups=z.shape[0])[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim_map_brute(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The same map by explicit window sums (loops), for pinning small inputs."""
    C, H, W = x.shape
    w = window_1d()
    r = WINDOW // 2
    out = np.zeros((C, H, W))
    for c in range(C):
        for i in range(H):
            for j in range(W):
                s = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
                for a in range(-r, r + 1):
                    for b in range(-r, r + 1):
                        ii, jj = i + a, j + b
                        if 0 <= ii < H and 0 <= jj < W:
                            g = w[a + r] * w[b + r]
                            xv, yv = x[c, ii, jj], y[c, ii, jj]
                            s["x"] += g * xv
                            s["y"] += g * yv
                            s["xx"] += g * xv * xv
                            s["yy"] += g * yv * yv
                            s["xy"] += g * xv * yv
                mx, my = s["x"], s["y"]
                vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
                out[c, i, j] = ((2 * mx * my + C1) * (2 * cxy + C2)) / \
                    ((mx * mx + my * my + C1) * (vx + vy + C2))
    return out


def dssim(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    return 1.0 - ssim_map(x, y).mean()
