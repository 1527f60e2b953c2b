"""float64 front-to-back alpha compositing of one tile's pixels (torch CPU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Image formation of the base 3DGS method (adopted unchanged, Supp.
"Implementation Details"), restated. For a pixel with centre (x + 1/2, y + 1/2)
and its Gaussians in front-to-back order (every Gaussian whose 3-sigma tile
rectangle holds the pixel's tile, by depth then index):

  d        = pixel centre - (u, v)
  power    = -1/2 (A dx^2 + C dy^2) - B dx dy
  alpha    = min(0.99, opacity * exp(power))
  skip the Gaussian when power > 0 or alpha < 1/255
  stop before a Gaussian when T (1 - alpha) < 1e-4 (it is not composited)
  C       += colour * alpha * T,   T *= (1 - alpha)
  C       += T * background at the end.

The discrete decisions (skip, stop, the 0.99 clamp) are taken here in float64.
A float32 implementation may take a different branch when a value sits on a
threshold; `near` flags those pixels (where the branch could move the result by
more than `value_tol`; `margin` is relative to the threshold) and
`near_ids` the Gaussians involved, so tests can
report them instead of comparing an ill-posed value.
"""
from __future__ import annotations

import torch

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def composite(u, v, conic, opacity, rgb, px, py, bg, margin: float = 1e-4,
              value_tol: float = 1e-4, grad_margin: float = 3e-4, du=None, dv=None):
    """Composite pixels (px, py) (integer pixel indices, [P]) over the ordered
    Gaussians given by 1-D tensors u, v, opacity [L], conic [L, 3], rgb [L, 3].

    Returns a dict: colour [P, 3], T_final [P], n_contrib [P] (one past the
    last list position composited), n_incl [P] (entries composited), stopped
    [P] (the stop rule ended the pixel inside the list), near [P] (bool),
    near_ids (list positions with a threshold decision) and ambiguous [P]:
    pixels with any reached decision (the 1/255 skip, the stop test, the 0.99
    clamp, the power > 0 guard) closer to its threshold than a float32
    evaluation can be trusted to resolve, whatever its effect on the value;
    there float32 may take the other branch, which moves the gradient that
    flows through the pixel's colour. Without `du`/`dv` "closer" means within
    a relative `grad_margin`. With them (per entry, the absolute error of the
    float32 centre u, v against these values) it is twice a first-order bound
    of the float32 error of the decided quantity: the exponent moves by
    |d power/du| du + |d power/dv| dv, plus 4e-6 of the size of its terms and
    1e-6 (conic, exponential and opacity rounding), alpha by the same
    relative amount, and the stop test by that of its own alpha plus the sum
    over the entries composited before it of alpha/(1 - alpha) times theirs
    (the transmittance's relative error), plus 1.2e-7 per factor."""
    P = px.shape[0]
    L = u.shape[0]
    dt = u.dtype
    if L == 0:
        zero = torch.zeros(P, dtype=torch.int64)
        return {"colour": bg[None, :].expand(P, 3).clone(), "T_final": torch.ones(P, dtype=dt),
                "n_contrib": zero, "n_incl": zero.clone(),
                "stopped": torch.zeros(P, dtype=torch.bool),
                "near": torch.zeros(P, dtype=torch.bool),
                "ambiguous": torch.zeros(P, dtype=torch.bool),
                "near_ids": torch.zeros(0, dtype=torch.int64)}
    dx = (px.to(dt)[:, None] + 0.5) - u[None, :]
    dy = (py.to(dt)[:, None] + 0.5) - v[None, :]
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    power = -0.5 * (A[None, :] * dx * dx + C[None, :] * dy * dy) - B[None, :] * dx * dy
    raw = opacity[None, :] * torch.exp(power)
    alpha = torch.clamp(raw, max=ALPHA_MAX)
    with torch.no_grad():
        skip = (power > 0) | (alpha < ALPHA_MIN)
    a_eff = torch.where(skip, torch.zeros_like(alpha), alpha)
    one_minus = 1.0 - a_eff
    ones = torch.ones((P, 1), dtype=dt)
    T_before = torch.cat([ones, torch.cumprod(one_minus, dim=1)[:, :-1]], dim=1)
    with torch.no_grad():
        test = T_before * (1.0 - alpha)
        stop = (~skip) & (test < T_MIN)
        before_stop = torch.cumsum(stop.to(torch.int64), dim=1) == 0
        incl = (~skip) & before_stop
    w = torch.where(incl, a_eff * T_before, torch.zeros_like(a_eff))
    T_final = torch.prod(torch.where(incl, one_minus, torch.ones_like(one_minus)), dim=1)
    colour = w @ rgb + T_final[:, None] * bg[None, :]
    with torch.no_grad():
        pos = torch.arange(1, L + 1, dtype=torch.int64)[None, :].expand(P, L)
        n_contrib = torch.where(incl, pos, torch.zeros_like(pos)).max(dim=1).values
        live = before_stop | stop  # decisions actually reached
        Tb = T_before.detach()
        al = alpha.detach()
        # alpha at the 1/255 threshold: the entry's share is ~alpha*T*(|c|+1)
        near_skip = live & (power <= 0) & ((al / ALPHA_MIN - 1.0).abs() < margin)
        sig_skip = near_skip & (ALPHA_MIN * Tb * 3.0 > value_tol)
        # stop test at its threshold: the entry's share is alpha*T*(|c|+1)
        near_stop = live & (~skip) & ((test / T_MIN - 1.0).abs() < margin)
        sig_stop = near_stop & (al * Tb * 3.0 > value_tol)
        # opacity clamp: value is continuous, gradient is not
        near_clamp = live & ((raw.detach() / ALPHA_MAX - 1.0).abs() < margin)
        near = (sig_skip | sig_stop).any(dim=1)
        near_ids = torch.nonzero((near_skip | near_stop | near_clamp).any(dim=0)).flatten()
        pw = power.detach()
        if du is None:
            m_alpha = torch.full_like(pw, grad_margin)
            m_stop = m_alpha
            m_guard = torch.full_like(pw, 1e-6)
        else:
            gx = (A[None, :] * dx + B[None, :] * dy).detach().abs()
            gy = (B[None, :] * dx + C[None, :] * dy).detach().abs()
            terms = (0.5 * (A[None, :].abs() * dx * dx + C[None, :].abs() * dy * dy) +
                     (B[None, :] * dx * dy).abs()).detach()
            dpow = gx * du.detach()[None, :] + gy * dv.detach()[None, :] + 4e-6 * terms + 1e-6
            m_alpha = 2.0 * dpow
            a_inc = torch.where(incl, al, torch.zeros_like(al))
            share = a_inc / (1.0 - a_inc) * dpow + 1.2e-7
            errT = torch.cumsum(share, dim=1) - share  # over the entries before
            m_stop = 2.0 * (errT + al / (1.0 - al) * dpow + 1e-6)
            m_guard = 2.0 * dpow
        amb = live & (((pw <= 0) & ((al / ALPHA_MIN - 1.0).abs() < m_alpha)) |
                      ((~skip) & ((test / T_MIN - 1.0).abs() < m_stop)) |
                      ((raw.detach() / ALPHA_MAX - 1.0).abs() < m_alpha) |
                      (pw.abs() < m_guard))
        ambiguous = amb.any(dim=1)
    return {"colour": colour, "T_final": T_final, "n_contrib": n_contrib,
            "n_incl": incl.sum(dim=1), "stopped": stop.any(dim=1), "near": near,
            "near_ids": near_ids, "ambiguous": ambiguous}
