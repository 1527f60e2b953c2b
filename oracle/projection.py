"""float64 EWA projection of 3D Gaussians (torch CPU, autograd-able).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper keeps the base 3DGS rasterizer (Supp. "Implementation Details") and
only restricts where it runs (Sec. 3.3 and Supp. "Local Optimization Kernel"),
so this is the base method's projection restated from its definition:

  camera point      p = R mu + t                      (world -> camera)
  image point       u = fx p_x / p_z + cx,  v = fy p_y / p_z + cy
  3D covariance     Sigma = R_q diag(s)^2 R_q^T,  s = exp(log_scale),
                    R_q the rotation of the normalised quaternion q/|q|
  2D covariance     Sigma' = T Sigma T^T + 0.3 I,   T = J R,
                    J = d(u, v)/d p at the point whose x/z, y/z are clamped to
                    1.3x the half field of view (EWA local affine
                    approximation of the perspective map)
  conic             Sigma'^{-1} = (A, B, C) for [[A, B], [B, C]]
  colour            max(0, sum_k sh_k Y_k(d) + 0.5), d = (mu - cam) / |mu - cam|
  opacity           sigmoid(opacity_logit)

Which Gaussians are culled and which tiles they touch are integer decisions
taken by `fp32_index`; this module only supplies the float64 values.
"""
from __future__ import annotations

from typing import Dict

import numpy as np
import torch

from . import sh as shb

T64 = torch.float64


def cam64(cam, dtype=T64) -> Dict[str, object]:
    """The camera as the library sees it: every field rounded to float32 once,
    then widened to float64 (or kept in float32 with dtype=torch.float32)."""
    f = lambda a: torch.tensor(np.asarray(a, dtype=np.float32).astype(np.float64), dtype=dtype)
    return {
        "R": f(np.asarray(cam["R"]).reshape(3, 3)), "t": f(cam["t"]), "pos": f(cam["pos"]),
        "fx": float(np.float32(cam["fx"])), "fy": float(np.float32(cam["fy"])),
        "cx": float(np.float32(cam["cx"])), "cy": float(np.float32(cam["cy"])),
        "W": int(cam["width"]), "H": int(cam["height"]),
    }


def scene64(scene: Dict[str, np.ndarray], requires_grad: bool = False,
            dtype=T64) -> Dict[str, torch.Tensor]:
    """Parameter tensors in float64 (the oracle), or in float32 with
    dtype=torch.float32: the same arithmetic rounded to single precision, which
    measures how far float32 rounding alone moves each value."""
    out = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        out[k] = torch.tensor(np.asarray(scene[k], dtype=np.float64), dtype=dtype,
                              requires_grad=requires_grad)
    return out


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of unit quaternions q = (w, x, y, z), shape [n, 3, 3]."""
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def covariance3d(log_scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    q = quats / torch.linalg.norm(quats, dim=-1, keepdim=True)
    Rq = quat_to_rotmat(q)
    s2 = torch.exp(log_scales) ** 2
    return Rq @ torch.diag_embed(s2) @ Rq.transpose(-1, -2)


def ewa_jacobian(p: torch.Tensor, c) -> torch.Tensor:
    """J = d(u, v)/dp at the clamped point, shape [n, 2, 3]."""
    px, py, pz = p.unbind(-1)
    limx = 1.3 * (0.5 * c["W"] / c["fx"])
    limy = 1.3 * (0.5 * c["H"] / c["fy"])
    tx = torch.clamp(px / pz, -limx, limx) * pz
    ty = torch.clamp(py / pz, -limy, limy) * pz
    zero = torch.zeros_like(pz)
    return torch.stack([
        torch.stack([c["fx"] / pz, zero, -c["fx"] * tx / (pz * pz)], -1),
        torch.stack([zero, c["fy"] / pz, -c["fy"] * ty / (pz * pz)], -1),
    ], -2)


def project(g: Dict[str, torch.Tensor], cam, sh_degree: int) -> Dict[str, torch.Tensor]:
    """2D quantities of every Gaussian for one camera (no culling here), in
    the precision of the parameter tensors."""
    c = cam64(cam, g["means"].dtype)
    p = g["means"] @ c["R"].T + c["t"]
    px, py, pz = p.unbind(-1)
    u = c["fx"] * px / pz + c["cx"]
    v = c["fy"] * py / pz + c["cy"]
    Sigma = covariance3d(g["log_scales"], g["quats"])
    T = ewa_jacobian(p, c) @ c["R"]
    S2 = T @ Sigma @ T.transpose(-1, -2)
    a = S2[:, 0, 0] + 0.3
    b = S2[:, 0, 1]
    cc = S2[:, 1, 1] + 0.3
    det = a * cc - b * b
    conic = torch.stack([cc / det, -b / det, a / det], -1)
    d = g["means"] - c["pos"]
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    Y = shb.basis(d[:, 0], d[:, 1], d[:, 2], sh_degree)
    k = len(Y)
    raw = sum(Y[i][:, None] * g["sh"][:, i, :] for i in range(k)) + 0.5
    rgb = torch.clamp(raw, min=0.0)
    opacity = torch.sigmoid(g["opacity_logits"])
    return {"u": u, "v": v, "z": pz, "conic": conic, "cov2d": torch.stack([a, b, cc], -1),
            "rgb": rgb, "rgb_raw": raw, "opacity": opacity}
