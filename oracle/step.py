"""Full-image render, loss and exact active-set gradient in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.3 ("Local Optimization Kernel") and Supp. "Local Optimization Kernel":
the local kernel renders only tiles touched by O^t and back-propagates only
into O^t, and must produce exactly the gradients that O^t receives in a
full-scene 3DGS step. This module computes that reference: the whole image of
every view (every tile, static Gaussians included), the loss over all pixels,
and the gradient of that loss by reverse-mode autodiff in float64, restricted
afterwards to O^t.

Loss reading (the paper adopts the base method's photometric loss; the
workloads use L1 or L2): L = (1/V) sum_views (1 / (3 H W)) sum_pixels,channels
l(C - C*), l = |.| or (.)^2, normalised by the full image so that the gradient
of O^t does not depend on how many tiles are rendered.

The per-pixel Gaussian lists use the float32 decisions of `fp32_index` (culling,
tile rectangles, depth order); all values are float64.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import fp32_index as fx
from .composite import composite
from .projection import project, scene64, T64

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def tile_list(pidx: Dict[str, np.ndarray], tx: int, ty: int) -> np.ndarray:
    """Gaussians whose rectangle holds tile (tx, ty), by (depth bits, index)."""
    sel = pidx["valid"] & (pidx["tx0"] <= tx) & (pidx["tx1"] >= tx) & \
        (pidx["ty0"] <= ty) & (pidx["ty1"] >= ty)
    ids = np.flatnonzero(sel)
    order = np.lexsort((ids, pidx["zbits"][ids]))
    return ids[order]


def saturated_length(u, v, conic, opacity, rgb, px, py, bg, start: int = 256) -> int:
    """Length of the list prefix that holds every composited entry of every
    pixel: the first of 256, 512, 1024, ... (or the whole list) at which the
    stop rule has ended all pixels. Entries behind it are composited at no
    pixel, so compositing the prefix gives the same result as the whole
    list (used to bound the oracle's work on long lists)."""
    L = int(u.shape[0])
    n = start
    with torch.no_grad():
        while n < L:
            if bool(composite(u[:n], v[:n], conic[:n], opacity[:n], rgb[:n], px, py,
                              bg)["stopped"].all()):
                return n
            n *= 2
    return L


def tile_pixels(cam, tx: int, ty: int):
    W, H = int(cam["width"]), int(cam["height"])
    xs = np.arange(tx * fx.TILE, min((tx + 1) * fx.TILE, W))
    ys = np.arange(ty * fx.TILE, min((ty + 1) * fx.TILE, H))
    X, Y = np.meshgrid(xs, ys)
    return torch.tensor(X.ravel()), torch.tensor(Y.ravel())


def loss_terms(colour, target, kind: str):
    d = colour - target
    return d.abs() if kind == "l1" else d * d


SSIM_LOSSES = ("ssim", "l1+ssim")
# |C - C*| below which the sign of an L1 term is ambiguous between float32 and
# float64 (the GPU's pixels agree with the oracle's to about 1e-6)
KINK_TOL = 1e-5


def view_loss_ssim(image, target, kind: str):
    """Per-view loss of the D-SSIM kinds over the whole image: "ssim" is
    D-SSIM alone, "l1+ssim" the base optimiser's (1 - lambda) L1 + lambda
    D-SSIM with the L1 mean over 3 H W values."""
    from . import ssim as os_
    d = os_.dssim(image, target)
    if kind == "ssim":
        return d
    return (1.0 - os_.LAMBDA) * (image - target).abs().mean() + os_.LAMBDA * d


def render(scene: Dict[str, np.ndarray], cams: Sequence, sh_degree: int,
           bg=(0.0, 0.0, 0.0), targets: Optional[Sequence[np.ndarray]] = None,
           loss: str = "l1", need_grad: bool = False,
           tiles: Optional[Sequence[Sequence[tuple]]] = None,
           margin: float = 1e-4, dtype=T64, truncate: bool = False,
           hold_ambiguous: bool = False, held: Optional[Sequence[np.ndarray]] = None):
    """Render every view (or only `tiles[j]` of view j).

    Returns a dict with per-view `image` [3, H, W] (NaN where not rendered),
    `T_final`, `n_contrib`, `n_incl`, `near` ([H, W] bools), the per-view index-mode
    projections `pidx`, `near_ids` (set of Gaussian ids with a threshold
    decision), `loss` (float, over rendered pixels) and, if `need_grad`, the
    float64 gradient of every parameter array (`grads`, numpy, same shapes as
    the scene). The loss is the mean over views of the per-view loss; for the
    D-SSIM kinds (`SSIM_LOSSES`, whole images only) `dL_dimage` holds the
    float64 gradient of the loss with respect to each view's image.

    hold_ambiguous=True holds the colour of every pixel with an ambiguous
    threshold decision (composite's `ambiguous`, and for the L1 kinds a
    channel within KINK_TOL of its target) constant in the loss: the
    loss value is unchanged, but no gradient flows through that pixel's
    compositing, so the gradient no longer depends on a branch that float32
    and float64 may take differently. `held` (per view, [H, W] bools) gives
    those pixels explicitly instead. The pixels held are returned in
    `held` (per view).

    truncate=True composites each tile over the list prefix that holds every
    composited entry (`saturated_length`): the same result with less work on
    long lists.

    dtype=torch.float32 runs the same arithmetic in single precision (every
    value, every sum); set against the float64 result it measures the rounding
    error that float32 arithmetic alone leaves in each pixel and gradient. The
    discrete decisions stay those of `fp32_index` either way."""
    if loss in SSIM_LOSSES and tiles is not None:
        raise ValueError("the D-SSIM losses are defined on whole images")
    V = len(cams)
    bg_t = torch.tensor(bg, dtype=dtype)
    g = scene64(scene, requires_grad=need_grad, dtype=dtype)
    out = {"image": [], "T_final": [], "n_contrib": [], "n_incl": [], "near": [], "pidx": [],
           "near_ids": set(), "loss": 0.0, "dL_dimage": [], "held": []}
    proj_outs, proj_grads = [], []
    for j, cam in enumerate(cams):
        W, H = int(cam["width"]), int(cam["height"])
        Tx, Ty = fx.tiles_of(cam)
        pidx = fx.project_index(scene, cam)
        out["pidx"].append(pidx)
        P = project(g, cam, sh_degree)
        leaves = {k: P[k].detach().clone().requires_grad_(need_grad)
                  for k in ("u", "v", "conic", "opacity", "rgb")}
        # how far the float32 centres (which the library computes exactly as
        # fp32_index does) lie from these values: the scale of the float32
        # error in every exponent, for the ambiguity test
        err_u = torch.from_numpy(np.abs(pidx["u"].astype(np.float64) -
                                        P["u"].detach().double().numpy()))
        err_v = torch.from_numpy(np.abs(pidx["v"].astype(np.float64) -
                                        P["v"].detach().double().numpy()))
        img = np.full((3, H, W), np.nan)
        Tf = np.full((H, W), np.nan)
        nc = np.full((H, W), -1, np.int64)
        ni = np.full((H, W), -1, np.int64)
        near = np.zeros((H, W), bool)
        hold = np.zeros((H, W), bool)
        tgt = None if targets is None else torch.tensor(
            np.asarray(targets[j], np.float64), dtype=dtype)
        norm = 1.0 / (3.0 * H * W * V)
        todo = tiles[j] if tiles is not None else [(x, y) for y in range(Ty) for x in range(Tx)]
        whole = torch.zeros(3, H * W, dtype=dtype) if loss in SSIM_LOSSES else None
        for (tx, ty) in todo:
            ids_np = tile_list(pidx, tx, ty)
            ids = torch.tensor(ids_np, dtype=torch.int64)
            px, py = tile_pixels(cam, tx, ty)
            if truncate:
                n_keep = saturated_length(leaves["u"][ids], leaves["v"][ids],
                                          leaves["conic"][ids], leaves["opacity"][ids],
                                          leaves["rgb"][ids], px, py, bg_t)
                ids_np, ids = ids_np[:n_keep], ids[:n_keep]
            cr = composite(leaves["u"][ids], leaves["v"][ids], leaves["conic"][ids],
                           leaves["opacity"][ids], leaves["rgb"][ids], px, py, bg_t, margin,
                           du=err_u[ids].to(dtype), dv=err_v[ids].to(dtype))
            col = cr["colour"]
            pxn, pyn = px.numpy(), py.numpy()
            if held is not None or hold_ambiguous:
                if held is not None:
                    h = torch.from_numpy(np.asarray(held[j], bool)[pyn, pxn])
                else:
                    h = cr["ambiguous"]
                    if tgt is not None and loss in ("l1", "l1+ssim"):
                        h = h | ((col.detach() - tgt[:, py, px].T).abs() < KINK_TOL).any(dim=1)
                hold[pyn, pxn] = h.numpy()
                col = torch.where(h[:, None], col.detach(), col)
            img[:, pyn, pxn] = col.detach().numpy().T
            Tf[pyn, pxn] = cr["T_final"].detach().numpy()
            nc[pyn, pxn] = cr["n_contrib"].numpy()
            ni[pyn, pxn] = cr["n_incl"].numpy()
            near[pyn, pxn] = cr["near"].numpy()
            out["near_ids"].update(ids_np[cr["near_ids"].numpy()].tolist())
            if whole is not None:
                whole = whole.index_put((torch.arange(3)[:, None], (py * W + px)[None, :]),
                                        col.T)
            elif tgt is not None:
                lt = loss_terms(col, tgt[:, py, px].T, loss).sum() * norm
                out["loss"] += float(lt.detach())
                if need_grad and lt.requires_grad:
                    lt.backward()
        if whole is not None and tgt is not None:
            image_t = whole.view(3, H, W)
            if need_grad:
                image_t.retain_grad()
            lv = view_loss_ssim(image_t, tgt, loss) / V
            out["loss"] += float(lv.detach())
            if need_grad and lv.requires_grad:
                lv.backward()
                out["dL_dimage"].append(image_t.grad.numpy().copy())
        out["image"].append(img)
        out["T_final"].append(Tf)
        out["n_contrib"].append(nc)
        out["n_incl"].append(ni)
        out["near"].append(near)
        out["held"].append(hold)
        if need_grad:
            for k, leaf in leaves.items():
                if leaf.grad is not None:
                    proj_outs.append(P[k])
                    proj_grads.append(leaf.grad)
    if need_grad:
        if proj_outs:
            torch.autograd.backward(proj_outs, proj_grads)
        out["grads"] = {k: (g[k].grad.numpy().astype(np.float64) if g[k].grad is not None
                            else np.zeros(g[k].shape)) for k in PARAM_KEYS}
    return out


def loss_value(scene, cams, sh_degree, targets, loss="l1", bg=(0.0, 0.0, 0.0)) -> float:
    return render(scene, cams, sh_degree, bg, targets, loss, need_grad=False)["loss"]


def active_tiles(scene, cams, active: np.ndarray) -> List[List[tuple]]:
    """Per view, the tiles touched by a non-culled Gaussian of O^t."""
    res = []
    for cam in cams:
        pidx = fx.project_index(scene, cam)
        m = fx.tile_mask(pidx, active, cam)
        ys, xs = np.nonzero(m)
        res.append(list(zip(xs.tolist(), ys.tolist())))
    return res


def local_step_reference(scene, cams, sh_degree, targets, active, loss="l1",
                         bg=(0.0, 0.0, 0.0), dtype=T64, hold_ambiguous: bool = False,
                         held=None):
    """Full-image gradient restricted to O^t (rows of static Gaussians are
    zero), plus the full-image render (`render` gives the options)."""
    r = render(scene, cams, sh_degree, bg, targets, loss, need_grad=True, dtype=dtype,
               hold_ambiguous=hold_ambiguous, held=held)
    for k in PARAM_KEYS:
        r["grads"][k][~active] = 0.0
    return r
