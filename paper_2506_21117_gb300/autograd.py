"""torch.autograd.Function over the local rasterizer.

Forward: cls_project_and_bin (active Gaussians re-projected), the per-tile
sort, cls_render_forward on the active tiles (no fused loss). Backward: the
hand-written adjoint cls_render_backward, which walks each pixel's list front
to back again up to its last contributor, recomputing the transmittance in
front of every Gaussian with the forward pass's own operations and taking the
colour behind it as the final colour minus what has been composited, so
nothing per (pixel, Gaussian) is stored. The gradient reaches only the rows
of the active set O^t (Supp. "Local Optimization Kernel", item 3); the rows of
frozen Gaussians get zero. Pixels of inactive tiles are returned as zero: no
Gaussian of O^t reaches them, so their gradient is not needed (Sec. 3.3).
"""
from __future__ import annotations

from typing import List

import torch

from .update import Batch, SceneState


class ActiveRasterizer:
    """Holds the device buffers of one scene and its views for the Function.

    The buffers are shared by every call: a forward must be followed by its
    own backward before the next forward (each call bumps `generation`, and a
    backward of an older call raises). The parameters must not change in place
    between a forward and its backward (torch's version check raises)."""

    def __init__(self, state: SceneState, cams, bg=(0.0, 0.0, 0.0), layout: int = 1):
        self.state = state
        self.cams = list(cams)
        self.bg = tuple(float(x) for x in bg)
        # the caller's optimiser may move any row, so the static prefix is
        # rebuilt on every call
        self.batch = Batch([state], [self.cams], state.params.device, layout,
                           prefix_cache=False)
        self.batch.plan_capacity()
        self.generation = 0

    def __call__(self, params: torch.Tensor) -> List[torch.Tensor]:
        """Images [3, H, W] per view; differentiable w.r.t. `params`, which must
        be the scene's parameter tensor (rows [n][row_stride] on the device)."""
        flat = _RasterizeActive.apply(params, self)
        return self.batch.per_view(flat, 3)


class _RasterizeActive(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, rast: ActiveRasterizer):
        st = rast.state
        if params.data_ptr() != st.params.data_ptr():
            raise ValueError("params must be the rasterizer's scene parameter tensor")
        b = rast.batch
        b.status.zero_()
        b.project_and_bin(1)
        need = int(b.n_pairs.item())
        if need > b.capacity:
            # the caller's optimiser moved or grew Gaussians past the planned
            # pair capacity: size the key buffers again and bin once more
            b.allocate_keys(int(need * 1.5) + (1 << 16))
            b.status.zero_()
            b.project_and_bin(1)
        b.sort()
        b.image.zero_()
        b.forward(0, rast.bg)
        b.check_status()
        rast.generation += 1
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.save_for_backward(params)
        return b.image.clone()

    @staticmethod
    def backward(ctx, grad_image: torch.Tensor):
        rast = ctx.rast
        ctx.saved_tensors  # raises if the parameters changed in place since the forward
        if ctx.generation != rast.generation:
            raise RuntimeError("ActiveRasterizer: the buffers hold a later forward call; run "
                               "each forward's backward before the next forward")
        b = rast.batch
        st = rast.state
        b.dL_dimage.copy_(grad_image.contiguous().view(-1))
        b.backward()
        grad = torch.zeros_like(st.params)
        A = st.n_active
        if A:
            rows = b.grads[: A * st.stride].view(A, st.stride)
            grad.index_copy_(0, st.active_idx[:A].long(), rows)
        return grad, None
