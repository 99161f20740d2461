"""Differentiable window fusion behind torch.autograd.Function (marshalling only: the forward
and the hand-written backward run in libvbh's kernels, see vbh_diff_* in include/vbh.h)."""
from __future__ import annotations

import torch

from . import vbh as V


class DiffFusion:
    """Fixed sample voxels and nominal poses of one window; call `loss(depth, xi)`.

    `T0` (n_frames x 3 x 4 float32 [R | t]) fixes the masks and cells; pass `T0=None` and the
    nominal twists `xi0` to take T0 = exp(xi0) rounded to float32 on the device."""

    def __init__(self, voxel_size, trunc, width, height, fx, fy, cx, cy, n_frames, samples,
                 depth0, T0=None, xi0=None):
        cfg = V.vbh_diff_config(voxel_size=voxel_size, trunc=trunc, width=width, height=height,
                                fx=fx, fy=fy, cx=cx, cy=cy, n_frames=n_frames)
        self.cfg = cfg
        self.h = V.vbh_diff_create(cfg, torch.cuda.current_stream().cuda_stream)
        self.samples = samples.to(torch.int32).contiguous()
        if T0 is None:
            T0 = torch.empty((n_frames, 3, 4), dtype=torch.float32, device=samples.device)
            V.vbh_diff_poses(self.h, xi0.to(torch.float32).contiguous(), T0)
        self.T0 = T0.to(torch.float32).contiguous()
        words = (n_frames + 31) // 32
        self.masks = torch.empty((self.samples.shape[0], words), dtype=torch.int32,
                                 device=self.samples.device)
        V.vbh_diff_masks(self.h, self.samples, depth0.contiguous(), self.T0, self.masks)

    def close(self):
        if getattr(self, "h", None):
            V.vbh_diff_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, depth, xi):
        c = self.cfg
        if depth.dtype != torch.float32 or tuple(depth.shape) != (c.n_frames, c.height, c.width):
            raise ValueError(f"depth must be float32 [{c.n_frames}, {c.height}, {c.width}], got "
                             f"{depth.dtype} {tuple(depth.shape)}")
        if xi.dtype != torch.float32 or tuple(xi.shape) != (c.n_frames, 6):
            raise ValueError(f"xi must be float32 [{c.n_frames}, 6], got {xi.dtype} "
                             f"{tuple(xi.shape)}")

    def forward_raw(self, depth, xi):
        self._check(depth, xi)
        F = torch.empty(self.samples.shape[0], dtype=torch.float32, device=depth.device)
        loss = torch.zeros((), dtype=torch.float64, device=depth.device)
        V.vbh_diff_forward(self.h, self.samples, depth.contiguous(), self.T0, xi.contiguous(),
                           self.masks, F, loss)
        return loss, F

    def backward_raw(self, depth, xi, F):
        self._check(depth, xi)
        # dense outputs: the kernels write them in the dense layout whatever the inputs' strides
        gd = torch.empty(depth.shape, dtype=torch.float32, device=depth.device)
        gx = torch.empty(xi.shape, dtype=torch.float32, device=xi.device)
        V.vbh_diff_backward(self.h, self.samples, depth.contiguous(), self.T0, xi.contiguous(),
                            self.masks, F, gd, gx)
        return gd, gx

    def loss(self, depth: torch.Tensor, xi: torch.Tensor) -> torch.Tensor:
        return _DiffFusionFn.apply(depth, xi, self)


class _DiffFusionFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, depth, xi, module):
        loss, F = module.forward_raw(depth, xi)
        ctx.module = module
        ctx.save_for_backward(depth, xi, F)
        return loss

    @staticmethod
    def backward(ctx, g):
        depth, xi, F = ctx.saved_tensors
        gd, gx = ctx.module.backward_raw(depth, xi, F)
        s = g.to(torch.float32)
        return gd * s, gx * s, None
