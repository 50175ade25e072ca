"""Differentiable projection operators for PyTorch.

ForwardProject: y = A x with the interpolated projector; its backward
applies the exact transpose of the same discretisation (every sample scatters
h * trilinear weight * grad into its 8 corner voxels), so gradients of any
loss of A x are exact up to FP32 rounding.

AdjointProject: x = A^T y (exact transpose); its backward is A.

Both run entirely in the CUDA library through the C ABI binding.
"""
from __future__ import annotations

import torch

from . import tigre


class ForwardProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol: torch.Tensor, geometry: "tigre.Geometry") -> torch.Tensor:
        ctx.geometry = geometry
        ctx.vol_dtype = vol.dtype
        return geometry.forward(vol.contiguous(), dtype=torch.float32)

    @staticmethod
    def backward(ctx, grad_proj: torch.Tensor):
        g = ctx.geometry.backward(grad_proj.contiguous().float(), weight="adjoint",
                                  dtype=torch.float32)
        return g.to(ctx.vol_dtype), None


class AdjointProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, proj: torch.Tensor, geometry: "tigre.Geometry") -> torch.Tensor:
        ctx.geometry = geometry
        ctx.proj_dtype = proj.dtype
        return geometry.backward(proj.contiguous(), weight="adjoint", dtype=torch.float32)

    @staticmethod
    def backward(ctx, grad_vol: torch.Tensor):
        g = ctx.geometry.forward(grad_vol.contiguous().float(), dtype=torch.float32)
        return g.to(ctx.proj_dtype), None


def forward_project(vol: torch.Tensor, geometry: "tigre.Geometry") -> torch.Tensor:
    """Differentiable A x (float32 projections)."""
    return ForwardProject.apply(vol, geometry)


def adjoint_project(proj: torch.Tensor, geometry: "tigre.Geometry") -> torch.Tensor:
    """Differentiable exact A^T y (float32 volume)."""
    return AdjointProject.apply(proj, geometry)
