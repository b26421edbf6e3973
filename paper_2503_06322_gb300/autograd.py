"""Differentiable multilevel transforms.

``recompose(coef, shape)`` maps a level-major coefficient stream to a field
and backpropagates through the library's adjoint kernels
(hpdr_recompose_adjoint); ``decompose(u)`` is the inverse map with
hpdr_decompose_adjoint as its backward.  Both maps are linear, so nothing of
the forward pass is saved: the backward pass runs its own level loop.
"""
import torch

from . import hpdr

__all__ = ["Recompose", "Decompose", "recompose", "decompose"]


class Recompose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, shape):
        ctx.shape = tuple(int(s) for s in shape)
        return hpdr.hpdr_recompose(coef.contiguous(), ctx.shape)

    @staticmethod
    def backward(ctx, grad_u):
        return hpdr.hpdr_recompose_adjoint(grad_u.contiguous()), None


class Decompose(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u):
        ctx.shape = tuple(u.shape)
        return hpdr.hpdr_decompose(u.contiguous())

    @staticmethod
    def backward(ctx, grad_coef):
        return hpdr.hpdr_decompose_adjoint(grad_coef.contiguous(), ctx.shape)


def recompose(coef, shape):
    return Recompose.apply(coef, shape)


def decompose(u):
    return Decompose.apply(u)
