"""torch.autograd wrappers around the C ABI.

The backward of the descriptor is the library's hand-written adjoint
(``dmcr_descriptor_vjp``): it recomputes every shifted pair instead of storing the N x K
ensemble (Sec. 3.4: the exact gradient through the convolve-threshold-reduce pipeline
and every multigrid level at once).
"""
from __future__ import annotations

import torch

from . import _lib


class S2Descriptor(torch.autograd.Function):
    """D = [w_1 S_bar_1, w_2 S_bar_2, ...] of one field (Sec. 3.2, Eq. mg)."""

    @staticmethod
    def forward(ctx, field, params):
        desc = _lib.descriptor(field.contiguous(), params)
        ctx.save_for_backward(field)
        ctx.params = params
        return desc

    @staticmethod
    def backward(ctx, grad_desc):
        (field,) = ctx.saved_tensors
        g = _lib.descriptor_vjp(field.contiguous(), grad_desc.contiguous().float(), ctx.params)
        return g, None


class S2DescriptorBatched(torch.autograd.Function):
    """Descriptors of many fields of mixed sizes, one fused launch per phase."""

    @staticmethod
    def forward(ctx, params, *fields):
        fields = [f.contiguous() for f in fields]
        descs = [torch.empty(_lib.dmcr_descriptor_length(p), dtype=torch.float32, device=f.device)
                 for p, f in zip(params, fields)]
        _lib.dmcr_descriptor_batched(list(params), fields, descs)
        ctx.save_for_backward(*fields)
        ctx.params = list(params)
        return tuple(descs)

    @staticmethod
    def backward(ctx, *grad_descs):
        fields = ctx.saved_tensors
        grads = [torch.zeros(_lib.dmcr_descriptor_length(p), dtype=torch.float32, device=f.device)
                 if g is None else g.contiguous().float() for p, f, g in zip(ctx.params, fields, grad_descs)]
        out = [torch.empty_like(f) for f in fields]
        _lib.dmcr_descriptor_vjp_batched(ctx.params, list(fields), grads, out)
        return (None, *out)


class DMCRLoss(torch.autograd.Function):
    """L = E (1 + lambda0 E_bc) of Sec. 3.1 (or its SQUARED form); forward and gradient come
    from one dmcr_loss_grad call, the gradient is kept for backward."""

    @staticmethod
    def forward(ctx, field, target_desc, params, opts):
        loss, grad = _lib.loss_grad(field.contiguous(), target_desc.contiguous(), params, opts)
        ctx.save_for_backward(grad)
        return loss[4].clone()

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad * grad_out, None, None, None


def s2_descriptor(field: torch.Tensor, params) -> torch.Tensor:
    return S2Descriptor.apply(field, params)


def s2_descriptor_batched(fields, params):
    return S2DescriptorBatched.apply(tuple(params), *fields)


def dmcr_loss(field: torch.Tensor, target_desc: torch.Tensor, params, opts=None) -> torch.Tensor:
    return DMCRLoss.apply(field, target_desc, params, opts or _lib.LossOpts())
