"""Autograd for the PAT operators (arXiv:1605.00133, Sec. 4.3-4.4).

`pat_forward(p0, op)` is f = C A p0 as a differentiable torch function whose backward is the library's
adjoint kernel sequence: d<w, C A p0>/d p0 = A^T C^T w.  `pat_adjoint(f, op)` is the reverse pair.
Both operators are linear in their input and independent of it, so the backward pass needs no
saved activations and no stored time steps: A^T runs its own reverse-time recurrence in O(N)
memory.  (Checkpointing the forward trajectory every sqrt(T) steps would only be needed for
gradients with respect to the medium, e.g. the sound speed, which this library does not expose.)
"""
from __future__ import annotations

import torch


class _Forward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0, op):
        ctx.op = op
        return op.forward(p0.contiguous())

    @staticmethod
    def backward(ctx, grad_f):
        return ctx.op.adjoint(grad_f.contiguous()), None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, op):
        ctx.op = op
        return op.adjoint(f.contiguous())

    @staticmethod
    def backward(ctx, grad_p):
        return ctx.op.forward(grad_p.contiguous()), None


def pat_forward(p0: torch.Tensor, op) -> torch.Tensor:
    """f = C A p0 with backward A^T C^T (op: a PatOperator)."""
    return _Forward.apply(p0, op)


def pat_adjoint(f: torch.Tensor, op) -> torch.Tensor:
    """p = A^T C^T f with backward C A (op: a PatOperator)."""
    return _Adjoint.apply(f, op)
