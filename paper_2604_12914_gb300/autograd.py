"""torch.autograd wrapper of the Jacobian-vector product (marshalling only).

``SigmaFn.apply(ctx, x1, x2)`` returns sigma = A X (Sec. 2.2 Jacobian) for CUDA complex128
tensors x1 [o, v], x2 [o, o, v, v] (x2 antisymmetric in (i,j) and (a,b)); its backward is
the transpose product computed by libcclr (cc_lr_sigma_T), so a graph built on sigma can be
differentiated without forming A.

Conventions.  sigma is complex-linear (holomorphic) in X, so PyTorch expects
grad_x = J^H grad_out = conj(J^T conj(grad_out)).  The library's transpose product is
defined with the unique-amplitude weights (1 for singles, 1/4 for doubles); for plain
tensor coordinates the doubles cotangent is passed scaled by 4 and the doubles result
divided by 4, which gives J^T on the antisymmetric subspace (the projection onto
antisymmetric tensors is part of the returned gradient).
"""
from __future__ import annotations

import torch

from . import binding


class SigmaFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cctx: "binding.Context", x1: torch.Tensor, x2: torch.Tensor):
        if not (x1.is_cuda and x2.is_cuda):
            raise ValueError("SigmaFn needs CUDA tensors (libcclr has no CPU path)")
        # resolve_conj: a lazily conjugated view would hand the library unconjugated memory
        x1c = x1.detach().to(torch.complex128).resolve_conj().contiguous()
        x2c = x2.detach().to(torch.complex128).resolve_conj().contiguous()
        s1 = torch.empty_like(x1c)
        s2 = torch.empty_like(x2c)
        torch.cuda.current_stream().synchronize()
        cctx.sigma_into(x1c, x2c, s1, s2)
        fctx.cctx = cctx
        return s1, s2

    @staticmethod
    def backward(fctx, g1: torch.Tensor, g2: torch.Tensor):
        cctx = fctx.cctx
        y1 = g1.conj().to(torch.complex128).resolve_conj().contiguous()
        y2 = (4.0 * g2.conj()).to(torch.complex128).resolve_conj().contiguous()
        z1 = torch.empty_like(y1)
        z2 = torch.empty_like(y2)
        torch.cuda.current_stream().synchronize()
        cctx.sigma_into(y1, y2, z1, z2, transpose=True)
        return None, z1.conj(), (0.25 * z2).conj()


def sigma(cctx: "binding.Context", x1: torch.Tensor, x2: torch.Tensor):
    """Differentiable sigma = A X."""
    return SigmaFn.apply(cctx, x1, x2)
