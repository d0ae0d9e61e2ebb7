"""Reverse-mode differentiation of the FP64-accurate transforms.

Every transform here is linear, so the gradient of a real loss with respect to
its input is the adjoint transform applied to the output gradient (PyTorch's
convention for complex tensors: the gradient is dL/dRe + i dL/dIm, and a
linear map A sends the output gradient g to A^H g).  The adjoints run through
the same pipeline as the transforms themselves, as two more plan directions of
libozfft:

    forward  y = F x            backward  F^H g = conj(F conj g)   (ADJOINT)
    inverse  y = (1/n) F^H x    backward  (1/n) F g                (INVERSE_ADJOINT)

F(k, j) = exp(-2 pi i jk / n) is the DFT of Eq. (3), F^H / n its inverse
(Eq. (4)).  The adjoint of an adjoint is the original direction, so the
backward pass is itself differentiable (higher-order gradients).
"""
from __future__ import annotations

import torch

from . import ozfft

_ADJ = {ozfft.FORWARD: ozfft.ADJOINT, ozfft.ADJOINT: ozfft.FORWARD,
        ozfft.INVERSE: ozfft.INVERSE_ADJOINT, ozfft.INVERSE_ADJOINT: ozfft.INVERSE}


class OzFFTFunction(torch.autograd.Function):
    """y = T x along the last axis for T in {F, F^H / n, F^H, F / n}."""

    @staticmethod
    def forward(ctx, x, direction, K, L, nprimes):
        ctx.cfg = (direction, K, L, nprimes)
        return ozfft.transform(x, direction, K, L, nprimes)

    @staticmethod
    def backward(ctx, g):
        direction, K, L, nprimes = ctx.cfg
        if g.dtype != torch.complex128:
            g = g.to(torch.complex128)
        return OzFFTFunction.apply(g.contiguous(), _ADJ[direction], K, L, nprimes), None, None, None, None


def fft(x, K=3, L=1, nprimes=2):
    """Differentiable DFT (Eq. (3)) of the last axis of a CUDA complex128 tensor."""
    return OzFFTFunction.apply(x, ozfft.FORWARD, K, L, nprimes)


def ifft(x, K=3, L=1, nprimes=2):
    """Differentiable inverse DFT (Eq. (4)) of the last axis."""
    return OzFFTFunction.apply(x, ozfft.INVERSE, K, L, nprimes)
