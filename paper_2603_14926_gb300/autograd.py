"""torch.autograd.Function wrappers: QD (or any precision) GEMM and batched
Horner evaluation with hand-written adjoint kernels.

Convention.  A K-component number is K float planes whose SUM is the value.
Autograd sees the planes as one tensor of shape (K, ...); the gradient it
carries through these functions is itself a K-component value: the planes of
an incoming gradient together encode d(loss)/d(value) to K-component
precision, and the returned gradients encode d(loss)/d(value) of each input
element the same way.  It is NOT the derivative with respect to each plane
separately (the planes are not independent variables), so mixing these
functions with ordinary elementwise torch arithmetic on the planes does not
give meaningful gradients.

MPGemm:   C = A B;            dA = dC B^T,  dB = A^T dC   (mp_gemm_P with op = T)
MPHorner: y_{b,m} = p_b(x_{b,m}) for real points;
          dcoef_{b,i} = sum_m dy_{b,m} x_{b,m}^i,  dx_{b,m} = dy_{b,m} p_b'(x_{b,m})
          (mp_polyeval_backward_P)
All of them run in the library's kernels; results equal the CPU oracle's bit for bit.
"""

from __future__ import annotations

import torch

from . import gemm, polyeval, polyeval_backward


class MPGemm(torch.autograd.Function):
    """C = A B in K-component arithmetic; A (K, m, k), B (K, k, n) -> C (K, m, n)."""

    @staticmethod
    def forward(ctx, prec, A, B):
        ctx.prec = prec
        ctx.save_for_backward(A, B)
        return gemm(prec, A.detach(), B.detach())

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        dA = gemm(ctx.prec, dC, B, opA=0, opB=1) if ctx.needs_input_grad[1] else None
        dB = gemm(ctx.prec, A, dC, opA=1, opB=0) if ctx.needs_input_grad[2] else None
        return None, dA, dB


class MPHorner(torch.autograd.Function):
    """Batched real-argument Horner: coef (K, sum(n_b+1)), x (K, npoly*npts) -> y."""

    @staticmethod
    def forward(ctx, prec, coef_off, npts, coef, x):
        ctx.prec, ctx.npts = prec, npts
        ctx.save_for_backward(coef_off, coef, x)
        return polyeval(prec, coef_off, coef.detach(), npts, x.detach())

    @staticmethod
    def backward(ctx, dy):
        coef_off, coef, x = ctx.saved_tensors
        want_c, want_x = ctx.needs_input_grad[3], ctx.needs_input_grad[4]
        dcoef, dx = polyeval_backward(ctx.prec, coef_off, coef, ctx.npts, x, dy.contiguous(),
                                      want_dcoef=want_c, want_dx=want_x)
        return None, None, None, dcoef, dx


def mp_gemm(prec, A, B):
    return MPGemm.apply(prec, A, B)


def mp_horner(prec, coef_off, npts, coef, x):
    return MPHorner.apply(prec, coef_off, npts, coef, x)
