"""PyTorch autograd wrapper of ln psi: forward nk_rbm_logpsi, backward the
hand-written analytic kernel nk_rbm_logpsi_backward (the RBM log-derivatives of
Sec. 2.2.5 contracted with the upstream gradient, theta recomputed from sigma).

Parameters are one flat tensor in the order (a, b, W row-major), complex128 for
a complex RBM (holomorphic; PyTorch's conjugate-Wirtinger convention, so the
backward returns sum_s conj(O_sk) g_s) or float64 for a real one.
"""
from __future__ import annotations

import torch

from . import nk


class RbmLogPsi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, rbm: nk.Rbm, sigma, prec: int = nk.NK_PREC_FP32):
        n, m = rbm.n, rbm.m
        with torch.no_grad():
            p = params.detach()
            if rbm.is_complex:
                p = torch.view_as_real(p.to(torch.complex128)).reshape(-1)
                rbm.a.copy_(p[:2 * n])
                rbm.b.copy_(p[2 * n:2 * (n + m)])
                rbm.w.copy_(p[2 * (n + m):])
            else:
                p = p.to(torch.float64)
                rbm.a.copy_(p[:n])
                rbm.b.copy_(p[n:n + m])
                rbm.w.copy_(p[n + m:])
            nk.nk_rbm_prepare(rbm)
            lp = nk.nk_rbm_logpsi(rbm, sigma, prec)
        ctx.rbm, ctx.prec = rbm, prec
        ctx.save_for_backward(sigma)
        return lp if rbm.is_complex else lp.real.contiguous()

    @staticmethod
    def backward(ctx, grad_out):
        (sigma,) = ctx.saved_tensors
        g = grad_out.to(torch.complex128).contiguous()
        grad = nk.nk_rbm_logpsi_backward(ctx.rbm, sigma, g, ctx.prec)
        return grad, None, None, None


def logpsi(params, rbm: nk.Rbm, sigma, prec: int = nk.NK_PREC_FP32):
    """ln psi(sigma) as a differentiable function of the flat parameter tensor."""
    return RbmLogPsi.apply(params, rbm, sigma, prec)


class FfnnLogPsi(torch.autograd.Function):
    """ln psi of a dense ln cosh network (Sec. 2.2.2, FFNN): forward
    nk_ffnn_logpsi, backward nk_ffnn_backward (the chain rule through the
    layers in hand-written kernels).  Parameters: one flat tensor in the
    network's order, complex128 (holomorphic) or float64."""

    @staticmethod
    def forward(ctx, params, net: nk.Ffnn, sigma):
        with torch.no_grad():
            p = params.detach()
            if net.is_complex:
                p = torch.view_as_real(p.to(torch.complex128)).reshape(-1)
            net.params.copy_(p.to(torch.float64))
            lp = nk.nk_ffnn_logpsi(net, sigma)
        ctx.net = net
        ctx.save_for_backward(sigma)
        return lp if net.is_complex else lp.real.contiguous()

    @staticmethod
    def backward(ctx, grad_out):
        (sigma,) = ctx.saved_tensors
        grad = nk.nk_ffnn_backward(ctx.net, sigma, grad_out.to(torch.complex128).contiguous())
        return grad, None, None


def ffnn_logpsi(params, net: nk.Ffnn, sigma):
    """ln psi(sigma) of the network as a differentiable function of its flat parameters."""
    return FfnnLogPsi.apply(params, net, sigma)
