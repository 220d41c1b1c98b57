"""torch.autograd binding of the sampled GCP loss.

Forward: the sampled loss F~ = sum_s w_s f(x_s, m_s) of one sample set
(Sec. 3.1.1 weights, Eq. gcp-model), reduced in FP64 by the fused kernel.
Backward: the same fused kernel in gradient mode -- it redraws the samples
from their counters and recomputes the Khatri-Rao row products, so nothing
per sample is stored between the passes -- scaled on the device by the
incoming gradient (Eq. gcp-gradient).  All arithmetic runs in libgcp.so;
this module only moves pointers.
"""
from __future__ import annotations

import torch

from . import GcpContext, _check, _ptr, load


def _stage_factors(ctx: GcpContext, factors):
    """Copy the factor tensors into the context (asynchronous, on its
    stream); returns the FP32 contiguous tensors, which must stay alive
    until the copies have run."""
    staged = []
    for k, a in enumerate(factors):
        t = a.detach()
        if t.dtype != torch.float32 or not t.is_contiguous():
            t = t.to(torch.float32).contiguous()
        if tuple(t.shape) != (ctx.dims[k], ctx.rank):
            raise ValueError(f"factor {k} has shape {tuple(t.shape)}, expected {(ctx.dims[k], ctx.rank)}")
        _check(load().gcp_set_factor(ctx.handle, k, _ptr(t)), ctx.handle)
        staged.append(t)
    return staged


class GcpSampledLoss(torch.autograd.Function):
    """loss = GcpSampledLoss.apply(ctx, iteration, p, q, A_0, ..., A_{d-1})

    ctx is a GcpContext (sparse: p nonzero and q zero samples; dense: p
    uniform cells and q = 0).  The factors are CUDA tensors I_k x R; the
    loss is a 0-dim float64 tensor."""

    @staticmethod
    def forward(fctx, ctx: GcpContext, iteration: int, p: int, q: int, *factors):
        staged = _stage_factors(ctx, factors)
        loss = torch.empty(1, dtype=torch.float64, device=factors[0].device)
        ctx.loss_async(iteration, p, q, loss)
        fctx.gcp = ctx
        fctx.args = (iteration, p, q)
        fctx.staged = staged
        fctx.save_for_backward(*factors)
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        ctx: GcpContext = fctx.gcp
        iteration, p, q = fctx.args
        factors = fctx.saved_tensors
        staged = _stage_factors(ctx, factors)  # the context may have served other calls since
        scale = grad_out.detach().to(torch.float32).reshape(1).contiguous()
        G = torch.empty(ctx.num_params, dtype=torch.float32, device=factors[0].device)
        ctx.grad_async(iteration, p, q, dscale=scale, G_out=G)
        grads, o = [], 0
        for I in ctx.dims:
            grads.append(G[o:o + I * ctx.rank].view(I, ctx.rank))
            o += I * ctx.rank
        fctx.staged = staged + [scale]  # alive until the stream has consumed them
        return (None, None, None, None, *grads)


def sampled_loss(ctx: GcpContext, iteration: int, p: int, q: int, factors):
    return GcpSampledLoss.apply(ctx, iteration, p, q, *factors)
