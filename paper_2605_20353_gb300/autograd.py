"""torch.autograd binding of the sampled GCP loss.

Forward: the sampled loss F~ = sum_s w_s f(x_s, m_s) of one sample set
(Sec. 3.1.1 weights, Eq. gcp-model), reduced in FP64 by the fused kernel.
When a factor needs a gradient, the same fused pass also forms the sampled
gradient (Eq. gcp-gradient) with a unit seed, so each sample is drawn and
its Khatri-Rao rows gathered once; nothing per sample is stored, only the
gradient itself (sum_k I_k R floats).  Backward multiplies that gradient by
the incoming one on the device.  Without factor gradients the forward pass
computes the loss alone.  The other split, GcpSampledLossAdjoint
(grad_in_forward=False), computes the loss alone in the forward and runs the
fused MTTKRP adjoint kernel in the backward, seeded with the incoming
gradient.  All arithmetic runs in libgcp.so; this module only moves
pointers.
"""
from __future__ import annotations

import ctypes

import torch

from . import GcpContext, _check, load


def _stage_factors(ctx: GcpContext, factors):
    """Copy the factor tensors into the context in one call (asynchronous,
    on its stream); returns the FP32 contiguous tensors, which must stay
    alive until the copies have run."""
    staged = []
    ptrs = (ctypes.c_void_p * len(factors))()
    for k, a in enumerate(factors):
        t = a.detach()
        if t.dtype != torch.float32 or not t.is_contiguous():
            t = t.to(torch.float32).contiguous()
        if t.shape[0] != ctx.dims[k] or t.shape[1] != ctx.rank or t.dim() != 2:
            raise ValueError(f"factor {k} has shape {tuple(t.shape)}, expected {(ctx.dims[k], ctx.rank)}")
        ptrs[k] = t.data_ptr()
        staged.append(t)
    _check(load().gcp_set_factor_list(ctx.handle, ptrs), ctx.handle)
    return staged


class GcpSampledLoss(torch.autograd.Function):
    """loss = GcpSampledLoss.apply(ctx, iteration, p, q, A_0, ..., A_{d-1})

    ctx is a GcpContext (sparse: p nonzero and q zero samples; dense: p
    uniform cells and q = 0).  The factors are CUDA tensors I_k x R; the
    loss is a 0-dim float64 tensor."""

    @staticmethod
    def forward(fctx, ctx: GcpContext, iteration: int, p: int, q: int, *factors):
        staged = _stage_factors(ctx, factors)
        dev = factors[0].device
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        fctx.gcp = ctx
        fctx.G = None
        if any(fctx.needs_input_grad[4:]):
            fctx.G = torch.empty(ctx.num_params, dtype=torch.float32, device=dev)
            ctx.grad_async(iteration, p, q, G_out=fctx.G, dloss=loss)
        else:
            ctx.loss_async(iteration, p, q, loss)
        fctx.staged = staged  # alive until the stream has consumed them
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        ctx: GcpContext = fctx.gcp
        scale = grad_out.detach().to(torch.float64).reshape(1).contiguous()  # no copy for an FP64 seed
        G = torch.empty_like(fctx.G)
        ctx.scale_async(scale, fctx.G, G)
        grads, o = [], 0
        for k, I in enumerate(ctx.dims):
            g = G[o:o + I * ctx.rank].view(I, ctx.rank)
            grads.append(g if fctx.needs_input_grad[4 + k] else None)
            o += I * ctx.rank
        fctx.staged = fctx.staged + [scale, fctx.G]  # alive until the stream has consumed them
        return (None, None, None, None, *grads)


class GcpSampledLossAdjoint(torch.autograd.Function):
    """Same loss, other split of the work: the forward computes the sampled
    loss alone; the backward runs the fused MTTKRP adjoint kernel once more
    over the same sample set (same iteration, so the same samples), seeded
    with the incoming gradient, recomputing the Khatri-Rao rows.  It costs a
    second sampling pass, and suits graphs whose backward may not run."""

    @staticmethod
    def forward(fctx, ctx: GcpContext, iteration: int, p: int, q: int, *factors):
        staged = _stage_factors(ctx, factors)
        loss = torch.empty(1, dtype=torch.float64, device=factors[0].device)
        ctx.loss_async(iteration, p, q, loss)
        fctx.gcp, fctx.args, fctx.staged = ctx, (iteration, p, q), staged
        fctx.save_for_backward(*[f.detach() for f in factors])
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        ctx: GcpContext = fctx.gcp
        factors = fctx.saved_tensors
        staged = _stage_factors(ctx, factors)  # the factors as of the forward pass
        seed = grad_out.detach().to(torch.float32).reshape(1).contiguous()
        G = torch.empty(ctx.num_params, dtype=torch.float32, device=seed.device)
        ctx.grad_async(*fctx.args, dscale=seed, G_out=G)
        grads, o = [], 0
        for k, I in enumerate(ctx.dims):
            g = G[o:o + I * ctx.rank].view(I, ctx.rank)
            grads.append(g if fctx.needs_input_grad[4 + k] else None)
            o += I * ctx.rank
        fctx.staged = fctx.staged + staged + [seed]  # alive until the stream has consumed them
        return (None, None, None, None, *grads)


def sampled_loss(ctx: GcpContext, iteration: int, p: int, q: int, factors, grad_in_forward: bool = True):
    """The sampled GCP loss of iteration `iteration` as a differentiable
    0-dim FP64 tensor.  grad_in_forward=True (default) forms the gradient in
    the forward's fused pass and only scales it in the backward; False runs
    the MTTKRP adjoint in the backward instead (GcpSampledLossAdjoint)."""
    fn = GcpSampledLoss if grad_in_forward else GcpSampledLossAdjoint
    return fn.apply(ctx, iteration, p, q, *factors)
