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


def _factor_ptrs(ctx: GcpContext, factors):
    """(pointer array, FP32 contiguous CUDA tensors) of the factor tensors;
    the tensors must stay alive until the stream has consumed them."""
    staged = []
    ptrs = (ctypes.c_void_p * len(factors))()
    for k, a in enumerate(factors):
        t = a.detach()
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            t = t.to(device="cuda", dtype=torch.float32).contiguous()
        if t.dim() != 2 or t.shape[0] != ctx.dims[k] or t.shape[1] != ctx.rank:
            raise ValueError(f"factor {k} has shape {tuple(t.shape)}, expected {(ctx.dims[k], ctx.rank)}")
        ptrs[k] = t.data_ptr()
        staged.append(t)
    return ptrs, staged


def _stage_and_run(ctx: GcpContext, factors, iteration, p, q, G, loss):
    """One C call: stage the factors into the context and run the fused pass
    (gradient into G when G is not None, loss into loss[0])."""
    ptrs, staged = _factor_ptrs(ctx, factors)
    _check(load().gcp_grad_factors_async(ctx.handle, ptrs, iteration, p, q, G.data_ptr() if G is not None else None,
                                         loss.data_ptr()), ctx.handle)
    return staged


def _grads_of(ctx: GcpContext, G, needs):
    grads, o = [], 0
    for k, I in enumerate(ctx.dims):
        grads.append(G[o:o + I * ctx.rank].view(I, ctx.rank) if needs[4 + k] else None)
        o += I * ctx.rank
    return grads


class GcpSampledLoss(torch.autograd.Function):
    """loss = GcpSampledLoss.apply(ctx, iteration, p, q, A_0, ..., A_{d-1})

    ctx is a GcpContext (sparse: p nonzero and q zero samples; dense: p
    uniform cells and q = 0).  The factors are CUDA tensors I_k x R; the
    loss is a 0-dim float64 tensor."""

    @staticmethod
    def forward(fctx, ctx: GcpContext, iteration: int, p: int, q: int, *factors):
        dev = factors[0].device
        loss = torch.empty(1, dtype=torch.float64, device=dev)
        fctx.gcp = ctx
        fctx.G = None
        if any(fctx.needs_input_grad[4:]):
            fctx.G = torch.empty(ctx.num_params, dtype=torch.float32, device=dev)
        fctx.staged = _stage_and_run(ctx, factors, iteration, p, q, fctx.G, loss)  # alive until consumed
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        ctx: GcpContext = fctx.gcp
        scale = grad_out.detach()
        if scale.dtype != torch.float64:
            scale = scale.to(torch.float64)
        scale = scale.reshape(1).contiguous()  # a view for the usual FP64 seed
        G = torch.empty_like(fctx.G)
        _check(load().gcp_scale_async(ctx.handle, scale.data_ptr(), fctx.G.data_ptr(), G.data_ptr(), G.numel()),
               ctx.handle)
        fctx.staged = fctx.staged + [scale, fctx.G]  # alive until the stream has consumed them
        return (None, None, None, None, *_grads_of(ctx, G, fctx.needs_input_grad))


class GcpSampledLossAdjoint(torch.autograd.Function):
    """Same loss, other split of the work: the forward computes the sampled
    loss alone; the backward runs the fused MTTKRP adjoint kernel once more
    over the same sample set (same iteration, so the same samples), seeded
    with the incoming gradient, recomputing the Khatri-Rao rows.  It costs a
    second sampling pass, and suits graphs whose backward may not run."""

    @staticmethod
    def forward(fctx, ctx: GcpContext, iteration: int, p: int, q: int, *factors):
        loss = torch.empty(1, dtype=torch.float64, device=factors[0].device)
        staged = _stage_and_run(ctx, factors, iteration, p, q, None, loss)
        fctx.gcp, fctx.args, fctx.staged = ctx, (iteration, p, q), staged
        fctx.save_for_backward(*[f.detach() for f in factors])
        return loss.reshape(())

    @staticmethod
    def backward(fctx, grad_out):
        ctx: GcpContext = fctx.gcp
        factors = fctx.saved_tensors
        ptrs, staged = _factor_ptrs(ctx, factors)  # the factors as of the forward pass
        _check(load().gcp_set_factor_list(ctx.handle, ptrs), ctx.handle)
        seed = grad_out.detach().to(torch.float32).reshape(1).contiguous()
        G = torch.empty(ctx.num_params, dtype=torch.float32, device=seed.device)
        ctx.grad_async(*fctx.args, dscale=seed, G_out=G)
        fctx.staged = fctx.staged + staged + [seed]  # alive until the stream has consumed them
        return (None, None, None, None, *_grads_of(ctx, G, fctx.needs_input_grad))


def sampled_loss(ctx: GcpContext, iteration: int, p: int, q: int, factors, grad_in_forward: bool = True):
    """The sampled GCP loss of iteration `iteration` as a differentiable
    0-dim FP64 tensor.  grad_in_forward=True (default) forms the gradient in
    the forward's fused pass and only scales it in the backward; False runs
    the MTTKRP adjoint in the backward instead (GcpSampledLossAdjoint)."""
    fn = GcpSampledLoss if grad_in_forward else GcpSampledLossAdjoint
    return fn.apply(ctx, iteration, p, q, *factors)
