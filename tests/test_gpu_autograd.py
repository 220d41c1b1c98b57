"""The autograd function of the sampled GCP loss against the FP64 oracle:
forward = sampled loss and, when a factor needs a gradient, the fused MTTKRP
adjoint from the same pass; backward = that gradient scaled on the device
by the incoming gradient."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def env(gpu_lib):
    import torch

    from paper_2605_20353_gb300 import autograd

    return gpu_lib, torch, autograd


def check(env, ctx, factors_np, iteration, p, q, loss_name, oracle_samples, scale=1.0):
    gcp, torch, ag = env
    A = [torch.tensor(a, device="cuda", requires_grad=True) for a in factors_np]
    loss = ag.sampled_loss(ctx, iteration, p, q, A)
    (scale * loss).backward()
    idx, x, w = oracle_samples
    Lo, Go = oracle.sampled_loss_grad(ctx.dims, factors_np, loss_name, idx, x, w)
    assert loss.dtype == torch.float64 and loss.dim() == 0
    assert abs(loss.item() - Lo) <= TOL * abs(Lo)
    for n, (a, g) in enumerate(zip(A, Go)):
        assert rel_err(a.grad.cpu().numpy(), scale * g) <= TOL, n


@pytest.mark.parametrize("scale", [1.0, -3.0])
def test_autograd_dense_five_way(env, scale):
    gcp, torch, ag = env
    dims = [10, 9, 8, 4, 5]
    X = synth.dense_cp_sinusoid(dims, 31, rank_true=4)
    fac = synth.factors_normal(dims, 16, 32, std=0.6)
    ctx = gcp.gcp_create_dense(dims, X, 16, "gaussian", seed=33)
    check(env, ctx, fac, 4, 6000, 0, "gaussian", oracle.uniform_samples(33, 4, 6000, dims, X), scale=scale)
    ctx.close()


def test_autograd_sparse_poisson_and_second_call(env):
    gcp, torch, ag = env
    dims = [40, 30, 20]
    coords, vals = synth.uniform_sparse(dims, 1500, 41, lam=2.0)
    fac = synth.factors_uniform(dims, 8, 42, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=43)
    for it in (1, 2):  # the context is reused across graph evaluations
        idx, x, w, _ = oracle.stratified_samples(43, it, 900, 1100, dims, coords, vals)
        check(env, ctx, fac, it, 900, 1100, "poisson", (idx, x, w))
    ctx.close()


def test_autograd_dense_simulation_full_size(env):
    """100x100x100x20x50 dense FP32 tensor (1e9 cells): rank-8 sinusoidal CP
    signal + N(0, 0.1^2) noise, Gaussian loss, rank 16, 2^22 uniform samples;
    loss and all five gradients against the oracle."""
    gcp, torch, ag = env
    dims = [100, 100, 100, 20, 50]
    X = synth.dense_cp_sinusoid(dims, 1003, rank_true=8, sigma=0.1)
    fac = synth.factors_normal(dims, 16, 2003, std=0.5)
    ctx = gcp.gcp_create_dense(dims, X, 16, "gaussian", seed=3003)
    s = 1 << 22
    samples = oracle.uniform_samples(3003, 7, s, dims, X)
    check(env, ctx, fac, 7, s, 0, "gaussian", samples)
    ctx.close()


def test_autograd_loss_only_and_partial_grads(env):
    """Without factor gradients the forward computes the loss alone, with
    the same value; with only some factors requiring gradients, the others
    get none and the rest match the oracle."""
    gcp, torch, ag = env
    dims = [30, 20, 10]
    coords, vals = synth.uniform_sparse(dims, 900, 51, lam=2.0)
    fac = synth.factors_uniform(dims, 8, 52, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=53)
    with torch.no_grad():
        L0 = ag.sampled_loss(ctx, 3, 700, 800, [torch.tensor(a, device="cuda") for a in fac])
    A = [torch.tensor(a, device="cuda", requires_grad=(k != 1)) for k, a in enumerate(fac)]
    L1 = ag.sampled_loss(ctx, 3, 700, 800, A)
    assert L0.item() == L1.item()  # the loss reduction is fixed-order in both passes
    (2.5 * L1).backward()
    idx, x, w, _ = oracle.stratified_samples(53, 3, 700, 800, dims, coords, vals)
    _, Go = oracle.sampled_loss_grad(dims, fac, "poisson", idx, x, w)
    assert A[1].grad is None
    for k in (0, 2):
        assert rel_err(A[k].grad.cpu().numpy(), 2.5 * Go[k]) <= TOL, k
    ctx.close()


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)


def test_autograd_bf16_padded_rank_and_fp64_noncontiguous_factors(env):
    """BF16 factor storage with rank 6 (rows padded to 8 columns): the
    factors are staged in one call into the padded layout and their BF16
    copy refreshed once; FP64 and transposed (non-contiguous) factor tensors
    are converted first.  Loss and gradients match the oracle run on the
    BF16-rounded factors."""
    gcp, torch, ag = env
    dims = [35, 25, 15]
    coords, vals = synth.uniform_sparse(dims, 1200, 61, lam=2.0)
    fac = synth.factors_uniform(dims, 6, 62, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, 6, "poisson", dtype="bf16", seed=63)
    A = [torch.tensor(fac[0], device="cuda", dtype=torch.float64, requires_grad=True),
         torch.tensor(fac[1].T.copy(), device="cuda").t().detach().requires_grad_(True),  # non-contiguous view
         torch.tensor(fac[2], device="cuda", requires_grad=True)]
    assert not A[1].is_contiguous()
    loss = ag.sampled_loss(ctx, 2, 800, 900, A)
    loss.backward()
    idx, x, w, _ = oracle.stratified_samples(63, 2, 800, 900, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, [bf16_round(a) for a in fac], "poisson", idx, x, w)
    assert abs(loss.item() - Lo) <= TOL * abs(Lo)
    for k in range(3):
        assert A[k].grad.shape == (dims[k], 6)
        assert rel_err(A[k].grad.double().cpu().numpy(), Go[k]) <= TOL, k
    ctx.close()


@pytest.mark.parametrize("scale", [1.0, -3.0])
def test_autograd_adjoint_in_backward(env, scale):
    """grad_in_forward=False: the forward computes the loss alone and the
    backward runs the fused MTTKRP adjoint over the same samples, seeded with
    the incoming gradient; loss and gradients match the oracle, also when
    the context's factors were changed between forward and backward."""
    gcp, torch, ag = env
    dims = [40, 30, 20]
    coords, vals = synth.uniform_sparse(dims, 1500, 71, lam=2.0)
    fac = synth.factors_uniform(dims, 8, 72, lo=0.1, hi=1.0)
    other = synth.factors_uniform(dims, 8, 73, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=74)
    A = [torch.tensor(a, device="cuda", requires_grad=True) for a in fac]
    loss = ag.sampled_loss(ctx, 5, 900, 1100, A, grad_in_forward=False)
    ctx.set_factors(other)  # the backward must use the forward's factors
    (scale * loss).backward()
    idx, x, w, _ = oracle.stratified_samples(74, 5, 900, 1100, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, fac, "poisson", idx, x, w)
    assert abs(loss.item() - Lo) <= TOL * abs(Lo)
    for n, (a, g) in enumerate(zip(A, Go)):
        assert rel_err(a.grad.cpu().numpy(), scale * g) <= TOL, n
    ctx.close()


def test_stage_and_gradient_call_matches_separate_calls_and_rejects_host_memory(env):
    """gcp_grad_factors_async (stage every factor matrix with one kernel, then
    the fused pass) gives the loss and gradient of gcp_set_factor_list +
    gcp_grad_async bit for bit, pads the rank with zeros, and rejects factor
    matrices in host memory with GCP_ERR_ARG."""
    import ctypes

    gcp, torch, _ = env
    dims, R = [30, 20, 10], 6  # rows padded to 8 columns
    coords, vals = synth.uniform_sparse(dims, 500, 4401, lam=2.0)
    fac = [torch.tensor(a, device="cuda") for a in synth.factors_uniform(dims, R, 4402, lo=0.1, hi=1.0)]
    lib = gcp.load()
    a = gcp.gcp_create(dims, coords, vals, R, "poisson", seed=4403)
    b = gcp.gcp_create(dims, coords, vals, R, "poisson", seed=4403)
    b.set_factors([f.cpu().numpy() for f in fac])
    ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in fac])
    Ga = torch.zeros(a.num_params, device="cuda")
    La = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert lib.gcp_grad_factors_async(a.handle, ptrs, 7, 300, 301, Ga.data_ptr(), La.data_ptr()) == 0
    Gb = torch.zeros(b.num_params, device="cuda")
    Lb = torch.zeros(1, dtype=torch.float64, device="cuda")
    b.grad_async(7, 300, 301, G_out=Gb, dloss=Lb)
    a.sync()
    b.sync()
    assert torch.equal(La, Lb)  # fixed-order loss reduction
    assert torch.linalg.norm(Ga - Gb) <= 1e-6 * torch.linalg.norm(Gb)  # atomic summation order only
    for x, y in zip(a.get_factors(), fac):
        assert np.array_equal(x, y.cpu().numpy())
    host = [f.cpu() for f in fac]
    hptrs = (ctypes.c_void_p * 3)(*[h.data_ptr() for h in host])
    assert lib.gcp_grad_factors_async(a.handle, hptrs, 7, 300, 301, Ga.data_ptr(), La.data_ptr()) == 1
    assert b"device or managed" in lib.gcp_last_error(a.handle)
    a.sync()  # the context stays usable
    a.close()
    b.close()
