"""The allocation-free entry point gcp_grad_samples_noalloc, called through
the C ABI, against the context-based gcp_grad on the same samples.

gcp_grad_samples_noalloc serves callers that cannot allocate device memory
(code under a device-memory budget fixed at start-up, e.g. a host framework
that owns every allocation through its own pool).  Its only scratch is a
file-scope device array shared by every call, so the test makes two calls in
a row with different sample counts: the second must not see the first's
partials.  This file is collected last so that a run stopping at the first
failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32 tolerance of the parity tests


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def env(gpu_lib):
    import torch

    return gpu_lib, torch


@pytest.mark.parametrize("loss", ["poisson", "gaussian"])
def test_noalloc_matches_gcp_grad_on_two_calls(env, loss):
    gcp, torch = env
    dims, R = [60, 45, 30, 7], 20
    coords, vals = synth.uniform_sparse(dims, 3000, 910, lam=2.0)
    factors = synth.factors_uniform(dims, R, 911, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, R, loss, seed=912)
    ctx.set_factors(factors)
    A = torch.from_numpy(np.concatenate([a.ravel() for a in factors])).cuda()
    lib = gcp.load()
    d = np.array(dims, dtype=np.int64)
    stream = torch.cuda.current_stream()
    for t, p, q in [(3, 2500, 2300), (4, 700, 611)]:  # second call: fewer blocks than the first
        idx, x, w = ctx.sample(t, p, q)
        G_ref = torch.zeros(ctx.num_params, device="cuda")
        L_ref, _ = ctx.grad(t, p, q, G_out=G_ref)
        G = torch.full((ctx.num_params,), float("nan"), device="cuda")  # must be overwritten
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.gcp_grad_samples_noalloc(len(dims), d.ctypes.data, R, gcp.LOSSES[loss], p + q, idx.data_ptr(),
                                          x.data_ptr(), w.data_ptr(), A.data_ptr(), G.data_ptr(), out.data_ptr(),
                                          ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.gcp_last_error(None)
        torch.cuda.synchronize()
        L, skipped = out.cpu().numpy()
        assert skipped == 0
        assert abs(L - L_ref) <= TOL * abs(L_ref), (t, L, L_ref)
        assert rel_err(G.cpu().numpy(), G_ref.cpu().numpy()) <= TOL, t
    ctx.close()


def test_noalloc_rejects_more_samples_than_its_scratch_holds(env):
    gcp, torch = env
    lib = gcp.load()
    d = np.array([4, 3, 2], dtype=np.int64)
    rc = lib.gcp_grad_samples_noalloc(3, d.ctypes.data, 2, 1, (1 << 24) + 1, 1, 1, 1, 1, 1, 1, None)
    assert rc == 1
    assert b"GCP_NOALLOC_MAX_SAMPLES" in lib.gcp_last_error(None)


@pytest.mark.parametrize("loss", ["gaussian", "poisson", "bernoulli", "gamma"])
def test_noalloc_skips_out_of_range_samples(env, loss):
    """Samples with a coordinate outside its mode (negative or past the end)
    are skipped and counted in loss_out[1]; the loss and gradient are those
    of the in-range samples, against the FP64 oracle on that subset, for
    every loss."""
    import oracle

    gcp, torch = env
    dims, R = [50, 40, 30], 12
    coords, vals = synth.uniform_sparse(dims, 2500, 920, lam=2.0)
    if loss == "bernoulli":
        vals = np.ones_like(vals)
    if loss in ("gaussian", "bernoulli"):
        factors = synth.factors_normal(dims, R, 921, std=0.6)
    else:
        factors = synth.factors_uniform(dims, R, 921, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, R, loss, seed=922)
    idx, x, w = ctx.sample(6, 1500, 1700)
    idx_h = idx.cpu().numpy().copy()
    rng = np.random.default_rng(923)
    bad = np.sort(rng.choice(idx_h.shape[0], 37, replace=False))
    for j, s in enumerate(bad):  # one coordinate off the end or negative, in varying modes
        k = j % 3
        idx_h[s, k] = dims[k] + j if j % 2 else -1 - j
    A = torch.from_numpy(np.concatenate([a.ravel() for a in factors])).cuda()
    G = torch.full((ctx.num_params,), float("nan"), device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    idx_d = torch.from_numpy(idx_h).cuda()
    lib = gcp.load()
    d = np.array(dims, dtype=np.int64)
    rc = lib.gcp_grad_samples_noalloc(3, d.ctypes.data, R, gcp.LOSSES[loss], idx_h.shape[0], idx_d.data_ptr(),
                                      x.data_ptr(), w.data_ptr(), A.data_ptr(), G.data_ptr(), out.data_ptr(),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.gcp_last_error(None)
    torch.cuda.synchronize()
    L, skipped = out.cpu().numpy()
    assert skipped == len(bad)
    keep = np.setdiff1d(np.arange(idx_h.shape[0]), bad)
    Lo, Go = oracle.sampled_loss_grad(dims, factors, loss, idx_h[keep], x.cpu().numpy()[keep].astype(np.float64),
                                      w.cpu().numpy()[keep].astype(np.float64))
    assert abs(L - Lo) <= TOL * abs(Lo), (L, Lo)
    assert rel_err(G.cpu().numpy(), np.concatenate([g.ravel() for g in Go])) <= TOL
    ctx.close()
