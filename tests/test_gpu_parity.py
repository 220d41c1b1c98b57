"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sampled indices must match bit for bit; the sampled loss and every mode's
gradient must match within relative Frobenius error 1e-5 with FP32 factors
and 5e-3 with BF16 factors.  Sizes span many 32-sample tiles with ragged
tails; edge cases cover empty sample sets, exhausted zero draws, duplicates
and every supported order and rank class.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16 = 5e-3


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def split(flat, dims, R):
    out, o = [], 0
    for I in dims:
        out.append(flat[o:o + I * R].reshape(I, R))
        o += I * R
    return out


def bf16_round(a):
    """Round-to-nearest-even of FP32 values to BF16, widened back to FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def problem(dims, nnz, R, loss, seed):
    coords, vals = synth.uniform_sparse(dims, nnz, seed, lam=2.0)
    if loss == "bernoulli":
        vals = np.ones_like(vals)
    if loss in ("gaussian", "bernoulli"):
        factors = synth.factors_normal(dims, R, seed + 1, std=0.6)
    else:
        factors = synth.factors_uniform(dims, R, seed + 1, lo=0.1, hi=1.0)
    return coords, vals, factors


def gpu_grad(gcp, torch, ctx, t, p, q):
    G = torch.zeros(ctx.num_params, dtype=torch.float32, device="cuda")
    loss, _ = ctx.grad(t, p, q, G_out=G)
    return loss, G.cpu().numpy()


def check_grad(gcp, torch, dims, coords, vals, R, loss, factors, p, q, t=0, seed=77, dtype="fp32", tol=TOL_FP32,
               sampling="stratified"):
    ctx = gcp.gcp_create(dims, coords, vals, R, loss, dtype=dtype, seed=seed, sampling=sampling)
    ctx.set_factors(factors)
    Lg, Gg = gpu_grad(gcp, torch, ctx, t, p, q)
    fac = [bf16_round(a) for a in factors] if dtype == "bf16" else factors
    if sampling == "semi":
        idx, x, w, semi = oracle.semi_stratified_samples(seed, t, p, q, dims, coords, vals)
    else:
        idx, x, w, _ = oracle.stratified_samples(seed, t, p, q, dims, coords, vals)
        semi = None
    Lo, Go = oracle.sampled_loss_grad(dims, fac, loss, idx, x, w, semi=semi)
    assert abs(Lg - Lo) <= tol * abs(Lo), (Lg, Lo)
    for n, (a, b) in enumerate(zip(split(Gg, dims, R), Go)):
        assert rel_err(a, b) <= tol, (n, rel_err(a, b))
    ctx.close()
    return Lg, Gg


@pytest.fixture(scope="module")
def env(gpu_lib):
    import torch

    return gpu_lib, torch


# ------------------------------------------------------------- sampling
@pytest.mark.parametrize("t", [0, 1, 7, 2**64 - 1])
def test_sample_bit_exact_small(env, t):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=3001)
    idx, x, wt = ctx.sample(t, 1000, 1000)
    ido, xo, wo, _ = oracle.stratified_samples(3001, t, 1000, 1000, w["dims"], w["coords"], w["vals"])
    assert np.array_equal(idx.cpu().numpy(), ido)
    assert np.array_equal(x.cpu().numpy(), xo.astype(np.float32))
    assert np.array_equal(wt.cpu().numpy(), wo.astype(np.float32))
    ctx.close()


def test_sample_bit_exact_over_2_24_counters(env):
    """2^23 nonzero + 2^23 zero draws (with about 2.9e5 rejected zero
    candidates redrawn) on the 50x40x30 tensor: every index equals the
    oracle's, so the device Philox and range map agree with the host's over
    2^24 counters."""
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=0x5EED)
    p = q = 1 << 23
    idx, _, _ = ctx.sample(12345, p, q)
    ido, _, _, att = oracle.stratified_samples(0x5EED, 12345, p, q, w["dims"], w["coords"], w["vals"])
    assert att > q  # some zero candidates were nonzeros and were redrawn
    assert np.array_equal(idx.cpu().numpy(), ido)
    ctx.close()


def test_sample_bit_exact_zipf_4way(env):
    gcp, torch = env
    w = synth.workload_zipf_count(scale=0.01)
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 32, "poisson", seed=3002)
    p, q = w["p"] + 13, w["q"] + 5  # ragged tail
    idx, x, _ = ctx.sample(3, p, q)
    ido, xo, _, _ = oracle.stratified_samples(3002, 3, p, q, w["dims"], w["coords"], w["vals"])
    assert np.array_equal(idx.cpu().numpy(), ido)
    assert np.array_equal(x.cpu().numpy(), xo.astype(np.float32))
    ctx.close()


@pytest.mark.parametrize("d", [2, 5, 8])
def test_sample_bit_exact_orders(env, d):
    gcp, torch = env
    dims = [7, 5, 9, 3, 4, 6, 2, 5][:d]
    coords, vals, _ = problem(dims, min(300, int(np.prod(dims)) // 3), 4, "poisson", 90 + d)
    ctx = gcp.gcp_create(dims, coords, vals, 4, "poisson", seed=11)
    idx, x, _ = ctx.sample(2, 555, 999)
    ido, xo, _, _ = oracle.stratified_samples(11, 2, 555, 999, dims, coords, vals)
    assert np.array_equal(idx.cpu().numpy(), ido)
    ctx.close()


def test_sample_semi_and_dense_bit_exact(env):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=5, sampling="semi")
    idx, x, wt = ctx.sample(4, 300, 700)
    ido, xo, wo, _ = oracle.semi_stratified_samples(5, 4, 300, 700, w["dims"], w["coords"], w["vals"])
    assert np.array_equal(idx.cpu().numpy(), ido)
    assert np.array_equal(wt.cpu().numpy(), wo.astype(np.float32))
    ctx.close()
    dims = [6, 5, 4, 3, 7]
    X = synth.dense_cp_sinusoid(dims, 4, rank_true=3)
    ctx = gcp.gcp_create_dense(dims, X, 8, "gaussian", seed=9)
    idx, x, wt = ctx.sample(1, 2049, 0)
    ido, xo, wo = oracle.uniform_samples(9, 1, 2049, dims, X)
    assert np.array_equal(idx.cpu().numpy(), ido)
    assert np.array_equal(x.cpu().numpy(), xo.astype(np.float32))
    ctx.close()


# --------------------------------------------------------- loss + grad
@pytest.mark.parametrize("loss", ["gaussian", "poisson", "bernoulli", "gamma"])
def test_grad_fp32_all_losses(env, loss):
    gcp, torch = env
    dims = [50, 40, 30]
    coords, vals, factors = problem(dims, 2000, 16, loss, 200)
    check_grad(gcp, torch, dims, coords, vals, 16, loss, factors, 1234, 777, t=3)


@pytest.mark.parametrize("d,R", [(2, 1), (3, 3), (4, 32), (5, 16), (6, 8), (8, 5), (3, 64), (3, 128), (4, 33)])
def test_grad_orders_and_ranks(env, d, R):
    gcp, torch = env
    dims = [23, 17, 11, 7, 5, 6, 4, 3][:d]
    coords, vals, factors = problem(dims, min(900, int(np.prod(dims)) // 4), R, "poisson", 300 + d * 7 + R)
    check_grad(gcp, torch, dims, coords, vals, R, "poisson", factors, 1500, 1001, t=1)


@pytest.mark.parametrize("loss", ["poisson", "bernoulli"])
def test_grad_bf16(env, loss):
    gcp, torch = env
    dims = [60, 50, 40]
    coords, vals, factors = problem(dims, 3000, 64, loss, 400)
    Lg, Gg = check_grad(gcp, torch, dims, coords, vals, 64, loss, factors, 2000, 2000, dtype="bf16", tol=1e-5)
    # against the FP32 factors: storage error, stated by the BF16 tolerance
    idx, x, w, _ = oracle.stratified_samples(77, 0, 2000, 2000, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, factors, loss, idx, x, w)
    assert abs(Lg - Lo) <= TOL_BF16 * abs(Lo)
    assert rel_err(Gg, np.concatenate([g.ravel() for g in Go])) <= TOL_BF16


def test_grad_semi_stratified(env):
    gcp, torch = env
    dims = [40, 30, 20]
    coords, vals, factors = problem(dims, 1500, 8, "poisson", 500)
    check_grad(gcp, torch, dims, coords, vals, 8, "poisson", factors, 999, 1501, sampling="semi")


def test_grad_dense_uniform(env):
    gcp, torch = env
    dims = [10, 9, 8, 4, 5]
    X = synth.dense_cp_sinusoid(dims, 21, rank_true=4)
    factors = synth.factors_normal(dims, 16, 22, std=0.5)
    ctx = gcp.gcp_create_dense(dims, X, 16, "gaussian", seed=4)
    ctx.set_factors(factors)
    Lg, Gg = gpu_grad(gcp, torch, ctx, 2, 5000, 0)
    idx, x, w = oracle.uniform_samples(4, 2, 5000, dims, X)
    Lo, Go = oracle.sampled_loss_grad(dims, factors, "gaussian", idx, x, w)
    assert abs(Lg - Lo) <= TOL_FP32 * abs(Lo)
    assert rel_err(Gg, np.concatenate([g.ravel() for g in Go])) <= TOL_FP32
    ctx.close()


def test_gradient_norm_in_fp64(env):
    """gcp_grad_norm: the FP64 Frobenius norm of the context's gradient
    equals the oracle gradient's norm, repeats bit for bit, and is zero once
    gcp_step has cleared the gradient."""
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=3001)
    ctx.set_factors(w["factors"])
    ctx.grad(2, w["p"], w["q"])
    n1, n2 = ctx.grad_norm(), ctx.grad_norm()
    idx, x, wt, _ = oracle.stratified_samples(3001, 2, w["p"], w["q"], w["dims"], w["coords"], w["vals"])
    _, Go = oracle.sampled_loss_grad(w["dims"], w["factors"], "gaussian", idx, x, wt)
    ref = float(np.linalg.norm(np.concatenate([g.ravel() for g in Go])))
    assert abs(n1 - ref) <= TOL_FP32 * ref, (n1, ref)
    assert n1 == n2
    ctx.step(3, w["p"], w["q"], gcp.AdamParams(lr=1e-3), 1)
    assert ctx.grad_norm() == 0.0
    # a NaN factor entry: the loss and the norm check both report it, and the
    # context stays usable once the factors are finite again
    bad = [a.copy() for a in w["factors"]]
    bad[0][0, 0] = np.nan
    ctx.set_factors(bad)
    with pytest.raises(gcp.GcpError):
        ctx.grad(4, w["p"], w["q"])
    with pytest.raises(gcp.GcpError):
        ctx.grad_norm()
    ctx.set_factors(w["factors"])
    ctx.grad(2, w["p"], w["q"])
    assert abs(ctx.grad_norm() - n1) <= TOL_FP32 * n1  # same samples; atomic order may differ
    ctx.close()


def test_loss_only_call_matches_grad_call(env):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=1)
    ctx.set_factors(w["factors"])
    L1 = ctx.loss_value(5, 800, 900)
    L2, _ = ctx.grad(5, 800, 900)
    assert L1 == L2  # same sample set, same fixed-order reduction
    ctx.close()


def test_grad_scale_and_async_loss(env):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=1)
    ctx.set_factors(w["factors"])
    G1 = torch.zeros(ctx.num_params, device="cuda")
    G2 = torch.zeros(ctx.num_params, device="cuda")
    dl = torch.zeros(1, dtype=torch.float64, device="cuda")
    L, _ = ctx.grad(2, 500, 500, G_out=G1)
    ctx.grad_async(2, 500, 500, dscale=torch.tensor([-2.5], device="cuda"), G_out=G2, dloss=dl)
    ctx.sync()
    assert dl.item() == L
    # atomic summation order differs between the two calls
    assert rel_err(G2.cpu().numpy(), -2.5 * G1.cpu().numpy()) <= 1e-6
    ctx.close()


# ---------------------------------------------------------------- Adam
def test_adam_step_parity(env):
    gcp, torch = env
    dims = [30, 20, 10]
    coords, vals, factors = problem(dims, 800, 8, "poisson", 600)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=3)
    ctx.set_factors(factors)
    A = oracle.flat_factors(factors)
    B, C = np.zeros_like(A), np.zeros_like(A)
    prm = gcp.AdamParams(lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)
    for t in range(1, 4):
        ctx.grad(t, 500, 500, want_loss=False)
        ctx.adam_step(prm, t)
        idx, x, w, _ = oracle.stratified_samples(3, t, 500, 500, dims, coords, vals)
        _, Go = oracle.sampled_loss_grad(dims, split(A, dims, 8), "poisson", idx, x, w)
        oracle.adam_step(A, B, C, np.concatenate([g.ravel() for g in Go]), 0.01, 0.9, 0.999, 1e-8, 0.0, t)
        Ag = np.concatenate([a.ravel() for a in ctx.get_factors()])
        assert rel_err(Ag, A) <= 1e-5, (t, rel_err(Ag, A))
        A = Ag.astype(np.float64)  # continue both from the GPU state
    ctx.close()


def test_fit_reduces_objective(env):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=8)
    ctx.set_factors(w["factors"])
    rep = ctx.fit(gcp.AdamParams(lr=1e-2), 1000, 1000, 5000, 5000, iters=100, max_epochs=20)
    assert rep["objective"] < 0.9 * rep["objective0"]
    assert rep["epochs"] >= 1 and rep["iterations"] >= 100
    assert 1.0 <= rep["attempts_per_zero"] < 1.2
    # the fit ends on the best accepted state: its objective estimate is
    # reproduced exactly, and the oracle agrees on those factors
    assert ctx.loss_value(gcp.GCP_ITER_OBJECTIVE, 5000, 5000) == rep["objective"]
    fac = ctx.get_factors()
    idx, x, wt, _ = oracle.stratified_samples(8, 2**64 - 1, 5000, 5000, w["dims"], w["coords"], w["vals"])
    Fo, _ = oracle.sampled_loss_grad(w["dims"], fac, "gaussian", idx, x, wt, grad=False)
    assert abs(rep["objective"] - Fo) <= TOL_FP32 * abs(Fo)
    assert rep["objective"] == min(rep["trace"] + [rep["objective0"]])
    ctx.close()


# ----------------------------------------------------------- edge cases
@pytest.mark.parametrize("mttkrp", ["atomic", "deterministic", "nonfused"])
def test_empty_sample_sets(env, mttkrp):
    gcp, torch = env
    w = synth.workload_small_gaussian()
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 4, "gaussian", seed=1, mttkrp=mttkrp)
    ctx.set_factors(w["factors"])
    L, G = gpu_grad(gcp, torch, ctx, 0, 0, 0)
    assert L == 0.0 and not np.any(G)
    L, G = gpu_grad(gcp, torch, ctx, 0, 37, 0)  # nonzeros only: one ragged tile
    idx, x, wt, _ = oracle.stratified_samples(1, 0, 37, 0, w["dims"], w["coords"], w["vals"])
    Lo, Go = oracle.sampled_loss_grad(w["dims"], w["factors"], "gaussian", idx, x, wt)
    assert abs(L - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(G, w["dims"], 4), Go)):
        assert rel_err(a, b) <= TOL_FP32, (n, rel_err(a, b))
    L, G = gpu_grad(gcp, torch, ctx, 0, 0, 0)  # and empty again after a non-empty call
    assert L == 0.0 and not np.any(G)
    ctx.close()


def test_exhausted_zero_draw_is_reported(env):
    gcp, torch = env
    dims = [3, 2, 2]
    coords = np.array(list(np.ndindex(*dims)), dtype=np.int32)
    ctx = gcp.gcp_create(dims, coords, np.ones(len(coords), np.float32), 2, "poisson", max_attempts=8)
    with pytest.raises(gcp.GcpError) as e:
        ctx.loss_value(0, 4, 4)
    assert e.value.status == "ERR_SAMPLER_EXHAUSTED"
    assert ctx.loss_value(0, 4, 0) == ctx.loss_value(0, 4, 0)  # context still usable
    ctx.close()


def test_half_dense_tensor_redraws(env):
    """Half of the cells are nonzeros, so about every other zero candidate
    is rejected and redrawn: bit-exact samples, and gradient parity through
    the fused pass's redraw path."""
    gcp, torch = env
    dims = [4, 5, 6]
    coords, vals, factors = problem(dims, 60, 8, "poisson", 910)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=13)
    idx, x, _ = ctx.sample(5, 3001, 2999)
    ido, xo, _, _ = oracle.stratified_samples(13, 5, 3001, 2999, dims, coords, vals)
    assert np.array_equal(idx.cpu().numpy(), ido)
    assert np.array_equal(x.cpu().numpy(), xo.astype(np.float32))
    ctx.close()
    check_grad(gcp, torch, dims, coords, vals, 8, "poisson", factors, 3001, 2999, t=5, seed=13)


@pytest.mark.parametrize("dims", [[1, 30, 20], [40, 1, 1, 9]])
def test_modes_of_size_one(env, dims):
    """Every sample falls in row 0 of a size-1 mode."""
    gcp, torch = env
    coords, vals, factors = problem(dims, int(np.prod(dims)) // 4, 4, "gaussian", 920 + len(dims))
    check_grad(gcp, torch, dims, coords, vals, 4, "gaussian", factors, 1000, 1003, t=2)


def test_largest_sample_count_per_call(env):
    """p + q = 2^31 - 1, the most one call accepts, on a problem whose
    sampled loss is known whatever is drawn: rank 1 with all factors 1 gives
    m = 1 in every cell, and all nonzeros are 1, so a nonzero costs 0, a zero
    costs (0 - 1)^2 = 1 and the loss is (M - N)/q * q = M - N.  Per-tile sums
    of ones are exact in FP32 and their total is exact in FP64, so the loss
    shows that every tile of the largest launch was taken exactly once."""
    gcp, torch = env
    dims = [50, 40, 30]
    M, N = 60000, 2000
    coords, _ = synth.uniform_sparse(dims, N, 930)
    ctx = gcp.gcp_create(dims, coords, np.ones(N, np.float32), 1, "gaussian", seed=17)
    ctx.set_factors([np.ones((I, 1), np.float32) for I in dims])
    p = 1 << 30
    q = (1 << 31) - 1 - p
    L, G = gpu_grad(gcp, torch, ctx, 0, p, q)
    assert L == pytest.approx(M - N, rel=1e-12)
    assert np.all(np.isfinite(G))
    # each zero adds w_z * f' = 2 (M - N) / q to one row per mode; a mode's
    # rows sum to 2 (M - N), up to FP32 rounding over ~2^30 additions
    for g in split(G, dims, 1):
        assert float(g.astype(np.float64).sum()) == pytest.approx(2 * (M - N), rel=0.05)
    ctx.close()


@pytest.mark.parametrize("loss,bad,status", [("gaussian", np.nan, "ERR_ARG"), ("gaussian", np.inf, "ERR_ARG"),
                                              ("poisson", -1.0, "ERR_DOMAIN"), ("bernoulli", 0.5, "ERR_DOMAIN")])
def test_dense_values_checked_at_creation(env, loss, bad, status):
    gcp, torch = env
    dims = [6, 5, 4]
    X = np.ones(int(np.prod(dims)), np.float32)
    X[77] = bad
    with pytest.raises(gcp.GcpError) as e:
        gcp.gcp_create_dense(dims, X, 4, loss)
    assert e.value.status == status
    X[77] = 0.0
    gcp.gcp_create_dense(dims, X, 4, loss).close()  # a valid tensor still builds


def test_duplicate_nonzeros_rejected(env):
    gcp, torch = env
    coords = np.array([[0, 1, 1], [2, 0, 1], [0, 1, 1]], dtype=np.int32)
    with pytest.raises(gcp.GcpError) as e:
        gcp.gcp_create([3, 2, 2], coords, np.ones(3, np.float32), 2, "poisson")
    assert e.value.status == "ERR_DUPLICATE"


# ------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def zipf_full():
    return synth.cached("zipf_count_full", lambda: synth.workload_zipf_count(scale=1.0))


@pytest.mark.parametrize("dtype,tol", [("fp32", TOL_FP32), ("bf16", 1e-5)])
def test_zipf_count_full_size(env, zipf_full, dtype, tol):
    """2000x1500x1000x200, 5e7 Zipf nonzeros, rank 32, Poisson, 2^20 + 2^20
    samples: every sampled index, the loss and all four gradients against
    the oracle, in the launch configuration the benchmark times."""
    gcp, torch = env
    w = zipf_full
    ctx = gcp.gcp_create(w["dims"], w["coords"], w["vals"], 32, "poisson", dtype=dtype, seed=3002)
    ctx.set_factors(w["factors"])
    skeys = oracle.sorted_keys(w["dims"], w["coords"])
    idx, x, wt, att = oracle.stratified_samples(3002, 5, w["p"], w["q"], w["dims"], w["coords"], w["vals"],
                                                skeys=skeys)
    gidx, gx, _ = ctx.sample(5, w["p"], w["q"])
    assert np.array_equal(gidx.cpu().numpy(), idx)
    assert np.array_equal(gx.cpu().numpy(), x.astype(np.float32))
    Lg, Gg = gpu_grad(gcp, torch, ctx, 5, w["p"], w["q"])
    fac = [bf16_round(a) for a in w["factors"]] if dtype == "bf16" else w["factors"]
    Lo, Go = oracle.sampled_loss_grad(w["dims"], fac, "poisson", idx, x, wt)
    assert abs(Lg - Lo) <= tol * abs(Lo), (Lg, Lo)
    for n, (a, b) in enumerate(zip(split(Gg, w["dims"], 32), Go)):
        assert rel_err(a, b) <= tol, (dtype, n, rel_err(a, b))
    if dtype == "bf16":
        Lf, Gf = oracle.sampled_loss_grad(w["dims"], w["factors"], "poisson", idx, x, wt)
        assert abs(Lg - Lf) <= TOL_BF16 * abs(Lf)
        assert rel_err(Gg, np.concatenate([g.ravel() for g in Gf])) <= TOL_BF16
    # the timed step (gcp_step: fused pass + epilogue with the replica fold)
    # consumes the same gradient
    g_max = max(np.abs(g).max() for g in Go)
    Gs = step_gradient(gcp, ctx, w["factors"], 5, w["p"], w["q"], g_max)
    for n, (a, b) in enumerate(zip(split(Gs, w["dims"], 32), Go)):
        assert rel_err(a, b) <= tol, (dtype, "step", n, rel_err(a, b))
    ctx.close()


# --------------------------------------------------- deterministic MTTKRP
@pytest.mark.parametrize("dims,R,loss,dtype,p,q", [
    ([2000, 1500, 1000, 200], 32, "poisson", "fp32", 20000, 20011),  # Zipf heads span many chunks
    ([60, 50, 40], 64, "bernoulli", "fp32", 3000, 2999),              # 8 columns per lane
    ([23, 17, 11, 7, 5], 16, "gamma", "bf16", 1500, 1001),
    ([5000, 3], 8, "gaussian", "fp32", 1 << 18, 1 << 18),             # rows of ~175k samples: 3 levels
    ([140000, 6, 5], 8, "gaussian", "fp32", (1 << 17) + 3, (1 << 17) - 1001),  # 18-bit rows: three sort passes
])
def test_deterministic_mttkrp_parity_and_bit_stability(env, dims, R, loss, dtype, p, q):
    gcp, torch = env
    if dims[0] == 2000:
        w = synth.workload_zipf_count(scale=0.01)
        coords, vals, factors = w["coords"], w["vals"], w["factors"]
    else:
        coords, vals, factors = problem(dims, min(3000, int(np.prod(dims)) // 3), R, loss, 700 + len(dims))
    det = gcp.gcp_create(dims, coords, vals, R, loss, dtype=dtype, seed=21, mttkrp="deterministic")
    det.set_factors(factors)
    L1, G1 = gpu_grad(gcp, torch, det, 6, p, q)
    L2, G2 = gpu_grad(gcp, torch, det, 6, p, q)
    assert L1 == L2 and np.array_equal(G1.view(np.uint32), G2.view(np.uint32))  # bit-identical
    fac = [bf16_round(a) for a in factors] if dtype == "bf16" else factors
    idx, x, wt, _ = oracle.stratified_samples(21, 6, p, q, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, fac, loss, idx, x, wt)
    assert abs(L1 - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(G1, dims, R), Go)):
        assert rel_err(a, b) <= TOL_FP32, (n, rel_err(a, b))
    atom = gcp.gcp_create(dims, coords, vals, R, loss, dtype=dtype, seed=21)
    atom.set_factors(factors)
    La, Ga = gpu_grad(gcp, torch, atom, 6, p, q)
    assert La == L1  # the loss reduction is fixed-order in both variants
    assert rel_err(G1, Ga) <= TOL_FP32
    det.close()
    atom.close()


def test_deterministic_mttkrp_semi_stratified_scaled_and_missing_samples(env):
    """The deterministic variant with semi-stratified samples (the
    f'(x,m) - f'(0,m) correction), a gradient scale from device memory, and
    a full tensor whose exhausted zero draws are reported and skipped:
    bit-stable, and equal to the oracle."""
    gcp, torch = env
    dims, R = [40, 30, 20], 16
    coords, vals, factors = problem(dims, 6000, R, "poisson", 771)
    det = gcp.gcp_create(dims, coords, vals, R, "poisson", seed=23, mttkrp="deterministic", sampling="semi")
    det.set_factors(factors)
    scale = torch.tensor([2.5], dtype=torch.float32, device="cuda")
    G = torch.zeros(det.num_params, dtype=torch.float32, device="cuda")
    dl = torch.zeros(1, dtype=torch.float64, device="cuda")
    det.grad_async(3, 2000, 2500, dscale=scale, G_out=G, dloss=dl)
    det.sync()
    G2 = torch.zeros_like(G)
    det.grad_async(3, 2000, 2500, dscale=scale, G_out=G2)
    det.sync()
    assert torch.equal(G, G2)
    idx, x, w, semi = oracle.semi_stratified_samples(23, 3, 2000, 2500, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, factors, "poisson", idx, x, w, semi=semi)
    assert abs(dl.item() - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(G.cpu().numpy(), dims, R), Go)):
        assert rel_err(a, 2.5 * b) <= TOL_FP32, (n, rel_err(a, 2.5 * b))
    det.close()
    # every cell a nonzero: each zero draw is exhausted, reported, and adds nothing
    dims = [3, 2, 2]
    coords = np.array(list(np.ndindex(*dims)), dtype=np.int32)
    full = gcp.gcp_create(dims, coords, np.ones(len(coords), np.float32), 2, "poisson", max_attempts=8,
                          mttkrp="deterministic")
    full.set_factors(synth.factors_uniform(dims, 2, 772, lo=0.1, hi=1.0))
    with pytest.raises(gcp.GcpError) as e:
        full.grad(0, 4, 4)
    assert e.value.status == "ERR_SAMPLER_EXHAUSTED"
    L, Gf = gpu_grad(gcp, torch, full, 0, 4, 0)  # still usable
    idx, x, w, _ = oracle.stratified_samples(0, 0, 4, 0, dims, coords, np.ones(len(coords), np.float32))
    Lo, Go = oracle.sampled_loss_grad(dims, synth.factors_uniform(dims, 2, 772, lo=0.1, hi=1.0), "poisson", idx, x, w)
    assert abs(L - Lo) <= TOL_FP32 * abs(Lo)
    full.close()


def test_deterministic_mttkrp_modes_sorted_in_two_groups(env):
    """An 8-way tensor with 8.4e6 samples: the sort buffers of all eight
    modes (16 B per sample and mode) pass 1 GiB, so the modes are sorted in
    a group of seven side by side and then one alone, with one-pass and
    two-pass modes and both digit widths in the group.  Bit-stable, and equal to
    the oracle."""
    gcp, torch = env
    dims, R = [2000, 600, 56, 52, 48, 44, 40, 36], 4  # 11-bit rows: two passes; 10-bit: one wide pass
    coords, vals, factors = problem(dims, 3000, R, "gaussian", 881)
    p = q = (1 << 22) + 5000
    assert 16 * (p + q) * 8 > 1 << 30 and 16 * (p + q) * 7 <= 1 << 30
    det = gcp.gcp_create(dims, coords, vals, R, "gaussian", seed=31, mttkrp="deterministic")
    det.set_factors(factors)
    L1, G1 = gpu_grad(gcp, torch, det, 2, p, q)
    L2, G2 = gpu_grad(gcp, torch, det, 2, p, q)
    assert L1 == L2 and np.array_equal(G1.view(np.uint32), G2.view(np.uint32))
    idx, x, wt, _ = oracle.stratified_samples(31, 2, p, q, dims, coords, vals)
    Lo, Go = oracle.sampled_loss_grad(dims, factors, "gaussian", idx, x, wt)
    assert abs(L1 - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(G1, dims, R), Go)):
        assert rel_err(a, b) <= TOL_FP32, (n, rel_err(a, b))
    det.close()


@pytest.fixture(scope="module")
def bernoulli_full():
    def make():
        dims = [10000, 10000, 1000]
        coords, vals = synth.bernoulli_logit_sparse(dims, 20_000_000, 1004, rank=16)
        return dict(dims=dims, coords=coords, vals=vals, factors=synth.factors_normal(dims, 64, 2004, std=0.5))
    return synth.cached("bernoulli_full", make)


@pytest.mark.parametrize("dtype,mttkrp", [("fp32", "atomic"), ("bf16", "atomic"), ("fp32", "deterministic")])
def test_bernoulli_binary_full_size(env, bernoulli_full, dtype, mttkrp):
    """10000x10000x1000 binary tensor with 2e7 ones from a rank-16 logistic
    generator, Bernoulli-logit loss, rank 64, 2^21 ones + 2^21 zeros (hash
    rejection); FP32 / BF16 factors, atomic / deterministic MTTKRP."""
    gcp, torch = env
    w = bernoulli_full
    dims, p = w["dims"], 1 << 21
    ctx = gcp.gcp_create(dims, w["coords"], w["vals"], 64, "bernoulli", dtype=dtype, mttkrp=mttkrp, seed=3004)
    ctx.set_factors(w["factors"])
    Lg, Gg = gpu_grad(gcp, torch, ctx, 2, p, p)
    if mttkrp == "deterministic":
        L2, G2 = gpu_grad(gcp, torch, ctx, 2, p, p)
        assert L2 == Lg and np.array_equal(G2.view(np.uint32), Gg.view(np.uint32))
    fac = [bf16_round(a) for a in w["factors"]] if dtype == "bf16" else w["factors"]
    idx, x, wt, _ = oracle.stratified_samples(3004, 2, p, p, dims, w["coords"], w["vals"])
    Lo, Go = oracle.sampled_loss_grad(dims, fac, "bernoulli", idx, x, wt)
    assert abs(Lg - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(Gg, dims, 64), Go)):
        assert rel_err(a, b) <= TOL_FP32, (n, rel_err(a, b))
    if dtype == "bf16":
        Lf, Gf = oracle.sampled_loss_grad(dims, w["factors"], "bernoulli", idx, x, wt)
        assert abs(Lg - Lf) <= TOL_BF16 * abs(Lf)
        assert rel_err(Gg, np.concatenate([g.ravel() for g in Gf])) <= TOL_BF16
    ctx.close()


# ------------------------------------------------------ non-fused MTTKRP
@pytest.mark.parametrize("sampling,dtype", [("stratified", "fp32"), ("semi", "fp32"), ("stratified", "bf16")])
def test_nonfused_mttkrp_matches_oracle_and_fused(env, sampling, dtype):
    """Sampling writes the gradient tensor and a separate MTTKRP reads it;
    the gradient equals the fused pass's (Sec. 3.1.2: fusion only removes
    memory traffic)."""
    gcp, torch = env
    w = synth.workload_zipf_count(scale=0.01)
    dims, p = w["dims"], 15000
    res = {}
    for mttkrp in ("nonfused", "atomic"):
        ctx = gcp.gcp_create(dims, w["coords"], w["vals"], 32, "poisson", dtype=dtype, mttkrp=mttkrp,
                             sampling=sampling, seed=31)
        ctx.set_factors(w["factors"])
        res[mttkrp] = gpu_grad(gcp, torch, ctx, 4, p, p + 7)
        ctx.close()
    fac = [bf16_round(a) for a in w["factors"]] if dtype == "bf16" else w["factors"]
    if sampling == "semi":
        idx, x, wt, semi = oracle.semi_stratified_samples(31, 4, p, p + 7, dims, w["coords"], w["vals"])
    else:
        idx, x, wt, _ = oracle.stratified_samples(31, 4, p, p + 7, dims, w["coords"], w["vals"])
        semi = None
    Lo, Go = oracle.sampled_loss_grad(dims, fac, "poisson", idx, x, wt, semi=semi)
    L, G = res["nonfused"]
    assert L == res["atomic"][0]  # same sampling pass, same fixed-order loss reduction
    assert abs(L - Lo) <= TOL_FP32 * abs(Lo)
    for n, (a, b) in enumerate(zip(split(G, dims, 32), Go)):
        assert rel_err(a, b) <= TOL_FP32, n
    assert rel_err(G, res["atomic"][1]) <= TOL_FP32


# ----------------------------------------------------------- fused step
@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_step_equals_grad_then_adam_and_oracle(env, dtype):
    """gcp_step (fused pass + one epilogue: loss, replica fold, Adam, G
    cleared) over several steps equals gcp_grad + gcp_adam_step, and the
    first step equals the oracle's gradient + Adam."""
    gcp, torch = env
    w = synth.workload_zipf_count(scale=0.01)
    dims, p = w["dims"], 9000
    adam = gcp.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)
    a = gcp.gcp_create(dims, w["coords"], w["vals"], 32, "poisson", dtype=dtype, seed=51)
    b = gcp.gcp_create(dims, w["coords"], w["vals"], 32, "poisson", dtype=dtype, seed=51)
    a.set_factors(w["factors"])
    b.set_factors(w["factors"])
    dl = torch.zeros(1, dtype=torch.float64, device="cuda")
    for t in range(1, 4):
        a.step(t, p, p, adam, t, dloss=dl)
        L, _ = b.grad(t, p, p)
        b.adam_step(adam, t)
        a.sync()
        if t == 1:  # identical factors: the same fused pass and loss reduction
            assert dl.item() == L
        else:  # the factors differ by the atomic summation order of earlier gradients
            assert dl.item() == pytest.approx(L, rel=1e-9)
        if t == 1:
            fac = [bf16_round(x) for x in w["factors"]] if dtype == "bf16" else w["factors"]
            idx, x, wt, _ = oracle.stratified_samples(51, 1, p, p, dims, w["coords"], w["vals"])
            _, Go = oracle.sampled_loss_grad(dims, fac, "poisson", idx, x, wt)
            A = oracle.flat_factors(w["factors"])
            oracle.adam_step(A, np.zeros_like(A), np.zeros_like(A), np.concatenate([g.ravel() for g in Go]),
                             1e-3, 0.9, 0.999, 1e-8, 0.0, 1)
            assert rel_err(np.concatenate([f.ravel() for f in a.get_factors()]), A) <= TOL_FP32
    fa = np.concatenate([f.ravel() for f in a.get_factors()])
    fb = np.concatenate([f.ravel() for f in b.get_factors()])
    assert rel_err(fa, fb) <= TOL_FP32
    a.close()
    b.close()


def step_gradient(gcp, ctx, factors, it, p, q, g_max):
    """The gradient that one gcp_step of iteration `it` folds and feeds to
    Adam, read back through a readout Adam step (tests/adam_readout.py)."""
    from adam_readout import flat, readout_params, recover_gradient

    prm = readout_params(gcp, g_max)
    ctx.set_factors(factors)
    ctx.reset_adam()
    ctx.step(it, p, q, prm, 1)
    ctx.sync()
    return recover_gradient(flat(factors), flat(ctx.get_factors()), prm)


@pytest.mark.parametrize("dtype,mttkrp", [("fp32", "atomic"), ("bf16", "atomic"), ("fp32", "deterministic"),
                                          ("fp32", "nonfused")])
def test_step_folded_gradient_matches_oracle(env, dtype, mttkrp):
    """The gradient inside gcp_step (fused pass, then the epilogue's replica
    fold; for the deterministic and non-fused variants their own gradient,
    then Adam) element by element against the oracle's sampled gradient (Eq.
    gcp-gradient), per mode, at 1e-5.  The Zipf tensor's 200-row mode is
    fully replicated, its other modes have replicated head rows carried in
    the nonzero records, and drawn zero cells reach unreplicated rows."""
    gcp, torch = env
    w = synth.workload_zipf_count(scale=0.01)
    dims, p, q, R = w["dims"], 9000, 9001, 32
    ctx = gcp.gcp_create(dims, w["coords"], w["vals"], R, "poisson", dtype=dtype, seed=53, mttkrp=mttkrp)
    fac = [bf16_round(x) for x in w["factors"]] if dtype == "bf16" else w["factors"]
    idx, x, wt, _ = oracle.stratified_samples(53, 2, p, q, dims, w["coords"], w["vals"])
    _, Go = oracle.sampled_loss_grad(dims, fac, "poisson", idx, x, wt)
    g_max = max(np.abs(g).max() for g in Go)
    G = step_gradient(gcp, ctx, w["factors"], 2, p, q, g_max)
    for n, (a, b) in enumerate(zip(split(G, dims, R), Go)):
        assert rel_err(a, b) <= TOL_FP32, (dtype, mttkrp, n, rel_err(a, b))
    ctx.close()


def test_fit_with_tuned_preset_on_count_data(env):
    """gcp_fit with the paper's tuned GCP-SGD hyperparameters on a Poisson
    count tensor: the objective estimate falls, at most max_fails epochs
    fail, and the reported objective is the best epoch's."""
    gcp, torch = env
    dims = [60, 50, 40]
    coords, vals = synth.uniform_sparse(dims, 6000, 81, lam=3.0)
    ctx = gcp.gcp_create(dims, coords, vals, 8, "poisson", seed=82)
    ctx.set_factors(synth.factors_uniform(dims, 8, 83, lo=0.1, hi=1.0))
    pre = gcp.FIT_PRESETS["gcp_sgd_tuned"]
    rep = ctx.fit(pre["adam"], 2000, 2000, 20000, 20000, iters=50, max_epochs=30, max_fails=3, decay=pre["decay"])
    assert rep["objective"] < rep["objective0"]
    assert rep["fails"] <= 3 and rep["epochs"] <= 30
    assert rep["objective"] == min(rep["trace"] + [rep["objective0"]])
    assert min(f for a in ctx.get_factors() for f in a.ravel()) >= 0.0  # lower bound 0
    ctx.close()


def test_small_gaussian_hundred_epochs_gradient_parity_along_the_fit(env):
    """50x40x30 Gaussian workload, Adam lr 1e-2 for 100 epochs of 100 steps:
    the trajectory is chaotic across precisions, so parity is checked per
    state -- the GPU gradient at the GPU's own factors after 0, 50 and 99
    epochs against the oracle's gradient at those factors."""
    gcp, torch = env
    w = synth.workload_small_gaussian()
    dims = w["dims"]
    ctx = gcp.gcp_create(dims, w["coords"], w["vals"], 4, "gaussian", seed=3001)
    ctx.set_factors(w["factors"])
    adam = gcp.AdamParams(lr=1e-2)
    F_start = None
    for epochs in (0, 50, 49):
        if epochs:
            rep = ctx.fit(adam, 1000, 1000, 10000, 10000, iters=100, max_epochs=epochs, max_fails=100, decay=0.5,
                          iter0=10_000 * (epochs + 1))
            F_start = F_start or rep["objective0"]
        fac = ctx.get_factors()
        L, G = gpu_grad(gcp, torch, ctx, 77, 1000, 1000)
        idx, x, wt, _ = oracle.stratified_samples(3001, 77, 1000, 1000, dims, w["coords"], w["vals"])
        Lo, Go = oracle.sampled_loss_grad(dims, fac, "gaussian", idx, x, wt)
        assert abs(L - Lo) <= TOL_FP32 * abs(Lo)
        for n, (a, b) in enumerate(zip(split(G, dims, 4), Go)):
            assert rel_err(a, b) <= TOL_FP32, (epochs, n)
    assert rep["objective"] < F_start
    ctx.close()


def test_fit_restores_state_after_failed_epochs(env):
    """An epoch that does not lower the objective estimate is undone (factors
    and moments restored exactly) and the rate decays; the fit stops after
    max_fails such epochs."""
    gcp, torch = env
    dims = [40, 30, 20]
    coords, vals = synth.uniform_sparse(dims, 1500, 91, lam=2.0)
    F0 = synth.factors_uniform(dims, 6, 92, lo=0.1, hi=1.0)
    ctx = gcp.gcp_create(dims, coords, vals, 6, "poisson", seed=93)
    ctx.set_factors(F0)
    # a rate this large with lower bound 0 drives factors to the bound: every epoch fails
    rep = ctx.fit(gcp.AdamParams(lr=50.0, lower=0.0), 500, 500, 4000, 4000, iters=20, max_epochs=10, max_fails=3,
                  decay=0.5)
    assert rep["fails"] == 3 and rep["epochs"] == 3 and rep["iterations"] == 0
    assert rep["objective"] == rep["objective0"]
    assert rep["lr"] == pytest.approx(50.0 * 0.5 ** 3)
    for a, b in zip(ctx.get_factors(), F0):
        assert np.array_equal(a, b)
    ctx.close()


def test_l2_probe_performs_every_row_operation(env):
    """The measured ceiling is only meaningful if the probe does its work:
    every reduction lands (the buffer's total equals the sum of all added
    values) and the load probe leaves the buffer unchanged."""
    gcp, torch = env
    Rp, d, ops, rows = 32, 4, 100_003, 4096
    buf = torch.zeros(rows * Rp, dtype=torch.float32, device="cuda")
    gcp.gcp_probe_l2("red", buf, Rp, d, ops)
    torch.cuda.synchronize()
    # op o adds 1e-30 (o mod 8) to each of the Rp columns of d rows
    k = np.arange(ops) % 8
    expect = d * Rp * 1e-30 * float(k.sum())
    total = float(buf.double().sum())
    assert abs(total - expect) <= 1e-4 * expect, (total, expect)
    before = buf.clone()
    gcp.gcp_probe_l2("load", buf, Rp, d, ops)
    torch.cuda.synchronize()
    assert torch.equal(buf, before)
    gcp.gcp_probe_l2("both", buf, 16, 3, ops)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(buf).all()) and float(buf.double().sum()) > total
    # rows wider than 32 floats: two quads per lane, as in the fused pass
    wide = torch.zeros(2048 * 64, dtype=torch.float32, device="cuda")
    gcp.gcp_probe_l2("red", wide, 64, 3, ops)
    torch.cuda.synchronize()
    expect = 3 * 64 * 1e-30 * float(k.sum())
    total = float(wide.double().sum())
    assert abs(total - expect) <= 1e-4 * expect, (total, expect)
    assert float(wide.view(2048, 64).double().sum(0).min()) > 0.0  # every column was reached
