"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks the oracle against something it does not share code with:
numpy's Philox4x64-10, Python integers, scipy.stats likelihoods, the
Gaussian closed-form gradient, an einsum MTTKRP on a dense tensor, exact
enumeration of the stratified estimator's expectation, central finite
differences, a chi-square test of the sampler and torch.optim.Adam.
"""
import math

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle
import synth

LOSSES = ["gaussian", "poisson", "bernoulli", "gamma"]


# ------------------------------------------------------------------ Philox
def _numpy_philox_block(ctr, key):
    """numpy's Philox4x64-10 increments its counter before producing a block,
    so the block of counter c is produced from state c - 1."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    c = (c - 1) % 2**256  # the counter is one 256-bit integer, word 0 lowest
    c = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((0, 0, 0, 0), (1, 2)),
    ((12345, 7, 3, 0), (2023, 1)),
    ((2**64 - 1, 2**63, 5, 9), (2**64 - 1, 2**32 + 5)),
    ((987654321, 4 * 63 + 1, 2**40, 0), (3002, 1)),
])
def test_philox_matches_numpy(ctr, key):
    assert [int(v) for v in oracle.philox(ctr, key)] == [int(v) for v in _numpy_philox_block(ctr, key)]


def test_philox_random_counters_match_numpy():
    rng = np.random.default_rng(5)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        assert [int(v) for v in oracle.philox(ctr, key)] == [int(v) for v in _numpy_philox_block(ctr, key)]


# ------------------------------------------------------------------- map64
def test_map64_is_exact_floor():
    rng = np.random.default_rng(0)
    cases = [(0, 1), (2**64 - 1, 1), (2**64 - 1, 7), (2**63, 2), (2**64 - 1, 2**63), (12345, 2**40 + 3)]
    cases += [(int(u), int(n)) for u, n in zip(rng.integers(0, 2**64 - 1, 500, dtype=np.uint64),
                                              rng.integers(1, 2**50, 500, dtype=np.uint64))]
    for u, n in cases:
        got = oracle.map64(u, n)
        assert 0 <= got < n
        assert got * 2**64 <= u * n < (got + 1) * 2**64  # the defining inequality


def test_map64_even_grid_is_balanced():
    n = 7
    us = [-(-i * 2**64 // 7000) for i in range(7000)]  # ceil grid: 1000 points per bucket
    counts = np.bincount([oracle.map64(u, n) for u in us], minlength=n)
    assert counts.tolist() == [1000] * n


# ------------------------------------------------------------------ losses
def _nll(loss, x, m):
    """Negative log-likelihood from scipy.stats, minus the data-only constant
    that the GCP loss drops."""
    if loss == "gaussian":  # variance 1/2 makes -log p = (x-m)^2 + log(pi)/2
        return -scipy.stats.norm.logpdf(x, loc=m, scale=math.sqrt(0.5)) - 0.5 * math.log(math.pi)
    if loss == "poisson":
        return -scipy.stats.poisson.logpmf(x, m) - scipy.special.gammaln(x + 1)
    if loss == "bernoulli":
        return -scipy.stats.bernoulli.logpmf(x, scipy.special.expit(m))
    if loss == "gamma":  # shape 1, mean m
        return -scipy.stats.gamma.logpdf(x, a=1.0, scale=m)
    raise ValueError(loss)


def _loss_points(loss):
    rng = np.random.default_rng(11)
    if loss == "gaussian":
        return rng.normal(size=50), rng.normal(size=50)
    if loss == "poisson":
        return rng.poisson(3, size=50).astype(float), rng.uniform(0.2, 6, size=50)
    if loss == "bernoulli":
        return rng.integers(0, 2, size=50).astype(float), rng.normal(scale=4, size=50)
    return rng.exponential(2.0, size=50) + 0.01, rng.uniform(0.3, 5, size=50)


@pytest.mark.parametrize("loss", LOSSES)
def test_loss_is_negative_log_likelihood(loss):
    x, m = _loss_points(loss)
    f, _ = oracle.loss_fn(loss, x, m)
    np.testing.assert_allclose(f, _nll(loss, x, m), rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("loss", LOSSES)
def test_loss_derivative_is_derivative_of_likelihood(loss):
    x, m = _loss_points(loss)
    _, df = oracle.loss_fn(loss, x, m)
    h = 1e-6
    fd = (_nll(loss, x, m + h) - _nll(loss, x, m - h)) / (2 * h)
    np.testing.assert_allclose(df, fd, rtol=1e-6, atol=1e-7)


def test_bernoulli_loss_is_stable_for_large_logits():
    f, df = oracle.loss_fn("bernoulli", np.array([1.0, 0.0, 1.0]), np.array([800.0, -800.0, -30.0]))
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(df))
    np.testing.assert_allclose(f, [0.0, 0.0, 30.0], atol=1e-12)


# ----------------------------------------------------- full gradient pins
def _dense_model(factors):
    d = len(factors)
    letters = "abcdefgh"[:d]
    spec = ",".join(f"{c}r" for c in letters) + "->" + letters
    return np.einsum(spec, *[np.asarray(a, np.float64) for a in factors])


def _einsum_mttkrp(Y, factors, n):
    d = len(factors)
    letters = "abcdefgh"[:d]
    ins = [letters] + [f"{letters[k]}r" for k in range(d) if k != n]
    spec = ",".join(ins) + f"->{letters[n]}r"
    return np.einsum(spec, Y, *[np.asarray(factors[k], np.float64) for k in range(d) if k != n])


def _tiny(dims, nnz, seed, loss):
    coords, vals = synth.uniform_sparse(dims, nnz, seed, lam=2.0)
    if loss == "bernoulli":
        vals = np.ones_like(vals)
    if loss in ("gaussian", "bernoulli"):
        factors = synth.factors_normal(dims, 3, seed + 1, std=0.7)
    else:
        factors = synth.factors_uniform(dims, 3, seed + 1, lo=0.2, hi=1.0)
    return coords, vals, factors


def test_gaussian_full_gradient_closed_form():
    """For f = (x-m)^2 the GCP gradient is 2 (A_n *_{k!=n} A_k^T A_k - X_(n) Z_n)."""
    w = synth.workload_small_gaussian()
    dims, factors = w["dims"], [a.astype(np.float64) for a in w["factors"]]
    X = oracle.densify(dims, w["coords"], w["vals"])
    F, G = oracle.full_loss_grad(dims, factors, "gaussian", X)
    Mfull = _dense_model(factors)
    assert F == pytest.approx(float(((X - Mfull) ** 2).sum()), rel=1e-12)
    for n in range(3):
        gram = np.ones((4, 4))
        for k in range(3):
            if k != n:
                gram *= factors[k].T @ factors[k]
        closed = 2.0 * (factors[n] @ gram - _einsum_mttkrp(X, factors, n))
        np.testing.assert_allclose(G[n], closed, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("dims,nnz", [([4, 3, 2], 7), ([3, 3, 3, 2], 20), ([5, 4], 6)])
def test_full_gradient_matches_einsum_mttkrp(loss, dims, nnz):
    coords, vals, factors = _tiny(dims, nnz, 31, loss)
    X = oracle.densify(dims, coords, vals)
    F, G = oracle.full_loss_grad(dims, factors, loss, X)
    Mfull = _dense_model(factors)
    f, df = oracle.loss_fn(loss, X.ravel(), Mfull.ravel())
    assert F == pytest.approx(float(_nll(loss, X.ravel(), Mfull.ravel()).sum()), rel=1e-9)
    Y = df.reshape(X.shape)
    for n in range(len(dims)):
        np.testing.assert_allclose(G[n], _einsum_mttkrp(Y, factors, n), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
def test_full_gradient_central_differences(loss):
    dims = [4, 3, 2]
    coords, vals, factors = _tiny(dims, 7, 41, loss)
    X = oracle.densify(dims, coords, vals)
    _, G = oracle.full_loss_grad(dims, factors, loss, X)
    h = 1e-6
    rng = np.random.default_rng(3)
    for _ in range(8):
        n = int(rng.integers(0, 3))
        i, r = int(rng.integers(0, dims[n])), int(rng.integers(0, 3))
        fp = [a.astype(np.float64).copy() for a in factors]
        fm = [a.astype(np.float64).copy() for a in factors]
        fp[n][i, r] += h
        fm[n][i, r] -= h
        fd = (oracle.full_loss_grad(dims, fp, loss, X)[0] - oracle.full_loss_grad(dims, fm, loss, X)[0]) / (2 * h)
        assert G[n][i, r] == pytest.approx(fd, rel=1e-6, abs=1e-7)


# ------------------------------------------- estimator expectation (exact)
@pytest.mark.parametrize("loss", LOSSES)
def test_stratified_estimator_is_unbiased_by_enumeration(loss):
    """p = q = 1: E[G~] = sum_e (1/N) G~(e; w=N) + sum_z 1/(M-N) G~(z; w=M-N)
    must equal the full gradient exactly (Sec. 3.1.1 weights)."""
    dims = [4, 3, 2]
    coords, vals, factors = _tiny(dims, 7, 51, loss)
    X = oracle.densify(dims, coords, vals)
    Ffull, Gfull = oracle.full_loss_grad(dims, factors, loss, X)
    N, M = len(vals), int(np.prod(dims))
    nzset = {tuple(c) for c in coords.tolist()}
    zeros = [c for c in np.ndindex(*dims) if c not in nzset]
    EG = [np.zeros_like(g) for g in Gfull]
    EF = 0.0
    for e in range(N):
        F, G = oracle.sampled_loss_grad(dims, factors, loss, coords[e:e + 1], [vals[e]], [N])
        EF += F / N
        for n in range(3):
            EG[n] += G[n] / N
    for z in zeros:
        F, G = oracle.sampled_loss_grad(dims, factors, loss, np.array([z]), [0.0], [M - N])
        EF += F / (M - N)
        for n in range(3):
            EG[n] += G[n] / (M - N)
    assert EF == pytest.approx(Ffull, rel=1e-12)
    for n in range(3):
        np.testing.assert_allclose(EG[n], Gfull[n], rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("loss", LOSSES)
def test_semi_stratified_gradient_is_unbiased_by_enumeration(loss):
    """Semi-stratified (Sec. 3.1.1): nonzero value f'(x,m) - f'(0,m) with weight
    N/p, zero candidates over all M cells with weight M/q; p = q = 1."""
    dims = [4, 3, 2]
    coords, vals, factors = _tiny(dims, 7, 61, loss)
    X = oracle.densify(dims, coords, vals)
    Ffull, Gfull = oracle.full_loss_grad(dims, factors, loss, X)
    N, M = len(vals), int(np.prod(dims))
    EG = [np.zeros_like(g) for g in Gfull]
    EF = 0.0
    for e in range(N):
        F, G = oracle.sampled_loss_grad(dims, factors, loss, coords[e:e + 1], [vals[e]], [N], semi=[1])
        EF += F / N
        for n in range(3):
            EG[n] += G[n] / N
    for z in np.ndindex(*dims):
        F, G = oracle.sampled_loss_grad(dims, factors, loss, np.array([z]), [0.0], [M], semi=[0])
        EF += F / M
        for n in range(3):
            EG[n] += G[n] / M
    assert EF == pytest.approx(Ffull, rel=1e-12)
    for n in range(3):
        np.testing.assert_allclose(EG[n], Gfull[n], rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------- sampler
def test_sampler_distribution_chi_square():
    w = synth.workload_small_gaussian()
    dims, coords, vals = w["dims"], w["coords"], w["vals"]
    N, M = len(vals), int(np.prod(dims))
    p, q = 100 * N, 10 * (M - N)
    idx, x, wts, attempts = oracle.stratified_samples(3001, 5, p, q, dims, coords, vals)
    keys = np.zeros(p + q, dtype=np.int64)
    for k in range(3):
        keys = keys * dims[k] + idx[:, k]
    nzkeys = set(oracle.sorted_keys(dims, coords).tolist())
    zkeys = keys[p:]
    assert not any(int(k) in nzkeys for k in np.unique(zkeys))
    assert np.all(x[p:] == 0) and np.all(wts[p:] == (M - N) / q) and np.all(wts[:p] == N / p)
    # zero samples uniform over the M - N zeros
    zero_cells = np.setdiff1d(np.arange(M), np.fromiter(nzkeys, dtype=np.int64))
    counts = np.bincount(np.searchsorted(zero_cells, zkeys), minlength=M - N)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    # nonzero samples uniform over the N nonzeros
    nz_sorted = np.sort(np.fromiter(nzkeys, dtype=np.int64))
    ncounts = np.bincount(np.searchsorted(nz_sorted, keys[:p]), minlength=N)
    assert scipy.stats.chisquare(ncounts).pvalue > 1e-4
    # nonzero samples carry their own value
    vmap = dict(zip(oracle.sorted_keys(dims, coords).tolist(), vals[np.lexsort(coords.T[::-1])].tolist()))
    assert all(vmap[int(k)] == xv for k, xv in zip(keys[:2000], x[:2000]))
    # rejection attempts per zero: geometric with mean 1 / (1 - N/M)
    mean, var = 1.0 / (1 - N / M), (N / M) / (1 - N / M) ** 2
    assert abs(attempts / q - mean) < 5 * math.sqrt(var / q)


def _counter_draw(seed, stream, t, j, sub0, dims):
    """A coordinate tuple of the documented counter layout, computed with
    numpy's independent Philox4x64-10 and Python integers: key (seed,
    stream), counter (j, sub0 + b, t, 0) for modes 4b..4b+3, word u of mode
    k mapped onto [0, I_k) as floor(u I_k / 2^64)."""
    out = []
    for b in range((len(dims) + 3) // 4):
        words = _numpy_philox_block((j, sub0 + b, t, 0), (seed, stream))
        for k in range(4 * b, min(len(dims), 4 * b + 4)):
            out.append(int(words[k - 4 * b]) * int(dims[k]) >> 64)
    return out


def test_semi_stratified_sampler_weights_values_and_layout():
    """Semi-stratified sample set (Sec. 3.1.1), checked without the GPU:
    nonzero samples are records with weight N/p; zero candidates carry x = 0
    and weight M/q (drawn over all M cells, so the unbiased weight is M/q,
    not (M-N)/q); flags mark the nonzeros; and the draws follow the counter
    layout (stream 0 for nonzeros, stream 3 for zero candidates) computed
    independently with numpy's Philox."""
    w = synth.workload_small_gaussian()
    dims, coords, vals = w["dims"], w["coords"], w["vals"]
    N, M = len(vals), int(np.prod(dims))
    seed, t, p, q = 3101, 9, 700, 900
    idx, x, wts, semi = oracle.semi_stratified_samples(seed, t, p, q, dims, coords, vals)
    assert np.all(wts[:p] == N / p)
    assert np.all(wts[p:] == M / q) and M / q != (M - N) / q
    assert np.all(semi[:p] == 1) and np.all(semi[p:] == 0)
    assert np.all(x[p:] == 0.0)
    for j in range(p):  # nonzero j: record e = floor(u N / 2^64) of stream 0
        e = int(_numpy_philox_block((j, 0, t, 0), (seed, 0))[0]) * N >> 64
        assert idx[j].tolist() == coords[e].tolist() and x[j] == float(vals[e])
    for j in range(q):
        assert idx[p + j].tolist() == _counter_draw(seed, 3, t, j, 0, dims)


def test_semi_stratified_zero_candidates_cover_every_cell():
    """Zero candidates of the semi-stratified sampler are uniform over all M
    cells, nonzero cells included: no rejection (Sec. 3.1.1).  Chi-square
    over the 60,000 cells of the 50 x 40 x 30 tensor, and the share of
    candidates that land on one of its 2,000 nonzeros is N/M."""
    w = synth.workload_small_gaussian()
    dims, coords, vals = w["dims"], w["coords"], w["vals"]
    N, M = len(vals), int(np.prod(dims))
    q = 20 * M
    idx, x, wts, _ = oracle.semi_stratified_samples(3102, 4, 0, q, dims, coords, vals)
    keys = np.zeros(q, dtype=np.int64)
    for k in range(3):
        keys = keys * dims[k] + idx[:, k]
    counts = np.bincount(keys, minlength=M)
    assert counts.size == M
    assert scipy.stats.chisquare(counts).pvalue > 1e-4
    on_nz = np.isin(keys, oracle.sorted_keys(dims, coords).astype(np.int64)).sum()
    share = N / M
    assert abs(on_nz / q - share) < 5 * math.sqrt(share * (1 - share) / q)
    assert on_nz > 0.9 * share * q  # a rejecting sampler would give none


def test_stratified_sampler_follows_counter_layout():
    """Stratified draws (Sec. 3.1.1) against numpy's Philox: nonzero j is
    record floor(u N / 2^64) of stream 0; zero draw j takes the first
    attempt a whose stream-1 tuple at sub-counter 4a is not a nonzero."""
    w = synth.workload_small_gaussian()
    dims, coords, vals = w["dims"], w["coords"], w["vals"]
    N = len(vals)
    seed, t, p, q = 3103, 2, 300, 400
    idx, x, _, _ = oracle.stratified_samples(seed, t, p, q, dims, coords, vals)
    for j in range(p):
        e = int(_numpy_philox_block((j, 0, t, 0), (seed, 0))[0]) * N >> 64
        assert idx[j].tolist() == coords[e].tolist() and x[j] == float(vals[e])
    nz = {tuple(c) for c in coords.tolist()}
    redrawn = 0
    for j in range(q):
        a = 0
        while tuple(cand := _counter_draw(seed, 1, t, j, 4 * a, dims)) in nz:
            a += 1
        redrawn += a > 0
        assert idx[p + j].tolist() == cand
    assert redrawn > 0  # the redraw path is exercised (about 3% of draws)


def test_sampler_reproducible_and_iteration_dependent():
    w = synth.workload_small_gaussian()
    a = oracle.stratified_samples(7, 3, 50, 50, w["dims"], w["coords"], w["vals"])
    b = oracle.stratified_samples(7, 3, 50, 50, w["dims"], w["coords"], w["vals"])
    c = oracle.stratified_samples(7, 4, 50, 50, w["dims"], w["coords"], w["vals"])
    assert np.array_equal(a[0], b[0]) and not np.array_equal(a[0], c[0])


def test_sampler_exhausted_on_full_tensor():
    dims = [3, 2, 2]
    coords = np.array(list(np.ndindex(*dims)), dtype=np.int32)
    vals = np.ones(len(coords), dtype=np.float32)
    with pytest.raises(oracle.SamplerExhausted):
        oracle.stratified_samples(1, 0, 4, 4, dims, coords, vals, cap=16)
    idx, _, _, _ = oracle.stratified_samples(1, 0, 4, 0, dims, coords, vals, cap=16)
    assert idx.shape == (4, 3)


def test_uniform_dense_sampler_weights_and_values():
    dims = [5, 4, 3, 2, 3]
    X = synth.dense_cp_sinusoid(dims, 3, rank_true=2)
    idx, x, wts = oracle.uniform_samples(9, 2, 5000, dims, X)
    assert np.all(wts == np.prod(dims) / 5000)
    np.testing.assert_array_equal(x, X[tuple(idx.T)].astype(np.float64))
    counts = np.bincount(np.ravel_multi_index(tuple(idx.T), dims), minlength=int(np.prod(dims)))
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


# --------------------------------------------------------- sampled gradient
@pytest.mark.parametrize("loss", LOSSES)
def test_sampled_gradient_central_differences(loss):
    dims = [6, 5, 4, 3]
    coords, vals, factors = _tiny(dims, 40, 71, loss)
    idx, x, wts, _ = oracle.stratified_samples(5, 1, 30, 30, dims, coords, vals)
    _, G = oracle.sampled_loss_grad(dims, factors, loss, idx, x, wts)
    h = 1e-6
    rng = np.random.default_rng(8)
    for _ in range(10):
        n = int(rng.integers(0, 4))
        i = int(idx[int(rng.integers(0, 60)), n])
        r = int(rng.integers(0, 3))
        fp = [a.astype(np.float64).copy() for a in factors]
        fm = [a.astype(np.float64).copy() for a in factors]
        fp[n][i, r] += h
        fm[n][i, r] -= h
        fd = (oracle.sampled_loss_grad(dims, fp, loss, idx, x, wts, grad=False)[0]
              - oracle.sampled_loss_grad(dims, fm, loss, idx, x, wts, grad=False)[0]) / (2 * h)
        assert G[n][i, r] == pytest.approx(fd, rel=1e-6, abs=1e-6 * max(1.0, abs(fd)))


def test_sampled_gradient_duplicates_count_separately():
    """Samples are drawn with replacement; a repeated sample adds twice."""
    dims = [4, 3, 2]
    coords, vals, factors = _tiny(dims, 7, 81, "poisson")
    one = oracle.sampled_loss_grad(dims, factors, "poisson", coords[:1], [vals[0]], [2.0])
    two = oracle.sampled_loss_grad(dims, factors, "poisson", np.repeat(coords[:1], 2, 0), [vals[0]] * 2, [1.0, 1.0])
    assert one[0] == pytest.approx(two[0], rel=1e-15)
    for a, b in zip(one[1], two[1]):
        np.testing.assert_allclose(a, b, rtol=1e-15)


# ------------------------------------------------------------------- Adam
def test_adam_matches_torch_when_eps_is_zero():
    """With eps = 0, Algorithm 1's sqrt(C^ + eps) equals Kingma's
    sqrt(C^) + eps, so torch.optim.Adam is an independent reference."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    A = rng.normal(size=300)
    B, C = np.zeros(300), np.zeros(300)
    p = torch.nn.Parameter(torch.tensor(A.copy(), dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.01, betas=(0.8, 0.95), eps=0.0)
    for t in range(1, 8):
        g = rng.normal(size=300)
        oracle.adam_step(A, B, C, g, 0.01, 0.8, 0.95, 0.0, -np.inf, t)
        p.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(A, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_adam_constant_gradient_closed_form_and_lower_bound():
    """Constant G: bias-corrected moments equal G and G^2 at every step, so each
    step moves by -lr G / sqrt(G^2 + eps); the lower bound clamps."""
    G = np.array([0.5, -2.0, 1e-3, 3.0])
    A = np.array([1.0, 1.0, 1.0, 0.001])
    B, C = np.zeros(4), np.zeros(4)
    lr, eps = 0.1, 1e-8
    expect = A.copy()
    for t in range(1, 6):
        oracle.adam_step(A, B, C, G, lr, 0.9, 0.999, eps, 0.0, t)
        expect = np.maximum(expect - lr * G / np.sqrt(G * G + eps), 0.0)
        np.testing.assert_allclose(A, expect, rtol=1e-12, atol=1e-15)
    assert A[3] == 0.0


# ---------------------------------------------------------- golden fixture
def test_oracle_matches_stored_golden():
    """Regression guard: values written by tests/golden/make_golden.py."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "small_gaussian.json")) as f:
        g = json.load(f)
    w = synth.workload_small_gaussian()
    idx, x, wts, att = oracle.stratified_samples(3001, 0, w["p"], w["q"], w["dims"], w["coords"], w["vals"])
    assert idx[:8].tolist() + idx[1000:1008].tolist() == g["first_samples"]
    assert att == g["zero_attempts"]
    F, G = oracle.sampled_loss_grad(w["dims"], w["factors"], w["loss"], idx, x, wts)
    assert F == pytest.approx(g["sampled_loss"], rel=1e-12)
    assert [float(np.linalg.norm(a)) for a in G] == pytest.approx(g["sampled_grad_fro"], rel=1e-12)


def test_dense_uniform_sampled_gradient_central_differences():
    """The dense five-way case: uniform samples of a sinusoidal CP tensor,
    Gaussian loss; the sampled gradient equals central differences (FP64,
    h = 1e-6) of the sampled loss."""
    dims = [6, 5, 4, 3, 4]
    X = synth.dense_cp_sinusoid(dims, 12, rank_true=2)
    factors = synth.factors_normal(dims, 3, 13, std=0.6)
    idx, x, w = oracle.uniform_samples(14, 3, 400, dims, X)
    _, G = oracle.sampled_loss_grad(dims, factors, "gaussian", idx, x, w)
    h = 1e-6
    rng = np.random.default_rng(15)
    for _ in range(12):
        n = int(rng.integers(0, 5))
        i, r = int(idx[int(rng.integers(0, 400)), n]), int(rng.integers(0, 3))
        fp = [a.astype(np.float64).copy() for a in factors]
        fm = [a.astype(np.float64).copy() for a in factors]
        fp[n][i, r] += h
        fm[n][i, r] -= h
        fd = (oracle.sampled_loss_grad(dims, fp, "gaussian", idx, x, w, grad=False)[0]
              - oracle.sampled_loss_grad(dims, fm, "gaussian", idx, x, w, grad=False)[0]) / (2 * h)
        assert G[n][i, r] == pytest.approx(fd, rel=1e-6, abs=1e-6 * max(1.0, abs(fd)))


# ------------------------------------------------------- FedAdam server
def test_fedadam_server_fixed_point_and_sign_step():
    """Algorithm 4's reconciliation: clients equal to U leave U and the server
    moments at zero; with beta1 = beta2 = 0 and eps = 0 each step moves U by
    lr * sign(U - mean(M)) (Adam's first step on D = U - mean of clients)."""
    rng = np.random.default_rng(21)
    U = rng.normal(size=50)
    B, C = np.zeros(50), np.zeros(50)
    oracle.fedadam_server([U.copy()] * 4, U, B, C, 0.1, 0.9, 0.999, 1e-8, -np.inf, 1)  # mean exact for 4
    assert not np.any(B) and not np.any(C)
    M = [U + rng.normal(size=50) for _ in range(4)]
    mean = np.mean(M, axis=0)
    U0 = U.copy()
    oracle.fedadam_server(M, U, np.zeros(50), np.zeros(50), 0.1, 0.0, 0.0, 0.0, -np.inf, 1)
    np.testing.assert_allclose(U, U0 - 0.1 * np.sign(U0 - mean), rtol=0, atol=1e-15)


def test_fedadam_server_is_adam_on_mean_pseudo_gradient():
    """Against torch.optim.Adam (eps = 0) fed the mean pseudo-gradient."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(22)
    U = rng.normal(size=40)
    B, C = np.zeros(40), np.zeros(40)
    p = torch.nn.Parameter(torch.tensor(U.copy()))
    opt = torch.optim.Adam([p], lr=0.05, betas=(0.7, 0.9), eps=0.0)
    for t in range(1, 5):
        M = [U + rng.normal(size=40) for _ in range(3)]
        D = U - np.mean(M, axis=0)
        oracle.fedadam_server(M, U, B, C, 0.05, 0.7, 0.9, 0.0, -np.inf, t)
        p.grad = torch.tensor(D)
        opt.step()
        np.testing.assert_allclose(U, p.detach().numpy(), rtol=1e-12, atol=1e-14)
