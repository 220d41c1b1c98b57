"""Seeded synthetic inputs for the stochastic GCP gradient.

This module only makes inputs: tensors, factor matrices and the client
batch.  It holds none of the method's arithmetic (no model evaluation of the
decomposition being fitted, no loss, no gradient, no sampling of the
estimator); both the GPU library's tests and the FP64 oracle read its
output.  Every generator is a pure function of its arguments and seed
(numpy PCG64).

Workload recipes (the paper's own tensors, Table 1, are not available; these
synthetic stand-ins keep the shape, sparsity and value statistics):
  * ``uniform_sparse``: distinct, uniformly placed nonzeros, values
    1 + Poisson(lam) (small 3-way test tensors; the federated clients).
  * ``zipf_sparse``: each coordinate drawn per mode from a Zipf(s) marginal
    P(i) ~ (i+1)^-s over 0..I_k-1, duplicates removed, a uniform subset of
    the distinct cells kept, values 1 + Poisson(lam); the skewed count
    tensor.
  * ``bernoulli_logit_sparse``: ones placed by a rank-R_true logistic model
    (cell probability sigma(m + b)), drawn by rejection from uniform cells.
  * ``dense_cp_sinusoid``: a dense FP32 tensor = rank-R_true CP signal with
    sinusoidal factor columns plus Gaussian noise.
"""
from __future__ import annotations

import math

import numpy as np


def _keys(dims, coords) -> np.ndarray:
    """uint64 linear index, last mode fastest."""
    keys = np.zeros(coords.shape[0], dtype=np.uint64)
    for k, I in enumerate(dims):
        keys = keys * np.uint64(I) + coords[:, k].astype(np.uint64)
    return keys


def _decode(dims, keys) -> np.ndarray:
    coords = np.zeros((keys.size, len(dims)), dtype=np.int32)
    rem = keys.copy()
    for k in range(len(dims) - 1, -1, -1):
        coords[:, k] = (rem % np.uint64(dims[k])).astype(np.int32)
        rem //= np.uint64(dims[k])
    return coords


def _sorted_unique(a):
    """Sorted distinct values (sort, then drop repeats)."""
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _draw_distinct(dims, nnz, draw_batch, rng, max_rounds=64):
    """Draw coordinate batches until at least nnz distinct cells exist, then
    keep a uniformly random subset of nnz of them.  Returns sorted keys."""
    M = math.prod(int(i) for i in dims)
    if nnz > M:
        raise ValueError("more nonzeros than cells")
    keys = np.zeros(0, dtype=np.uint64)
    rate = 1.0  # distinct cells gained per draw, re-estimated each round
    for _ in range(max_rounds):
        need = nnz - keys.size
        if need <= 0:
            break
        n = max(1024, int(1.1 * need / max(rate, 0.05)))
        before = keys.size
        keys = _sorted_unique(np.concatenate([keys, _keys(dims, draw_batch(n, rng))]))
        rate = max((keys.size - before) / n, 1e-3)
    if keys.size < nnz:
        raise RuntimeError("could not draw enough distinct cells")
    if keys.size > nnz:
        keys = np.sort(keys[rng.permutation(keys.size)[:nnz]])
    return keys


def uniform_sparse(dims, nnz, seed, lam=2.0):
    """nnz distinct uniformly placed cells, values 1 + Poisson(lam).

    Returns (coords [nnz x d] int32 sorted lexicographically, vals float32)."""
    dims = [int(i) for i in dims]
    rng = np.random.default_rng(seed)

    def draw(n, rng):
        return np.stack([rng.integers(0, I, size=n, dtype=np.int64) for I in dims], axis=1)

    keys = _draw_distinct(dims, nnz, draw, rng)
    vals = (1 + rng.poisson(lam, size=nnz)).astype(np.float32)
    return _decode(dims, keys), vals


def zipf_pmf(I, s):
    p = (np.arange(1, I + 1, dtype=np.float64)) ** (-s)
    return p / p.sum()


def zipf_sparse(dims, nnz, seed, s=1.1, lam=3.0):
    """nnz distinct cells with per-mode Zipf(s) marginals, values 1 + Poisson(lam)."""
    dims = [int(i) for i in dims]
    rng = np.random.default_rng(seed)
    cdfs = [np.cumsum(zipf_pmf(I, s)) for I in dims]

    def draw(n, rng):
        cols = []
        for I, cdf in zip(dims, cdfs):
            u = rng.random(n) * cdf[-1]
            cols.append(np.minimum(np.searchsorted(cdf, u, side="right"), I - 1).astype(np.int64))
        return np.stack(cols, axis=1)

    keys = _draw_distinct(dims, nnz, draw, rng)
    vals = (1 + rng.poisson(lam, size=nnz)).astype(np.float32)
    return _decode(dims, keys), vals


def bernoulli_logit_sparse(dims, nnz, seed, rank=16, logit_std=0.5, density=None, chunk=1 << 22):
    """nnz distinct ones placed by a rank-`rank` logistic model.

    True factors are N(0, sigma^2) with sigma chosen so the logit has standard
    deviation ~logit_std; the bias b puts the expected density at
    nnz / M.  Cells are drawn uniformly and accepted with probability
    sigma(m+b) / sigma(c+b), c = 4 logit_std (cells with m > c, a ~3e-5
    tail, are accepted with probability 1).  Returns (coords, vals=1)."""
    dims = [int(i) for i in dims]
    d = len(dims)
    M = math.prod(dims)
    rng = np.random.default_rng(seed)
    sig = (logit_std / math.sqrt(rank)) ** (1.0 / d)
    U = [rng.normal(0.0, sig, size=(I, rank)).astype(np.float32) for I in dims]
    dens = nnz / M if density is None else density
    b = math.log(dens) - 0.5 * logit_std ** 2
    c = 4.0 * logit_std
    top = 1.0 / (1.0 + math.exp(-(c + b)))

    def draw(n, rng):
        out = []
        got = 0
        while got < n:
            cand = np.stack([rng.integers(0, I, size=chunk, dtype=np.int64) for I in dims], axis=1)
            prod = U[0][cand[:, 0]]
            for k in range(1, d):
                prod *= U[k][cand[:, k]]
            logit = prod.sum(axis=1, dtype=np.float64) + b
            acc = rng.random(chunk) * top < 1.0 / (1.0 + np.exp(-logit))
            out.append(cand[acc])
            got += int(acc.sum())
        return np.concatenate(out)[:n]

    keys = _draw_distinct(dims, nnz, draw, rng)
    return _decode(dims, keys), np.ones(nnz, dtype=np.float32)


def dense_cp_sinusoid(dims, seed, rank_true=8, sigma=0.1):
    """Dense FP32 tensor: sum_r prod_k S_k(:, r) + N(0, sigma^2) noise with
    S_k(i, r) = sin(2 pi (r+1)(i+0.5)/I_k + r).  Row-major, last mode fastest."""
    dims = [int(i) for i in dims]
    rng = np.random.default_rng(seed)
    S = []
    for I in dims:
        i = np.arange(I, dtype=np.float64)[:, None] + 0.5
        r = np.arange(rank_true, dtype=np.float64)[None, :]
        S.append(np.sin(2 * np.pi * (r + 1) * i / I + r))
    X = np.empty(dims, dtype=np.float32)
    rest = S[1:]
    letters = "abcdefgh"[: len(dims) - 1]
    spec = "r," + ",".join(f"{c}r" for c in letters) + "->" + letters
    for i0 in range(dims[0]):
        X[i0] = np.einsum(spec, S[0][i0], *rest, optimize=True)
        X[i0] += rng.standard_normal(size=dims[1:], dtype=np.float32) * np.float32(sigma)
    return X


def factors_uniform(dims, rank, seed, lo=0.0, hi=1.0):
    """Per-mode I_k x rank FP32 factor matrices with U(lo, hi) entries."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(lo, hi, size=(int(I), rank)).astype(np.float32) for I in dims]


def factors_normal(dims, rank, seed, std=1.0):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal(size=(int(I), rank)) * std).astype(np.float32) for I in dims]


def client_batch(nclients, seed, dim_lo=200, dim_hi=5000, nnz_lo=1e4, nnz_hi=2e6, lam=2.0, ndim=3,
                 max_fill=0.5):
    """Independent sparse 3-way client shards: mode sizes U{dim_lo..dim_hi},
    nnz log-uniform in [nnz_lo, nnz_hi] (at most max_fill of the cells),
    distinct uniform placement, values 1 + Poisson(lam).
    Returns a list of (dims, coords, vals)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(nclients):
        dims = [int(x) for x in rng.integers(dim_lo, dim_hi + 1, size=ndim)]
        nnz = int(math.exp(rng.uniform(math.log(nnz_lo), math.log(nnz_hi))))
        nnz = min(nnz, int(max_fill * math.prod(dims)))
        coords, vals = uniform_sparse(dims, nnz, int(rng.integers(0, 2**31)), lam=lam)
        out.append((dims, coords, vals))
    return out


# Named workloads.  Sizes follow the benchmark configurations; each returns
# a dict the tests and the benchmark both consume.
def workload_small_gaussian(seed=1001):
    """50 x 40 x 30, 2,000 distinct uniform nonzeros, 1 + Poisson(2), rank 4."""
    dims = [50, 40, 30]
    coords, vals = uniform_sparse(dims, 2000, seed, lam=2.0)
    return dict(dims=dims, coords=coords, vals=vals, rank=4, loss="gaussian",
                factors=factors_uniform(dims, 4, seed + 1000), p=1000, q=1000)


def workload_zipf_count(scale=1.0, seed=1002, nnz=None):
    """2000 x 1500 x 1000 x 200 Zipf(1.1) count tensor with 5e7 nonzeros,
    Poisson loss, rank 32, 2^20 + 2^20 samples.  `scale` < 1 shrinks the
    nonzero count and samples proportionally for quick tests; `nnz` sets
    the nonzero count alone (full sample counts), for profiling captures."""
    dims = [2000, 1500, 1000, 200]
    nnz = int(nnz) if nnz else max(1000, int(5e7 * scale))
    coords, vals = zipf_sparse(dims, nnz, seed, s=1.1, lam=3.0)
    S = max(256, int((1 << 20) * scale))
    return dict(dims=dims, coords=coords, vals=vals, rank=32, loss="poisson",
                factors=factors_uniform(dims, 32, seed + 1000), p=S, q=S)


def cached(name, make, cache_dir=None):
    """Return make()'s dict of arrays and scalars, stored once under
    `cache_dir` (default: <repo>/_cache, or $GCP_CACHE_DIR) as a pickle so that
    several processes of one run generate a large workload only once."""
    import os
    import pickle

    d = cache_dir or os.environ.get("GCP_CACHE_DIR") or os.path.join(
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache")
    path = os.path.join(d, name + ".pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    w = make()
    os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        pickle.dump(w, f, protocol=pickle.HIGHEST_PROTOCOL)
    os.replace(tmp, path)
    return w
