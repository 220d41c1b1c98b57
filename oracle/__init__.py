"""FP64 CPU oracle of the stochastic GCP gradient (Myers & Phipps, Sec. 3.1).

TEST INFRASTRUCTURE ONLY: this package exists to check the GPU library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the GPU library never does, and it imports
nothing from the GPU library.  It wraps the plain C in ``gcp_oracle.c``
(compiled with gcc at first use, or by ``build()``) through ctypes and adds
numpy marshalling only: every arithmetic step lives in the C file, one
sample at a time, in sample order, in double precision.

Parity pins live in ``tests/test_oracle_pins.py``: Philox against numpy's
independent Philox4x64-10, the losses against scipy.stats negative
log-likelihoods, the full gradient against the Gaussian closed form and an
einsum MTTKRP, the stratified estimator's expectation by exact enumeration,
central finite differences, the samplers' distributions, weights and counter
layout (the semi-stratified sampler's included, against numpy's Philox),
and Adam against torch.optim.Adam.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gcp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")

GAUSSIAN, POISSON, BERNOULLI_LOGIT, GAMMA = 0, 1, 2, 3
LOSSES = {"gaussian": GAUSSIAN, "poisson": POISSON, "bernoulli": BERNOULLI_LOGIT, "gamma": GAMMA}

_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile gcp_oracle.c into a shared library with gcc (plain -O2, IEEE)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
    lib.orc_map64.restype = ctypes.c_uint64
    lib.orc_map64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.orc_draw_nonzero.restype = ctypes.c_int64
    lib.orc_draw_nonzero.argtypes = [ctypes.c_uint64] * 3 + [ctypes.c_int64]
    lib.orc_draw_zero.restype = ctypes.c_int
    lib.orc_draw_zero.argtypes = [ctypes.c_uint64] * 3 + [ctypes.c_int, _i64p, _u64p, ctypes.c_int64,
                                                           ctypes.c_int, _i64p]
    lib.orc_stratified_samples.restype = ctypes.c_int64
    lib.orc_stratified_samples.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int, _i64p, ctypes.c_int64, _i32p, _f32p, _u64p,
                                           ctypes.c_int, _i32p, _f64p, _f64p, _i64p]
    lib.orc_uniform_samples.restype = None
    lib.orc_uniform_samples.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, _i64p,
                                        _f32p, _i32p, _f64p, _f64p]
    lib.orc_semi_stratified_samples.restype = None
    lib.orc_semi_stratified_samples.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int, _i64p, ctypes.c_int64, _i32p,
                                                _f32p, _i32p, _f64p, _f64p]
    lib.orc_loss_vec.restype = None
    lib.orc_loss_vec.argtypes = [ctypes.c_int, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p]
    lib.orc_model.restype = ctypes.c_double
    lib.orc_model.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _f64p, _i32p]
    lib.orc_sampled_loss_grad.restype = ctypes.c_double
    lib.orc_sampled_loss_grad.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _f64p, ctypes.c_int, ctypes.c_int64,
                                          _i32p, _f64p, _f64p, _u8p, _f64p]
    lib.orc_full_loss_grad.restype = ctypes.c_double
    lib.orc_full_loss_grad.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _f64p, ctypes.c_int, _f64p, _f64p]
    lib.orc_fedadam_server.restype = None
    lib.orc_fedadam_server.argtypes = [ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, _f64p, _f64p] + [
        ctypes.c_double] * 5 + [ctypes.c_int64]
    lib.orc_adam_step.restype = None
    lib.orc_adam_step.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p] + [ctypes.c_double] * 5 + [
        ctypes.c_int64]
    _lib = lib
    return lib


def _p(a, ptype):
    return a.ctypes.data_as(ptype) if a is not None else None


def _dims(dims):
    return np.ascontiguousarray(dims, dtype=np.int64)


def _loss_id(loss):
    return LOSSES[loss] if isinstance(loss, str) else int(loss)


# ------------------------------------------------------------------ random
def philox(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for a 4-word counter and a 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_p(c, _u64p), _p(k, _u64p), _p(out, _u64p))
    return out


def map64(u: int, n: int) -> int:
    """floor(u * n / 2**64)."""
    return int(_load().orc_map64(ctypes.c_uint64(int(u)), ctypes.c_uint64(int(n))))


def draw_nonzero(seed, t, j, nnz) -> int:
    return int(_load().orc_draw_nonzero(seed, t, j, nnz))


def sorted_keys(dims, coords) -> np.ndarray:
    """Sorted uint64 linear indices (last mode fastest) of the nonzeros; the
    sorted coordinate list searched by the zero check of Sec. 3.1.1."""
    dims = _dims(dims)
    keys = np.zeros(coords.shape[0], dtype=np.uint64)
    for k in range(len(dims)):
        keys = keys * np.uint64(dims[k]) + coords[:, k].astype(np.uint64)
    return np.sort(keys)


def draw_zero(seed, t, j, dims, skeys, cap=64):
    """(coords, attempts) of zero draw j, or (None, -1) if exhausted."""
    dims = _dims(dims)
    idx = np.zeros(len(dims), dtype=np.int64)
    a = _load().orc_draw_zero(seed, t, j, len(dims), _p(dims, _i64p), _p(skeys, _u64p), len(skeys), cap,
                              _p(idx, _i64p))
    return (idx if a > 0 else None), a


# ----------------------------------------------------------------- samples
class SamplerExhausted(RuntimeError):
    pass


def stratified_samples(seed, t, p, q, dims, coords, vals, skeys=None, cap=64):
    """Stratified sample set of iteration t (Sec. 3.1.1).

    Returns (idx [(p+q) x d] int32, x [p+q] f64, w [p+q] f64, attempts)."""
    dims = _dims(dims)
    d = len(dims)
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    if skeys is None:
        skeys = sorted_keys(dims, coords)
    S = p + q
    idx = np.zeros((S, d), dtype=np.int32)
    x = np.zeros(S, dtype=np.float64)
    w = np.zeros(S, dtype=np.float64)
    att = ctypes.c_int64(0)
    rc = _load().orc_stratified_samples(seed, t, p, q, d, _p(dims, _i64p), coords.shape[0], _p(coords, _i32p),
                                        _p(vals, _f32p), _p(skeys, _u64p), cap, _p(idx, _i32p), _p(x, _f64p),
                                        _p(w, _f64p), ctypes.byref(att))
    if rc != 0:
        raise SamplerExhausted(f"zero draw {-rc - 1} found no zero in {cap} attempts")
    return idx, x, w, int(att.value)


def uniform_samples(seed, t, s, dims, X=None):
    """Uniform sample set of a dense tensor: s cells, weight M/s."""
    dims = _dims(dims)
    d = len(dims)
    idx = np.zeros((s, d), dtype=np.int32)
    x = np.zeros(s, dtype=np.float64)
    w = np.zeros(s, dtype=np.float64)
    Xf = None if X is None else np.ascontiguousarray(X, dtype=np.float32).reshape(-1)
    _load().orc_uniform_samples(seed, t, s, d, _p(dims, _i64p), _p(Xf, _f32p), _p(idx, _i32p), _p(x, _f64p),
                                _p(w, _f64p))
    return idx, x, w


def semi_stratified_samples(seed, t, p, q, dims, coords, vals):
    """Semi-stratified sample set (Sec. 3.1.1): zeros drawn over all cells,
    no search.  Returns (idx, x, w, semi) with semi[s] = 1 for nonzeros."""
    dims = _dims(dims)
    d = len(dims)
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float32)
    S = p + q
    idx = np.zeros((S, d), dtype=np.int32)
    x = np.zeros(S, dtype=np.float64)
    w = np.zeros(S, dtype=np.float64)
    _load().orc_semi_stratified_samples(seed, t, p, q, d, _p(dims, _i64p), coords.shape[0], _p(coords, _i32p),
                                        _p(vals, _f32p), _p(idx, _i32p), _p(x, _f64p), _p(w, _f64p))
    semi = np.zeros(S, dtype=np.uint8)
    semi[:p] = 1
    return idx, x, w, semi


# ------------------------------------------------------- loss and gradient
def loss_fn(loss, x, m):
    """Elementwise (f, df/dm) of one of the four losses."""
    x = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), np.shape(m)))
    m = np.ascontiguousarray(m, dtype=np.float64)
    f = np.zeros_like(m)
    df = np.zeros_like(m)
    _load().orc_loss_vec(_loss_id(loss), m.size, _p(x, _f64p), _p(m, _f64p), _p(f, _f64p), _p(df, _f64p))
    return f, df


def flat_factors(factors) -> np.ndarray:
    """Concatenate per-mode I_k x R factor matrices into one FP64 vector."""
    return np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in factors])


def split_factors(flat, dims, R):
    out, o = [], 0
    for I in dims:
        out.append(flat[o:o + I * R].reshape(I, R))
        o += I * R
    return out


def model(dims, factors, idx) -> float:
    dims = _dims(dims)
    A = flat_factors(factors)
    R = np.asarray(factors[0]).shape[1]
    i = np.ascontiguousarray(idx, dtype=np.int32)
    return float(_load().orc_model(len(dims), _p(dims, _i64p), R, _p(A, _f64p), _p(i, _i32p)))


def sampled_loss_grad(dims, factors, loss, idx, x, w, semi=None, grad=True):
    """Sampled loss sum_s w_s f(x_s, m_s) and per-mode sampled gradients."""
    dims = _dims(dims)
    d = len(dims)
    R = np.asarray(factors[0]).shape[1]
    A = flat_factors(factors)
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, d)
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    sm = None if semi is None else np.ascontiguousarray(semi, dtype=np.uint8)
    G = np.zeros(A.size, dtype=np.float64) if grad else None
    F = _load().orc_sampled_loss_grad(d, _p(dims, _i64p), R, _p(A, _f64p), _loss_id(loss), idx.shape[0],
                                      _p(idx, _i32p), _p(x, _f64p), _p(w, _f64p), _p(sm, _u8p), _p(G, _f64p))
    return float(F), (split_factors(G, dims, R) if grad else None)


def full_loss_grad(dims, factors, loss, X):
    """Full GCP loss and gradient of a dense tensor X by enumeration."""
    dims = _dims(dims)
    d = len(dims)
    R = np.asarray(factors[0]).shape[1]
    A = flat_factors(factors)
    Xd = np.ascontiguousarray(X, dtype=np.float64).reshape(-1)
    G = np.zeros(A.size, dtype=np.float64)
    F = _load().orc_full_loss_grad(d, _p(dims, _i64p), R, _p(A, _f64p), _loss_id(loss), _p(Xd, _f64p),
                                   _p(G, _f64p))
    return float(F), split_factors(G, dims, R)


def adam_step(A, B, C, G, lr, beta1, beta2, eps, lower, t):
    """Algorithm 1 on flat FP64 vectors, in place."""
    for a in (A, B, C):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    G = np.ascontiguousarray(G, dtype=np.float64)
    _load().orc_adam_step(A.size, _p(A, _f64p), _p(B, _f64p), _p(C, _f64p), _p(G, _f64p), lr, beta1, beta2, eps,
                          lower, t)


def fedadam_server(M, U, B, C, lr, beta1, beta2, eps, lower, t):
    """Algorithm 4 reconciliation in place on U, B, C (flat FP64); M is the
    list of client models (flat FP64).  Returns the new U."""
    Ms = np.ascontiguousarray(np.stack([np.asarray(m, np.float64) for m in M]))
    for a in (U, B, C):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _load().orc_fedadam_server(Ms.shape[0], Ms.shape[1], _p(Ms, _f64p), _p(U, _f64p), _p(B, _f64p), _p(C, _f64p),
                               lr, beta1, beta2, eps, lower, t)
    return U


def densify(dims, coords, vals) -> np.ndarray:
    """Dense FP64 array of a COO tensor (tiny tensors only)."""
    X = np.zeros(tuple(int(i) for i in dims), dtype=np.float64)
    X[tuple(np.asarray(coords).T)] = vals
    return X
