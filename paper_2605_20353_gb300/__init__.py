"""Python binding of libgcp.so, the GB300 stochastic GCP gradient library.

Argument marshalling only: every step of the sampled gradient (sampling,
model evaluation, loss, MTTKRP, Adam) runs in the CUDA kernels behind the C
ABI declared in include/gcp.h.  Functions carry the C names; ``GcpContext``
wraps a context handle.  Device buffers are torch tensors (PyTorch supplies
device memory and streams only).  There is no CPU fallback: ``load()``
raises if the library has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcp.so")

GCP_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_DUPLICATE", 5: "ERR_HASH_FULL",
          6: "ERR_SAMPLER_EXHAUSTED", 7: "ERR_NONFINITE", 8: "ERR_DOMAIN", 9: "ERR_STATE"}
LOSSES = {"gaussian": 0, "poisson": 1, "bernoulli": 2, "gamma": 3}
DTYPES = {"fp32": 0, "bf16": 1}
MTTKRP = {"atomic": 0, "deterministic": 1, "nonfused": 2}
SAMPLING = {"stratified": 0, "semi": 1, "uniform": 2}
GCP_ITER_OBJECTIVE = 2**64 - 1
GCP_FIT_TRACE = 256


class GcpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class gcp_options(ctypes.Structure):
    _fields_ = [("factor_dtype", ctypes.c_int32), ("mttkrp", ctypes.c_int32), ("sampling", ctypes.c_int32),
                ("max_attempts", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("hash_max_load", ctypes.c_double), ("lane_cols", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gcp_adam_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("lower", ctypes.c_double)]


class gcp_fit_params(ctypes.Structure):
    _fields_ = [("adam", gcp_adam_params), ("p", ctypes.c_int64), ("q", ctypes.c_int64),
                ("p_obj", ctypes.c_int64), ("q_obj", ctypes.c_int64), ("iters", ctypes.c_int32),
                ("max_epochs", ctypes.c_int32), ("max_fails", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("decay", ctypes.c_double), ("iter0", ctypes.c_uint64)]


class gcp_fit_report(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("fails", ctypes.c_int32), ("iterations", ctypes.c_int64),
                ("objective0", ctypes.c_double), ("objective", ctypes.c_double), ("lr", ctypes.c_double),
                ("seconds", ctypes.c_double), ("grad_samples_per_s", ctypes.c_double),
                ("attempts_per_zero", ctypes.c_double), ("trace", ctypes.c_double * GCP_FIT_TRACE)]


_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double

# name -> (restype, argtypes): every entry point of include/gcp.h
SIGNATURES = {
    "gcp_options_default": (None, [ctypes.POINTER(gcp_options)]),
    "gcp_create": (_i32, [_i32, _vp, _i64, _vp, _vp, _i32, _i32, ctypes.POINTER(gcp_options), ctypes.POINTER(_vp)]),
    "gcp_create_dense": (_i32, [_i32, _vp, _vp, _i32, _i32, ctypes.POINTER(gcp_options), ctypes.POINTER(_vp)]),
    "gcp_destroy": (None, [_vp]),
    "gcp_last_error": (ctypes.c_char_p, [_vp]),
    "gcp_ndim": (_i32, [_vp]),
    "gcp_rank": (_i32, [_vp]),
    "gcp_nnz": (_i64, [_vp]),
    "gcp_num_params": (_i64, [_vp]),
    "gcp_set_factors": (_i32, [_vp, _vp]),
    "gcp_set_factor": (_i32, [_vp, _i32, _vp]),
    "gcp_set_factor_list": (_i32, [_vp, _vp]),
    "gcp_grad_factors_async": (_i32, [_vp, _vp, _u64, _i64, _i64, _vp, _vp]),
    "gcp_get_factors": (_i32, [_vp, _vp]),
    "gcp_reset_adam": (_i32, [_vp]),
    "gcp_sample": (_i32, [_vp, _u64, _i64, _i64, _vp, _vp, _vp]),
    "gcp_loss": (_i32, [_vp, _u64, _i64, _i64, ctypes.POINTER(_f64)]),
    "gcp_loss_async": (_i32, [_vp, _u64, _i64, _i64, _vp]),
    "gcp_grad": (_i32, [_vp, _u64, _i64, _i64, _vp, _vp]),
    "gcp_grad_async": (_i32, [_vp, _u64, _i64, _i64, _vp, _vp, _vp]),
    "gcp_scale_async": (_i32, [_vp, _vp, _vp, _vp, _i64]),
    "gcp_grad_norm": (_i32, [_vp, ctypes.POINTER(_f64)]),
    "gcp_adam_step": (_i32, [_vp, ctypes.POINTER(gcp_adam_params), _i64]),
    "gcp_step": (_i32, [_vp, _u64, _i64, _i64, ctypes.POINTER(gcp_adam_params), _i64, _vp]),
    "gcp_sync": (_i32, [_vp]),
    "gcp_fit": (_i32, [_vp, ctypes.POINTER(gcp_fit_params), ctypes.POINTER(gcp_fit_report)]),
    "gcp_profile": (_i32, [_vp, _i32]),
    "gcp_profile_read": (_i32, [_vp, ctypes.POINTER(_f64), ctypes.POINTER(_i64)]),
    "gcp_batch_create": (_i32, [_i32, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "gcp_batch_destroy": (None, [_vp]),
    "gcp_batch_last_error": (ctypes.c_char_p, [_vp]),
    "gcp_batch_tune": (_i32, [_vp, _i32, _i32]),
    "gcp_batch_tune_tile": (_i32, [_vp, _i32]),
    "gcp_batch_local_steps": (_i32, [_vp, _i32, ctypes.POINTER(gcp_adam_params), _u64, _i64]),
    "gcp_batch_losses": (_i32, [_vp, _vp]),
    "gcp_batch_server_init": (_i32, [_vp]),
    "gcp_batch_server_step": (_i32, [_vp, ctypes.POINTER(gcp_adam_params), _i64]),
    "gcp_grad_samples_noalloc": (_i32, [_i32, _vp, _i32, _i32, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gcp_probe_l2": (_i32, [_i32, _i32, _i32, _vp, _i64, _i64, _vp]),
}


def load():
    """Load libgcp.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2605_20353_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, handle=None):
    if rc != GCP_OK:
        msg = load().gcp_last_error(handle)
        raise GcpError(rc, msg.decode() if msg else "")


def _ptr(t):
    """Device/host address of a torch tensor or numpy array (or None)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check_buf(t, n, dtype, name):
    """The C ABI cannot see buffer sizes: refuse a buffer that is too small,
    of another element type, or not contiguous before its address is passed."""
    if t is None:
        return
    if isinstance(t, np.ndarray):
        ok_type = t.dtype == np.dtype(dtype)
        size, contiguous = t.size, t.flags["C_CONTIGUOUS"]
    else:
        import torch

        ok_type = t.dtype == {"float32": torch.float32, "float64": torch.float64}[dtype]
        size, contiguous = t.numel(), t.is_contiguous()
    if not ok_type or size < n or not contiguous:
        raise ValueError(f"{name} must be a contiguous {dtype} buffer of at least {n} elements")


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


@dataclass
class AdamParams:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    lower: float = -math.inf

    def c(self):
        return gcp_adam_params(self.lr, self.beta1, self.beta2, self.eps, self.lower)


# Hyperparameter presets for gcp_fit (Alg. 2) and the FedAdam server step
# (Alg. 4): the default column of the paper's parameter-range table and the
# values its Latin-hypercube study tuned on synthetic count data (Sec. 5.2,
# tuned-parameter table).  The lower bound 0 keeps count-data factors
# nonnegative.
FIT_PRESETS = {
    "paper_default": dict(adam=AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0), decay=0.1),
    "gcp_sgd_tuned": dict(adam=AdamParams(lr=0.035817, beta1=0.630219, beta2=0.966996, eps=1.388768e-13, lower=0.0),
                          decay=0.123013),
    "gcp_fedadam_tuned": dict(adam=AdamParams(lr=0.002185, beta1=0.603286, beta2=0.991181, eps=5.523877e-14,
                                              lower=0.0),
                              decay=0.000148, meta_rate=0.029976),
}


class GcpContext:
    """Owns one gcp_ctx (a sparse or dense tensor plus model, gradient and
    Adam state on the GPU)."""

    def __init__(self, handle, dims, rank, loss, dtype, stream):
        self.handle = handle
        self.dims = [int(i) for i in dims]
        self.rank = int(rank)
        self.loss = loss
        self.dtype = dtype
        self.stream = stream
        self._num_params = None

    # ------------------------------------------------------------ life
    def close(self):
        if self.handle:
            load().gcp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_params(self):
        """sum_k I_k * R, fixed for the context's life (asked once)."""
        if self._num_params is None:
            self._num_params = int(load().gcp_num_params(self.handle))
        return self._num_params

    @property
    def nnz(self):
        return int(load().gcp_nnz(self.handle))

    # --------------------------------------------------------- factors
    def set_factors(self, factors):
        """factors: flat FP32 tensor/array (host or device) or a list of
        per-mode I_k x R matrices."""
        import torch

        if isinstance(factors, (list, tuple)):
            if len(factors) != len(self.dims):
                raise ValueError(f"expected {len(self.dims)} factor matrices, got {len(factors)}")
            staged = []
            ptrs = (ctypes.c_void_p * len(factors))()
            for k, a in enumerate(factors):
                if isinstance(a, np.ndarray):
                    a = np.ascontiguousarray(a, dtype=np.float32)
                else:
                    a = a.detach().to(torch.float32).contiguous()
                if tuple(a.shape) != (self.dims[k], self.rank):
                    raise ValueError(f"factor {k} has shape {tuple(a.shape)}, expected {(self.dims[k], self.rank)}")
                ptrs[k] = _ptr(a)
                staged.append(a)
            _check(load().gcp_set_factor_list(self.handle, ptrs), self.handle)
            self.sync()  # the copies have run: the staged arrays may go
            return
        a = factors
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=np.float32)
        _check_buf(a, self.num_params, "float32", "factors")
        _check(load().gcp_set_factors(self.handle, _ptr(a)), self.handle)
        self.sync()

    def get_factors(self):
        """FP32 master factors as a list of host numpy I_k x R arrays."""
        out = np.zeros(self.num_params, dtype=np.float32)
        _check(load().gcp_get_factors(self.handle, out.ctypes.data), self.handle)
        res, o = [], 0
        for I in self.dims:
            res.append(out[o:o + I * self.rank].reshape(I, self.rank))
            o += I * self.rank
        return res

    def reset_adam(self):
        _check(load().gcp_reset_adam(self.handle), self.handle)

    # ---------------------------------------------------------- compute
    def sample(self, iter, p, q, device="cuda"):
        """(idx [(p+q) x d] int32, x [p+q] f32, w [p+q] f32) as device tensors."""
        import torch

        S = p + q
        idx = torch.empty((S, len(self.dims)), dtype=torch.int32, device=device)
        x = torch.empty(S, dtype=torch.float32, device=device)
        w = torch.empty(S, dtype=torch.float32, device=device)
        _check(load().gcp_sample(self.handle, iter, p, q, _ptr(idx), _ptr(x), _ptr(w)), self.handle)
        self.sync()
        return idx, x, w

    def loss_value(self, iter, p, q):
        out = ctypes.c_double(0.0)
        _check(load().gcp_loss(self.handle, iter, p, q, ctypes.byref(out)), self.handle)
        return out.value

    def grad(self, iter, p, q, G_out=None, want_loss=True):
        """Sampled gradient; returns (loss or None, G_out)."""
        _check_buf(G_out, self.num_params, "float32", "G_out")
        out = ctypes.c_double(0.0)
        _check(load().gcp_grad(self.handle, iter, p, q, _ptr(G_out), ctypes.byref(out) if want_loss else None),
               self.handle)
        return (out.value if want_loss else None), G_out

    def grad_async(self, iter, p, q, dscale=None, G_out=None, dloss=None):
        _check_buf(dscale, 1, "float32", "dscale")
        _check_buf(G_out, self.num_params, "float32", "G_out")
        _check_buf(dloss, 1, "float64", "dloss")
        _check(load().gcp_grad_async(self.handle, iter, p, q, _ptr(dscale), _ptr(G_out), _ptr(dloss)),
               self.handle)

    def scale_async(self, dscale, x, y):
        """y = dscale[0] * x on the context's stream (device tensors; dscale
        holds one FP64 value)."""
        _check_buf(dscale, 1, "float64", "dscale")
        _check_buf(x, 0, "float32", "x")
        _check_buf(y, x.numel(), "float32", "y")
        _check(load().gcp_scale_async(self.handle, _ptr(dscale), _ptr(x), _ptr(y), x.numel()), self.handle)

    def loss_async(self, iter, p, q, dloss):
        _check_buf(dloss, 1, "float64", "dloss")
        _check(load().gcp_loss_async(self.handle, iter, p, q, _ptr(dloss)), self.handle)

    def grad_norm(self):
        """||G||_F of the gradient the context holds, in FP64 (synchronises)."""
        v = ctypes.c_double(0.0)
        _check(load().gcp_grad_norm(self.handle, ctypes.byref(v)), self.handle)
        return v.value

    def adam_step(self, prm: AdamParams, t: int):
        c = prm.c()
        _check(load().gcp_adam_step(self.handle, ctypes.byref(c), t), self.handle)

    def step(self, iter, p, q, prm: AdamParams, t: int, dloss=None):
        """Sampled gradient + Adam step t in one call (G is cleared after)."""
        _check_buf(dloss, 1, "float64", "dloss")
        c = prm.c()
        _check(load().gcp_step(self.handle, iter, p, q, ctypes.byref(c), t, _ptr(dloss)), self.handle)

    def sync(self):
        _check(load().gcp_sync(self.handle), self.handle)

    def profile(self, enable=True):
        _check(load().gcp_profile(self.handle, int(enable)), self.handle)

    def profile_read(self):
        """(summed fused-kernel milliseconds, launches) since the last read."""
        ms, n = ctypes.c_double(0.0), ctypes.c_int64(0)
        _check(load().gcp_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n)), self.handle)
        return ms.value, n.value

    def fit(self, adam: AdamParams, p, q, p_obj, q_obj, iters=100, max_epochs=100, max_fails=3, decay=0.1,
            iter0=0):
        prm = gcp_fit_params(adam.c(), p, q, p_obj, q_obj, iters, max_epochs, max_fails, 0, decay, iter0)
        rep = gcp_fit_report()
        _check(load().gcp_fit(self.handle, ctypes.byref(prm), ctypes.byref(rep)), self.handle)
        d = {f: getattr(rep, f) for f, _ in gcp_fit_report._fields_ if f != "trace"}
        d["trace"] = list(rep.trace)[: rep.epochs]
        return d


def _options(dtype, mttkrp, sampling, seed, stream, max_attempts, hash_max_load, lane_cols=0):
    opt = gcp_options()
    load().gcp_options_default(ctypes.byref(opt))
    opt.factor_dtype = DTYPES[dtype]
    opt.mttkrp = MTTKRP[mttkrp]
    opt.sampling = SAMPLING[sampling]
    opt.seed = seed
    opt.stream = _stream_handle(stream)
    opt.max_attempts = max_attempts
    opt.hash_max_load = hash_max_load
    opt.lane_cols = lane_cols
    return opt


def gcp_create(dims, coords, vals, rank, loss, dtype="fp32", mttkrp="atomic", sampling="stratified", seed=0,
               stream=None, max_attempts=64, hash_max_load=0.3, lane_cols=0) -> GcpContext:
    """Sparse tensor context: coords (nnz x d int32) and vals (nnz float32) on the host."""
    lib = load()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    c = np.ascontiguousarray(coords, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.float32)
    opt = _options(dtype, mttkrp, sampling, seed, stream, max_attempts, hash_max_load, lane_cols)
    h = ctypes.c_void_p()
    rc = lib.gcp_create(len(d), d.ctypes.data, len(v), c.ctypes.data, v.ctypes.data, rank, LOSSES[loss],
                        ctypes.byref(opt), ctypes.byref(h))
    _check(rc, None)
    return GcpContext(h.value, d, rank, loss, dtype, stream)


def gcp_create_dense(dims, X, rank, loss, dtype="fp32", seed=0, stream=None, lane_cols=0) -> GcpContext:
    """Dense tensor context; X is a host numpy array or a device tensor."""
    lib = load()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    if isinstance(X, np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
    _check_buf(X, int(np.prod(d, dtype=np.float64)), "float32", "X")
    opt = _options(dtype, "atomic", "uniform", seed, stream, 64, 0.3, lane_cols)
    h = ctypes.c_void_p()
    _check(lib.gcp_create_dense(len(d), d.ctypes.data, _ptr(X), rank, LOSSES[loss], ctypes.byref(opt),
                                ctypes.byref(h)), None)
    return GcpContext(h.value, d, rank, loss, dtype, stream)


class GcpBatch:
    """Many client contexts advanced together (one multi-client launch per
    kernel, tau local steps in one CUDA graph)."""

    def __init__(self, clients, p, q):
        lib = load()
        self.clients = list(clients)  # keep the contexts alive
        arr = (ctypes.c_void_p * len(self.clients))(*[c.handle for c in self.clients])
        pp = np.ascontiguousarray(p, dtype=np.int64).reshape(-1)
        qq = np.ascontiguousarray(q, dtype=np.int64).reshape(-1)
        if len(pp) != len(self.clients) or len(qq) != len(self.clients):
            raise ValueError("p and q need one entry per client")
        h = ctypes.c_void_p()
        rc = lib.gcp_batch_create(len(self.clients), ctypes.cast(arr, ctypes.c_void_p), pp.ctypes.data,
                                  qq.ctypes.data, ctypes.byref(h))
        if rc != GCP_OK:
            raise GcpError(rc, lib.gcp_batch_last_error(None).decode())
        self.handle = h.value
        self.p, self.q = pp, qq

    def _check(self, rc):
        if rc != GCP_OK:
            raise GcpError(rc, load().gcp_batch_last_error(self.handle).decode())

    def tune(self, lane_cols=0, blocks=0, samples_per_warp=None):
        """Knobs of the multi-client fused kernel: factor columns per lane,
        persistent grid size (0 = all resident blocks) and, if given,
        samples per warp tile (16, 32 or 64)."""
        if samples_per_warp is not None:
            self._check(load().gcp_batch_tune_tile(self.handle, samples_per_warp))
        self._check(load().gcp_batch_tune(self.handle, lane_cols, blocks))

    def local_steps(self, tau, adam: AdamParams, iter0, t0):
        c = adam.c()
        self._check(load().gcp_batch_local_steps(self.handle, tau, ctypes.byref(c), iter0, t0))

    def server_init(self):
        """GCP-FedAdam: server model = client 0's factors, broadcast to all."""
        self._check(load().gcp_batch_server_init(self.handle))

    def server_step(self, adam: AdamParams, t: int):
        """GCP-FedAdam reconciliation (Alg. 4) with the server Adam step t."""
        c = adam.c()
        self._check(load().gcp_batch_server_step(self.handle, ctypes.byref(c), t))

    def losses(self):
        out = np.zeros(len(self.clients), dtype=np.float64)
        self._check(load().gcp_batch_losses(self.handle, out.ctypes.data))
        return out

    def close(self):
        if self.handle:
            load().gcp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gcp_grad_samples_noalloc(dims, rank, loss, idx, x, w, A, G, loss_out, stream=None):
    """Loss and gradient of a given sample list with no device allocation
    (for callers that cannot allocate).  idx/x/w/A/G/loss_out are device
    tensors; loss_out holds 2 doubles (loss, skipped samples).  Asynchronous."""
    import torch

    d = np.ascontiguousarray(dims, dtype=np.int64)
    S = int(idx.shape[0])
    if idx.dtype != torch.int32 or tuple(idx.shape) != (S, len(d)) or not idx.is_contiguous():
        raise ValueError(f"idx must be a contiguous int32 tensor of shape (nsamples, {len(d)})")
    nparam = int(d.sum()) * int(rank)
    _check_buf(x, S, "float32", "x")
    _check_buf(w, S, "float32", "w")
    _check_buf(A, nparam, "float32", "A")
    _check_buf(G, nparam, "float32", "G")
    _check_buf(loss_out, 2, "float64", "loss_out")
    _check(load().gcp_grad_samples_noalloc(len(d), d.ctypes.data, rank, LOSSES[loss], int(idx.shape[0]), _ptr(idx),
                                           _ptr(x), _ptr(w), _ptr(A), _ptr(G), _ptr(loss_out),
                                           _stream_handle(stream)), None)


PROBES = {"red": 0, "load": 1, "both": 2}


def gcp_probe_l2(kind, buf, row_floats, rows_per_op, ops, stream=None):
    """Row traffic of the fused pass's pattern on an L2-resident buffer
    (measurement support): `ops` groups of row_floats/4 lanes each reduce
    into ("red"), read ("load") or read then reduce ("both") rows_per_op
    random rows of buf, a device float32 tensor of rows x row_floats.
    Asynchronous on `stream`; the caller times it."""
    if buf.numel() % row_floats:
        raise ValueError("buf must hold whole rows of row_floats floats")
    _check_buf(buf, buf.numel(), "float32", "buf")
    rows = buf.numel() // row_floats
    _check(load().gcp_probe_l2(PROBES[kind], row_floats, rows_per_op, _ptr(buf), rows, int(ops),
                               _stream_handle(stream)), None)


# C-named conveniences over a context
def gcp_sample(ctx: GcpContext, iter, p, q):
    return ctx.sample(iter, p, q)


def gcp_loss(ctx: GcpContext, iter, p, q):
    return ctx.loss_value(iter, p, q)


def gcp_grad(ctx: GcpContext, iter, p, q, G_out=None):
    return ctx.grad(iter, p, q, G_out)


def gcp_adam_step(ctx: GcpContext, prm: AdamParams, t):
    return ctx.adam_step(prm, t)


def gcp_fit(ctx: GcpContext, *a, **k):
    return ctx.fit(*a, **k)
