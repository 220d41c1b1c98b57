"""Benchmark of the stochastic GCP gradient step on GB300.

Workload: a 4-way sparse count tensor 2000 x 1500 x 1000 x 200 with 5e7
distinct nonzeros whose coordinates follow per-mode Zipf(1.1) marginals,
values 1 + Poisson(3), Poisson loss, rank 32, FP32 factors, 2^20 nonzero +
2^20 zero samples per gradient.  One step = one fused sampled gradient
(sampling, model, loss, all-mode MTTKRP) plus one Adam update, through the
C ABI.  The metric is gradient samples per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica (the path
does not shard); value = all ranks' samples / the slowest rank's time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCP gradient samples/s & % HBM peak; BF16/batched vs plain FP32 at rel-err≤5e-3"
WORKLOAD = ("zipf-count 4-way 2000x1500x1000x200, 5e7 nnz Zipf(1.1) coords, 1+Poisson(3) values, "
            "Poisson loss, rank 32, p=q=2^20 stratified samples")
# what stays resident where; both arms print the same config
L2_NOTE = ("inputs larger than L2 (1.6 GB records, 2.1 GB hash set); factors and gradient (0.6 MB each) stay "
           "L2-resident across steps as in training")
CONFIG = {"workload": WORKLOAD, "l2": L2_NOTE}
KERNEL_SOURCES = ["paper_2605_20353_gb300/csrc/gcp_kernels.cu", "paper_2605_20353_gb300/csrc/gcp_device.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_grad_zipf_count_traffic.json")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload(nnz=None):
    import synth

    if nnz:
        return synth.cached(f"zipf_count_nnz{int(nnz)}", lambda: synth.workload_zipf_count(nnz=nnz))
    return synth.cached("zipf_count_full", lambda: synth.workload_zipf_count(scale=1.0))


def algorithmic_bytes_per_sample(d, R, nnz, M, elt_bytes):
    """Bytes one sample must move by the definition of the step: a nonzero
    reads its d coordinates and value (4(d+1) B); a zero reads one 32-byte
    hash bucket per rejection attempt (expected 1/(1-N/M)); both gather d
    factor rows (elt_bytes R each) and add d gradient rows (4R each)."""
    attempts = 1.0 / (1.0 - nnz / M)
    rows = d * R * (elt_bytes + 4)
    return 0.5 * (4 * (d + 1) + rows) + 0.5 * (32 * attempts + rows)


def compulsory_bytes_per_sample(d, R, nnz, M, rows, access_bytes=128, elt_bytes=4):
    """HBM bytes a sample cannot avoid when the model stays in L2: one
    random access for a nonzero's record, one per rejection attempt for a
    zero's hash bucket, plus the model (factors read, gradient read and
    written once per step: rows x R x 3 x 4 B) spread over the step's 2^21
    samples.  On this GPU a random access that misses L2 moves a whole
    128-byte DRAM line whatever its width (`bench.py --only dramprobe`
    under ncu: 124 B of DRAM reads per random 16-128 B access);
    access_bytes=32 gives the 32-byte-sector reading instead."""
    attempts = 1.0 / (1.0 - nnz / M)
    return 0.5 * access_bytes + 0.5 * access_bytes * attempts + rows * R * (elt_bytes + 8) / float(1 << 21)


# the fused pass's part of gcp_kernels.cu ends where the replica fold begins
FUSED_SECTION_END = b"// G(hot row) += sum over replicas"


def kernel_source_hash():
    """Hash of the fused kernel's source: the device header and the part of
    gcp_kernels.cu up to the replica fold (the whole file if that marker
    moved), so that edits to other kernels keep the captured counters."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            text = fh.read()
        if f.endswith("gcp_kernels.cu") and FUSED_SECTION_END in text:
            text = text[:text.index(FUSED_SECTION_END)]
        h.update(text)
    return h.hexdigest()[:16]


def measured_traffic(key="dram_bytes_per_launch"):
    """A per-launch byte count from the committed ncu capture of the fused
    kernel, or None once the kernel sources have changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        if t.get("kernel_sha") == kernel_source_hash():
            return t[key]
    except (OSError, ValueError, KeyError):
        pass
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (read-only
    queries, via ctypes) every `period` seconds from a thread while running.
    The timed loop of the benchmark lasts a few milliseconds, shorter than
    nvidia-smi's sampling interval; this reader samples inside it.  `ok` is
    False where NVML or the device cannot be found."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}
    NVML_CLOCK_SM = 1

    def __init__(self, device, period=0.0005):
        self.device = device
        self.period = period
        self.ok = False
        self.samples = []
        self.max_mhz = None

    def _open(self):
        import ctypes
        import threading
        import torch

        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            return False
        self.nv, self.ct = nv, ctypes
        h = ctypes.c_void_p()
        uuid = str(torch.cuda.get_device_properties(self.device).uuid)
        found = False
        for u in (uuid, "GPU-" + uuid):
            if nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0:
                found = True
                break
        if not found:
            return False
        self.h = h
        mx = ctypes.c_uint()
        if nv.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        self.reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)
        return True

    def _run(self):
        ct = self.ct
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, self.NVML_CLOCK_SM, ct.byref(clk)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(self.period)

    def __enter__(self):
        try:
            self.ok = self._open()
        except (OSError, AttributeError, RuntimeError):
            self.ok = False
        if self.ok:
            self.thread.start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 1.0:  # running before the loop starts
                time.sleep(self.period)
        return self

    def __exit__(self, *a):
        if self.ok:
            self.stop.set()
            self.thread.join(timeout=2)
            self.nv.nvmlShutdown()

    def summary(self):
        sm = [c for c, _ in self.samples]
        reasons = sorted({n for _, r in self.samples for bit, n in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": self.max_mhz if self.max_mhz else (max(sm) if sm else None),
                "reasons": reasons, "samples": len(sm), "source": "nvml, every 0.5 ms"}


class ClockRecord:
    """Clocks during a timed region: NVML when it can be read, else
    nvidia-smi every 20 ms."""

    def __init__(self, device):
        self.device = device

    def __enter__(self):
        self.src = NvmlClocks(self.device).__enter__()
        if not self.src.ok:
            self.src = ClockSampler(self.device).__enter__()
        return self

    def __exit__(self, *a):
        self.src.__exit__(*a)

    def summary(self):
        return self.src.summary()


class ClockSampler:
    """nvidia-smi clock/throttle samples every 20 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, every 20 ms"}


def cpu_oracle_rate(w, skeys, n_samples, seed=3002, t=5):
    """Oracle samples/s on n_samples of the workload (half nonzero, half zero)."""
    import oracle

    p = n_samples // 2
    q = n_samples - p
    t0 = time.perf_counter()
    idx, x, wt, _ = oracle.stratified_samples(seed, t, p, q, w["dims"], w["coords"], w["vals"], skeys=skeys)
    oracle.sampled_loss_grad(w["dims"], w["factors"], w["loss"], idx, x, wt)
    return n_samples / (time.perf_counter() - t0)


_POOL_W = None


def _pool_init(paths):
    """Spawned oracle worker: map the workload's arrays read-only (shared
    page cache, no per-worker copy)."""
    global _POOL_W
    import numpy as np

    _POOL_W = {k: np.load(v, mmap_mode="r") for k, v in paths.items()}


def _pool_task(task):
    """One worker's share: the oracle as it stands on n samples of iteration t."""
    import oracle

    seed, t, n, dims, factors, loss = task
    W = _POOL_W
    p = n // 2
    t0 = time.perf_counter()
    idx, x, wt, _ = oracle.stratified_samples(seed, t, p, n - p, dims, W["coords"], W["vals"], skeys=W["skeys"])
    oracle.sampled_loss_grad(dims, factors, loss, idx, x, wt)
    return n, time.perf_counter() - t0


class OraclePool:
    """The unmodified oracle on all host cores: `workers` spawned processes
    that map the workload's arrays read-only; run() gives each worker its own
    iteration's samples and returns (samples, wall seconds of the slowest)."""

    def __init__(self, w, skeys, workers, name="zipf_count_full"):
        import multiprocessing as mp

        import numpy as np

        self.w, self.workers = w, workers
        d = os.path.join(os.environ.get("GCP_CACHE_DIR") or os.path.join(ROOT, "_cache"), f"pool_{name}")
        os.makedirs(d, exist_ok=True)
        paths = {}
        for k, a in (("coords", w["coords"]), ("vals", w["vals"]), ("skeys", skeys)):
            paths[k] = os.path.join(d, k + ".npy")
            if not os.path.exists(paths[k]):
                tmp = paths[k] + f".tmp{os.getpid()}.npy"
                np.save(tmp, np.ascontiguousarray(a))
                os.replace(tmp, paths[k])
        ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
        self.pool = ctx.Pool(workers, initializer=_pool_init, initargs=(paths,))
        self.run(256, 10_000)  # start-up and first page faults, untimed

    def run(self, n_per_worker, t0, seed=3002):
        w = self.w
        tasks = [(seed, t0 + i, n_per_worker, w["dims"], w["factors"], w["loss"]) for i in range(self.workers)]
        start = time.perf_counter()
        out = self.pool.map(_pool_task, tasks, chunksize=1)
        return sum(n for n, _ in out), time.perf_counter() - start

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(w, target_s=10.0):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample."""
    import numpy as np

    import oracle

    skeys = oracle.sorted_keys(w["dims"], w["coords"])
    probe = cpu_oracle_rate(w, skeys, 1 << 14)
    n = int(min(w["p"] + w["q"], max(1 << 14, probe * target_s)))
    rate = cpu_oracle_rate(w, skeys, n)
    single = {"value": rate, "unit": "samples/s", "cores": 1, "kind": "oracle",
              "sample": f"{n} samples ({n // 2} nonzero + {n - n // 2} zero) of the same workload, "
                        f"sampling + FP64 loss + all-mode gradient, one thread"}
    cores = os.cpu_count() or 1
    if cores < 2:
        return single
    try:
        n_core = max(1 << 12, int(probe * target_s))
        pool = OraclePool(w, skeys, cores)
        try:
            done, wall = pool.run(n_core, 1000)
        finally:
            pool.close()
        all_rate = done / wall
    except Exception as e:  # report the one-thread figure rather than none
        single["all_cores_error"] = repr(e)[:200]
        return single
    return {"value": all_rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} spawned processes, each {n_core} samples ({n_core // 2} nonzero + "
                      f"{n_core - n_core // 2} zero) of its own iteration of the same workload; sampling + FP64 "
                      f"loss + all-mode gradient; total samples / wall time",
            "single_thread": single}


def run_reference(args):
    """The oracle arm: each step = the oracle on a bounded sample of the
    workload, sized so the whole run stays within a few minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    w = workload()
    skeys = oracle.sorted_keys(w["dims"], w["coords"])
    probe = cpu_oracle_rate(w, skeys, 1 << 12)
    cores = os.cpu_count() or 1
    # each step: every core runs the oracle on its share of a bounded sample,
    # sized so warm-up + timed steps take about 90 s in all
    per_core = max(64, int(probe * 90.0 / max(1, args.steps + args.warmup)))
    per_core = min(per_core, (w["p"] + w["q"]) // cores)
    pool = OraclePool(w, skeys, cores)
    try:
        for i in range(args.warmup):
            pool.run(per_core, 100 + 64 * i)
        done, dt = 0, 0.0
        for i in range(args.steps):
            n, s = pool.run(per_core, 1_000_000 + 64 * i)
            done += n
            dt += s
    finally:
        pool.close()
    per_step = done // args.steps
    value = done / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG),
            "step": {"what": "the FP64 oracle (stratified sampling, loss, all-mode gradient) on a bounded sample "
                             "of the workload, split over the host cores", "samples": per_step},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} samples per step of the same workload ({per_core} per core, "
                                       f"{cores} spawned processes, each on its own iteration)"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_rate(run, n0=1 << 12, target_s=4.0, cap=None):
    """Single-thread oracle samples/s: run(n) draws and differentiates n
    samples; a probe of n0 sizes one bounded run of about target_s seconds."""
    t = time.perf_counter()
    k = run(n0) or n0
    r = k / (time.perf_counter() - t)
    n = max(n0, int(r * target_s))
    if cap:
        n = min(n, cap)
    t = time.perf_counter()
    k = run(n) or n
    return {"value": k / (time.perf_counter() - t), "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} samples, one thread"}


def batched_variant(gcp, torch, stream, steps=20, with_oracle=True):
    """64 independent 3-way client shards (federated clients simulated on one
    GPU): mode sizes U{200..5000}, nnz log-uniform in [1e4, 2e6], values
    1+Poisson(2), Poisson loss, rank 16, BF16 factors, p_c = q_c =
    ceil(nnz_c / 8), tau = 8 local Adam steps per graph launch with autotuned
    tiles, against the same clients stepped by 64 sequential plain launches."""
    import synth
    from paper_2605_20353_gb300 import autotune

    shards = synth.cached("client_batch_64", lambda: synth.client_batch(64, 1005))
    tau = 8
    P = [math.ceil(len(v) / 8) for _, _, v in shards]
    samples_per_step = 2 * sum(P)
    adam = gcp.AdamParams(lr=1e-3, lower=0.0)

    def make(dtype):
        out = []
        for i, (dims, coords, vals) in enumerate(shards):
            c = gcp.gcp_create(dims, coords, vals, 16, "poisson", dtype=dtype, seed=5000 + i, stream=stream)
            c.set_factors(synth.factors_uniform(dims, 16, 6000 + i, lo=0.1, hi=1.0))
            out.append(c)
        return out

    res = {"workload": "64 clients, dims U{200..5000}^3, nnz log-uniform [1e4, 2e6], Poisson, rank 16",
           "samples_per_local_step": samples_per_step, "tau": tau}
    if with_oracle:
        import oracle

        skeys = [oracle.sorted_keys(dims, coords) for dims, coords, _ in shards]
        facs = [synth.factors_uniform(dims, 16, 6000 + i, lo=0.1, hi=1.0) for i, (dims, _, _) in enumerate(shards)]

        def run(n):  # about n samples over the clients in proportion to their p_c + q_c
            done = 0
            for i, (dims, coords, vals) in enumerate(shards):
                m = max(2, int(n * P[i] / sum(P)))
                idx, x, wt, _ = oracle.stratified_samples(5000 + i, 3, m // 2, m - m // 2, dims, coords, vals,
                                                          skeys=skeys[i])
                oracle.sampled_loss_grad(dims, facs[i], "poisson", idx, x, wt)
                done += m
            return done

        res["cpu_oracle"] = oracle_rate(run, n0=1 << 14)
    clients = make("bf16")
    batch = gcp.GcpBatch(clients, P, P)
    best, times = autotune.tune_batch(batch, adam, tau=tau, reps=2)
    res["autotune"] = {"best_lane_cols": best[0], "best_blocks": best[1], "best_samples_per_warp": best[2],
                       "ms_per_step": {f"cols{c}_blocks{g}_tile{t}": ms for (c, g, t), ms in times.items()}}
    batch.local_steps(tau, adam, 0, 0)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        batch.local_steps(tau, adam, (k + 1) * tau, (k + 1) * tau)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    res["batched_graph"] = {"value": samples_per_step * tau * steps / (ms / 1e3), "unit": "samples/s"}
    batch.close()
    for c in clients:
        c.close()
    # 64 sequential single-client steps: gcp_step (fused pass + one epilogue,
    # two launches per client, the best single-client path) and gradient +
    # Adam as separate calls (five launches per client)
    nseq = max(2, steps // 4)
    for form in ("step", "grad_adam"):
        for dtype in ("bf16", "fp32"):
            clients = make(dtype)
            for i, c in enumerate(clients):
                if form == "step":
                    c.step(0, P[i], P[i], adam, 1)
                else:
                    c.grad_async(0, P[i], P[i])
                    c.adam_step(adam, 1)
            stream.synchronize()
            e0.record(stream)
            for k in range(nseq * tau):
                for i, c in enumerate(clients):
                    if form == "step":
                        c.step(k + 1, P[i], P[i], adam, k + 2)
                    else:
                        c.grad_async(k + 1, P[i], P[i])
                        c.adam_step(adam, k + 2)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            key = f"sequential_{form}_{dtype}"
            res[key] = {"value": samples_per_step * tau * nseq / (ms / 1e3), "unit": "samples/s",
                        "launches_per_client_step": 2 if form == "step" else 5}
            for c in clients:
                c.close()
    for key in [k for k in res if k.startswith("sequential_")]:
        res["speedup_vs_" + key] = res["batched_graph"]["value"] / res[key]["value"]
    return res


def hbm_resident_variant(gcp, torch, stream, launches=20, dtypes=("fp32", "bf16"), ranks=(16, 32)):
    """Factors too large for L2: mode sizes near the paper's Amazon tensor
    (4.8M x 1.7M x 1.1M; its third mode is shortened from 1.8M so the cell
    count stays below 2^63), 2e7 uniform nonzeros with values 1+Poisson(2),
    Poisson loss, p = q = 2^20, ranks 16 and 32.  Gathers now come from HBM,
    so BF16 factor storage halves their bytes; fused-kernel time FP32 vs
    BF16.  HBM moves whole 64-byte atoms, so the halving only shows where a
    BF16 row is at least 64 bytes (rank 32)."""
    import numpy as np

    import synth

    dims = [4_800_000, 1_700_000, 1_100_000]

    def gen():
        coords, vals = synth.uniform_sparse(dims, 20_000_000, 1006, lam=2.0)
        return dict(coords=coords, vals=vals)

    w = synth.cached("hbm_resident_amazon_dims", gen)
    S = 1 << 20
    adam = gcp.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)
    res = {"workload": "4.8Mx1.7Mx1.1M, 2e7 uniform nnz, Poisson, p=q=2^20; rank 16 (factors 486 MB FP32) "
                       "and rank 32 (973 MB)"}
    for R in ranks:
        fac = synth.factors_uniform(dims, R, 2006, lo=0.1, hi=1.0)
        out = res if R == 16 else res.setdefault(f"rank{R}", {})
        for dtype in dtypes:
            ctx = gcp.gcp_create(dims, w["coords"], w["vals"], R, "poisson", dtype=dtype, seed=9, stream=stream)
            ctx.set_factors(fac)
            for i in range(3):
                ctx.grad_async(i, S, S)
            ctx.sync()
            ctx.profile(True)
            ctx.profile_read()
            for i in range(launches):
                ctx.grad_async(100 + i, S, S)
            kms, nl = ctx.profile_read()
            # the whole training step (gcp_step: fused pass + the epilogue
            # that streams every parameter through Adam), CUDA events
            for i in range(3):
                ctx.step(200 + i, S, S, adam, i + 1)
            ctx.profile_read()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(launches):
                ctx.step(300 + i, S, S, adam, 4 + i)
            e1.record(stream)
            e1.synchronize()
            step_ms = e0.elapsed_time(e1) / launches
            skms, snl = ctx.profile_read()
            ctx.profile(False)
            nparam = ctx.num_params
            ctx.close()
            per = kms / nl
            bps = algorithmic_bytes_per_sample(3, R, len(w["vals"]), float(np.prod(dims, dtype=np.float64)),
                                               4 if dtype == "fp32" else 2)
            epi_ms = step_ms - skms / max(1, snl)
            # epilogue bytes per parameter: G, A, B, C read; A, B, C written,
            # G cleared; the BF16 copy written when there is one
            epi_bytes = nparam * (32 + (2 if dtype == "bf16" else 0))
            out[dtype] = {"kernel_ms_per_launch": per, "samples_per_s": 2 * S / (per / 1e3),
                          "achieved_gbs": bps * 2 * S / (per / 1e3) / 1e9, "bytes_per_sample": bps,
                          "step_ms": step_ms, "step_samples_per_s": 2 * S / (step_ms / 1e3),
                          "epilogue_ms": epi_ms, "epilogue_bytes": epi_bytes,
                          "epilogue_gbs": epi_bytes / (epi_ms / 1e3) / 1e9 if epi_ms > 0 else None}
        if "fp32" in out and "bf16" in out:
            out["bf16_speedup"] = out["fp32"]["kernel_ms_per_launch"] / out["bf16"]["kernel_ms_per_launch"]
    return res


def fused_vs_nonfused_variant(gcp, torch, stream, launches=10):
    """The comparison of Sec. 5.1: fused vs non-fused sampling + MTTKRP with
    semi-stratified samples, on a synthetic tensor with the arXiv tensor's
    shape and nonzero count (172 x 25,000 x 300, 3e7 uniform nonzeros with
    values 1+Poisson(2)), Poisson loss, rank 16, p = q varied."""
    import synth

    dims = [172, 25000, 300]

    def gen():
        coords, vals = synth.uniform_sparse(dims, 30_000_000, 1007, lam=2.0)
        return dict(coords=coords, vals=vals)

    w = synth.cached("arxiv_shape_3e7", gen)
    fac = synth.factors_uniform(dims, 16, 2007, lo=0.1, hi=1.0)
    res = {"workload": "172x25000x300, 3e7 uniform nnz, Poisson, rank 16, semi-stratified", "points": []}
    ctxs = {m: gcp.gcp_create(dims, w["coords"], w["vals"], 16, "poisson", mttkrp=m, sampling="semi", seed=11,
                              stream=stream) for m in ("atomic", "nonfused")}
    for c in ctxs.values():
        c.set_factors(fac)
    for S in (1 << 16, 1 << 18, 1 << 20, 1 << 22):
        pt = {"p": S, "q": S}
        for m, c in ctxs.items():
            for i in range(2):
                c.grad_async(i, S, S)
            c.sync()
            c.profile(True)
            c.profile_read()
            for i in range(launches):
                c.grad_async(10 + i, S, S)
            kms, nl = c.profile_read()
            c.profile(False)
            pt["fused_ms" if m == "atomic" else "nonfused_ms"] = kms / nl
        pt["fused_speedup"] = pt["nonfused_ms"] / pt["fused_ms"]
        res["points"].append(pt)
    for c in ctxs.values():
        c.close()
    return res


def l2_flushed_variant(make, torch, p, q, launches=20):
    """The benchmark's fused launch timed alone, warm (factors and gradient
    rows left in L2 by the previous launch, as in training) and cold (L2
    flushed by writing 512 MiB just before each launch): medians of
    `launches` fused-kernel times from the library's own CUDA events."""
    ctx = make("fp32")
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    for i in range(3):
        ctx.grad_async(30_000 + i, p, q)
    ctx.sync()
    ctx.profile(True)
    ctx.profile_read()
    res = {}
    for mode in ("warm", "cold"):
        times = []
        for i in range(launches):
            if mode == "cold":
                flush.fill_(float(i))
            ctx.grad_async(40_000 + i, p, q)
            ms, n = ctx.profile_read()
            times.append(ms / max(1, n))
        res[f"{mode}_ms_median"] = statistics.median(times)
    ctx.profile(False)
    ctx.close()
    res["cold_over_warm"] = res["cold_ms_median"] / res["warm_ms_median"]
    res["workload"] = "the benchmark launch (2^21 samples); flush = 512 MiB written before each cold launch"
    return res


def l2_ceiling(gcp, torch, stream, d, Rp, S, reps=10, rows=1 << 15):
    """Measured ceiling of the fused pass's model traffic: the same number
    of row operations (S samples x d rows of Rp FP32 columns, each gathered
    and each reduced with red.v4) on uniformly random rows of a 4 MB
    L2-resident buffer, with no sampling, loss or hot rows.  Median of
    `reps` launches per kind, CUDA events on the launching stream."""
    buf = torch.zeros(rows * Rp, dtype=torch.float32, device="cuda")
    out = {"rows": rows, "row_bytes": 4 * Rp, "ops": S, "rows_per_op": d}
    for kind in ("red", "load", "both"):
        for _ in range(3):
            gcp.gcp_probe_l2(kind, buf, Rp, d, S, stream)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gcp.gcp_probe_l2(kind, buf, Rp, d, S, stream)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        nbytes = S * d * 4 * Rp * (2 if kind == "both" else 1)
        out[kind] = {"ms": ms, "gbs": nbytes / (ms / 1e3) / 1e9}
    del buf
    return out


def dram_access_cost(gcp, torch, stream, ops=1 << 21, gib=2):
    """Random row accesses that miss L2: gcp_probe_l2's row operations, one
    uniformly random row per op, on a 2 GiB buffer (16 times L2).  Rows of
    16, 32, 64 and 128 B are read and rows of 64 and 128 B reduced, 2^21
    ops each, one launch per kind; under ncu (dram__bytes_read.sum,
    dram__bytes_write.sum) the launches give the DRAM bytes that one random
    access of each width costs.  CUDA-event times are reported beside."""
    buf = torch.zeros(gib << 28, dtype=torch.float32, device="cuda")
    out = {"buffer_gib": gib, "ops": ops}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for kind, rf in (("load", 4), ("load", 8), ("load", 16), ("load", 32), ("red", 16), ("red", 32)):
        e0.record(stream)
        gcp.gcp_probe_l2(kind, buf, rf, 1, ops, stream)
        e1.record(stream)
        e1.synchronize()
        out[f"{kind}_{4 * rf}B_ms"] = e0.elapsed_time(e1)
    del buf
    return out


def combine_ranks(seconds, units_per_rank, world, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: every rank processed
    units_per_rank units; the job took as long as its slowest rank (max over
    ranks of the local timed seconds).  Returns (units per second, max s)."""
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return world * units_per_rank / slowest, slowest


def bernoulli_variant(gcp, torch, stream, launches=10, with_oracle=True):
    """10000 x 10000 x 1000 binary tensor with 2e7 ones from a rank-16
    logistic generator, Bernoulli-logit loss, rank 64, 2^21 ones + 2^21
    zeros: gradient time with FP32 / BF16 factors and atomic /
    deterministic MTTKRP."""
    import synth

    dims = [10000, 10000, 1000]

    def gen():
        coords, vals = synth.bernoulli_logit_sparse(dims, 20_000_000, 1004, rank=16)
        return dict(coords=coords, vals=vals)

    w = synth.cached("bernoulli_full_cv", gen)
    fac = synth.factors_normal(dims, 64, 2004, std=0.5)
    S = 1 << 21
    res = {"workload": "10000x10000x1000, 2e7 ones, Bernoulli-logit, rank 64, p=q=2^21"}
    if with_oracle:
        import oracle

        skeys = oracle.sorted_keys(dims, w["coords"])

        def run(n):
            idx, x, wt, _ = oracle.stratified_samples(7, 5, n // 2, n - n // 2, dims, w["coords"], w["vals"],
                                                      skeys=skeys)
            oracle.sampled_loss_grad(dims, fac, "bernoulli", idx, x, wt)

        res["cpu_oracle"] = oracle_rate(run)
        del skeys
    for name, dtype, mttkrp in (("fp32_atomic", "fp32", "atomic"), ("bf16_atomic", "bf16", "atomic"),
                                ("fp32_deterministic", "fp32", "deterministic")):
        ctx = gcp.gcp_create(dims, w["coords"], w["vals"], 64, "bernoulli", dtype=dtype, mttkrp=mttkrp, seed=7,
                             stream=stream)
        ctx.set_factors(fac)
        ctx.grad_async(0, S, S)
        ctx.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(launches):
            ctx.grad_async(1 + i, S, S)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / launches
        res[name] = {"gradient_ms": ms, "samples_per_s": 2 * S / (ms / 1e3)}
        ctx.close()
    # the same row traffic (3 rows of 256 B gathered and reduced per sample)
    # alone on an L2-resident buffer: the atomic gradient's measured ceiling
    ceil = l2_ceiling(gcp, torch, stream, 3, 64, 2 * S, reps=5)
    res["l2_rows_probe_ms"] = ceil["both"]["ms"]
    res["fp32_atomic"]["l2_rows_frac"] = ceil["both"]["ms"] / res["fp32_atomic"]["gradient_ms"]
    return res


def autograd_variant(gcp, torch, stream, steps=10, with_oracle=True):
    """Dense 100x100x100x20x50 FP32 tensor (rank-8 sinusoidal CP signal +
    N(0, 0.1^2) noise), Gaussian loss, rank 16, 2^22 uniform samples:
    forward (sampled loss and, in the same fused pass, the gradient) +
    backward (the gradient scaled by the incoming one) through the autograd
    function."""
    import synth
    from paper_2605_20353_gb300 import autograd

    dims = [100, 100, 100, 20, 50]
    X = synth.dense_cp_sinusoid(dims, 1003, rank_true=8, sigma=0.1)
    ctx = gcp.gcp_create_dense(dims, X, 16, "gaussian", seed=3003, stream=stream)
    fac = synth.factors_normal(dims, 16, 2003, std=0.5)
    cpu = None
    if with_oracle:
        import oracle

        def run(n):
            idx, x, wt = oracle.uniform_samples(3003, 5, n, dims, X)
            oracle.sampled_loss_grad(dims, fac, "gaussian", idx, x, wt)

        cpu = oracle_rate(run)
    del X
    A = [torch.tensor(a, device="cuda", requires_grad=True) for a in fac]
    s = 1 << 22
    loss = autograd.sampled_loss(ctx, 0, s, 0, A)
    loss.backward()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h0 = time.perf_counter()
    for i in range(steps):
        for a in A:
            a.grad = None
        loss = autograd.sampled_loss(ctx, 1 + i, s, 0, A)
        loss.backward()
    host_ms = (time.perf_counter() - h0) * 1e3 / steps  # host time to issue one iteration
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the other split: loss-only forward, MTTKRP adjoint in the backward
    for i in range(2):
        loss = autograd.sampled_loss(ctx, 50 + i, s, 0, A, grad_in_forward=False)
        loss.backward()
    e0.record(stream)
    for i in range(steps):
        for a in A:
            a.grad = None
        loss = autograd.sampled_loss(ctx, 60 + i, s, 0, A, grad_in_forward=False)
        loss.backward()
    e1.record(stream)
    e1.synchronize()
    ms_adjoint = e0.elapsed_time(e1) / steps
    # the fused pass's own time, from the library's events, in a second loop
    # (a first untimed one creates the events)
    ctx.profile(True)
    for rep in range(2):
        ctx.profile_read()
        for i in range(steps):
            for a in A:
                a.grad = None
            loss = autograd.sampled_loss(ctx, 100 + i, s, 0, A)
            loss.backward()
    kms, nl = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    # the fused pass's row traffic (5 rows of 64 B gathered and reduced per
    # sample) alone on an L2-resident buffer
    ceil = l2_ceiling(gcp, torch, stream, 5, 16, s, reps=5)
    fused_ms = kms / max(1, nl)
    out = {"workload": "dense 100x100x100x20x50, Gaussian, rank 16, 2^22 uniform samples",
           "forward_backward_ms": ms, "samples_per_s": s / (ms / 1e3), "host_issue_ms": host_ms,
           "forward_backward_ms_adjoint_in_backward": ms_adjoint,
           "fused_kernel_ms": fused_ms,
           "l2_rows_probe_ms": ceil["both"]["ms"], "l2_rows_frac": ceil["both"]["ms"] / fused_ms if nl else None}
    if cpu:
        out["cpu_oracle"] = cpu
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_2605_20353_gb300 as gcp
    from paper_2605_20353_gb300 import build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    gcp.load()
    if args.only:  # profiling captures: one variant alone
        stream = torch.cuda.current_stream()
        fn = {"batched": batched_variant, "hbm": hbm_resident_variant, "nonfused": fused_vs_nonfused_variant,
              "bernoulli": bernoulli_variant, "autograd": autograd_variant, "dramprobe": dram_access_cost}.get(args.only)
        if args.only == "l2probe":
            res = l2_ceiling(gcp, torch, stream, 4, 32, 1 << 21)
        else:
            kw = {"dtypes": (args.dtype,)} if args.only == "hbm" else {}
            if args.only in ("batched", "bernoulli", "autograd"):
                kw["with_oracle"] = False
            res = fn(gcp, torch, stream, **kw)
        print(json.dumps({"variant": args.only, **res}), flush=True)
        return
    if rank == 0:
        w = workload(args.nnz)
    if dist:
        dist.barrier()
    if rank != 0:
        w = workload(args.nnz)
    dims, R, p, q = w["dims"], w["rank"], w["p"], w["q"]
    S = p + q
    stream = torch.cuda.current_stream()

    def make(dtype):
        ctx = gcp.gcp_create(dims, w["coords"], w["vals"], R, "poisson", dtype=dtype, seed=3002 + rank,
                             stream=stream)
        ctx.set_factors(w["factors"])
        return ctx

    adam = gcp.AdamParams(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)

    def timed_loop(ctx, steps, warmup, profile):
        if profile:  # one untimed pass creates the library's per-launch timing events
            ctx.profile(True)
            for i in range(steps):
                ctx.step(50_000 + i, p, q, adam, i + 1)
            ctx.profile_read()
            ctx.profile(False)
            ctx.set_factors(w["factors"])  # back to the starting state
            ctx.reset_adam()
        for i in range(warmup):
            ctx.step(10_000 + i, p, q, adam, i + 1)
        ctx.sync()
        if profile:
            ctx.profile(True)
            ctx.profile_read()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            ctx.step(i, p, q, adam, warmup + i + 1)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ctx.sync()
        ms = e0.elapsed_time(e1)
        kms, nl = ctx.profile_read() if profile else (0.0, 0)
        ctx.profile(False)
        return ms, kms, nl

    if args.kernel_only:  # profiling captures: the timed loop of one variant only
        ctx = make(args.dtype)
        ms, kernel_ms, launches = timed_loop(ctx, args.steps, args.warmup, profile=True)
        log(f"kernel-only {args.dtype}: {kernel_ms / max(1, launches):.4f} ms per fused launch")
        ctx.close()
        return
    ctx = make("fp32")
    with ClockRecord(local) as clk:
        ms, _, _ = timed_loop(ctx, args.steps, args.warmup, profile=False)
    clocks = clk.summary()
    # the fused kernel's launch duration: the same K steps again, each fused
    # launch between the library's timing events.  Those events cost about
    # 4 us per step, so the throughput loop above runs without them.
    ctx.set_factors(w["factors"])
    ctx.reset_adam()
    ms_events, kernel_ms, launches = timed_loop(ctx, args.steps, args.warmup, profile=True)
    value, slowest_s = combine_ranks(ms / 1e3, S * args.steps, world, dist, device="cuda")
    ms = slowest_s * 1e3
    ms_per_step = ms / args.steps

    # end to end through the public API with host buffers, the same step as
    # `value` (gcp_step): every step the factors come in from pinned host
    # memory and the host reads the step's loss (8 B back).  The host reads
    # step i's loss after it has issued step i + 1, as a training loop that
    # logs its losses does, so the GPU does not wait on the host between steps
    n_e2e = max(3, min(args.steps, 200))
    A_host = torch.from_numpy(np.concatenate([a.ravel() for a in w["factors"]])).pin_memory()
    dl = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(2)]
    dl_host = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def e2e_issue(i):
        assert gcp.load().gcp_set_factors(ctx.handle, A_host.data_ptr()) == 0
        ctx.step(i, p, q, adam, i + 1, dloss=dl[i % 2])
        dl_host[i % 2].copy_(dl[i % 2], non_blocking=True)
        done[i % 2].record(stream)

    def e2e_read(i):
        done[i % 2].synchronize()
        return dl_host[i % 2].item()

    def e2e_loop(first, n):
        losses = []
        for i in range(first, first + n):
            e2e_issue(i)
            if i > first:
                losses.append(e2e_read(i - 1))
        losses.append(e2e_read(first + n - 1))
        return losses

    e2e_loop(20_000, 3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_losses = e2e_loop(0, n_e2e)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    assert len(e2e_losses) == n_e2e and all(math.isfinite(v) for v in e2e_losses)
    e2e_value, _ = combine_ranks(e2e_s, S * n_e2e, world, dist, device="cuda")
    # the same with the whole gradient out instead (gcp_grad to pinned host
    # memory, then gcp_adam_step): the gradient API's round trip
    G_host = torch.empty(ctx.num_params, dtype=torch.float32).pin_memory()
    for i in range(3):
        ctx.set_factors(A_host.numpy())
        ctx.grad(20_000 + i, p, q, G_out=G_host)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        assert gcp.load().gcp_set_factors(ctx.handle, A_host.data_ptr()) == 0
        ctx.grad(i, p, q, G_out=G_host)
        ctx.adam_step(adam, i + 1)
    torch.cuda.synchronize()
    e2e_g_value, _ = combine_ranks(time.perf_counter() - t0, S * n_e2e, world, dist, device="cuda")
    ctx.close()

    # BF16 factor storage, same workload
    ctx_bf = make("bf16")
    ms_bf, _, _ = timed_loop(ctx_bf, max(3, args.steps // 2), args.warmup, profile=False)
    ctx_bf.set_factors(w["factors"])
    ctx_bf.reset_adam()
    _, kms_bf, nl_bf = timed_loop(ctx_bf, max(3, args.steps // 2), args.warmup, profile=True)
    ctx_bf.close()
    bf16_value = S * max(3, args.steps // 2) / (ms_bf / 1e3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    bps = algorithmic_bytes_per_sample(4, R, len(w["vals"]), float(np.prod(dims, dtype=np.float64)), 4)
    bps_bf = algorithmic_bytes_per_sample(4, R, len(w["vals"]), float(np.prod(dims, dtype=np.float64)), 2)
    kernel_avg_s = kernel_ms / 1e3 / launches
    # The binding resource: the factor and gradient rows are L2-resident, so
    # the fused pass is bound by its row traffic between the SMs and L2
    # (d = 4 rows of 128 B gathered and 4 reduced per sample).  Its ceiling
    # is the same row operations alone on uniformly random rows of an
    # L2-resident buffer (gcp_probe_l2), measured in this run.
    ceil = l2_ceiling(gcp, torch, stream, 4, 32, S)
    row_bytes = 2 * S * 4 * 32 * 4
    achieved = row_bytes / kernel_avg_s / 1e9
    dram = measured_traffic()
    compulsory = compulsory_bytes_per_sample(4, R, len(w["vals"]), float(np.prod(dims, dtype=np.float64)),
                                             sum(dims))
    sector_bytes = compulsory_bytes_per_sample(4, R, len(w["vals"]), float(np.prod(dims, dtype=np.float64)),
                                               sum(dims), access_bytes=32)
    roofline = {"bound": "l2", "achieved": achieved, "peak": ceil["both"]["gbs"], "unit": "GB/s",
                "frac": achieved / ceil["both"]["gbs"], "traffic": dram, "kernel": "k_fused<4,float,4>",
                "kernel_ms_per_launch": kernel_avg_s * 1e3,
                "kernel_timing": "CUDA events around each fused launch on the context's stream, over a second "
                                 f"pass of the same {args.steps} timed steps (that pass: "
                                 f"{ms_events / args.steps:.4f} ms per step; the events cost a few us per step, "
                                 "so the throughput loop runs without them)",
                "what": "fused pass's factor-row gathers + gradient-row reductions (4 rows of 128 B each per sample) "
                        "per launch / its CUDA-event time, against the same row operations alone on uniformly "
                        "random rows of an L2-resident buffer (gcp_probe_l2, measured in this run: a builder-"
                        "measured ceiling, not a driver peak); traffic = ncu DRAM bytes per launch",
                "peak_source": "gcp_probe_l2 'both' rate, this run",
                "reductions": {"achieved": row_bytes / 2 / kernel_avg_s / 1e9, "peak": ceil["red"]["gbs"],
                               "frac": (row_bytes / 2 / kernel_avg_s / 1e9) / ceil["red"]["gbs"]},
                "probe": ceil,
                # HBM: what the kernel moves through DRAM (ncu bytes per launch
                # over the live kernel time), against the measured copy peak
                "hbm": {"achieved": dram / kernel_avg_s / 1e9 if dram else None, "peak": peak, "unit": "GB/s",
                        "frac": dram / kernel_avg_s / 1e9 / peak if dram else None,
                        "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                        "dram_bytes_per_sample": dram / S if dram else None,
                        "compulsory_bytes_per_sample": compulsory,
                        "compulsory_note": "one 128-B DRAM line per random record or bucket access (measured "
                                           "granularity of this GPU) + the model amortised over the step",
                        "dram_over_compulsory": dram / S / compulsory if dram else None,
                        "sector_bytes_per_sample": sector_bytes},
                # the scope table's logical bytes (record or bucket, gathers,
                # reductions) over the kernel time: most are served by L2, so
                # this is not an HBM fraction
                "logical": {"bytes_per_sample": bps, "achieved": bps * S / kernel_avg_s / 1e9, "unit": "GB/s",
                            "over_hbm_peak": bps * S / kernel_avg_s / 1e9 / peak}}
    base = cpu_baseline(w)
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(CONFIG),
            "step": {"what": "gcp_step: fused sampled gradient (sampling, model, loss, all-mode MTTKRP) + one "
                             "epilogue (loss finish, replica fold, Adam)", "samples": S,
                     "parallelism": f"replicas{world}"},
            "roofline": roofline, "cpu_baseline": base,
            "e2e": {"value": e2e_value, "unit": "samples/s", "h2d_bytes_per_step": int(A_host.numel() * 4),
                    "d2h_bytes_per_step": 8,
                    "what": "gcp_step per step with the factors copied in from pinned host memory and the "
                            "loss read back by the host (step i's loss read once step i + 1 is issued)",
                    "gradient_out": {"value": e2e_g_value, "unit": "samples/s",
                                     "h2d_bytes_per_step": int(A_host.numel() * 4),
                                     "d2h_bytes_per_step": int(G_host.numel() * 4 + 8),
                                     "what": "gcp_grad with the gradient and loss copied to pinned host "
                                             "memory, then gcp_adam_step"}},
            # per step (gcp_step): k_fused and the k_post_step epilogue
            "gpu_launches": 2 * args.steps, "clocks": clocks,
            "variants": {"bf16_factors": {"value": bf16_value, "unit": "samples/s",
                                          "kernel_ms_per_launch": kms_bf / max(1, nl_bf),
                                          "achieved_gbs": bps_bf * S / (kms_bf / 1e3 / max(1, nl_bf)) / 1e9}}}
    if not args.no_variants:
        line["variants"]["l2_warm_vs_flushed"] = l2_flushed_variant(make, torch, p, q)
        line["variants"]["batched_clients"] = batched_variant(gcp, torch, stream)
        line["variants"]["hbm_resident_factors"] = hbm_resident_variant(gcp, torch, stream)
        line["variants"]["fused_vs_nonfused"] = fused_vs_nonfused_variant(gcp, torch, stream)
        line["variants"]["bernoulli_binary"] = bernoulli_variant(gcp, torch, stream)
        line["variants"]["autograd_dense"] = autograd_variant(gcp, torch, stream)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nnz", type=float, default=None,
                    help="nonzero count of a smaller tensor of the same shape (profiling captures)")
    ap.add_argument("--kernel-only", action="store_true", help="time the step loop only (profiling)")
    ap.add_argument("--no-variants", action="store_true", help="skip the batched and HBM-resident variants")
    ap.add_argument("--only", default=None,
                    choices=["batched", "hbm", "nonfused", "bernoulli", "autograd", "l2probe", "dramprobe"],
                    help="run one variant alone (profiling captures)")
    ap.add_argument("--dtype", default="fp32", choices=["fp32", "bf16"], help="factor storage for --kernel-only")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
