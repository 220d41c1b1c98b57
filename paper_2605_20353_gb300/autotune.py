"""Autotuner for the batched multi-client kernel.

The knobs are the factor columns each GPU lane owns (4 or 8; the rank
split of a sample across lanes), the samples each warp takes per tile (16,
32 or 64) and the size of the persistent grid (thread blocks, i.e. how
many tiles are in flight per SM).  Each candidate replays tau local steps
a few times; the fastest, by CUDA-event time on the clients' stream, is
kept.  Timing changes the clients' models, so callers tune on a scratch
copy of the batch (or accept the extra steps).
"""
from __future__ import annotations

import torch


def candidates(rank: int, sms: int, max_per_sm: int = 4, tiles=(16, 32, 64)):
    """(lane_cols, blocks, samples_per_warp) triples; blocks 0 = every block
    that fits on the GPU at once."""
    cols = [4, 8] if rank > 4 else [4]
    grids = sorted({sms * k for k in range(1, max_per_sm + 1)} | {0})
    return [(c, g, t) for t in tiles for c in cols for g in grids]


def tune_batch(batch, adam, tau: int = 4, reps: int = 3, cands=None, stream=None):
    """Pick (lane_cols, blocks, samples_per_warp) for `batch`; returns
    (best, {candidate: ms per local step})."""
    stream = stream or torch.cuda.current_stream()
    if cands is None:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        cands = candidates(batch.clients[0].rank, sms)
    times = {}
    it = 1_000_000  # iteration numbers reserved for tuning
    for cols, blocks, ts in cands:
        batch.tune(cols, blocks, samples_per_warp=ts)
        batch.local_steps(tau, adam, it, 0)  # build the graph, warm up
        it += tau
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            batch.local_steps(tau, adam, it, 0)
            it += tau
        e1.record(stream)
        e1.synchronize()
        times[(cols, blocks, ts)] = e0.elapsed_time(e1) / (reps * tau)
    best = min(times, key=times.get)
    batch.tune(best[0], best[1], samples_per_warp=best[2])
    return best, times
