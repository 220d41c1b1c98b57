"""The N > 1 path of the benchmark on CPU: world_size-2 gloo ranks combine
their replica timings as the GPU run does (max over ranks, whole-job
throughput = all ranks' units / slowest rank)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_s = 1.0 + rank  # rank 1 is the slow replica
    value, slowest = bench.combine_ranks(local_s, 1000, world, dist)
    dist.barrier()
    q.put((rank, value, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_gpu_run():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in out:
        assert slowest == pytest.approx(2.0)
        assert value == pytest.approx(2 * 1000 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench

    value, slowest = bench.combine_ranks(0.5, 100, 1, None)
    assert value == pytest.approx(200.0) and slowest == 0.5


def test_clock_record_summaries():
    """The bench's clock records: NVML clock-event reason bits decode to the
    names the timing rules use, and nvidia-smi lines parse the same way; with
    neither available the record is empty, not an error."""
    import bench

    nv = bench.NvmlClocks(0)
    nv.samples = [(2070.0, 0x0), (2070.0, 0x4), (1995.0, 0x4 | 0x40), (2070.0, 0x1)]
    nv.max_mhz = 2070.0
    s = nv.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]  # 0x1 (idle) is not a slowdown
    smi = bench.ClockSampler(0)
    smi.lines = ["0, 2070, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active",
                 "0, 1800, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Not Active"]
    s = smi.summary()
    assert s["sm_mhz"] == 1935.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    if not torch_cuda_available():
        rec = bench.ClockRecord(0)
        with rec:
            pass
        assert rec.summary()["samples"] == 0


def torch_cuda_available():
    import torch

    return torch.cuda.is_available()
