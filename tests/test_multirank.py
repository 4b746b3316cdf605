"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2).

Ranks run independent ensemble members (weak scaling, no data-path
collective); only the timing is reduced with a max across ranks.
"""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    t = bench.reduce_max(1.5 + rank, w)          # rank 1 is the slow one
    seed = bench.rank_seed(7, r)
    dist.barrier()
    q.put((r, w, loc, t, seed))
    dist.destroy_process_group()


def test_two_rank_timing_reduction_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 2.5 for r in res)            # max over ranks on every rank
    assert res[0][4] != res[1][4]                   # independent ensemble members


def test_aggregate_is_whole_job_over_slowest_rank():
    import bench
    v, t = bench.aggregate([2.0, 4.0], sites_per_rank=1000, steps=10)
    assert t == 4.0 and v == pytest.approx(2 * 1000 * 10 / 4.0 / 1e6)


def test_clock_samples_summary():
    """NVML clock-event reason bits map to the names the benchmark line
    reports (sw_power_cap 0x4, hw_slowdown 0x8, sw_thermal_slowdown 0x20,
    hw_thermal_slowdown 0x40); idle (0x1) and other bits are not reasons; the
    SM clock is the median of the samples."""
    import bench
    s = bench.NvmlClocks.summarise([(2070, 0x0), (2070, 0x1), (1980, 0x4), (2070, 0x100)], 2070)
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.NvmlClocks.summarise([(1500, 0x8 | 0x40), (1600, 0x20)], 2070)
    assert s["sm_mhz"] == 1550 and s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown",
                                                     "sw_thermal_slowdown"]
    assert bench.NvmlClocks.summarise([], 2070) is None
