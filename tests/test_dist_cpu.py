"""The N > 1 path of bench.py on the CPU: world-size-2 gloo ranks (the path is replicas only, so the one
exchange is the timing: every rank reports its time and the job takes the maximum over ranks)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench

    class Args:
        impl = "reference"   # the gloo backend (the GPU arm uses NCCL)

    try:
        wsz, r, local = bench.dist_setup(Args)
        bench.barrier(wsz)
        v = bench.barrier_max(wsz, 10.0 * (rank + 1))
        q.put((r, wsz, local, v))
    finally:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


def test_replicas_take_the_maximum_time_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in range(2))
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    assert got == [(0, 2, 0, 20.0), (1, 2, 1, 20.0)]
    assert all(p.exitcode == 0 for p in ps)


def test_single_rank_needs_no_process_group():
    import bench

    class Args:
        impl = "ours"

    saved = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        assert bench.dist_setup(Args) == (1, 0, 0)
        assert bench.barrier_max(1, 3.5) == 3.5
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v


def test_clock_summary_parses_samples_and_throttle_reasons():
    """The clock record of the timed region: median SM clock, the maximum clock and every throttle reason
    seen active (the ones that reject a run, and sw_power_cap, which is kept and noted)."""
    import bench
    cs = bench.ClockSampler()
    na = "Not Active"
    cs.lines = [
        f"0, 2070, 2070, 812.4, 0x0, {na}, {na}, {na}, {na}",
        f"0, 1980, 2070, 1390.2, 0x4, {na}, {na}, {na}, Active",
        f"0, 2055, 2070, 1201.0, 0x0, {na}, {na}, {na}, {na}",
        "0, [N/A], 2070, 0, 0x0",              # malformed and short lines are skipped
        "",
    ]
    s = cs.summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.lines.append(f"0, 1500, 2070, 1400.0, 0x40, {na}, Active, {na}, {na}")
    assert cs.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler().summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
