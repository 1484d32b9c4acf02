"""The replica path of the multi-GPU bench, on CPU with gloo and two ranks.

Each rank solves its own problems; the only collective is the max of the wall
time, and the job throughput counts every rank's units against that maximum.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_13046_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = replicas.dist_env()
        secs = replicas.max_over_ranks(times[rank])
        value = replicas.job_throughput(5, secs, ws)
        out.put((rank, env, secs, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_max_over_ranks_gloo(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.75, 1.25, 0.5, 2.0][:ws]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, times, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, (rank, env, secs, value) in enumerate(res):
        assert env == (ws, r, r)
        assert secs == max(times)                  # every rank sees the slowest rank's time
        assert value == pytest.approx(ws * 5 / max(times))


def test_single_process_passthrough():
    assert not dist.is_initialized()
    assert replicas.max_over_ranks(0.3) == 0.3
    assert replicas.job_throughput(10, 2.0, 1) == 5.0
    with pytest.raises(ValueError):
        replicas.job_throughput(1, 0.0, 1)
