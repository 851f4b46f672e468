"""The N-GPU path of bench.py is N independent replicas (the single solve does not
shard): the job time is the slowest rank's and the rate counts every rank's DoFs.
Checked with two gloo ranks on the CPU (the reduction bench.py does over NCCL)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]  # rank 1 is the slower replica
    slowest = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, slowest, bench.replica_throughput(529984, 5, world, slowest)))
    dist.destroy_process_group()


def test_two_gloo_replicas_report_the_slowest_time_and_all_units():
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
    assert [o[1] for o in out] == [150.0, 150.0]
    assert out[0][2] == pytest.approx(529984 * 5 * 2 / 0.150)
    assert out[0][2] == out[1][2]
