"""The N > 1 path of bench.py: independent replicas, one per rank, timed with a
barrier and the slowest rank's time. Two gloo ranks on the CPU check the
aggregation the NCCL run uses: under weak scaling every replica solves a whole
time step per step, so value = the slowest replica's ms per time step, and the
job's throughput (time steps per second over all ranks) is reported apart."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms_local = [800.0, 1200.0][rank]   # the replicas ran 4 steps each
        q.put((rank,) + bench.replica_ms_per_step(ms_local, 4))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_step, ms_max, rate in got:
        assert ms_max == 1200.0                 # both ranks see the slowest rank's time
        assert ms_step == 1200.0 / 4            # the slowest replica's ms per time step
        assert rate == pytest.approx(8 / 1.2)   # 8 time steps in 1.2 s for the whole job


def test_single_process_is_plain_average():
    assert bench.replica_ms_per_step(900.0, 3) == (300.0, 900.0, pytest.approx(3 / 0.9))
