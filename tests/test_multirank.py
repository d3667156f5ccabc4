"""The multi-GPU path is replicas only (each rank solves its own batch, seed = rank, no
data-path collective); what the ranks share is the timing: the step time is the maximum
over ranks and the throughput counts every rank's units. This host logic runs here as two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench._dist()
        ms = bench._max_over_ranks(10.0 + 5.0 * rank)   # rank 1 is the slow one
        p = bench._problem(rank, batch=2)
        out[rank] = (ws, r, ms, bench._whole_job_rate(1000, ws, ms),
                     float(p["params"].sum()), float(p["s0"].sum()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_problems():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        ws, r, ms, rate, _, _ = res[rank]
        assert (ws, r) == (2, rank)
        assert ms == 15.0                      # max over ranks, same on every rank
        assert rate == pytest.approx(2 * 1000 / 0.015)
    # replicas: each rank draws its own systems (seed = rank)
    assert res[0][4] != res[1][4] and res[0][5] != res[1][5]


def test_single_process_is_identity():
    import bench
    assert bench._max_over_ranks(3.5) == 3.5
    assert bench._whole_job_rate(100, 1, 1000.0) == pytest.approx(100.0)
