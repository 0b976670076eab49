"""Host side of the multi-GPU path (weak scaling over independent images):
two gloo ranks on the CPU exchange their step times the way bench.py does
under torchrun, and the whole-job value uses the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_setup()
        assert (r, w, local) == (rank, world, rank)
        ms_local = 10.0 + 5.0 * rank          # rank 1 is the slower one
        ms = bench.max_over_ranks_tensor(torch, ms_local, world, "cpu")
        value = bench.weak_scaling_value(world, 1_000_000, 4, ms)
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 ranks x 1 Mpx x 4 steps in 15 ms
    assert res[0][1] == pytest.approx(2 * 1e6 * 4 / 15e-3 / 1e9)
    assert res[0][1] == res[1][1]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks_tensor(torch, 3.5, 1, "cpu") == 3.5
    assert bench.weak_scaling_value(1, 2_000_000, 10, 20.0) == pytest.approx(1.0)
