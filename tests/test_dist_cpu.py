"""Multi-process host logic of the benchmark (one shot per rank, max-over-ranks
timing, barrier, stacking of the ranks' gradients and misfits), on CPU with
the gloo backend and world_size 2."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        t = bench.max_over_ranks(dist, 1.0 + rank)
        args = type("A", (), {"grid": "48,40,24", "nt": 10})()
        shot, _ = bench.workload(args, rank)
        out[rank] = (t, tuple(shot.src))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_max_time_and_distinct_shots():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0          # max over ranks
    assert res[0][1] != res[1][1]                 # each rank models its own shot
    assert all(0 <= c for c in res[0][1] + res[1][1])


def _stack_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = torch.Generator().manual_seed(100 + rank)
        grad = torch.randn((5, 6, 7), generator=g)
        phi = bench.stack(dist, grad, 1.5 + rank)
        out[rank] = (grad.numpy().copy(), phi)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_stack_gradients_and_misfits():
    """Stacking (Sec. 2: the objective and its gradient are sums over shots):
    after the step every rank holds the sum of both ranks' gradients and
    misfits."""
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_stack_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    expect = sum(torch.randn((5, 6, 7), generator=torch.Generator().manual_seed(100 + r)) for r in range(world))
    for r in range(world):
        assert torch.equal(torch.from_numpy(res[r][0]), expect)
        assert res[r][1] == 1.5 + 2.5
