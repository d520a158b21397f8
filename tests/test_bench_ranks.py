"""The multi-rank logic of bench.py on CPU ranks (gloo, world size 2): independent replicas, the
slowest rank's time, and the whole-job value (units of all ranks over that time).  No GPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        mine = 10.0 * (rank + 1)               # rank 1 is the slow replica
        slowest = bench.max_over_ranks(mine, world, device="cpu")
        q.put((rank, slowest, bench.replica_value(5, 32, world, slowest)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    assert out[0][2] == pytest.approx(5 * 32 * 2 / 0.020)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_value(20, 32, 1, 1000.0) == pytest.approx(640.0)
