"""The bench's multi-GPU combination on CPU: world_size-2 gloo ranks, each
with its own time and work; every rank must see the slowest time and the
total work (the figures rank 0 prints)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as tdist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        q.put((rank, bench.combine_ranks(1.5 + rank, 1e9 * (rank + 1), "cpu"), bench.dist_env()[:2]))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_combine_ranks_max_time_total_work(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (t, w), (r_env, w_env) in res:
        assert t == 1.5 + (world - 1)
        assert w == 1e9 * world * (world + 1) / 2
        assert (r_env, w_env) == (rank, world)
