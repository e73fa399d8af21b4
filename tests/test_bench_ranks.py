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


def test_bench_workload_pieces_keep_the_big_workload_physics():
    """The 1024^2 workload's pieces (bench legs, profiles) have its element
    size, degree, subdomain shape, frequency and medium."""
    import bench

    w3 = bench.workload("cfg3")
    h3 = (w3.box[1] - w3.box[0]) / w3.nx
    for name, S in (("cfg3p4", 4), ("cfg3p8", 8), ("cfg3p16", 16)):
        w = bench.workload(name)
        assert w.nx == w.ny == 32 * S and w.L == S * S
        assert abs((w.box[1] - w.box[0]) / w.nx - h3) < 1e-15
        assert (w.P, w.sub_nx, w.sub_ny, w.omega, w.speed_kind, w.speed_seed, w.corr_len) == \
               (w3.P, w3.sub_nx, w3.sub_ny, w3.omega, w3.speed_kind, w3.speed_seed, w3.corr_len)


def test_served_pool_is_the_cheapest_draws_of_the_sampler():
    import bench
    from workloads import configs

    pool = bench._serve_pool(16)
    names = {w.name for w in configs.config4(64, seed0=500)}
    assert len(pool) == 16 and {w.name for w in pool} <= names
    assert [w.name for w in bench._serve_pool(16)] == [w.name for w in pool]  # deterministic


def test_oracle_pool_on_two_cores():
    """The CPU baseline's worker pool: spawned single-threaded processes, a
    timed sample with a positive rate."""
    import bench

    pool = bench.OraclePool("cfg1", m_wh=1, cores=2)
    try:
        r = pool.sample(0.2)
    finally:
        pool.close()
    assert r["cores"] == 2 and r["value"] > 0 and r["nl"] == 17 * 17
