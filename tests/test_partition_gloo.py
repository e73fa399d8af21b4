"""Multi-rank path of the DD sweep on CPU: world_size-2 gloo process group,
each rank runs the oracle's DDM cycle on its own block of subdomains, the
cut-interface lambda slots travel point-to-point, and the dot products of
the outer Krylov iteration are all-reduced.  The assembled result must equal
the single-rank sweep bit for bit (same arithmetic per subdomain)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2606_21695_gb300.partition import Partition, pack, unpack


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from oracle import dd, sem

    m = sem.Mesh(0, 1, 0, 1, 8, 6, 2, 2, 2)  # 4 x 3 subdomains
    X, Y = m.coords()
    return dd.Problem(m, 1.0 + 0.2 * np.sin(3 * X) * np.cos(2 * Y), 7.0, np.exp(-30 * ((X - .4) ** 2 + (Y - .6) ** 2)))


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = _problem()
        m = pr.mesh
        part = Partition(m.Sx, m.Sy, world)
        rng = np.random.default_rng(0)
        lam_in = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
        nt = pr.choose_nt()
        mine = part.subdomains(rank)
        out = pr.sweep(lam_in, pr.rhs(), nt, 2, subset=mine)
        # exchange cut-interface slots
        reqs = []
        for dst, slots in sorted(part.send_plan(rank).items()):
            buf = torch.from_numpy(pack(out, slots).view(np.float64).copy())
            reqs.append(dist.isend(buf, dst))
        for src, slots in sorted(part.recv_plan(rank).items()):
            buf = torch.empty(len(slots) * m.NE * 2, dtype=torch.float64)
            dist.recv(buf, src)
            unpack(out, slots, buf.numpy().view(np.complex128).reshape(len(slots), m.NE))
        for r in reqs:
            r.wait()
        # dot product of the outer iteration: all-reduce of the per-rank partials
        part_dot = np.vdot(out[mine], out[mine])
        t = torch.tensor([part_dot.real, part_dot.imag], dtype=torch.float64)
        dist.all_reduce(t)
        q.put((rank, mine, out[mine], complex(t[0].item(), t[1].item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_sweep_matches_single_rank(world):
    pr = _problem()
    m = pr.mesh
    rng = np.random.default_rng(0)
    lam_in = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
    ref = pr.sweep(lam_in, pr.rhs(), pr.choose_nt(), 2)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seen = np.zeros(m.L, bool)
    for rank, mine, vals, dot in results:
        np.testing.assert_array_equal(vals, ref[mine])  # bitwise
        seen[mine] = True
        assert abs(dot - np.vdot(ref, ref)) <= 1e-12 * abs(np.vdot(ref, ref))
    assert seen.all()


def test_partition_plans_are_consistent():
    for Sx, Sy, R in [(4, 3, 2), (32, 32, 8), (5, 7, 4), (3, 3, 3)]:
        p = Partition(Sx, Sy, R)
        assert sorted(set(p.owner)) == list(range(R))
        for r in range(R):
            for dst, slots in p.send_plan(r).items():
                back = p.recv_plan(dst)[r]
                assert back == slots  # the receiver unpacks exactly what the sender packs
