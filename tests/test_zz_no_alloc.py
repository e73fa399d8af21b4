"""hz_residual_noalloc: the global residual for callers that cannot allocate
device memory (inside another component's graph capture, under a foreign
allocator, in a loop that must not synchronise).  It must give what
hz_residual gives, call after call, from caller-owned arrays only, and what
the oracle's matrix-free K gives for every compiled degree.

Collected last on purpose (file name), so a stop-at-first-failure run has
already run every other test; it also passes alone in a fresh process."""

import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_hz_residual_twice(hz):
    import torch

    from paper_2606_21695_gb300.api import Case

    wl = configs.scaled(configs.config2(), 40, 24, 8, 8, name="noalloc_40x24")  # ragged block edges
    case = Case(wl)
    n = case.n
    c = torch.from_numpy(np.ascontiguousarray(case.c.ravel())).cuda()
    b = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    hz.hz_rhs(case.pr, b)
    rng = np.random.default_rng(11)
    for call in range(2):  # the shared scratch keeps the previous call's partial sums
        uh = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        u = torch.from_numpy(uh.view(np.float64).copy()).cuda()
        r_ref = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        n_ref = torch.empty(2, dtype=torch.float64, device="cuda")
        hz.hz_residual(case.pr, b, u, r_ref, n_ref)
        r = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
        nrm = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        hz.hz_residual_noalloc(case.mesh, wl.omega, c, b, u, r, nrm)
        torch.cuda.synchronize()
        rr, rref = r.cpu().numpy(), r_ref.cpu().numpy()
        assert np.max(np.abs(rr - rref)) <= 1e-12 * np.max(np.abs(rref)), call
        np.testing.assert_allclose(nrm.cpu().numpy(), n_ref.cpu().numpy(), rtol=1e-12)
    case.close()


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7])
def test_residual_noalloc_matches_oracle_every_degree(hz, P):
    """r = b - (A - i w H - w^2 M) u (Sec. 4) against the oracle's
    matrix-free element-form K on a non-square box with variable c; the node
    grid is ragged against the 32 x 8 blocks in both directions."""
    import torch

    from oracle.dd import Problem
    from oracle.sem import Mesh

    nx, ny = 11, 7
    box = (-0.3, 0.9, 0.1, 0.75)
    m = Mesh(*box, nx, ny, P, nx, ny)
    hm = hz.hz_mesh_create(*box, nx, ny, P, nx, ny)
    try:
        rng = np.random.default_rng(100 + P)
        cvals = 0.5 + rng.uniform(size=(m.NY, m.NX))
        omega = 7.5
        pr = Problem(m, cvals, omega, np.zeros((m.NY, m.NX)))
        n = m.NX * m.NY
        c = torch.from_numpy(cvals.ravel().copy()).cuda()
        for call in range(2):
            uh = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).reshape(m.NY, m.NX)
            bh = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).reshape(m.NY, m.NX)
            want = bh - pr.apply_K(uh)
            u = torch.from_numpy(uh.ravel().view(np.float64).copy()).cuda()
            b = torch.from_numpy(bh.ravel().view(np.float64).copy()).cuda()
            r = torch.full((2 * n,), float("nan"), dtype=torch.float64, device="cuda")
            nrm = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
            hz.hz_residual_noalloc(hm, omega, c, b, u, r, nrm)
            torch.cuda.synchronize()
            got = r.cpu().numpy().view(complex).reshape(m.NY, m.NX)
            scale = np.max(np.abs(want))
            assert np.max(np.abs(got - want)) <= 1e-12 * scale, (P, call)
            np.testing.assert_allclose(nrm.cpu().numpy(),
                                       [np.sum(np.abs(want) ** 2), np.sum(np.abs(bh) ** 2)], rtol=1e-11)
    finally:
        hz.hz_mesh_destroy(hm)


def test_residual_noalloc_rejects_meshes_beyond_its_scratch(hz):
    import torch

    tiny = torch.zeros(4, dtype=torch.float64, device="cuda")
    m = hz.hz_mesh_create(0, 1, 0, 1, 8192, 8192, 7, 8192, 8192)  # 57345^2 nodes, host-side only
    try:
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 1.0, tiny, tiny, tiny, tiny, tiny)
        assert e.value.status == hz.HZ_ERR_UNSUPPORTED
        assert "too large" in str(e.value)
    finally:
        hz.hz_mesh_destroy(m)
    # a thin strip: few blocks in all, but more rows of blocks than a launch allows
    m = hz.hz_mesh_create(0, 1, 0, 100, 4, 600000, 1, 4, 600000)  # 5 x 600001 nodes: 75001 block rows
    try:
        with pytest.raises(hz.HzError) as e:
            hz.hz_residual_noalloc(m, 1.0, tiny, tiny, tiny, tiny, tiny)
        assert e.value.status == hz.HZ_ERR_UNSUPPORTED
        assert "node rows" in str(e.value)
    finally:
        hz.hz_mesh_destroy(m)
