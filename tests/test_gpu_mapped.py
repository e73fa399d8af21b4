"""General convex quadrilaterals (HZ_NODE_COORDS) through the C ABI against
the oracle's mapped discretisation (oracle/geom.py, pinned on the CPU).

Tolerances as in test_gpu_parity.py: FP64 sweep 1e-11 relative (both sides
use the element form; summation orders differ), FP32 sweep FP32_REL = 2e-5
(tests/_tolerances.py), solutions against the direct solve 1e-7 after a
1e-11 residual (cond(K) times the residual on these small meshes).
"""

import numpy as np
import pytest

from oracle import dd, geom, sem
from workloads import configs

import _tolerances as _tol
from _tolerances import FP32_REL

pytestmark = pytest.mark.gpu


def _wl(nx, ny, sx, sy, P, omega=9.0, amp=0.05, kind="channel"):
    w = configs.Workload(f"m{nx}x{ny}p{P}", (0.0, 1.0, 0.0, 1.0), nx, ny, P, sx, sy, omega, kind, (0.37, 0.58),
                         0.08, extra={"warp": amp})
    return w


def _pair(hz, wl, g_seed=3):
    from paper_2606_21695_gb300.api import Case, boundary_vector

    case = Case(wl, device=0)
    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    X, Y = wl.node_xy(*m.coords_1d())
    rng = np.random.default_rng(g_seed)
    g = {k: rng.standard_normal(len(v)) + 1j * rng.standard_normal(len(v)) for k, v in wl.boundary().items()}
    hz.hz_problem_set(case.pr, hz.HZ_BOUNDARY, boundary_vector(g))
    pr = geom.MappedProblem(m, X, Y, wl.speed_at(X, Y), wl.omega, wl.source_at(X, Y), g)
    assert np.max(np.abs(case.X - X)) < 1e-15 and np.max(np.abs(case.c - pr.c)) < 1e-15
    return case, pr


def _rand_lam(pr, seed):
    m = pr.mesh
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
    for l in range(m.L):
        for e in range(4):
            n = m.nly if e < 2 else m.nlx
            lam[l, e, n:] = 0
            if pr.nbr[l, e] < 0:
                lam[l, e] = 0
    return lam


def _dev(x):
    import torch

    a = np.ascontiguousarray(x)
    if np.iscomplexobj(a):
        a = a.astype(np.complex128).reshape(-1).view(np.float64)
    return torch.from_numpy(a.copy()).cuda()


def _host_c(t):
    return t.cpu().numpy().view(np.complex128)


def _rel(a, b):
    return _tol.record(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run_sweep(hz, case, pr, precision, nt, m_wh, lam, with_rhs):
    import torch

    m = pr.mesh
    nl = hz.hz_lambda_size(case.pr)
    lin = _dev(lam)
    lout = torch.full((2 * nl,), float("nan"), dtype=torch.float64, device="cuda")
    usub = torch.zeros(2 * m.L * m.nly * m.nlx, dtype=torch.float64, device="cuda")
    rhs = None
    if with_rhs:
        rhs = torch.empty(2 * case.n, dtype=torch.float64, device="cuda")
        hz.hz_rhs(case.pr, rhs)
    hz.hz_sweep(case.pr, precision, nt, m_wh, 0.0, lin, lout, rhs, usub)
    torch.cuda.synchronize()
    return _host_c(lout).reshape(m.L, 4, m.NE), _host_c(usub).reshape(m.L, m.nly, m.nlx)


LAYOUTS = [
    (16, 16, 8, 8, 3),  # the benchmark's subdomain shape (25 x 25 nodes), 2x2 subdomains
    (8, 8, 4, 4, 2),    # cross point, P = 2
    (6, 6, 2, 2, 3),    # 3x3 subdomains
    (8, 4, 2, 4, 1),    # strips, P = 1
    (4, 6, 4, 2, 4),    # P = 4, non-square subdomains
    (4, 4, 2, 2, 5),    # P = 5
    (2, 4, 2, 2, 7),    # P = 7
    (4, 4, 1, 1, 2),    # single-element subdomains
]


@pytest.mark.parametrize("nx,ny,sx,sy,P", LAYOUTS)
def test_mapped_sweep_fp64_matches_oracle(hz, nx, ny, sx, sy, P):
    case, pr = _pair(hz, _wl(nx, ny, sx, sy, P))
    nt = pr.choose_nt()
    lam = _rand_lam(pr, 1)
    got_l, got_u = _run_sweep(hz, case, pr, hz.HZ_FP64, nt, 2, lam, True)
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 2, want_u=True)
    assert _rel(got_u, ref_u) < 1e-11
    assert _rel(got_l, ref_l) < 1e-11
    got_h, _ = _run_sweep(hz, case, pr, hz.HZ_FP64, nt, 2, lam, False)
    assert _rel(got_h, pr.sweep(lam, None, nt, 2)) < 1e-11
    case.close()


@pytest.mark.parametrize("nx,ny,sx,sy,P", LAYOUTS[:4])
def test_mapped_sweep_fp32_error(hz, nx, ny, sx, sy, P):
    case, pr = _pair(hz, _wl(nx, ny, sx, sy, P))
    nt = pr.choose_nt()
    lam = _rand_lam(pr, 2)
    got_l, got_u = _run_sweep(hz, case, pr, hz.HZ_FP32_REFINE, nt, 2, lam, True)
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 2, want_u=True)
    assert _rel(got_u, ref_u) < FP32_REL
    assert _rel(got_l, ref_l) < FP32_REL
    case.close()


def test_mapped_rhs_residual_and_assembly_match_oracle(hz):
    import torch

    case, pr = _pair(hz, _wl(12, 8, 4, 4, 3))
    m = pr.mesh
    b = torch.empty(2 * case.n, dtype=torch.float64, device="cuda")
    hz.hz_rhs(case.pr, b)
    assert _rel(_host_c(b).reshape(m.NY, m.NX), pr.rhs()) < 1e-13
    rng = np.random.default_rng(7)
    u = rng.standard_normal((m.NY, m.NX)) + 1j * rng.standard_normal((m.NY, m.NX))
    r = torch.empty_like(b)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    hz.hz_residual(case.pr, b, _dev(u), r, norms)
    ref_r = pr.residual(u)
    assert _rel(_host_c(r).reshape(m.NY, m.NX), ref_r) < 1e-12
    assert abs(norms[0].item() - np.sum(np.abs(ref_r) ** 2)) < 1e-10 * np.sum(np.abs(ref_r) ** 2)
    us = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    acc = torch.zeros_like(b)
    hz.hz_assemble_add(case.pr, _dev(us), acc)
    assert _rel(_host_c(acc), pr.assemble_u(us).ravel()) < 1e-14
    case.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_mapped_solve_matches_direct(hz, precision):
    case, pr = _pair(hz, _wl(16, 16, 4, 4, 3, omega=14.0))
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_FP32_REFINE
    st, u, rep = hz.hz_solve(case.pr, hz.hz_default_opts(precision=prec, tol=1e-11, max_sweeps=4000), n=case.n)
    assert st == hz.HZ_OK and rep["rel_residual"] <= 1e-11 and rep["sweep_variant"] == 6
    ud = pr.direct_solve()
    assert _rel(u, ud.ravel()) < 1e-7
    case.close()


def test_identity_coordinates_reproduce_the_cartesian_path(hz):
    """Setting the Cartesian grid's own coordinates switches to the mapped
    kernels; the sweep equals the Cartesian kernels' to FP64 rounding."""
    from paper_2606_21695_gb300.api import Case

    wl = configs.Workload("id", (0.0, 1.0, 0.0, 1.0), 8, 8, 3, 4, 4, 9.0, "channel", (0.37, 0.58), 0.08)
    cart = Case(wl)
    mapd = Case(wl)
    X, Y = np.meshgrid(mapd.gx, mapd.gy)
    hz.hz_problem_set(mapd.pr, hz.HZ_NODE_COORDS, np.stack([X.ravel(), Y.ravel()], 1).ravel())
    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    ref = dd.Problem(m, wl.speed(*m.coords_1d()), wl.omega, wl.source(*m.coords_1d()), wl.boundary())
    nt = hz.hz_problem_nt(cart.pr)
    lam = _rand_lam(ref, 4)
    a_l, a_u = _run_sweep(hz, cart, ref, hz.HZ_FP64, nt, 2, lam, True)
    b_l, b_u = _run_sweep(hz, mapd, ref, hz.HZ_FP64, nt, 2, lam, True)
    assert _rel(b_u, a_u) < 1e-12 and _rel(b_l, a_l) < 1e-12
    cart.close()
    mapd.close()


def test_time_step_rule_matches_the_oracle_bound(hz):
    case, pr = _pair(hz, _wl(8, 8, 4, 4, 3))
    nt = hz.hz_problem_nt(case.pr)
    ref = pr.choose_nt()
    # host power iteration with a 1% margin vs the oracle's exact element eigenvalues
    assert ref <= nt <= int(np.ceil(ref * 1.006)) + 1
    case.close()


def test_invalid_geometry_is_refused(hz):
    from paper_2606_21695_gb300.api import Case

    wl = configs.Workload("bad", (0.0, 1.0, 0.0, 1.0), 4, 4, 2, 2, 2, 5.0, "const", (0.5, 0.5), 0.1)
    case = Case(wl)
    X, Y = np.meshgrid(case.gx, case.gy)
    Xf = X.copy()
    Xf[2, 1], Xf[2, 3] = X[2, 3], X[2, 1]  # fold an element: negative Jacobian
    with pytest.raises(hz.HzError) as e:
        hz.hz_problem_set(case.pr, hz.HZ_NODE_COORDS, np.stack([Xf.ravel(), Y.ravel()], 1).ravel())
    assert e.value.status == hz.HZ_ERR_INVALID_ARG
    with pytest.raises(hz.HzError) as e:
        hz.hz_problem_set(case.pr, hz.HZ_NODE_COORDS, X.ravel())  # n values instead of 2n
    assert e.value.status == hz.HZ_ERR_INVALID_ARG
    case.close()
    big = Case(configs.Workload("big", (0.0, 1.0, 0.0, 1.0), 32, 32, 2, 16, 16, 5.0, "const", (0.5, 0.5), 0.1),
               fields=False)  # 33 x 33 = 1089 subdomain nodes
    Xb, Yb = np.meshgrid(big.gx, big.gy)
    with pytest.raises(hz.HzError) as e:
        hz.hz_problem_set(big.pr, hz.HZ_NODE_COORDS, np.stack([Xb.ravel(), Yb.ravel()], 1).ravel())
    assert e.value.status == hz.HZ_ERR_UNSUPPORTED
    big.close()


def test_mapped_problem_in_batch_and_server_equals_solo(hz):
    from paper_2606_21695_gb300.api import Case

    cases = [Case(_wl(8, 8, 4, 4, 2, omega=8.0)), Case(configs.scaled(configs.config1(), 16, 16, 8, 8, name="c"))]
    o = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8)
    solo = []
    for c in cases:
        st, u, rep = hz.hz_solve(c.pr, o, n=c.n)
        assert st == hz.HZ_OK
        solo.append(u.copy())
    st, sts, us, reps = hz.hz_solve_batch([c.pr for c in cases], [c.n for c in cases], o)
    assert st == hz.HZ_OK and reps[0]["sweep_variant"] == 6
    assert np.array_equal(us[0], solo[0])
    srv = hz.hz_server_create(0, 1 << 30)
    try:
        t = hz.hz_server_submit(srv, cases[0].pr, o)
        done, st, u, rep = hz.hz_server_poll(srv, t, -1, n=cases[0].n)
        assert done and st == hz.HZ_OK and np.array_equal(u, solo[0])
    finally:
        hz.hz_server_destroy(srv)
    for c in cases:
        c.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mapped_full_size_sampled_sweep(hz, precision):
    """The curved-quadrilateral benchmark workload (cfg2m: 256x256 warped quads,
    P=3, 32x32 subdomains) at full size: one sweep as the solve launches it,
    sampled subdomains recomputed by the mapped oracle (each subdomain's cycle
    depends only on its own data and incoming lambda)."""
    from paper_2606_21695_gb300.api import Case

    wl = configs.config2m()
    case = Case(wl)
    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    X, Y = wl.node_xy(*m.coords_1d())
    pr = geom.MappedProblem(m, X, Y, wl.speed_at(X, Y), wl.omega, wl.source_at(X, Y), wl.boundary())
    nt = hz.hz_problem_nt(case.pr)
    lam = _rand_lam(pr, 7) * 1e-2
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_FP32_REFINE
    got_l, got_u = _run_sweep(hz, case, pr, prec, nt, 3, lam, True)
    sample = [0, m.Sx - 1, 17 * m.Sx + 9, m.L - m.Sx, m.L - 1, 511]
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 3, want_u=True, subset=sample)
    tol = 1e-11 if precision == "fp64" else FP32_REL
    scale = max(np.max(np.abs(ref_u[sample])), 1e-300)
    for l in sample:
        assert np.max(np.abs(got_u[l] - ref_u[l])) < tol * scale, l
        for e in range(4):
            r = pr.nbr[l, e]
            if r >= 0:
                o = dd.OPPOSITE[e]
                sl = np.max(np.abs(ref_l[r, o])) + 1e-300
                assert np.max(np.abs(got_l[r, o] - ref_l[r, o])) < tol * max(sl, np.max(np.abs(lam))), (l, e)
            else:
                assert np.all(got_l[l, e] == 0)
    case.close()


def test_mapped_generalised_transmission_matches_oracle(hz):
    """Interface condition d_n + k (eta - i zeta) on a mapped mesh: the boundary
    mass and the zeta-scaled damping use the arc-length edge weights."""
    from paper_2606_21695_gb300.api import Case, boundary_vector

    wl = _wl(8, 8, 4, 4, 3)
    case = Case(wl, device=0)
    hz.hz_problem_set(case.pr, hz.HZ_TRANSMISSION, np.array([0.3, 0.8]))
    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    X, Y = wl.node_xy(*m.coords_1d())
    pr = geom.MappedProblem(m, X, Y, wl.speed_at(X, Y), wl.omega, wl.source_at(X, Y), wl.boundary(),
                            robin=(0.3, 0.8))
    nt = pr.choose_nt()
    lam = _rand_lam(pr, 9)
    for prec, tol in ((hz.HZ_FP64, 1e-11), (hz.HZ_FP32_REFINE, FP32_REL)):
        got_l, got_u = _run_sweep(hz, case, pr, prec, nt, 2, lam, True)
        ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 2, want_u=True)
        assert _rel(got_u, ref_u) < tol and _rel(got_l, ref_l) < tol, prec
    case.close()


def test_coordinates_set_from_device_memory(hz):
    import torch

    from paper_2606_21695_gb300.api import Case

    wl = _wl(8, 8, 4, 4, 2)
    a = Case(wl)
    b = Case(configs.Workload(wl.name, wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny, wl.omega, wl.speed_kind,
                              wl.src_center, wl.src_width, extra={}))
    xy = torch.from_numpy(np.stack([a.X.ravel(), a.Y.ravel()], 1).ravel().copy()).cuda()
    hz.hz_problem_set_device(b.pr, hz.HZ_NODE_COORDS, xy, 2 * b.n)
    hz.hz_problem_set(b.pr, hz.HZ_WAVE_SPEED, a.c.ravel())
    hz.hz_problem_set(b.pr, hz.HZ_SOURCE, a.f.ravel())
    o = hz.hz_default_opts(precision=hz.HZ_FP64, tol=1e-10)
    _, ua, ra = hz.hz_solve(a.pr, o, n=a.n)
    _, ub, rb = hz.hz_solve(b.pr, o, n=b.n)
    assert ra["sweep_variant"] == rb["sweep_variant"] == 6
    assert np.array_equal(ua, ub)
    a.close()
    b.close()
