"""Warm-started WaveHoltz (hz_sweep_from, opts.wh_warm; Sec. 8): the sweep
started from given subdomain solutions against the oracle's sweep with the
same start (FP64 1e-11, FP32 FP32_REL = 2e-5 of tests/_tolerances.py), on the one-warp,
block and mapped-mesh kernels; the plain fixed-point iteration with warm
starts reaches the global tolerance with fewer WaveHoltz iterations; the
GMRES outer iterations refuse it."""

import numpy as np
import pytest

from oracle import dd, geom, sem
from workloads import configs

import _tolerances as _tol
from _tolerances import FP32_REL

pytestmark = pytest.mark.gpu


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


def _lam(pr, seed):
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


def _case(hz, nx, ny, sx, sy, P, amp=0.0):
    from paper_2606_21695_gb300.api import Case

    extra = {"warp": amp} if amp > 0 else {}
    wl = configs.Workload(f"w{nx}x{ny}p{P}", (0.0, 1.0, 0.0, 1.0), nx, ny, P, sx, sy, 9.0, "channel", (0.37, 0.58),
                          0.08, extra=extra)
    case = Case(wl)
    m = sem.Mesh(*wl.box, nx, ny, P, sx, sy)
    if amp > 0:
        X, Y = wl.node_xy(*m.coords_1d())
        pr = geom.MappedProblem(m, X, Y, wl.speed_at(X, Y), wl.omega, wl.source_at(X, Y), wl.boundary())
    else:
        gx, gy = m.coords_1d()
        pr = dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary())
    return case, pr


@pytest.mark.parametrize("nx,ny,sx,sy,P,amp,precision", [
    (16, 16, 8, 8, 3, 0.0, "fp32"),   # one-warp kernel (25 columns)
    (16, 16, 8, 8, 3, 0.0, "fp64"),   # block kernel
    (8, 8, 4, 4, 2, 0.0, "fp32"),
    (4, 4, 2, 2, 7, 0.0, "fp64"),
    (8, 8, 4, 4, 3, 0.05, "fp64"),    # mapped kernel
    (8, 8, 4, 4, 3, 0.05, "fp32"),
])
def test_warm_sweep_matches_oracle(hz, nx, ny, sx, sy, P, amp, precision):
    import torch

    case, pr = _case(hz, nx, ny, sx, sy, P, amp)
    m = pr.mesh
    nt = hz.hz_problem_nt(case.pr)
    lam = _lam(pr, 3)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 2, want_u=True, u0=u0)
    prec = hz.HZ_FP64 if precision == "fp64" else hz.HZ_FP32_REFINE
    rhs = torch.empty(2 * case.n, dtype=torch.float64, device="cuda")
    hz.hz_rhs(case.pr, rhs)
    lout = torch.full((2 * hz.hz_lambda_size(case.pr),), float("nan"), dtype=torch.float64, device="cuda")
    ubuf = _dev(u0)  # in place: the start is read and the result written into the same buffer
    hz.hz_sweep_from(case.pr, prec, nt, 2, 0.0, _dev(lam), lout, rhs, ubuf, ubuf)
    torch.cuda.synchronize()
    tol = 1e-11 if precision == "fp64" else FP32_REL
    assert _rel(_host_c(ubuf).reshape(ref_u.shape), ref_u) < tol
    assert _rel(_host_c(lout).reshape(ref_l.shape), ref_l) < tol
    # a warm start from zero is the cold sweep
    ref0 = pr.sweep(lam, pr.rhs(), nt, 2)
    z = torch.zeros_like(ubuf)
    hz.hz_sweep_from(case.pr, prec, nt, 2, 0.0, _dev(lam), lout, rhs, z, z)
    torch.cuda.synchronize()
    assert _rel(_host_c(lout).reshape(ref0.shape), ref0) < tol
    case.close()


@pytest.mark.parametrize("warps", ["2", "4"])
def test_warm_sweep_on_warp_bands(hz, monkeypatch, warps):
    """The 2- and 4-warp band kernels read the start too (each band its own rows)."""
    import torch

    monkeypatch.setenv("HZ_SWEEP_WARPS", warps)
    case, pr = _case(hz, 16, 16, 8, 8, 3)
    m = pr.mesh
    nt = hz.hz_problem_nt(case.pr)
    lam = _lam(pr, 5)
    rng = np.random.default_rng(6)
    u0 = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 2, want_u=True, u0=u0)
    rhs = torch.empty(2 * case.n, dtype=torch.float64, device="cuda")
    hz.hz_rhs(case.pr, rhs)
    lout = torch.zeros(2 * hz.hz_lambda_size(case.pr), dtype=torch.float64, device="cuda")
    ubuf = _dev(u0)
    hz.hz_sweep_from(case.pr, hz.HZ_FP32_REFINE, nt, 2, 0.0, _dev(lam), lout, rhs, ubuf, ubuf)
    torch.cuda.synchronize()
    assert _rel(_host_c(ubuf).reshape(ref_u.shape), ref_u) < FP32_REL
    assert _rel(_host_c(lout).reshape(ref_l.shape), ref_l) < FP32_REL
    case.close()


def test_plain_iteration_warm_start_saves_waveholtz_iterations(hz):
    from paper_2606_21695_gb300.api import Case

    wl = configs.Workload("pw", (0.0, 1.0, 0.0, 1.0), 8, 4, 2, 4, 4, 6.0, "const", (0.4, 0.5), 0.1)  # 2 subdomains
    case = Case(wl)
    reps, us = {}, {}
    for warm in (0, 1):
        o = hz.hz_default_opts(precision=hz.HZ_FP64, tol=1e-8, outer=hz.HZ_OUTER_PLAIN, wh_iters=80, wh_tol=1e-9,
                               max_sweeps=3000, wh_warm=warm)
        st, u, rep = hz.hz_solve(case.pr, o, n=case.n)
        assert st == hz.HZ_OK and rep["rel_residual"] <= 1e-8, (warm, rep)
        reps[warm], us[warm] = rep, u.copy()
    assert reps[1]["dof_updates"] < 0.9 * reps[0]["dof_updates"], (reps[1]["dof_updates"], reps[0]["dof_updates"])
    assert np.max(np.abs(us[1] - us[0])) < 1e-6 * np.max(np.abs(us[0]))
    with pytest.raises(hz.HzError) as e:
        hz.hz_solve(case.pr, hz.hz_default_opts(wh_warm=1), n=case.n)  # GMRES outer
    assert e.value.status == hz.HZ_ERR_INVALID_ARG
    case.close()
