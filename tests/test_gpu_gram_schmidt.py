"""Gram-Schmidt passes of the Arnoldi step (opts.gs_passes): one classical
pass and two (one reorthogonalisation) both reach the global FP64 tolerance,
agree with each other and with the oracle's direct solve, and other values
are refused."""

import numpy as np
import pytest

from oracle import dd, sem
from workloads import configs

pytestmark = pytest.mark.gpu


def _wl():
    return configs.Workload("gsp", (0, 1, 0, 1), 24, 24, 3, 4, 4, 26.0, "channel", (0.45, 0.3), 0.03)


@pytest.mark.parametrize("precision", ["fp32_refine", "fp64"])
def test_one_and_two_passes_reach_the_tolerance_and_agree(hz, precision):
    from paper_2606_21695_gb300.api import Case

    wl = _wl()
    case = Case(wl)
    prec = hz.HZ_FP32_REFINE if precision == "fp32_refine" else hz.HZ_FP64
    sols, reps = {}, {}
    for passes in (1, 2):
        o = hz.hz_default_opts(precision=prec, tol=1e-9, gs_passes=passes)
        st, u, rep = hz.hz_solve(case.pr, o, n=case.n)
        assert st == hz.HZ_OK and rep["rel_residual"] <= 1e-9, (passes, rep)
        sols[passes], reps[passes] = u.copy(), rep
    # both stop at a relative residual of 1e-9 of the same FP64 system
    scale = np.max(np.abs(sols[2]))
    assert np.max(np.abs(sols[1] - sols[2])) <= 1e-6 * scale
    # the direct solve of the oracle's assembled system
    m = sem.Mesh(*wl.box, wl.nx, wl.ny, wl.P, wl.sub_nx, wl.sub_ny)
    gx, gy = m.coords_1d()
    pr = dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary())
    ref = pr.direct_solve()
    assert np.max(np.abs(sols[1] - ref.ravel())) <= 1e-6 * np.max(np.abs(ref))
    # one pass costs at most a few more iterations here
    assert reps[1]["gmres_iters"] <= 1.2 * reps[2]["gmres_iters"] + 5
    case.close()


@pytest.mark.parametrize("bad", [0, 3, -1])
def test_other_pass_counts_are_refused(hz, bad):
    from paper_2606_21695_gb300.api import Case

    case = Case(_wl())
    with pytest.raises(hz.HzError) as e:
        hz.hz_solve(case.pr, hz.hz_default_opts(gs_passes=bad), n=case.n)
    assert e.value.status == hz.HZ_ERR_INVALID_ARG
    case.close()
