"""CUDA graphs of the Arnoldi step's vector work: a solve with the graphs
replays exactly the launches of the solve without them (bitwise equal
solutions, same sweep and iteration counts, same number of kernels), also
on a second solve that reuses the captured graphs."""

import numpy as np
import pytest

from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("outer", ["gmres", "rgmres"])
@pytest.mark.parametrize("gs_passes", [1, 2])
def test_graphs_replay_the_same_launches(hz, outer, gs_passes):
    from paper_2606_21695_gb300.api import Case

    case = Case(configs.Workload("gr", (0, 1, 0, 1), 16, 16, 3, 4, 4, 17.0, "channel", (0.45, 0.3), 0.03))
    out = hz.HZ_OUTER_GMRES if outer == "gmres" else hz.HZ_OUTER_RGMRES
    res = {}
    # the first solve of a shape also runs the autotuner: keep it out of the counts
    hz.hz_solve(case.pr, hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8, outer=out), n=case.n)
    for graphs in (0, 1, 1):  # the second graphs=1 solve replays the cached graphs
        o = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8, gmres_restart=12, outer=out, graphs=graphs,
                               gs_passes=gs_passes)
        k0 = hz.hz_kernel_launches()
        st, u, rep = hz.hz_solve(case.pr, o, n=case.n)
        assert st == hz.HZ_OK and rep["rel_residual"] <= 1e-8
        res.setdefault(graphs, []).append((u.copy(), rep, hz.hz_kernel_launches() - k0))
    (u0, r0, k0), = res[0]
    for u1, r1, k1 in res[1]:
        assert np.array_equal(u0, u1)
        assert (r1["sweeps"], r1["gmres_iters"], r1["refinements"]) == (r0["sweeps"], r0["gmres_iters"],
                                                                        r0["refinements"])
        assert k1 == k0
    case.close()


def test_device_solve_on_default_and_side_streams(hz):
    """hz_solve_device on the default stream (joined by events, solved on the
    problem's stream with the step graphs) and on a side stream give the
    solution of hz_solve bitwise."""
    import torch

    from paper_2606_21695_gb300.api import Case

    case = Case(configs.Workload("gs", (0, 1, 0, 1), 16, 16, 2, 4, 4, 11.0, "random", (0.5, 0.4), 0.04,
                                 corr_len=0.3))
    o = hz.hz_default_opts(precision=hz.HZ_FP32_REFINE, tol=1e-8, gmres_restart=10)
    st, ref, _ = hz.hz_solve(case.pr, o, n=case.n)
    assert st == hz.HZ_OK
    side = torch.cuda.Stream()
    for stream in (None, torch.cuda.current_stream(), side):
        u = torch.full((2 * case.n,), float("nan"), dtype=torch.float64, device="cuda")
        st, rep = hz.hz_solve_device(case.pr, o, u, stream)
        torch.cuda.synchronize()
        assert st == hz.HZ_OK
        assert np.array_equal(u.cpu().numpy().view(np.complex128), ref)
    case.close()
