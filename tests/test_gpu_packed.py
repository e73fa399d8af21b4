"""Packed multi-problem sweep (one launch for several problems of different
meshes, degrees, frequencies and N_t) against the FP64 oracle, and against
the single-problem register-resident kernel it shares its body with.

Tolerance for FP32 against the oracle: FP32_REL = 2e-5 relative, derived in
tests/_tolerances.py."""

import numpy as np
import pytest

from oracle import dd, sem
from workloads import configs

import _tolerances as _tol
from _tolerances import FP32_REL

pytestmark = pytest.mark.gpu

# (nx, ny, sub_nx, sub_ny, P, omega): packable shapes of different sizes,
# degrees and frequencies (so different N_t), plus a non-square subdomain
MEMBERS = [
    (8, 8, 4, 4, 2, 9.0),    # (P, sub_ny) = (2, 4): 9 x 9 nodes, 2 x 2 subdomains
    (16, 8, 8, 8, 3, 21.0),  # (3, 8): 25 x 25 nodes (the benchmark's shape), 2 x 1
    (12, 12, 4, 4, 3, 14.0),  # (3, 4): 13 x 13 nodes, 3 x 3
    (8, 8, 2, 4, 5, 11.0),   # (5, 4), 11 x 21 nodes (sub_nx = 2): 4 x 2
    (16, 16, 8, 16, 1, 6.0),  # (1, 16): 9 x 17 nodes, 2 x 1
]


def _case(hz, nx, ny, sx, sy, P, omega, seed):
    from paper_2606_21695_gb300.api import Case

    wl = configs.Workload(f"pk{nx}x{ny}p{P}", (0.0, 1.0, 0.0, 1.0), nx, ny, P, sx, sy, omega, "random",
                          (0.41, 0.57), 0.08, speed_seed=seed, corr_len=0.3)
    case = Case(wl, device=0)
    m = sem.Mesh(*wl.box, nx, ny, P, sx, sy)
    gx, gy = m.coords_1d()
    pr = dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary())
    assert np.max(np.abs(case.c - pr.c)) < 1e-12
    return case, pr


def _lam(pr, seed):
    m = pr.mesh
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
    for l in range(m.L):
        for e in range(4):
            n = m.nly if e < 2 else m.nlx
            if pr.nbr[l, e] < 0:
                lam[l, e] = 0
            else:
                lam[l, e, n:] = 0
    return lam


def _dev(x):
    import torch

    a = np.ascontiguousarray(x).astype(np.complex128).reshape(-1).view(np.float64)
    return torch.from_numpy(a.copy()).cuda()


def _host(t):
    return t.cpu().numpy().view(np.complex128)


def _rel(a, b):
    return _tol.record(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _buffers(hz, case, pr, lam, with_rhs):
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
    return lin, lout, rhs, usub


def _packed(hz, members, wh, with_rhs):
    import torch

    bufs = [_buffers(hz, c, p, lam, r) for (c, p, lam, nt), r in zip(members, with_rhs)]
    hz.hz_sweep_packed([c.pr for c, _, _, _ in members], [nt for _, _, _, nt in members], wh,
                       [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs], [b[3] for b in bufs])
    torch.cuda.synchronize()
    out = []
    for (c, p, lam, nt), b in zip(members, bufs):
        m = p.mesh
        out.append((_host(b[1]).reshape(m.L, 4, m.NE), _host(b[3]).reshape(m.L, m.nly, m.nlx)))
    return out


@pytest.fixture(scope="module")
def members(hz):
    ms = []
    for k, (nx, ny, sx, sy, P, om) in enumerate(MEMBERS):
        case, pr = _case(hz, nx, ny, sx, sy, P, om, seed=20 + k)
        nt = hz.hz_problem_nt(case.pr)
        assert nt == pr.choose_nt()
        ms.append((case, pr, _lam(pr, 100 + k), nt))
    yield ms
    for c, _, _, _ in ms:
        c.close()


def test_packed_sweep_matches_oracle(hz, members):
    """One launch for all five problems, with and without their sources."""
    wh = 3
    with_rhs = [k % 2 == 0 for k in range(len(members))]
    got = _packed(hz, members, wh, with_rhs)
    for (case, pr, lam, nt), (gl, gu), r in zip(members, got, with_rhs):
        ref_l, ref_u, _ = pr.sweep(lam, pr.rhs() if r else None, nt, wh, want_u=True)
        assert np.all(np.isfinite(gl))
        assert _rel(gu, ref_u) < FP32_REL, pr.mesh.P
        assert _rel(gl, ref_l) < FP32_REL, pr.mesh.P


def test_packed_result_does_not_depend_on_the_mix(hz, members):
    """Each problem's outputs are bitwise the same swept alone or packed with
    the others (in any order)."""
    wh = 2
    alone = [_packed(hz, [m], wh, [True])[0] for m in members]
    mixed = _packed(hz, members[::-1], wh, [True] * len(members))[::-1]
    for (al, au), (ml, mu) in zip(alone, mixed):
        assert np.array_equal(al, ml)
        assert np.array_equal(au, mu)


def test_packed_equals_single_problem_warp_kernel(hz, members, monkeypatch):
    """The packed launch runs the same per-subdomain body as the
    one-problem register-resident kernel: same results to FP32 rounding of
    a different compilation (and normally bitwise)."""
    import torch

    monkeypatch.setenv("HZ_SWEEP_VARIANT", "warp")
    wh = 2
    packed = _packed(hz, members, wh, [True] * len(members))
    for (case, pr, lam, nt), (pl, pu) in zip(members, packed):
        lin, lout, rhs, usub = _buffers(hz, case, pr, lam, True)
        hz.hz_sweep(case.pr, hz.HZ_FP32_REFINE, nt, wh, 0.0, lin, lout, rhs, usub)
        torch.cuda.synchronize()
        m = pr.mesh
        assert _rel(pl, _host(lout).reshape(m.L, 4, m.NE)) < 1e-6
        assert _rel(pu, _host(usub).reshape(m.L, m.nly, m.nlx)) < 1e-6


def test_packed_rejects_unsupported_shapes(hz):
    """More than 32 node columns, or a (degree, sub_ny) pair without a packed
    variant: HZ_ERR_UNSUPPORTED and nothing launched."""
    import torch

    for nx, ny, sx, sy, P in [(16, 8, 16, 4, 3), (8, 8, 4, 4, 6)]:
        case, pr = _case(hz, nx, ny, sx, sy, P, 5.0, seed=7)
        nt = hz.hz_problem_nt(case.pr)
        lin, lout, rhs, usub = _buffers(hz, case, pr, _lam(pr, 1), False)
        before = hz.hz_kernel_launches()
        with pytest.raises(hz.HzError) as e:
            hz.hz_sweep_packed([case.pr], [nt], 2, [lin], [lout])
        assert e.value.status == hz.HZ_ERR_UNSUPPORTED
        assert hz.hz_kernel_launches() == before
        torch.cuda.synchronize()
        case.close()


def test_packed_sweep_with_generalised_transmission(hz):
    """A member with the generalised interface condition (eta = 0.3,
    zeta = 0.8) in a packed launch, against the oracle."""
    from paper_2606_21695_gb300.api import Case

    nx, ny, sx, sy, P, om = MEMBERS[2]
    wl = configs.Workload("pkr", (0.0, 1.0, 0.0, 1.0), nx, ny, P, sx, sy, om, "random", (0.41, 0.57), 0.08,
                          speed_seed=31, corr_len=0.3)
    case = Case(wl, device=0)
    hz.hz_problem_set(case.pr, hz.HZ_TRANSMISSION, np.array([0.3, 0.8]))
    m = sem.Mesh(*wl.box, nx, ny, P, sx, sy)
    gx, gy = m.coords_1d()
    pr = dd.Problem(m, wl.speed(gx, gy), wl.omega, wl.source(gx, gy), wl.boundary(), robin=(0.3, 0.8))
    nt = hz.hz_problem_nt(case.pr)
    lam = _lam(pr, 77)
    (gl, gu), = _packed(hz, [(case, pr, lam, nt)], 3, [True])
    ref_l, ref_u, _ = pr.sweep(lam, pr.rhs(), nt, 3, want_u=True)
    assert _rel(gu, ref_u) < FP32_REL and _rel(gl, ref_l) < FP32_REL
    case.close()
