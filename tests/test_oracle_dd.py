"""Pins of the oracle's WaveHoltz + domain-decomposition pieces.

* Pi(u*) = u*  -- exact evolution of e^{-i w t} by the modified leapfrog plus
  the filter (Sec. 5): pins the leapfrog, filter sign and 2/N_t scaling.
* WaveHoltz -> dense solve of the subdomain system (Sec. 5, fixed point).
* DD fixed point == sparse direct global solve (Sec. 3, eq.
  (lambda-iteration) with the -2ik reading, cross points included).
* plane wave e^{ik d.x}: O(h^{P+1}) convergence (Sec. 2 and 4 as a whole).
* interface continuity, plain == GMRES, linearity of the sweep, N_t rule.
Negative controls plant a mistake in the oracle (CPU only) and show the pin
catches it.
"""

import math

import numpy as np
import pytest

from oracle import dd, sem
from workloads import fields


def _problem(nx, ny, sx, sy, P, omega=6.0, seed=0, box=(0.0, 1.0, 0.0, 1.0), g=True, var_c=True, robin=(0.0, 1.0)):
    m = sem.Mesh(*box, nx, ny, P, sx, sy)
    X, Y = m.coords()
    rng = np.random.default_rng(seed)
    c = 1.0 + (0.3 * np.sin(2.1 * X + 0.4) * np.cos(1.7 * Y) if var_c else 0.0 * X)
    f = fields.gaussian_source(X, Y, (0.37, 0.61), 0.15) * (1.0 + 0.5j)
    gg = None
    if g:
        gg = {k: rng.standard_normal(n) + 1j * rng.standard_normal(n)
              for k, n in (("S", m.NX), ("N", m.NX), ("W", m.NY), ("E", m.NY))}
    return dd.Problem(m, c, omega, f, gg, robin=robin)


@pytest.mark.parametrize("P,Nt", [(1, 7), (2, 12), (3, 40), (4, 25)])
def test_waveholtz_exact_fixed_point(P, Nt):
    """b := K_l u* for random complex u*; one WaveHoltz iteration from u*
    returns u* (to rounding) for any N_t >= 3 satisfying the CFL rule."""
    pr = _problem(4, 4, 2, 2, P, omega=5.0, seed=P)
    Nt = max(Nt, pr.choose_nt())
    rng = np.random.default_rng(10 + P)
    m = pr.mesh
    subs = np.arange(m.L)
    us = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    b = np.stack([(pr.sub_matrix(l) @ us[l].ravel()).reshape(us[l].shape) for l in subs])
    u1, _ = pr.waveholtz(b, Nt, 1, u0=us, subs=subs)
    assert np.max(np.abs(u1 - us)) < 1e-11 * np.max(np.abs(us))


def test_waveholtz_fixed_point_negative_control():
    """Plant Algorithm 1's printed filter sign (+1/(i w) on the p-dot term) in
    a copy of the oracle loop: Pi(u*) = u* then fails by O(1)."""
    pr = _problem(4, 4, 2, 2, 2, omega=5.0)
    Nt = pr.choose_nt()
    m = pr.mesh
    rng = np.random.default_rng(3)
    us = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    b = np.stack([(pr.sub_matrix(l) @ us[l].ravel()).reshape(us[l].shape) for l in range(m.L)])
    u_good, _ = pr.waveholtz(b, Nt, 1, u0=us)
    w = pr.omega
    alpha, beta, sigma = pr.leapfrog_coeffs(Nt)
    c0 = -0.25 + 0.25 * math.tan(math.pi / Nt) ** 2

    def kap(nu):
        return math.cos(2 * math.pi * nu / Nt) + c0

    p = us.real.copy()
    pd = (-1j * w * us * np.exp(-1j * math.pi / Nt)).real
    v = kap(0) * p - (1j / w) * kap(0.5) * pd
    for nu in range(1, Nt):
        p = p + sigma * pd
        pd = alpha * pd + beta * (-pr.apply_A_sub(p) + (b * np.exp(-2j * math.pi * nu / Nt)).real)
        v = v + kap(nu) * p - (1j / w) * kap(nu + 0.5) * pd
    u_bad = (2.0 / Nt) * v
    assert np.max(np.abs(u_good - us)) < 1e-11 * np.max(np.abs(us))
    assert np.max(np.abs(u_bad - us)) > 1e-2 * np.max(np.abs(us))


def test_waveholtz_converges_to_dense_subdomain_solve():
    pr = _problem(4, 4, 2, 2, 2, omega=4.0, seed=4)
    m = pr.mesh
    rng = np.random.default_rng(5)
    b = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    exact = np.stack([np.linalg.solve(pr.sub_matrix(l).toarray(), b[l].ravel()).reshape(b[l].shape)
                      for l in range(m.L)])
    u, it = pr.waveholtz(b, pr.choose_nt(), 80)
    err = np.max(np.abs(u - exact)) / np.max(np.abs(exact))
    assert err < 1e-10, err
    u5, _ = pr.waveholtz(b, pr.choose_nt(), 5)
    assert np.max(np.abs(u5 - exact)) / np.max(np.abs(exact)) > err


@pytest.mark.parametrize("robin", [(0.4, 0.7), (1.0, 1.5)])
def test_waveholtz_with_interface_boundary_mass_converges_to_dense_solve(robin):
    """Generalised interface condition d_n + k (eta - i zeta): the subdomain
    operator gains zeta-scaled damping and a boundary mass on interface
    edges; WaveHoltz with the boundary mass in the time stepping converges
    to the dense solve of that operator, and Pi(u*) = u* holds exactly."""
    pr = _problem(4, 4, 2, 2, 2, omega=4.0, seed=4, robin=robin)
    m = pr.mesh
    assert np.max(pr.Hm_sub) > 0
    rng = np.random.default_rng(5)
    b = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    exact = np.stack([np.linalg.solve(pr.sub_matrix(l).toarray(), b[l].ravel()).reshape(b[l].shape)
                      for l in range(m.L)])
    u, _ = pr.waveholtz(b, pr.choose_nt(), 120)
    assert np.max(np.abs(u - exact)) / np.max(np.abs(exact)) < 1e-9
    u1, _ = pr.waveholtz(b, pr.choose_nt(), 1, u0=exact)
    assert np.max(np.abs(u1 - exact)) < 1e-11 * np.max(np.abs(exact))


LAYOUTS = [
    (4, 4, 2, 2, 2),  # 2x2 subdomains, one cross point
    (6, 6, 2, 2, 1),  # 3x3, four cross points, P = 1
    (4, 2, 1, 2, 3),  # 4x1 strips
    (3, 6, 3, 2, 2),  # 1x3 strips
    (4, 4, 1, 1, 2),  # 4x4 single-element subdomains
    (4, 6, 2, 3, 4),  # non-square subdomains, P = 4
]


@pytest.mark.parametrize("nx,ny,sx,sy,P", LAYOUTS)
def test_dd_fixed_point_equals_global_direct_solve(nx, ny, sx, sy, P):
    pr = _problem(nx, ny, sx, sy, P, omega=7.0, seed=nx + P)
    ud = pr.direct_solve()
    u, info = pr.dd_solve(pr.rhs(), outer="gmres", restart=200, tol=1e-13, max_sweeps=400, inner="direct")
    err = np.linalg.norm(u - ud) / np.linalg.norm(ud)
    assert err < 1e-10, (err, info["sweeps"])
    # interface continuity of the subdomain copies at the converged lambda
    us = info["u_sub"]
    m = pr.mesh
    for l in range(m.L):
        for e in range(4):
            r = pr.nbr[l, e]
            if r < 0:
                continue
            rows, cols, _ = pr.edge_nodes(e)
            rr, rc, _ = pr.edge_nodes(dd.OPPOSITE[e])
            assert np.max(np.abs(us[l, rows, cols] - us[r, rr, rc])) < 1e-9 * np.max(np.abs(ud))


@pytest.mark.parametrize("robin", [(0.3, 0.8), (0.5, 1.3)])
@pytest.mark.parametrize("nx,ny,sx,sy,P", [(4, 4, 2, 2, 2), (6, 6, 2, 2, 1), (4, 6, 2, 3, 4)])
def test_dd_fixed_point_with_generalised_transmission_condition(nx, ny, sx, sy, P, robin):
    """Interface condition d_n + k (eta - i zeta) with update
    lambda_r = -lambda_l + 2k(eta - i zeta) u: the DD fixed point is still the
    global discrete solution (cross points included), the iteration count is
    what changes."""
    pr = _problem(nx, ny, sx, sy, P, omega=7.0, seed=nx + P, robin=robin)
    ud = pr.direct_solve()
    u, info = pr.dd_solve(pr.rhs(), outer="gmres", restart=200, tol=1e-13, max_sweeps=400, inner="direct")
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-10, info["sweeps"]


def test_generalised_condition_negative_control():
    """Plant a wrong update (the eta term with the opposite sign): the DD
    fixed point is no longer the global solution."""
    pr = _problem(4, 4, 2, 2, 2, omega=7.0, seed=6, robin=(0.5, 1.0))
    ud = pr.direct_solve()
    orig = dd.Problem.sweep

    def wrong(self, lam_in, *a, **k):
        k2 = dict(k)
        k2["want_u"] = True
        lam_out, u, it = orig(self, lam_in, *a, **k2)
        w = self.omega
        for e in range(4):
            rows, cols, _ = self.edge_nodes(e)
            n = len(rows)
            for l in np.where(self.nbr[:, e] >= 0)[0]:
                r = self.nbr[l, e]
                kk = w / self.c_sub[l, rows, cols]
                lam_out[r, dd.OPPOSITE[e], :n] -= 4 * kk * self.eta * u[l, rows, cols]
        return (lam_out, u, it) if k.get("want_u", False) else lam_out

    u_ok, _ = pr.dd_solve(pr.rhs(), restart=200, tol=1e-13, max_sweeps=400, inner="direct")
    assert np.linalg.norm(u_ok - ud) / np.linalg.norm(ud) < 1e-10
    dd.Problem.sweep = wrong
    try:
        u_bad, _ = pr.dd_solve(pr.rhs(), restart=200, tol=1e-13, max_sweeps=400, inner="direct")
    finally:
        dd.Problem.sweep = orig
    assert np.linalg.norm(u_bad - ud) / np.linalg.norm(ud) > 1e-3


def test_dd_paper_sign_does_not_give_global_solution(monkeypatch):
    """Negative control: the printed +2ik update converges to something that
    is not the discrete Helmholtz solution (or does not converge)."""
    pr = _problem(4, 4, 2, 2, 2, omega=7.0, seed=1)
    ud = pr.direct_solve()
    orig = dd.Problem.sweep

    def plus_sign(self, lam_in, *a, **k):
        want_u = k.get("want_u", False)
        res = orig(self, lam_in, *a, **k)
        lam_out = res[0] if want_u else res
        # undo -2iku and apply +2iku:  new = -lam_in + 2iku  = lam_out + 4iku
        k2 = dict(k)
        k2["want_u"] = True
        _, u, _ = orig(self, lam_in, *a, **k2)
        fixed = np.zeros_like(lam_out)
        for l in range(self.mesh.L):
            for e in range(4):
                r = self.nbr[l, e]
                if r < 0:
                    continue
                rows, cols, _ = self.edge_nodes(e)
                n = len(rows)
                kk = self.omega / self.c_sub[l, rows, cols]
                fixed[r, dd.OPPOSITE[e], :n] = lam_out[r, dd.OPPOSITE[e], :n] + 4j * kk * u[l, rows, cols]
        return (fixed,) + tuple(res[1:]) if want_u else fixed

    monkeypatch.setattr(dd.Problem, "sweep", plus_sign)
    u, _ = pr.dd_solve(pr.rhs(), restart=200, tol=1e-13, max_sweeps=300, inner="direct")
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) > 1e-3


def test_dd_with_waveholtz_inner_and_refinement_reaches_direct_solution():
    pr = _problem(8, 8, 4, 4, 3, omega=10.0, seed=2)
    ud = pr.direct_solve()
    u, info = pr.solve(m_wh=5, tol=1e-11, inner_tol=1e-9, restart=60, max_refine=12)
    assert info["rel_residual"] <= 1e-11
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-8


def test_fgmres_refinement_reaches_direct_solution():
    """Flexible GMRES around inexact DD solves (5 WaveHoltz iterations, DD
    solves stopped at 1e-2): the same global solution as the direct solve."""
    pr = _problem(8, 8, 4, 4, 3, omega=10.0, seed=2)
    ud = pr.direct_solve()
    u, info = pr.solve(m_wh=5, tol=1e-11, inner_tol=1e-2, restart=60, max_refine=40, refine="fgmres",
                       refine_restart=20)
    assert info["rel_residual"] <= 1e-11, info["hist"]
    assert np.linalg.norm(pr.residual(u)) <= 1.0001e-11 * np.linalg.norm(pr.rhs())
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-8
    assert info["refinements"] <= 40 and info["sweeps"] > 0


def test_real_gmres_reaches_inexact_fixed_point():
    """With a fixed WaveHoltz count the DD map is real-linear; real GMRES on
    the interleaved vector converges to its fixed point (checked against the
    plain fixed-point iteration), complex GMRES stalls above it."""
    pr = _problem(4, 2, 2, 2, 2, omega=5.0, seed=8)
    Nt = pr.choose_nt()
    ur, ir = pr.dd_solve(pr.rhs(), Nt=Nt, m_wh=2, outer="rgmres", restart=200, tol=1e-13, max_sweeps=300)
    up, ip = pr.dd_solve(pr.rhs(), Nt=Nt, m_wh=2, outer="plain", tol=1e-14, max_sweeps=4000)
    assert np.linalg.norm(ur - up) / np.linalg.norm(up) < 1e-9, (ir["sweeps"], ip["sweeps"])


def test_plain_and_gmres_outer_agree():
    pr = _problem(4, 2, 2, 2, 2, omega=5.0, seed=7)
    ug, _ = pr.dd_solve(pr.rhs(), outer="gmres", restart=100, tol=1e-13, max_sweeps=200, inner="direct")
    up, info = pr.dd_solve(pr.rhs(), outer="plain", tol=1e-13, max_sweeps=3000, inner="direct")
    assert np.linalg.norm(ug - up) / np.linalg.norm(ug) < 1e-9, info["sweeps"]


def test_homogeneous_sweep_is_linear_and_subset_consistent():
    pr = _problem(6, 4, 2, 2, 2, omega=6.0, seed=3)
    m = pr.mesh
    rng = np.random.default_rng(9)
    shape = (m.L, 4, m.NE)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    y = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    Nt = pr.choose_nt()
    # a fixed number of WaveHoltz iterations is real-linear in lambda ...
    a = -1.7
    lhs = pr.sweep(a * x + y, None, Nt, 3)
    rhs = a * pr.sweep(x, None, Nt, 3) + pr.sweep(y, None, Nt, 3)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    # ... but not complex-linear (WaveHoltz evolves Re w only) ...
    ci = pr.sweep(1j * x, None, Nt, 3)
    assert np.max(np.abs(ci - 1j * pr.sweep(x, None, Nt, 3))) > 1e-4 * np.max(np.abs(ci))
    # ... while an exact subdomain solve is complex-linear
    a = 0.7 - 1.3j
    lhs = pr.sweep(a * x + y, None, Nt, inner="direct")
    rhs = a * pr.sweep(x, None, Nt, inner="direct") + pr.sweep(y, None, Nt, inner="direct")
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))
    full, uf, _ = pr.sweep(x, pr.rhs(), Nt, 3, want_u=True)
    sub, us, _ = pr.sweep(x, pr.rhs(), Nt, 3, want_u=True, subset=[1, 4])
    for l in (1, 4):
        np.testing.assert_allclose(us[l], uf[l], rtol=0, atol=1e-14 * np.max(np.abs(uf)))
        for e in range(4):
            r = pr.nbr[l, e]
            if r >= 0:
                o = dd.OPPOSITE[e]
                np.testing.assert_allclose(sub[r, o], full[r, o], rtol=0, atol=1e-14 * np.max(np.abs(full)))


@pytest.mark.parametrize("P,rate_min", [(1, 1.7), (2, 2.7), (3, 3.7)])
def test_plane_wave_convergence_order(P, rate_min):
    """u = exp(i k d.x), c = 1, f = 0, g = (d_n - ik) u = ik(d.n - 1) u on each
    edge.  The discrete solution converges at O(h^{P+1}) in the mass norm."""
    k = 6.0
    th = 0.4
    d = (math.cos(th), math.sin(th))
    errs = []
    for n in (4, 8, 16):
        m = sem.Mesh(0, 1, 0, 1, n, n, P, n, n)
        X, Y = m.coords()
        gx, gy = m.coords_1d()
        ue = lambda x, y: np.exp(1j * k * (d[0] * x + d[1] * y))  # noqa: E731
        g = {
            "S": 1j * k * (-d[1] - 1) * ue(gx, 0 * gx),
            "N": 1j * k * (d[1] - 1) * ue(gx, 0 * gx + 1),
            "W": 1j * k * (-d[0] - 1) * ue(0 * gy, gy),
            "E": 1j * k * (d[0] - 1) * ue(0 * gy + 1, gy),
        }
        pr = dd.Problem(m, np.ones_like(X), k, 0 * X, g)
        u = pr.direct_solve()
        e = u - ue(X, Y)
        errs.append(math.sqrt(np.sum(pr.W2 * np.abs(e) ** 2)))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate >= rate_min, (errs, rate)


def test_nt_rule_matches_2d_operator_and_is_stable():
    """lx + ly equals the largest eigenvalue of M^-1 A for the 2D subdomain
    (tensor-product identity, c = 1); the chosen N_t gives a bounded
    leapfrog, a step 10% above the limit does not."""
    pr = _problem(4, 4, 2, 2, 3, omega=3.0, var_c=False, g=False)
    m = pr.mesh
    A = pr.sub_matrix(0)  # complex; rebuild real A
    A = pr._A_sub.toarray()
    Ws = np.outer(pr.Wys, pr.Wxs).ravel()
    lam2d = np.max(np.linalg.eigvals(A / Ws[:, None]).real)
    lx = dd._max_gen_eig_1d(m, m.sub_nx, m.hx)
    ly = dd._max_gen_eig_1d(m, m.sub_ny, m.hy)
    assert abs(lam2d - (lx + ly)) < 1e-10 * lam2d
    Nt = pr.choose_nt()
    rng = np.random.default_rng(0)
    b = rng.standard_normal((m.L, m.nly, m.nlx)) + 0j
    u_ok, _ = pr.waveholtz(b, Nt, 3)
    assert np.all(np.isfinite(u_ok)) and np.max(np.abs(u_ok)) < 1e3 * np.max(np.abs(b))
    # a time step beyond the limit: sigma*sqrt(lam) > 2.2
    T = 2 * math.pi / pr.omega
    nt_bad = max(3, int(T * math.sqrt(lam2d) / 2.3))
    u_bad, _ = pr.waveholtz(b, nt_bad, 3)
    assert not np.all(np.isfinite(u_bad)) or np.max(np.abs(u_bad)) > 1e6 * np.max(np.abs(u_ok))


def test_single_subdomain_and_zero_rhs():
    pr = _problem(3, 3, 3, 3, 2, omega=4.0)
    u, info = pr.dd_solve(pr.rhs(), inner="direct")
    np.testing.assert_allclose(u, pr.direct_solve(), rtol=1e-12, atol=1e-14)
    z, info = pr.dd_solve(0 * pr.rhs())
    assert np.all(z == 0)


def test_warm_started_waveholtz_plain_iteration():
    """Warm start (each sweep's WaveHoltz from the previous sweep's subdomain
    solutions, plain fixed-point iteration, tolerance-controlled WaveHoltz):
    the same fixed point -- the global direct solve -- with fewer WaveHoltz
    iterations than cold starts from zero."""
    pr = _problem(4, 2, 2, 2, 2, omega=4.0, seed=11)  # two subdomains: the plain iteration converges
    b = pr.rhs()
    ud = pr.direct_solve()
    res = {}
    for warm in (False, True):
        u, info = pr.dd_solve(b, outer="plain", m_wh=80, wh_tol=1e-10, tol=1e-7, max_sweeps=300, warm=warm)
        assert np.max(np.abs(u - ud)) < 1e-5 * np.max(np.abs(ud)), warm
        res[warm] = info
    assert res[True]["wh_iters"] < 0.7 * res[False]["wh_iters"], (res[True]["wh_iters"], res[False]["wh_iters"])
    # the outer iterates agree to the WaveHoltz tolerance, so the sweep counts match
    assert abs(res[True]["sweeps"] - res[False]["sweeps"]) <= 2


def test_nested_dissection_direct_solve_equals_plain_direct_solve():
    """The nested-dissection ordered LU (used for the larger test meshes) is a
    permutation of the node grid and gives the plain sparse direct solve's
    result; its separators are element-boundary node lines, which the
    stiffness does not couple across."""
    from oracle.sem import nested_dissection_order

    m = sem.Mesh(0, 1, 0, 1, 12, 10, 3, 4, 5)
    X, Y = m.coords()
    pr = dd.Problem(m, 1.0 + 0.3 * np.sin(4 * X) * np.cos(3 * Y), 17.0, np.exp(-40 * ((X - .4) ** 2 + (Y - .6) ** 2)))
    perm = nested_dissection_order(m.NX, m.NY, m.P, leaf=16)
    assert np.array_equal(np.sort(perm), np.arange(m.NX * m.NY))
    ud = pr.direct_solve()
    un = pr.direct_solve(ordering="nd")
    assert np.max(np.abs(un - ud)) <= 1e-12 * np.max(np.abs(ud))
    b = pr.rhs()
    assert np.linalg.norm(pr.residual(un, b)) <= 1e-13 * np.linalg.norm(b)
    # an element-boundary column separates: no stiffness coupling across it
    K = pr.matrix().tocoo()
    I0, I1 = K.row % m.NX, K.col % m.NX
    s = 2 * m.P
    assert not np.any((I0 < s) & (I1 > s)) and not np.any((I0 > s) & (I1 < s))
