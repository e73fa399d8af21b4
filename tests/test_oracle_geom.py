"""Pins of the oracle's general-quadrilateral (mapped) discretisation
(oracle/geom.py), each against something other than the code itself:

* identity map == the tensor-product Cartesian oracle (an independent code
  path: 1D stiffness products and lumped 1D weights);
* rotation invariance (the Laplacian, lumped mass and edge lengths of a
  rotated mesh are those of the unrotated one);
* affine (sheared) mesh: patch test A(a x + b y) = 0 on interior nodes, the
  energy product v^T A u = integral of grad u . grad v for quadratics, area
  and edge lengths, all exact (GLL is exact for these integrands);
* curved mesh: A symmetric, A 1 = 0; quarter-annulus area converges;
* plane wave e^{ik d.x} on a curved mesh: O(h^{P+1}) convergence;
* DD fixed point (direct subdomain solves + GMRES) == global direct solve on
  a curved mesh with variable c (per-subdomain edge weights, cross points);
* WaveHoltz exact fixed point Pi(u*) = u* on curved subdomains.
A negative control drops the cross term G12 and shows the energy pin fails.
"""

import math

import numpy as np
import pytest

from oracle import dd, geom, sem
from workloads import fields


def _rand_g(m, rng):
    return {k: rng.standard_normal(n) + 1j * rng.standard_normal(n)
            for k, n in (("S", m.NX), ("N", m.NX), ("W", m.NY), ("E", m.NY))}


def _fields(X, Y):
    c = 1.0 + 0.3 * np.sin(2.1 * X + 0.4) * np.cos(1.7 * Y)
    f = fields.gaussian_source(X, Y, (0.37, 0.61), 0.15) * (1.0 + 0.5j)
    return c, f


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_identity_map_equals_cartesian_oracle():
    m = sem.Mesh(0, 1.3, 0, 0.9, 6, 4, 3, 3, 2)
    X, Y = m.coords()
    c, f = _fields(X, Y)
    g = _rand_g(m, np.random.default_rng(1))
    ref = dd.Problem(m, c, 7.0, f, g)
    mp = geom.MappedProblem(m, X, Y, c, 7.0, f, g)
    assert _rel(mp.W2, ref.W2) < 1e-13 and _rel(mp.Hdiag, ref.Hdiag) < 1e-13
    assert _rel(mp.rhs(), ref.rhs()) < 1e-13
    rng = np.random.default_rng(2)
    u = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
    assert _rel(mp.apply_K(u), ref.apply_K(u)) < 1e-12
    assert _rel(mp.M_sub, ref.M_sub) < 1e-13 and _rel(mp.H_sub, ref.H_sub) < 1e-13
    assert _rel(mp.share, ref.share) < 1e-13
    lam = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
    a = mp.sweep(lam, mp.rhs(), Nt=20, m_wh=2)
    b = ref.sweep(lam, ref.rhs(), Nt=20, m_wh=2)
    assert _rel(a, b) < 1e-11


def test_rotation_invariance():
    m = sem.Mesh(0, 1, 0, 1, 4, 4, 2, 2, 2)
    X, Y = m.coords()
    c, f = _fields(X, Y)
    g = _rand_g(m, np.random.default_rng(3))
    th = 0.7
    Xr = math.cos(th) * X - math.sin(th) * Y + 0.2
    Yr = math.sin(th) * X + math.cos(th) * Y - 0.1
    ref = dd.Problem(m, c, 5.0, f, g)
    mp = geom.MappedProblem(m, Xr, Yr, c, 5.0, f, g)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
    assert _rel(mp.apply_K(u), ref.apply_K(u)) < 1e-12
    assert _rel(mp.rhs(), ref.rhs()) < 1e-12
    lam = rng.standard_normal((m.L, 4, m.NE)) + 1j * rng.standard_normal((m.L, 4, m.NE))
    assert _rel(mp.sweep(lam, None, Nt=15, m_wh=2), ref.sweep(lam, None, Nt=15, m_wh=2)) < 1e-11


def _sheared(P=3, G12_zero=False):
    m = sem.Mesh(0, 1, 0, 1, 4, 3, P, 2, 3)
    X0, Y0 = m.coords()
    X, Y = X0 + 0.35 * Y0, 0.8 * Y0
    met = list(geom.metric(X, Y, m.P, m.D, m.w, m.nx, m.ny))
    if G12_zero:
        met[2] = 0 * met[2]
    return m, X, Y, met


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_affine_patch_test_area_and_edges(P):
    m, X, Y, (Jw, G11w, G12w, G22w, s_xi, s_eta) = _sheared(P)
    u = 0.7 * X - 1.9 * Y + 0.3
    Au = geom.stiffness_apply(u, m.P, m.D, G11w, G12w, G22w)
    assert np.max(np.abs(Au[1:-1, 1:-1])) < 1e-12 * np.max(np.abs(Au))
    assert abs(np.sum(Jw) - 0.8) < 1e-13
    bw = geom.block_edge_weights(m.P, m.w, s_xi, s_eta)
    assert abs(np.sum(bw["S"]) - 1.0) < 1e-13 and abs(np.sum(bw["N"]) - 1.0) < 1e-13
    assert abs(np.sum(bw["W"]) - math.hypot(0.35, 0.8)) < 1e-13
    if P >= 2:
        assert abs(_energy_xy_x2(m, X, Y, G11w, G12w, G22w) - _ENERGY_EXACT) < 1e-12


# v^T A u for u = x y, v = x^2 on the parallelogram {(s + 0.35 t, 0.8 t)}:
# integral of grad u . grad v = 2 x y over it = 1.28 (1/4 + 0.35/3), exact for
# P >= 2 (quadratics are in the space, the integrand is quadratic in xi, eta)
_ENERGY_EXACT = 1.28 * (0.25 + 0.35 / 3.0)


def _energy_xy_x2(m, X, Y, G11w, G12w, G22w):
    u, v = X * Y, X * X
    return float(np.sum(v * geom.stiffness_apply(u, m.P, m.D, G11w, G12w, G22w)))


def test_negative_control_energy_pin_catches_dropped_cross_term():
    """A planted mistake (G12 dropped) keeps the linear patch test (any
    constant tensor passes it) but breaks the exact energy product."""
    m, X, Y, (Jw, G11w, G12w, G22w, s_xi, s_eta) = _sheared(3, G12_zero=True)
    assert abs(_energy_xy_x2(m, X, Y, G11w, G12w, G22w) - _ENERGY_EXACT) > 1e-2


def test_curved_symmetry_and_constants():
    m = sem.Mesh(0, 1, 0, 1, 4, 4, 3, 2, 2)
    X, Y = fields.warp_nodes(*m.coords(), (0, 1, 0, 1), 0.08)
    _, G11w, G12w, G22w, _, _ = geom.metric(X, Y, m.P, m.D, m.w, m.nx, m.ny)
    A = geom.stiffness_matrix(m.P, m.D, G11w, G12w, G22w).toarray()
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-12 * np.max(np.abs(A))
    # the element form applied matrix-free equals the assembled matrix
    u = np.random.default_rng(5).standard_normal(X.shape)
    assert _rel(geom.stiffness_apply(u, m.P, m.D, G11w, G12w, G22w).ravel(), A @ u.ravel()) < 1e-13


def test_quarter_annulus_area_converges():
    errs = []
    for P in (2, 4, 6):
        m = sem.Mesh(0, 1, 0, 1, 3, 3, P, 3, 3)
        S, T = m.coords()
        r, th = 1.0 + S, 0.5 * math.pi * T
        X, Y = r * np.cos(th), r * np.sin(th)
        Jw = geom.metric(X, Y, m.P, m.D, m.w, m.nx, m.ny)[0]
        errs.append(abs(np.sum(Jw) - 0.75 * math.pi))
    assert errs[0] < 1e-3 and errs[2] < 1e-9 and errs[2] < errs[1] < errs[0]


@pytest.mark.parametrize("P,rate_min", [(2, 2.6), (3, 3.5)])
def test_plane_wave_convergence_on_curved_mesh(P, rate_min):
    k, th = 6.0, 0.4
    d = (math.cos(th), math.sin(th))
    errs = []
    for n in (4, 8, 16):
        m = sem.Mesh(0, 1, 0, 1, n, n, P, n, n)
        X, Y = fields.warp_nodes(*m.coords(), (0, 1, 0, 1), 0.06)
        gx, gy = m.coords_1d()
        ue = lambda x, y: np.exp(1j * k * (d[0] * x + d[1] * y))  # noqa: E731
        g = {"S": 1j * k * (-d[1] - 1) * ue(gx, 0 * gx), "N": 1j * k * (d[1] - 1) * ue(gx, 0 * gx + 1),
             "W": 1j * k * (-d[0] - 1) * ue(0 * gy, gy), "E": 1j * k * (d[0] - 1) * ue(0 * gy + 1, gy)}
        pr = geom.MappedProblem(m, X, Y, np.ones_like(X), k, 0 * X, g)
        e = pr.direct_solve() - ue(X, Y)
        errs.append(math.sqrt(np.sum(pr.W2 * np.abs(e) ** 2)))
    rate = math.log2(errs[-2] / errs[-1])
    assert rate >= rate_min, (errs, rate)


def test_dd_fixed_point_equals_direct_on_curved_mesh():
    m = sem.Mesh(0, 1, 0, 1, 8, 8, 2, 4, 4)
    X, Y = fields.warp_nodes(*m.coords(), (0, 1, 0, 1), 0.07)
    c, f = _fields(X, Y)
    pr = geom.MappedProblem(m, X, Y, c, 9.0, f, _rand_g(m, np.random.default_rng(6)))
    u, info = pr.dd_solve(pr.rhs(), outer="gmres", restart=60, tol=1e-13, max_sweeps=200, inner="direct")
    ud = pr.direct_solve()
    assert _rel(u, ud) < 1e-9


@pytest.mark.parametrize("P", [2, 3])
def test_waveholtz_exact_fixed_point_on_curved_subdomains(P):
    m = sem.Mesh(0, 1, 0, 1, 4, 4, P, 2, 2)
    X, Y = fields.warp_nodes(*m.coords(), (0, 1, 0, 1), 0.08)
    c, f = _fields(X, Y)
    pr = geom.MappedProblem(m, X, Y, c, 5.0, f)
    Nt = pr.choose_nt() + 3
    rng = np.random.default_rng(P)
    us = rng.standard_normal((m.L, m.nly, m.nlx)) + 1j * rng.standard_normal((m.L, m.nly, m.nlx))
    b = np.stack([(pr.sub_matrix(l) @ us[l].ravel()).reshape(us[l].shape) for l in range(m.L)])
    u1, _ = pr.waveholtz(b, Nt, 1, u0=us)
    assert _rel(u1, us) < 1e-10


def test_element_bound_dominates_the_subdomain_operator():
    m = sem.Mesh(0, 1, 0, 1, 4, 4, 3, 2, 2)
    X, Y = fields.warp_nodes(*m.coords(), (0, 1, 0, 1), 0.08)
    Jw, G11w, G12w, G22w, _, _ = geom.metric(X, Y, m.P, m.D, m.w, m.nx, m.ny)
    mu = geom.element_eig_bound(m.P, m.D, Jw, G11w, G12w, G22w)
    A = geom.stiffness_matrix(m.P, m.D, G11w, G12w, G22w).toarray()
    W = geom.scatter_add(Jw, m.P, m.nx, m.ny, X.shape).ravel()
    lam = np.max(np.linalg.eigvalsh(A / np.sqrt(np.outer(W, W))))
    assert lam <= mu * (1 + 1e-12) and mu < 2.5 * lam
