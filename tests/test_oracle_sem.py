"""Pins of the oracle's spectral-element pieces against closed forms and
exact quadrature identities (Sec. 4: GLL nodal basis, lumped M and H,
stiffness A_ij = (grad phi_j, grad phi_i))."""

import math

import numpy as np
import pytest

from oracle import sem
from oracle.dd import Problem


CLOSED_FORM_GLL = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    5: (
        [-1.0, -math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), -math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21),
         math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21), math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21), 1.0],
        [1 / 15, (14 - math.sqrt(7)) / 30, (14 + math.sqrt(7)) / 30, (14 + math.sqrt(7)) / 30,
         (14 - math.sqrt(7)) / 30, 1 / 15],
    ),
}


@pytest.mark.parametrize("P", sorted(CLOSED_FORM_GLL))
def test_gll_closed_forms(P):
    x, w = sem.gll(P)
    xe, we = CLOSED_FORM_GLL[P]
    np.testing.assert_allclose(x, xe, atol=1e-15)
    np.testing.assert_allclose(w, we, rtol=1e-14)


@pytest.mark.parametrize("P", range(1, 9))
def test_gll_exactness_degree(P):
    x, w = sem.gll(P)
    for k in range(0, 2 * P):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x**k) - exact) < 1e-13
    # degree 2P is not integrated exactly by GLL (guards against a Gauss rule)
    assert abs(np.sum(w * x ** (2 * P)) - 2.0 / (2 * P + 1)) > 1e-6


@pytest.mark.parametrize("P", range(1, 9))
def test_diff_matrix_exact_on_polynomials(P):
    x, _ = sem.gll(P)
    D = sem.diff_matrix(x)
    for k in range(0, P + 1):
        d = D @ x**k
        exact = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(d, exact, atol=1e-11 * max(1, k))


def _mesh(P, nx=3, ny=2, box=(-0.5, 1.5, 0.25, 1.0)):
    return sem.Mesh(box[0], box[1], box[2], box[3], nx, ny, P, 1, 1)


def _poly_integral_2d(cx, cy, box):
    """Integral over box of sum_k cx[k] x^i y^j given as dict {(i,j): coef}."""
    x0, x1, y0, y1 = box
    tot = 0.0
    for (i, j), c in cx.items():
        tot += c * (x1 ** (i + 1) - x0 ** (i + 1)) / (i + 1) * (y1 ** (j + 1) - y0 ** (j + 1)) / (j + 1)
    return tot


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
def test_stiffness_kernel_and_symmetry(P):
    m = _mesh(P)
    rng = np.random.default_rng(P)
    one = np.ones((m.NY, m.NX))
    A1 = sem.stiffness_apply(one, P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    assert np.max(np.abs(A1)) < 1e-11
    u = rng.standard_normal((m.NY, m.NX))
    v = rng.standard_normal((m.NY, m.NX))
    Au = sem.stiffness_apply(u, P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    Av = sem.stiffness_apply(v, P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    assert abs(np.sum(v * Au) - np.sum(u * Av)) < 1e-10 * np.sum(np.abs(u * Au))
    assert np.sum(u * Au) > 0
    # matrix-free and assembled forms agree
    A = sem.stiffness_matrix(P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    np.testing.assert_allclose((A @ u.ravel()).reshape(u.shape), Au, atol=1e-11 * np.max(np.abs(Au)))


@pytest.mark.parametrize("P", [2, 3, 4])
def test_stiffness_bilinear_form_exact(P):
    """v^T A u = integral grad u . grad v for u = x^2 y, v = x y^2 (exact for
    P >= 2: the integrand has degree 3 <= 2P-1 per variable).  A non-square
    box with hx != hy catches a swapped metric or transposed operand."""
    box = (-0.5, 1.5, 0.25, 1.0)
    m = _mesh(P, 3, 2, box)
    X, Y = m.coords()
    u = X**2 * Y
    v = X * Y**2
    Au = sem.stiffness_apply(u, P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    got = np.sum(v * Au)
    # grad u . grad v = (2xy)(y^2) + (x^2)(2xy) = 2 x y^3 + 2 x^3 y
    exact = _poly_integral_2d({(1, 3): 2.0, (3, 1): 2.0}, None, box)
    assert abs(got - exact) < 1e-12 * abs(exact)
    # u = x^2 + y: |grad u|^2 = 4x^2 + 1
    u2 = X**2 + Y
    Au2 = sem.stiffness_apply(u2, P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
    exact2 = _poly_integral_2d({(2, 0): 4.0, (0, 0): 1.0}, None, box)
    assert abs(np.sum(u2 * Au2) - exact2) < 1e-12 * exact2


@pytest.mark.parametrize("P", [2, 3, 4])
def test_lumped_mass_and_boundary(P):
    box = (-0.5, 1.5, 0.25, 1.0)
    m = sem.Mesh(*box, 3, 2, P, 1, 1)
    X, Y = m.coords()
    c = 0.5 + 0.0 * X
    pr = Problem(m, c, 3.0, 0.0 * X)
    area = (box[1] - box[0]) * (box[3] - box[2])
    perim = 2 * (box[1] - box[0]) + 2 * (box[3] - box[2])
    assert abs(pr.Mdiag.sum() - area / 0.25) < 1e-12 * area / 0.25
    assert abs(pr.Hdiag.sum() - perim / 0.5) < 1e-12 * perim / 0.5
    u = X + Y  # u^2 has degree 2 <= 2P-1
    exact = _poly_integral_2d({(2, 0): 1.0, (1, 1): 2.0, (0, 2): 1.0}, None, box) / 0.25
    assert abs(np.sum(pr.Mdiag * u * u) - exact) < 1e-12 * exact
    # boundary integral of x^2 / c along the perimeter
    x0, x1, y0, y1 = box
    bx = (x1**3 - x0**3) / 3
    edge = 2 * bx + (y1 - y0) * (x0**2 + x1**2)
    assert abs(np.sum(pr.Hdiag * X * X) - edge / 0.5) < 1e-12 * edge / 0.5


def test_real_block_form_matches_complex_system():
    """eq. (matrix-system): the real 2x2 block system is the complex system."""
    m = sem.Mesh(0, 1, 0, 1, 3, 3, 2, 1, 1)
    X, Y = m.coords()
    rng = np.random.default_rng(0)
    c = 1.0 + 0.3 * np.sin(3 * X) * np.cos(2 * Y)
    f = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
    pr = Problem(m, c, 7.0, f)
    K = pr.matrix().toarray()
    w = pr.omega
    A = (K + 1j * w * np.diag(pr.Hdiag.ravel()) + w * w * np.diag(pr.Mdiag.ravel())).real
    M = np.diag(pr.Mdiag.ravel())
    H = np.diag(pr.Hdiag.ravel())
    blk = np.block([[A - w * w * M, w * H], [w * H, w * w * M - A]])
    assert np.allclose(blk, blk.T)
    b = pr.rhs().ravel()
    sol = np.linalg.solve(blk, np.concatenate([b.real, -b.imag]))
    u = np.linalg.solve(K, b)
    n = u.size
    np.testing.assert_allclose(sol[:n] + 1j * sol[n:], u, rtol=1e-10, atol=1e-12 * np.abs(u).max())
