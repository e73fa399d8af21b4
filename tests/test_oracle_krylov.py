"""Pins of the oracle's GMRES against dense linear algebra (Sec. 3, Krylov
acceleration of the transmission-data iteration)."""

import numpy as np
import pytest

from oracle import krylov


def _system(n, seed, shift=3.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A / np.sqrt(n) + shift * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_gmres_full_space_solves_exactly():
    A, b = _system(30, 1)
    x, hist, nmv = krylov.gmres(lambda v: A @ v, b, restart=30, tol=0.0, maxit=30)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    assert nmv == 30


@pytest.mark.parametrize("k", [1, 3, 7])
def test_gmres_minimal_residual_property(k):
    """After k steps x_k minimises ||b - A x|| over span{b, Ab, ..., A^{k-1} b}
    (computed here from an explicit, orthonormalised Krylov matrix)."""
    A, b = _system(25, 2, shift=1.0)
    x, hist, _ = krylov.gmres(lambda v: A @ v, b, restart=50, tol=0.0, maxit=k)
    Kr = np.empty((b.size, k), complex)
    v = b.copy()
    for j in range(k):
        Kr[:, j] = v
        v = A @ v
    Q, _ = np.linalg.qr(Kr)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    xbest = Q @ y
    np.testing.assert_allclose(x, xbest, rtol=1e-9, atol=1e-12)
    assert abs(hist[-1] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-12


def test_gmres_restart_counts_matvecs_and_converges():
    A, b = _system(40, 3, shift=4.0)
    x, hist, nmv = krylov.gmres(lambda v: A @ v, b, restart=5, tol=1e-12, maxit=200)
    assert np.linalg.norm(b - A @ x) <= 1.01e-12 * np.linalg.norm(b)
    cycles = -(-len(hist) // 5)
    assert nmv == len(hist) + (cycles - 1)  # one residual matvec per restart


def test_gmres_zero_rhs():
    x, hist, nmv = krylov.gmres(lambda v: v, np.zeros(5, complex), restart=3, maxit=10)
    assert np.all(x == 0) and nmv == 0


# ---- flexible GMRES (the FP64 refinement around the DD solve, Sec. 7)


def test_fgmres_with_identity_preconditioner_is_gmres():
    """M_j = I: the same iterate and least-squares residuals as GMRES."""
    A, b = _system(30, 4, shift=1.5)
    xg, hg, _ = krylov.gmres(lambda v: A @ v, b, restart=12, tol=0.0, maxit=12)
    xf, info = krylov.fgmres(lambda v: A @ v, lambda v: v, b, restart=12, tol=0.0, maxit=12)
    np.testing.assert_allclose(xf, xg, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(info["est"], hg, rtol=1e-9, atol=1e-14)
    assert info["precond"] == 12


def test_fgmres_with_fixed_preconditioner_is_right_preconditioned_gmres():
    """One fixed linear M: x = M y with y the GMRES iterate for A M y = b."""
    A, b = _system(30, 5, shift=0.5)
    rng = np.random.default_rng(9)
    M = np.eye(30) + 0.3 * (rng.standard_normal((30, 30)) + 1j * rng.standard_normal((30, 30))) / np.sqrt(30)
    y, hg, _ = krylov.gmres(lambda v: A @ (M @ v), b, restart=9, tol=0.0, maxit=9)
    xf, info = krylov.fgmres(lambda v: A @ v, lambda v: M @ v, b, restart=9, tol=0.0, maxit=9)
    np.testing.assert_allclose(xf, M @ y, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(info["est"], hg, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("k", [2, 5, 8])
def test_fgmres_minimises_over_its_preconditioned_directions(k):
    """A preconditioner that changes every step (a random perturbation of the
    identity per call): after k steps of one cycle x minimises ||b - A x|| over
    span{z_1 .. z_k}, the vectors the preconditioner returned (least squares on
    the explicit A Z), and the estimate is that minimum."""
    A, b = _system(24, 6, shift=1.0)
    rng = np.random.default_rng(11)
    Z = []

    def precond(v):
        E = 0.5 * (rng.standard_normal((24, 24)) + 1j * rng.standard_normal((24, 24))) / np.sqrt(24)
        z = v + E @ v
        Z.append(z.copy())
        return z

    x, info = krylov.fgmres(lambda v: A @ v, precond, b, restart=50, tol=0.0, maxit=k)
    Zm = np.array(Z).T
    y, *_ = np.linalg.lstsq(A @ Zm, b, rcond=None)
    np.testing.assert_allclose(x, Zm @ y, rtol=1e-9, atol=1e-12)
    bn = np.linalg.norm(b)
    assert abs(info["est"][-1] - np.linalg.norm(b - A @ x) / bn) < 1e-12
    assert abs(info["hist"][-1] - np.linalg.norm(b - A @ x) / bn) < 1e-12


def test_fgmres_exact_preconditioner_solves_in_one_step():
    A, b = _system(20, 7)
    Ainv = np.linalg.inv(A)
    x, info = krylov.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, restart=5, tol=1e-12, maxit=5)
    assert info["precond"] == 1
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


def test_fgmres_restarts_from_the_true_residual_and_converges():
    """Cycles of 3 steps with an inexact preconditioner (a rough inverse):
    every cycle starts from b - A x, the recorded true residuals fall to the
    tolerance, and the preconditioner count is the budget actually used."""
    A, b = _system(40, 8, shift=4.0)
    rng = np.random.default_rng(12)
    Ainv = np.linalg.inv(A)

    def precond(v):
        E = 0.2 * (rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))) / np.sqrt(40)
        return (Ainv + E @ Ainv) @ v

    x, info = krylov.fgmres(lambda v: A @ v, precond, b, restart=3, tol=1e-12, maxit=60)
    rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert rel <= 1e-12 and abs(info["hist"][-1] - rel) < 1e-14
    assert all(h2 < h1 for h1, h2 in zip(info["hist"], info["hist"][1:]))
    assert info["precond"] == len(info["est"])


def test_fgmres_zero_rhs():
    x, info = krylov.fgmres(lambda v: v, lambda v: v, np.zeros(4, complex), restart=3, maxit=5)
    assert np.all(x == 0) and info["precond"] == 0
