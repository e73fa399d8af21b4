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
