"""Plain restarted GMRES for the oracle (test infrastructure only).

Sec. 3 of the paper notes that the fixed-point iteration on the transmission
data can be accelerated by a Krylov method.  GMRES(m) from x0 = 0 is defined
by its minimal-residual property: after k steps of a cycle, x = x_start + V_k y
with y minimising || r_start - A V_k y ||_2 over the Krylov space.  This file
builds the Arnoldi basis with modified Gram-Schmidt and takes y from a
least-squares solve of the small Hessenberg system (numpy.linalg.lstsq), with
no Givens shortcut, so the iterate is the textbook definition.

Restart policy (matched by the CUDA-path driver): each cycle after the first
recomputes r = b - A x with one extra matvec; the first cycle uses r = b.
Pinned in tests/test_oracle_krylov.py against dense solves and the
minimal-residual property on random complex systems.

Flexible GMRES (``fgmres``) is the same minimal-residual definition with a
preconditioner applied to each basis vector, z_j = M_j(v_j), where M_j may
change from step to step (Sec. 7 of the paper uses the DD cycle, run in lower
precision and stopped at a tolerance, as the preconditioner of the FP64
problem: such an M_j is not one fixed linear map).  After k steps of a cycle
x = x_start + Z_k y, y minimising || r_start - A Z_k y ||_2; the Arnoldi
relation A Z_k = V_{k+1} H_k gives that as the small least-squares problem
|| beta e1 - H_k y ||.  With M_j = I it is GMRES; with one fixed linear M it is
GMRES on A M followed by x = M y (right preconditioning).  Both special cases,
the least-squares definition over the preconditioner's own outputs, the
one-step solve with the exact inverse and the restarts are pinned in
tests/test_oracle_krylov.py.
"""

from __future__ import annotations

import numpy as np


def gmres(matvec, b, restart=50, tol=0.0, maxit=100, x0=None):
    """Solve A x = b.  Returns (x, hist, n_matvec) with hist[k] the relative
    residual ||b - A x_k|| / ||b|| (least-squares value) after iteration k+1."""
    b = np.asarray(b, dtype=complex)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex)
    hist = []
    nmv = 0
    if bnorm == 0.0:
        return np.zeros_like(b), hist, nmv
    it = 0
    first = x0 is None
    while it < maxit:
        if first:
            r = b.copy()
            first = False
        else:
            r = b - matvec(x)
            nmv += 1
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        m = min(restart, maxit - it)
        V = np.zeros((m + 1, b.size), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        V[0] = r / beta
        y = np.zeros(0, dtype=complex)
        k = 0
        done = False
        for j in range(m):
            w = matvec(V[j])
            nmv += 1
            it += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=complex)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y)
            hist.append(res / bnorm)
            k = j + 1
            if res <= tol * bnorm or H[j + 1, j] == 0.0:
                done = True
                break
            V[j + 1] = w / H[j + 1, j]
        x = x + V[:k].T @ y
        if done:
            break
    return x, hist, nmv


def fgmres(matvec, precond, b, restart=30, tol=0.0, maxit=100, x0=None, cycle_tol=0.5):
    """Solve A x = b by flexible GMRES(restart) with right preconditioners
    z_j = precond(v_j).  Every cycle starts from the true residual r = b - A x
    (r = b when x0 is None, without a matvec), and ends after `restart` steps,
    at a lucky breakdown, or once the least-squares residual of the cycle is
    at most cycle_tol * tol * ||b|| (the margin leaves room for the difference
    between that estimate and the true residual the next cycle recomputes).
    Stops when the true relative residual is <= tol or after maxit
    preconditioner applications.  Returns (x, info): info["hist"] the true
    relative residual at the start of every cycle and at the end,
    info["est"] the least-squares estimate after every step,
    info["precond"] the number of preconditioner applications."""
    b = np.asarray(b, dtype=complex)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=complex)
    hist, est = [], []
    napp = 0
    if bnorm == 0.0:
        return np.zeros_like(b), {"hist": [0.0], "est": est, "precond": 0}
    first = x0 is None
    while True:
        r = b.copy() if first else b - matvec(x)
        first = False
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm or napp >= maxit:
            break
        m = min(restart, maxit - napp)
        V = np.zeros((m + 1, b.size), dtype=complex)
        Z = np.zeros((m, b.size), dtype=complex)
        H = np.zeros((m + 1, m), dtype=complex)
        V[0] = r / beta
        y = np.zeros(0, dtype=complex)
        k = 0
        for j in range(m):
            Z[j] = precond(V[j])
            napp += 1
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=complex)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[: j + 2, : j + 1] @ y)
            est.append(res / bnorm)
            k = j + 1
            if res <= cycle_tol * tol * bnorm or H[j + 1, j] == 0.0:
                break
            V[j + 1] = w / H[j + 1, j]
        x = x + Z[:k].T @ y
    return x, {"hist": hist, "est": est, "precond": napp}
