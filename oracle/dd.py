"""Domain decomposition + WaveHoltz oracle (test infrastructure only).

Follows the paper step by step, in FP64, vectorised over subdomains (the DDM
cycle of Algorithm 1 runs on every subdomain independently, Sec. 6):

* Global problem (Sec. 2, eq. (Helmholtz); Sec. 4, eq. (discrete-helmholtz)):
  (A - i w H - w^2 M) u = b with A_ij = (grad phi_j, grad phi_i),
  M = (c^-2 phi_j, phi_i), H = <c^-1 phi_j, phi_i> on the outer boundary,
  b = (f, phi) + <g, phi>, all by lumped GLL quadrature.
* Subdomain problem (Sec. 3): same operator on the subdomain's own elements;
  H over all four subdomain edges (outer boundary and interfaces, the
  zeroth-order transmission condition B = d_n - i k); interface data enters
  the right-hand side as <lambda, phi>.
* WaveHoltz (Sec. 5, eq. (WaveHoltz) and the modified leapfrog) on each
  subdomain, Algorithm 1's loop order.
* Transmission update (eq. (lambda-iteration), Algorithm 1 last step):
  lambda_{r,l} <- -lambda_{l,r} - 2 i k u_l on Gamma_{l,r}.
* Optional generalised transmission condition (the improved transmission
  conditions the paper names as future work, Sec. 8): B = d_n + k (eta - i zeta)
  on interfaces; eta = 0, zeta = 1 is the paper's condition.  In the subdomain
  operator the interface edges then carry zeta times the impedance damping
  and a boundary mass w eta <c^-1 phi_j, phi_i> (time domain:
  d_n u + (zeta/c) u_t + (w eta / c) u), and the update reads
  lambda_{r,l} <- -lambda_{l,r} + 2 k (eta - i zeta) u_l.

Readings of the paper taken here (each pinned by a test):
  1. lambda update sign -2ik (the paper prints +2ik; with outward normals and
     B = d_n - ik the derivation gives -2ik; pinned by DD == global solve).
  2. filter sign of the p-dot term from eq. (WaveHoltz): -1/(i w) = +i/w
     (Algorithm 1 prints +1/(i w); pinned by Pi(u*) = u*).
  3. the 2/N_t normalisation of eq. (WaveHoltz) is applied (Algorithm 1
     omits it; pinned by Pi(u*) = u*).
  4. t_nu = nu * dt, dt = (2 pi / w) / N_t.
  5. per-edge lambda including edge end points; corner nodes receive one
     contribution per edge (pinned by DD == global solve on cross points).
  6. N_t from the stable step of the subdomain operator:
     dt_max = cfl * 2 / (c_max sqrt(lx + ly)) with lx, ly the largest
     generalised eigenvalues of the 1D subdomain stiffness/lumped mass.
  7. outer iteration: GMRES(m) on (I - S) lambda = g (Krylov acceleration),
     plain fixed point as an option; global RHS split by lumped-mass share.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import krylov
from .sem import Mesh, nested_dissection_order, stiffness_apply, stiffness_matrix

EDGE_W, EDGE_E, EDGE_S, EDGE_N = 0, 1, 2, 3
OPPOSITE = {EDGE_W: EDGE_E, EDGE_E: EDGE_W, EDGE_S: EDGE_N, EDGE_N: EDGE_S}


class Problem:
    """One Helmholtz problem on a Mesh: nodal wave speed c (NY,NX), omega,
    nodal source f (NY,NX) complex, outer boundary data g (dict S,E,N,W)."""

    def __init__(self, mesh: Mesh, c, omega, f, g=None, robin=(0.0, 1.0)):
        self.mesh = mesh
        self.eta, self.zeta = float(robin[0]), float(robin[1])
        self.c = np.asarray(c, dtype=float).reshape(mesh.NY, mesh.NX)
        self.omega = float(omega)
        self.f = np.asarray(f, dtype=complex).reshape(mesh.NY, mesh.NX)
        if g is None:
            g = {"S": np.zeros(mesh.NX), "N": np.zeros(mesh.NX), "W": np.zeros(mesh.NY), "E": np.zeros(mesh.NY)}
        self.g = {k: np.asarray(v, dtype=complex) for k, v in g.items()}
        if np.any(~np.isfinite(self.c)) or np.any(self.c <= 0):
            raise ValueError("wave speed must be finite and positive")
        self.W2, Hw = self._global_weights()
        self.Mdiag = self.W2 / self.c**2
        self.Hdiag = Hw / self.c
        self._sub_setup()

    def _global_weights(self):
        """Lumped node weights W (the GLL rule's sum of w_a w_b |J| over the
        elements at a node) and outer-boundary edge weights, (NY, NX) each."""
        m = self.mesh
        self.Wx = m.lumped_1d(m.nx, m.hx)
        self.Wy = m.lumped_1d(m.ny, m.hy)
        Hw = np.zeros((m.NY, m.NX))
        Hw[0, :] += self.Wx
        Hw[-1, :] += self.Wx
        Hw[:, 0] += self.Wy
        Hw[:, -1] += self.Wy
        return np.outer(self.Wy, self.Wx), Hw

    # ------------------------------------------------------------ global --
    def rhs(self):
        """b_j = (f, phi_j) + <g, phi_j> (Sec. 4), lumped GLL quadrature."""
        return self.W2 * self.f + self.mesh.boundary_rhs(self.g)

    def apply_K(self, u):
        """(A - i w H - w^2 M) u on the whole mesh, matrix-free (Sec. 4)."""
        m = self.mesh
        Au = stiffness_apply(u, m.P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
        w = self.omega
        return Au - 1j * w * self.Hdiag * u - w * w * self.Mdiag * u

    def residual(self, u, b=None):
        b = self.rhs() if b is None else b
        return b - self.apply_K(u)

    def matrix(self):
        """Assembled sparse global matrix (the plain definition of the result)."""
        m = self.mesh
        A = stiffness_matrix(m.P, m.D, m.w, m.hx, m.hy, m.nx, m.ny)
        w = self.omega
        return (A - 1j * w * sp.diags(self.Hdiag.ravel()) - w * w * sp.diags(self.Mdiag.ravel())).tocsc()

    def direct_solve(self, b=None, ordering="default"):
        """K^{-1} b by a sparse LU.  ordering="nd": the matrix is permuted by
        nested dissection of the node grid first (sem.nested_dissection_order)
        and factorised in that order with diagonal pivots (far less fill on
        meshes of 10^5 nodes); without pivoting the factors are less accurate
        (residual 4e-10 on the 148k-node channel mesh), so two steps of FP64
        iterative refinement with the same factors follow (x += LU^{-1}(b - K x):
        residual 9e-15 there)."""
        b = self.rhs() if b is None else b
        if ordering != "nd":
            return spla.spsolve(self.matrix(), b.ravel()).reshape(b.shape)
        m = self.mesh
        perm = nested_dissection_order(m.NX, m.NY, m.P)
        Kp = self.matrix()[perm][:, perm].tocsc()
        lu = spla.splu(Kp, permc_spec="NATURAL", diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
        bp = b.ravel()[perm]
        up = lu.solve(bp)
        for _ in range(2):
            up = up + lu.solve(bp - Kp @ up)
        u = np.empty_like(up)
        u[perm] = up
        return u.reshape(b.shape)

    # -------------------------------------------------------- subdomains --
    def _sub_setup(self):
        m = self.mesh
        P = m.P
        L = m.L
        self.ox = np.array([(l % m.Sx) * m.sub_nx * P for l in range(L)])
        self.oy = np.array([(l // m.Sx) * m.sub_ny * P for l in range(L)])
        jj, ii = np.meshgrid(np.arange(m.nly), np.arange(m.nlx), indexing="ij")
        self.gJ = self.oy[:, None, None] + jj[None]  # (L, nly, nlx) global row
        self.gI = self.ox[:, None, None] + ii[None]  # global column
        Ws = self._sub_weights()  # (1 or L, nly, nlx)
        # neighbours and interface flags per edge
        self.nbr = -np.ones((L, 4), dtype=int)
        for l in range(L):
            sx, sy = l % m.Sx, l // m.Sx
            if sx > 0:
                self.nbr[l, EDGE_W] = l - 1
            if sx < m.Sx - 1:
                self.nbr[l, EDGE_E] = l + 1
            if sy > 0:
                self.nbr[l, EDGE_S] = l - m.Sx
            if sy < m.Sy - 1:
                self.nbr[l, EDGE_N] = l + m.Sx
        # edge quadrature weights, split into outer-boundary and interface edges
        Hout = np.zeros((L, m.nly, m.nlx))
        Hif = np.zeros((L, m.nly, m.nlx))
        for e in range(4):
            rows, cols, wts = self.edge_nodes(e)
            for l in range(L):
                (Hif if self.nbr[l, e] >= 0 else Hout)[l, rows, cols] += wts[l] if np.ndim(wts) == 2 else wts
        self.c_sub = self.c[self.gJ, self.gI]
        self.M_sub = Ws / self.c_sub**2
        self.H_sub = (Hout + self.zeta * Hif) / self.c_sub          # damping: outer impedance, zeta on interfaces
        self.Hm_sub = self.omega * self.eta * Hif / self.c_sub      # interface boundary mass (eta)
        self.share = Ws / self.W2[self.gJ, self.gI]  # lumped-mass share of each copy

    def _sub_weights(self):
        """Lumped node weights of a subdomain's own elements, (1, nly, nlx)
        (the same for every subdomain of a uniform mesh)."""
        m = self.mesh
        self.Wxs = m.lumped_1d(m.sub_nx, m.hx)
        self.Wys = m.lumped_1d(m.sub_ny, m.hy)
        return np.outer(self.Wys, self.Wxs)[None]

    def edge_nodes(self, e):
        """(rows, cols, weights) of subdomain edge e in local node indices
        (weights (n,) shared by all subdomains, or (L, n) per subdomain)."""
        m = self.mesh
        if e == EDGE_W:
            return np.arange(m.nly), np.zeros(m.nly, int), self.Wys
        if e == EDGE_E:
            return np.arange(m.nly), np.full(m.nly, m.nlx - 1), self.Wys
        if e == EDGE_S:
            return np.zeros(m.nlx, int), np.arange(m.nlx), self.Wxs
        return np.full(m.nlx, m.nly - 1), np.arange(m.nlx), self.Wxs

    def lam_size(self):
        return self.mesh.L * 4 * self.mesh.NE

    def split_rhs(self, rhs_glob):
        """Subdomain right-hand sides from a global weak-form vector, by the
        lumped-mass share of each copy (equal to assembling f and g on the
        subdomain's own elements and edges)."""
        return self.share * rhs_glob[self.gJ, self.gI]

    def assemble_u(self, u_sub):
        """Global field from subdomain copies, mass-weighted average."""
        m = self.mesh
        out = np.zeros((m.NY, m.NX), complex)
        np.add.at(out, (self.gJ, self.gI), self.share * u_sub)
        return out

    # ------------------------------------------------------------ timing --
    def choose_nt(self, cfl=0.9):
        """Reading 6: N_t = max(3, ceil(T / dt_max)), T = 2 pi / w."""
        m = self.mesh
        lx = _max_gen_eig_1d(m, m.sub_nx, m.hx)
        ly = _max_gen_eig_1d(m, m.sub_ny, m.hy)
        lam = float(np.max(self.c)) ** 2 * (lx + ly)
        dt_max = cfl * 2.0 / math.sqrt(lam)
        return max(3, int(math.ceil((2.0 * math.pi / self.omega) / dt_max)))

    # ------------------------------------------------------------- sweep --
    def sweep(self, lam_in, rhs_glob=None, Nt=None, m_wh=5, wh_tol=0.0, want_u=False, inner="waveholtz", subset=None,
              u0=None):
        """One DDM cycle (Algorithm 1) on every subdomain.

        lam_in: (L, 4, NE) complex, incoming data per subdomain edge (W,E,S,N),
        nodes along increasing x or y; slots of outer-boundary edges unused.
        rhs_glob: global weak-form source (None = homogeneous sweep).
        Returns lam_out (same layout) and, if want_u, the subdomain solutions
        (L, nly, nlx) and the number of WaveHoltz iterations taken.
        inner="direct" replaces WaveHoltz by an exact sparse solve of each
        subdomain system (isolates the DD fixed point in tests).
        subset: optional list of subdomains to solve (others get u = 0 and
        send nothing); used for sampled checks of large problems.
        u0: optional (L, nly, nlx) start of the WaveHoltz iteration instead of
        zero (warm start from a previous sweep's subdomain solutions).
        """
        m = self.mesh
        Nt = self.choose_nt() if Nt is None else Nt
        b = np.zeros((m.L, m.nly, m.nlx), complex)
        if rhs_glob is not None:
            b += self.split_rhs(rhs_glob)
        for e in range(4):
            rows, cols, wts = self.edge_nodes(e)
            n = len(rows)
            for l in np.where(self.nbr[:, e] >= 0)[0]:
                wl = wts[l] if np.ndim(wts) == 2 else wts
                b[l, rows, cols] += wl * lam_in[l, e, :n]  # <lambda, phi> on the interface
        sel = np.arange(m.L) if subset is None else np.asarray(subset, dtype=int)
        u = np.zeros_like(b)
        if inner == "direct":
            u[sel] = self.direct_sub(b[sel], sel)
            iters = np.zeros(m.L, int)
        else:
            u_sel, it_sel = self.waveholtz(b[sel], Nt, m_wh, wh_tol, subs=sel, u0=None if u0 is None else u0[sel])
            u[sel] = u_sel
            iters = np.zeros(m.L, int)
            iters[sel] = it_sel
        lam_out = np.zeros_like(lam_in)
        w = self.omega
        for e in range(4):
            rows, cols, _ = self.edge_nodes(e)
            n = len(rows)
            for l in sel[self.nbr[sel, e] >= 0]:
                r = self.nbr[l, e]
                k = w / self.c_sub[l, rows, cols]
                lam_out[r, OPPOSITE[e], :n] = -lam_in[l, e, :n] + 2 * k * (self.eta - 1j * self.zeta) * u[l, rows, cols]
        if want_u:
            return lam_out, u, iters
        return lam_out

    def leapfrog_coeffs(self, Nt, subs=None):
        """alpha, beta, sigma of the modified leapfrog (Sec. 5):
        theta = tan(w dt/2)/w, sigma = sin(w dt/2)/(w/2),
        alpha = (M - theta H)/(M + theta H), beta = sigma/(M + theta H)."""
        w = self.omega
        dt = (2.0 * math.pi / w) / Nt
        theta = math.tan(w * dt / 2.0) / w
        sigma = math.sin(w * dt / 2.0) / (w / 2.0)
        M = self.M_sub if subs is None else self.M_sub[subs]
        H = self.H_sub if subs is None else self.H_sub[subs]
        alpha = (M - theta * H) / (M + theta * H)
        beta = sigma / (M + theta * H)
        return alpha, beta, sigma

    def sub_matrix(self, l):
        """Sparse subdomain matrix A_l - i w H_l - w^2 M_l (all four edges in H)."""
        m = self.mesh
        if not hasattr(self, "_A_sub"):
            self._A_sub = stiffness_matrix(m.P, m.D, m.w, m.hx, m.hy, m.sub_nx, m.sub_ny)
        w = self.omega
        d = self.Hm_sub[l].ravel() - 1j * w * self.H_sub[l].ravel() - w * w * self.M_sub[l].ravel()
        return (self._A_sub + sp.diags(d)).tocsc()

    def direct_sub(self, b, sel):
        out = np.empty_like(b)
        for k, l in enumerate(sel):
            out[k] = spla.spsolve(self.sub_matrix(l), b[k].ravel()).reshape(b[k].shape)
        return out

    def apply_A_sub(self, p, subs=None):
        """A p on subdomain arrays p (len(subs) or L, nly, nlx); a uniform
        mesh has one subdomain operator, so subs is not needed here."""
        m = self.mesh
        return stiffness_apply(p, m.P, m.D, m.w, m.hx, m.hy, m.sub_nx, m.sub_ny)

    def waveholtz(self, b, Nt, m_wh, wh_tol=0.0, u0=None, time_steps=None, subs=None):
        """WaveHoltz fixed-point iteration u <- Pi u (eq. (WaveHoltz)) on every
        subdomain, Algorithm 1's loop.  With wh_tol > 0 a subdomain stops once
        ||u^{m+1} - u^m|| <= wh_tol ||u^{m+1}|| (at most m_wh iterations).
        time_steps limits the inner loop to nu = 1..time_steps (tests only).
        subs: the subdomains b belongs to (default: all, in order).
        Returns (u, iterations per subdomain)."""
        w = self.omega
        alpha, beta, sigma = self.leapfrog_coeffs(Nt, subs)
        Hm = self.Hm_sub if subs is None else self.Hm_sub[subs]
        c0 = -0.25 + 0.25 * math.tan(math.pi / Nt) ** 2

        def kappa(nu):
            return math.cos(2.0 * math.pi * nu / Nt) + c0

        u = np.zeros_like(b) if u0 is None else np.array(u0, dtype=complex)
        L = b.shape[0]
        active = np.ones(L, bool)
        iters = np.zeros(L, int)
        last = Nt - 1 if time_steps is None else time_steps
        for _ in range(m_wh):
            if not active.any():
                break
            p = u.real.copy()
            pd = (-1j * w * u * np.exp(-1j * math.pi / Nt)).real
            v = kappa(0) * p + (1j / w) * kappa(0.5) * pd
            for nu in range(1, last + 1):
                p = p + sigma * pd
                Ap = self.apply_A_sub(p, subs) + Hm * p  # interface boundary mass (zero unless eta != 0)
                force = (b * np.exp(-2j * math.pi * nu / Nt)).real
                pd = alpha * pd + beta * (-Ap + force)
                v = v + kappa(nu) * p + (1j / w) * kappa(nu + 0.5) * pd
            unew = (2.0 / Nt) * v
            iters[active] += 1
            if wh_tol > 0.0:
                dn = np.sqrt(np.sum(np.abs(unew - u) ** 2, axis=(1, 2)))
                un = np.sqrt(np.sum(np.abs(unew) ** 2, axis=(1, 2)))
                conv = dn <= wh_tol * un
                u[active] = unew[active]
                active &= ~conv
            else:
                u = unew
        return u, iters

    # ------------------------------------------------------ outer solves --
    def dd_solve(self, rhs_glob, Nt=None, m_wh=5, wh_tol=0.0, outer="gmres", restart=50, tol=1e-10, max_sweeps=500,
                 inner="waveholtz", warm=False):
        """Approximate K^{-1} rhs_glob by the DD method (one refinement step).

        gmres / rgmres: solve (I - S) lam = g with g = sweep(0, rhs), S the
        homogeneous sweep, by complex GMRES / real GMRES on the interleaved
        (re, im) vector; plain: lam <- sweep(lam, rhs), with warm=True each
        sweep's WaveHoltz starting from the previous sweep's subdomain
        solutions.  A final sweep at lam returns the subdomain solutions,
        assembled by mass-weighted averaging; info["wh_iters"] sums the
        WaveHoltz iterations of the plain iteration's sweeps and the final one.
        Returns (u_global, info dict with sweeps and residual history)."""
        Nt = self.choose_nt() if Nt is None else Nt
        shape = (self.mesh.L, 4, self.mesh.NE)
        sweeps = 0
        g, u_first, it = self.sweep(np.zeros(shape, complex), rhs_glob, Nt, m_wh, wh_tol, inner=inner, want_u=True)
        wh_total = int(np.sum(it))  # WaveHoltz iterations summed over subdomains and sweeps
        sweeps += 1
        hist = []
        if outer == "gmres":
            # complex GMRES: exact when the subdomain solve is complex-linear
            # (converged WaveHoltz or direct inner solve)
            def mv(x):
                return x - self.sweep(x.reshape(shape), None, Nt, m_wh, wh_tol, inner=inner).ravel()

            lam, hist, nmv = krylov.gmres(mv, g.ravel(), restart=restart, tol=tol, maxit=max(0, max_sweeps - 2))
            sweeps += nmv
            lam = lam.reshape(shape)
        elif outer == "rgmres":
            # real GMRES on the (re, im)-interleaved lambda vector: exact for
            # any fixed WaveHoltz count, where the sweep is only real-linear
            def to_c(xr):
                return np.ascontiguousarray(xr.real).view(complex).reshape(shape)

            def mvr(xr):
                x = to_c(xr)
                y = x - self.sweep(x, None, Nt, m_wh, wh_tol, inner=inner)
                return y.reshape(-1).view(float).astype(complex)

            lam_r, hist, nmv = krylov.gmres(mvr, g.reshape(-1).view(float).astype(complex), restart=restart,
                                           tol=tol, maxit=max(0, max_sweeps - 2))
            sweeps += nmv
            lam = to_c(lam_r)
        elif outer == "plain":
            # warm: every sweep starts WaveHoltz from the previous sweep's
            # subdomain solutions (Sec. 8's loose-then-tight inner solves; the
            # sweep then depends on the previous iterate, so only the plain
            # fixed-point iteration can use it)
            lam = g
            gn = np.linalg.norm(g)
            u_prev = u_first if warm else None
            for _ in range(max(0, max_sweeps - 2)):
                if warm:
                    new, u_prev, it = self.sweep(lam, rhs_glob, Nt, m_wh, wh_tol, want_u=True, inner=inner, u0=u_prev)
                    wh_total += int(np.sum(it))
                else:
                    new, _, it = self.sweep(lam, rhs_glob, Nt, m_wh, wh_tol, want_u=True, inner=inner)
                    wh_total += int(np.sum(it))
                sweeps += 1
                d = np.linalg.norm(new - lam)
                lam = new
                hist.append(d / gn if gn > 0 else 0.0)
                if gn == 0 or d <= tol * gn:
                    break
        else:
            raise ValueError(outer)
        _, u_sub, it = self.sweep(lam, rhs_glob, Nt, m_wh, wh_tol, want_u=True, inner=inner,
                                  u0=u_prev if (outer == "plain" and warm) else None)
        wh_total += int(np.sum(it))
        sweeps += 1
        return self.assemble_u(u_sub), {"sweeps": sweeps, "hist": hist, "lam": lam, "u_sub": u_sub,
                                        "wh_iters": wh_total}

    def solve(self, Nt=None, m_wh=5, wh_tol=0.0, tol=1e-8, outer="gmres", restart=50, inner_tol=1e-10,
              max_sweeps=500, max_refine=10, inner="waveholtz", refine="defect", refine_restart=30):
        """FP64 refinement around the DD solve (Sec. 7: the DDM acts as a
        preconditioner) until ||b - K u|| <= tol ||b||.

        refine="defect": u_{k+1} = u_k + DD(b - K u_k).
        refine="fgmres": flexible GMRES(refine_restart) on K u = b with the DD
        solve of each basis vector as the right preconditioner
        (krylov.fgmres; the DD solve stops at a tolerance and, with a fixed
        WaveHoltz count, is only real-linear, so it is a different map at
        every step).  max_refine bounds the DD solves in both.
        Returns (u, info)."""
        if refine == "fgmres":
            Nt = self.choose_nt() if Nt is None else Nt
            b = self.rhs()
            shape = b.shape
            sweeps = [0]

            def precond(v):
                e, info = self.dd_solve(v.reshape(shape), Nt, m_wh, wh_tol, outer, restart, inner_tol, max_sweeps,
                                        inner)
                sweeps[0] += info["sweeps"]
                return e.ravel()

            u, info = krylov.fgmres(lambda x: self.apply_K(x.reshape(shape)).ravel(), precond, b.ravel(),
                                    restart=refine_restart, tol=tol, maxit=max_refine)
            return u.reshape(shape), {"rel_residual": info["hist"][-1], "hist": info["hist"], "est": info["est"],
                       "sweeps": sweeps[0], "refinements": info["precond"]}
        if refine != "defect":
            raise ValueError(refine)
        b = self.rhs()
        bn = np.linalg.norm(b)
        u = np.zeros_like(b)
        r = b.copy()
        hist = []
        sweeps = 0
        refinements = 0
        while True:
            rel = np.linalg.norm(r) / bn if bn > 0 else 0.0
            hist.append(rel)
            if rel <= tol or refinements >= max_refine:
                break
            e, info = self.dd_solve(r, Nt, m_wh, wh_tol, outer, restart, inner_tol, max_sweeps, inner)
            sweeps += info["sweeps"]
            u = u + e
            r = b - self.apply_K(u)
            refinements += 1
        return u, {"rel_residual": hist[-1], "hist": hist, "sweeps": sweeps, "refinements": refinements}


def _max_gen_eig_1d(m: Mesh, n_el, h):
    """Largest eigenvalue of W^-1 K for the 1D subdomain stiffness K and
    lumped mass W over n_el elements (free ends)."""
    P = m.P
    K1 = m.D.T @ np.diag(m.w) @ m.D * (2.0 / h)
    n = n_el * P + 1
    K = np.zeros((n, n))
    for e in range(n_el):
        K[e * P : e * P + P + 1, e * P : e * P + P + 1] += K1
    W = m.lumped_1d(n_el, h)
    return float(sla.eigh(K, np.diag(W), eigvals_only=True)[-1])
