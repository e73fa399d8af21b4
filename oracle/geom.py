"""Spectral elements on general convex quadrilaterals (test infrastructure only).

Sec. 4 of the paper allows convex quadrilateral elements; the tensor-product
basis is then composed with each element's map from the reference square.
Here the map is isoparametric: the element's (P+1)^2 GLL nodes carry their
physical coordinates (x, y), and x(xi, eta), y(xi, eta) are the degree-P
Lagrange interpolants of them (bilinear quads are the special case of nodes
placed by the bilinear map).  With the collocated GLL rule:

  J       = x_xi y_eta - x_eta y_xi                     (must be > 0)
  A_e     = sum over GLL points of w_a w_b (grad phi_i . grad phi_j) J, i.e.
            with u_xi = sum_c D[a,c] u(c,b), u_eta = sum_c D[b,c] u(a,c):
            F1 = w_a w_b (G11 u_xi + G12 u_eta),  F2 = w_a w_b (G12 u_xi + G22 u_eta)
            (A u)(a',b') = sum_a D[a,a'] F1(a,b') + sum_b D[b,b'] F2(a',b)
            G = J (dxi/dx)(dxi/dx)^T:  G11 = (x_eta^2 + y_eta^2)/J,
            G12 = -(x_xi x_eta + y_xi y_eta)/J,  G22 = (x_xi^2 + y_xi^2)/J
  M       = lumped: sum over elements of w_a w_b J / c^2 at each node
  edges   = GLL rule along the edge with the arc-length factor
            |(x_xi, y_xi)| (edges eta = const) or |(x_eta, y_eta)| (xi = const)

Arrays on node grids are [y, x] (x fastest) as in sem.py; element-local
arrays are [..., ey, ex, b, a] (b along eta, a along xi).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dd
from .sem import element_view, scatter_add


def metric(X, Y, P, D, w, nex, ney):
    """Per element node: (Jw, G11w, G12w, G22w, s_xi, s_eta) with Jw = w_a w_b J,
    Gkw = w_a w_b Gk, s_xi = |(x_xi, y_xi)|, s_eta = |(x_eta, y_eta)|.
    X, Y: (..., ney*P+1, nex*P+1) node coordinates."""
    Xe = element_view(np.asarray(X, float), P, nex, ney)
    Ye = element_view(np.asarray(Y, float), P, nex, ney)
    # d/dxi at (b, q): sum_a D[q,a] X[b,a];  d/deta at (r, a): sum_b D[r,b] X[b,a]
    x_xi = np.einsum("...ba,qa->...bq", Xe, D)
    y_xi = np.einsum("...ba,qa->...bq", Ye, D)
    x_eta = np.einsum("...ba,rb->...ra", Xe, D)
    y_eta = np.einsum("...ba,rb->...ra", Ye, D)
    J = x_xi * y_eta - x_eta * y_xi
    if np.any(~(J > 0)):
        raise ValueError("element map is not positively oriented (J <= 0 at a GLL node)")
    ww = np.outer(w, w)  # [b, a] = w_b w_a
    G11 = (x_eta**2 + y_eta**2) / J
    G12 = -(x_xi * x_eta + y_xi * y_eta) / J
    G22 = (x_xi**2 + y_xi**2) / J
    s_xi = np.sqrt(x_xi**2 + y_xi**2)
    s_eta = np.sqrt(x_eta**2 + y_eta**2)
    return ww * J, ww * G11, ww * G12, ww * G22, s_xi, s_eta


def stiffness_apply(u, P, D, G11w, G12w, G22w):
    """(A u) on a block of mapped elements, element form (see module doc).
    u: (..., ney*P+1, nex*P+1); G*: (..., ney, nex, P+1, P+1)."""
    ney, nex = G11w.shape[-4], G11w.shape[-3]
    ue = element_view(u, P, nex, ney)
    u_xi = np.einsum("...ra,qa->...rq", ue, D)
    u_eta = np.einsum("...bq,rb->...rq", ue, D)
    F1 = G11w * u_xi + G12w * u_eta
    F2 = G12w * u_xi + G22w * u_eta
    contrib = np.einsum("...bq,qa->...ba", F1, D) + np.einsum("...ra,rb->...ba", F2, D)
    return scatter_add(contrib, P, nex, ney, u.shape)


def element_matrices(P, D, G11w, G12w, G22w):
    """Dense element stiffness matrices (..., n, n), n = (P+1)^2, local index
    b*(P+1)+a, by applying the element form to each unit vector."""
    n = (P + 1) ** 2
    E = np.eye(n).reshape(n, P + 1, P + 1)  # [k, b, a]
    g11, g12, g22 = (g[..., None, :, :] for g in (G11w, G12w, G22w))
    u_xi = np.einsum("kra,qa->krq", E, D)
    u_eta = np.einsum("kbq,rb->krq", E, D)
    F1 = g11 * u_xi + g12 * u_eta
    F2 = g12 * u_xi + g22 * u_eta
    out = np.einsum("...kbq,qa->...kba", F1, D) + np.einsum("...kra,rb->...kba", F2, D)
    # column k of A_e is A_e e_k
    return np.swapaxes(out.reshape(out.shape[:-2] + (n,)), -1, -2)


def stiffness_matrix(P, D, G11w, G12w, G22w):
    """Assembled sparse A on one block of mapped elements (ney, nex, P+1, P+1)."""
    ney, nex = G11w.shape[0], G11w.shape[1]
    Ae = element_matrices(P, D, G11w, G12w, G22w)
    nX = nex * P + 1
    loc = np.array([[b * nX + a for a in range(P + 1)] for b in range(P + 1)]).ravel()
    rows, cols, vals = [], [], []
    for ey in range(ney):
        for ex in range(nex):
            g = loc + ey * P * nX + ex * P
            rows.append(np.repeat(g, len(g)))
            cols.append(np.tile(g, len(g)))
            vals.append(Ae[ey, ex].ravel())
    n = nX * (ney * P + 1)
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()


def block_edge_weights(P, w, s_xi, s_eta):
    """GLL arc-length weights along the four outer edges of a block of
    elements: dict W,E (length ney*P+1, along y) and S,N (nex*P+1, along x)."""
    ney, nex = s_xi.shape[-4], s_xi.shape[-3]
    lead = s_xi.shape[:-4]
    out = {"S": np.zeros(lead + (nex * P + 1,)), "N": np.zeros(lead + (nex * P + 1,)),
           "W": np.zeros(lead + (ney * P + 1,)), "E": np.zeros(lead + (ney * P + 1,))}
    for ex in range(nex):
        out["S"][..., ex * P: ex * P + P + 1] += w * s_xi[..., 0, ex, 0, :]
        out["N"][..., ex * P: ex * P + P + 1] += w * s_xi[..., ney - 1, ex, P, :]
    for ey in range(ney):
        out["W"][..., ey * P: ey * P + P + 1] += w * s_eta[..., ey, 0, :, 0]
        out["E"][..., ey * P: ey * P + P + 1] += w * s_eta[..., ey, nex - 1, :, P]
    return out


def element_eig_bound(P, D, Jw, G11w, G12w, G22w):
    """max over elements of the largest eigenvalue of W_e^-1 A_e (W_e = diag
    of w_a w_b J).  Since x^T A x = sum_e x_e^T A_e x_e and x^T W x >=
    sum_e x_e^T W_e x_e, it bounds lambda_max(W^-1 A) of any assembly."""
    Ae = element_matrices(P, D, G11w, G12w, G22w)
    s = 1.0 / np.sqrt(Jw.reshape(Jw.shape[:-2] + (-1,)))
    B = Ae * s[..., :, None] * s[..., None, :]
    return float(np.max(np.linalg.eigvalsh(B)[..., -1]))


class MappedProblem(dd.Problem):
    """dd.Problem on a mesh whose GLL nodes sit at given physical positions
    X, Y (NY, NX); the mesh's logical structure (elements, subdomains,
    lambda slots) is unchanged.  Outer boundary data g as in dd.Problem."""

    def __init__(self, mesh, X, Y, c, omega, f, g=None, robin=(0.0, 1.0)):
        m = mesh
        self.X = np.asarray(X, float).reshape(m.NY, m.NX)
        self.Y = np.asarray(Y, float).reshape(m.NY, m.NX)
        met = metric(self.X, self.Y, m.P, m.D, m.w, m.nx, m.ny)
        self.Jw, self.G11w, self.G12w, self.G22w, self.s_xi, self.s_eta = met
        self.bw = block_edge_weights(m.P, m.w, self.s_xi, self.s_eta)
        super().__init__(mesh, c, omega, f, g, robin)

    # global weights and operator ------------------------------------------
    def _global_weights(self):
        m = self.mesh
        W2 = scatter_add(self.Jw, m.P, m.nx, m.ny, (m.NY, m.NX))
        Hw = np.zeros((m.NY, m.NX))
        Hw[0, :] += self.bw["S"]
        Hw[-1, :] += self.bw["N"]
        Hw[:, 0] += self.bw["W"]
        Hw[:, -1] += self.bw["E"]
        return W2, Hw

    def rhs(self):
        b = self.W2 * self.f
        b[0, :] += self.bw["S"] * self.g["S"]
        b[-1, :] += self.bw["N"] * self.g["N"]
        b[:, 0] += self.bw["W"] * self.g["W"]
        b[:, -1] += self.bw["E"] * self.g["E"]
        return b

    def apply_K(self, u):
        m = self.mesh
        Au = stiffness_apply(u, m.P, m.D, self.G11w, self.G12w, self.G22w)
        w = self.omega
        return Au - 1j * w * self.Hdiag * u - w * w * self.Mdiag * u

    def matrix(self):
        m = self.mesh
        A = stiffness_matrix(m.P, m.D, self.G11w, self.G12w, self.G22w)
        w = self.omega
        return (A - 1j * w * sp.diags(self.Hdiag.ravel()) - w * w * sp.diags(self.Mdiag.ravel())).tocsc()

    # subdomains -------------------------------------------------------------
    def _sub_blocks(self, arr):
        """Element-local array (ny, nx, P+1, P+1) -> per subdomain (L, sny, snx, P+1, P+1)."""
        m = self.mesh
        out = np.empty((m.L, m.sub_ny, m.sub_nx) + arr.shape[2:], arr.dtype)
        for l in range(m.L):
            sx, sy = l % m.Sx, l // m.Sx
            out[l] = arr[sy * m.sub_ny:(sy + 1) * m.sub_ny, sx * m.sub_nx:(sx + 1) * m.sub_nx]
        return out

    def _sub_weights(self):
        m = self.mesh
        self.G11s, self.G12s, self.G22s = (self._sub_blocks(a) for a in (self.G11w, self.G12w, self.G22w))
        self.Jws = self._sub_blocks(self.Jw)
        Ws = scatter_add(self.Jws, m.P, m.sub_nx, m.sub_ny, (m.L, m.nly, m.nlx))
        bw = block_edge_weights(m.P, m.w, self._sub_blocks(self.s_xi), self._sub_blocks(self.s_eta))
        self.sub_edge_w = {dd.EDGE_W: bw["W"], dd.EDGE_E: bw["E"], dd.EDGE_S: bw["S"], dd.EDGE_N: bw["N"]}
        return Ws

    def edge_nodes(self, e):
        """(rows, cols, weights (L, n)) of subdomain edge e: arc-length GLL
        weights differ per subdomain on a mapped mesh."""
        m = self.mesh
        if e == dd.EDGE_W:
            rows, cols = np.arange(m.nly), np.zeros(m.nly, int)
        elif e == dd.EDGE_E:
            rows, cols = np.arange(m.nly), np.full(m.nly, m.nlx - 1)
        elif e == dd.EDGE_S:
            rows, cols = np.zeros(m.nlx, int), np.arange(m.nlx)
        else:
            rows, cols = np.full(m.nlx, m.nly - 1), np.arange(m.nlx)
        return rows, cols, self.sub_edge_w[e]

    def apply_A_sub(self, p, subs=None):
        m = self.mesh
        sel = slice(None) if subs is None else subs
        return stiffness_apply(p, m.P, m.D, self.G11s[sel], self.G12s[sel], self.G22s[sel])

    def sub_matrix(self, l):
        m = self.mesh
        A = stiffness_matrix(m.P, m.D, self.G11s[l], self.G12s[l], self.G22s[l])
        w = self.omega
        d = self.Hm_sub[l].ravel() - 1j * w * self.H_sub[l].ravel() - w * w * self.M_sub[l].ravel()
        return (A + sp.diags(d)).tocsc()

    def choose_nt(self, cfl=0.9):
        """N_t = max(3, ceil(T / dt_max)), dt_max = cfl * 2 / sqrt(lambda),
        lambda = c_max^2 * the element eigenvalue bound (element_eig_bound)."""
        m = self.mesh
        mu = element_eig_bound(m.P, m.D, self.Jw, self.G11w, self.G12w, self.G22w)
        lam = float(np.max(self.c)) ** 2 * mu
        dt_max = cfl * 2.0 / math.sqrt(lam)
        return max(3, int(math.ceil((2.0 * math.pi / self.omega) / dt_max)))
