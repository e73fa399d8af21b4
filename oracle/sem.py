"""Spectral-element pieces of the oracle (test infrastructure only).

Sec. 4 of the paper: degree-P tensor-product Lagrange basis on
Gauss-Lobatto-Legendre (GLL) nodes, quadrilateral elements, integrals
evaluated by the collocated GLL rule so that M and H are diagonal (mass
lumping).  The stiffness apply follows Sec. 6.1: the gradient of p is formed
at every quadrature point from rows of the 1D differentiation matrix D, scaled
by the quadrature weight and metric, then contracted with D^T and summed into
the nodes it belongs to.

Arrays on node grids are indexed ``[y, x]`` (x fastest in memory).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as npleg


# ---------------------------------------------------------------- 1D basis --
def gll(P: int):
    """GLL nodes x_0=-1 < ... < x_P=1 and weights (Sec. 4, lumped quadrature).

    Interior nodes are the roots of L_P'(x) (NumPy's Legendre root finder,
    polished by Newton steps); w_i = 2 / (P (P+1) L_P(x_i)^2).
    Pinned by closed forms for P = 1..4 and by exactness on polynomials of
    degree <= 2P-1 (tests/test_oracle_sem.py).
    """
    if P < 1:
        raise ValueError("degree must be >= 1")
    cP = np.zeros(P + 1)
    cP[P] = 1.0
    dcP = npleg.legder(cP)
    d2cP = npleg.legder(dcP)
    if P >= 2:
        r = np.sort(npleg.legroots(dcP).real)
        for _ in range(4):
            r = r - npleg.legval(r, dcP) / npleg.legval(r, d2cP)
        x = np.concatenate(([-1.0], r, [1.0]))
    else:
        x = np.array([-1.0, 1.0])
    LP = npleg.legval(x, cP)
    w = 2.0 / (P * (P + 1) * LP**2)
    return x, w


def diff_matrix(x):
    """D[q, a] = l_a'(x_q) for the Lagrange basis on nodes x (barycentric form).

    Pinned: D applied to nodal values of x^k equals k x^(k-1) for k <= P.
    """
    n = len(x)
    lam = np.array([1.0 / np.prod([x[a] - x[b] for b in range(n) if b != a]) for a in range(n)])
    D = np.zeros((n, n))
    for q in range(n):
        for a in range(n):
            if a != q:
                D[q, a] = (lam[a] / lam[q]) / (x[q] - x[a])
        D[q, q] = -np.sum(D[q, :])
    return D


# -------------------------------------------------------------------- mesh --
@dataclass
class Mesh:
    """Structured quad mesh of [x0,x1]x[y0,y1], nx*ny elements, degree P,
    split into non-overlapping subdomains of sub_nx*sub_ny elements (Sec. 3,
    Fig. 1).  Global nodes: (nx*P+1)*(ny*P+1), x fastest."""

    x0: float
    x1: float
    y0: float
    y1: float
    nx: int
    ny: int
    P: int
    sub_nx: int
    sub_ny: int

    def __post_init__(self):
        if self.nx % self.sub_nx or self.ny % self.sub_ny:
            raise ValueError("subdomain size must divide the mesh")
        self.hx = (self.x1 - self.x0) / self.nx
        self.hy = (self.y1 - self.y0) / self.ny
        self.xi, self.w = gll(self.P)
        self.D = diff_matrix(self.xi)
        self.NX = self.nx * self.P + 1
        self.NY = self.ny * self.P + 1
        self.Sx = self.nx // self.sub_nx
        self.Sy = self.ny // self.sub_ny
        self.L = self.Sx * self.Sy
        self.nlx = self.sub_nx * self.P + 1
        self.nly = self.sub_ny * self.P + 1
        self.NE = max(self.nlx, self.nly)

    # node coordinates ------------------------------------------------------
    def coords_1d(self):
        P = self.P
        gx = np.empty(self.NX)
        for e in range(self.nx):
            gx[e * P : e * P + P + 1] = self.x0 + e * self.hx + (self.xi + 1.0) * self.hx / 2.0
        gy = np.empty(self.NY)
        for e in range(self.ny):
            gy[e * P : e * P + P + 1] = self.y0 + e * self.hy + (self.xi + 1.0) * self.hy / 2.0
        return gx, gy

    def coords(self):
        """(NY, NX) arrays X, Y of node positions."""
        gx, gy = self.coords_1d()
        return np.meshgrid(gx, gy)

    # lumped 1D weights ------------------------------------------------------
    def lumped_1d(self, n_el, h):
        """Assembled lumped 1D mass over n_el elements of size h: sum of
        w_a*h/2 over the elements touching each node."""
        P = self.P
        W = np.zeros(n_el * P + 1)
        for e in range(n_el):
            W[e * P : e * P + P + 1] += self.w * h / 2.0
        return W

    def boundary_rhs(self, g):
        """<g, phi> on the outer boundary by GLL quadrature along each edge.

        g: dict with keys 'S','E','N','W', complex arrays along increasing x
        (S,N) or y (E,W).  Returns the (NY, NX) complex weak-form vector.
        """
        Wx = self.lumped_1d(self.nx, self.hx)
        Wy = self.lumped_1d(self.ny, self.hy)
        out = np.zeros((self.NY, self.NX), complex)
        out[0, :] += Wx * g["S"]
        out[-1, :] += Wx * g["N"]
        out[:, 0] += Wy * g["W"]
        out[:, -1] += Wy * g["E"]
        return out


# ---------------------------------------------- element-form operator apply --
def element_view(u, P, nex, ney):
    """u on a block of ney x nex elements -> (..., ney, nex, P+1, P+1)
    element-local copies indexed [.., ey, ex, b(y), a(x)]."""
    out = np.empty(u.shape[:-2] + (ney, nex, P + 1, P + 1), dtype=u.dtype)
    for b in range(P + 1):
        for a in range(P + 1):
            out[..., b, a] = u[..., b : b + ney * P : P, a : a + nex * P : P]
    return out


def scatter_add(ue, P, nex, ney, shape):
    """Sum element-local contributions back onto the node grid (assembly)."""
    out = np.zeros(shape, dtype=ue.dtype)
    for b in range(P + 1):
        for a in range(P + 1):
            out[..., b : b + ney * P : P, a : a + nex * P : P] += ue[..., b, a]
    return out


def stiffness_apply(u, P, D, w, hx, hy, nex, ney):
    """(A u) for A_ij = (grad phi_j, grad phi_i) on a block of uniform
    rectangular elements, matrix-free (Sec. 4 eq. for A; Sec. 6.1 procedure).

    Per element: gradient of u at each GLL point (q,r) from rows of D,
    scaled by w_q w_r |J| and the squared metric (2/h)^2, then contracted with
    D^T and summed into the nodes (assembly).  u: (..., ney*P+1, nex*P+1).
    Pinned: A 1 = 0; v^T A u = integral grad u . grad v for polynomials
    (tests/test_oracle_sem.py).
    """
    ue = element_view(u, P, nex, ney)
    J = hx * hy / 4.0
    wq = w[None, :]  # weight along x index q
    wr = w[:, None]  # weight along y index r
    # d/dxi at (r, q): sum_a D[q,a] u[r,a];  d/deta at (r, q): sum_b D[r,b] u[b,q]
    dxi = np.einsum("...ra,qa->...rq", ue, D)
    deta = np.einsum("...bq,rb->...rq", ue, D)
    gx = dxi * (wr * wq) * J * (2.0 / hx) ** 2
    gy = deta * (wr * wq) * J * (2.0 / hy) ** 2
    # contract with D^T: (A u)[b', a'] = sum_q D[q,a'] gx[b',q] + sum_r D[r,b'] gy[r,a']
    contrib = np.einsum("...bq,qa->...ba", gx, D) + np.einsum("...ra,rb->...ba", gy, D)
    return scatter_add(contrib, P, nex, ney, u.shape)


def stiffness_matrix(P, D, w, hx, hy, nex, ney):
    """Assembled sparse A on a block of elements (same quadrature), built from
    element matrices K_e = (hy/hx) (D^T W D) (x) W + (hx/hy) W (x) (D^T W D).
    Used by the direct global solve (the plain definition of the result)."""
    import scipy.sparse as sp

    W = np.diag(w)
    K1 = D.T @ W @ D  # 1D reference stiffness (integral l_a' l_b' on [-1,1])
    Ke = (hy / hx) * np.kron(W, K1) + (hx / hy) * np.kron(K1, W)  # index (b,a) row-major: y outer
    nX = nex * P + 1
    rows, cols, vals = [], [], []
    loc = np.array([[b * nX + a for a in range(P + 1)] for b in range(P + 1)]).ravel()
    for ey in range(ney):
        for ex in range(nex):
            g = loc + ey * P * nX + ex * P
            rows.append(np.repeat(g, len(g)))
            cols.append(np.tile(g, len(g)))
            vals.append(Ke.ravel())
    n = nX * (ney * P + 1)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A.tocsr()


def nested_dissection_order(NX, NY, P, leaf=256):
    """Fill-reducing elimination order of the NX x NY node grid (x fastest)
    for a sparse direct solve: recursive bisection by node lines.  A node row
    or column on an element boundary separates the nodes on its two sides
    (they share no element, so the stiffness couples them only through it);
    each half is ordered first, the separator last.  Blocks of at most `leaf`
    nodes keep their natural order.  Returns a permutation of range(NX NY).
    Used only to make the oracle's direct solves of the larger test meshes
    affordable (the factorisation is the same LU)."""
    out = []

    def natural(i0, i1, j0, j1):
        out.extend(J * NX + I for J in range(j0, j1) for I in range(i0, i1))

    def rec(i0, i1, j0, j1):
        w, h = i1 - i0, j1 - j0
        if w * h <= leaf:
            natural(i0, i1, j0, j1)
            return
        if w >= h:
            s = i0 + ((w // 2) // P) * P  # an element-boundary column
            if s <= i0 or s >= i1 - 1:
                natural(i0, i1, j0, j1)
                return
            rec(i0, s, j0, j1)
            rec(s + 1, i1, j0, j1)
            out.extend(J * NX + s for J in range(j0, j1))
        else:
            s = j0 + ((h // 2) // P) * P
            if s <= j0 or s >= j1 - 1:
                natural(i0, i1, j0, j1)
                return
            rec(i0, i1, j0, s)
            rec(i0, i1, s + 1, j1)
            out.extend(s * NX + I for I in range(i0, i1))

    rec(0, NX, 0, NY)
    return np.asarray(out)

