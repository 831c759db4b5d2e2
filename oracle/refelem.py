"""Reference elements of the Galerkin spectral element discretisation (Section 3.1).

The paper's V^p is the space of continuous piecewise polynomials of degree p
with a nodal (cardinal) basis N_i(x_j) = delta_ij.  It leaves the nodal set on
triangles/prisms open beyond naming Fekete points; the reading used here (and,
independently written, by the CUDA library) is:

* triangle: Warburton's warp & blend nodes with alpha = 0 (edge nodes are the
  Gauss-Lobatto-Legendre (GLL) points), on the reference triangle
  T = {r, s >= -1, r + s <= 0} with vertices v0=(-1,-1), v1=(1,-1), v2=(-1,1);
  lattice order: for j = 0..p, for i = 0..p-j, node (i, j);
* prism: triangle nodes x GLL nodes in t in [-1, 1]; local index k*NT + n;
* quadrature: collapsed Gauss rule on T with n = p+1 points per direction
  (Gauss-Legendre in a, Gauss-Jacobi(1,0) in b, r = (1+a)(1-b)/2 - 1, s = b,
  w = w_a w_b / 2) times Gauss-Legendre with p+1 points in t.

The oracle builds the Lagrange basis from the orthonormal collapsed-coordinate
modal basis (Jacobi polynomials from SciPy); any basis of P^p gives the same
Lagrange functions, this one keeps the Vandermonde matrix well conditioned.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import eval_jacobi, roots_jacobi


# ------------------------------------------------------------------ 1D rules
@lru_cache(maxsize=None)
def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (exact to degree 2n-1)."""
    x, w = npleg.leggauss(n)
    return np.asarray(x), np.asarray(w)


@lru_cache(maxsize=None)
def gauss_jacobi10(n: int):
    """n-point Gauss-Jacobi rule for the weight (1-b) on [-1, 1]."""
    x, w = roots_jacobi(n, 1.0, 0.0)
    return np.asarray(x), np.asarray(w)


@lru_cache(maxsize=None)
def gll(p: int) -> np.ndarray:
    """p+1 Gauss-Lobatto-Legendre points: -1, 1 and the roots of L_p'(x)."""
    if p == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(c))))
    return np.concatenate([[-1.0], inner, [1.0]])


def lagrange1d(xn: np.ndarray, x: np.ndarray):
    """Values and derivatives of the 1D Lagrange basis on nodes xn at points x.

    Returns (B, D) with B[q, k] = l_k(x_q), D[q, k] = l_k'(x_q), computed from
    the product formula l_k(x) = prod_{m != k} (x - x_m) / (x_k - x_m)."""
    xn = np.asarray(xn, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = xn.size
    B = np.ones((x.size, n))
    D = np.zeros((x.size, n))
    for k in range(n):
        den = 1.0
        for m in range(n):
            if m != k:
                den *= xn[k] - xn[m]
        for q in range(x.size):
            val = 1.0
            for m in range(n):
                if m != k:
                    val *= x[q] - xn[m]
            B[q, k] = val / den
            # derivative: sum over the dropped factor
            d = 0.0
            for j in range(n):
                if j == k:
                    continue
                prod = 1.0
                for m in range(n):
                    if m != k and m != j:
                        prod *= x[q] - xn[m]
                d += prod
            D[q, k] = d / den
    return B, D


# ------------------------------------------------------------------ triangle nodes
def lattice(p: int):
    """Lattice indices (i, j) of the order-p triangle in node order."""
    return [(i, j) for j in range(p + 1) for i in range(p + 1 - j)]


def _warp(p: int, tau: np.ndarray) -> np.ndarray:
    """Warp function of Warburton's construction: the equispaced-grid interpolant
    of (GLL - equispaced) displacements, divided by (1 - tau^2) inside (-1, 1)."""
    g = gll(p)
    e = np.linspace(-1.0, 1.0, p + 1)
    Beq, _ = lagrange1d(e, tau)
    w = Beq @ (g - e)
    out = np.zeros_like(tau)
    inside = np.abs(tau) < 1.0 - 1e-10
    out[inside] = w[inside] / (1.0 - tau[inside] ** 2)
    return out


@lru_cache(maxsize=None)
def tri_nodes(p: int) -> np.ndarray:
    """Warp & blend (alpha = 0) nodes on the reference triangle, shape [NT, 2] (r, s).

    Each lattice point starts at equispaced barycentrics (mu0, mu1, mu2) =
    (1 - (i+j)/p, i/p, j/p).  Along each edge (a, b) the point is displaced by
    d = 4 mu_a mu_b warp(mu_b - mu_a) in edge-length units (edge length 2),
    i.e. mu_b += d/2, mu_a -= d/2; the three edge displacements add up."""
    if p == 0:
        return np.array([[-1.0 / 3, -1.0 / 3]])
    lat = lattice(p)
    mu = np.array([[1.0 - (i + j) / p, i / p, j / p] for (i, j) in lat])
    new = mu.copy()
    for (a, b) in ((0, 1), (1, 2), (2, 0)):
        tau = mu[:, b] - mu[:, a]
        d = 4.0 * mu[:, a] * mu[:, b] * _warp(p, tau)
        new[:, b] += d / 2.0
        new[:, a] -= d / 2.0
    r = -1.0 + 2.0 * new[:, 1]
    s = -1.0 + 2.0 * new[:, 2]
    return np.stack([r, s], axis=1)


# ------------------------------------------------------------------ triangle basis
def _modal_tri(p: int, r: np.ndarray, s: np.ndarray):
    """Orthonormal collapsed-coordinate modal basis on T and its r/s derivatives.

    psi_ij(r, s) = sqrt(2) Pn_i^(0,0)(a) Pn_j^(2i+1,0)(b) (1-b)^i, i + j <= p, with
    a = 2(1+r)/(1-s) - 1 (a = -1 at s = 1), b = s and Pn the L2-normalised Jacobi
    polynomials; Jacobi values come from scipy.special.eval_jacobi and derivatives
    from d/dx P_n^(al,be) = (n+al+be+1)/2 P_{n-1}^(al+1,be+1)."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    one_m_s = 1.0 - s
    safe = np.abs(one_m_s) > 1e-14
    a = np.where(safe, 2.0 * (1.0 + r) / np.where(safe, one_m_s, 1.0) - 1.0, -1.0)
    b = s

    def norm(n, al, be):
        return math.sqrt(2.0 ** (al + be + 1) / (2 * n + al + be + 1)
                         * math.gamma(n + al + 1) * math.gamma(n + be + 1)
                         / (math.gamma(n + al + be + 1) * math.factorial(n)))

    def P(n, al, be, x):
        return eval_jacobi(n, al, be, x) / norm(n, al, be)

    def dP(n, al, be, x):
        if n == 0:
            return np.zeros_like(x)
        return 0.5 * (n + al + be + 1) * eval_jacobi(n - 1, al + 1, be + 1, x) / norm(n, al, be)

    cols, cr, cs = [], [], []
    for i in range(p + 1):
        for j in range(p + 1 - i):
            fa, dfa = P(i, 0, 0, a), dP(i, 0, 0, a)
            gb, dgb = P(j, 2 * i + 1, 0, b), dP(j, 2 * i + 1, 0, b)
            cols.append(math.sqrt(2.0) * fa * gb * one_m_s ** i)
            if i == 0:
                dr = np.zeros_like(r)
                ds = math.sqrt(2.0) * fa * dgb
            else:
                pim1 = one_m_s ** (i - 1)
                dr = math.sqrt(2.0) * 2.0 * dfa * gb * pim1
                ds = math.sqrt(2.0) * (dfa * (1.0 + a) * gb * pim1
                                       + fa * dgb * one_m_s ** i
                                       - i * fa * gb * pim1)
            cr.append(dr)
            cs.append(ds)
    return np.stack(cols, axis=1), np.stack(cr, axis=1), np.stack(cs, axis=1)


def tri_basis(p: int, pts: np.ndarray):
    """Order-p triangle Lagrange basis (cardinal at tri_nodes(p)) at points pts [npt, 2].

    Returns (B, Dr, Ds), each [npt, NT]: values and reference derivatives."""
    nodes = tri_nodes(p)
    V, _, _ = _modal_tri(p, nodes[:, 0], nodes[:, 1])
    Vinv = np.linalg.inv(V)
    M, Mr, Ms = _modal_tri(p, pts[:, 0], pts[:, 1])
    return M @ Vinv, Mr @ Vinv, Ms @ Vinv


@lru_cache(maxsize=None)
def tri_quadrature(n: int):
    """Collapsed Gauss rule on the reference triangle with n x n points: (pts [n*n, 2], w [n*n])."""
    a, wa = gauss_legendre(n)
    b, wb = gauss_jacobi10(n)
    pts, w = [], []
    for jb in range(n):
        for ia in range(n):
            r = (1.0 + a[ia]) * (1.0 - b[jb]) / 2.0 - 1.0
            pts.append((r, b[jb]))
            w.append(wa[ia] * wb[jb] / 2.0)
    return np.asarray(pts), np.asarray(w)


# ------------------------------------------------------------------ element objects
class RefTri:
    """Order-p reference triangle: nodes, quadrature (n = p+1), basis at quadrature points."""

    def __init__(self, p: int):
        self.p = p
        self.nodes = tri_nodes(p)
        self.NT = self.nodes.shape[0]
        self.Np = self.NT
        self.qpts, self.qw = tri_quadrature(p + 1)
        self.Nq = self.qw.size
        self.B, self.Dr, self.Ds = tri_basis(p, self.qpts)
        self.grads = np.stack([self.Dr, self.Ds])        # [2, Nq, Np]

    def face_nodes(self, f: int):
        lat = lattice(self.p)
        p = self.p
        if f == 0:
            return [n for n, (i, j) in enumerate(lat) if j == 0]
        if f == 1:
            return [n for n, (i, j) in enumerate(lat) if i + j == p]
        return [n for n, (i, j) in enumerate(lat) if i == 0]

    def basis_at(self, pts):
        """(B, grads[2]) of this order's basis at arbitrary reference points."""
        B, Dr, Ds = tri_basis(self.p, pts)
        return B, np.stack([Dr, Ds])


class RefPrism:
    """Reference prism T x [-1, 1] of order p on the triangle and pz in the vertical
    (pz = p unless given; Section 6 uses P_xy != P_z): nodes (triangle x GLL, index
    k*NT + n), quadrature (collapsed (p+1)^2 on T times (pz+1) Gauss-Legendre in t)."""

    def __init__(self, p: int, pz: int | None = None):
        pz = p if pz is None else pz
        self.p, self.pz = p, pz
        self.tri = RefTri(p)
        self.NT = self.tri.NT
        self.NZ = pz + 1
        self.Np = self.NT * self.NZ
        self.zn = gll(pz)
        tn = self.tri.nodes
        self.nodes = np.array([(tn[n, 0], tn[n, 1], self.zn[k])
                               for k in range(self.NZ) for n in range(self.NT)])
        zq, zw = gauss_legendre(pz + 1)
        tq, tw = self.tri.qpts, self.tri.qw
        self.qpts = np.array([(tq[a, 0], tq[a, 1], zq[c]) for c in range(zq.size) for a in range(tw.size)])
        self.qw = np.array([tw[a] * zw[c] for c in range(zq.size) for a in range(tw.size)])
        self.Nq = self.qw.size
        self.B, g = self.basis_at(self.qpts)
        self.grads = g

    def basis_at(self, pts):
        """(B [npt, Np], grads [3, npt, Np]) of the prism basis l_n(r,s) h_k(t) at points."""
        pts = np.asarray(pts)
        Bt, Drt, Dst = tri_basis(self.p, pts[:, :2])
        Bz, Dz = lagrange1d(self.zn, pts[:, 2])
        npt = pts.shape[0]
        B = np.empty((npt, self.Np))
        Gr = np.empty((npt, self.Np))
        Gs = np.empty((npt, self.Np))
        Gt = np.empty((npt, self.Np))
        for k in range(self.NZ):
            sl = slice(k * self.NT, (k + 1) * self.NT)
            B[:, sl] = Bt * Bz[:, k:k + 1]
            Gr[:, sl] = Drt * Bz[:, k:k + 1]
            Gs[:, sl] = Dst * Bz[:, k:k + 1]
            Gt[:, sl] = Bt * Dz[:, k:k + 1]
        return B, np.stack([Gr, Gs, Gt])

    def face_nodes(self, f: int):
        if f < 3:
            tf = self.tri.face_nodes(f)
            return [k * self.NT + n for k in range(self.NZ) for n in tf]
        k = 0 if f == 3 else self.pz
        return [k * self.NT + n for n in range(self.NT)]


def ref_element(dim: int, p: int, pz: int | None = None):
    return RefTri(p) if dim == 2 else RefPrism(p, pz)


def interpolation_matrix(dim: int, pf: int, pc: int, pzf: int | None = None, pzc: int | None = None) -> np.ndarray:
    """Element prolongation I [Np_f, Np_c]: the coarse basis (order pc, vertical pzc) at the
    fine nodes (order pf, vertical pzf).

    Nested spaces (Section 4.1; semi-coarsening of Section 6 lowers one direction only):
    a coarse polynomial is reproduced exactly at the fine nodes, so I is the element block
    of the global prolongation P."""
    fine = ref_element(dim, pf, pzf)
    coarse = ref_element(dim, pc, pzc)
    B, _ = coarse.basis_at(fine.nodes)
    return B
