"""Geometry and the assembled stiffness matrix (Section 3.1, Eq. laplaceproblemdiscrete).

For the order-p level the element matrix is the Galerkin stiffness

    A_e[i, j] = sum_q w_q |det J_q| (J_q^{-T} grad N_i(xi_q)) . (J_q^{-T} grad N_j(xi_q)),

i.e. minus the paper's L^p_ij (the sign is flipped so that A is symmetric
positive definite on the free nodes).  J_q is the Jacobian of the isoparametric
order-P geometry map x(xi) = sum_i X_i N^P_i(xi) (the finest order P, also on
the coarse levels: coarse operators are re-discretised with the finest
geometry, the "direct assembly" option of Section 4.4).  In 3D the nodes of the
order-P map are x, y affine over the base triangle and z = -h + sigma (h + eta)
in sigma layers, which reproduces the sigma-transform of Section 3.1.  A mesh may
instead give curved base triangles (x, y from the blended map of oracle.mesh at the
order-P nodes) and layer interfaces z_k = a_k + b_k eta (two vertical zones around
a hull): within layer l the node at local t sits at
z = (1 - tau) z_l + tau z_{l+1}, tau = (t + 1)/2.

The global matrix is A = sum_e Q_e^T A_e Q_e (COO with duplicates summed).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Level, blended_xy, interfaces
from .refelem import RefPrism, RefTri, tri_basis


class Problem:
    """Mesh + p-levels (finest first) + the order-P geometry.

    ``levels``: orders p, or (p, pz) pairs for prisms whose vertical order differs
    (semi-coarsening, Section 6).  The geometry is the order-P map of the finest triangle
    order P (the sigma map is linear in t within a layer, so its vertical order is exact).
    ``eta_nodal``: eta at the finest level's 2D nodes (canonical numbering); by
    default the mesh's eta evaluated there."""

    def __init__(self, mesh, levels, eta_nodal=None):
        self.mesh = mesh
        self.dim = mesh.dim
        self.levels = [Level(mesh, *(spec if isinstance(spec, (tuple, list)) else (spec,))) for spec in levels]
        fin = self.levels[0]
        self.P = fin.p
        if mesh.dim == 3:
            if eta_nodal is None:
                eta_nodal = np.zeros(fin.N2)
                for b in range(mesh.tri.shape[0]):
                    xy = self.base_xy_P(b)
                    eta_nodal[fin.map2[b]] = mesh.eta(xy[:, 0], xy[:, 1])
            self.eta_nodal = np.asarray(eta_nodal, dtype=np.float64)
        else:
            self.eta_nodal = None
        self._A = {}

    # ----------------------------------------------------------- coordinates
    def general(self) -> bool:
        """True for meshes with curved base triangles, partial columns or given
        layer interfaces (the hull tank)."""
        m = self.mesh
        return m.dim == 3 and (m.edge_arc is not None or m.col_layers is not None or m.z_iface is not None)

    def _tri_nodes(self, p: int) -> np.ndarray:
        """Reference nodes of the order-p triangle (built once per order: the per-triangle
        loops below would otherwise rebuild the same reference element thousands of times)."""
        cache = self.__dict__.setdefault("_tn_cache", {})
        if p not in cache:
            cache[p] = RefTri(p).nodes
        return cache[p]

    def base_xy_P(self, b: int) -> np.ndarray:
        """(x, y) of the order-P nodes of base triangle b [NT_P, 2]."""
        tn = self._tri_nodes(self.P)
        if self.mesh.dim == 3 and self.mesh.edge_arc is not None:
            return blended_xy(self.mesh, b, tn)
        return self.levels[0].tri_node_xy(b, tn)

    def base_xy(self, li: int, b: int) -> np.ndarray:
        """(x, y) of level li's 2D nodes in base triangle b: the order-P map (the
        interpolant of the order-P nodes) at the level's nodes."""
        lev = self.levels[li]
        tn = self._tri_nodes(lev.p)
        if self.mesh.dim == 3 and self.mesh.edge_arc is not None:
            B, _, _ = tri_basis(self.P, tn)
            return B @ self.base_xy_P(b)
        return lev.tri_node_xy(b, tn)

    def eta_at_level(self, li: int) -> np.ndarray:
        """eta_P (the order-P surface interpolant) at level li's 2D nodes."""
        lev, fin = self.levels[li], self.levels[0]
        if li == 0:
            return self.eta_nodal.copy()
        B, _, _ = tri_basis(self.P, RefTri(lev.p).nodes)
        out = np.zeros(lev.N2)
        for b in range(self.mesh.tri.shape[0]):
            out[lev.map2[b]] = B @ self.eta_nodal[fin.map2[b]]
        return out

    def coords(self, li: int) -> np.ndarray:
        """Physical coordinates [N, dim] of level li's global nodes; in 3D
        z = -h + sigma (h + eta_P) at the node."""
        lev, mesh = self.levels[li], self.mesh
        xy2 = np.zeros((lev.N2, 2))
        for b in range(mesh.tri.shape[0]):
            xy2[lev.map2[b]] = self.base_xy(li, b)
        if self.dim == 2:
            return xy2
        eta2 = self.eta_at_level(li)
        zn = RefPrism(lev.p, lev.pz).zn
        nl, h = mesh.nlayers, mesh.depth
        zif = interfaces(mesh)
        out = np.zeros((lev.N, 3))
        for kz in range(nl * lev.pz + 1):
            l, k = divmod(kz, lev.pz)
            if l == nl:
                l, k = nl - 1, lev.pz
            sl = slice(kz * lev.N2, (kz + 1) * lev.N2)
            out[sl, :2] = xy2
            out[sl, 2] = self._z(l, zn[k], eta2, zif)
        return out

    def _z(self, l, t, eta, zif):
        """z of the point at local t in layer l over surface elevation eta."""
        mesh = self.mesh
        if not self.general():
            nl, h = mesh.nlayers, mesh.depth
            return -h + (l + (t + 1.0) / 2.0) / nl * (h + eta)
        tau = (t + 1.0) / 2.0
        return ((1 - tau) * (zif[l, 0] + zif[l, 1] * eta) + tau * (zif[l + 1, 0] + zif[l + 1, 1] * eta))

    # ----------------------------------------------------------- geometry
    def element_nodes_P(self, elements=None) -> np.ndarray:
        """Coordinates of the order-P nodes of the given elements (default all), [E, Np_P, dim]."""
        mesh, P = self.mesh, self.P
        fin = self.levels[0]
        tn = RefTri(P).nodes
        elems = np.arange(mesh.nelem) if elements is None else np.asarray(elements)
        if self.dim == 2:
            X = np.empty((elems.size, tn.shape[0], 2))
            for i, b in enumerate(elems):
                X[i] = fin.tri_node_xy(b, tn)
            return X
        ref = RefPrism(P)
        cb, cl = mesh.columns()
        zif = interfaces(mesh)
        X = np.empty((elems.size, ref.Np, 3))
        for i, e in enumerate(elems):
            b, l = int(cb[e]), int(cl[e])
            xy = self.base_xy_P(b)
            eta = self.eta_nodal[fin.map2[b]]
            for k in range(P + 1):
                sl = slice(k * ref.NT, (k + 1) * ref.NT)
                X[i, sl, :2] = xy
                X[i, sl, 2] = self._z(l, ref.zn[k], eta, zif)
        return X

    def jacobians(self, li: int, elements=None) -> np.ndarray:
        """J[e, q, d, a] = d x_d / d xi_a of the order-P map at level li's quadrature points."""
        lev = self.levels[li]
        refP = RefTri(self.P) if self.dim == 2 else RefPrism(self.P)
        _, gP = refP.basis_at(lev.ref.qpts)            # [dim, Nq, NpP]
        X = self.element_nodes_P(elements)
        return np.einsum("eid,aqi->eqda", X, gP)

    def geometric_factors(self, li: int, elements=None) -> np.ndarray:
        """G[e, q, a, b] = w_q |det J| (J^{-1} J^{-T})_{ab} at level li's quadrature points."""
        J = self.jacobians(li, elements)
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)                          # [e, q, a, d]
        w = self.levels[li].ref.qw
        return (w[None, :, None, None] * np.abs(det)[:, :, None, None]
                * np.einsum("eqad,eqbd->eqab", Jinv, Jinv))

    # ----------------------------------------------------------- matrices
    def element_matrices(self, li: int, elements=None) -> np.ndarray:
        """A_e [E, Np, Np] of level li from the definition (sum over quadrature points)."""
        lev = self.levels[li]
        G = self.geometric_factors(li, elements)
        g = lev.ref.grads                                  # [dim, Nq, Np]
        dim, Nq, Np = g.shape
        # H[e, a, q, j] = sum_b G[e, q, a, b] g[b, q, j]; A_e = sum_{a,q} g[a, q, i] H[e, a, q, j]
        H = np.einsum("eqab,bqj->eaqj", G, g)
        return np.matmul(g.reshape(dim * Nq, Np).T[None], H.reshape(-1, dim * Nq, Np))

    def stiffness(self, li: int) -> sp.csr_matrix:
        """Assembled global A (all nodes, no boundary conditions), CSR."""
        if li in self._A:
            return self._A[li]
        lev = self.levels[li]
        Ae = self.element_matrices(li)
        E, Np = lev.emap.shape
        rows = np.repeat(lev.emap, Np, axis=1).ravel()
        cols = np.tile(lev.emap, (1, Np)).ravel()
        A = sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(lev.N, lev.N)).tocsr()
        A.sum_duplicates()
        self._A[li] = A
        return A

    def free_matrix(self, li: int) -> sp.csr_matrix:
        """A_FF: rows and columns of the free (non-Dirichlet) nodes."""
        lev = self.levels[li]
        A = self.stiffness(li)
        return A[lev.free][:, lev.free].tocsr()

    def masked_apply(self, li: int, x: np.ndarray) -> np.ndarray:
        """The library's sem_apply convention: y_F = A_FF x_F, y_D = x_D."""
        lev = self.levels[li]
        A = self.stiffness(li)
        xf = np.where(lev.dmask, 0.0, x)
        y = A @ xf
        return np.where(lev.dmask, x, y)

    def apply_rows(self, li: int, x: np.ndarray, rows: np.ndarray, masked: bool = True) -> np.ndarray:
        """Rows of the masked apply (y_F = A_FF x_F, y_D = x_D), or of the plain
        product A x (masked=False), computed one by one from the element matrices
        of the elements containing each row's node."""
        lev = self.levels[li]
        rows = np.asarray(rows)
        hit = np.isin(lev.emap, rows)
        elems = np.flatnonzero(hit.any(axis=1))
        Ae = self.element_matrices(li, elems)
        xf = np.where(lev.dmask, 0.0, x) if masked else x
        out = {int(r): 0.0 for r in rows}
        for k, e in enumerate(elems):
            ye = Ae[k] @ xf[lev.emap[e]]
            for l, g in enumerate(lev.emap[e]):
                if int(g) in out:
                    out[int(g)] += ye[l]
        return np.array([x[r] if (masked and lev.dmask[r]) else out[int(r)] for r in rows])
