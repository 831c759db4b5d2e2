"""Global node numbering, Dirichlet node sets and node coordinates (Section 3.1).

The global basis {N_i^p} of V^p is identified with the distinct mesh nodes.
The canonical numbering (shared as a *definition* with the CUDA library, which
implements it independently) is:

* triangles (2D, and the base of the 3D mesh): first appearance when visiting
  elements in order and their local nodes in lattice order; a vertex node is
  identified by its vertex id, an edge node by (edge, position counted from the
  lower vertex id), an interior node is new;
* prisms: global id = kz * N2 + g2, with g2 the 2D id of the base-triangle node
  and kz = l*p + k the vertical node index (l layer, k local GLL index).  Prisms
  are taken column by column, bottom up (mesh.columns()); a column may hold fewer
  than nlayers prisms (the hull tank).

A node is Dirichlet when it lies on a face flagged Dirichlet (closure).  On a mesh
whose columns are not all full some ids belong to no element (above the hull): no
basis function lives there, and the library keeps them as identity rows listed with
the Dirichlet nodes, so this numbering does the same.

Curved base triangles (the hull's rounded corners) are given by the circle each
curved edge follows.  The exact map of a base triangle is the straight-sided
(affine) map plus, for every curved edge (a, b), the edge's displacement from its
chord carried into the triangle by the blending factor 4 l_a l_b / (1 - xi^2),
xi = l_b - l_a (l the barycentric coordinates): the blending-function method for
triangles of Szabo and Babuska (Finite Element Analysis, 1991, Ch. 6), with the arc
point at angle theta_a + (1 + xi)/2 (theta_b - theta_a).  The factor is one on the
edge and zero on the other two; the element geometry is the order-P interpolant of
this map at the order-P nodes (isoparametric).
"""
from __future__ import annotations

import math

import numpy as np

from .refelem import RefPrism, RefTri, lattice


def tri_numbering(tri: np.ndarray, p: int):
    """First-appearance global numbering of the order-p triangle nodes.

    Returns (emap [ntri, NT] int64, N2)."""
    lat = lattice(p)
    keys = {}
    emap = np.empty((tri.shape[0], len(lat)), dtype=np.int64)
    for e in range(tri.shape[0]):
        v0, v1, v2 = (int(v) for v in tri[e])
        for n, (i, j) in enumerate(lat):
            if (i, j) == (0, 0):
                key = ("V", v0)
            elif (i, j) == (p, 0):
                key = ("V", v1)
            elif (i, j) == (0, p):
                key = ("V", v2)
            else:
                if j == 0:
                    va, vb, pos = v0, v1, i
                elif i + j == p:
                    va, vb, pos = v1, v2, j
                elif i == 0:
                    va, vb, pos = v2, v0, p - j
                else:
                    va = None
                if va is None:
                    key = ("I", e, n)
                else:
                    if va > vb:
                        va, vb, pos = vb, va, p - pos
                    key = ("E", va, vb, pos)
            g = keys.get(key)
            if g is None:
                g = len(keys)
                keys[key] = g
            emap[e, n] = g
    return emap, len(keys)


class Level:
    """One p-level of the mesh: numbering, Dirichlet set, reference element."""

    def __init__(self, mesh, p: int, pz: int | None = None):
        pz = p if pz is None else pz
        self.mesh = mesh
        self.p, self.pz = p, pz                      # triangle order, vertical order (3D)
        self.dim = mesh.dim
        map2, N2 = tri_numbering(mesh.tri, p)
        self.map2, self.N2 = map2, N2
        if mesh.dim == 2:
            self.ref = RefTri(p)
            self.emap = map2
            self.N = N2
        else:
            self.ref = RefPrism(p, pz)
            nl = mesh.nlayers
            NT = self.ref.NT
            cb, cl = mesh.columns()
            emap = np.empty((cb.size, self.ref.Np), dtype=np.int64)
            for e in range(cb.size):
                b, l = int(cb[e]), int(cl[e])
                for k in range(pz + 1):
                    kz = l * pz + k
                    emap[e, k * NT:(k + 1) * NT] = kz * N2 + map2[b]
            self.emap = emap
            self.N = N2 * (nl * pz + 1)
        dmask = np.zeros(self.N, dtype=bool)
        fb = mesh.face_bc
        faces = [np.asarray(self.ref.face_nodes(f)) for f in range(fb.shape[1])]
        for e, f in zip(*np.nonzero(fb)):
            dmask[self.emap[e, faces[f]]] = True
        held = np.zeros(self.N, dtype=bool)
        held[self.emap.ravel()] = True
        dmask |= ~held                       # ids in no element: identity rows
        self.dmask = dmask
        self.free = np.flatnonzero(~dmask)
        self.dirichlet = np.flatnonzero(dmask)

    # ------------------------------------------------------------ coordinates
    def tri_node_xy(self, b: int, pts: np.ndarray) -> np.ndarray:
        """Physical (x, y) of reference triangle points pts [n, 2] in base triangle b:
        the affine map x = -(r+s)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2 (straight triangles;
        curved ones go through blended_xy and the order-P interpolant)."""
        v = self.mesh.vxy[self.mesh.tri[b]]
        r, s = pts[:, 0], pts[:, 1]
        return (np.outer(-(r + s) / 2, v[0]) + np.outer((1 + r) / 2, v[1])
                + np.outer((1 + s) / 2, v[2]))


def blended_xy(mesh, b: int, pts: np.ndarray) -> np.ndarray:
    """Exact map of base triangle b at reference points pts [n, 2]: the affine map plus
    the blended displacement of every curved edge (module docstring)."""
    v = mesh.vxy[mesh.tri[b]]
    r, s = pts[:, 0], pts[:, 1]
    lam = (-(r + s) / 2, (1 + r) / 2, (1 + s) / 2)
    x = lam[0][:, None] * v[0] + lam[1][:, None] * v[1] + lam[2][:, None] * v[2]
    if mesh.edge_arc is None:
        return x
    for f, (ia, ib) in enumerate(((0, 1), (1, 2), (2, 0))):
        cx, cy, R = mesh.edge_arc[b, f]
        if R <= 0.0:
            continue
        c = np.array([cx, cy])
        ta = math.atan2(v[ia, 1] - cy, v[ia, 0] - cx)
        tb = math.atan2(v[ib, 1] - cy, v[ib, 0] - cx)
        dth = math.remainder(tb - ta, 2 * math.pi)       # the shorter way round
        xi = lam[ib] - lam[ia]
        th = ta + 0.5 * (1 + xi) * dth
        arcpt = c + R * np.stack([np.cos(th), np.sin(th)], axis=1)
        chord = (0.5 * (1 - xi))[:, None] * v[ia] + (0.5 * (1 + xi))[:, None] * v[ib]
        den = 1.0 - xi * xi
        fac = np.where(den > 1e-13, 4.0 * lam[ia] * lam[ib] / np.where(den > 1e-13, den, 1.0), 0.0)
        x = x + fac[:, None] * (arcpt - chord)
    return x


def interfaces(mesh) -> np.ndarray:
    """[nlayers+1, 2]: interface k at z = a_k + b_k eta (sigma layers when not given)."""
    if mesh.z_iface is not None:
        return np.asarray(mesh.z_iface, dtype=np.float64)
    nl, h = mesh.nlayers, mesh.depth
    k = np.arange(nl + 1) / nl
    return np.stack([-h * (1 - k), k], axis=1)
