"""Global node numbering, Dirichlet node sets and node coordinates (Section 3.1).

The global basis {N_i^p} of V^p is identified with the distinct mesh nodes.
The canonical numbering (shared as a *definition* with the CUDA library, which
implements it independently) is:

* triangles (2D, and the base of the 3D mesh): first appearance when visiting
  elements in order and their local nodes in lattice order; a vertex node is
  identified by its vertex id, an edge node by (edge, position counted from the
  lower vertex id), an interior node is new;
* prisms: global id = kz * N2 + g2, with g2 the 2D id of the base-triangle node
  and kz = l*p + k the vertical node index (l layer, k local GLL index).

A node is Dirichlet when it lies on a face flagged Dirichlet (closure).
"""
from __future__ import annotations

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
            E = mesh.tri.shape[0] * nl
            emap = np.empty((E, self.ref.Np), dtype=np.int64)
            for b in range(mesh.tri.shape[0]):
                for l in range(nl):
                    e = b * nl + l
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
        self.dmask = dmask
        self.free = np.flatnonzero(~dmask)
        self.dirichlet = np.flatnonzero(dmask)

    # ------------------------------------------------------------ coordinates
    def tri_node_xy(self, b: int, pts: np.ndarray) -> np.ndarray:
        """Physical (x, y) of reference triangle points pts [n, 2] in base triangle b:
        the affine map x = -(r+s)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2."""
        v = self.mesh.vxy[self.mesh.tri[b]]
        r, s = pts[:, 0], pts[:, 1]
        return (np.outer(-(r + s) / 2, v[0]) + np.outer((1 + r) / 2, v[1])
                + np.outer((1 + s) / 2, v[2]))
