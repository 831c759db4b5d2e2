"""Oracle of the overlapping additive Schwarz smoother (test infrastructure: plain CPU
FP64, imported only by tests and the benchmark's CPU baseline).

Section 4.3, Eqs. sec_form, Mass and weights: one smoothing step is the defect
correction u <- u + S^{-1} (f - A u) with

    S^{-1} = W sum_k R_k^T (R_k A R_k^T)^{-1} R_k,     W = (sum_k R_k R_k^T)^{-1},

R_k restricting to the subdomain of element k: the element's nodes and an overlap
zone of `overlap` nodes in every direction (Fig. schwarzsmoother, one node by
default; the "refined Schwarz" variant of Section 6 uses ceil((p+1)/2) nodes on
the order-p level).

Readings (the paper draws the subdomain on a structured picture only):
* lattice step: two nodes of one element whose local lattice indices -- (i, j),
  i + j <= p, of the triangle and k of the vertical GLL line -- differ by at most
  one in i, in j, in i + j and in k, and are not the same node.  The triangle
  steps are the six neighbours of the triangular lattice; with the vertical one
  this is "one node further in every direction, the diagonal corners included".
* the subdomain of element k with overlap l: the nodes within l lattice steps of
  element k's nodes (distance on the graph of all nodes, steps taken in any
  element), of which the free (non-Dirichlet) nodes form the block.  l = 0 is
  block Jacobi over the element node sets.
* R_k A R_k^T is the principal submatrix of the free-node matrix A_FF on those
  nodes; W counts, per free node, the subdomains holding it.
* the pre-smoothing steps apply S^{-1}; the post-smoothing steps apply its adjoint
  S^{-T} = sum_k R_k^T (R_k A R_k^T)^{-1} R_k W, so that the V-cycle is a
  symmetric operator, as the conjugate gradient outer iteration needs (the paper
  uses one form in both places; with W a multiple of the identity the two agree).
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

from .assemble import Problem
from .refelem import lattice


def local_lattice(dim: int, p: int, pz: int | None = None) -> np.ndarray:
    """Lattice indices (i, j, k) of the element's local nodes in local node order
    (k = 0 for triangles; k = 0..pz on the vertical line, pz = p unless given)."""
    tl = lattice(p)
    if dim == 2:
        return np.array([(i, j, 0) for (i, j) in tl], dtype=np.int64)
    pz = p if pz is None else pz
    return np.array([(i, j, k) for k in range(pz + 1) for (i, j) in tl], dtype=np.int64)


def lattice_steps(dim: int, p: int, pz: int | None = None):
    """For every local node, the local nodes one lattice step away."""
    lat = local_lattice(dim, p, pz)
    out = []
    for a in range(lat.shape[0]):
        nb = []
        for b in range(lat.shape[0]):
            if a == b:
                continue
            di, dj, dk = lat[b] - lat[a]
            if abs(di) <= 1 and abs(dj) <= 1 and abs(di + dj) <= 1 and abs(dk) <= 1:
                nb.append(b)
        out.append(nb)
    return out


def overlap_of(p: int, overlap: int) -> int:
    """Overlap in nodes on an order-p level (p the triangle order); overlap < 0 selects
    the refined Schwarz variant, ceil((p + 1) / 2)."""
    return math.ceil((p + 1) / 2) if overlap < 0 else overlap


def subdomains(prob: Problem, li: int, overlap: int = 1):
    """Sorted free global node ids of every element's subdomain on level li."""
    lev = prob.levels[li]
    ell = overlap_of(lev.p, overlap)
    steps = lattice_steps(prob.dim, lev.p, lev.pz)
    incid = [[] for _ in range(lev.N)]                 # node -> (element, local index)
    for e in range(lev.emap.shape[0]):
        for a, g in enumerate(lev.emap[e]):
            incid[g].append((e, a))
    subs = []
    for e in range(lev.emap.shape[0]):
        dist = {int(g): 0 for g in lev.emap[e]}
        queue = deque(dist)
        while queue:
            g = queue.popleft()
            if dist[g] == ell:
                continue
            for (e2, a) in incid[g]:
                for b in steps[a]:
                    h = int(lev.emap[e2, b])
                    if h not in dist:
                        dist[h] = dist[g] + 1
                        queue.append(h)
        nodes = np.array(sorted(dist), dtype=np.int64)
        subs.append(nodes[~lev.dmask[nodes]])
    return subs


def weights(prob: Problem, li: int, subs) -> np.ndarray:
    """Diagonal of W (Eq. weights): 1 / (number of subdomains holding the node) on the
    free nodes, 0 at the Dirichlet nodes."""
    lev = prob.levels[li]
    cnt = np.zeros(lev.N)
    for s in subs:
        cnt[s] += 1.0
    return np.where(cnt > 0, 1.0 / np.where(cnt > 0, cnt, 1.0), 0.0)


class Schwarz:
    """S^{-1} of one level: the subdomains, their dense blocks R_k A R_k^T and W."""

    def __init__(self, prob: Problem, li: int, A, overlap: int = 1):
        self.subs = subdomains(prob, li, overlap)
        self.w = weights(prob, li, self.subs)
        A = A.tocsr()
        self.blocks = [A[s][:, s].toarray() for s in self.subs]

    def apply(self, r: np.ndarray, adjoint: bool = False) -> np.ndarray:
        """S^{-1} r (Eq. Mass), or S^{-T} r with adjoint=True."""
        x = self.w * r if adjoint else r
        z = np.zeros_like(r)
        for s, Ak in zip(self.subs, self.blocks):
            if s.size:
                z[s] += np.linalg.solve(Ak, x[s])
        return z if adjoint else self.w * z

    def smooth(self, A, f, u, adjoint: bool = False) -> np.ndarray:
        """One step of Eq. sec_form: u + S^{-1} (f - A u)."""
        return u + self.apply(f - A @ u, adjoint)
