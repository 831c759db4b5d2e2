"""Pins of the additive Schwarz smoother's oracle (Section 4.3, Eqs. sec_form, Mass,
weights; Fig. schwarzsmoother).

* the lattice step: the six neighbours of the triangular lattice (interior 6, edge 4,
  vertex 2 in one triangle) and the vertical line (prism counts as products);
* subdomain sizes in closed form: on two triangles sharing an edge the overlap of
  element 0 is the first l rows of the other triangle parallel to the edge; on two
  prism columns of two layers it is the product of that row with one vertical level;
* at order 1 the subdomain with one node of overlap is the closed vertex
  neighbourhood of the element along the mesh edges (2D) and the union of the
  elements sharing a node with it (prisms), computed here from the mesh alone;
* zero overlap: the element's own free nodes, W = 1 / (elements sharing the node);
* a subdomain covering every free node makes S^{-1} = A_FF^{-1}: one step solves;
* the V-cycle with S^{-1} before and S^{-T} after the coarse correction is symmetric,
  while S^{-1} on both sides is not (W is not a multiple of the identity);
* ASM-preconditioned PCG reaches the direct solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import schwarz as SZ
from oracle import solvers as S
from oracle.assemble import Problem


def _tri_counts(p):
    # number of lattice steps from each triangle node inside one triangle
    steps = SZ.lattice_steps(2, p)
    lat = SZ.local_lattice(2, p)
    out = {}
    for a, (i, j, _) in enumerate(lat):
        vert = (i, j) in ((0, 0), (p, 0), (0, p))
        edge = (j == 0 or i == 0 or i + j == p) and not vert
        kind = "vertex" if vert else ("edge" if edge else "interior")
        out.setdefault(kind, set()).add(len(steps[a]))
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_triangle_lattice_steps(p):
    c = _tri_counts(p)
    assert c["vertex"] == {2}
    if p >= 2:
        assert c["edge"] == {4}
    if p >= 3:
        assert c["interior"] == {6}


@pytest.mark.parametrize("p", [1, 2, 4])
def test_prism_lattice_steps(p):
    tri = SZ.lattice_steps(2, p)
    pr = SZ.lattice_steps(3, p)
    NT = len(tri)
    for k in range(p + 1):
        nz = 2 if k in (0, p) else 3
        for n in range(NT):
            assert len(pr[k * NT + n]) == (len(tri[n]) + 1) * nz - 1


def _no_dirichlet(mesh):
    mesh.face_bc = np.zeros_like(mesh.face_bc)
    return mesh


@pytest.mark.parametrize("p", [1, 2, 3, 5])
@pytest.mark.parametrize("ell", [0, 1, 2])
def test_two_triangles_closed_form(p, ell):
    mesh = _no_dirichlet(W.slice2d(1, 1))
    prob = Problem(mesh, [p])
    sub = SZ.subdomains(prob, 0, ell)
    NT = (p + 1) * (p + 2) // 2
    rows = sum(p + 1 - j for j in range(1, min(ell, p) + 1))
    assert len(sub[0]) == NT + rows
    assert len(sub[1]) == NT + rows


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_two_prism_columns_closed_form(p):
    mesh = _no_dirichlet(W.box3d(1, 1, 2))       # base: two triangles; two layers
    prob = Problem(mesh, [p])
    NT = (p + 1) * (p + 2) // 2
    sub0 = SZ.subdomains(prob, 0, 0)
    sub1 = SZ.subdomains(prob, 0, 1)
    # element 0 = column 0, layer 0
    assert len(sub0[0]) == NT * (p + 1)
    assert len(sub1[0]) == (NT + p) * (p + 2)


def test_order1_triangles_vertex_neighbourhood():
    mesh = W.slice2d(4, 3)
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    adj = {v: {v} for v in range(mesh.vxy.shape[0])}
    for t in mesh.tri:
        for a in t:
            for b in t:
                adj[int(a)].add(int(b))
    # order 1: global node id = first-appearance vertex numbering; map it back through emap
    vid = {}
    for e, t in enumerate(mesh.tri):
        for n in range(3):
            vid[int(t[n])] = int(lev.emap[e, n])
    sub = SZ.subdomains(prob, 0, 1)
    for e, t in enumerate(mesh.tri):
        verts = set().union(*(adj[int(v)] for v in t))
        want = sorted(g for g in (vid[v] for v in verts) if not lev.dmask[g])
        assert list(sub[e]) == want


def test_order1_prisms_element_neighbourhood():
    mesh = W.box3d(3, 2, 3)
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    sub = SZ.subdomains(prob, 0, 1)
    for e in range(lev.emap.shape[0]):
        mine = set(lev.emap[e].tolist())
        touch = [f for f in range(lev.emap.shape[0]) if mine & set(lev.emap[f].tolist())]
        want = sorted(g for g in set(lev.emap[touch].ravel().tolist()) if not lev.dmask[g])
        assert list(sub[e]) == want


def test_zero_overlap_is_block_jacobi_over_elements():
    mesh = W.slice2d(3, 2)
    prob = Problem(mesh, [3])
    lev = prob.levels[0]
    sub = SZ.subdomains(prob, 0, 0)
    w = SZ.weights(prob, 0, sub)
    cnt = np.bincount(lev.emap.ravel(), minlength=lev.N)
    for e in range(lev.emap.shape[0]):
        assert list(sub[e]) == sorted(g for g in lev.emap[e] if not lev.dmask[g])
    assert np.allclose(w[lev.free], 1.0 / cnt[lev.free], rtol=0, atol=0)
    assert np.all(w[lev.dirichlet] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_covering_subdomains_solve_exactly(dim):
    mesh = W.slice2d(2, 1) if dim == 2 else W.box3d(1, 1, 2)
    prob = Problem(mesh, [2, 1])
    ops = S.MGOperators(prob, smoother="asm", overlap=20)
    lev = prob.levels[0]
    sz = ops.asm[0]
    assert all(np.array_equal(s, lev.free) for s in sz.subs)
    f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=4))
    u0 = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=5))
    exact = S.direct_solve(prob, f)
    for adjoint in (False, True):
        u = sz.smooth(ops.A[0], f, u0, adjoint)
        assert np.abs(u - exact).max() <= 1e-11 * np.abs(exact).max()


@pytest.mark.parametrize("dim,levels", [(2, [4, 2, 1]), (3, [3, 1])])
def test_vcycle_with_adjoint_post_smoothing_is_symmetric(dim, levels):
    mesh = W.slice2d(4, 2) if dim == 2 else W.box3d(2, 2, 2, eta_modes=W.eta_sinx_cosy(0.1))
    prob = Problem(mesh, levels)
    ops = S.MGOperators(prob, nu1=2, nu2=2, smoother="asm", overlap=1)
    lev = prob.levels[0]
    f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=1))
    g = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=2))
    a, b = g @ ops.vcycle(f), f @ ops.vcycle(g)
    assert abs(a - b) <= 1e-12 * abs(a)
    # the same cycle with S^{-1} after the correction as well is not symmetric
    asym = S.MGOperators(prob, nu1=2, nu2=2, smoother="asm", overlap=1)
    asym.smooth = lambda li, ff, x, post=False: asym.asm[li].smooth(asym.A[li], ff, x, adjoint=False)
    a2, b2 = g @ asym.vcycle(f), f @ asym.vcycle(g)
    assert abs(a2 - b2) > 1e-8 * abs(a2)


@pytest.mark.parametrize("overlap,nu,bound", [(0, 1, 25), (1, 1, 20), (1, 3, 8), (-1, 3, 8)])
def test_asm_pcg_reaches_the_direct_solution(overlap, nu, bound):
    # with larger overlaps the weighted smoother contracts in spectral radius but not in
    # the A-norm, so one sweep on each side can leave the V-cycle indefinite; the paper's
    # (3,3) sweeps do not
    mesh = W.box3d(3, 2, 2, eta_modes=W.eta_sinx_cosy(0.1))
    prob = Problem(mesh, [4, 2, 1])
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    f = S.lift(prob, phiD)
    ops = S.MGOperators(prob, nu1=nu, nu2=nu, smoother="asm", overlap=overlap)
    res = S.pcg(ops, f, rtol=1e-12)
    exact = S.direct_solve(prob, f)
    assert np.abs(res.u - exact).max() <= 1e-9 * np.abs(exact).max()
    assert res.iters <= bound
