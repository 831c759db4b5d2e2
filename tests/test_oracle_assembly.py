"""Pins of the oracle's discretisation (Section 3.1, Eq. laplaceproblemdiscrete).

Each check is fixed by mathematics outside the oracle: the P=1 cotangent
stiffness, exact symbolic integration on a 2-element mesh, exact reproduction
of harmonic polynomials in V^p, the closed-form sigma-transform tensor K,
Galerkin identities between levels and spectral convergence to the Airy
potential."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import solvers as S
from oracle.assemble import Problem
from oracle.mesh import Level
from oracle.refelem import RefTri


def test_p1_triangle_is_cotangent_stiffness():
    vxy = np.array([[0.3, -0.2], [2.0, 0.1], [0.7, 1.4]])
    m = W.Mesh(dim=2, vxy=vxy, tri=np.array([[0, 1, 2]], dtype=np.int32),
               face_bc=np.zeros((1, 3), dtype=np.int8))
    Ae = Problem(m, [1]).element_matrices(0)[0]
    x, y = vxy[:, 0], vxy[:, 1]
    area = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]))
    b = np.array([y[1] - y[2], y[2] - y[0], y[0] - y[1]])
    c = np.array([x[2] - x[1], x[0] - x[2], x[1] - x[0]])
    K = (np.outer(b, b) + np.outer(c, c)) / (4 * area)
    assert np.allclose(Ae, K, atol=1e-14)


def test_two_element_p2_brute_force_exact_integration():
    sympy = pytest.importorskip("sympy")
    X, Y = sympy.symbols("x y")
    R = sympy.Rational
    verts = [(R(0), R(0)), (R(2), R(0)), (R(3, 2), R(1)), (R(0), R(5, 4))]
    tris = [(0, 1, 2), (0, 2, 3)]
    # exact P2 Lagrange basis on each physical triangle; nodes = vertices + edge midpoints
    glob = {}
    entries = {}
    for (a, b, c) in tris:
        pa, pb, pc = (sympy.Matrix(verts[v]) for v in (a, b, c))
        nodes = [pa, pb, pc, (pa + pb) / 2, (pb + pc) / 2, (pc + pa) / 2]
        mons = [1, X, Y, X * X, X * Y, Y * Y]
        V = sympy.Matrix([[sympy.sympify(mm).subs({X: n[0], Y: n[1]}) for mm in mons] for n in nodes])
        Cinv = V.inv()
        basis = [sum(Cinv[k, i] * mons[k] for k in range(6)) for i in range(6)]
        # integrate over the triangle with the affine map u, v in the unit simplex
        U, Vv = sympy.symbols("u v")
        xm = pa[0] + (pb[0] - pa[0]) * U + (pc[0] - pa[0]) * Vv
        ym = pa[1] + (pb[1] - pa[1]) * U + (pc[1] - pa[1]) * Vv
        jac = abs((pb[0] - pa[0]) * (pc[1] - pa[1]) - (pc[0] - pa[0]) * (pb[1] - pa[1]))
        keys = [tuple(n) for n in nodes]
        for i in range(6):
            for j in range(6):
                integrand = (sympy.diff(basis[i], X) * sympy.diff(basis[j], X)
                             + sympy.diff(basis[i], Y) * sympy.diff(basis[j], Y))
                integrand = sympy.expand(integrand.subs({X: xm, Y: ym}, simultaneous=True))
                val = sympy.integrate(sympy.integrate(integrand, (Vv, 0, 1 - U)), (U, 0, 1)) * jac
                k = (keys[i], keys[j])
                entries[k] = entries.get(k, 0) + val
        for kk in keys:
            glob.setdefault(kk, len(glob))
    vxy = np.array([[float(a), float(b)] for (a, b) in verts])
    m = W.Mesh(dim=2, vxy=vxy, tri=np.array(tris, dtype=np.int32), face_bc=np.zeros((2, 3), dtype=np.int8))
    prob = Problem(m, [2])
    A = prob.stiffness(0).toarray()
    coords = prob.coords(0)
    idx = {}
    for kk, g in glob.items():
        d = np.linalg.norm(coords - np.array([float(kk[0]), float(kk[1])]), axis=1)
        assert d.min() < 1e-14
        idx[kk] = int(d.argmin())
    assert len(set(idx.values())) == len(idx) == A.shape[0]
    for (ki, kj), val in entries.items():
        assert abs(A[idx[ki], idx[kj]] - float(val)) < 1e-13, (ki, kj)


def _check_sym_rowsum(prob, li):
    A = prob.stiffness(li)
    assert abs(A - A.T).max() < 1e-13 * abs(A).max()
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12 * abs(A).max()


def test_symmetry_and_zero_row_sums_2d_and_curved_3d():
    _check_sym_rowsum(Problem(W.config_slice2d(), [4, 2, 1]), 0)
    prob = Problem(W.config_box3d(4, 2), [4, 2, 1])
    for li in range(3):
        _check_sym_rowsum(prob, li)


def test_numbering_shared_nodes_have_one_position():
    for mesh, P in [(W.config_slice2d(), 5), (W.config_box3d(3, 2), 3)]:
        prob = Problem(mesh, [P])
        lev = prob.levels[0]
        X = prob.element_nodes_P()
        C = prob.coords(0)
        for e in range(lev.emap.shape[0]):
            assert np.abs(X[e] - C[lev.emap[e]]).max() < 1e-13
        # every global node is used, and distinct global nodes are at distinct places
        assert np.unique(lev.emap).size == lev.N
        key = np.round(C, 9)
        assert np.unique(key, axis=0).shape[0] == lev.N


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
def test_harmonic_polynomials_reproduced_2d(P):
    mesh = W.all_boundary_dirichlet(W.slice2d(4, 2))
    prob = Problem(mesh, [P])
    lev = prob.levels[0]
    C = prob.coords(0)
    u = lambda x, z: ((x - 3.0) + 1j * (z + 0.5)) ** P
    ex = u(C[:, 0], C[:, 1]).real
    phi = S.solve_laplace_direct(prob, ex[lev.dirichlet])
    assert np.abs(phi - ex).max() < 1e-11 * max(1.0, np.abs(ex).max())


@pytest.mark.parametrize("P", [2, 3, 4])
def test_harmonic_polynomials_reproduced_3d_flat(P):
    mesh = W.all_boundary_dirichlet(W.box3d(3, 2, 2))
    prob = Problem(mesh, [P])
    lev = prob.levels[0]
    C = prob.coords(0)
    x, y, z = C[:, 0] - 3, C[:, 1] - 3, C[:, 2] + 0.5
    ex = x * x + y * y - 2 * z * z + (x * y * z if P >= 3 else 0) + (
        (x ** 4 - 6 * x * x * z * z + z ** 4) if P >= 4 else 0)
    phi = S.solve_laplace_direct(prob, ex[lev.dirichlet])
    assert np.abs(phi - ex).max() < 1e-10 * np.abs(ex).max()


def test_sigma_transform_tensor_closed_form():
    # eta quadratic: exactly represented by the order-P interpolant (P >= 2), so
    # eta_x, eta_y at a quadrature point are known in closed form.
    P, h, nl = 3, 1.3, 2
    mesh = W.box3d(3, 2, nl, depth=h)
    c0, cx, cy, cxx = 0.05, 0.02, -0.03, 0.004
    eta_f = lambda x, y: c0 + cx * x + cy * y + cxx * x * x
    lev = Level(mesh, P)
    tn = RefTri(P).nodes
    eta_nodal = np.zeros(lev.N2)
    for b in range(mesh.tri.shape[0]):
        xy = lev.tri_node_xy(b, tn)
        eta_nodal[lev.map2[b]] = eta_f(xy[:, 0], xy[:, 1])
    prob = Problem(mesh, [P], eta_nodal=eta_nodal)
    G = prob.geometric_factors(0)
    ref = prob.levels[0].ref
    for e in [0, 3, 7]:
        b, l = divmod(e, nl)
        v = mesh.vxy[mesh.tri[b]]
        M = np.array([[(v[1, 0] - v[0, 0]) / 2, (v[2, 0] - v[0, 0]) / 2],
                      [(v[1, 1] - v[0, 1]) / 2, (v[2, 1] - v[0, 1]) / 2]])
        Axi = np.zeros((3, 3))
        Axi[:2, :2] = M
        Axi[2, 2] = 1.0 / (2 * nl)                      # d sigma / d t
        xy = lev.tri_node_xy(b, ref.qpts[:, :2])
        for q in range(0, ref.Nq, 7):
            x, y = xy[q]
            sig = (l + (ref.qpts[q, 2] + 1) / 2) / nl
            d = h + eta_f(x, y)
            ex, ey = cx + 2 * cxx * x, cy
            K = np.array([[d, 0, -sig * ex], [0, d, -sig * ey],
                          [-sig * ex, -sig * ey, (1 + (sig * ex) ** 2 + (sig * ey) ** 2) / d]])
            want = ref.qw[q] * abs(np.linalg.det(Axi)) * np.linalg.inv(Axi) @ K @ np.linalg.inv(Axi).T
            assert np.allclose(G[e, q], want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_coarse_rediscretisation_equals_galerkin_rap_on_affine_meshes(dim):
    mesh = W.slice2d(4, 2) if dim == 2 else W.box3d(2, 2, 2)
    prob = Problem(mesh, [4, 2, 1])
    for li in range(2):
        Pm = S.prolongation(prob, li)
        lf, lc = prob.levels[li], prob.levels[li + 1]
        Af = prob.stiffness(li).toarray()
        Ac = prob.stiffness(li + 1).toarray()
        Pd = Pm.toarray()[np.ix_(lf.free, lc.free)]
        rap = Pd.T @ Af[np.ix_(lf.free, lf.free)] @ Pd
        assert np.allclose(rap, Ac[np.ix_(lc.free, lc.free)], atol=1e-12 * abs(Ac).max())


def test_prolongation_reproduces_coarse_functions_on_curved_mesh():
    prob = Problem(W.config_box3d(3, 2), [4, 2, 1])
    for li in range(2):
        lf, lc = prob.levels[li], prob.levels[li + 1]
        Cf, Cc = prob.coords(li), prob.coords(li + 1)
        Pm = S.prolongation(prob, li)
        # a coarse function that vanishes on the Dirichlet top: the mapped reference
        # coordinate structure is preserved, so use sigma-layer index functions
        uc = np.where(lc.dmask, 0.0, np.cos(Cc[:, 0]) * (1 + Cc[:, 2]))
        uf = Pm @ uc
        # check against element-wise interpolation done independently per element
        from oracle.refelem import interpolation_matrix
        I = interpolation_matrix(3, lf.p, lc.p)
        for e in range(lf.emap.shape[0]):
            vals = I @ uc[lc.emap[e]]
            free = ~lf.dmask[lf.emap[e]]
            assert np.allclose(uf[lf.emap[e]][free], vals[free], atol=1e-13)


def test_airy_spectral_convergence_in_p():
    errs = []
    for P in range(1, 8):
        prob = Problem(W.slice2d(4, 2), [P])
        lev = prob.levels[0]
        C = prob.coords(0)
        ex = W.airy2d(C[:, 0], C[:, 1])
        phi = S.solve_laplace_direct(prob, ex[lev.dirichlet])
        errs.append(np.abs(phi - ex).max())
    errs = np.array(errs)
    assert errs[-1] < 1e-7
    rates = errs[2:] / errs[1:-1]
    assert np.all(rates < 0.35), errs


@pytest.mark.parametrize("mesh_fn,levels", [(lambda: W.slice2d(4, 2), [4, 2, 1]),
                                            (lambda: W.config_box3d(3, 2), [3, 1]),
                                            (lambda: W.hull_tank(8), [2, 1])])
def test_apply_rows_equal_the_assembled_product(mesh_fn, levels):
    # the row-by-row apply (used for sampled rows at full size) against the assembled
    # sparse product, masked (y_F = A_FF x_F, y_D = x_D) and plain (y = A x), on rows that
    # include Dirichlet nodes, nodes shared by many elements and the last node
    prob = Problem(mesh_fn(), levels)
    for li in range(len(levels)):
        lev = prob.levels[li]
        x = W.random_vector(lev.N, seed=40 + li)
        rng = np.random.default_rng(li)
        rows = np.unique(np.concatenate([rng.choice(lev.N, size=min(25, lev.N), replace=False),
                                         lev.dirichlet[:3], lev.emap[0], [lev.N - 1]]))
        full_m = prob.masked_apply(li, x)
        full_p = prob.stiffness(li) @ x
        got_m = prob.apply_rows(li, x, rows, masked=True)
        got_p = prob.apply_rows(li, x, rows, masked=False)
        scale = np.abs(full_p).max()
        assert np.abs(got_m - full_m[rows]).max() <= 1e-12 * scale
        assert np.abs(got_p - full_p[rows]).max() <= 1e-12 * scale
        assert lev.dmask[rows].any() and (~lev.dmask[rows]).any()
