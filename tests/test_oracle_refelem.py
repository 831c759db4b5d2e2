"""Pins of the oracle's reference elements (Section 3.1) against closed forms.

Nodes, quadrature and Lagrange bases define the discrete problem; every check
here compares with mathematics fixed independently of the oracle code."""
import math
from itertools import permutations

import numpy as np
import pytest

from oracle import refelem as R


def test_gll_closed_forms():
    assert np.allclose(R.gll(2), [-1, 0, 1], atol=1e-15)
    assert np.allclose(R.gll(3), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    assert np.allclose(R.gll(4), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    a = math.sqrt(1 / 3 - 2 * math.sqrt(7) / 21)
    b = math.sqrt(1 / 3 + 2 * math.sqrt(7) / 21)
    assert np.allclose(R.gll(5), [-1, -b, -a, a, b, 1], atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8])
def test_triangle_quadrature_exact_on_dirichlet_integrals(n):
    # int_T (1+r)^a (1+s)^b dr ds = 2^(a+b+2) a! b! / (a+b+2)!  (substitute u=(1+r)/2, v=(1+s)/2)
    pts, w = R.tri_quadrature(n)
    for a in range(2 * n):
        for b in range(2 * n - a):
            exact = 2.0 ** (a + b + 2) * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = np.sum(w * (1 + pts[:, 0]) ** a * (1 + pts[:, 1]) ** b)
            assert abs(got - exact) <= 1e-13 * max(1.0, exact), (n, a, b)


@pytest.mark.parametrize("n", [1, 3, 7])
def test_gauss_legendre_and_jacobi_exactness(n):
    x, w = R.gauss_legendre(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - (0.0 if k % 2 else 2.0 / (k + 1))) < 1e-14
    x, w = R.gauss_jacobi10(n)
    for k in range(2 * n):
        # int (1-x) x^k dx over [-1, 1]
        ex = (0.0 if k % 2 else 2.0 / (k + 1)) - (2.0 / (k + 2) if k % 2 else 0.0)
        assert abs(np.sum(w * x ** k) - ex) < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_warp_blend_edges_are_gll_and_counts(p):
    nodes = R.tri_nodes(p)
    assert nodes.shape == ((p + 1) * (p + 2) // 2, 2)
    lat = R.lattice(p)
    g = R.gll(p)
    edge0 = np.array([nodes[n, 0] for n, (i, j) in enumerate(lat) if j == 0])
    assert np.allclose(np.sort(edge0), g, atol=1e-14)
    s_on_edge2 = np.array([nodes[n, 1] for n, (i, j) in enumerate(lat) if i == 0])
    assert np.allclose(np.sort(s_on_edge2), g, atol=1e-14)
    # hypotenuse r + s = 0: parameter r runs through the GLL points
    hyp = np.array([nodes[n] for n, (i, j) in enumerate(lat) if i + j == p])
    assert np.allclose(hyp.sum(axis=1), 0.0, atol=1e-14)
    assert np.allclose(np.sort(hyp[:, 0]), g, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 8))
def test_warp_blend_nodes_invariant_under_vertex_permutations(p):
    nodes = R.tri_nodes(p)
    mu = np.stack([-(nodes[:, 0] + nodes[:, 1]) / 2, (1 + nodes[:, 0]) / 2, (1 + nodes[:, 1]) / 2], axis=1)
    key = lambda m: np.array(sorted(map(tuple, np.round(m, 12))))
    ref = key(mu)
    for perm in permutations(range(3)):
        assert np.allclose(key(mu[:, perm]), ref, atol=1e-11)


def test_warp_blend_low_orders():
    assert np.allclose(R.tri_nodes(1), [[-1, -1], [1, -1], [-1, 1]])
    eq2 = [[-1, -1], [0, -1], [1, -1], [-1, 0], [0, 0], [-1, 1]]
    assert np.allclose(R.tri_nodes(2), eq2, atol=1e-15)
    n3 = R.tri_nodes(3)
    interior = [n3[k] for k, (i, j) in enumerate(R.lattice(3)) if i > 0 and j > 0 and i + j < 3]
    assert np.allclose(interior, [[-1 / 3, -1 / 3]], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 8))
def test_triangle_lagrange_cardinal_and_exact_derivatives(p):
    nodes = R.tri_nodes(p)
    B, Dr, Ds = R.tri_basis(p, nodes)
    assert np.abs(B - np.eye(nodes.shape[0])).max() < 1e-13
    rng = np.random.default_rng(p)
    pts = rng.uniform(-1, 1, (40, 2))
    pts = pts[pts.sum(axis=1) <= 0]
    B, Dr, Ds = R.tri_basis(p, pts)
    for a in range(p + 1):
        for b in range(p + 1 - a):
            f = nodes[:, 0] ** a * nodes[:, 1] ** b
            assert np.allclose(B @ f, pts[:, 0] ** a * pts[:, 1] ** b, atol=1e-12)
            fr = a * pts[:, 0] ** max(a - 1, 0) * pts[:, 1] ** b
            fs = b * pts[:, 0] ** a * pts[:, 1] ** max(b - 1, 0)
            assert np.allclose(Dr @ f, fr, atol=1e-11)
            assert np.allclose(Ds @ f, fs, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_prism_basis_exact_on_polynomials(p):
    ref = R.RefPrism(p)
    X = ref.nodes
    pts = ref.qpts
    f = (X[:, 0] ** (p // 2)) * X[:, 1] * X[:, 2] ** p + X[:, 2]
    fx = lambda r, s, t: (r ** (p // 2)) * s * t ** p + t
    B, g = ref.basis_at(pts)
    assert np.allclose(B @ f, fx(pts[:, 0], pts[:, 1], pts[:, 2]), atol=1e-12)
    dt = (pts[:, 0] ** (p // 2)) * pts[:, 1] * p * pts[:, 2] ** (p - 1) + 1
    assert np.allclose(g[2] @ f, dt, atol=1e-11)
    assert abs(ref.qw.sum() - 4.0) < 1e-13          # |T| * 2


@pytest.mark.parametrize("dim,pf,pc", [(2, 4, 2), (2, 6, 3), (3, 4, 2), (3, 6, 3), (3, 3, 1)])
def test_interpolation_matrix_reproduces_coarse_polynomials(dim, pf, pc):
    fine, coarse = R.ref_element(dim, pf), R.ref_element(dim, pc)
    I = R.interpolation_matrix(dim, pf, pc)
    assert I.shape == (fine.Np, coarse.Np)
    assert np.allclose(I.sum(axis=1), 1.0, atol=1e-13)
    c = coarse.nodes
    f = fine.nodes
    poly = lambda X: X[:, 0] ** pc + 0.5 * X[:, 1] * X[:, 0] ** max(pc - 1, 0) + (X[:, -1] ** pc if dim == 3 else 0)
    assert np.allclose(I @ poly(c), poly(f), atol=1e-12)
