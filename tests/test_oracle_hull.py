"""Pins of the oracle's hull tank: curved base triangles (blended map), columns that stop
at the hull, and two vertical zones with interfaces z_k = a_k + b_k eta.

* the blended map in closed form: a curved edge's points lie on its circle at the angle
  theta_a + (1 + xi)/2 (theta_b - theta_a), the other two edges stay straight, and the
  centroid moves by 4/9 of the displacement of the edge's midpoint;
* volumes: on a flat surface the quadrature sum of |det J| over the mesh converges to the
  exact volume of the fluid (the tank minus the rounded-box hull below its draft); at
  P = 1 the straight chords miss the corner arcs' segments, at P = 6 the curved elements
  hit the volume to 1e-12; the flat lower zone holds exactly 0.7 of the tank's volume;
* numbering: the ids above the hull belong to no element and are exactly the 2D nodes
  strictly inside the footprint at the vertical levels of the upper zone; they are
  identity rows, listed with the Dirichlet nodes;
* node placement: interface nodes sit at a_k + b_k eta_P;
* the discretisation: zero row sums and symmetry of the unconstrained matrix, and with
  Dirichlet data on every boundary face the solve converges exponentially in P to a
  harmonic function.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import solvers as S
from oracle.assemble import Problem
from oracle.mesh import blended_xy, interfaces
from oracle.refelem import RefTri

L = 2 * math.pi


def _fluid_volume(depth=1.0, draft=0.3, hl=0.3, hw=0.1, corner=0.25):
    rc = corner * hw * L
    footprint = hl * L * hw * L - (4.0 - math.pi) * rc * rc
    return L * L * depth - footprint * draft * depth


def _volume(prob, li=0, elements=None):
    J = prob.jacobians(li, elements)
    w = prob.levels[li].ref.qw
    return float((w[None] * np.abs(np.linalg.det(J))).sum())


def test_blended_map_closed_form():
    m = W.hull_tank(8)
    curved = np.argwhere(m.edge_arc[:, :, 2] > 0)
    assert len(curved) == 16                 # 8 curved edges, each seen from both sides
    for (b, f) in curved[:4]:
        cx, cy, R = m.edge_arc[b, f]
        ia, ib = ((0, 1), (1, 2), (2, 0))[f]
        v = m.vxy[m.tri[b]]
        # reference points along edge f: barycentric (l_a, l_b) = ((1 - xi)/2, (1 + xi)/2)
        xi = np.linspace(-1, 1, 9)
        lam = np.zeros((9, 3))
        lam[:, ia], lam[:, ib] = (1 - xi) / 2, (1 + xi) / 2
        pts = np.stack([2 * lam[:, 1] - 1, 2 * lam[:, 2] - 1], axis=1)
        x = blended_xy(m, b, pts)
        assert np.allclose(np.hypot(x[:, 0] - cx, x[:, 1] - cy), R, atol=1e-14)
        ta = math.atan2(v[ia, 1] - cy, v[ia, 0] - cx)
        tb = math.atan2(v[ib, 1] - cy, v[ib, 0] - cx)
        dth = math.remainder(tb - ta, 2 * math.pi)
        assert 0 < abs(dth) < math.pi / 2 + 1e-12
        th = ta + (1 + xi) / 2 * dth
        assert np.allclose(x, np.stack([cx + R * np.cos(th), cy + R * np.sin(th)], 1), atol=1e-14)
        # the two other edges: the affine map
        for g, (ja, jb) in enumerate(((0, 1), (1, 2), (2, 0))):
            if g == f or m.edge_arc[b, g, 2] > 0:
                continue
            lam = np.zeros((9, 3))
            lam[:, ja], lam[:, jb] = (1 - xi) / 2, (1 + xi) / 2
            pts = np.stack([2 * lam[:, 1] - 1, 2 * lam[:, 2] - 1], axis=1)
            assert np.allclose(blended_xy(m, b, pts), lam @ v, atol=1e-14)
        if (m.edge_arc[b, :, 2] > 0).sum() == 1:
            cen = blended_xy(m, b, np.array([[-1 / 3, -1 / 3]]))[0]
            mid = np.array([cx, cy]) + R * np.array([math.cos(ta + dth / 2), math.sin(ta + dth / 2)])
            assert np.allclose(cen, v.mean(0) + 4.0 / 9.0 * (mid - 0.5 * (v[ia] + v[ib])), atol=1e-14)


def test_hull_volume_converges_to_the_fluid_volume():
    m = W.hull_tank(8)
    exact = _fluid_volume()
    errs = {}
    for P in (1, 2, 4, 6):
        prob = Problem(m, [P])
        errs[P] = abs(_volume(prob) - exact)
        cb, cl = m.columns()
        lower = np.flatnonzero(cl < 2)
        assert abs(_volume(prob, 0, lower) - 0.7 * L * L) < 1e-12
    assert errs[1] > 1e-4                    # chords cut the corner arcs' segments off
    assert errs[2] < errs[1] / 50 and errs[4] < 1e-8 and errs[6] < 1e-12


def test_hull_numbering_and_interfaces():
    m = W.hull_tank(8, eta_modes=W.eta_sinx_cosy(0.1))
    P = 3
    prob = Problem(m, [P])
    lev = prob.levels[0]
    held = np.zeros(lev.N, bool)
    held[lev.emap.ravel()] = True
    # 2D nodes strictly inside the footprint: in no full column's triangle
    full = np.flatnonzero(m.col_layers == m.nlayers)
    on_full = np.zeros(lev.N2, bool)
    on_full[lev.map2[full].ravel()] = True
    kz_low = 2 * P                                     # top of the lower zone
    expect = np.zeros(lev.N, bool)
    for kz in range(kz_low + 1, m.nlayers * P + 1):
        expect[kz * lev.N2 + np.flatnonzero(~on_full)] = True
    assert np.array_equal(~held, expect) and expect.sum() > 0
    assert lev.dmask[~held].all()
    # Dirichlet nodes that are held: the free surface of the full columns
    top = m.nlayers * P * lev.N2 + np.flatnonzero(on_full)
    assert np.array_equal(np.flatnonzero(lev.dmask & held), top)
    # node placement on the layer interfaces
    C = prob.coords(0)
    eta = prob.eta_at_level(0)
    zif = interfaces(m)
    for k in range(m.nlayers + 1):
        zk = C[k * P * lev.N2:(k * P + 1) * lev.N2, 2]
        assert np.allclose(zk, zif[k, 0] + zif[k, 1] * eta, atol=1e-14)
    # x, y of the order-P nodes are the blended map at the order-P reference nodes
    tn = RefTri(P).nodes
    for b in np.flatnonzero((m.edge_arc[:, :, 2] > 0).any(1))[:3]:
        assert np.allclose(C[lev.map2[b], :2], blended_xy(m, b, tn), atol=1e-13)


def test_hull_matrix_invariants():
    m = W.hull_tank(8, eta_modes=W.eta_powerlaw(32))
    prob = Problem(m, [4])
    A = prob.stiffness(0)
    assert abs(A - A.T).max() < 1e-13 * abs(A).max()
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-12 * abs(A).max()


def test_hull_harmonic_convergence():
    m = W.all_boundary_dirichlet(W.hull_tank(8))

    def phi(x, y, z):
        return np.exp(math.sqrt(2) * z) * np.cos(x) * np.cos(y) + 0.3 * np.exp(z) * np.sin(x)

    errs = []
    for P in (2, 4, 6):
        prob = Problem(m, [P])
        lev = prob.levels[0]
        C = prob.coords(0)
        ex = phi(*C.T)
        held = np.zeros(lev.N, bool)
        held[lev.emap.ravel()] = True
        u = S.solve_laplace_direct(prob, ex[lev.dirichlet])
        errs.append(np.abs(u - ex)[held].max())
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 50 and errs[2] < 1e-5, errs


@pytest.mark.parametrize("n", [8, 16, 64])
def test_hull_mesh_shape(n):
    m = W.hull_tank(n)
    v = m.vxy[m.tri]
    area2 = (v[:, 1, 0] - v[:, 0, 0]) * (v[:, 2, 1] - v[:, 0, 1]) - (v[:, 2, 0] - v[:, 0, 0]) * (v[:, 1, 1] - v[:, 0, 1])
    assert area2.min() > 0 and abs(area2.sum() / 2 - L * L) < 1e-10
    assert m.tri.shape[0] == 2 * n * n
    assert m.nelem == 4 * 2 * n * n - 2 * int((m.col_layers == 2).sum())
    assert int((m.edge_arc[:, :, 2] > 0).sum()) == 2 * 4 * (2 if n >= 32 else 1) * 2
    assert m.face_bc[:, 4].sum() == int((m.col_layers == 4).sum())
