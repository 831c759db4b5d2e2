"""Pins of the oracle's anisotropic prism orders and semi-coarsening (Section 6: P_xy != P_z,
the hierarchy first lowers P_xy until the orders agree, then both).

* the (p, pz) reference prism: GLL vertical nodes of order pz, Gauss-Legendre quadrature
  with pz + 1 points in t (exact to degree 2 pz + 1), node and quadrature counts;
* the discrete space holds exactly the polynomials of degree p horizontally and pz
  vertically: on a flat box with Dirichlet data on every face the solve reproduces a
  harmonic polynomial of degrees (4, 2) at (p, pz) = (4, 2) and one of degrees (4, 4) at
  (4, 4), and misses them when the order in one direction is two too low;
* nested spaces under semi-coarsening: the element prolongation reproduces coarse
  polynomials, and on affine meshes P^T A_f P equals the coarse re-discretisation;
* the semi-coarsened V-cycle (5,3) -> (3,3) -> (1,1) is symmetric, and PCG with it reaches
  the direct solution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import refelem as R
from oracle import solvers as S
from oracle.assemble import Problem


@pytest.mark.parametrize("p,pz", [(4, 2), (5, 3), (2, 4), (6, 4)])
def test_anisotropic_reference_prism(p, pz):
    ref = R.RefPrism(p, pz)
    NT = (p + 1) * (p + 2) // 2
    assert ref.NT == NT and ref.NZ == pz + 1 and ref.Np == NT * (pz + 1)
    assert ref.Nq == (p + 1) ** 2 * (pz + 1)
    assert np.allclose(ref.zn, R.gll(pz))
    # t^(2 pz + 1) integrates to 0 and t^(2 pz) to 2 / (2 pz + 1) (times |T| = 2)
    t = ref.qpts[:, 2]
    assert abs(ref.qw @ t ** (2 * pz + 1)) < 1e-13
    assert abs(ref.qw @ t ** (2 * pz) - 2.0 * 2.0 / (2 * pz + 1)) < 1e-12
    # the top face is the vertical node pz
    top = ref.face_nodes(4)
    assert np.allclose(ref.nodes[top, 2], 1.0)


def _solve_box(p, pz, u):
    mesh = W.all_boundary_dirichlet(W.box3d(2, 2, 2))
    prob = Problem(mesh, [(p, pz)])
    lev = prob.levels[0]
    C = prob.coords(0)
    x, y, z = C[:, 0] - 3.0, C[:, 1] - 3.0, C[:, 2] + 0.5
    ex = u(x, y, z)
    phi = S.solve_laplace_direct(prob, ex[lev.dirichlet])
    return np.abs(phi - ex).max() / np.abs(ex).max()


def test_space_holds_the_horizontal_and_vertical_degrees():
    # degree p + 1 is reproduced at the nodes of this structured box even when it is not in
    # the space (nodal superconvergence), so the "too low" cases miss by two degrees
    quartic_h = lambda x, y, z: x ** 4 - 6 * x * x * y * y + y ** 4 + x * x - z * z       # degrees (4, 2)
    quartic_v = lambda x, y, z: 8 * z ** 4 - 24 * z * z * (x * x + y * y) + 3 * (x * x + y * y) ** 2  # (4, 4)
    assert _solve_box(4, 2, quartic_h) < 1e-10
    assert _solve_box(2, 2, quartic_h) > 1e-4        # horizontal order too low
    assert _solve_box(4, 4, quartic_v) < 1e-10
    assert _solve_box(4, 2, quartic_v) > 1e-6        # vertical order too low (z spans only [-0.5, 0.5])


@pytest.mark.parametrize("pf,pzf,pc,pzc", [(5, 3, 3, 3), (4, 2, 2, 2), (6, 4, 4, 4), (3, 3, 1, 1)])
def test_semi_coarsened_interpolation_reproduces_coarse_polynomials(pf, pzf, pc, pzc):
    fine, coarse = R.RefPrism(pf, pzf), R.RefPrism(pc, pzc)
    I = R.interpolation_matrix(3, pf, pc, pzf, pzc)
    assert I.shape == (fine.Np, coarse.Np)
    assert np.allclose(I.sum(axis=1), 1.0, atol=1e-13)
    poly = lambda X: X[:, 0] ** pc + 0.5 * X[:, 1] * X[:, 0] ** max(pc - 1, 0) + X[:, 2] ** pzc * (1 + X[:, 1])
    assert np.allclose(I @ poly(coarse.nodes), poly(fine.nodes), atol=1e-12)
    if (pc, pzc) == (pf - 2, pzf) and pzf == pzc:
        # pure horizontal semi-coarsening: the vertical factor is the identity
        NTf, NTc = fine.NT, coarse.NT
        for k in range(pzf + 1):
            for kc in range(pzc + 1):
                blk = I[k * NTf:(k + 1) * NTf, kc * NTc:(kc + 1) * NTc]
                if k != kc:
                    assert np.abs(blk).max() < 1e-13


def test_semi_coarsened_rap_equals_rediscretisation_on_affine_meshes():
    prob = Problem(W.box3d(2, 2, 2), [(5, 3), (3, 3), (1, 1)])
    for li in range(2):
        Pm = S.prolongation(prob, li)
        lf, lc = prob.levels[li], prob.levels[li + 1]
        Af = prob.stiffness(li).toarray()
        Ac = prob.stiffness(li + 1).toarray()
        Pd = Pm.toarray()[np.ix_(lf.free, lc.free)]
        rap = Pd.T @ Af[np.ix_(lf.free, lf.free)] @ Pd
        assert np.allclose(rap, Ac[np.ix_(lc.free, lc.free)], atol=1e-12 * abs(Ac).max())


@pytest.mark.parametrize("smoother", ["chebyshev", "asm"])
def test_semi_coarsened_vcycle_symmetric_and_pcg_converges(smoother):
    mesh = W.box3d(3, 2, 2, eta_modes=W.eta_sinx_cosy(0.1))
    prob = Problem(mesh, [(5, 3), (3, 3), (1, 1)])
    kw = dict(smoother="asm", nu1=3, nu2=3) if smoother == "asm" else dict(k_cheb=5, lo=0.01, hi=1.05)
    ops = S.MGOperators(prob, **kw)
    lev = prob.levels[0]
    f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=1))
    g = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=2))
    a, b = g @ ops.vcycle(f), f @ ops.vcycle(g)
    assert abs(a - b) <= 1e-12 * abs(a)
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    rhs = S.lift(prob, phiD)
    res = S.pcg(ops, rhs, rtol=1e-12)
    exact = S.direct_solve(prob, rhs)
    assert np.abs(res.u - exact).max() <= 1e-9 * np.abs(exact).max()
    assert res.iters <= 20
