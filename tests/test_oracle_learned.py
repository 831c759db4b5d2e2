"""Pins of the oracle's learned correction sweep (oracle/learned.py).

* An identity network (y = relu(x) - relu(-x)) returns each element's scaled
  input, so the sweep must reduce to the minimal-residual Jacobi step
  delta = D^{-1} r, alpha = (r, A D^{-1} r) / ||A D^{-1} r||^2: this fixes the
  gather, the per-element scale s_e, the weights W and the scatter at once.
* For any network the sweep is positively homogeneous of degree one in (f, u):
  the network only ever sees unit-norm inputs and its output is scaled back.
* alpha minimises ||r - alpha A delta||, and the reported residual after the
  step is the residual of the new iterate.
* A network that returns zero, or tau = 0, is rejected and the Chebyshev sweep
  runs instead."""
import numpy as np
import pytest

import workloads as W
from oracle import learned as Lr
from oracle import solvers as S
from oracle.assemble import Problem


def _ops(mesh_fn=lambda: W.config_box3d(3, 2), levels=(3, 2, 1)):
    prob = Problem(mesh_fn(), list(levels))
    return prob, S.MGOperators(prob, k_cheb=3, lo=0.1, hi=1.05)


def _vec(prob, seed):
    lev = prob.levels[0]
    return np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=seed))


def _identity_net(npe):
    I = np.eye(npe)
    return (np.vstack([I, -I]), np.zeros(2 * npe), np.hstack([I, -I]), np.zeros(npe))


def _random_net(npe, H=24, seed=3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((H, npe)) * 0.3, rng.standard_normal(H) * 0.1,
            rng.standard_normal((npe, H)) * 0.3, rng.standard_normal(npe) * 0.1)


@pytest.mark.parametrize("mesh_fn,levels", [(lambda: W.config_box3d(3, 2), (3, 2, 1)),
                                            (lambda: W.hull_tank(8), (2, 1))])
def test_identity_network_gives_the_minimal_residual_jacobi_step(mesh_fn, levels):
    prob, ops = _ops(mesh_fn, levels)
    lev = prob.levels[0]
    f, u = _vec(prob, 1), 0.3 * _vec(prob, 2)
    res = Lr.learned_sweep(ops, _identity_net(lev.ref.Np), f, u, tau=1.0)
    r = f - ops.A[0] @ u
    d = ops.Dinv[0] * r
    q = ops.A[0] @ d
    alpha = (r @ q) / (q @ q)
    assert np.abs(res.delta - d).max() <= 1e-12 * np.abs(d).max()
    assert res.accepted and abs(res.alpha - alpha) <= 1e-12 * alpha
    assert np.abs(res.u - (u + alpha * d)).max() <= 1e-12 * np.abs(u + alpha * d).max()


def test_sweep_is_positively_homogeneous_for_any_network():
    prob, ops = _ops()
    npe = prob.levels[0].ref.Np
    net = _random_net(npe)
    f, u = _vec(prob, 3), 0.5 * _vec(prob, 4)
    for tau in (1.0, 0.0):                       # accepted and rejected branches
        a = Lr.learned_sweep(ops, net, f, u, tau)
        b = Lr.learned_sweep(ops, net, 3.7 * f, 3.7 * u, tau)
        assert a.accepted == b.accepted
        assert np.abs(b.delta - 3.7 * a.delta).max() <= 1e-12 * np.abs(b.delta).max()
        assert np.abs(b.u - 3.7 * a.u).max() <= 1e-12 * np.abs(b.u).max()
    assert np.abs(a.delta).max() > 0


def test_alpha_minimises_the_residual_and_the_reported_residual_is_the_new_one():
    prob, ops = _ops()
    net = _random_net(prob.levels[0].ref.Np, seed=9)
    f, u = _vec(prob, 5), 0.2 * _vec(prob, 6)
    res = Lr.learned_sweep(ops, net, f, u, tau=1.0)
    r = f - ops.A[0] @ u
    q = ops.A[0] @ res.delta
    a = (r @ q) / (q @ q)
    for beta in (0.9 * a, 1.1 * a, -a, 0.0):
        assert np.linalg.norm(r - a * q) <= np.linalg.norm(r - beta * q) + 1e-14
    rn = f - ops.A[0] @ (u + a * res.delta)
    assert abs(res.rr_after - rn @ rn) <= 1e-10 * (r @ r)
    assert abs(res.rr - r @ r) <= 1e-12 * (r @ r)


def test_rejected_sweeps_fall_back_to_the_chebyshev_sweep():
    prob, ops = _ops()
    npe = prob.levels[0].ref.Np
    f, u = _vec(prob, 7), 0.1 * _vec(prob, 8)
    b = ops.hi * ops.lam[0]
    cheb = S.chebyshev(lambda v: ops.A[0] @ v, ops.Dinv[0], f, u, ops.k, ops.lo * b, b)
    zero = (np.zeros((4, npe)), np.zeros(4), np.zeros((npe, 4)), np.zeros(npe))
    for net, tau in ((zero, 1.0), (_identity_net(npe), 0.0)):
        res = Lr.learned_sweep(ops, net, f, u, tau)
        assert not res.accepted and res.alpha == 0.0
        assert np.array_equal(res.u, cheb)


def test_element_weights_are_a_partition_of_unity():
    prob, _ = _ops()
    lev = prob.levels[0]
    w = Lr.element_weights(lev.emap, lev.N)
    tot = np.zeros(lev.N)
    np.add.at(tot, lev.emap.ravel(), w[lev.emap].ravel())
    assert np.allclose(tot, 1.0)
