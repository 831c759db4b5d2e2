"""Pins of the oracle's solvers: Chebyshev smoothing against its closed-form error
polynomial, the Lanczos eigenvalue estimate against a closed form and eigen-solvers, the V-cycle
(Algorithm 1) against dense two-level algebra and its symmetry, and the outer
iterations (Algorithms 2, 3 and FGMRES) against the direct solve."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import chebyshev as C

import workloads as W
from oracle import solvers as S
from oracle.assemble import Problem


def _cheb_poly(lam, k, a, b):
    theta, delta = (a + b) / 2, (b - a) / 2
    Tk = np.zeros(k + 1)
    Tk[k] = 1.0
    return C.chebval((theta - lam) / delta, Tk) / C.chebval(theta / delta, Tk)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_chebyshev_error_is_scaled_chebyshev_polynomial(k):
    rng = np.random.default_rng(k)
    lam = np.linspace(0.05, 2.0, 40)
    d = rng.uniform(0.5, 2.0, 40)            # A = diag(d * lam), D = diag(d)
    A = d * lam
    xs = rng.standard_normal(40)
    f = A * xs
    x0 = rng.standard_normal(40)
    a, b = 0.3, 2.1
    x = S.chebyshev(lambda v: A * v, 1.0 / d, f, x0, k, a, b)
    assert np.allclose(x - xs, _cheb_poly(lam, k, a, b) * (x0 - xs), atol=1e-12)


def test_lanczos_estimate_matches_closed_form_of_1d_laplacian():
    # A = tridiag(-1, 2, -1) of n interior nodes: D^{-1} A = A / 2 has eigenvalues
    # 1 - cos(j pi / (n + 1)), so lambda_max = 1 + cos(pi / (n + 1)).
    for n in (7, 40):
        A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
        dinv = np.full(n, 0.5)
        lam = S.lanczos_lambda(A, dinv, np.zeros(n, dtype=bool), steps=n)
        assert abs(lam - (1 + np.cos(np.pi / (n + 1)))) < 1e-12


def test_lanczos_estimate_is_a_converging_lower_bound():
    prob = Problem(W.slice2d(4, 2), [3, 1])
    ops = S.MGOperators(prob)
    lev = prob.levels[0]
    A = ops.A[0].toarray()[np.ix_(lev.free, lev.free)]
    dd = 1.0 / ops.Dinv[0][lev.free]
    Ds = np.diag(1 / np.sqrt(dd))
    lmax = np.linalg.eigvalsh(Ds @ A @ Ds).max()
    # Ritz values interlace: the largest grows with the step count towards lambda_max
    est = [S.lanczos_lambda(ops.A[0], ops.Dinv[0], lev.dmask, k) for k in (3, 6, 12, 24)]
    assert all(b >= a - 1e-12 for a, b in zip(est, est[1:]))
    assert est[-1] <= lmax * (1 + 1e-12) and est[-1] >= 0.99 * lmax
    assert ops.lam[0] <= lmax * (1 + 1e-12) and ops.lam[0] >= 0.99 * lmax
    full = S.lanczos_lambda(ops.A[0], ops.Dinv[0], lev.dmask, len(lev.free))
    assert abs(full - lmax) < 1e-9 * lmax


@pytest.mark.parametrize("n,P", [(6, 6), (10, 3)])
def test_lanczos_estimate_on_sigma_prism_tanks(n, P):
    # wavy-surface prism tanks: 30 steps come within 2 % of lambda_max (ARPACK)
    mesh = W.box3d(n, n, 4, eta_modes=W.random_tank(1019)[0].eta_modes)
    prob = Problem(mesh, [P, 1])
    ops = S.MGOperators(prob)
    lev = prob.levels[0]
    A = prob.free_matrix(0)
    d = A.diagonal()
    B = sp.diags(1 / np.sqrt(d)) @ A @ sp.diags(1 / np.sqrt(d))
    lmax = spla.eigsh(B, k=1, which="LA", tol=1e-10, return_eigenvectors=False)[0]
    assert 0.98 * lmax <= ops.lam[0] <= lmax * (1 + 1e-10)


def test_two_level_vcycle_equals_dense_algebra():
    prob = Problem(W.slice2d(2, 1), [3, 1])            # 4 triangles
    ops = S.MGOperators(prob, nu1=1, nu2=1, k_cheb=3, lo=0.2, hi=1.1)
    lf, lc = prob.levels
    F = lf.free
    A = ops.A[0].toarray()[np.ix_(F, F)]
    Dinv = ops.Dinv[0][F]
    Pm = ops.P[0].toarray()[np.ix_(F, lc.free)]
    Ac = Pm.T @ A @ Pm          # affine + exact quadrature: equals the re-discretised coarse matrix
    b = ops.hi * ops.lam[0]
    a = ops.lo * b
    # smoother error propagator p_k(D^{-1} A) through the symmetric similarity transform
    Dh = np.diag(np.sqrt(Dinv))
    w, Q = np.linalg.eigh(Dh @ A @ Dh)
    # D^{-1} A = Dh (Dh A Dh) Dh^{-1} with Dh = D^{-1/2}
    Smat = Dh @ Q @ np.diag(_cheb_poly(w, 3, a, b)) @ Q.T @ np.diag(1 / np.sqrt(Dinv))
    Ecg = np.eye(len(F)) - Pm @ np.linalg.solve(Ac, Pm.T @ A)
    E = Smat @ Ecg @ Smat
    Minv = (np.eye(len(F)) - E) @ np.linalg.inv(A)
    rng = np.random.default_rng(0)
    for _ in range(3):
        f = np.zeros(lf.N)
        f[F] = rng.standard_normal(len(F))
        z = ops.vcycle(f)
        assert np.allclose(z[F], Minv @ f[F], atol=1e-12 * np.abs(z).max())
        assert np.all(z[lf.dirichlet] == 0)


@pytest.mark.parametrize("mesh_fn,levels", [(lambda: W.config_slice2d(), [4, 2, 1]),
                                             (lambda: W.config_box3d(4, 2), [4, 2, 1]),
                                             (lambda: W.config_box3d(3, 2), [6, 3, 1])])
def test_vcycle_is_symmetric_and_positive(mesh_fn, levels):
    prob = Problem(mesh_fn(), levels)
    ops = S.MGOperators(prob)
    lev = prob.levels[0]
    rng = np.random.default_rng(1)
    x = np.where(lev.dmask, 0.0, rng.standard_normal(lev.N))
    y = np.where(lev.dmask, 0.0, rng.standard_normal(lev.N))
    Mx, My = ops.vcycle(x), ops.vcycle(y)
    assert abs(Mx @ y - x @ My) < 1e-11 * np.linalg.norm(Mx) * np.linalg.norm(y)
    assert Mx @ x > 0


@pytest.mark.parametrize("outer", ["pcg", "pdc", "fgmres"])
def test_outer_iterations_reach_the_direct_solution(outer):
    prob = Problem(W.config_box3d(4, 2), [4, 2, 1])
    lev = prob.levels[0]
    X = prob.coords(0)
    phiD = W.potential3d(*X[lev.dirichlet].T)
    f = S.lift(prob, phiD)
    exact = S.direct_solve(prob, f)
    ops = S.MGOperators(prob, lo=0.1)
    res = getattr(S, outer)(ops, f, rtol=1e-12)
    assert res.resids[-1] <= 1e-12 * res.fnorm
    assert np.abs(res.u - exact).max() < 1e-10 * np.abs(exact).max()
    assert res.iters < 60


def test_pcg_residual_drop_per_iteration_is_multigrid_like():
    # qualitative check in the spirit of the paper's tables (about an order of
    # magnitude per iteration): mean contraction below 0.25 on the 2D slice.
    prob = Problem(W.config_slice2d(), [4, 2, 1])
    lev = prob.levels[0]
    X = prob.coords(0)
    f = S.lift(prob, W.airy2d(*X[lev.dirichlet].T))
    res = S.pcg(S.MGOperators(prob, lo=0.1), f, rtol=1e-10)
    q = (res.resids[-1] / res.resids[0]) ** (1.0 / res.iters)
    assert q < 0.25
