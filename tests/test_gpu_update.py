"""sem_update_eta: a new surface elevation with the paper's operator-reuse strategies
(Section 5, strategies I-III).

ALL must leave the handle equal to one set up from scratch with the new elevation
(apply on every level and the diagonals to 1e-12, lambda_hat to 1e-10, the solve to the
oracle's direct solution to 1e-10 at rtol 1e-13).  FINEST changes the finest
operator (and re-estimates its lambda_hat) while the diagonals and coarse levels keep the
old elevation's operators; the solve still reaches the new problem's solution.
LINEAR_COARSE puts the flat-surface operators on the coarse levels (compared with the
oracle on a flat mesh)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers as S  # noqa: E402
from oracle.assemble import Problem  # noqa: E402

LEVELS = [5, 3, 1]
MODES0 = W.eta_sinx_cosy(0.08)
MODES1 = [(0.06, 2.0, 1.0, 0.3), (0.04, 1.0, 3.0, 1.1)]


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    pkg.lib()
    return pkg


def _mesh(modes):
    return W.box3d(5, 4, 3, eta_modes=modes)


def _solver(sem, modes, **o):
    mesh = _mesh(modes)
    xy = sem.sem_mesh_nodes2d(mesh, LEVELS[0])
    return mesh, xy, sem.Solver(mesh, LEVELS[0], eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=LEVELS,
                                coarse_rtol=1e-14, **o)


def _apply(s, level, x):
    y = torch.zeros_like(x)
    s.apply(level, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _solve_vs_oracle(s, mesh1, tol, bound):
    prob = Problem(mesh1, LEVELS)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ref = S.solve_laplace_direct(prob, phiD)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=tol)
    torch.cuda.synchronize()
    assert st["status"] == 0
    assert _rel(phi.cpu().numpy(), ref) <= bound
    return st


def test_update_all_equals_a_fresh_setup(sem):
    mesh1, xy, fresh = _solver(sem, MODES1)
    _, _, s = _solver(sem, MODES0)
    try:
        s.update_eta(mesh1.eta(xy[:, 0], xy[:, 1]), "all")
        for li in range(len(LEVELS)):
            x = torch.tensor(W.random_vector(s.query(li)["ndof"], seed=li), device="cuda")
            assert _rel(_apply(s, li, x), _apply(fresh, li, x)) <= 1e-12
            assert _rel(s.diagonal(li), fresh.diagonal(li)) <= 1e-12
        lam, lam_f = s.lambdas(), fresh.lambdas()
        assert np.all(np.abs(lam - lam_f) <= 1e-10 * np.abs(lam_f).max())
        _solve_vs_oracle(s, mesh1, 1e-13, 1e-10)
    finally:
        s.close()
        fresh.close()


def test_update_finest_keeps_the_t0_preconditioner(sem):
    mesh1, xy, fresh = _solver(sem, MODES1)
    _, _, old = _solver(sem, MODES0)
    _, _, s = _solver(sem, MODES0)
    try:
        lam0, diag0 = s.lambdas(), s.diagonal(0)
        s.update_eta(mesh1.eta(xy[:, 0], xy[:, 1]), "finest")
        lam1 = s.lambdas()
        x0 = torch.tensor(W.random_vector(s.query(0)["ndof"], seed=3), device="cuda")
        assert _rel(_apply(s, 0, x0), _apply(fresh, 0, x0)) <= 1e-12
        x1 = torch.tensor(W.random_vector(s.query(1)["ndof"], seed=4), device="cuda")
        assert _rel(_apply(s, 1, x1), _apply(old, 1, x1)) <= 1e-12
        # the diagonal of t = 0 stays; lambda_hat of the finest level follows the operator
        assert np.array_equal(s.diagonal(0), diag0)
        assert np.array_equal(lam1[1:], lam0[1:])
        _solve_vs_oracle(s, mesh1, 1e-11, 1e-8)
    finally:
        s.close()
        old.close()
        fresh.close()


def test_update_linear_coarse_uses_flat_coarse_operators(sem):
    mesh1, xy, fresh = _solver(sem, MODES1)
    _, _, s = _solver(sem, MODES0)
    flat = Problem(_mesh([]), LEVELS)
    try:
        s.update_eta(mesh1.eta(xy[:, 0], xy[:, 1]), "linear_coarse")
        x0 = torch.tensor(W.random_vector(s.query(0)["ndof"], seed=5), device="cuda")
        assert _rel(_apply(s, 0, x0), _apply(fresh, 0, x0)) <= 1e-12
        assert abs(s.lambdas()[0] - fresh.lambdas()[0]) <= 1e-10 * fresh.lambdas()[0]
        for li in (1, 2):
            x = W.random_vector(s.query(li)["ndof"], seed=6 + li)
            got = _apply(s, li, torch.tensor(x, device="cuda"))
            assert _rel(got, flat.masked_apply(li, x)) <= 1e-12
        _solve_vs_oracle(s, mesh1, 1e-11, 1e-8)
        # a second update keeps the flat coarse levels and refreshes the finest one
        s.update_eta(_mesh(MODES0).eta(xy[:, 0], xy[:, 1]), "linear_coarse")
        _solve_vs_oracle(s, _mesh(MODES0), 1e-11, 1e-8)
    finally:
        s.close()
        fresh.close()


def test_update_rejects_2d_handles_and_unknown_strategies(sem):
    s2 = sem.Solver(W.config_slice2d(), 4, levels=[4, 2, 1])
    _, xy, s3 = _solver(sem, MODES0)
    try:
        with pytest.raises(sem.SemError) as e:
            s2.update_eta(np.zeros(10), "all")
        assert e.value.status == sem.SEM_EINVAL
        with pytest.raises(sem.SemError) as e:
            s3.update_eta(np.zeros(len(xy)), 3)
        assert e.value.status == sem.SEM_EINVAL
    finally:
        s2.close()
        s3.close()


def test_mixed_handles_reestimate_with_the_single_precision_operator(sem):
    # the FP32 operator differs from the FP64 one by rounding (~1e-7 of its size), so the
    # largest Ritz value of the same 30 Lanczos steps moves by about that much
    mesh1, xy, fresh = _solver(sem, MODES1)
    _, _, s = _solver(sem, MODES0, precision="mixed_fp32")
    try:
        s.update_eta(mesh1.eta(xy[:, 0], xy[:, 1]), "all")
        lam, lam_f = s.lambdas(), fresh.lambdas()
        assert np.all(np.abs(lam - lam_f) <= 1e-4 * np.abs(lam_f))
        _solve_vs_oracle(s, mesh1, 1e-11, 1e-8)
    finally:
        s.close()
        fresh.close()
