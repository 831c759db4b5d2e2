"""The block-Jacobi preconditioned coarse CG (sem_options.coarse_bj): the coarse solve of a
single-level order-1 handle against a sparse direct solve of the oracle's free-node matrix
(coarse_rtol 1e-12, so 1e-9 relative), on a sigma-prism box and on a hull tank; the
pipelined form that loose tolerances take (coarse_rtol >= 1e-6) through the true residual
of the oracle's matrix; fewer
coarse iterations than the point-Jacobi CG at the default tolerance with the same FP64
solution of the full problem; and the block inverses follow a surface update (strategy III
reassembles the coarse matrix: the next solve equals a fresh handle's)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers as S  # noqa: E402
from oracle.assemble import Problem  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


@pytest.mark.parametrize("bj", [1, 0])
@pytest.mark.parametrize("mesh_fn", [lambda: W.config_box3d(24, 4), lambda: W.hull_tank(8)])
def test_coarse_solve_matches_sparse_direct_solve(sem, mesh_fn, bj):
    mesh = mesh_fn()
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    A = prob.free_matrix(0).tocsc()
    s = sem.Solver(mesh, 1, eta_nodal=prob.eta_nodal, levels=[1], coarse_rtol=1e-12, coarse_imax=20000, coarse_bj=bj)
    try:
        r = np.zeros(lev.N)
        r[lev.free] = W.random_vector(len(lev.free), seed=33)
        z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        s.vcycle(torch.tensor(r, device="cuda"), z)
        torch.cuda.synchronize()
        exact = np.zeros(lev.N)
        exact[lev.free] = spla.spsolve(A, r[lev.free])
        got = z.cpu().numpy()
        assert np.abs(got - exact).max() <= 1e-9 * np.abs(exact).max()
        assert np.all(got[lev.dirichlet] == 0.0)
    finally:
        s.close()


@pytest.mark.parametrize("mesh_fn", [lambda: W.config_box3d(24, 4), lambda: W.hull_tank(8)])
def test_pipelined_coarse_solve_reaches_its_tolerance(sem, mesh_fn):
    mesh = mesh_fn()
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    A = prob.free_matrix(0).tocsr()
    s = sem.Solver(mesh, 1, eta_nodal=prob.eta_nodal, levels=[1], coarse_rtol=1e-6, coarse_bj=1)
    try:
        for seed in (34, 35):
            r = np.zeros(lev.N)
            r[lev.free] = W.random_vector(len(lev.free), seed=seed)
            z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
            s.vcycle(torch.tensor(r, device="cuda"), z)
            torch.cuda.synchronize()
            got = z.cpu().numpy()
            res = np.linalg.norm(A @ got[lev.free] - r[lev.free]) / np.linalg.norm(r[lev.free])
            assert res <= 2e-6, res
    finally:
        s.close()


def test_block_jacobi_takes_fewer_coarse_iterations_same_solution(sem):
    mesh = W.config_box3d(32, 4)
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    eta = mesh.eta(xy[:, 0], xy[:, 1])
    out = {}
    for bj in (1, 0):
        s = sem.Solver(mesh, 6, eta_nodal=eta, levels=[6, 3, 1], coarse_bj=bj)
        try:
            C = s.coords(0)
            d = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
            phi = torch.zeros(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
            st = s.solve(d, phi, tol=1e-10)
            torch.cuda.synchronize()
            assert st["status"] == 0
            out[bj] = (st["coarse_iters_max"], phi.cpu().numpy())
        finally:
            s.close()
    assert out[1][0] < 0.7 * out[0][0], (out[1][0], out[0][0])
    assert np.abs(out[1][1] - out[0][1]).max() <= 1e-8 * np.abs(out[0][1]).max()


def test_block_inverses_follow_a_surface_update(sem):
    mesh = W.config_box3d(8, 3)
    levels = [4, 2, 1]
    xy = sem.sem_mesh_nodes2d(mesh, 4)
    eta1 = 0.08 * np.sin(2 * xy[:, 0]) * np.cos(xy[:, 1])
    s = sem.Solver(mesh, 4, levels=levels, coarse_rtol=1e-14)
    fresh = sem.Solver(mesh, 4, eta_nodal=eta1, levels=levels, coarse_rtol=1e-14)
    try:
        s.update_eta(eta1, "all")
        N = s.query(0)["ndof"]
        r = torch.tensor(W.random_vector(N, seed=41), device="cuda")
        za, zb = torch.zeros_like(r), torch.zeros_like(r)
        s.vcycle(r, za)
        fresh.vcycle(r, zb)
        torch.cuda.synchronize()
        assert (za - zb).abs().max().item() <= 1e-10 * zb.abs().max().item()
    finally:
        s.close()
        fresh.close()


def test_solve_with_block_jacobi_matches_direct_solution(sem):
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ref = S.solve_laplace_direct(prob, phiD)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=levels, coarse_rtol=1e-14, coarse_bj=1)
    try:
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-13)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    finally:
        s.close()
