"""The one-launch solve of small problems (sem_options.fused_small): lifting, FGMRES or PCG
and the V-cycle with a direct coarse solve in one CTA.  Checks: the config-1 slice (128
triangles, P = 4, FGMRES(30), pMG 4-2-1) against the oracle's direct solution (1e-10 at
rtol 1e-13) and the oracle's own FGMRES with the same V-cycle (iteration count), against the
multi-kernel path; PCG on a small sigma-prism box, with a source term; a surface update (the
plan's element matrices follow the geometry); a non-finite Dirichlet value ends in SEM_NAN.
One kernel launch per solve (the solve statistics report it)."""
import numpy as np
import pytest

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


def _slice(sem, **opts):
    mesh = W.config_slice2d()
    prob = Problem(mesh, [4, 2, 1])
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.airy2d(*C[lev.dirichlet].T)
    s = sem.Solver(mesh, 4, levels=[4, 2, 1], outer="fgmres", gmres_m=30, imax=100, **opts)
    return mesh, prob, lev, phiD, s


def test_slice_fgmres_matches_direct_solution_in_one_launch(sem):
    mesh, prob, lev, phiD, s = _slice(sem)
    try:
        ref = S.solve_laplace_direct(prob, phiD)
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-13)
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["kernel_launches"] == 1
        got = phi.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
        np.testing.assert_array_equal(got[lev.dirichlet], phiD)
        # the oracle's FGMRES(30) with the same V-cycle (Chebyshev k = 5 on [0.01 b, b], b = 1.05
        # lambda_hat, exact coarse solve) takes the same number of iterations
        ops = S.MGOperators(prob, k_cheb=5, lo=0.01, hi=1.05)
        res = S.fgmres(ops, S.lift(prob, phiD), rtol=1e-13, m=30)
        assert abs(st["iters"] - res.iters) <= 1, (st["iters"], res.iters)
    finally:
        s.close()


def test_slice_fused_equals_multi_kernel_path(sem):
    _, prob, lev, phiD, s1 = _slice(sem)
    _, _, _, _, s0 = _slice(sem, fused_small=0, coarse_rtol=1e-14)
    try:
        d = torch.tensor(phiD, device="cuda")
        a = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        b = torch.zeros_like(a)
        sa = s1.solve(d, a, tol=1e-12)
        sb = s0.solve(d, b, tol=1e-12)
        torch.cuda.synchronize()
        assert sa["kernel_launches"] == 1 and sb["kernel_launches"] > 100
        assert abs(sa["iters"] - sb["iters"]) <= 1
        assert (a - b).abs().max().item() <= 1e-9 * b.abs().max().item()
    finally:
        s1.close()
        s0.close()


def test_small_box_pcg_with_source_matches_direct_solution(sem):
    mesh = W.config_box3d(2, 2)
    levels = [3, 2, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    rhs = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=61))
    ref = S.solve_laplace_direct(prob, phiD, rhs=rhs)
    s = sem.Solver(mesh, 3, eta_nodal=prob.eta_nodal, levels=levels, outer="pcg")
    try:
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-13, rhs=torch.tensor(rhs, device="cuda"))
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["kernel_launches"] == 1
        assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    finally:
        s.close()


def test_small_box_after_surface_update_equals_fresh_handle(sem):
    mesh = W.config_box3d(2, 2)
    levels = [3, 2, 1]
    xy = sem.sem_mesh_nodes2d(mesh, 3)
    eta1 = 0.07 * np.sin(xy[:, 0] + 0.3) * np.cos(2 * xy[:, 1])
    s = sem.Solver(mesh, 3, levels=levels, outer="fgmres")
    fresh = sem.Solver(mesh, 3, eta_nodal=eta1, levels=levels, outer="fgmres")
    try:
        s.update_eta(eta1, "all")
        C = fresh.coords(0)
        d = torch.tensor(W.potential3d(*C[fresh.dirichlet_nodes(0)].T), device="cuda")
        a = torch.zeros(fresh.query(0)["ndof"], dtype=torch.float64, device="cuda")
        b = torch.zeros_like(a)
        sa = s.solve(d, a, tol=1e-12)
        sb = fresh.solve(d, b, tol=1e-12)
        torch.cuda.synchronize()
        assert sa["kernel_launches"] == 1 and sb["kernel_launches"] == 1
        assert (a - b).abs().max().item() <= 1e-10 * b.abs().max().item()
    finally:
        s.close()
        fresh.close()


def test_non_finite_dirichlet_value_ends_in_sem_nan(sem):
    _, prob, lev, phiD, s = _slice(sem)
    try:
        bad = phiD.copy()
        bad[3] = np.nan
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        with pytest.raises(sem.SemError) as e:
            s.solve(torch.tensor(bad, device="cuda"), phi, tol=1e-10)
        assert e.value.status == sem.SEM_NAN
    finally:
        s.close()
