"""The FP64 apply from precomputed element matrices (sem_options.elem_matrices: FP64
matrices, kind 1, and the double-FP32 upper block triangle, kind 2) against the
sum-factorised contraction and the oracle's assembled matrix, on every level of a
sigma-prism box and of a hull tank (curved base edges; orders 4 and 2 exercise the
double-FP32 layouts of 3 and 1 row blocks), with the lifting apply and after a surface
update (the matrices are recomputed with the geometry); and the FP64 and MIXED_TF32 solves
of every form against the oracle's direct solution.  Tolerance: 1e-12 of max|y| as for the
apply parity elsewhere.  The FP64 forms sum the same quadrature in FP64; the double-FP32
form represents every entry and x to 2^-48 and sums each 28-or-so-term block with exact
TwoProduct/TwoSum steps and FP32 compensation sums folded into FP64, so its error stays
within a few 1e-13 of sum_j |A_ij x_j|."""
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


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("mesh_fn,levels", [(lambda: W.config_box3d(4, 2), [6, 3, 1]),
                                            (lambda: W.hull_tank(8), [4, 2, 1])])
def test_element_matrix_apply_on_every_level(sem, mesh_fn, levels, kind):
    mesh = mesh_fn()
    prob = Problem(mesh, levels)
    on = sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, levels=levels, elem_matrices=kind)
    off = sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, levels=levels, elem_matrices=0)
    try:
        assert on.elem_matrices(0) == kind and off.elem_matrices(0) == 0
        for li in range(len(levels) - 1):
            assert on.elem_matrices(li) == kind
            lev = prob.levels[li]
            x = W.random_vector(lev.N, seed=90 + li)
            xd = torch.tensor(x, device="cuda")
            ya, yb = (torch.empty(lev.N, dtype=torch.float64, device="cuda") for _ in range(2))
            on.apply(li, xd, ya)
            off.apply(li, xd, yb)
            torch.cuda.synchronize()
            ref = prob.masked_apply(li, x)
            scale = np.abs(ref).max()
            assert np.abs(ya.cpu().numpy() - ref).max() <= 1e-12 * scale
            assert np.abs(ya.cpu().numpy() - yb.cpu().numpy()).max() <= 1e-12 * scale
    finally:
        on.close()
        off.close()


@pytest.mark.parametrize("elem", [2, 1, 0])
def test_fp64_solve_of_every_apply_form_matches_direct_solution(sem, elem):
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ref = S.solve_laplace_direct(prob, phiD)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=levels, elem_matrices=elem, coarse_rtol=1e-14)
    try:
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-13)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    finally:
        s.close()


@pytest.mark.parametrize("kind", [1, 2])
def test_element_matrices_follow_a_surface_update(sem, kind):
    # strategy III rebuilds every level's geometry: the element matrices must match the new
    # surface, i.e. the apply must equal a fresh handle's on the new eta
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    s = sem.Solver(mesh, 6, levels=levels, elem_matrices=kind)
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    eta = 0.05 * np.cos(xy[:, 0]) * np.sin(2 * xy[:, 1])
    fresh = sem.Solver(mesh, 6, eta_nodal=eta, levels=levels, elem_matrices=kind)
    try:
        s.update_eta(eta, "all")
        N = s.query(0)["ndof"]
        x = torch.tensor(W.random_vector(N, seed=97), device="cuda")
        ya, yb = torch.empty_like(x), torch.empty_like(x)
        s.apply(0, x, ya)
        fresh.apply(0, x, yb)
        torch.cuda.synchronize()
        assert (ya - yb).abs().max().item() <= 1e-12 * yb.abs().max().item()
    finally:
        s.close()
        fresh.close()


def test_mixed_tf32_residual_from_double_fp32_matrices_matches_oracle(sem):
    # the mixed path's FP64 residual through the double-FP32 element matrices (the default of a
    # mixed handle where they fit): the outer iteration still reaches the oracle's solution
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ref = S.solve_laplace_direct(prob, phiD)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=levels, precision="mixed_tf32", outer="pdc",
                   coarse_rtol=1e-14)
    try:
        assert s.elem_matrices(0) == 2 and s.elem_matrices(1) == 0
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-11)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert np.abs(phi.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    finally:
        s.close()


def test_deterministic_double_fp32_apply_is_bit_identical(sem):
    # element results summed per node in a fixed order: repeated applies and solves are equal
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=levels, elem_matrices=2, deterministic=1)
    try:
        x = torch.tensor(W.random_vector(prob.levels[0].N, seed=98), device="cuda")
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        s.apply(0, x, y1)
        s.apply(0, x, y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        ref = prob.masked_apply(0, x.cpu().numpy())
        assert np.abs(y1.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        s.close()


def test_auto_element_matrices_give_way_to_a_moving_surface(sem):
    # the auto rule serves a fixed geometry: the first surface update returns the handle to the
    # sum-factorised apply, which then equals a fresh handle's element-matrix apply
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    s = sem.Solver(mesh, 6, levels=levels)
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    eta = 0.04 * np.sin(xy[:, 0]) * np.sin(xy[:, 1])
    fresh = sem.Solver(mesh, 6, eta_nodal=eta, levels=levels)
    try:
        assert s.elem_matrices(0) == 1 and fresh.elem_matrices(0) == 1
        s.update_eta(eta, "finest")
        assert s.elem_matrices(0) == 0 and s.elem_matrices(1) == 0
        N = s.query(0)["ndof"]
        x = torch.tensor(W.random_vector(N, seed=99), device="cuda")
        ya, yb = torch.empty_like(x), torch.empty_like(x)
        s.apply(0, x, ya)
        fresh.apply(0, x, yb)
        torch.cuda.synchronize()
        assert (ya - yb).abs().max().item() <= 1e-12 * yb.abs().max().item()
    finally:
        s.close()
        fresh.close()
