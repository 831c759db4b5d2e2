"""Atomic-free direct-stiffness summation (sem_options.deterministic = 1).

The FP64 applies and restrictions write element results that every node then sums
over its precomputed segment of the node -> element-slot map, in a fixed order.
Checks: the operator on every level against the oracle's assembled matrix (1e-12)
and against the atomic form; bit-identical repeated applies and repeated solves
(on the test box and at the benchmark's full size); the solve against the
oracle's direct solution at rtol 1e-13 (1e-10)."""
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


@pytest.mark.parametrize("mesh_fn,levels", [(lambda: W.config_box3d(4, 2), [6, 3, 1]),
                                            (lambda: W.hull_tank(8), [4, 2, 1])])
def test_deterministic_apply_matches_oracle_and_atomic_form(sem, mesh_fn, levels):
    mesh = mesh_fn()
    prob = Problem(mesh, levels)
    det = sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, levels=levels, deterministic=1)
    ato = sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, levels=levels)
    try:
        for li in range(len(levels)):
            lev = prob.levels[li]
            x = W.random_vector(lev.N, seed=70 + li)
            xd = torch.tensor(x, device="cuda")
            y1, y2, ya = (torch.empty(lev.N, dtype=torch.float64, device="cuda") for _ in range(3))
            det.apply(li, xd, y1)
            det.apply(li, xd, y2)
            ato.apply(li, xd, ya)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2)
            ref = prob.masked_apply(li, x)
            got = y1.cpu().numpy()
            scale = np.abs(ref).max()
            assert np.abs(got - ref).max() <= 1e-12 * scale
            assert np.abs(got - ya.cpu().numpy()).max() <= 1e-13 * scale
            # the assembled diagonal (all nodes) is summed the same way at setup
            dref = prob.stiffness(li).diagonal()
            assert np.abs(det.diagonal(li) - dref).max() <= 1e-12 * np.abs(dref).max()
    finally:
        det.close()
        ato.close()


def test_deterministic_solves_are_bit_identical_and_match_direct_solution(sem):
    mesh = W.config_box3d(4, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ref = S.solve_laplace_direct(prob, phiD)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=levels, deterministic=1, coarse_rtol=1e-14)
    try:
        d = torch.tensor(phiD, device="cuda")
        outs = []
        for _ in range(2):
            phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
            st = s.solve(d, phi, tol=1e-13)
            torch.cuda.synchronize()
            assert st["status"] == 0
            outs.append(phi)
        assert torch.equal(outs[0], outs[1])
        assert np.abs(outs[0].cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    finally:
        s.close()


def test_deterministic_full_size_solves_are_bit_identical(sem):
    # the benchmark's workload (64 x 64 x 4 prisms, P = 6, FP64 PCG to 1e-8), two handles
    mesh = W.config_box3d(64, 4)
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    eta = mesh.eta(xy[:, 0], xy[:, 1])
    res = []
    for _ in range(2):
        s = sem.Solver(mesh, 6, eta_nodal=eta, levels=[6, 3, 1], deterministic=1)
        try:
            C = s.coords(0)
            d = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
            phi = torch.empty(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
            st = s.solve(d, phi, tol=1e-8)
            torch.cuda.synchronize()
            assert st["status"] == 0 and st["res_final"] <= 1e-8 * st["fnorm"]
            res.append(phi)
        finally:
            s.close()
    assert torch.equal(res[0], res[1])
