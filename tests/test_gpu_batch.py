"""Batched lockstep solves of several uneven tanks (random element counts and
orders P in {3,...,6}) against the individual solves and the oracle."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers as S  # noqa: E402
from oracle.assemble import Problem  # noqa: E402

LEVELS = {6: [6, 3, 1], 5: [5, 3, 1], 4: [4, 2, 1], 3: [3, 2, 1]}


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


@pytest.mark.parametrize("precision,mode", [("mixed_fp32", 0), ("mixed_fp32", 1), ("fp64", 0), ("mixed_tf32", 0)])
def test_batched_tanks_match_individual_solves_and_oracle(sem, precision, mode):
    # mode 0: the whole batch as one graph launch with device-side loops; 1: host-stepped lockstep
    tanks = []
    for i in range(6):
        mesh, P, modes = W.random_tank(i, count_range=(64, 700))
        prob = Problem(mesh, LEVELS[P])
        solver = sem.Solver(mesh, P, eta_nodal=prob.eta_nodal, levels=LEVELS[P], precision=precision, batch=1,
                            outer="pdc", imax=400, batch_mode=mode)
        C = solver.coords(0)
        dn = solver.dirichlet_nodes(0)
        phiD = W.tank_potential(*C[dn].T, modes)
        tanks.append((mesh, P, prob, solver, torch.tensor(phiD, device="cuda"), phiD))
    try:
        _check_batch(sem, tanks)
    finally:
        for t in tanks:
            t[3].close()


def _check_batch(sem, tanks):
    phis = [torch.zeros(t[3].query(0)["ndof"], dtype=torch.float64, device="cuda") for t in tanks]
    stats = sem.laplace_solve_batch([t[3].h for t in tanks], [t[4] for t in tanks], 1e-10, phis)
    torch.cuda.synchronize()
    # a second batched call reuses the captured iteration graphs
    stats2 = sem.laplace_solve_batch([t[3].h for t in tanks], [t[4] for t in tanks], 1e-10, phis)
    torch.cuda.synchronize()
    for (mesh, P, prob, solver, dD, phiD), phi, st, st2 in zip(tanks, phis, stats, stats2):
        e64, e32 = solver.tile_shapes(0)
        assert e64 in (4, 8, 16, 32) and e32 in (4, 8, 16, 32)
        assert st["status"] == 0 and st["res_final"] <= 1e-10 * st["fnorm"]
        assert abs(st2["iters"] - st["iters"]) <= 1
        # every iteration of the second call runs inside a graph (the batch graph, or the
        # tank's iteration graph in lockstep mode)
        assert st2["graph_iterations"] == st2["iters"], (st["graph_iterations"], st2)
        single = torch.zeros_like(phi)
        st1 = solver.solve(dD, single, tol=1e-10)
        assert abs(st1["iters"] - st["iters"]) <= 1
        got = phi.cpu().numpy()
        assert np.abs(got - single.cpu().numpy()).max() <= 1e-8 * np.abs(got).max()
        ref = S.solve_laplace_direct(prob, phiD)
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_batch_rejects_handles_not_prepared_for_it(sem):
    mesh, P, modes = W.random_tank(0, count_range=(64, 100))
    xy = sem.sem_mesh_nodes2d(mesh, P)
    s = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), precision="mixed_fp32")
    try:
        x = torch.zeros(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
        with pytest.raises(sem.SemError) as e:
            sem.laplace_solve_batch([s.h], [x], 1e-8, [x])
        assert e.value.status == sem.SEM_EINVAL, sem.sem_last_error()
    finally:
        s.close()
    b = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), precision="mixed_fp32", outer="pdc", batch=1)
    try:
        x = torch.zeros(b.query(0)["ndof"], dtype=torch.float64, device="cuda")
        with pytest.raises(sem.SemError) as e:
            sem.laplace_solve_batch([b.h, b.h], [x, x], 1e-8, [x, x])
        assert e.value.status == sem.SEM_EINVAL and "twice" in sem.sem_last_error()
    finally:
        b.close()


def test_full_size_tanks_whose_spectrum_defeats_power_iteration(sem):
    """Two tanks of the 32-tank benchmark draw (3528 prisms at P = 6 and 6728 at
    P = 3) whose lambda_max the 20-step power iteration underestimated by 16-22 %,
    which made the Chebyshev sweep amplify the top modes: with the Lanczos estimate
    both converge, batched and alone, and lambda_hat matches the oracle's."""
    from oracle.solvers import MGOperators
    tanks = []
    try:
        for i in (1019, 1031):
            mesh, P, modes = W.random_tank(i)
            xy = sem.sem_mesh_nodes2d(mesh, P)
            s = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=LEVELS[P],
                           precision="mixed_fp32", outer="pdc", batch=1, imax=100)
            C = s.coords(0)
            dD = torch.tensor(W.tank_potential(*C[s.dirichlet_nodes(0)].T, modes), device="cuda")
            tanks.append((mesh, P, s, dD))
        phis = [torch.zeros(t[2].query(0)["ndof"], dtype=torch.float64, device="cuda") for t in tanks]
        stats = sem.laplace_solve_batch([t[2].h for t in tanks], [t[3] for t in tanks], 1e-8, phis)
        for (mesh, P, s, dD), phi, st in zip(tanks, phis, stats):
            assert st["status"] == 0 and st["iters"] <= 40 and st["res_final"] <= 1e-8 * st["fnorm"], st
            alone = torch.zeros_like(phi)
            st1 = s.solve(dD, alone, tol=1e-8)
            assert abs(st1["iters"] - st["iters"]) <= 1
        mesh, P, s, _ = tanks[1]
        ops = MGOperators(Problem(mesh, LEVELS[P][:2]))
        assert abs(s.lambdas()[0] - ops.lam[0]) <= 1e-10 * ops.lam[0]
    finally:
        for t in tanks:
            t[2].close()
