"""GPU checks at the benchmark's full size (3D box 64x64 quads x 4 sigma layers,
P = 4 and P = 6), in the launch configuration bench.py times.  The oracle cannot
assemble these meshes whole, so it computes sampled rows one by one from the
element matrices of the elements around each sampled node, and the solve is
checked through properties that hold at any size: the residual of the discrete
system at sampled rows and the distance to the exact harmonic potential."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.assemble import Problem  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


LEVELS = {4: [4, 2, 1], 6: [6, 3, 1]}


@pytest.fixture(scope="module", params=[4, 6])
def full(request, sem):
    P = request.param
    mesh = W.config_box3d(64, 4)
    prob = Problem(mesh, LEVELS[P])
    solver = sem.Solver(mesh, P, eta_nodal=prob.eta_nodal, levels=LEVELS[P])
    yield P, mesh, prob, solver
    solver.close()


def test_full_size_apply_sampled_rows(full):
    P, mesh, prob, solver = full
    lev = prob.levels[0]
    rng = np.random.default_rng(5)
    rows = np.concatenate([rng.choice(lev.free, 48, replace=False), rng.choice(lev.dirichlet, 8, replace=False),
                           [lev.free[0], lev.free[-1]]])
    x = W.random_vector(lev.N, seed=9)
    y = torch.empty(lev.N, dtype=torch.float64, device="cuda")
    solver.apply(0, torch.tensor(x, device="cuda"), y)
    got = y.cpu().numpy()[rows]
    ref = prob.apply_rows(0, x, rows)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_full_size_solve_residual_and_exact_potential(full, sem, precision):
    P, mesh, prob, solver = full
    lev = prob.levels[0]
    if precision != "fp64":
        solver = sem.Solver(mesh, P, eta_nodal=prob.eta_nodal, levels=LEVELS[P], precision=precision)
    C = solver.coords(0)
    dn = solver.dirichlet_nodes(0)
    phiD = W.potential3d(*C[dn].T)
    phi = torch.empty(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-8)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["res_final"] <= 1e-8 * st["fnorm"]
    u = phi.cpu().numpy()
    np.testing.assert_array_equal(u[dn], phiD)
    rng = np.random.default_rng(6)
    rows = rng.choice(lev.free, 40, replace=False)
    r = prob.apply_rows(0, u, rows, masked=False)       # (A phi)_i = 0 on free rows for the exact discrete phi
    assert np.abs(r).max() <= 1e-8 * st["fnorm"]
    exact = W.potential3d(*C.T)
    err = np.abs(u - exact).max()
    assert err < (2e-5 if P == 4 else 2e-7), err
    if precision != "fp64":
        solver.close()
