"""GPU checks on the largest configuration: the 3D box of 256 x 256 quads x 6 sigma
layers at P = 6 (786,432 prisms, 87.4 M nodes, 85.0 M free), in the launch
configuration bench.py times.  The oracle builds the mesh's numbering but not its
assembled matrix, so it computes sampled rows one by one from the element matrices
around each sampled node; the solves are checked through properties that hold at
any size: the residual of the discrete system at sampled rows and the distance to
the exact harmonic potential."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.assemble import Problem  # noqa: E402

LEVELS = [6, 3, 1]


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    mesh = W.config_box3d(256, 6)
    prob = Problem(mesh, LEVELS)
    return pkg, mesh, prob


def test_256_apply_sampled_rows(big):
    sem, mesh, prob = big
    lev = prob.levels[0]
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, levels=LEVELS, autotune=0)
    try:
        assert s.query(0)["nelem"] == 786432 and s.query(0)["ndof"] == lev.N == 87407653
        rng = np.random.default_rng(15)
        rows = np.concatenate([rng.choice(lev.free, 40, replace=False), rng.choice(lev.dirichlet, 6, replace=False),
                               [lev.free[0], lev.free[-1]]])
        x = W.random_vector(lev.N, seed=19)
        y = torch.empty(lev.N, dtype=torch.float64, device="cuda")
        s.apply(0, torch.tensor(x, device="cuda"), y)
        got = y.cpu().numpy()[rows]
        ref = prob.apply_rows(0, x, rows)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["mixed_tf32", "fp64"])
def test_256_solve_residual_and_exact_potential(big, precision):
    sem, mesh, prob = big
    lev = prob.levels[0]
    opts = dict(levels=LEVELS, imax=400)
    if precision != "fp64":
        opts.update(precision=precision, outer="pdc", inner_imax=40, inner_rtol=1e-4)
    s = sem.Solver(mesh, 6, eta_nodal=prob.eta_nodal, **opts)
    try:
        C = s.coords(0)
        dn = s.dirichlet_nodes(0)
        phiD = W.potential3d(*C[dn].T)
        phi = torch.empty(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-8)
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["res_final"] <= 1e-8 * st["fnorm"]
        u = phi.cpu().numpy()
        np.testing.assert_array_equal(u[dn], phiD)
        rows = np.random.default_rng(16).choice(lev.free, 30, replace=False)
        r = prob.apply_rows(0, u, rows, masked=False)     # (A phi)_i = 0 on free rows of the exact discrete phi
        assert np.abs(r).max() <= 1e-8 * st["fnorm"]
        err = np.abs(u - W.potential3d(*C.T)).max()
        assert err < 2e-7, err
    finally:
        s.close()
