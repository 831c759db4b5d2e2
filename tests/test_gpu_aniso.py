"""Anisotropic prism orders and semi-coarsening on the GPU (Section 6: P_xy != P_z, the
hierarchy lowers P_xy until the orders agree, then both) against the oracle.

Bars: numbering, Dirichlet sets exact; coordinates 1e-13; assembled diagonal and the
FP64 apply 1e-12 relative on every level; the FP32 apply 1e-5; the V-cycle 1e-10 (coarse CG
to 1e-14); PCG solves 1e-10 against the direct solution at rtol 1e-13, the mixed precisions
1e-8 at rtol 1e-11; the Schwarz subdomains exact; the free-surface right-hand sides 1e-9.
Unsupported order pairs and growing orders are refused.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fnpf as F  # noqa: E402
from oracle import schwarz as SZ  # noqa: E402
from oracle import solvers as S  # noqa: E402
from oracle.assemble import Problem  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    pkg.lib()
    return pkg


HIER = {
    "53": [(5, 3), (3, 3), (1, 1)],
    "42": [(4, 2), (2, 2), (1, 1)],
    "64": [(6, 4), (4, 4), (2, 2), (1, 1)],
    "65": [(6, 5), (3, 3), (1, 1)],
}


def _mesh():
    return W.box3d(3, 3, 2, eta_modes=W.eta_sinx_cosy(0.1))


def _make(sem, key, **o):
    mesh = _mesh()
    levels = HIER[key]
    P = levels[0][0]
    xy = sem.sem_mesh_nodes2d(mesh, P)
    eta = mesh.eta(xy[:, 0], xy[:, 1])
    s = sem.Solver(mesh, P, eta_nodal=eta, levels=levels, coarse_rtol=1e-14, imax=400, **o)
    return mesh, Problem(mesh, levels, eta_nodal=eta), s


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("key", list(HIER))
def test_numbering_coordinates_diagonal_and_apply(sem, key):
    mesh, prob, s = _make(sem, key)
    try:
        for li, lev in enumerate(prob.levels):
            q = s.query(li)
            assert q["ndof"] == lev.N and q["np"] == lev.ref.Np
            np.testing.assert_array_equal(s.element_map(li), lev.emap)
            np.testing.assert_array_equal(s.dirichlet_nodes(li), lev.dirichlet)
            np.testing.assert_allclose(s.coords(li), prob.coords(li), atol=1e-13)
            assert _rel(s.diagonal(li), prob.stiffness(li).diagonal()) < 1e-12
            x = W.random_vector(lev.N, seed=li)
            y = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
            s.apply(li, torch.tensor(x, device="cuda"), y)
            torch.cuda.synchronize()
            assert _rel(y.cpu().numpy(), prob.masked_apply(li, x)) < 1e-12
            y32 = torch.zeros(lev.N, dtype=torch.float32, device="cuda")
            s.apply32(li, torch.tensor(x, dtype=torch.float32, device="cuda"), y32)
            torch.cuda.synchronize()
            assert _rel(y32.cpu().numpy().astype(np.float64), prob.masked_apply(li, x)) < 1e-5
    finally:
        s.close()


@pytest.mark.parametrize("key", ["53", "64"])
def test_semi_coarsened_vcycle(sem, key):
    mesh, prob, s = _make(sem, key, k_cheb=3, cheb_lo=0.1, cheb_hi=1.1)
    try:
        ops = S.MGOperators(prob, k_cheb=3, lo=0.1, hi=1.1, lambdas=list(s.lambdas()[:-1]))
        lev = prob.levels[0]
        f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=3))
        z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        s.vcycle(torch.tensor(f, device="cuda"), z)
        torch.cuda.synchronize()
        assert _rel(z.cpu().numpy(), ops.vcycle(f)) < 1e-10
        # the library's lambda_hat is the oracle's Lanczos estimate
        lam = [S.lanczos_lambda(ops.A[li], ops.Dinv[li], prob.levels[li].dmask) for li in range(len(HIER[key]) - 1)]
        assert np.allclose(s.lambdas()[:-1], lam, rtol=1e-10)
    finally:
        s.close()


def _phid(prob):
    lev = prob.levels[0]
    C = prob.coords(0)
    return W.potential3d(*C[lev.dirichlet].T)


@pytest.mark.parametrize("key,opts,tol,bound", [
    ("53", dict(), 1e-13, 1e-10),
    ("42", dict(outer="fgmres"), 1e-13, 1e-10),
    ("64", dict(outer="pdc"), 1e-13, 1e-10),
    ("53", dict(precision="mixed_fp32", outer="pdc", inner_imax=40), 1e-11, 1e-8),
    ("53", dict(precision="mixed_tf32", outer="pdc", inner_imax=40), 1e-11, 1e-8),
    ("53", dict(smoother="asm", nu1=3, nu2=3), 1e-13, 1e-10),
])
def test_solves_reach_the_direct_solution(sem, key, opts, tol, bound):
    mesh, prob, s = _make(sem, key, **opts)
    try:
        phiD = _phid(prob)
        ref = S.solve_laplace_direct(prob, phiD)
        phi = torch.zeros(prob.levels[0].N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=tol)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert _rel(phi.cpu().numpy(), ref) <= bound
    finally:
        s.close()


def test_schwarz_subdomains_on_anisotropic_levels(sem):
    mesh, prob, s = _make(sem, "53", smoother="asm", precision="mixed_fp32")
    try:
        for li in range(2):
            got = s.asm_subdomains(li)
            want = SZ.subdomains(prob, li, 1)
            assert all(np.array_equal(g, w) for g, w in zip(got, want))
    finally:
        s.close()


def test_free_surface_rhs_on_anisotropic_prisms(sem):
    mesh = W.box3d(3, 2, 2)
    levels = HIER["53"]
    xy = sem.sem_mesh_nodes2d(mesh, 5)
    x, y = xy[:, 0], xy[:, 1]
    eta = 0.05 * np.cos(x) * np.cos(y)
    phis = 0.03 * np.cos(x) * np.cos(2 * y)
    s = sem.Solver(mesh, 5, eta_nodal=np.zeros(len(xy)), levels=levels, surface_ops=1, coarse_rtol=1e-14, imax=400)
    try:
        de = torch.zeros(len(xy), dtype=torch.float64, device="cuda")
        dp = torch.zeros_like(de)
        s.fnpf_rhs(torch.tensor(eta, device="cuda"), torch.tensor(phis, device="cuda"), de, dp, tol=1e-13)
        re, rp = F.fnpf_rhs(mesh, levels, eta, phis)
        assert _rel(de.cpu().numpy(), re) <= 1e-9
        assert _rel(dp.cpu().numpy(), rp) <= 1e-9
    finally:
        s.close()


def test_refusals(sem):
    mesh = _mesh()
    for levels in ([(5, 2), (2, 2), (1, 1)],          # vertical order three below: not compiled
                   [(4, 2), (4, 3), (1, 1)],          # an order grows
                   [(4, 2), (4, 2), (1, 1)],          # no order falls
                   [(3, 3), (2, 2), (1, 2)]):         # coarsest not (1, 1)
        with pytest.raises(sem.SemError) as e:
            sem.Solver(mesh, levels[0][0], levels=levels)
        assert e.value.status == sem.SEM_EINVAL
    with pytest.raises(sem.SemError) as e:
        sem.Solver(W.slice2d(4, 2), 4, levels=[(4, 2), (2, 2), (1, 1)])   # 2D has no vertical order
    assert e.value.status == sem.SEM_EINVAL
    s = sem.Solver(mesh, 5, levels=HIER["53"], precision="mixed_tf32")
    try:
        n = s.query(0)["ndof"]
        x = torch.zeros(n, dtype=torch.float32, device="cuda")
        with pytest.raises(sem.SemError):
            s.apply32(0, x, x.clone(), tensor_cores=True)        # tensor-core apply: isotropic levels only
    finally:
        s.close()
