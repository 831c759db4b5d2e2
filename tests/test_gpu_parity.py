"""GPU parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64 path): operator apply and assembled diagonal 1e-12 relative to
the largest entry (rounding of a different summation order, O(10) terms per
entry, is ~1e-15); V-cycle 1e-10 (the coarse CG is run to 1e-14 instead of the
oracle's direct coarse solve); solution of the discrete problem 1e-10 relative
(solve run at rtol 1e-13, the criterion of the FP64 path).
"""
import math

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
    pkg.lib()
    return pkg


CASES = {
    "slice2d_p4": (lambda: W.config_slice2d(), [4, 2, 1]),
    "slice2d_p6": (lambda: W.slice2d(5, 3), [6, 3, 1]),
    "box3d_p4": (lambda: W.config_box3d(4, 2), [4, 2, 1]),
    "box3d_p6": (lambda: W.config_box3d(3, 3), [6, 3, 1]),
    "box3d_p5_ragged": (lambda: W.box3d(5, 3, 3, eta_modes=W.eta_sinx_cosy(0.08)), [5, 3, 1]),
    "box3d_p3": (lambda: W.box3d(4, 3, 2, eta_modes=W.eta_sinx_cosy(0.1)), [3, 2, 1]),
}


def make(sem, name, **opts):
    mesh_fn, levels = CASES[name]
    mesh = mesh_fn()
    prob = Problem(mesh, levels)
    o = dict(levels=levels, coarse_rtol=1e-14, cheb_lo=0.1, cheb_hi=1.1, k_cheb=3)
    o.update(opts)
    solver = sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, **o)
    return mesh, prob, solver


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_numbering_coordinates_and_dirichlet_sets(sem, name):
    mesh, prob, solver = make(sem, name)
    for li, lev in enumerate(prob.levels):
        q = solver.query(li)
        assert q["ndof"] == lev.N and q["nelem"] == lev.emap.shape[0] and q["np"] == lev.ref.Np
        np.testing.assert_array_equal(solver.element_map(li), lev.emap)
        np.testing.assert_array_equal(solver.dirichlet_nodes(li), lev.dirichlet)
        np.testing.assert_allclose(solver.coords(li), prob.coords(li), atol=1e-13)


@pytest.mark.parametrize("name", list(CASES))
def test_assembled_diagonal(sem, name):
    mesh, prob, solver = make(sem, name)
    for li in range(len(prob.levels)):
        d_ref = prob.stiffness(li).diagonal()
        assert relerr(solver.diagonal(li), d_ref) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_apply_every_level(sem, name):
    mesh, prob, solver = make(sem, name)
    for li, lev in enumerate(prob.levels):
        for seed in (1, 2):
            x = W.random_vector(lev.N, seed=seed)
            y = torch.full((lev.N,), float("nan"), dtype=torch.float64, device="cuda")
            solver.apply(li, dev(x), y)
            torch.cuda.synchronize()
            assert relerr(y.cpu().numpy(), prob.masked_apply(li, x)) < 1e-12, (li, seed)


@pytest.mark.parametrize("name", ["slice2d_p4", "box3d_p4", "box3d_p6"])
def test_chebyshev_bounds_from_power_iteration(sem, name):
    mesh, prob, solver = make(sem, name)
    ops = S.MGOperators(prob, lo=0.1, hi=1.1)
    lam = solver.lambdas()
    for li in range(len(prob.levels) - 1):
        assert abs(lam[li] - ops.lam[li]) < 1e-10 * ops.lam[li]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("nu,k", [((1, 1), 3), ((2, 2), 2)])
def test_vcycle(sem, name, nu, k):
    mesh, prob, solver = make(sem, name, nu1=nu[0], nu2=nu[1], k_cheb=k)
    ops = S.MGOperators(prob, nu1=nu[0], nu2=nu[1], k_cheb=k, lo=0.1, hi=1.1)
    lev = prob.levels[0]
    r = W.random_vector(lev.N, seed=7)
    z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    solver.vcycle(dev(r), z)
    torch.cuda.synchronize()
    z_ref = ops.vcycle(np.where(lev.dmask, 0.0, r))
    assert relerr(z.cpu().numpy(), z_ref) < 1e-10


def _dirichlet_data(prob, name):
    lev = prob.levels[0]
    C = prob.coords(0)
    if prob.dim == 2:
        return W.airy2d(*C[lev.dirichlet].T)
    return W.potential3d(*C[lev.dirichlet].T)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("outer", ["pcg", "fgmres", "pdc"])
def test_solve_matches_direct_solution(sem, name, outer):
    mesh, prob, solver = make(sem, name, outer=outer, imax=400)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, name)
    phi_ref = S.solve_laplace_direct(prob, phiD)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-13)
    torch.cuda.synchronize()
    assert st["status"] == 0
    assert st["res_final"] <= 1e-13 * st["fnorm"]
    assert relerr(phi.cpu().numpy(), phi_ref) < 1e-10


@pytest.mark.parametrize("name", ["slice2d_p4", "box3d_p4", "box3d_p6"])
def test_iteration_counts_match_oracle(sem, name):
    mesh, prob, solver = make(sem, name)
    ops = S.MGOperators(prob, lo=0.1, hi=1.1)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, name)
    f = S.lift(prob, phiD)
    ref = S.pcg(ops, f, rtol=1e-8)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-8)
    assert abs(st["iters"] - ref.iters) <= 1
    assert abs(st["fnorm"] - ref.fnorm) < 1e-12 * ref.fnorm


@pytest.mark.parametrize("name", ["slice2d_p4", "box3d_p4", "box3d_p6"])
@pytest.mark.parametrize("outer", ["pdc", "pcg", "fgmres"])
def test_mixed_precision_solve_error_vs_oracle(sem, name, outer):
    # FP32 V-cycle inside the FP64 outer iteration: the FP64 residual still reaches
    # the tolerance, so the error against the oracle is that of the tolerance.
    mesh, prob, solver = make(sem, name, outer=outer, precision="mixed_fp32", imax=400)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, name)
    phi_ref = S.solve_laplace_direct(prob, phiD)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-11)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["res_final"] <= 1e-11 * st["fnorm"]
    err = relerr(phi.cpu().numpy(), phi_ref)
    print(f"{name} mixed {outer}: iters {st['iters']} rel err vs oracle {err:.2e}")
    assert err < 1e-8


def test_host_buffer_solve_equals_device_solve(sem):
    mesh, prob, solver = make(sem, "box3d_p4")
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, "box3d_p4")
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    solver.solve(dev(phiD), phi, tol=1e-10)
    phi_h = np.zeros(lev.N)
    solver.solve_host(np.ascontiguousarray(phiD), phi_h, tol=1e-10)
    # same computation; the FP64 atomic summation order may differ between runs
    assert relerr(phi_h, phi.cpu().numpy()) < 1e-8


def test_rhs_load_vector(sem):
    mesh, prob, solver = make(sem, "box3d_p4")
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, "box3d_p4")
    rhs = W.random_vector(lev.N, seed=11)
    ref = S.lift(prob, phiD, rhs)
    u = S.direct_solve(prob, ref)
    u[lev.dirichlet] = phiD
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    solver.solve(dev(phiD), phi, tol=1e-13, rhs=dev(rhs))
    assert relerr(phi.cpu().numpy(), u) < 1e-10


# ---------------------------------------------------------------- edge cases
def test_single_element_and_single_level(sem):
    vxy = np.array([[0.0, -1.0], [1.0, -1.0], [0.0, 0.0]])
    mesh = W.Mesh(dim=2, vxy=vxy, tri=np.array([[0, 1, 2]], dtype=np.int32),
                  face_bc=np.array([[0, 0, 1]], dtype=np.int8))
    for levels in ([1], [3, 1], [5, 2, 1]):
        prob = Problem(mesh, levels)
        solver = sem.Solver(mesh, levels[0], levels=levels, coarse_rtol=1e-14)
        lev = prob.levels[0]
        x = W.random_vector(lev.N, seed=3)
        y = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        solver.apply(0, dev(x), y)
        assert relerr(y.cpu().numpy(), prob.masked_apply(0, x)) < 1e-12
        phiD = np.cos(prob.coords(0)[lev.dirichlet, 0])
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        solver.solve(dev(phiD), phi, tol=1e-13)
        assert relerr(phi.cpu().numpy(), S.solve_laplace_direct(prob, phiD)) < 1e-10


def test_all_neumann_is_rejected(sem):
    mesh = W.config_box3d(2, 2)
    mesh.face_bc[:] = 0
    with pytest.raises(sem.SemError) as e:
        sem.Solver(mesh, 3)
    assert e.value.status == sem.SEM_EINVAL and "singular" in sem.sem_last_error()


def test_nan_dirichlet_data_reports_nan(sem):
    mesh, prob, solver = make(sem, "box3d_p3")
    lev = prob.levels[0]
    phiD = np.full(lev.dirichlet.size, np.nan)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        solver.solve(dev(phiD), phi, tol=1e-8)
    assert e.value.status == sem.SEM_NAN


def test_imax_zero_returns_not_converged_with_stats(sem):
    mesh, prob, solver = make(sem, "box3d_p3", imax=0)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, "box3d_p3")
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-8, allow_not_converged=True)
    assert st["status"] == sem.SEM_NOT_CONVERGED and st["iters"] == 0
    # phi holds the Dirichlet data and the zero initial guess
    out = phi.cpu().numpy()
    np.testing.assert_array_equal(out[lev.dirichlet], phiD)
    assert np.all(out[lev.free] == 0)


def test_invalid_arguments(sem):
    mesh, prob, solver = make(sem, "box3d_p3")
    x = torch.zeros(prob.levels[0].N, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError):
        solver.apply(0, x, x)
    with pytest.raises(sem.SemError):
        solver.apply(9, x, torch.zeros_like(x))
    with pytest.raises(sem.SemError):
        sem.Solver(mesh, 7)
    with pytest.raises(sem.SemError):
        sem.Solver(mesh, 4, levels=[4, 3, 3, 1])


@pytest.mark.parametrize("name", ["slice2d_p4", "box3d_p4", "box3d_p6", "box3d_p5_ragged"])
def test_mixed_precision_inner_pcg(sem, name):
    # FP64 defect correction (Algorithm 2) around an FP32 PCG whose preconditioner is
    # the FP32 V-cycle: the FP64 residual reaches the tolerance, so the solution
    # matches the oracle's to the tolerance.
    mesh, prob, solver = make(sem, name, outer="pdc", precision="mixed_fp32", inner_imax=50, inner_rtol=1e-4,
                              imax=100)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, name)
    phi_ref = S.solve_laplace_direct(prob, phiD)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-11)
    torch.cuda.synchronize()
    assert st["status"] == 0 and st["res_final"] <= 1e-11 * st["fnorm"]
    assert st["inner_iters"] > 0 and st["iters"] <= 8
    err = relerr(phi.cpu().numpy(), phi_ref)
    print(f"{name} mixed inner PCG: outer {st['iters']} inner {st['inner_iters']} rel err {err:.2e}")
    assert err < 1e-8


@pytest.mark.parametrize("coarse_rtol", [1e-3, 1e-6])
def test_loose_coarse_tolerance_still_converges(sem, coarse_rtol):
    mesh, prob, solver = make(sem, "box3d_p6", coarse_rtol=coarse_rtol)
    lev = prob.levels[0]
    phiD = _dirichlet_data(prob, "box3d_p6")
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    st = solver.solve(dev(phiD), phi, tol=1e-12)
    assert st["status"] == 0
    assert relerr(phi.cpu().numpy(), S.solve_laplace_direct(prob, phiD)) < 1e-9
