"""The TF32 tensor-core prism apply (Chebyshev sweeps of the MIXED_TF32 V-cycle).

Tolerance: the MMA operands are rounded to TF32 (unit roundoff 2^-11 = 4.9e-4)
and the geometric factors come from a BF16 copy (unit roundoff 2^-9 = 2.0e-3);
products accumulate in FP32.  An entry of y = A x therefore carries an error of
a few 1e-3 of the terms it sums; for random x the entries are of the size of
their terms, and the bound is 1e-2 of max|y| entrywise and 4e-3 of ||y||_2.
The solves that use the kernel still reach an FP64 residual of 1e-11, so their
error against the oracle's direct solution is the tolerance's (1e-8)."""
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


SMALL = {
    "p6": (lambda: W.config_box3d(3, 3), [6, 3, 1]),
    "p5_ragged": (lambda: W.box3d(5, 3, 3, eta_modes=W.eta_sinx_cosy(0.08)), [5, 3, 1]),
    "p4": (lambda: W.config_box3d(4, 2), [4, 2, 1]),
    "p3": (lambda: W.box3d(4, 3, 2, eta_modes=W.eta_sinx_cosy(0.1)), [3, 2, 1]),
}


def _solver(sem, mesh, prob, levels, **o):
    return sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, levels=levels, coarse_rtol=1e-14, **o)


def _check_apply(y_tc, y_ref):
    scale = np.abs(y_ref).max()
    e_max = np.abs(y_tc - y_ref).max() / scale
    e_2 = np.linalg.norm(y_tc - y_ref) / np.linalg.norm(y_ref)
    print(f"tensor-core apply: max error {e_max:.2e} of max|y|, 2-norm error {e_2:.2e}")
    assert e_max <= 1e-2 and e_2 <= 4e-3


@pytest.mark.parametrize("name", list(SMALL))
def test_tensor_core_apply_matches_oracle_on_every_level(sem, name):
    mesh_fn, levels = SMALL[name]
    mesh = mesh_fn()
    prob = Problem(mesh, levels)
    s = _solver(sem, mesh, prob, levels)
    try:
        for li, p in enumerate(levels):
            if p < 2:
                continue
            N = prob.levels[li].N
            x = W.random_vector(N, seed=100 + li).astype(np.float32)
            xd = torch.tensor(x, device="cuda")
            y_tc = torch.zeros(N, dtype=torch.float32, device="cuda")
            y_32 = torch.zeros(N, dtype=torch.float32, device="cuda")
            s.apply32(li, xd, y_tc, tensor_cores=True)
            s.apply32(li, xd, y_32, tensor_cores=False)
            torch.cuda.synchronize()
            ref = prob.masked_apply(li, x.astype(np.float64))
            y32 = y_32.cpu().numpy().astype(np.float64)
            assert np.abs(y32 - ref).max() <= 1e-5 * np.abs(ref).max()
            _check_apply(y_tc.cpu().numpy().astype(np.float64), ref)
    finally:
        s.close()


def test_tensor_core_apply_many_passes_per_cta(sem):
    # 19 x 19 x 3 prisms at P = 6: 2166 elements = 542 passes of 4 over at most 304
    # CTAs (two per SM), the last pass ragged (2 elements); rows sampled against the oracle
    mesh = W.box3d(19, 19, 3, eta_modes=W.eta_sinx_cosy(0.1))
    levels = [6, 3, 1]
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    s = sem.Solver(mesh, 6, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=levels)
    try:
        q = s.query(0)
        N = q["ndof"]
        x = W.random_vector(N, seed=7).astype(np.float32)
        xd = torch.tensor(x, device="cuda")
        y_tc = torch.zeros(N, dtype=torch.float32, device="cuda")
        y_32 = torch.zeros(N, dtype=torch.float32, device="cuda")
        s.apply32(0, xd, y_tc, tensor_cores=True)
        s.apply32(0, xd, y_32, tensor_cores=False)
        torch.cuda.synchronize()
        _check_apply(y_tc.cpu().numpy().astype(np.float64), y_32.cpu().numpy().astype(np.float64))
        prob = Problem(mesh, [6, 1])
        rows = np.random.default_rng(3).choice(N, 200, replace=False)
        ref = prob.apply_rows(0, x.astype(np.float64), rows)
        got = y_tc.cpu().numpy().astype(np.float64)[rows]
        assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max()
    finally:
        s.close()


def test_tensor_core_apply_rejects_triangles_and_order_one(sem):
    mesh = W.config_slice2d()
    s = sem.Solver(mesh, 4, levels=[4, 2, 1])
    try:
        x = torch.zeros(s.query(0)["ndof"], dtype=torch.float32, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(sem.SemError) as e:
            s.apply32(0, x, y, tensor_cores=True)
        assert e.value.status == sem.SEM_EINVAL
    finally:
        s.close()


@pytest.mark.parametrize("name", ["p6", "p5_ragged"])
def test_mixed_tf32_solve_matches_oracle(sem, name):
    mesh_fn, levels = SMALL[name]
    mesh = mesh_fn()
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    phi_ref = S.solve_laplace_direct(prob, phiD)
    its = {}
    for prec in ("mixed_fp32", "mixed_tf32"):
        s = _solver(sem, mesh, prob, levels, outer="pdc", precision=prec, inner_imax=50, inner_rtol=1e-4,
                    imax=100)
        try:
            phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
            st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-11)
            torch.cuda.synchronize()
            assert st["status"] == 0 and st["res_final"] <= 1e-11 * st["fnorm"]
            got = phi.cpu().numpy()
            assert np.abs(got - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
            its[prec] = (st["iters"], st["inner_iters"])
        finally:
            s.close()
    # the smoothing operator's rounding leaves the convergence essentially unchanged
    assert its["mixed_tf32"][1] <= its["mixed_fp32"][1] + 3, its


@pytest.mark.parametrize("n,nl", [(3, 3), (40, 4)])
def test_tcgen05_apply_against_warp_mma_and_oracle(sem, n, nl):
    # order 6: the tcgen05 kernel (16 elements per pass, M = 128 rows) against the warp-MMA kernel,
    # the FP32 apply and the oracle's rows; 3x3x3 = 54 prisms is four passes, the last ragged (6
    # elements); 40x40x4 = 12,800 prisms is 800 passes, five or six per CTA
    mesh = W.box3d(n, n, nl, eta_modes=W.eta_sinx_cosy(0.1))
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    s = sem.Solver(mesh, 6, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=[6, 3, 1])
    try:
        N = s.query(0)["ndof"]
        x = W.random_vector(N, seed=29).astype(np.float32)
        xd = torch.tensor(x, device="cuda")
        ys = {k: torch.zeros(N, dtype=torch.float32, device="cuda") for k in (0, 1, 2)}
        for k, y in ys.items():
            s.apply32(0, xd, y, tensor_cores=k)
        torch.cuda.synchronize()
        y32, ymma, y5 = (ys[k].cpu().numpy().astype(np.float64) for k in (0, 1, 2))
        _check_apply(y5, y32)
        _check_apply(ymma, y32)
        # the two tensor-core forms round alike (TF32 operands, BF16 factors): they agree more
        # closely with each other than either with the FP32 apply
        assert np.linalg.norm(y5 - ymma) <= 2e-3 * np.linalg.norm(y32)
        prob = Problem(mesh, [6, 1])
        rows = np.random.default_rng(4).choice(N, 120, replace=False)
        ref = prob.apply_rows(0, x.astype(np.float64), rows)
        assert np.abs(y5[rows] - ref).max() <= 1e-2 * np.abs(ref).max()
        # repeated launches give the same result up to the order of the atomic summation
        y2 = torch.zeros(N, dtype=torch.float32, device="cuda")
        s.apply32(0, xd, y2, tensor_cores=2)
        torch.cuda.synchronize()
        assert np.abs(y2.cpu().numpy() - y5).max() <= 1e-5 * np.abs(y5).max()
        # the tcgen05 kernel exists for order 6 only
        if n == 3:
            xc = torch.zeros(s.query(1)["ndof"], dtype=torch.float32, device="cuda")
            with pytest.raises(sem.SemError):
                s.apply32(1, xc, torch.zeros_like(xc), tensor_cores=2)
    finally:
        s.close()


@pytest.mark.parametrize("autotune", [0, 1])
def test_mixed_tf32_solve_with_the_tcgen05_smoother_matches_oracle(sem, autotune):
    # the V-cycle's Chebyshev sweeps on the order-6 level run the tcgen05 kernel (autotune = 0
    # takes it; autotune = 1 keeps whichever kernel is faster on the mesh and says which); the
    # solve still reaches the FP64 residual and the oracle's direct solution
    mesh = W.box3d(6, 6, 3, eta_modes=W.eta_sinx_cosy(0.1))
    levels = [6, 3, 1]
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    phi_ref = S.solve_laplace_direct(prob, phiD)
    s = _solver(sem, mesh, prob, levels, outer="pdc", precision="mixed_tf32", inner_imax=50, inner_rtol=1e-4,
                imax=100, autotune=autotune)
    try:
        kind = s.tc_kernel(0)
        assert kind == 2 if autotune == 0 else kind in (1, 2)
        assert s.tc_kernel(1) == 1 and s.tc_kernel(2) == 0      # order 3: warp MMA; order 1: FP32
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-11)
        torch.cuda.synchronize()
        assert st["status"] == 0 and st["res_final"] <= 1e-11 * st["fnorm"]
        assert np.abs(phi.cpu().numpy() - phi_ref).max() <= 1e-8 * np.abs(phi_ref).max()
    finally:
        s.close()
