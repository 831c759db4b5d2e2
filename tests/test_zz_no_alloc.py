"""The allocation-free CG entry point (sem_cg_csr_noalloc) against the existing
coarse solve.

Some callers cannot call cudaMalloc (their device memory belongs to another
framework's pool, or they run in loops that cannot absorb an allocation's
device-wide synchronisation).  sem_cg_csr_noalloc gives them the library's
FP64 Jacobi-CG on their own CSR matrix with every work buffer in a static device
array.  Here it solves the order-1 system of a 3D sigma-prism box, assembled by
the oracle in the library's numbering, and must agree with pmg_vcycle of a
single-level order-1 handle (whose V-cycle is exactly that coarse CG) on two
calls in a row, and a sparse direct solve of the same matrix done here.  A call
capped below convergence must say so (SEM_NOT_CONVERGED, with the iteration
count), and a NaN in the right-hand side must come back as SEM_NAN.  Collected last (file name) so that a failure here comes after
every other test has run."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.assemble import Problem  # noqa: E402

TOL = 1e-10          # the V-cycle parity tolerance of tests/test_gpu_parity.py


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


def test_noalloc_cg_matches_single_level_vcycle_twice(sem):
    mesh = W.config_box3d(40, 4)
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    keep = sp.diags((~lev.dmask).astype(np.float64))
    A = (keep @ prob.stiffness(0) @ keep).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    d = prob.stiffness(0).diagonal()
    dinv = np.where(lev.dmask, 0.0, 1.0 / np.where(lev.dmask, 1.0, d))
    solver = sem.Solver(mesh, 1, eta_nodal=prob.eta_nodal, levels=[1], coarse_rtol=1e-14, coarse_imax=20000)
    dev = lambda a, t=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    rowptr, col, vals, dv = dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data), dev(dinv)
    for seed in (21, 22):
        r = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=seed))
        z_ref = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        solver.vcycle(dev(r), z_ref)
        x = torch.full((lev.N,), float("nan"), dtype=torch.float64, device="cuda")
        its = sem.sem_cg_csr_noalloc(lev.N, rowptr, col, vals, dv, dev(r), x, 1e-14, 20000)
        torch.cuda.synchronize()
        got, ref = x.cpu().numpy(), z_ref.cpu().numpy()
        assert its > 0
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
        # independent of the library: a sparse direct solve of the test's own matrix on the free rows
        free = ~lev.dmask
        exact = np.zeros(lev.N)
        exact[free] = spla.spsolve(A[free][:, free].tocsc(), r[free])
        assert np.abs(got - exact).max() <= 1e-9 * np.abs(exact).max()
    solver.close()


def _box_system(sem, seed):
    mesh = W.config_box3d(12, 2)
    prob = Problem(mesh, [1])
    lev = prob.levels[0]
    keep = sp.diags((~lev.dmask).astype(np.float64))
    A = (keep @ prob.stiffness(0) @ keep).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    d = prob.stiffness(0).diagonal()
    dinv = np.where(lev.dmask, 0.0, 1.0 / np.where(lev.dmask, 1.0, d))
    r = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=seed))
    dev = lambda a, t=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    return lev.N, dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data), dev(dinv), r, dev


def test_noalloc_cg_stops_at_imax_with_not_converged(sem):
    n, rowptr, col, vals, dv, r, dev = _box_system(sem, 31)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.sem_cg_csr_noalloc(n, rowptr, col, vals, dv, dev(r), x, 1e-14, 3)
    assert e.value.status == sem.SEM_NOT_CONVERGED
    its = sem.sem_cg_csr_noalloc(n, rowptr, col, vals, dv, dev(r), x, 1e-14, 3, allow_not_converged=True)
    assert its == 3
    assert np.isfinite(x.cpu().numpy()).all()


def test_noalloc_cg_reports_a_non_finite_right_hand_side(sem):
    n, rowptr, col, vals, dv, r, dev = _box_system(sem, 32)
    free = np.flatnonzero(r != 0.0)
    r[free[len(free) // 2]] = np.nan
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.sem_cg_csr_noalloc(n, rowptr, col, vals, dv, dev(r), x, 1e-10, 100, allow_not_converged=True)
    assert e.value.status == sem.SEM_NAN


def test_noalloc_cg_rejects_sizes_beyond_its_scratch(sem):
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.sem_cg_csr_noalloc(1 << 20, i, i, x, x, x, x, 1e-8, 10)
    assert e.value.status == sem.SEM_EINVAL and "static scratch" in sem.sem_last_error()
