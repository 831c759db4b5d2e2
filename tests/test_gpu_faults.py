"""Failure detection on the GPU without faulting it: a bounded device-side wait
that is made to run out reports SEM_TIMEOUT, and the context stays usable."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


def _solve(sem, **opts):
    mesh = W.config_box3d(3, 2)
    P = 3
    xy = sem.sem_mesh_nodes2d(mesh, P)
    s = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), **opts)
    C = s.coords(0)
    phiD = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
    phi = torch.zeros(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
    return s, phiD, phi


@pytest.mark.parametrize("bj", [1, 0])
def test_coarse_barrier_wait_runs_out_into_sem_timeout(sem, bj):
    # the block-Jacobi and the point-Jacobi coarse CG both wait on the same bounded barrier
    s, phiD, phi = _solve(sem, debug_barrier_extra=1, coarse_bj=bj)
    with pytest.raises(sem.SemError) as e:
        s.solve(phiD, phi, tol=1e-8)
    assert e.value.status == sem.SEM_TIMEOUT
    assert "timeout" in sem.sem_last_error()
    s.close()
    # the context is still usable: a normal solve on a fresh handle succeeds
    s2, phiD2, phi2 = _solve(sem)
    st = s2.solve(phiD2, phi2, tol=1e-8)
    assert st["status"] == 0 and torch.isfinite(phi2).all()
    s2.close()
