"""Free-surface time stepping on the GPU (Section 2, Eqs. FSeta, FSphi, ERK4) against
the oracle (oracle/fnpf.py) and the linear standing wave's closed form.

Tolerances: the right-hand sides come from Laplace solves at rtol 1e-13 against the
oracle's direct solve, so they agree to ~1e-10 of their size (1e-9 asserted); three
ERK4 steps compound that (1e-8); the standing wave is held to the oracle's own pin
(1e-4 of the amplitude after half a period)."""
import math

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fnpf as F  # noqa: E402

LEVELS = [4, 2, 1]


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    pkg.lib()
    return pkg


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _setup(sem, mesh, levels, eta0):
    return sem.Solver(mesh, levels[0], eta_nodal=eta0, levels=levels, surface_ops=1, coarse_rtol=1e-14, imax=400)


def _fields(sem, mesh, P):
    xy = sem.sem_mesh_nodes2d(mesh, P)
    x, y = xy[:, 0], xy[:, 1]
    eta = 0.05 * np.cos(x) * np.cos(y) + 0.02 * np.cos(2 * x + 0.3)
    phis = 0.03 * np.cos(x) * np.cos(2 * y) - 0.01 * np.sin(y + 0.2)
    return xy, eta, phis


def test_right_hand_sides_match_the_oracle(sem):
    mesh = W.box3d(4, 3, 2)
    xy, eta, phis = _fields(sem, mesh, LEVELS[0])
    s = _setup(sem, mesh, LEVELS, np.zeros(len(xy)))
    try:
        for linear in (False, True):
            de, dp = torch.zeros(len(xy), dtype=torch.float64, device="cuda"), torch.zeros(len(xy), dtype=torch.float64,
                                                                                             device="cuda")
            s.fnpf_rhs(_dev(eta), _dev(phis), de, dp, linear=linear, tol=1e-13)
            re, rp = F.fnpf_rhs(mesh, LEVELS, eta, phis, linear=linear)
            assert _rel(de.cpu().numpy(), re) <= 1e-9, linear
            assert _rel(dp.cpu().numpy(), rp) <= 1e-9, linear
            if not linear:
                s.update_eta(np.zeros(len(xy)), "all")      # the linear form runs on the flat geometry
    finally:
        s.close()


def test_erk4_steps_match_the_oracle(sem):
    mesh = W.box3d(4, 3, 2)
    xy, eta, phis = _fields(sem, mesh, LEVELS[0])
    s = _setup(sem, mesh, LEVELS, eta)
    try:
        e, p = _dev(eta), _dev(phis)
        re, rp = eta.copy(), phis.copy()
        for _ in range(3):
            st = s.fnpf_step(e, p, 0.05, tol=1e-13, strategy="all")
            assert st["status"] == 0 and st["iters"] > 0
            re, rp = F.erk4_step(mesh, LEVELS, re, rp, 0.05)
        assert _rel(e.cpu().numpy(), re) <= 1e-8
        assert _rel(p.cpu().numpy(), rp) <= 1e-8
    finally:
        s.close()


def test_reuse_strategies_reach_the_same_step(sem):
    # FINEST keeps the t = 0 smoother and coarse operators: a different preconditioner for
    # the same finest problem, so the step agrees to the solver tolerance
    mesh = W.box3d(4, 3, 2)
    xy, eta, phis = _fields(sem, mesh, LEVELS[0])
    out = {}
    for strat in ("all", "finest", "linear_coarse"):
        s = _setup(sem, mesh, LEVELS, eta)
        try:
            e, p = _dev(eta), _dev(phis)
            for _ in range(2):
                s.fnpf_step(e, p, 0.05, tol=1e-12, strategy=strat)
            out[strat] = (e.cpu().numpy(), p.cpu().numpy())
        finally:
            s.close()
    for strat in ("finest", "linear_coarse"):
        assert _rel(out[strat][0], out["all"][0]) <= 1e-9
        assert _rel(out[strat][1], out["all"][1]) <= 1e-9


def test_linear_standing_wave_on_the_gpu(sem):
    mesh = W.box3d(6, 2, 2)
    levels = [6, 3, 1]
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    s = _setup(sem, mesh, levels, np.zeros(len(xy)))
    try:
        a, g = 1e-2, 9.81
        omega = math.sqrt(g * math.tanh(1.0))
        steps = 20
        dt = 0.5 * 2 * math.pi / omega / steps
        e, p = _dev(a * np.cos(xy[:, 0])), _dev(np.zeros(len(xy)))
        for _ in range(steps):
            s.fnpf_step(e, p, dt, g=g, linear=True, tol=1e-12)
        assert np.abs(e.cpu().numpy() + a * np.cos(xy[:, 0])).max() < 1e-4 * a
    finally:
        s.close()


def test_surface_operations_need_their_setup(sem):
    mesh = W.box3d(3, 2, 2)
    xy = sem.sem_mesh_nodes2d(mesh, 3)
    s = sem.Solver(mesh, 3, levels=[3, 2, 1])
    try:
        z = _dev(np.zeros(len(xy)))
        with pytest.raises(sem.SemError) as e:
            s.fnpf_step(z, z.clone(), 0.01)
        assert e.value.status == sem.SEM_EINVAL
    finally:
        s.close()
    with pytest.raises(sem.SemError) as e:
        sem.Solver(W.all_boundary_dirichlet(W.box3d(3, 2, 2)), 3, levels=[3, 2, 1], surface_ops=1)
    assert e.value.status == sem.SEM_EINVAL
