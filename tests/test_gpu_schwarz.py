"""The additive Schwarz smoother on the GPU (Section 4.3, Eqs. sec_form, Mass, weights)
against the oracle (oracle/schwarz.py).

* subdomains: the free node sets of every element's subdomain equal the oracle's exactly
  (index work), on every smoothed level, for overlaps 0, 1 and the refined variant;
* S^{-1} r and S^{-T} r with the FP64 blocks: 1e-11 relative to the oracle's dense
  solves (the blocks are inverted by Gauss-Jordan at condition numbers up to ~1e4);
  with the FP32 blocks of a mixed-precision handle: 2e-3 (FP32 inversion at that
  condition number, and the FP32 element matrices);
* the V-cycle with ASM smoothing: 1e-10 against the oracle's (exact coarse solve, coarse
  CG to 1e-14 here); PCG solves: 1e-10 against the direct solution at rtol 1e-13, the
  mixed precisions 1e-8 at rtol 1e-11;
* sem_update_eta: ALL gives the blocks of a fresh setup (1e-11), FINEST keeps the t = 0
  blocks (the same apply up to the order of the atomic scatter, 1e-14).
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


CASES = {
    "slice2d_p6": (lambda: W.slice2d(6, 3), [6, 3, 1]),
    "box3d_p6": (lambda: W.box3d(3, 3, 3, eta_modes=W.eta_sinx_cosy(0.1)), [6, 3, 1]),
    "box3d_p4": (lambda: W.box3d(4, 3, 2, eta_modes=W.eta_sinx_cosy(0.1)), [4, 2, 1]),
}


def _eta(sem, mesh, P):
    if mesh.dim != 3:
        return None
    xy = sem.sem_mesh_nodes2d(mesh, P)
    return mesh.eta(xy[:, 0], xy[:, 1])


def _setup(sem, name, overlap=1, **o):
    mk, levels = CASES[name]
    mesh = mk()
    s = sem.Solver(mesh, levels[0], eta_nodal=_eta(sem, mesh, levels[0]), levels=levels, smoother="asm",
                   asm_overlap=overlap, coarse_rtol=1e-14, imax=400, **o)
    return mesh, levels, s


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name,overlap", [(n, o) for n in CASES for o in (0, 1, -1) if (n, o) != ("box3d_p6", -1)])
def test_subdomains_match_the_oracle(sem, name, overlap):
    # (refined overlap at order 6 in 3D makes 2400-node blocks: allowed in FP32, but their
    # inversion streams O(n^3 / 16) words per block, too slow for a test)
    mesh, levels, s = _setup(sem, name, overlap, precision="mixed_fp32")
    try:
        prob = Problem(mesh, levels)
        for li in range(len(levels) - 1):
            got = s.asm_subdomains(li)
            want = SZ.subdomains(prob, li, overlap)
            assert len(got) == len(want)
            for g, w in zip(got, want):
                assert np.array_equal(g, w)
    finally:
        s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_block_apply_fp64(sem, name):
    mesh, levels, s = _setup(sem, name)
    try:
        prob = Problem(mesh, levels)
        ops = S.MGOperators(prob, smoother="asm", overlap=1)
        for li in range(len(levels) - 1):
            lev = prob.levels[li]
            r = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=10 + li))
            for adjoint in (False, True):
                z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
                s.asm_apply(li, torch.tensor(r, device="cuda"), z, adjoint)
                torch.cuda.synchronize()
                want = ops.asm[li].apply(r, adjoint)
                assert _rel(z.cpu().numpy(), want) <= 1e-11, (li, adjoint)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["box3d_p6", "slice2d_p6"])
def test_block_apply_fp32(sem, name):
    mesh, levels, s = _setup(sem, name, precision="mixed_fp32")
    try:
        prob = Problem(mesh, levels)
        ops = S.MGOperators(prob, smoother="asm", overlap=1)
        for li in range(len(levels) - 1):
            lev = prob.levels[li]
            r = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=20 + li))
            for adjoint in (False, True):
                z = torch.zeros(lev.N, dtype=torch.float32, device="cuda")
                s.asm_apply32(li, torch.tensor(r, dtype=torch.float32, device="cuda"), z, adjoint)
                torch.cuda.synchronize()
                want = ops.asm[li].apply(r, adjoint)
                assert _rel(z.cpu().numpy().astype(np.float64), want) <= 2e-3, (li, adjoint)
    finally:
        s.close()


@pytest.mark.parametrize("name", ["box3d_p6", "slice2d_p6"])
def test_vcycle_matches_the_oracle(sem, name):
    mesh, levels, s = _setup(sem, name, nu1=2, nu2=2)
    try:
        prob = Problem(mesh, levels)
        ops = S.MGOperators(prob, nu1=2, nu2=2, smoother="asm", overlap=1)
        lev = prob.levels[0]
        f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=3))
        z = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        s.vcycle(torch.tensor(f, device="cuda"), z)
        torch.cuda.synchronize()
        assert _rel(z.cpu().numpy(), ops.vcycle(f)) <= 1e-10
    finally:
        s.close()


def _dirichlet_data(prob):
    lev = prob.levels[0]
    C = prob.coords(0)
    if prob.dim == 3:
        return W.potential3d(*C[lev.dirichlet].T)
    return W.airy2d(C[lev.dirichlet, 0], C[lev.dirichlet, 1])


@pytest.mark.parametrize("name", list(CASES))
def test_pcg_with_asm_reaches_the_direct_solution(sem, name):
    mesh, levels, s = _setup(sem, name, nu1=3, nu2=3)
    try:
        prob = Problem(mesh, levels)
        lev = prob.levels[0]
        phiD = _dirichlet_data(prob)
        ref = S.solve_laplace_direct(prob, phiD)
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-13)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert _rel(phi.cpu().numpy(), ref) <= 1e-10
        # the same iteration as the oracle's PCG (same V-cycle up to rounding)
        ops = S.MGOperators(prob, nu1=3, nu2=3, smoother="asm", overlap=1)
        res = S.pcg(ops, S.lift(prob, phiD), rtol=1e-13)
        assert abs(st["iters"] - res.iters) <= 1
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["mixed_fp32", "mixed_tf32"])
def test_mixed_asm_solves(sem, precision):
    mesh, levels, s = _setup(sem, "box3d_p6", nu1=3, nu2=3, precision=precision, outer="pdc")
    try:
        prob = Problem(mesh, levels)
        lev = prob.levels[0]
        phiD = _dirichlet_data(prob)
        ref = S.solve_laplace_direct(prob, phiD)
        phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
        st = s.solve(torch.tensor(phiD, device="cuda"), phi, tol=1e-11)
        torch.cuda.synchronize()
        assert st["status"] == 0
        assert _rel(phi.cpu().numpy(), ref) <= 1e-8
        assert st["asm_launches"] >= 0
    finally:
        s.close()


def test_update_eta_rebuilds_or_keeps_the_blocks(sem):
    modes1 = [(0.06, 2.0, 1.0, 0.3), (0.04, 1.0, 3.0, 1.1)]
    mesh1 = W.box3d(3, 3, 3, eta_modes=modes1)
    xy = sem.sem_mesh_nodes2d(mesh1, 6)
    eta1 = mesh1.eta(xy[:, 0], xy[:, 1])
    fresh = sem.Solver(mesh1, 6, eta_nodal=eta1, levels=[6, 3, 1], smoother="asm", coarse_rtol=1e-14)
    _, _, s_all = _setup(sem, "box3d_p6")
    _, _, s_fin = _setup(sem, "box3d_p6")
    try:
        n = s_all.query(0)["ndof"]
        r = torch.tensor(W.random_vector(n, seed=8), device="cuda")

        def z_of(h):
            z = torch.zeros(n, dtype=torch.float64, device="cuda")
            h.asm_apply(0, r, z)
            torch.cuda.synchronize()
            return z.cpu().numpy()

        before = z_of(s_fin)
        s_all.update_eta(eta1, "all")
        s_fin.update_eta(eta1, "finest")
        assert _rel(z_of(s_all), z_of(fresh)) <= 1e-11
        # the same blocks; the atomic scatter into z adds in a varying order
        assert _rel(z_of(s_fin), before) <= 1e-14
    finally:
        for h in (fresh, s_all, s_fin):
            h.close()


def test_refusals(sem):
    # refined overlap at order 6 in 3D makes subdomains of ~2400 nodes: too large for FP64
    mk, levels = CASES["box3d_p6"]
    with pytest.raises(sem.SemError) as e:
        sem.Solver(mk(), 6, levels=levels, smoother="asm", asm_overlap=-1)
    assert e.value.status == sem.SEM_EINVAL
    cheb = sem.Solver(mk(), 6, levels=levels)
    _, _, s = _setup(sem, "box3d_p4", precision="mixed_fp32")
    try:
        n = cheb.query(0)["ndof"]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(sem.SemError):
            cheb.asm_apply(0, x, x.clone())                 # no blocks on a Chebyshev handle
        n4 = s.query(0)["ndof"]
        x4 = torch.zeros(n4, dtype=torch.float64, device="cuda")
        with pytest.raises(sem.SemError):
            s.asm_apply(0, x4, x4.clone())                   # FP32 blocks: asm_apply32 only
        with pytest.raises(sem.SemError):
            s.asm_apply32(len(CASES["box3d_p4"][1]) - 1, x4.float(), x4.float().clone())   # coarsest level
    finally:
        cheb.close()
        s.close()
