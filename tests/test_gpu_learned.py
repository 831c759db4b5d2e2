"""The learned smoothing sweep: network forward/gradients and Adam against the FP64
oracle, one whole sweep (network correction, minimal-residual step, verdict,
Chebyshev fallback) against the oracle's sweep, training on solver-generated
residual/error pairs, and what the trained network gains over the plain method."""
import time

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import learned as L  # noqa: E402
from oracle import mlp as M  # noqa: E402
from oracle import solvers as S  # noqa: E402
from oracle.assemble import Problem  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2009_00705_gb300 as pkg
    from paper_2009_00705_gb300 import build as B
    B.build()
    return pkg


def _solver(sem, mesh, levels, **opts):
    prob = Problem(mesh, levels)
    o = dict(levels=levels, precision="mixed_fp32", smoother="learned", outer="pdc")
    o.update(opts)
    return prob, sem.Solver(mesh, levels[0], eta_nodal=prob.eta_nodal, **o)


@pytest.mark.parametrize("levels,hidden,mesh_fn", [([4, 2, 1], 40, lambda: W.config_box3d(4, 2)),
                                                    ([6, 3, 1], 256, lambda: W.config_box3d(3, 3))])
def test_network_forward_and_gradients_match_the_oracle(sem, levels, hidden, mesh_fn):
    prob, s = _solver(sem, mesh_fn(), levels, mlp_hidden=hidden)
    npe = prob.levels[0].ref.Np
    E = prob.levels[0].emap.shape[0]
    rng = np.random.default_rng(17)
    # bf16-representable weights: the library's GEMMs read W1, W2 as bf16
    W1 = M.bf16_round(rng.standard_normal((hidden, npe)) * 0.2).astype(np.float32)
    W2 = M.bf16_round(rng.standard_normal((npe, hidden)) * 0.2).astype(np.float32)
    b1 = (rng.standard_normal(hidden) * 0.1).astype(np.float32)
    b2 = (rng.standard_normal(npe) * 0.1).astype(np.float32)
    s.set_mlp_weights(W1, b1, W2, b2)
    B = E - 3                                        # a ragged batch
    X = rng.standard_normal((B, npe)).astype(np.float32)
    T = rng.standard_normal((B, npe)).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    Y = torch.zeros((B, npe), dtype=torch.float32, device="cuda")
    s.mlp_forward(B, Xd, Y)
    args = [a.astype(np.float64) for a in (W1, b1, W2, b2)]
    _, _, y_ref = M.forward(*args, X.astype(np.float64))
    assert np.abs(Y.cpu().numpy() - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    loss, g = s.mlp_gradient(B, Xd, Td)
    loss_ref, (gW1, gb1, gW2, gb2) = M.loss_and_grads(*args, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    for got, ref in ((g["W1"], gW1), (g["b1"], gb1), (g["W2"], gW2), (g["b2"], gb2)):
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    s.close()


def test_checkpoint_round_trip(sem):
    mesh = W.config_box3d(4, 2)
    prob, s1 = _solver(sem, mesh, [4, 2, 1], mlp_hidden=32)
    s1.train(1, 2, lr=1e-3, seed=5)
    w = s1.mlp_weights()
    _, s2 = _solver(sem, mesh, [4, 2, 1], mlp_hidden=32, mlp_seed=999)
    s2.set_mlp_weights(w["W1"], w["b1"], w["W2"], w["b2"])
    E, npe = prob.levels[0].emap.shape
    X = torch.randn((E, npe), dtype=torch.float32, device="cuda")
    Y1 = torch.zeros_like(X)
    Y2 = torch.zeros_like(X)
    s1.mlp_forward(E, X, Y1)
    s2.mlp_forward(E, X, Y2)
    assert torch.equal(Y1, Y2)
    s1.close()
    s2.close()


def test_training_and_what_the_network_gains(sem):
    mesh = W.config_box3d(8, 4)
    levels = [6, 3, 1]
    prob, learned = _solver(sem, mesh, levels, mlp_hidden=256, imax=300)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    l0, l1 = learned.train(snapshots=60, steps=6, lr=1e-3, seed=7)
    assert l1 < 0.5 * l0, (l0, l1)
    phi = torch.zeros(lev.N, dtype=torch.float64, device="cuda")
    dD = torch.tensor(phiD, device="cuda")
    learned.solve(dD, phi, tol=1e-10)
    torch.cuda.synchronize()
    t = time.perf_counter()
    st_l = learned.solve(dD, phi, tol=1e-10)
    torch.cuda.synchronize()
    t_l = time.perf_counter() - t
    ref = S.solve_laplace_direct(prob, phiD)
    err = np.abs(phi.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert st_l["status"] == 0 and err < 1e-8
    # every V-cycle judges the network's sweep until a solve has rejected it three times
    # without accepting it once; then the rest of the solve runs the plain cycle
    acc, fb = st_l["learned_accepts"], st_l["learned_fallbacks"]
    if acc == 0:
        assert fb == min(3, st_l["vcycles"]), st_l
    else:
        assert acc + fb == st_l["vcycles"], st_l
    _, plain = _solver(sem, mesh, levels, smoother="chebyshev", imax=300)
    plain.solve(dD, phi, tol=1e-10)
    torch.cuda.synchronize()
    t = time.perf_counter()
    st_p = plain.solve(dD, phi, tol=1e-10)
    torch.cuda.synchronize()
    t_p = time.perf_counter() - t
    print(f"\nlearned sweep: loss {l0:.3e} -> {l1:.3e}; PDC iterations {st_l['iters']} (plain {st_p['iters']}), "
          f"accepted {st_l['learned_accepts']}/{st_l['vcycles']} sweeps, time {t_l * 1e3:.1f} ms "
          f"(plain {t_p * 1e3:.1f} ms), q {st_l['q_mean']:.3f} (plain {st_p['q_mean']:.3f})")
    learned.close()
    plain.close()


def test_trained_sweep_gains_on_a_16x16x4_box(sem):
    # 16 x 16 x 4 prisms at P = 6 (element aspect ratio d_z / d_xy 0.64): trained on 200 snapshots x
    # 20 steps, the network's sweep is accepted at tau = 0.7 and the defect correction needs fewer
    # iterations than the same cycle without it (15 against 20 on a GB300)
    mesh = W.config_box3d(16, 4)
    levels = [6, 3, 1]
    xy = sem.sem_mesh_nodes2d(mesh, 6)
    eta = mesh.eta(xy[:, 0], xy[:, 1])
    its = {}
    for form in ("plain", "learned"):
        o = dict(levels=levels, precision="mixed_fp32", outer="pdc", imax=300)
        if form == "learned":
            o.update(smoother="learned", learned_tau=0.7)
        s = sem.Solver(mesh, 6, eta_nodal=eta, **o)
        try:
            if form == "learned":
                l0, l1 = s.train(200, 20, lr=1e-3, seed=7)
                assert l1 < 0.3 * l0, (l0, l1)
            C = s.coords(0)
            d = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
            phi = torch.zeros(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
            st = s.solve(d, phi, tol=1e-8)
            assert st["status"] == 0 and st["res_final"] <= 1e-8 * st["fnorm"]
            its[form] = (st["iters"], st["learned_accepts"])
        finally:
            s.close()
    print(f"\n16x16x4 box: PDC iterations plain {its['plain'][0]}, with the trained sweep {its['learned'][0]} "
          f"({its['learned'][1]} sweeps accepted)")
    assert its["learned"][0] < its["plain"][0] and its["learned"][1] > 0, its


def test_adam_kernel_matches_the_oracle_over_three_steps(sem):
    # the library's Adam (FP32 masters) against oracle.mlp.adam_step in FP64 from the same
    # FP32 weights and gradients: three steps with different gradients, so the bias
    # corrections and both decay rates matter; a wrong beta moves a weight by ~1e-4 here
    mesh = W.config_box3d(3, 2)
    prob, s = _solver(sem, mesh, [3, 2, 1], mlp_hidden=24)
    npe = prob.levels[0].ref.Np
    rng = np.random.default_rng(23)
    w = {"W1": rng.standard_normal((24, npe)) * 0.3, "b1": rng.standard_normal(24) * 0.1,
         "W2": rng.standard_normal((npe, 24)) * 0.3, "b2": rng.standard_normal(npe) * 0.1}
    w = {k: v.astype(np.float32) for k, v in w.items()}
    s.set_mlp_weights(w["W1"], w["b1"], w["W2"], w["b2"])
    keys = ("W1", "b1", "W2", "b2")
    params = [w[k].astype(np.float64) for k in keys]
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    lr = 1e-2
    for t in range(1, 4):
        g = {k: rng.standard_normal(w[k].shape).astype(np.float32) for k in keys}
        s.adam_step(g, lr, reset=(t == 1))
        M.adam_step(params, [g[k].astype(np.float64) for k in keys], m, v, t=t, lr=lr)
    got = s.mlp_weights()
    for k, ref in zip(keys, params):
        assert np.abs(got[k] - ref).max() <= 1e-6, k
    s.close()


def _sweep_case(sem, hidden, tau, weights_fn):
    mesh = W.config_box3d(3, 2)
    levels = [3, 2, 1]
    prob, s = _solver(sem, mesh, levels, mlp_hidden=hidden, learned_tau=tau)
    lev = prob.levels[0]
    npe = lev.ref.Np
    W1, b1, W2, b2 = weights_fn(npe, hidden)
    s.set_mlp_weights(W1, b1, W2, b2)
    ops = S.MGOperators(prob, k_cheb=5, lo=0.01, hi=1.05)    # the library's default smoother
    f = np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=51)).astype(np.float32)
    u = (0.3 * np.where(lev.dmask, 0.0, W.random_vector(lev.N, seed=52))).astype(np.float32)
    fd = torch.tensor(f, device="cuda")
    ud = torch.tensor(u, device="cuda")
    acc, alpha = s.learned_sweep(fd, ud)
    # the oracle takes the weights the GEMMs read (BF16 copies of W1, W2)
    net = (M.bf16_round(W1), b1.astype(np.float64), M.bf16_round(W2), b2.astype(np.float64))
    ref = L.learned_sweep(ops, net, f.astype(np.float64), u.astype(np.float64), tau)
    s.close()
    return acc, alpha, ud.cpu().numpy().astype(np.float64), ref


# FP32 arithmetic throughout the sweep (apply, Jacobi scaling, network with K <= 2 Np
# accumulations, scatter): each result within a few 1e-6 of the FP64 oracle; 5e-5 is the bound
SWEEP_TOL = 5e-5


def test_learned_sweep_with_an_identity_network_matches_the_oracle(sem):
    def identity(npe, H):
        I = np.eye(npe, dtype=np.float32)
        return (np.vstack([I, -I]), np.zeros(H, np.float32), np.hstack([I, -I]), np.zeros(npe, np.float32))
    acc, alpha, u, ref = _sweep_case(sem, 80, 1.0, identity)
    assert ref.accepted and acc
    assert abs(alpha - ref.alpha) <= SWEEP_TOL * ref.alpha
    assert np.abs(u - ref.u).max() <= SWEEP_TOL * np.abs(ref.u).max()


@pytest.mark.parametrize("tau", [1.0, 0.05])
def test_learned_sweep_with_a_random_network_matches_the_oracle(sem, tau):
    def rand(npe, H):
        rng = np.random.default_rng(61)
        return ((rng.standard_normal((H, npe)) * 0.2).astype(np.float32), (rng.standard_normal(H) * 0.05).astype(np.float32),
                (rng.standard_normal((npe, H)) * 0.2).astype(np.float32), (rng.standard_normal(npe) * 0.05).astype(np.float32))
    acc, alpha, u, ref = _sweep_case(sem, 32, tau, rand)
    # the verdict is compared where the oracle's margin from the threshold exceeds the FP32 error
    margin = abs(ref.rr_after - tau * tau * ref.rr) / ref.rr
    if margin > 1e-3:
        assert acc == ref.accepted
    if acc == ref.accepted:
        assert abs(alpha - ref.alpha) <= SWEEP_TOL * max(abs(ref.alpha), 1e-30)
        assert np.abs(u - ref.u).max() <= SWEEP_TOL * np.abs(ref.u).max()
    if tau == 0.05:
        assert not ref.accepted          # the Chebyshev fallback path
