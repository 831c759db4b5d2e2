"""What an element-local correction can do after the coarse-grid correction (the role of the
learned sweep, which replaces the first finest-level post-smoothing sweep), computed with the
oracle on a small P = 6 box: the least-squares-best linear map shared by all elements, from the
scaled element residual d_e / s_e (d = D^{-1} r, s_e = ||d_e||) to the scaled error e_e / s_e,
fitted on the post-coarse-correction states of the plain iteration, taken with the
minimal-residual step, cuts the residual several times more than the Chebyshev sweep it
replaces on held-out states.  This is the bound the correction network is trained towards."""
import numpy as np

import workloads as W
from oracle import solvers as S
from oracle.assemble import Problem


def test_element_local_map_bound_after_coarse_correction():
    mesh = W.config_box3d(4, 4)
    prob = Problem(mesh, [6, 3, 1])
    lev = prob.levels[0]
    ops = S.MGOperators(prob, k_cheb=5, lo=0.01, hi=1.05)
    A, Dinv, emap = ops.A[0], ops.Dinv[0], lev.emap
    free = ~lev.dmask
    mult = np.bincount(emap.ravel(), minlength=lev.N).astype(float)
    wm = np.where(mult > 0, 1.0 / np.maximum(mult, 1.0), 0.0)
    rng = np.random.default_rng(3)
    u_star = np.zeros(lev.N)
    u_star[free] = rng.standard_normal(free.sum())
    f = A @ u_star

    def after_coarse_correction(u):
        u = ops.smooth(0, f, u)
        fc = ops.P[0].T @ (f - A @ u)
        u1 = ops.smooth(1, fc, np.zeros_like(fc))
        u1 = u1 + ops.P[1] @ ops.coarse_solve(ops.P[1].T @ (fc - ops.A[1] @ u1))
        u1 = ops.smooth(1, fc, u1, post=True)
        return u + ops.P[0] @ u1

    def scaled(u):
        r = f - A @ u
        X = (Dinv * r)[emap]
        s = np.linalg.norm(X, axis=1, keepdims=True)
        s[s == 0] = 1.0
        return X / s, (u_star - u)[emap] / s, s, r

    Xs, Ts = [], []
    for k in range(4):
        u = np.zeros(lev.N)
        u[free] = 0.3 * (k + 1) * rng.standard_normal(free.sum())
        for _ in range(2):
            uc = after_coarse_correction(u)
            X, T, _, _ = scaled(uc)
            Xs.append(X)
            Ts.append(T)
            u = ops.smooth(0, f, uc, post=True)
    M, *_ = np.linalg.lstsq(np.concatenate(Xs), np.concatenate(Ts), rcond=None)

    u = np.zeros(lev.N)
    u[free] = rng.standard_normal(free.sum())
    uc = after_coarse_correction(u)
    X, _, s, r = scaled(uc)
    rn = np.linalg.norm(r)
    cheb = np.linalg.norm(f - A @ ops.smooth(0, f, uc, post=True)) / rn
    delta = np.zeros(lev.N)
    np.add.at(delta, emap.ravel(), ((X @ M) * s).ravel())
    delta *= wm
    delta[~free] = 0.0
    q = A @ delta
    local = np.linalg.norm(r - (r @ q) / (q @ q) * q) / rn
    print(f"\nresidual factor after the coarse-grid correction: Chebyshev k = 5 {cheb:.3f}, "
          f"best shared linear element map + minimal-residual step {local:.3f}")
    assert 0.0 < local < 0.5 * cheb < 1.0
