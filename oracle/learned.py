"""FP64 oracle of the learned correction sweep.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports or calls this module.

The paper has no learned component.  Its nearest counterpart is the weighted
element-block Schwarz correction of Section 4.3 (Eqs. Mass and weights): local
corrections computed on element patches from the local residual, scaled by the
weight W and summed into the global correction.  The learned sweep keeps that
shape and replaces the local solve by a small network applied to each
element's Jacobi-scaled residual.  One sweep, in order:

1. residual r = f - A u on the free nodes (A the masked operator of the level,
   zero at the Dirichlet nodes);
2. Jacobi scaling z = D^{-1} r, D the diagonal of the assembled matrix;
3. per element e: z_e = Q_e z (its nodal values), s_e = ||z_e||_2 (1 when
   z_e = 0), network input x_e = z_e / s_e;
4. y_e = MLP(x_e) (oracle.mlp.forward);
5. delta = W sum_e Q_e^T s_e y_e on the free nodes, W = diag(1 / number of
   elements holding the node), the element-level weight of the Schwarz sum;
6. q = A delta and the step alpha = (r, q) / (q, q) that minimises
   ||r - alpha q||_2;
7. verdict: the step is kept when alpha > 0 and ||r - alpha q||^2 < tau^2 ||r||^2
   (u <- u + alpha delta); otherwise the Chebyshev sweep that the learned sweep
   replaces runs instead (oracle.solvers.chebyshev).

Pins: tests/test_oracle_learned.py (an identity network turns the sweep into a
minimal-residual Jacobi step, positive homogeneity of the sweep in (f, u), the
minimal-residual property of alpha, the rejection paths).
"""
from __future__ import annotations

import numpy as np

from . import mlp as M
from .solvers import MGOperators, chebyshev


class SweepResult:
    def __init__(self, u, delta, alpha, accepted, rr, rr_after):
        self.u = u                  # iterate after the sweep (u + alpha delta, or the Chebyshev sweep)
        self.delta = delta          # network correction (step 5)
        self.alpha = alpha          # minimal-residual step (0 when rejected)
        self.accepted = accepted
        self.rr = rr                # ||r||^2 before
        self.rr_after = rr_after    # ||r - alpha_mr q||^2 at the minimising alpha (step 7's test value)


def element_weights(emap: np.ndarray, N: int) -> np.ndarray:
    """W_g = 1 / (number of elements whose node list holds g)."""
    count = np.bincount(emap.ravel(), minlength=N).astype(np.float64)
    return np.where(count > 0, 1.0 / np.where(count > 0, count, 1.0), 0.0)


def network_correction(ops: MGOperators, weights, r: np.ndarray) -> np.ndarray:
    """Steps 2-5: delta = W sum_e Q_e^T s_e MLP(Q_e D^{-1} r / s_e) on the free nodes."""
    lev = ops.prob.levels[0]
    emap, dmask = lev.emap, lev.dmask
    z = ops.Dinv[0] * r
    Z = np.where(dmask[emap], 0.0, z[emap])                # [E, Np], zero at Dirichlet nodes
    s = np.sqrt(np.sum(Z * Z, axis=1))
    s = np.where(s > 0.0, s, 1.0)
    _, _, Y = M.forward(*weights, Z / s[:, None])
    w = element_weights(emap, lev.N)
    delta = np.zeros(lev.N)
    np.add.at(delta, emap.ravel(), (s[:, None] * Y).ravel())
    delta *= w
    delta[dmask] = 0.0
    return delta


def learned_sweep(ops: MGOperators, weights, f: np.ndarray, u: np.ndarray, tau: float) -> SweepResult:
    """One learned sweep on the finest level of ``ops`` (steps 1-7 above).  ``weights`` =
    (W1, b1, W2, b2) in the library's layout (W1 [H][Np], W2 [Np][H])."""
    r = f - ops.A[0] @ u
    rr = float(r @ r)
    delta = network_correction(ops, weights, r)
    q = ops.A[0] @ delta
    rq, qq = float(r @ q), float(q @ q)
    a = rq / qq if qq > 0.0 else 0.0
    after = rr - a * rq
    accepted = bool(a > 0.0 and np.isfinite(a) and after < tau * tau * rr)
    if accepted:
        return SweepResult(u + a * delta, delta, a, True, rr, after)
    b = ops.hi * ops.lam[0]
    un = chebyshev(lambda v: ops.A[0] @ v, ops.Dinv[0], f, u, ops.k, ops.lo * b, b)
    return SweepResult(un, delta, 0.0, False, rr, after)
