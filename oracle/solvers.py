"""Solvers of the oracle: Dirichlet lifting, direct solve, p-transfers, Chebyshev
smoothing, the p-multigrid V-cycle (Algorithm 1), PDC (Algorithm 2), PCG
(Algorithm 3) and right-preconditioned flexible GMRES.

Vectors are full length N (all global nodes of a level) with zeros at the
Dirichlet nodes: the free-node system A_FF u_F = f_F is solved in place.

Readings of the paper used here (the CUDA library follows the same ones):
* Algorithm 1 at the level just above the coarsest restricts and solves
  directly on the coarsest level (order 1); the residual uses the current
  iterate u_{h,p}.
* Algorithm 2 forms the residual before testing it; MultigridCycle(-r) followed
  by u <- u - delta is the same as u <- u + M^{-1} r.
* Algorithm 3's "q <- A delta" is q <- A p (delta is a scalar).
* Stop test ||r||_2 <= rtol ||f||_2 + atol on the unpreconditioned free residual.
* Smoother: the paper's overlapping additive Schwarz (smoother="asm", the readings
  in oracle/schwarz.py), or Chebyshev
  iteration of degree k on D^{-1} A (D = diagonal of A) for the interval
  [lo*b, b], b = hi * lambda_hat.  lambda_hat is the largest Ritz value of
  30 Lanczos steps on D^{-1/2} A D^{-1/2} (free nodes) started from D^{-1/2} x0,
  x0_i = sin(i + 1): a lower bound of lambda_max that converges far faster than
  the power iteration (which stayed 16-22 % below lambda_max after 20 steps on
  some sigma-prism meshes, enough for the smoother to amplify the top modes).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import Problem
from .refelem import interpolation_matrix


# ----------------------------------------------------------------- boundary data
def lift(prob: Problem, phi_dirichlet: np.ndarray, rhs: np.ndarray | None = None, li: int = 0):
    """Right-hand side of the free system: f_F = rhs_F - A_FD phi_D (Eq. laplaceproblem:
    phi = phi~ on the free surface), zeros at the Dirichlet nodes."""
    lev = prob.levels[li]
    A = prob.stiffness(li)
    uD = np.zeros(lev.N)
    uD[lev.dirichlet] = phi_dirichlet
    f = -(A @ uD)
    if rhs is not None:
        f = f + rhs
    f[lev.dirichlet] = 0.0
    return f


def direct_solve(prob: Problem, f: np.ndarray, li: int = 0) -> np.ndarray:
    """Exact solution of A_FF u_F = f_F by sparse LU (SuperLU) plus one step of
    iterative refinement; zeros at the Dirichlet nodes."""
    lev = prob.levels[li]
    AFF = prob.free_matrix(li).tocsc()
    lu = spla.splu(AFF, permc_spec="MMD_AT_PLUS_A")
    ff = f[lev.free]
    u = lu.solve(ff)
    u = u + lu.solve(ff - AFF @ u)
    out = np.zeros(lev.N)
    out[lev.free] = u
    return out


def solve_laplace_direct(prob: Problem, phi_dirichlet: np.ndarray, rhs=None) -> np.ndarray:
    """phi on all nodes of the finest level: phi_D = phi~, phi_F from the direct solve."""
    lev = prob.levels[0]
    f = lift(prob, phi_dirichlet, rhs)
    u = direct_solve(prob, f)
    u[lev.dirichlet] = phi_dirichlet
    return u


# ----------------------------------------------------------------- operators
class MGOperators:
    """Matrices of every level for the free-node system (Dirichlet rows/cols zeroed)."""

    def __init__(self, prob: Problem, nu1=1, nu2=1, k_cheb=3, lo=0.25, hi=1.1,
                 lanczos_steps=30, lambdas=None, smoother="chebyshev", overlap=1):
        self.prob = prob
        self.smoother = smoother
        self.L = len(prob.levels)
        self.nu1, self.nu2, self.k = nu1, nu2, k_cheb
        self.lo, self.hi = lo, hi
        self.A = []
        self.Dinv = []
        for li, lev in enumerate(prob.levels):
            A = prob.stiffness(li)
            keep = sp.diags((~lev.dmask).astype(np.float64))
            Am = (keep @ A @ keep).tocsr()
            self.A.append(Am)
            d = A.diagonal()
            dinv = np.where(lev.dmask, 0.0, 1.0 / np.where(lev.dmask, 1.0, d))
            self.Dinv.append(dinv)
        self.P = [prolongation(prob, li) for li in range(self.L - 1)]
        self.lam = []
        self.asm = []
        if smoother == "asm":
            # the overlapping additive Schwarz smoother of Section 4.3 (oracle/schwarz.py)
            from .schwarz import Schwarz
            self.asm = [Schwarz(prob, li, self.A[li], overlap) for li in range(self.L - 1)]
            lambdas = [float("nan")] * (self.L - 1)
        elif smoother != "chebyshev":
            raise ValueError("smoother: chebyshev or asm")
        for li in range(self.L - 1):
            lam = lanczos_lambda(self.A[li], self.Dinv[li], prob.levels[li].dmask, lanczos_steps) \
                if lambdas is None else lambdas[li]
            self.lam.append(lam)
        c = prob.levels[-1]
        self._coarse = spla.splu(prob.free_matrix(self.L - 1).tocsc(), permc_spec="MMD_AT_PLUS_A")
        self._cfree = c.free
        self.fine_applies = 0

    def apply(self, li, x):
        if li == 0:
            self.fine_applies += 1
        return self.A[li] @ x

    def coarse_solve(self, f):
        out = np.zeros_like(f)
        out[self._cfree] = self._coarse.solve(f[self._cfree])
        return out

    def smooth(self, li, f, x, post=False):
        if self.asm:
            return self.asm[li].smooth(self.A[li], f, x, adjoint=post)
        b = self.hi * self.lam[li]
        a = self.lo * b
        return chebyshev(lambda v: self.apply(li, v), self.Dinv[li], f, x, self.k, a, b)

    def vcycle(self, f):
        """Algorithm 1 with u = 0 on entry at every level: z = M^{-1} f."""
        L = self.L
        fs = [None] * L
        us = [None] * L
        fs[0] = f
        for li in range(L - 1):
            u = np.zeros_like(fs[li])
            for _ in range(self.nu1):
                u = self.smooth(li, fs[li], u)
            r = fs[li] - self.apply(li, u)
            fs[li + 1] = self.P[li].T @ r
            us[li] = u
        us[L - 1] = self.coarse_solve(fs[L - 1])
        for li in range(L - 2, -1, -1):
            us[li] = us[li] + self.P[li] @ us[li + 1]
            for _ in range(self.nu2):
                us[li] = self.smooth(li, fs[li], us[li], post=True)
        return us[0]


def prolongation(prob: Problem, li: int) -> sp.csr_matrix:
    """Global prolongation P from level li+1 (coarse) to level li (fine), free nodes only.

    P[i, J] = value of the coarse basis function J at fine node i (Section 4.1,
    nested spaces), taken from any element that contains node i."""
    fine, coarse = prob.levels[li], prob.levels[li + 1]
    I = interpolation_matrix(prob.dim, fine.p, coarse.p, fine.pz, coarse.pz)   # [Np_f, Np_c]
    done = np.zeros(fine.N, dtype=bool)
    rows, cols, vals = [], [], []
    for e in range(fine.emap.shape[0]):
        for l, i in enumerate(fine.emap[e]):
            if done[i] or fine.dmask[i]:
                continue
            done[i] = True
            for c, J in enumerate(coarse.emap[e]):
                if coarse.dmask[J] or I[l, c] == 0.0:
                    continue
                rows.append(i)
                cols.append(J)
                vals.append(I[l, c])
    P = sp.coo_matrix((vals, (rows, cols)), shape=(fine.N, coarse.N)).tocsr()
    P.sum_duplicates()
    return P


def lanczos_lambda(A, Dinv, dmask, steps=30) -> float:
    """Largest eigenvalue estimate of D^{-1} A: the largest eigenvalue of the
    tridiagonal matrix T_k of k = ``steps`` Lanczos steps (no reorthogonalisation)
    on the symmetric B = D^{-1/2} A_FF D^{-1/2}, started from v0 = D^{-1/2} x0 / ||.||
    with x0_i = sin(i + 1) on the free nodes (Lanczos, e.g. Saad, Iterative
    Methods for Sparse Linear Systems, Sec. 6.6).  Stops early when the Krylov
    space is exhausted (beta_j = 0), where T_j is exact."""
    free = ~np.asarray(dmask, dtype=bool)
    n = A.shape[0]
    x0 = np.sin(np.arange(n) + 1.0)[free]
    s = np.sqrt(Dinv[free])                     # D^{-1/2}
    Aff = A[free][:, free]
    v = s * x0
    v = v / np.linalg.norm(v)
    v_prev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = s * (Aff @ (s * v)) - beta * v_prev
        a = float(w @ v)
        w = w - a * v
        alphas.append(a)
        beta = float(np.linalg.norm(w))
        if beta <= 1e-14 * abs(a):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    k = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    return float(np.linalg.eigvalsh(T).max())


def chebyshev(apply, Dinv, f, x, k, a, b):
    """k steps of the Chebyshev iteration for A x = f preconditioned by D^{-1} on the
    eigenvalue interval [a, b] (three-term recurrence of the scaled Chebyshev
    polynomials, e.g. Saad, Iterative Methods for Sparse Linear Systems, Sec. 12.1).
    The residual is recomputed as f - A x at every step."""
    theta = 0.5 * (b + a)
    delta = 0.5 * (b - a)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = f - apply(x)
    d = Dinv * r / theta
    x = x + d
    for _ in range(1, k):
        r = f - apply(x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * r)
        x = x + d
        rho = rho_new
    return x


# ----------------------------------------------------------------- outer iterations
class Result:
    def __init__(self, u, iters, resids, fnorm):
        self.u = u
        self.iters = iters
        self.resids = resids
        self.fnorm = fnorm


def pcg(ops: MGOperators, f, rtol=1e-8, atol=0.0, imax=200, u0=None):
    """Algorithm 3 (PCG-pMG) on the free system."""
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    r = f - ops.apply(0, u)
    z = ops.vcycle(r)
    p = z.copy()
    delta = z @ r
    res = [np.linalg.norm(r)]
    i = 0
    while i < imax and res[-1] > rtol * fn + atol:
        q = ops.apply(0, p)
        alpha = delta / (p @ q)
        u = u + alpha * p
        r = r - alpha * q
        z = ops.vcycle(r)
        dnew = z @ r
        beta = dnew / delta
        p = z + beta * p
        delta = dnew
        i += 1
        res.append(np.linalg.norm(r))
    return Result(u, i, res, fn)


def pdc(ops: MGOperators, f, rtol=1e-8, atol=0.0, imax=200, u0=None):
    """Algorithm 2 (PDC-pMG): residual, test, u <- u + MultigridCycle(r)."""
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    res = []
    i = 0
    while True:
        r = f - ops.apply(0, u)
        res.append(np.linalg.norm(r))
        if i >= imax or res[-1] <= rtol * fn + atol:
            break
        u = u + ops.vcycle(r)
        i += 1
    return Result(u, i, res, fn)


def fgmres(ops: MGOperators, f, rtol=1e-8, atol=0.0, imax=200, m=30, u0=None):
    """Right-preconditioned flexible GMRES(m) with modified Gram-Schmidt and Givens
    rotations (Saad, Sec. 9.4.1); preconditioner = one V-cycle."""
    u = np.zeros_like(f) if u0 is None else u0.copy()
    fn = np.linalg.norm(f)
    tol = rtol * fn + atol
    r = f - ops.apply(0, u)
    beta = np.linalg.norm(r)
    res = [beta]
    it = 0
    while it < imax and beta > tol:
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j = 0
        while j < m and it < imax:
            z = ops.vcycle(V[j])
            Z.append(z)
            w = ops.apply(0, z)
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            it += 1
            res.append(abs(g[j]))
            if abs(g[j]) <= tol:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        for i in range(j):
            u = u + y[i] * Z[i]
        r = f - ops.apply(0, u)
        beta = np.linalg.norm(r)
        res[-1] = beta
    return Result(u, it, res, fn)
