"""Oracle of the free-surface time stepping around the Laplace solve (test
infrastructure: plain CPU FP64, imported only by tests and the benchmark's CPU
baseline).

Section 2: the surface elevation eta and the surface potential phi~ evolve by the
kinematic and dynamic conditions (Eqs. FSeta, FSphi)

    d eta/dt  = -grad eta . grad phi~ + w~ (1 + grad eta . grad eta)
    d phi~/dt = -g eta - (grad phi~ . grad phi~ - w~^2 (1 + grad eta . grad eta)) / 2

where w~ is the vertical velocity d phi/dz at the surface of the solution of the
Laplace problem (Eq. laplaceproblem) with phi = phi~ on z = eta; the small-amplitude
version keeps the domain flat (z <= 0) and reads d eta/dt = w~, d phi~/dt = -g eta.
The benchmarks integrate in time with the classical four-stage explicit Runge-Kutta
method (ERK4).

Readings: the fields live at the order-P 2D nodes of the surface; horizontal
gradients of a surface field are those of its order-P interpolant on each base
triangle at the triangle's nodes, averaged over the triangles sharing a node; w~ is
the vertical derivative of the discrete solution along the node's vertical line
(the same in every element of the column), dphi/dz = (dphi/dt) / (dz/dt) with
dz/dt = (h + eta) / (2 N_layers) in the top sigma layer.
"""
from __future__ import annotations

import numpy as np

from . import solvers as S
from .assemble import Problem
from .refelem import RefTri, gll, lagrange1d, tri_basis


def surface_gradient(prob: Problem, f2: np.ndarray):
    """(df/dx, df/dy) at the order-P 2D nodes of a field f2 given at those nodes."""
    lev, mesh = prob.levels[0], prob.mesh
    tn = RefTri(lev.p).nodes
    _, Dr, Ds = tri_basis(lev.p, tn)              # derivatives of the basis at its own nodes
    gx = np.zeros(lev.N2)
    gy = np.zeros(lev.N2)
    cnt = np.zeros(lev.N2)
    for b in range(mesh.tri.shape[0]):
        v = mesh.vxy[mesh.tri[b]]
        # x = -(r+s)/2 v0 + (1+r)/2 v1 + (1+s)/2 v2:  [[x_r, x_s], [y_r, y_s]]
        J = 0.5 * np.array([[v[1, 0] - v[0, 0], v[2, 0] - v[0, 0]],
                            [v[1, 1] - v[0, 1], v[2, 1] - v[0, 1]]])
        Ji = np.linalg.inv(J)                       # [[r_x, r_y], [s_x, s_y]]
        ids = lev.map2[b]
        fr, fs = Dr @ f2[ids], Ds @ f2[ids]
        gx[ids] += Ji[0, 0] * fr + Ji[1, 0] * fs
        gy[ids] += Ji[0, 1] * fr + Ji[1, 1] * fs
        cnt[ids] += 1.0
    return gx / cnt, gy / cnt


def surface_w(prob: Problem, phi: np.ndarray, eta2: np.ndarray) -> np.ndarray:
    """d phi/dz at the surface nodes from phi on all nodes of the finest level; eta2 is the
    surface elevation the geometry was built with (zeros for the flat domain)."""
    lev, mesh = prob.levels[0], prob.mesh
    pz, nl, N2 = lev.pz, mesh.nlayers, lev.N2
    _, D = lagrange1d(gll(pz), np.array([1.0]))     # h_k'(+1) of the vertical GLL basis
    phit = np.zeros(N2)
    for k in range(pz + 1):
        kz = (nl - 1) * pz + k
        phit += D[0, k] * phi[kz * N2:(kz + 1) * N2]
    return phit / ((mesh.depth + eta2) / (2.0 * nl))


def _surface_problem(mesh, levels, eta2):
    prob = Problem(mesh, levels, eta_nodal=eta2)
    lev = prob.levels[0]
    top = (mesh.nlayers * lev.pz) * lev.N2 + np.arange(lev.N2)
    if not np.array_equal(lev.dirichlet, top):
        raise ValueError("the free-surface fields need the surface nodes to be exactly the Dirichlet nodes")
    return prob


def fnpf_rhs(mesh, levels, eta: np.ndarray, phis: np.ndarray, g: float = 9.81, linear: bool = False):
    """(d eta/dt, d phi~/dt) at the order-P surface nodes (Eqs. FSeta, FSphi or their
    small-amplitude version), from a direct solve of the Laplace problem."""
    eta2 = np.zeros_like(eta) if linear else np.asarray(eta, dtype=np.float64)
    prob = _surface_problem(mesh, levels, eta2)
    phi = S.solve_laplace_direct(prob, phis)
    w = surface_w(prob, phi, eta2)
    if linear:
        return w, -g * eta
    ex, ey = surface_gradient(prob, eta)
    px, py = surface_gradient(prob, phis)
    gg = 1.0 + ex * ex + ey * ey
    deta = -(ex * px + ey * py) + w * gg
    dphi = -g * eta - 0.5 * (px * px + py * py - w * w * gg)
    return deta, dphi


def erk4_step(mesh, levels, eta, phis, dt: float, g: float = 9.81, linear: bool = False):
    """One step of the classical four-stage Runge-Kutta method for (eta, phi~)."""
    k1 = fnpf_rhs(mesh, levels, eta, phis, g, linear)
    k2 = fnpf_rhs(mesh, levels, eta + 0.5 * dt * k1[0], phis + 0.5 * dt * k1[1], g, linear)
    k3 = fnpf_rhs(mesh, levels, eta + 0.5 * dt * k2[0], phis + 0.5 * dt * k2[1], g, linear)
    k4 = fnpf_rhs(mesh, levels, eta + dt * k3[0], phis + dt * k3[1], g, linear)
    eta_n = eta + dt / 6.0 * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0])
    phis_n = phis + dt / 6.0 * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1])
    return eta_n, phis_n
