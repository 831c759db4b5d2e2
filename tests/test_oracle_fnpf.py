"""Pins of the free-surface time-stepping oracle (Section 2, Eqs. FSeta, FSphi):
exact surface gradients of polynomials, the exact vertical derivative of a field
polynomial in z, the linear standing wave against its closed form
(eta = a cos(kx) cos(omega t), omega^2 = g k tanh(k h)), and the nonlinear
equations reducing to the linear ones at small amplitude."""
import math

import numpy as np

import workloads as W
from oracle import fnpf as F
from oracle.assemble import Problem


def test_surface_gradient_is_exact_for_polynomials_of_degree_p():
    mesh = W.box3d(3, 2, 2, eta_modes=W.eta_sinx_cosy(0.1))
    prob = Problem(mesh, [4, 1])
    C = prob.coords(0)[: prob.levels[0].N2, :2]          # the 2D nodes (bottom layer)
    x, y = C[:, 0], C[:, 1]
    f = x * x * y - 3 * x * y + 2 + y ** 3 - 0.5 * x ** 4
    gx, gy = F.surface_gradient(prob, f)
    assert np.abs(gx - (2 * x * y - 3 * y - 2 * x ** 3)).max() < 1e-11
    assert np.abs(gy - (x * x - 3 * x + 3 * y * y)).max() < 1e-11


def test_surface_w_is_exact_for_a_field_cubic_in_z():
    mesh = W.box3d(3, 2, 3, eta_modes=W.eta_sinx_cosy(0.1))
    prob = Problem(mesh, [4, 1])
    C = prob.coords(0)
    phi = C[:, 2] ** 3 + 2 * C[:, 2] + C[:, 0]           # cubic along every vertical line
    w = F.surface_w(prob, phi, prob.eta_nodal)
    eta = prob.eta_nodal
    assert np.abs(w - (3 * eta ** 2 + 2)).max() < 1e-11


def _standing_wave(a, steps, T_frac, linear):
    mesh = W.box3d(6, 2, 2)
    levels = [6, 3, 1]
    prob = Problem(mesh, levels, eta_nodal=np.zeros(Problem(mesh, [6, 1]).levels[0].N2))
    x = prob.coords(0)[: prob.levels[0].N2, 0]
    g, k, h = 9.81, 1.0, 1.0
    omega = math.sqrt(g * k * math.tanh(k * h))
    dt = T_frac * 2 * math.pi / omega / steps
    eta, phis = a * np.cos(x), np.zeros_like(x)
    for _ in range(steps):
        eta, phis = F.erk4_step(mesh, levels, eta, phis, dt, g, linear)
    return x, eta, phis, omega, dt * steps


def test_linear_standing_wave_reverses_after_half_a_period():
    a = 1e-2
    x, eta, phis, omega, t = _standing_wave(a, 20, 0.5, True)
    # eta = a cos(x) cos(omega t) = -a cos(x) at t = T/2; phi~ = -(a g / omega) cos(x) sin(omega t) = 0
    assert np.abs(eta + a * np.cos(x)).max() < 1e-4 * a
    assert np.abs(phis).max() < 1e-3 * a * 9.81 / omega


def test_nonlinear_equations_reduce_to_the_linear_ones_at_small_amplitude():
    a = 1e-5
    _, e_lin, p_lin, _, _ = _standing_wave(a, 3, 0.1, True)
    _, e_nl, p_nl, _, _ = _standing_wave(a, 3, 0.1, False)
    # the nonlinear terms and the moving domain change the result at O(a^2)
    assert np.abs(e_nl - e_lin).max() < 1e-3 * a
    assert np.abs(p_nl - p_lin).max() < 1e-3 * np.abs(p_lin).max()
    assert np.abs(e_nl - e_lin).max() > 0.0
