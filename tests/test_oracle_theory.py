"""Pins of the linear-theory oracle (Eq. (LT), Sec. 2) against what the paper
and the mathematics fix: the printed coefficients, the steady-shear closed form
(S -> R^2 (I + (35/8) tau_sigma E) at chi = 1, beta -> 1/sqrt(2)), that the
exponential solves the ODE, the semigroup property, the trace for a traceless
gradient, the relaxation rate, and an independent adaptive ODE solver."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou


def test_coefficients(golden):
    g = golden["linear_theory_chi1"]["value"]
    c_r, c_s = O.lt_coefficients(1.0)
    assert abs(c_r - g["relax_coeff"]) < 1e-15 and abs(c_s - g["strain_coeff"]) < 1e-15
    # inviscid droplet chi = 0: 40/(3*16), 5/3; rigid limit chi -> inf: both -> 0
    c_r0, c_s0 = O.lt_coefficients(0.0)
    assert abs(c_r0 - 40 / 48) < 1e-15 and abs(c_s0 - 5 / 3) < 1e-15
    c_rb, c_sb = O.lt_coefficients(1e9)
    assert c_rb < 2e-9 and c_sb < 3e-9


def test_steady_shear_closed_form(golden):
    """Simple shear of rate g at chi = 1 from a sphere: lambda_max/R^2 ->
    1 + (35/16) Ca, D -> (35/32) Ca to first order, beta -> 1/sqrt(2)."""
    R, tau, g = 7.0, 900.0, 1e-5
    A = np.zeros((3, 3))
    A[0, 2] = g
    Ca = tau * g
    S = O.lt_trajectory(np.repeat(A[None], 200, axis=0), 1000.0, tau, R, 1.0)[-1]
    ob = O.lt_observables(S, A, R)
    assert abs(ob["lam_max_R2"] - (1 + 35 / 16 * Ca)) < 1e-12
    assert abs(ob["beta"] - golden["beta_steady_shear"]["value"]) < 1e-12
    assert abs(ob["D"] - 35 / 32 * Ca) < 2 * Ca * Ca


def test_exponential_solves_the_ode():
    """Central difference of S(t) against the right-hand side of Eq. (LT)."""
    rng = np.random.default_rng(3)
    for chi in (0.0, 1.0, 4.0):
        c_r, c_s = O.lt_coefficients(chi)
        R, tau = 5.0, 300.0
        E = O.strain(rng.standard_normal((3, 3)) * 1e-3)
        S0 = R * R * np.eye(3) + np.diag([0.3, -0.1, -0.2])
        for t in (10.0, 250.0, 900.0):
            h = 1e-3
            dS = (O.lt_propagate(S0, E, t + h, tau, R, chi) - O.lt_propagate(S0, E, t - h, tau, R, chi)) / (2 * h)
            S = O.lt_propagate(S0, E, t, tau, R, chi)
            rhs = -(c_r / tau) * (S - R * R * np.eye(3)) + 2 * R * R * c_s * E
            assert np.abs(dS - rhs).max() < 1e-9 * max(1.0, np.abs(rhs).max()) + 1e-12


def test_semigroup_trace_and_relaxation():
    R, tau = 6.0, 500.0
    rng = np.random.default_rng(4)
    E = O.strain(rng.standard_normal((3, 3)) * 2e-3)
    E -= np.trace(E) / 3 * np.eye(3)
    S0 = R * R * np.eye(3)
    a = O.lt_propagate(O.lt_propagate(S0, E, 120.0, tau, R, 1.0), E, 380.0, tau, R, 1.0)
    b = O.lt_propagate(S0, E, 500.0, tau, R, 1.0)
    assert np.abs(a - b).max() < 1e-12 * R * R
    assert abs(np.trace(b) - 3 * R * R) < 1e-12 * R * R
    # no flow: a deformed droplet relaxes to the sphere at rate (16/35)/tau
    Sd = R * R * np.eye(3) + np.diag([1.0, -0.5, -0.5])
    Z = np.zeros((3, 3))
    s1 = O.lt_propagate(Sd, Z, 700.0, tau, R, 1.0)
    assert abs((s1[0, 0] - R * R) - np.exp(-16 / 35 * 700.0 / tau)) < 1e-13


def test_trajectory_against_adaptive_solver():
    """A held OU gradient sequence: the exact propagation against scipy's
    adaptive Runge-Kutta (DOP853) integrating Eq. (LT) frame by frame."""
    integrate = pytest.importorskip("scipy.integrate")
    fr = frames_ou(12, 6, 3e-3).reshape(6, 3, 3)
    R, tau, hold, chi = 5.0, 400.0, 150.0, 1.0
    c_r, c_s = O.lt_coefficients(chi)
    ref = O.lt_trajectory(fr, hold, tau, R, chi)
    y = (R * R * np.eye(3)).ravel()
    for k in range(6):
        E = O.strain(fr[k])

        def f(t, y):
            S = y.reshape(3, 3)
            return (-(c_r / tau) * (S - R * R * np.eye(3)) + 2 * R * R * c_s * E).ravel()

        sol = integrate.solve_ivp(f, (0.0, hold), y, method="DOP853", rtol=1e-12, atol=1e-12)
        y = sol.y[:, -1]
        assert np.abs(y.reshape(3, 3) - ref[k]).max() < 1e-9 * R * R
