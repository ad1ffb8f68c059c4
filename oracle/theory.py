"""Oracle of the linear theory of Eq. (LT) (Sec. 2) along a sequence of
velocity-gradient frames, each held for a fixed time (Sec. 3.2).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

Eq. (LT) reads dS/dt = -(c_r / tau_sigma) (S - R^2 I) + 2 R^2 c_s E(t) with
c_r = 40(chi+1)/((2chi+3)(19chi+16)) and c_s = 5/(2chi+3), E the symmetric
part of the gradient.  With E constant over a frame this is a linear ODE with
constant coefficients, so its solution over a frame of length h is the plain
exponential

    S(t + h) = S_inf + (S(t) - S_inf) exp(-c_r h / tau_sigma),
    S_inf    = R^2 I + (2 R^2 c_s tau_sigma / c_r) E,

which is what this module evaluates (no time stepping).  The droplet starts
spherical, S(0) = R^2 I.  Observables follow Sec. 2: lambda_max of S (numpy
``eigh``), D from the extreme eigenvalues, and beta of Eq. (beta) with the E of
the frame in force.
"""
from __future__ import annotations

import numpy as np


def lt_coefficients(chi: float):
    """(c_r, c_s) of Eq. (LT) for viscosity ratio chi."""
    c_r = 40.0 * (chi + 1.0) / ((2.0 * chi + 3.0) * (19.0 * chi + 16.0))
    c_s = 5.0 / (2.0 * chi + 3.0)
    return c_r, c_s


def strain(A) -> np.ndarray:
    """E = (grad u + grad u^T)/2 of a frame A[a, b] = du_a/dx_b."""
    A = np.asarray(A, dtype=np.float64).reshape(3, 3)
    return 0.5 * (A + A.T)


def lt_propagate(S, E, h: float, tau_sigma: float, R: float, chi: float) -> np.ndarray:
    """S after a time h under constant strain E (exact solution of Eq. (LT))."""
    c_r, c_s = lt_coefficients(chi)
    S_inf = R * R * np.eye(3) + (2.0 * R * R * c_s * tau_sigma / c_r) * np.asarray(E, dtype=np.float64)
    return S_inf + (np.asarray(S, dtype=np.float64) - S_inf) * np.exp(-c_r * h / tau_sigma)


def lt_trajectory(frames, hold: float, tau_sigma: float, R: float, chi: float = 1.0, S0=None) -> np.ndarray:
    """S at the end of every frame (n_frames, 3, 3); frame k acts for `hold`."""
    fr = np.asarray(frames, dtype=np.float64).reshape(-1, 3, 3)
    S = R * R * np.eye(3) if S0 is None else np.asarray(S0, dtype=np.float64)
    out = np.zeros((fr.shape[0], 3, 3))
    for k in range(fr.shape[0]):
        S = lt_propagate(S, strain(fr[k]), hold, tau_sigma, R, chi)
        out[k] = S
    return out


def lt_observables(S, A, R: float) -> dict:
    """lambda_max / R^2, beta (Eq. (beta), E of frame A; NaN when E = 0) and
    D = (sqrt(l_max) - sqrt(l_min))/(sqrt(l_max) + sqrt(l_min)) of one S."""
    lam, vec = np.linalg.eigh(np.asarray(S, dtype=np.float64))
    v = vec[:, 2]
    E = strain(A)
    nE = np.sqrt((E * E).sum())
    beta = float(v @ E @ v / nE) if nE > 0 else float("nan")
    p, q = np.sqrt(lam[2]), np.sqrt(lam[0])
    return {"lam_max_R2": lam[2] / (R * R), "beta": beta, "D": (p - q) / (p + q), "lam": lam}
