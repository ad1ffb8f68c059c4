"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.  This module holds none of the method's arithmetic: it
only draws velocity-gradient sequences that stand in for the turbulent
trajectories of the TURB-Lagr database used in Sec. 3.2 of arXiv:2403.01161
(the database itself is not available offline).

Recipe (traceless Ornstein-Uhlenbeck process in lattice units):
    A_0     = s P(xi_0)
    A_{k+1} = exp(-dt/T) A_k + sqrt(1 - exp(-2 dt/T)) s P(xi_{k+1})
with xi_k a 3x3 standard normal draw from numpy.random.default_rng(seed), in
that order, P the traceless projection X - tr(X)/3 I, s = a_rms / sqrt(8) (a
traceless 3x3 Gaussian has 8 degrees of freedom, so E|A|_F^2 = a_rms^2), dt
the frame interval and T the correlation time.  Row a of A_k holds du_a/dx_b.
"""
from __future__ import annotations

import numpy as np


def traceless(x: np.ndarray) -> np.ndarray:
    """x minus its trace part (over the last two axes, so stacks work too)."""
    return x - (np.trace(x, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def ou_gradients(seed: int, n_frames: int, dt: float, T: float, a_rms: float) -> np.ndarray:
    """(n_frames, 3, 3) float64 traceless OU gradient frames (see module doc)."""
    rng = np.random.default_rng(seed)
    s = a_rms / np.sqrt(8.0)
    out = np.empty((n_frames, 3, 3), dtype=np.float64)
    a = np.exp(-dt / T)
    b = np.sqrt(1.0 - np.exp(-2.0 * dt / T))
    out[0] = s * traceless(rng.standard_normal((3, 3)))
    for k in range(1, n_frames):
        out[k] = a * out[k - 1] + b * s * traceless(rng.standard_normal((3, 3)))
    return out


def ou_gradients_batch(seed: int, n_traj: int, n_frames: int, dt: float, T: float, a_rms: float) -> np.ndarray:
    """(n_traj, n_frames, 3, 3) float64: n_traj independent traceless OU
    gradient sequences of the same law as ou_gradients, drawn from one seeded
    generator (vectorised over trajectories)."""
    rng = np.random.default_rng(seed)
    s = a_rms / np.sqrt(8.0)
    a = np.exp(-dt / T)
    b = np.sqrt(1.0 - np.exp(-2.0 * dt / T))
    out = np.empty((n_frames, n_traj, 3, 3), dtype=np.float64)
    out[0] = s * traceless(rng.standard_normal((n_traj, 3, 3)))
    for k in range(1, n_frames):
        out[k] = a * out[k - 1] + b * s * traceless(rng.standard_normal((n_traj, 3, 3)))
    return np.ascontiguousarray(out.transpose(1, 0, 2, 3))


def simple_shear(rate: float, flow_axis: int = 0, gradient_axis: int = 2) -> np.ndarray:
    """(1, 3, 3) frame of steady simple shear u_flow = rate * x_gradient."""
    A = np.zeros((1, 3, 3))
    A[0, flow_axis, gradient_axis] = rate
    return A


def jitter(r: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """Node positions displaced by seeded Gaussian noise (mesh test inputs)."""
    rng = np.random.default_rng(seed)
    return r + amplitude * rng.standard_normal(r.shape)


def ensemble_members(n: int = 64, seed0: int = 1000):
    """Box sides and radii of the uneven droplet ensemble: seed0 + k draws
    L_k uniformly from {48, 56, ..., 96} and R_k uniformly in [6, 10] rounded
    to 0.5, redrawing L_k until L_k >= 6 R_k; icosphere level 3 if R_k < 8
    else 4."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed0 + k)
        R = round(rng.uniform(6.0, 10.0) * 2.0) / 2.0
        L = int(rng.choice(np.arange(48, 97, 8)))
        while L < 6 * R:
            L = int(rng.choice(np.arange(48, 97, 8)))
        out.append({"seed": seed0 + k, "L": L, "R": R, "level": 3 if R < 8 else 4})
    return out
