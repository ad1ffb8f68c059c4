"""GPU lattice kernel against the oracle, element by element: D3Q19 BGK with
Guo forcing, AA in-place streaming, Zou-He faces/edges/corners, periodic
axes, several frames, both parities of the step count.  FP64 storage must
agree to round-off; FP32 deviation storage to the stated tolerance."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou, lib_to_oracle_perm, make_pair, rel, run_both

pytestmark = pytest.mark.gpu

# n, bc, tau, steps, edge rule.  Odd and even step counts, several tiles of
# 256 nodes with a ragged tail, periodic and Zou-He axes.
CASES = [
    ((12, 10, 9), (0, 0, 0), 1.0, 7, 0),
    ((12, 10, 9), (0, 0, 0), 1.5, 8, 0),
    ((13, 11, 10), (0, 0, 0), 0.8, 9, 1),
    ((16, 8, 10), (1, 1, 0), 1.2, 9, 0),
    ((9, 14, 11), (0, 1, 0), 1.0, 6, 0),
    ((10, 9, 15), (1, 0, 0), 0.9, 5, 0),
]


def _frames(bc, seed):
    fr = frames_ou(seed, 6, 2e-3)
    for a in range(3):
        if bc[a] == 1:  # the linear flow must not vary along a periodic axis
            fr[:, :, a] = 0.0
    return fr


@pytest.mark.parametrize("n,bc,tau,steps,rule", CASES)
def test_lattice_fp64_matches_oracle(n, bc, tau, steps, rule):
    fr = _frames(bc, 3)
    g, o = make_pair(n, tau, fr, 2, bc=bc, precision="fp64", rule=rule)
    run_both(g, o, steps)
    rho_g, u_g, F_g = g.fields()
    rho_o, u_o, F_o = o.fields()
    assert np.abs(rho_g - rho_o).max() < 1e-13
    assert np.abs(u_g - u_o).max() < 1e-14
    assert np.abs(u_o).max() > 1e-3
    perm = lib_to_oracle_perm()
    fg = g.populations()[perm]
    fo = o.populations()
    assert np.abs(fg - fo).max() < 1e-14
    assert g.status() == 0


@pytest.mark.parametrize("n,bc,tau,steps,rule", CASES)
def test_lattice_fp32_matches_oracle(n, bc, tau, steps, rule):
    """FP32 deviations against the FP64 oracle: rel 1e-5 on u (the stated
    tolerance), density deviation and populations to FP32 resolution of
    the deviations."""
    fr = _frames(bc, 4)
    g, o = make_pair(n, tau, fr, 3, bc=bc, precision="fp32", rule=rule)
    run_both(g, o, steps)
    rho_g, u_g, _ = g.fields()
    rho_o, u_o, _ = o.fields()
    assert rel(u_g, u_o) < 1e-5
    assert np.abs(rho_g - rho_o).max() < 1e-6
    perm = lib_to_oracle_perm()
    assert np.abs(g.populations()[perm] - o.populations()).max() < 1e-6


def test_lattice_long_run_fp32():
    """A few hundred steps of a sheared and strained box: FP32 deviation
    storage stays within 1e-5 relative on u of the FP64 oracle."""
    n = (20, 18, 16)
    fr = frames_ou(11, 8, 3e-3)
    g, o = make_pair(n, 1.0, fr, 40, precision="fp32")
    run_both(g, o, 300)
    _, u_g, _ = g.fields()
    _, u_o, _ = o.fields()
    assert rel(u_g, u_o) < 1e-5


def test_periodic_body_free_rest_state():
    """A fully periodic box at rest stays exactly at rest (no spurious source)."""
    g, o = make_pair((8, 8, 8), 1.0, np.zeros((1, 3, 3)), 1, bc=(1, 1, 1), precision="fp32")
    run_both(g, o, 4)
    rho, u, F = g.fields()
    assert np.abs(u).max() == 0.0 and np.abs(rho - 1).max() == 0.0
