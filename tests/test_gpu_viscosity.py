"""Viscosity ratio chi != 1 (Sec. 2; the paper's runs have chi = 1): the
library against the oracle with an off-centre droplet in FP64 and FP32,
eager and as replayed graphs with regularisation, and the refusals."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou, make_pair, rel, run_both

pytestmark = pytest.mark.gpu

N = (24, 22, 26)
CENTRE = (10.7, 11.2, 12.9)


def _pair(precision, frames, n_hold, chi, R=4.5, level=2):
    g, o = make_pair(N, 1.0, frames, n_hold, precision=precision)
    g.add_icosphere(level, R, 0.02, center=CENTRE)
    r, t = O.icosphere(level, R, CENTRE)
    o.set_mesh(r, t, 0.02)
    g.set_viscosity_ratio(chi)
    o.set_viscosity_ratio(chi)
    return g, o


@pytest.mark.parametrize("steps", [1, 12])
def test_viscosity_ratio_fp64_matches_oracle(steps):
    fr = frames_ou(91, 4, 4e-3)
    g, o = _pair("fp64", fr, 4, 3.0)
    run_both(g, o, steps)
    assert np.abs(g.mesh()[0] - o.mesh()[0]).max() < 1e-12
    rho_g, u_g, _ = g.fields()
    rho_o, u_o, _ = o.fields()
    assert np.abs(u_g - u_o).max() < 1e-14
    assert np.abs(rho_g - rho_o).max() < 1e-13
    assert o.indicator().sum() > 200  # the droplet's interior relaxes with tau_in
    if steps > 1:
        # chi = 3 changes the flow against chi = 1 from the second step on (the
        # first step's velocity is a moment of the initial populations)
        b = O.OracleSim(N, 1.0, fr, 4)
        b.set_mesh(*O.icosphere(2, 4.5, CENTRE), 0.02)
        b.step(steps)
        assert np.abs(b.fields()[1] - u_o).max() > 1e-9
    assert g.status() == 0


def test_viscosity_ratio_fp32_and_graph_replay():
    """FP32 storage over 60 steps at chi = 0.4 within the droplet-test
    tolerances; FP64 graph replay (regularisation every 10 steps) equals
    eager stepping at chi = 5."""
    fr = frames_ou(92, 6, 4e-3)
    g, o = _pair("fp32", fr, 10, 0.4)
    run_both(g, o, 60)
    assert np.abs(g.mesh()[0] - o.mesh()[0]).max() < 1e-6 * 4.5
    assert rel(g.fields()[1], o.fields()[1]) < 1e-5
    out = []
    for graphs in (True, False):
        h, _ = _pair("fp64", fr, 10, 5.0)
        h.set_graphs(graphs)
        h.set_regularization(every=10)
        h.step(7)
        h.step(80)
        h.sync()
        out.append(h.mesh()[0])
        assert h.status() == 0
    assert np.abs(out[0] - out[1]).max() < 1e-12


def test_viscosity_ratio_refusals():
    from paper_2403_01161_gb300 import _lib as L
    from paper_2403_01161_gb300.sim import Ensemble, Sim

    fr = frames_ou(93, 3, 4e-3)
    g, _ = _pair("fp64", fr, 10, 2.0)
    with pytest.raises(L.IblError) as e:
        g.adjoint(5, 5)
    assert e.value.code == L.IBL_EINVAL
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(L.IblError):
            g.set_viscosity_ratio(bad)
    with pytest.raises(L.IblError):
        Ensemble([g])
    p = Sim(N, 1.0, fr, 10, bc=(0, 1, 0), precision="fp64")
    p.add_icosphere(2, 4.0, 0.02, center=CENTRE)
    with pytest.raises(L.IblError) as e:
        p.set_viscosity_ratio(2.0)
    assert e.value.code == L.IBL_EINVAL
    # chi = 1 switches it off: the plain trajectory
    g.set_viscosity_ratio(1.0)
    g.step(10)
    o = O.OracleSim(N, 1.0, fr, 10)
    o.set_mesh(*O.icosphere(2, 4.5, CENTRE), 0.02)
    o.step(10)
    assert np.abs(g.mesh()[0] - o.mesh()[0]).max() < 1e-12
