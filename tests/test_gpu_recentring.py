"""Re-centring of the boundary field on the droplet's centre of mass (the
Sec. 3.2 remark; off by default): the library against the oracle with an
off-centre droplet, in FP64 and FP32, eager and as replayed graphs, in the
batched ensemble, and the argument checks."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou, lib_to_oracle_perm, make_pair, rel, run_both

pytestmark = pytest.mark.gpu

N = (24, 22, 26)
CENTRE = (10.2, 11.6, 12.1)  # off the box centre (11.5, 10.5, 12.5) on every axis


def _pair(precision, frames, n_hold, n=N, centre=CENTRE, R=4.5, level=2):
    g, o = make_pair(n, 1.0, frames, n_hold, precision=precision)
    g.add_icosphere(level, R, 0.02, center=centre)
    r, t = O.icosphere(level, R, centre)
    o.set_mesh(r, t, 0.02)
    g.set_recentring(True)
    o.set_recentring(True)
    return g, o, t


@pytest.mark.parametrize("steps", [1, 12])
def test_recentring_fp64_matches_oracle(steps):
    fr = frames_ou(71, 4, 4e-3)
    g, o, t = _pair("fp64", fr, 4)
    run_both(g, o, steps)
    r_g, _, _ = g.mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-12
    rho_g, u_g, _ = g.fields()
    rho_o, u_o, _ = o.fields()
    assert np.abs(u_g - u_o).max() < 1e-14
    assert np.abs(rho_g - rho_o).max() < 1e-13
    # the faces carry the field about the centre of mass, not the box centre
    b = O.OracleSim(N, 1.0, fr, 4)
    b.set_mesh(*O.icosphere(2, 4.5, CENTRE), 0.02)
    b.step(steps)
    assert np.abs(b.fields()[1] - u_o).max() > 1e-4
    assert g.status() == 0


def test_recentring_fp32_and_graph_replay_match_oracle():
    """FP32 storage over 60 steps (whole chunks replay as graphs): positions
    within 1e-6 of the droplet size, velocities within 1e-5 relative; the
    eager FP64 run and its graph replay agree to rounding."""
    fr = frames_ou(72, 6, 4e-3)
    g, o, t = _pair("fp32", fr, 10)
    run_both(g, o, 60)
    r_g, _, _ = g.mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-6 * 4.5
    _, u_g, _ = g.fields()
    _, u_o, _ = o.fields()
    assert rel(u_g, u_o) < 1e-5
    out = []
    for graphs in (True, False):
        h, _, _ = _pair("fp64", fr, 10)
        h.set_graphs(graphs)
        h.set_regularization(every=10)
        h.step(7)
        h.step(80)
        h.sync()
        out.append(h.mesh()[0])
        assert h.status() == 0
    assert np.abs(out[0] - out[1]).max() < 1e-12


def test_recentring_in_the_ensemble():
    """Batched members with re-centring (one of them without) against the
    same droplets stepped one at a time, and one member against the oracle."""
    from paper_2403_01161_gb300.sim import Ensemble, Sim

    specs = [((24, 26, 22), (10.0, 13.4, 11.0), True), ((26, 24, 28), (13.1, 10.9, 12.2), True),
             ((20, 20, 20), (9.5, 9.5, 9.5), False)]

    def member(n, c, on, seed):
        g = Sim(n, 1.0, frames_ou(seed, 4, 4e-3), 7, precision="fp64")
        g.add_icosphere(2, 4.0, 0.02, center=c)
        if on:
            g.set_recentring(True)
        return g

    ens = [member(n, c, on, 80 + k) for k, (n, c, on) in enumerate(specs)]
    ind = [member(n, c, on, 80 + k) for k, (n, c, on) in enumerate(specs)]
    E = Ensemble(ens)
    E.step(30)
    E.sync()
    for g in ind:
        g.step(30)
        g.sync()
    for a, b in zip(ens, ind):
        assert np.abs(a.mesh()[0] - b.mesh()[0]).max() < 1e-12
        assert np.abs(a.populations() - b.populations()).max() < 1e-13
    n, c, _ = specs[1]
    o = O.OracleSim(n, 1.0, frames_ou(81, 4, 4e-3), 7)
    o.set_mesh(*O.icosphere(2, 4.0, c), 0.02)
    o.set_recentring(True)
    o.step(30)
    assert np.abs(ens[1].mesh()[0] - o.mesh()[0]).max() < 1e-11
    perm = lib_to_oracle_perm()
    assert np.abs(ens[1].populations()[perm] - o.populations()).max() < 1e-13


def test_recentring_argument_checks():
    """The adjoint refuses re-centring; switching it off restores the box
    centre (the trajectory of a run that never had it)."""
    from paper_2403_01161_gb300 import _lib as L

    fr = frames_ou(73, 3, 4e-3)
    g, _, _ = _pair("fp64", fr, 10)
    with pytest.raises(L.IblError) as e:
        g.adjoint(5, 5)
    assert e.value.code == L.IBL_EINVAL
    g.set_recentring(False)
    g.step(10)
    h, _, _ = _pair("fp64", fr, 10)
    h.set_recentring(False)
    h.step(10)
    o = O.OracleSim(N, 1.0, fr, 10)
    o.set_mesh(*O.icosphere(2, 4.5, CENTRE), 0.02)
    o.step(10)
    for s in (g, h):
        assert np.abs(s.mesh()[0] - o.mesh()[0]).max() < 1e-12
