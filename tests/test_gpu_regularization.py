"""The adaptive regularisation trigger: a threshold never reached leaves the
trajectory exactly as without regularisation; a threshold always exceeded
gives the scheduled regularisation of Sec. 3.3; the measured mesh quality is
the oracle's; ibl_regularize_now ignores the trigger; bad thresholds are
rejected."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou

pytestmark = pytest.mark.gpu

N = (24, 22, 26)


def _sim(every=0, trigger=None):
    from paper_2403_01161_gb300.sim import Sim

    s = Sim(N, 1.0, frames_ou(21, 4, 4e-3), 8, precision="fp64")
    s.add_icosphere(2, 4.5, 0.02, center=tuple(0.5 * (k - 1) for k in N))
    if every:
        s.set_regularization(every=every)
    if trigger is not None:
        s.set_regularization_trigger(trigger)
    return s


def test_unreached_trigger_leaves_the_trajectory_alone():
    a = _sim(every=5, trigger=1e6)
    a.step(20)
    b = _sim()
    b.step(20)
    ra, _, t = a.mesh()
    rb, _, _ = b.mesh()
    assert np.abs(ra - rb).max() < 1e-12
    count, q = a.regularization_stats()
    assert count == 0
    # the last check ran on the positions after step 20
    assert abs(q - O.mesh_quality(ra, t)) < 1e-12 * q
    assert a.status() == 0


def test_always_exceeded_trigger_is_the_scheduled_regularisation():
    a = _sim(every=5, trigger=1.0)
    a.step(20)
    b = _sim(every=5)
    b.step(20)
    ra, _, _ = a.mesh()
    rb, _, _ = b.mesh()
    assert np.abs(ra - rb).max() < 1e-12
    assert a.regularization_stats()[0] == 4
    assert b.regularization_stats()[0] == 4


def test_regularize_now_ignores_the_trigger_and_bad_thresholds():
    from paper_2403_01161_gb300 import _lib as L

    a = _sim(every=5, trigger=1e6)
    a.step(3)
    it = a.regularize_now()
    assert it >= 1
    assert a.regularization_stats()[0] == 1
    for bad in (-1.0, 0.5, float("inf")):
        with pytest.raises(L.IblError) as e:
            a.set_regularization_trigger(bad)
        assert e.value.code == L.IBL_EINVAL
    a.set_regularization_trigger(0.0)
    a.close()


def test_keep_volume_matches_oracle():
    """The volume-restoring option: a one-off regularisation of a stretched,
    jittered icosphere and a coupled FP64 run with regularisation every 5
    steps give the oracle's positions, and the one-off keeps the volume."""
    from paper_2403_01161_gb300 import inputs
    from paper_2403_01161_gb300.sim import Sim

    r0, t = O.icosphere(3, 5.0, (15.5, 15.5, 15.5))
    r0 = inputs.jitter((r0 - 15.5) * [1.5, 0.8, 0.9] + 15.5, 0.15, 3)
    g = Sim((32, 32, 32), 1.0, np.zeros((1, 3, 3)), 1, precision="fp32")
    g.add_mesh(r0, t, 0.01)
    g.set_regularization_keep_volume(True)
    g.regularize_now()
    ptr, idx = O.one_ring(t, r0.shape[0])
    x, _, conv = O.regularize(r0, ptr, idx, tris=t, keep_volume=True)
    r_g, _, _ = g.mesh()
    assert conv and np.abs(r_g - x).max() < 1e-12
    V0 = O.enclosed_volume(r0, t)[0]
    assert abs(O.enclosed_volume(r_g, t)[0] - V0) < 1e-12 * V0
    assert O.enclosed_volume(O.regularize(r0, ptr, idx)[0], t)[0] < (1 - 1e-4) * V0
    g.close()

    fr = frames_ou(31, 3, 6e-3)
    c = (12.5, 12.5, 12.5)
    g = Sim((26, 26, 26), 1.0, fr, 8, precision="fp64")
    g.add_icosphere(2, 5.0, 0.01, center=c)
    g.set_regularization(every=5)
    g.set_regularization_keep_volume(True)
    o = O.OracleSim((26, 26, 26), 1.0, fr, 8)
    rr, tt = O.icosphere(2, 5.0, c)
    o.set_mesh(rr, tt, 0.01)
    o.set_regularization(every=5, keep_volume=True)
    g.step(20)
    o.step(20)
    r_g, _, _ = g.mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-11
    assert g.regularization_stats()[0] == 4
    g.close()
    o.close()
