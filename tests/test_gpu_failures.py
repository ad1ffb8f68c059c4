"""Failure detection with inputs made on the host: a non-finite gradient
frame or position (refused before any device work), a gradient frame whose
wall velocity breaks the Mach limit |u| <= 0.3 (the lattice kernels flag it,
the next synchronising call reports IBL_EUNSTABLE), a regularisation that
cannot meet its tolerance in max_iter iterations (Sec. 3.3 exit criterion;
IBL_ENOCONV), an ensemble naming the member that failed, and a bounded
device wait that runs out (IBL_ETIMEOUT).  No case faults the GPU: the
kernels bound every access whatever the values, and every wait in time."""
import numpy as np
import pytest

from paper_2403_01161_gb300 import _lib as L
from parity import frames_ou

pytestmark = pytest.mark.gpu

N = (22, 20, 24)


def _sim(precision="fp32", frames=None, hold=5, graphs=True):
    from paper_2403_01161_gb300.sim import Sim

    fr = frames_ou(11, 6, 3e-3) if frames is None else frames
    g = Sim(N, 1.0, fr, hold, precision=precision)
    g.add_icosphere(2, 4.0, 0.02)
    g.set_graphs(graphs)
    return g


def _over_mach():
    """A frame whose wall velocity reaches |A| (n - 1)/2 = 0.05 * 11.5 > 0.3."""
    A = np.zeros((3, 3))
    A[0, 2] = 0.05
    A[2, 0] = -0.05
    return A


def test_non_finite_inputs_are_refused_on_the_host():
    from paper_2403_01161_gb300.sim import Sim

    fr = frames_ou(11, 4, 3e-3)
    bad = fr.copy()
    bad[2, 1, 0] = np.nan
    with pytest.raises(L.IblError) as e:
        Sim(N, 1.0, bad, 5)
    assert e.value.code == L.IBL_EINVAL
    g = _sim()
    with pytest.raises(L.IblError) as e:
        g.set_frame(1, np.full((3, 3), np.inf))
    assert e.value.code == L.IBL_EINVAL
    h = Sim(N, 1.0, fr, 5)
    r, t = __import__("oracle").icosphere(2, 4.0, tuple(0.5 * (k - 1) for k in N))
    r[7, 1] = np.nan
    with pytest.raises(L.IblError) as e:
        h.add_mesh(r, t, 0.02)
    assert e.value.code == L.IBL_EINVAL
    g.step(10)
    assert g.status() == L.IBL_OK  # the refused frame changed nothing


@pytest.mark.parametrize("precision,graphs", [("fp32", True), ("fp64", False)])
def test_over_mach_frame_reports_unstable_at_the_next_sync(precision, graphs):
    g = _sim(precision, graphs=graphs)
    g.step(12)
    assert g.status() == L.IBL_OK
    g.set_frame(3, _over_mach())  # applied from step 15
    g.step(2)
    assert g.status() == L.IBL_OK  # steps 12, 13 still use frame 2
    g.step(30)
    assert g.status() == L.IBL_EUNSTABLE
    with pytest.raises(L.IblError) as e:
        g.sync()
    assert e.value.code == L.IBL_EUNSTABLE and "0.3" in str(e.value)
    g.step(6)  # the bits are sticky; stepping on stays in bounds
    assert g.status() == L.IBL_EUNSTABLE
    rec = g.readout  # a synchronising readout reports the same status
    with pytest.raises(L.IblError):
        rec()
    g.close()
    # the context is still usable: a fresh box runs clean
    h = _sim(precision)
    h.step(20)
    assert h.status() == L.IBL_OK
    h.close()


def test_regularisation_without_convergence_reports_noconv():
    g = _sim("fp64")
    g.set_regularization(alpha=0.1, gamma=0.51, tol=1e-12, max_iter=1, every=5)
    g.step(4)
    assert g.status() == L.IBL_OK
    g.step(1)  # the first scheduled regularisation stops after one iteration
    assert g.status() == L.IBL_ENOCONV
    g.close()
    h = _sim("fp64")
    h.set_regularization(alpha=0.1, gamma=0.51, tol=1e-12, max_iter=1, every=0)
    with pytest.raises(L.IblError) as e:
        h.regularize_now()
    assert e.value.code == L.IBL_ENOCONV
    h.close()
    k = _sim("fp64")
    k.set_regularization(alpha=0.1, gamma=0.51, tol=0.01, max_iter=100, every=5)
    k.step(20)
    assert k.status() == L.IBL_OK  # the paper's tolerance converges on the same mesh
    k.close()


def test_ensemble_names_the_failing_member():
    from paper_2403_01161_gb300.sim import Ensemble

    members = [_sim("fp32") for _ in range(3)]
    E = Ensemble(members)
    E.step(10)
    E.sync()
    members[1].set_frame(4, _over_mach())  # frame 4: steps 20..24
    E.step(40)
    with pytest.raises(L.IblError) as e:
        E.sync()
    assert e.value.code == L.IBL_EUNSTABLE
    assert "ensemble member 1" in str(e.value)
    assert members[0].status() == L.IBL_OK and members[2].status() == L.IBL_OK
    E.close()


def test_staged_update_wait_runs_out_and_reports_timeout():
    """The staged outside update waits on mbarriers for its own bulk copies,
    each wait bounded in time.  With the test hook its stages never complete
    (more bytes announced than copied): every block gives up after 1 s, sets
    the sticky timeout bit and returns; the next synchronising call reports
    IBL_ETIMEOUT, and the device stays usable for the next lattice."""
    import time

    from paper_2403_01161_gb300.sim import Sim

    fr = frames_ou(12, 4, 3e-3)
    g = Sim(N, 1.0, fr, 5, precision="fp32")
    g.set_graphs(False)
    g.set_outside_update(1)
    L.check(g.lib.ibl_test_stage_timeout(g.h, 1))
    t0 = time.time()
    g.step(1)
    assert g.status() == L.IBL_ETIMEOUT
    assert time.time() - t0 < 30.0
    g.close()
    h = Sim(N, 1.0, fr, 5, precision="fp32")
    h.set_outside_update(1)
    h.step(4)
    assert h.status() == 0
    ref = Sim(N, 1.0, fr, 5, precision="fp32")
    ref.step(4)
    assert np.array_equal(h.populations(), ref.populations())
    h.close()
    ref.close()
