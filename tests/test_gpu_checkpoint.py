"""Checkpoint and resume: a droplet run saved mid-way and resumed in a new
lattice continues exactly as the uninterrupted run (regularisation and
shape records on), and mismatched or damaged files are refused."""
import numpy as np
import pytest

from parity import frames_ou

pytestmark = pytest.mark.gpu

N = (24, 22, 26)


def _sim(precision="fp64", n=N):
    from paper_2403_01161_gb300.sim import Sim

    s = Sim(n, 1.0, frames_ou(61, 4, 4e-3), 9, precision=precision)
    s.add_icosphere(2, 4.5, 0.02, center=(11.2, 10.4, 12.6))
    s.set_regularization(every=10)
    s.set_readout(5)
    return s


def test_resume_continues_the_run(tmp_path):
    path = str(tmp_path / "ck.bin")
    a = _sim()
    a.step(37)
    a.save(path)
    a.step(23)
    a.sync()
    b = _sim()
    b.step(4)  # some other state, overwritten by the load
    b.load(path)
    assert b.steps_done == 37
    b.step(23)
    b.sync()
    assert b.steps_done == a.steps_done == 60
    assert np.abs(a.mesh()[0] - b.mesh()[0]).max() < 1e-12
    assert np.abs(a.populations() - b.populations()).max() < 1e-13
    sa, sb = a.series(), b.series()
    assert [x["step"] for x in sa] == [x["step"] for x in sb] == list(range(5, 61, 5))
    assert max(abs(x["D"] - y["D"]) for x, y in zip(sa, sb)) < 1e-12
    assert a.status() == 0 and b.status() == 0


def test_mismatched_or_damaged_checkpoints_are_refused(tmp_path):
    from paper_2403_01161_gb300 import _lib as L

    path = str(tmp_path / "ck.bin")
    a = _sim()
    a.step(3)
    a.save(path)
    for other in (_sim(precision="fp32"), _sim(n=(24, 22, 28))):
        with pytest.raises(L.IblError) as e:
            other.load(path)
        assert e.value.code == L.IBL_EINVAL
    data = open(path, "rb").read()
    short = str(tmp_path / "short.bin")
    open(short, "wb").write(data[: len(data) // 2])
    with pytest.raises(L.IblError):
        _sim().load(short)
    with pytest.raises(L.IblError):
        _sim().load(str(tmp_path / "missing.bin"))
