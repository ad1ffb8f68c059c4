"""Batched ensemble of uneven droplets against the same droplets stepped one
at a time (and one member against the oracle): the batched kernels compute
exactly what the single-droplet kernels compute, up to the order of the
atomic additions in the spread."""
import numpy as np
import pytest

import oracle as O
from parity import frames_ou, lib_to_oracle_perm

pytestmark = pytest.mark.gpu

SPECS = [((24, 26, 22), 4.0, 2, 1), ((30, 28, 32), 5.0, 3, 2), ((20, 20, 20), 3.5, 2, 3), ((26, 24, 28), 4.5, 2, 4)]


def _member(n, R, level, seed, precision, reg=0, readout=0):
    from paper_2403_01161_gb300.sim import Sim

    g = Sim(n, 1.0, frames_ou(seed, 4, 4e-3), 7, precision=precision)
    g.add_icosphere(level, R, 0.02)
    if reg:
        g.set_regularization(every=reg)
    if readout:
        g.set_readout(readout)
    return g


@pytest.mark.parametrize("precision,tol_r,tol_f", [("fp64", 1e-12, 1e-13), ("fp32", 1e-6, 1e-6)])
def test_ensemble_matches_one_at_a_time(precision, tol_r, tol_f):
    from paper_2403_01161_gb300.sim import Ensemble

    ens = [_member(*s, precision, reg=10, readout=5) for s in SPECS]
    ind = [_member(*s, precision, reg=10, readout=5) for s in SPECS]
    E = Ensemble(ens)
    E.step(3)
    E.step(45)  # eager head, graph replays of whole chunks, eager tail
    E.sync()
    for g in ind:
        g.step(48)
        g.sync()
    for a, b in zip(ens, ind):
        assert a.steps_done == b.steps_done == 48
        ra, _, _ = a.mesh()
        rb, _, _ = b.mesh()
        assert np.abs(ra - rb).max() < tol_r
        assert np.abs(a.populations() - b.populations()).max() < tol_f
        sa, sb = a.series(), b.series()
        assert [x["step"] for x in sa] == [x["step"] for x in sb] == list(range(5, 49, 5))
        assert max(abs(x["D"] - y["D"]) for x, y in zip(sa, sb)) < tol_r


def test_ensemble_graph_chunks_match_one_at_a_time():
    """Long enough to replay whole graph chunks of the two-stream ensemble
    step (chunk 60 with regularisation every 10 and records every 5)."""
    from paper_2403_01161_gb300.sim import Ensemble

    ens = [_member(*s, "fp64", reg=10, readout=5) for s in SPECS]
    ind = [_member(*s, "fp64", reg=10, readout=5) for s in SPECS]
    E = Ensemble(ens)
    E.step(3)
    E.step(130)  # eager to 60, one chunk replay to 120, eager tail
    E.sync()
    for g in ind:
        g.step(133)
        g.sync()
    for a, b in zip(ens, ind):
        ra, _, _ = a.mesh()
        rb, _, _ = b.mesh()
        assert np.abs(ra - rb).max() < 1e-12
        assert np.abs(a.populations() - b.populations()).max() < 1e-13
        assert [x["step"] for x in a.series()] == list(range(5, 134, 5))


@pytest.mark.parametrize("precision,tol_r,tol_f", [("fp64", 1e-12, 1e-13), ("fp32", 1e-6, 1e-6)])
def test_every_launch_shape_computes_the_same_step(precision, tol_r, tol_f):
    """The batched lattice update's launch shapes (threads per block, L2
    prefetch distance) change only the launch geometry; the autotuner keeps
    one of them and the members stay on the one-at-a-time trajectory."""
    from paper_2403_01161_gb300 import _lib as L
    from paper_2403_01161_gb300.sim import Ensemble

    ref = [_member(*s, precision) for s in SPECS]
    for g in ref:
        g.step(24)
        g.sync()
    for shape in range(L.ENSEMBLE_SHAPES):
        ens = [_member(*s, precision) for s in SPECS]
        E = Ensemble(ens)
        E.set_shape(shape)
        assert E.shape()[0] == shape
        E.step(24)
        E.sync()
        for a, b in zip(ens, ref):
            assert np.abs(a.mesh()[0] - b.mesh()[0]).max() < tol_r
            assert np.abs(a.populations() - b.populations()).max() < tol_f
        E.close()
    ens = [_member(*s, precision) for s in SPECS]
    E = Ensemble(ens)
    k, ms = E.tune(4)
    assert 0 <= k < L.ENSEMBLE_SHAPES and ms.shape == (L.ENSEMBLE_SHAPES,) and (ms > 0).all()
    assert ms[k] == ms.min() and E.shape()[0] == k
    assert all(g.steps_done == L.ENSEMBLE_SHAPES * 6 for g in ens)
    E.step(12)
    E.sync()
    for g in ref:
        g.step(L.ENSEMBLE_SHAPES * 6 + 12 - 24)
        g.sync()
    for a, b in zip(ens, ref):
        assert np.abs(a.mesh()[0] - b.mesh()[0]).max() < tol_r
        assert np.abs(a.populations() - b.populations()).max() < tol_f


def test_ensemble_member_matches_oracle():
    from paper_2403_01161_gb300.sim import Ensemble

    ens = [_member(*s, "fp64") for s in SPECS]
    E = Ensemble(ens)
    E.step(20)
    E.sync()
    n, R, level, seed = SPECS[1]
    o = O.OracleSim(n, 1.0, frames_ou(seed, 4, 4e-3), 7)
    r0, t = O.icosphere(level, R, tuple(0.5 * (k - 1) for k in n))
    o.set_mesh(r0, t, 0.02)
    o.step(20)
    r_g, _, _ = ens[1].mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-11
    perm = lib_to_oracle_perm()
    assert np.abs(ens[1].populations()[perm] - o.populations()).max() < 1e-13


def test_ensemble_rejects_desynchronised_members():
    from paper_2403_01161_gb300 import _lib as L
    from paper_2403_01161_gb300.sim import Ensemble

    ens = [_member(*s, "fp32") for s in SPECS[:2]]
    E = Ensemble(ens)
    ens[0].step(1)
    with pytest.raises(L.IblError):
        E.step(1)
