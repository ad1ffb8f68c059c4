"""Whole trajectories of the measured FP32 workloads against the FP64
oracle (the trajectory loop of Sec. 3.2, steps 1-4, with the shape readout
of Sec. 2): the 128^3 single droplet over 20000 steps, the 256^3 precision
stress workload over 5000 steps (rms Ca 0.5, regularisation of Sec. 3.3
every 50 steps), and the first 8 members of the 64-droplet ensemble over
10000 steps, batched.  The oracle's series are stored by
tests/golden/make_oracle_series.py, which calls only the oracle.

Per-observable bounds (FP32 deviation populations, FP64 mesh geometry):
  D       relative 1e-4, against max(|D_oracle|, 0.05): a nearly spherical
          droplet has D -> 0, where a relative error means nothing, so the
          first records are held to 5e-6 absolute;
  beta    absolute 1e-4, on records whose leading eigenvalue of S stands
          clear of the second by 1% of itself (the direction v_max of a
          droplet with a degenerate leading pair is undefined; its error
          is |dS| / (lam_1 - lam_2));
  V, lam_max   relative 1e-5;
  u       relative 1e-5 in the 2-norm over the stored node sample (the box
          around the final droplet plus seeded nodes of the whole box);
  r       relative 1e-6: |r_gpu - r_oracle|_2 / |r_oracle - mean(r_oracle)|_2,
          i.e. against the droplet's size, not its place in the box.
A trajectory the oracle stopped at a flagged record (a stencil reaching a
wall) is compared up to its last clean record."""
import os

import numpy as np
import pytest

from paper_2403_01161_gb300 import config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RECORD_EVERY = 100


def _golden(name):
    path = os.path.join(GOLDEN, "oracle_%s.npz" % name)
    if not os.path.exists(path):
        pytest.skip("missing %s: run tests/golden/make_oracle_series.py %s" % (path, name))
    return np.load(path)


def _sim(w, record_fields):
    from paper_2403_01161_gb300.sim import Sim

    g = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, record_fields=record_fields)
    g.add_icosphere(w.level, w.R, w.sigma)
    if w.reg_every:
        g.set_regularization(every=w.reg_every)
    g.set_readout(RECORD_EVERY)
    return g


def _check_records(series, d, prefix, last_step, label):
    """Every GPU shape record up to last_step against the oracle's."""
    by_step = {int(s["step"]): s for s in series}
    steps = d[prefix + "rec_step"]
    worst = {"D": 0.0, "beta": 0.0, "V": 0.0, "lam": 0.0}
    n_beta = 0
    for k, st in enumerate(steps):
        st = int(st)
        if st > last_step:
            break
        assert st in by_step, "%s: GPU has no record at step %d" % (label, st)
        s = by_step[st]
        assert s["err"] == 0, "%s: GPU flagged error bits %d at step %d" % (label, s["err"], st)
        D_o = float(d[prefix + "rec_D"][k])
        eD = abs(s["D"] - D_o) / max(abs(D_o), 0.05)
        V_o = float(d[prefix + "rec_V"][k])
        eV = abs(s["V"] - V_o) / abs(V_o)
        lam_o = np.asarray(d[prefix + "rec_lam"][k], dtype=np.float64)
        lmax_o = float(lam_o.max())
        eL = abs(max(s["lam"]) - lmax_o) / lmax_o
        worst["D"] = max(worst["D"], eD)
        worst["V"] = max(worst["V"], eV)
        worst["lam"] = max(worst["lam"], eL)
        assert eD <= 1e-4, "%s step %d: D %.9f vs oracle %.9f" % (label, st, s["D"], D_o)
        assert eV <= 1e-5, "%s step %d: V %.9f vs oracle %.9f" % (label, st, s["V"], V_o)
        assert eL <= 1e-5, "%s step %d: lam_max %.9f vs oracle %.9f" % (label, st, max(s["lam"]), lmax_o)
        ls = np.sort(lam_o)[::-1]
        b_o = float(d[prefix + "rec_beta"][k])
        if ls[0] - ls[1] >= 1e-2 * ls[0] and np.isfinite(b_o):
            eb = abs(s["beta"] - b_o)
            worst["beta"] = max(worst["beta"], eb)
            n_beta += 1
            assert eb <= 1e-4, "%s step %d: beta %.8f vs oracle %.8f" % (label, st, s["beta"], b_o)
    print("%s: %d records to step %d, worst D %.2e, beta %.2e (%d records), V %.2e, lam_max %.2e"
          % (label, len([s for s in steps if s <= last_step]), last_step, worst["D"], worst["beta"], n_beta,
             worst["V"], worst["lam"]))


def _check_positions(r_g, r_o, label):
    e = np.linalg.norm(r_g - r_o) / np.linalg.norm(r_o - r_o.mean(axis=0))
    print("%s: positions relative %.2e" % (label, e))
    assert e <= 1e-6, "%s: positions differ by %.3e relative" % (label, e)


def _trajectory(w, name):
    d = _golden(name)
    last = int(d["last_step"])
    g = _sim(w, record_fields=True)
    g.step(last - 1)
    g.step_record()
    assert g.status() == 0
    _check_records(g.series(), d, "", last, name)
    r_g, _, tris = g.mesh()
    assert np.array_equal(tris, d["tris"])
    _check_positions(r_g, d["r_last"], name)
    _, u, _ = g.fields()
    u = u.reshape(3, -1)
    idx = d["u_idx"]
    u_o = d["u_sample"]
    eu = np.linalg.norm(u[:, idx] - u_o) / np.linalg.norm(u_o)
    en = abs(np.linalg.norm(u) - float(d["u_norm_all"])) / float(d["u_norm_all"])
    print("%s: u sample relative %.2e (%d nodes), whole-field norm %.2e" % (name, eu, idx.size, en))
    assert eu <= 1e-5
    assert en <= 1e-5
    g.close()


def test_single_droplet_128_trajectory():
    """128^3, R 12, level 4, OU seed 2, rms Ca 0.2: 20000 FP32 steps."""
    _trajectory(config.single_droplet_128(steps=20000), "single_droplet_128")


@pytest.mark.slow
def test_precision_stress_256_trajectory():
    """256^3, R 24, level 5, R/eta 1, rms Ca 0.5, regularisation every 50
    steps: 5000 FP32 steps."""
    _trajectory(config.precision_stress_256(steps=5000, Ca_rms=0.5), "precision_stress_256")


def test_ensemble_members_trajectories():
    """The first 8 members of the uneven ensemble (seeds 1000-1007, boxes
    48^3-96^3), stepped together by the batched kernels for 10000 steps."""
    from paper_2403_01161_gb300.sim import Ensemble

    d = _golden("ensemble8")
    ws = config.ensemble_workloads(8, steps=10000)
    members = [_sim(w, record_fields=False) for w in ws]
    E = Ensemble(members)
    last = [int(d["m%d_last_step" % k]) for k in range(8)]
    # members the oracle found clean to the end run the full length; a
    # flagged member stops every member at its last clean record
    stop = min(last)
    E.step(stop)
    E.sync()
    for k, (g, w) in enumerate(zip(members, ws)):
        _check_records(g.series(), d, "m%d_" % k, min(last[k], stop), "ensemble member %d (%s)" % (k, w.name))
        if last[k] == stop:
            r_g, _, _ = g.mesh()
            _check_positions(r_g, d["m%d_r_last" % k], "ensemble member %d" % k)
    E.close()
    for g in members:
        g.close()
