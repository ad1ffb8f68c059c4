"""The adjoint at the size of the 64^3 adjoint workload (R 8, icosphere level
3, 2000 steps, checkpoints every K = 100 steps), for 4 of its 16 seeds (OU
gradients of seeds 500-503): dD/dsigma and the derivative of D along 4
seeded unit directions in the space of the gradient frames, from the
library's discrete adjoint, against central differences of the FP64
oracle's final Taylor deformation D (Sec. 2) stored by
tests/golden/make_oracle_series.py (adjoint_64_fd, adjoint_64_fd_s501..503)."""
import os

import numpy as np
import pytest

from paper_2403_01161_gb300 import config

pytestmark = pytest.mark.gpu

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(seed):
    name = "oracle_adjoint_64_fd.npz" if seed == 500 else "oracle_adjoint_64_fd_s%d.npz" % seed
    path = os.path.join(GOLDEN_DIR, name)
    if not os.path.exists(path):
        pytest.fail("missing %s: run tests/golden/make_oracle_series.py" % path)
    return np.load(path)


def _gradients(precision, seed):
    from paper_2403_01161_gb300.sim import Sim

    w = config.adjoint_member(seed, steps=2000)
    g = Sim(w.n, w.tau, w.frames, w.n_hold, precision=precision)
    g.add_icosphere(w.level, w.R, w.sigma)
    res = g.adjoint(2000, 100)
    assert g.status() == 0
    g.close()
    return res


@pytest.mark.parametrize("seed", [500, 501, 502, 503])
@pytest.mark.parametrize("precision,tol_D,tol_g", [("fp64", 1e-10, 1e-6), ("fp32", 1e-4, 1e-3)])
def test_adjoint_64_matches_oracle_central_differences(precision, tol_D, tol_g, seed):
    """FP64: the adjoint of the same discrete map as the oracle's, so it
    agrees with the oracle's central differences to their truncation error.
    FP32 (the measured configuration): within 1e-3 relative.  A directional
    derivative is compared relative to the gradient's norm |dD/dA| (the
    scale of a derivative along a unit direction of the 117-entry frame
    space) and to its own magnitude, whichever is larger."""
    d = _golden(seed)
    assert int(d["seed"]) == seed
    res = _gradients(precision, seed)
    assert abs(res["D"] - d["D0"]) <= tol_D * abs(d["D0"])
    assert abs(res["dD_dsigma"] - d["dD_dsigma"]) <= tol_g * abs(d["dD_dsigma"])
    gA = res["dD_dA"]
    assert gA.shape == d["V"].shape[1:]
    scale = np.linalg.norm(gA)
    for k in range(d["V"].shape[0]):
        proj = float((gA * d["V"][k]).sum())
        fd = float(d["dD_dV"][k])
        assert abs(proj - fd) <= tol_g * max(abs(fd), scale), (k, proj, fd, scale)
        if precision == "fp64":
            assert abs(proj - fd) <= tol_g * abs(fd), (k, proj, fd)
