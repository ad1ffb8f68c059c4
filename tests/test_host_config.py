"""Host-side parameter mapping (Sec. 3.2) and the seeded input generators."""
import numpy as np
import pytest

from paper_2403_01161_gb300 import config, inputs


def test_steps_per_frame_matches_paper(golden):
    """Eq. (N_Reta) with the TURB-Lagr numbers of Sec. 3.2 and the production
    setup (R_LBU = 19, tau_f = 1.5) at R/eta = 0.472 gives N ~ 500."""
    d = golden["dns_units"]["value"]
    for k in ("eta", "tau_eta", "nu", "epsilon", "dt_frame"):
        assert config.DNS[k] == d[k]
    p = golden["production_setup"]["value"]
    c = config.dns_to_lbu(p["R_over_eta"], p["R_lbu"], p["tau_f"], 0.05)
    assert abs(c["N"] / golden["steps_per_frame_example"]["value"]["N"] - 1) < 0.01
    # N scales as (eta/R)^2
    c2 = config.dns_to_lbu(p["R_over_eta"] / 2, p["R_lbu"], p["tau_f"], 0.05)
    assert abs(c2["N"] / c["N"] - 4) < 1e-12
    # sigma = mu R / tau_sigma with tau_sigma = Ca tau_eta converted to lattice time
    assert abs(c["sigma_lbu"] - config.nu_lbu(1.5) * 19 / (0.05 * c["tau_eta_lbu"])) < 1e-15


def test_lattice_turbulence_scales():
    s = config.lattice_turbulence(12.0, 1.0, 0.472, 0.2)
    assert abs(s["tau_eta"] - 3878.2) < 0.1
    assert abs(s["a_rms"] - 2.5785e-4) < 1e-7
    assert s["n_hold"] == 379
    assert abs(s["sigma"] - 2.5785e-3) < 1e-6


def test_ou_generator_statistics():
    dt, T, a = 1.0, 10.0, 2e-3
    A = inputs.ou_gradients(5, 40000, dt, T, a)
    tr = A[:, 0, 0] + A[:, 1, 1] + A[:, 2, 2]
    assert np.abs(tr).max() < 1e-17
    rms = np.sqrt((A * A).sum((1, 2)).mean())
    assert abs(rms / a - 1) < 0.03
    x = A[:, 0, 1]
    rho1 = (x[1:] * x[:-1]).mean() / (x * x).mean()
    assert abs(rho1 - np.exp(-dt / T)) < 0.02
    assert np.array_equal(A, inputs.ou_gradients(5, 40000, dt, T, a))


def test_workloads():
    w = config.single_droplet_128()
    assert w.n == (128, 128, 128) and w.level == 4 and w.R == 12.0
    assert w.frames.shape[0] * w.n_hold >= w.steps
    members = inputs.ensemble_members()
    assert len(members) == 64
    for m in members:
        assert 48 <= m["L"] <= 96 and m["L"] % 8 == 0 and m["L"] >= 6 * m["R"]
        assert 6 <= m["R"] <= 10 and m["level"] == (3 if m["R"] < 8 else 4)
    t = config.taylor_shear_fp64()
    assert t.precision == "fp64" and abs(t.frames[0, 0, 2] - 1 / 6 * 0.472 ** 2 / 25) < 1e-15
