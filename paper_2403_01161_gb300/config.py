"""Parameter mapping of Sec. 3.2 of arXiv:2403.01161 and the synthetic
workloads the library is measured and tested on.

Units (Sec. 3.2): a quantity A in DNS units equals A_LBU * C_A.  With the
droplet radius fixing the length scale, C_x = R / R_LBU (Eq. (cl)); the
viscosity fixes time, C_t = C_x^2 nu_LBU / nu (Eq. (ct)); gradients convert
as (grad u)_LBU = C_t grad u (Eq. (strain_conversion)); each gradient frame
is held N = dt / C_t lattice steps (Eq. (N_Reta)); and the surface tension
follows from the capillary number Ca = tau_sigma / tau_eta (Eq. (capillary))
as sigma_LBU = mu_LBU R_LBU / tau_sigma,LBU (Eq. (surfacetensionconversion)).
In lattice units nu_LBU = (tau_f - 1/2)/3 (Eq. (tau_to_nu)) and mu = rho nu
with rho = 1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Tuple

import numpy as np

from . import inputs

# TURB-Lagr values in DNS units, Sec. 3.2
DNS = {"eta": 4.2e-3, "tau_eta": 2.3e-2, "nu": 8e-4, "epsilon": 1.4, "dt_frame": 2.25e-3}


def nu_lbu(tau_f: float) -> float:
    """Eq. (tau_to_nu): nu = c_s^2 (tau_f - 1/2), c_s^2 = 1/3."""
    return (tau_f - 0.5) / 3.0


def dns_to_lbu(R_over_eta: float, R_lbu: float, tau_f: float, Ca: float, dns=DNS) -> dict:
    """Conversion factors and lattice parameters of Sec. 3.2 for a droplet of
    radius R = (R/eta) eta in DNS units drawn with R_lbu lattice units."""
    nu_l = nu_lbu(tau_f)
    R = R_over_eta * dns["eta"]
    C_x = R / R_lbu                                  # Eq. (cl)
    C_t = C_x ** 2 * nu_l / dns["nu"]                # Eq. (ct)
    N = dns["dt_frame"] / C_t                        # steps per frame
    tau_sigma = Ca * dns["tau_eta"]                  # Eq. (capillary)
    tau_sigma_l = tau_sigma / C_t
    sigma_l = nu_l * R_lbu / tau_sigma_l             # Eq. (surfacetensionconversion), mu = rho nu
    return {"C_x": C_x, "C_t": C_t, "N": N, "tau_sigma_lbu": tau_sigma_l, "sigma_lbu": sigma_l,
            "tau_eta_lbu": dns["tau_eta"] / C_t, "grad_scale": C_t}


def lattice_turbulence(R: float, tau_f: float, R_over_eta: float, Ca_rms: float) -> dict:
    """Lattice-unit scales of a sub-Kolmogorov droplet of radius R (lattice
    units): tau_eta = R^2 / (nu (R/eta)^2) (from eta^2 = nu tau_eta), rms
    gradient 1/tau_eta (epsilon = nu <grad u : grad u>, Sec. 2), frame interval
    dt_frame/tau_eta of the DNS, and sigma = mu R / (Ca tau_eta)."""
    nu = nu_lbu(tau_f)
    tau_eta = R * R / (nu * R_over_eta ** 2)
    dt = DNS["dt_frame"] / DNS["tau_eta"] * tau_eta
    return {"nu": nu, "tau_eta": tau_eta, "a_rms": 1.0 / tau_eta, "dt_frame": dt,
            "n_hold": max(1, int(round(dt))), "sigma": nu * R / (Ca_rms * tau_eta)}


@dataclasses.dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    tau: float
    level: int
    R: float
    sigma: float
    frames: np.ndarray            # (n_frames, 3, 3), lattice units
    n_hold: int
    steps: int
    precision: str = "fp32"       # "fp32" (FP32 deviations) or "fp64"
    reg_every: int = 0            # 0: no mesh regularisation
    readout_every: int = 100
    center: Optional[Tuple[float, float, float]] = None

    @property
    def nodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def _ou_workload(name, N, R, level, seed, steps, R_over_eta=0.472, Ca_rms=0.2, tau=1.0,
                 T_over_tau_eta=20.0, **kw) -> Workload:
    s = lattice_turbulence(R, tau, R_over_eta, Ca_rms)
    n_frames = steps // s["n_hold"] + 2
    frames = inputs.ou_gradients(seed, n_frames, s["n_hold"], T_over_tau_eta * s["tau_eta"], s["a_rms"])
    return Workload(name, (N, N, N), tau, level, R, s["sigma"], frames, s["n_hold"], steps, **kw)


def taylor_shear_fp64(N: int = 32, R: float = 5.0, Ca: float = 0.1, steps: int = 1000,
                      level: int = 3) -> Workload:
    """Steady simple shear on the box walls with shear rate 1/tau_eta at
    R/eta = 0.472 and sigma = mu R rate / Ca; FP64 populations."""
    nu = nu_lbu(1.0)
    rate = nu * 0.472 ** 2 / (R * R)
    sigma = nu * R * rate / Ca
    return Workload("taylor_shear_fp64", (N, N, N), 1.0, level, R, sigma, inputs.simple_shear(rate),
                    10 ** 9, steps, precision="fp64")


def single_droplet_128(steps: int = 20000) -> Workload:
    """128^3 box, R = 12, icosphere level 4, OU gradients (seed 2), rms Ca 0.2."""
    return _ou_workload("single_droplet_128", 128, 12.0, 4, 2, steps)


def precision_stress_256(steps: int = 5000, Ca_rms: float = 0.5) -> Workload:
    """256^3 box, R = 24, icosphere level 5, OU gradients (seed 4) at R/eta = 1,
    mesh regularisation every 50 steps."""
    return _ou_workload("precision_stress_256", 256, 24.0, 5, 4, steps, R_over_eta=1.0, Ca_rms=Ca_rms,
                        reg_every=50)


def production_200(steps: int = 2 * 1488, seed: int = 6, Ca: float = 0.2, R_over_eta: float = 0.472) -> Workload:
    """The paper's production setup (Sec. 3.2): 200^3 box, R = 19 lattice
    units, 20480-triangle mesh (icosphere level 5), tau_f = 1.5, with the DNS
    conversion of Eqs. (cl), (ct), (N_Reta), (capillary) and
    (surfacetensionconversion) at R/eta = 0.472: N = 496 steps per frame,
    rms gradient 1/tau_eta in lattice units, sigma from Ca.  OU gradients
    (seed) stand in for the database trajectory; one shape record per frame."""
    d = dns_to_lbu(R_over_eta, 19.0, 1.5, Ca)
    n_hold = int(round(d["N"]))
    tau_eta = d["tau_eta_lbu"]
    n_frames = steps // n_hold + 2
    frames = inputs.ou_gradients(seed, n_frames, n_hold, 20.0 * tau_eta, 1.0 / tau_eta)
    return Workload("production_200", (200, 200, 200), 1.5, 5, 19.0, d["sigma_lbu"], frames, n_hold, steps,
                    readout_every=n_hold)


def adjoint_member(seed: int, steps: int = 2000) -> Workload:
    """64^3 box, R = 8, icosphere level 3, OU gradients (seed), rms Ca 0.2."""
    return _ou_workload("adjoint_64_seed%d" % seed, 64, 8.0, 3, seed, steps)


def ensemble_workloads(n: int = 64, steps: int = 10000):
    """The uneven ensemble: per member its own box, radius, level and OU seed."""
    out = []
    for m in inputs.ensemble_members(n):
        out.append(_ou_workload("ensemble_seed%d" % m["seed"], m["L"], m["R"], m["level"], m["seed"],
                                steps))
    return out


def small_ou(N: int = 32, R: float = 5.0, level: int = 3, seed: int = 7, steps: int = 200,
             precision: str = "fp32", scale: float = 1.0, Ca_rms: float = 0.2, **kw) -> Workload:
    """A reduced-size OU workload for parity tests (gradients scaled by
    `scale` so that few steps still deform the droplet)."""
    w = _ou_workload("small_ou_%d" % N, N, R, level, seed, steps, Ca_rms=Ca_rms, precision=precision,
                     **kw)
    w.frames = w.frames * scale
    return w


def box_center(n) -> Tuple[float, float, float]:
    return tuple(0.5 * (k - 1) for k in n)


def total_frames_needed(steps: int, n_hold: int) -> int:
    return int(math.ceil(steps / max(1, n_hold)))
