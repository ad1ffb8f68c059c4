"""Shape statistics of droplets along many synthetic gradient trajectories,
the synthetic analogue of the paper's ensemble results (Sec. 4: the
distributions of lambda_max/R^2 and of the orientation beta of Eq. (beta)
over many Lagrangian trajectories, compared with the linear theory of
Eq. (LT)).  Each trajectory drives one IBLB droplet; all droplets step as
one batched ensemble on the GPU, and the linear theory runs along the same
frames.  This module only sets the runs up and collects their records: the
droplet steps run in the library's kernels, the theory in its integrator."""
from __future__ import annotations

import numpy as np

from . import config, inputs


def trajectories(n_members: int, n_frames: int, Ca: float, R: float = 6.0, box: int = 48, level: int = 3,
                 seed: int = 900, R_over_eta: float = 0.472, tau: float = 1.0, reg_every: int = 10,
                 keep_volume: bool = True, recentre: bool = True, device=None):
    """Runs n_members IBLB droplets (box^3, radius R, icosphere level, rms
    capillary number Ca at R/eta, seeded OU gradients, one per droplet) for
    n_frames gradient frames each, and the linear theory (chi = 1) along the
    same frames.  Over trajectories of many frames the droplet needs the
    mesh regularisation of Sec. 3.3 (here every reg_every steps, with the
    paper's parameters, and by default restoring the volume each time) and
    the boundary field centred on its centre of mass (Sec. 3.2), else the
    mesh degrades and leaks volume and the droplet drifts into a wall.
    Returns a dict of (n_members, n_frames) arrays of lambda_max/R^2 and beta
    at the end of every frame ("iblb_lam", "iblb_beta", "lt_lam", "lt_beta")
    and the run parameters."""
    import torch

    from .sim import Ensemble, Sim
    from .theory import linear_theory

    s = config.lattice_turbulence(R, tau, R_over_eta, Ca)
    hold = s["n_hold"]
    tau_eta = s["tau_eta"]
    frames = inputs.ou_gradients_batch(seed, n_members, n_frames + 1, float(hold), 20.0 * tau_eta, s["a_rms"])
    sims = []
    for k in range(n_members):
        g = Sim((box,) * 3, tau, frames[k], hold, device=device)
        g.add_icosphere(level, R, s["sigma"])
        g.set_readout(hold)
        if reg_every > 0:
            g.set_regularization(every=reg_every)
            g.set_regularization_keep_volume(keep_volume)
        if recentre:
            g.set_recentring(True)
        sims.append(g)
    E = Ensemble(sims)
    E.step(n_frames * hold)
    E.sync()
    lam = np.empty((n_members, n_frames))
    beta = np.empty((n_members, n_frames))
    for k, g in enumerate(sims):
        ser = g.series(n_frames + 8)[:n_frames]
        assert [x["step"] for x in ser] == [hold * (j + 1) for j in range(n_frames)]
        lam[k] = [x["lam"][2] / (R * R) for x in ser]
        beta[k] = [x["beta"] for x in ser]
    E.close()
    for g in sims:
        g.close()
    lt = linear_theory(torch.as_tensor(frames[:, :n_frames]), Ca * tau_eta, R, float(hold), 1.0, substeps=8,
                       device=device).cpu().numpy()
    return {"iblb_lam": lam, "iblb_beta": beta, "lt_lam": lt[..., 6], "lt_beta": lt[..., 7], "hold": hold,
            "tau_eta": tau_eta, "sigma": s["sigma"], "R": R, "box": box, "Ca": Ca, "seed": seed,
            "reg_every": reg_every, "keep_volume": keep_volume, "recentre": recentre}


def quantiles(res: dict, skip: int, q=(5, 25, 50, 75, 95)) -> dict:
    """Quantiles over members and frames (after the first `skip` frames) of
    lambda_max/R^2 and beta for the IBLB droplets and the linear theory."""
    out = {}
    for key in ("iblb_lam", "iblb_beta", "lt_lam", "lt_beta"):
        v = res[key][:, skip:].ravel()
        v = v[np.isfinite(v)]
        out[key] = [float(x) for x in np.percentile(v, q)]
    return out
