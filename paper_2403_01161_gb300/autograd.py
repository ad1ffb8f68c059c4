"""torch.autograd face of the library's discrete adjoint: the Taylor
deformation D of a droplet after a trajectory, as a differentiable function
of the surface tension sigma and the velocity-gradient frames A_k.

The forward builds a box with an icosphere droplet (Sec. 3.1), runs the
trajectory through the library and, when a gradient is wanted, obtains
dD/dsigma and dD/dA_k in the same call by the library's checkpointed
adjoint sweep; backward only scales them by the incoming gradient."""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from .sim import Sim


@dataclass(frozen=True)
class DropletSpec:
    """One trajectory: box n, relaxation time tau, frames held n_hold steps
    each, icosphere of `level` and radius R at `center` (None = box centre),
    n_steps steps, adjoint checkpoint every K steps, storage precision."""
    n: Sequence[int]
    tau: float
    n_hold: int
    level: int
    R: float
    n_steps: int
    K: int = 100
    precision: str = "fp32"
    center: Optional[Sequence[float]] = None


def _run(spec: DropletSpec, sigma: float, frames: np.ndarray, want_grad: bool, device):
    s = Sim(spec.n, spec.tau, frames, spec.n_hold, precision=spec.precision, device=device)
    try:
        s.add_icosphere(spec.level, spec.R, sigma, center=spec.center)
        if want_grad:
            return s.adjoint(spec.n_steps, spec.K)
        s.step(spec.n_steps)
        return {"D": s.readout()["D"]}
    finally:
        s.close()


class DeformationFn(torch.autograd.Function):
    """D = DeformationFn.apply(sigma, frames, spec); sigma a scalar tensor,
    frames (n_frames, 3, 3) with frames[k, a, b] = du_a/dx_b of frame k."""

    @staticmethod
    def forward(ctx, sigma: torch.Tensor, frames: torch.Tensor, spec: DropletSpec):
        want = bool(sigma.requires_grad or frames.requires_grad)
        fr = frames.detach().to("cpu", torch.float64).numpy().reshape(-1, 3, 3)
        device = frames.device if frames.is_cuda else None
        out = _run(spec, float(sigma.detach().cpu()), fr, want, device)
        if want:
            ctx.save_for_backward(torch.tensor(out["dD_dsigma"], dtype=sigma.dtype, device=sigma.device),
                                  torch.as_tensor(out["dD_dA"], dtype=frames.dtype, device=frames.device))
        return torch.tensor(out["D"], dtype=torch.float64, device=frames.device)

    @staticmethod
    def backward(ctx, g):
        ds, dA = ctx.saved_tensors
        gs = (g.to(ds.dtype) * ds).to(ds.device) if ctx.needs_input_grad[0] else None
        gA = (g.to(dA.dtype).to(dA.device) * dA).reshape(dA.shape) if ctx.needs_input_grad[1] else None
        return gs, gA, None


def deformation(sigma: torch.Tensor, frames: torch.Tensor, spec: DropletSpec) -> torch.Tensor:
    return DeformationFn.apply(sigma, frames, spec)
