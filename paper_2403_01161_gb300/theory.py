"""Python face of the library's linear-theory integrator (Eq. (LT), Sec. 2):
many gradient trajectories at once on the GPU.  Argument marshalling only;
the integration runs in the library's kernel."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L

FIELDS = ("S_xx", "S_yy", "S_zz", "S_xy", "S_xz", "S_yz", "lam_max_R2", "beta", "D")


def linear_theory(frames, tau_sigma, R, hold, chi=1.0, substeps: int = 8, device=None, stream=None) -> torch.Tensor:
    """frames: (n_traj, n_frames, 3, 3) gradients (tensor or array; rows
    du_a/dx_b); tau_sigma, R, hold, chi: scalars or per-trajectory sequences.
    Returns a device tensor (n_traj, n_frames, 9) of S at each frame end and
    lambda_max/R^2, beta, D (see FIELDS)."""
    lib = L.load()
    dev = torch.device(device if device is not None else "cuda")
    A = frames if torch.is_tensor(frames) else torch.as_tensor(np.asarray(frames, dtype=np.float64))
    A = A.to(device=dev, dtype=torch.float64)
    if A.dim() == 3:
        A = A.unsqueeze(0)
    n_traj, n_frames = A.shape[0], A.shape[1]
    A = A.reshape(n_traj, n_frames, 9).contiguous()
    p = np.zeros((n_traj, 4))
    for j, v in enumerate((tau_sigma, R, chi, hold)):
        p[:, j] = np.broadcast_to(np.asarray(v, dtype=np.float64), (n_traj,))
    params = torch.as_tensor(p, dtype=torch.float64, device=dev).contiguous()
    out = torch.empty((n_traj, n_frames, 9), dtype=torch.float64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    L.check(lib.ibl_linear_theory(n_traj, n_frames, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(params.data_ptr()),
                                  int(substeps), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
    return out
