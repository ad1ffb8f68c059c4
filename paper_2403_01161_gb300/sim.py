"""Python face of libiblb: a lattice with an optional droplet, stepping on a
torch CUDA stream, with device workspaces allocated as torch tensors.
Every step of the method runs in the library's CUDA kernels; this module
only marshals arguments and owns the torch buffers."""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def velocity_set():
    """(c (19,3) int32, w (19,) float64) in the library's population order."""
    lib = L.load()
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    L.check(lib.ibl_velocity_set(_ip(c), _dp(w)))
    return c, w


def icosphere_size(level: int):
    lib = L.load()
    nv, nt = ctypes.c_int(), ctypes.c_int()
    L.check(lib.ibl_icosphere_size(level, ctypes.byref(nv), ctypes.byref(nt)))
    return nv.value, nt.value


def icosphere(level: int, R: float = 1.0, center=(0.0, 0.0, 0.0)):
    """The library's icosphere (host only): positions (nv,3), triangles (nt,3)."""
    lib = L.load()
    nv, nt = icosphere_size(level)
    r = np.zeros((nv, 3))
    t = np.zeros((nt, 3), dtype=np.int32)
    c = np.ascontiguousarray(center, dtype=np.float64)
    L.check(lib.ibl_icosphere(int(level), float(R), _dp(c), _dp(r), _ip(t)))
    return r, t


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


class Sim:
    """IBLB box of n = (nx, ny, nz) lattice nodes.

    frames: (n_frames, 3, 3) velocity gradients (row a = du_a/dx_b, lattice
    units), frame k applied for steps [k*n_hold, (k+1)*n_hold).
    """

    def __init__(self, n: Sequence[int], tau: float, frames, n_hold: int, *, bc=(L.BC_ZOU_HE,) * 3,
                 precision: str = "fp32", edge_rule: int = L.EDGE_COUNTER_SLIP, record_fields: bool = False,
                 device=None, stream: Optional[torch.cuda.Stream] = None):
        self.lib = L.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n = tuple(int(v) for v in n)
        self.nodes = self.n[0] * self.n[1] * self.n[2]
        fr = np.ascontiguousarray(np.asarray(frames, dtype=np.float64).reshape(-1, 9))
        self.n_frames = fr.shape[0]
        self.n_hold = int(n_hold)
        p = L.LbParams()
        p.version = L.IBL_ABI_VERSION
        for a in range(3):
            p.n[a] = self.n[a]
            p.bc[a] = int(bc[a])
        p.tau = float(tau)
        p.edge_rule = int(edge_rule)
        p.precision = L.FP64 if precision == "fp64" else L.FP32_DEV
        p.record_fields = 1 if record_fields else 0
        self.params = p
        nbytes = ctypes.c_size_t()
        L.check(self.lib.ibl_lb_workspace_size(ctypes.byref(p), self.n_frames, ctypes.byref(nbytes)))
        self.ws = _workspace(nbytes.value, self.device)
        h = ctypes.c_void_p()
        L.check(self.lib.ibl_lb_create(ctypes.byref(p), _dp(fr), self.n_frames, self.n_hold,
                                       ctypes.c_void_p(self.ws.data_ptr()), nbytes.value,
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.mesh_h = None
        self.mesh_ws = None
        self.nv = self.nt = 0

    # ---- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "mesh_h", None):
            self.lib.ibl_mesh_destroy(self.mesh_h)
            self.mesh_h = None
        if getattr(self, "h", None):
            self.lib.ibl_lb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- droplet -----------------------------------------------------------
    def add_icosphere(self, level: int, R: float, sigma: float, center=None):
        self.nv, self.nt = icosphere_size(level)
        self._alloc_mesh()
        c = None if center is None else np.ascontiguousarray(center, dtype=np.float64)
        h = ctypes.c_void_p()
        L.check(self.lib.ibl_mesh_create_icosphere(self.h, int(level), float(R), float(sigma),
                                                   _dp(c) if c is not None else None,
                                                   ctypes.c_void_p(self.mesh_ws.data_ptr()),
                                                   self.mesh_ws.numel(), ctypes.byref(h)))
        self.mesh_h = h
        return self

    def add_mesh(self, r, tris, sigma: float):
        r = np.ascontiguousarray(r, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        self.nv, self.nt = r.shape[0], t.shape[0]
        self._alloc_mesh()
        h = ctypes.c_void_p()
        L.check(self.lib.ibl_mesh_create(self.h, self.nv, _dp(r), self.nt, _ip(t), float(sigma),
                                         ctypes.c_void_p(self.mesh_ws.data_ptr()), self.mesh_ws.numel(),
                                         ctypes.byref(h)))
        self.mesh_h = h
        return self

    def _alloc_mesh(self):
        nbytes = ctypes.c_size_t()
        L.check(self.lib.ibl_mesh_workspace_size(self.nv, self.nt, ctypes.byref(nbytes)))
        self.mesh_ws = _workspace(nbytes.value, self.device)

    def set_regularization(self, alpha=0.1, gamma=0.51, tol=0.01, max_iter=100, every=0, plus_sign=True):
        L.check(self.lib.ibl_set_regularization(self.mesh_h, alpha, gamma, tol, max_iter, every,
                                                1 if plus_sign else 0))

    def set_regularization_trigger(self, max_edge_ratio: float):
        """Smooth at a scheduled step only when the mesh quality (max over
        triangles of longest/shortest edge) exceeds max_edge_ratio; 0 = always."""
        L.check(self.lib.ibl_set_regularization_trigger(self.mesh_h, float(max_edge_ratio)))

    def set_regularization_keep_volume(self, keep: bool):
        """Rescale the mesh after every regularisation to the volume it
        enclosed before (about its volume centroid)."""
        L.check(self.lib.ibl_set_regularization_keep_volume(self.mesh_h, 1 if keep else 0))

    def set_recentring(self, on: bool = True):
        """Centre the linear boundary field of every step on the droplet's
        centre of mass (volume centroid at the start of the step) instead of
        the box centre (Sec. 3.2)."""
        L.check(self.lib.ibl_set_recentring(self.mesh_h, 1 if on else 0))

    def set_viscosity_ratio(self, chi: float):
        """Droplet viscosity chi times the carrier's (Sec. 2): nodes inside the
        droplet relax with tau_in = 1/2 + chi (tau - 1/2).  Needs Zou-He walls
        on every axis; 1 switches it off."""
        L.check(self.lib.ibl_set_viscosity_ratio(self.mesh_h, float(chi)))

    def regularization_stats(self):
        """(regularisations performed, mesh quality at the latest check)."""
        n = ctypes.c_int()
        q = np.zeros(1)
        L.check(self.lib.ibl_regularization_stats(self.mesh_h, ctypes.byref(n), _dp(q)))
        return n.value, float(q[0])

    def set_readout(self, every: int):
        L.check(self.lib.ibl_set_readout(self.mesh_h, int(every)))

    # ---- stepping ----------------------------------------------------------
    def step(self, n: int = 1):
        L.check(self.lib.ibl_step(self.h, int(n)))

    def prepare(self, n: int):
        """Capture (without running) the graphs the next step(n) replays."""
        L.check(self.lib.ibl_prepare_steps(self.h, int(n)))

    def set_outside_update(self, kind: int):
        """Kernel of the update outside the droplet patch: 0 direct loads,
        1..2 the staged shared-memory pipeline in one of its launch shapes."""
        L.check(self.lib.ibl_set_outside_update(self.h, int(kind)))

    @property
    def outside_update(self) -> int:
        k = ctypes.c_int()
        L.check(self.lib.ibl_outside_update(self.h, ctypes.byref(k)))
        return k.value

    def set_graphs(self, enable: bool):
        """Replay whole chunks of steps as a captured CUDA graph (default on)."""
        L.check(self.lib.ibl_set_graphs(self.h, 1 if enable else 0))

    def step_paths(self):
        """(steps run eagerly, steps run by graph replay) by step() so far."""
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        L.check(self.lib.ibl_step_paths(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def step_record(self):
        L.check(self.lib.ibl_step_record(self.h))

    def sync(self):
        L.check(self.lib.ibl_sync(self.h))

    def save(self, path: str):
        """Write the dynamic state between steps to `path` (ibl_save)."""
        L.check(self.lib.ibl_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        """Resume from a file written by `save` for a Sim built the same way
        (box, boundaries, precision, tau, frames, mesh size); settings such as
        the regularisation schedule are applied to this Sim as before."""
        L.check(self.lib.ibl_load(self.h, os.fsencode(path)))

    def status(self) -> int:
        """Synchronise and return the status code instead of raising."""
        return self.lib.ibl_sync(self.h)

    @property
    def steps_done(self) -> int:
        return int(self.lib.ibl_steps_done(self.h))

    def set_frame(self, k: int, A):
        a = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
        L.check(self.lib.ibl_set_frame(self.h, int(k), _dp(a)))
        self.sync()

    # ---- readout -----------------------------------------------------------
    def readout(self) -> dict:
        o = L.Observables()
        L.check(self.lib.ibl_readout(self.mesh_h, ctypes.byref(o)))
        return o.as_dict()

    def series(self, max_records: int = 4096, allow_error: bool = False):
        """The shape-record ring, oldest first.  With allow_error the records
        are returned even when the lattice carries a sticky device error
        (each record holds the error bits of its own step)."""
        buf = (L.Observables * max_records)()
        cnt = ctypes.c_int()
        st = self.lib.ibl_read_series(self.mesh_h, buf, max_records, ctypes.byref(cnt))
        if not (allow_error and st in (L.IBL_EUNSTABLE, L.IBL_ENOCONV, L.IBL_EWALL, L.IBL_ETIMEOUT)):
            L.check(st)
        return [buf[k].as_dict() for k in range(cnt.value)]

    def fields(self):
        """(rho, u, F) of the last step_record(): (nz,ny,nx), (3,nz,ny,nx) x2."""
        rho = np.zeros(self.nodes)
        u = np.zeros(3 * self.nodes)
        F = np.zeros(3 * self.nodes)
        L.check(self.lib.ibl_copy_fields(self.h, _dp(rho), _dp(u), _dp(F)))
        nx, ny, nz = self.n
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx), F.reshape(3, nz, ny, nx)

    def populations(self):
        """Pre-collision f of the next step, (19, nz, ny, nx), library order."""
        f = np.zeros(19 * self.nodes)
        L.check(self.lib.ibl_copy_populations(self.h, _dp(f)))
        nx, ny, nz = self.n
        return f.reshape(19, nz, ny, nx)

    def mesh(self):
        """(positions (nv,3), nodal forces of the last step (nv,3), triangles (nt,3))."""
        r = np.zeros((self.nv, 3))
        F = np.zeros((self.nv, 3))
        t = np.zeros((self.nt, 3), dtype=np.int32)
        L.check(self.lib.ibl_copy_mesh(self.mesh_h, _dp(r), _dp(F), _ip(t)))
        return r, F, t

    def neighbours(self):
        ptr = np.zeros(self.nv + 1, dtype=np.int32)
        nnz = ctypes.c_int()
        L.check(self.lib.ibl_copy_neighbours(self.mesh_h, _ip(ptr), None, ctypes.byref(nnz)))
        idx = np.zeros(nnz.value, dtype=np.int32)
        L.check(self.lib.ibl_copy_neighbours(self.mesh_h, None, _ip(idx), ctypes.byref(nnz)))
        return ptr, idx

    def regularize_now(self) -> int:
        it = ctypes.c_int()
        L.check(self.lib.ibl_regularize_now(self.mesh_h, ctypes.byref(it)))
        return it.value

    def run_frames(self, frames, steps_per_frame: int):
        """Sec. 3.2 trajectory loop with host buffers (synchronising per frame)."""
        fr = np.ascontiguousarray(np.asarray(frames, dtype=np.float64).reshape(-1, 9))
        out = (L.Observables * fr.shape[0])()
        L.check(self.lib.ibl_run_frames(self.h, self.mesh_h, _dp(fr), fr.shape[0], int(steps_per_frame), out))
        return [out[k].as_dict() for k in range(fr.shape[0])]

    def adjoint(self, n_steps: int, K: int = 100) -> dict:
        """Runs n_steps steps from step 0 and returns the Taylor deformation D
        of the final droplet with its gradients by the library's discrete
        adjoint (checkpoint every K steps, recomputation per segment):
        {"D", "dD_dsigma", "dD_dA" (n_frames, 3, 3), "dD_dr0" (nv, 3)}.
        Leaves the box at step n_steps."""
        nbytes = ctypes.c_size_t()
        L.check(self.lib.ibl_adjoint_workspace_size(self.h, int(n_steps), int(K), ctypes.byref(nbytes)))
        ws = _workspace(nbytes.value, self.device)
        D = np.zeros(1)
        ds = np.zeros(1)
        dA = np.zeros(9 * self.n_frames)
        dr = np.zeros(3 * self.nv)
        L.check(self.lib.ibl_adjoint(self.h, int(n_steps), int(K), ctypes.c_void_p(ws.data_ptr()), nbytes.value,
                                     _dp(D), _dp(ds), _dp(dA), _dp(dr)))
        del ws
        return {"D": float(D[0]), "dD_dsigma": float(ds[0]), "dD_dA": dA.reshape(self.n_frames, 3, 3),
                "dD_dr0": dr.reshape(self.nv, 3)}

    def patch(self):
        """(lo (3,), ext (3,)) of the droplet patch of the next step."""
        lo = np.zeros(3, dtype=np.int32)
        ext = np.zeros(3, dtype=np.int32)
        L.check(self.lib.ibl_patch(self.h, _ip(lo), _ip(ext)))
        return lo, ext

    # ---- timing --------------------------------------------------------------
    def profile(self, enable, mask: int = 7, every: int = 1):
        """Time kernels with CUDA events (mask bit 0 lattice, 1 spread, 2 interpolation;
        bit 3: only launches inside replayed graph chunks), one launch in `every`."""
        L.check(self.lib.ibl_profile_enable(self.h, mask if enable else 0, int(every)))

    def profile_read(self):
        ms = np.zeros(3)
        cnt = (ctypes.c_longlong * 3)()
        L.check(self.lib.ibl_profile_read(self.h, _dp(ms), cnt))
        return {"lattice": (float(ms[0]), int(cnt[0])), "spread": (float(ms[1]), int(cnt[1])),
                "interp": (float(ms[2]), int(cnt[2]))}


class Ensemble:
    """Droplets advanced together by batched kernels (one launch per phase
    for all members).  members: Sim objects, each with a droplet, same
    precision and stream, same step count.  The members stay alive with the
    ensemble and keep their per-member readouts."""

    def __init__(self, members):
        self.lib = L.load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        self._arr = arr
        nbytes = ctypes.c_size_t()
        L.check(self.lib.ibl_ensemble_workspace_size(len(self.members), arr, ctypes.byref(nbytes)))
        self.ws = _workspace(nbytes.value, self.members[0].device)
        h = ctypes.c_void_p()
        L.check(self.lib.ibl_ensemble_create(len(self.members), arr, ctypes.c_void_p(self.ws.data_ptr()),
                                             nbytes.value, ctypes.byref(h)))
        self.h = h

    def step(self, n: int = 1):
        L.check(self.lib.ibl_ensemble_step(self.h, int(n)))

    def sync(self):
        L.check(self.lib.ibl_ensemble_sync(self.h))

    def tune(self, steps_per_candidate: int = 8):
        """Autotunes the launch shape of the batched lattice update by timing
        real ensemble steps with each candidate (the members advance by
        ENSEMBLE_SHAPES * (steps_per_candidate + 2) steps); returns
        (chosen shape, ms per step of every candidate)."""
        ms = np.zeros(L.ENSEMBLE_SHAPES)
        k = ctypes.c_int()
        L.check(self.lib.ibl_ensemble_tune(self.h, int(steps_per_candidate), _dp(ms), ctypes.byref(k)))
        return k.value, ms

    def set_shape(self, shape: int):
        L.check(self.lib.ibl_ensemble_set_shape(self.h, int(shape)))

    def shape(self):
        """(shape index, threads per block, prefetch distance in waves)."""
        k, t, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(self.lib.ibl_ensemble_shape(self.h, ctypes.byref(k), ctypes.byref(t), ctypes.byref(w)))
        return k.value, t.value, w.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibl_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
