"""ctypes declarations of libiblb (include/iblb.h).  Argument marshalling
only; the library must have been built in-tree (``__graft_entry__.build()``
or ``python -m paper_2403_01161_gb300.build``).  There is no fallback: a
missing library raises."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libiblb.so")

IBL_ABI_VERSION = 1
IBL_OK, IBL_EINVAL, IBL_ENOMEM, IBL_ECUDA, IBL_EUNSTABLE, IBL_ENOCONV, IBL_EWALL, IBL_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
BC_ZOU_HE, BC_PERIODIC = 0, 1
EDGE_COUNTER_SLIP, EDGE_PAPER_LITERAL = 0, 1
FP32_DEV, FP64 = 0, 1
ENSEMBLE_SHAPES = 32
ERRBIT_UNSTABLE, ERRBIT_NOCONV, ERRBIT_WALL = 1, 2, 4


class LbParams(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int), ("n", ctypes.c_int * 3), ("tau", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("edge_rule", ctypes.c_int), ("precision", ctypes.c_int),
                ("record_fields", ctypes.c_int)]


class Observables(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("frame", ctypes.c_int), ("reg_iters", ctypes.c_int),
                ("err", ctypes.c_int), ("pad_", ctypes.c_int), ("volume", ctypes.c_double),
                ("area", ctypes.c_double), ("centroid", ctypes.c_double * 3), ("S", ctypes.c_double * 6),
                ("lam", ctypes.c_double * 3), ("vmax", ctypes.c_double * 3), ("D", ctypes.c_double),
                ("beta", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"step": self.step, "frame": self.frame, "reg_iters": self.reg_iters, "err": self.err,
                "V": self.volume, "area": self.area, "xc": list(self.centroid), "S6": list(self.S),
                "lam": list(self.lam), "vmax": list(self.vmax), "D": self.D, "beta": self.beta}


class IblError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libiblb error %d: %s" % (code, msg))
        self.code = code


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_SZ = ctypes.POINTER(ctypes.c_size_t)

# (name, restype, argtypes)
SIGNATURES = [
    ("ibl_lb_workspace_size", ctypes.c_int, [ctypes.POINTER(LbParams), ctypes.c_int, _SZ]),
    ("ibl_lb_create", ctypes.c_int, [ctypes.POINTER(LbParams), _D, ctypes.c_int, ctypes.c_int, _P, ctypes.c_size_t,
                                     _P, ctypes.POINTER(_P)]),
    ("ibl_lb_destroy", None, [_P]),
    ("ibl_set_frame", ctypes.c_int, [_P, ctypes.c_int, _D]),
    ("ibl_icosphere_size", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("ibl_icosphere", ctypes.c_int, [ctypes.c_int, ctypes.c_double, _D, _D, _I32]),
    ("ibl_mesh_workspace_size", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _SZ]),
    ("ibl_mesh_create_icosphere", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _P,
                                                 ctypes.c_size_t, ctypes.POINTER(_P)]),
    ("ibl_mesh_create", ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.c_int, _I32, ctypes.c_double, _P,
                                       ctypes.c_size_t, ctypes.POINTER(_P)]),
    ("ibl_mesh_destroy", None, [_P]),
    ("ibl_set_regularization", ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int]),
    ("ibl_set_readout", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_set_regularization_trigger", ctypes.c_int, [_P, ctypes.c_double]),
    ("ibl_regularization_stats", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _D]),
    ("ibl_set_regularization_keep_volume", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_set_recentring", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_set_viscosity_ratio", ctypes.c_int, [_P, ctypes.c_double]),
    ("ibl_save", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("ibl_load", ctypes.c_int, [_P, ctypes.c_char_p]),
    ("ibl_step", ctypes.c_int, [_P, ctypes.c_longlong]),
    ("ibl_prepare_steps", ctypes.c_int, [_P, ctypes.c_longlong]),
    ("ibl_set_outside_update", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_outside_update", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("ibl_test_stage_timeout", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_step_record", ctypes.c_int, [_P]),
    ("ibl_set_graphs", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_step_paths", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    ("ibl_sync", ctypes.c_int, [_P]),
    ("ibl_steps_done", ctypes.c_longlong, [_P]),
    ("ibl_readout", ctypes.c_int, [_P, ctypes.POINTER(Observables)]),
    ("ibl_read_series", ctypes.c_int, [_P, ctypes.POINTER(Observables), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("ibl_copy_fields", ctypes.c_int, [_P, _D, _D, _D]),
    ("ibl_copy_populations", ctypes.c_int, [_P, _D]),
    ("ibl_copy_mesh", ctypes.c_int, [_P, _D, _D, _I32]),
    ("ibl_copy_neighbours", ctypes.c_int, [_P, _I32, _I32, ctypes.POINTER(ctypes.c_int)]),
    ("ibl_regularize_now", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("ibl_regularize_noalloc", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P]),
    ("ibl_run_frames", ctypes.c_int, [_P, _P, _D, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Observables)]),
    ("ibl_adjoint_workspace_size", ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_int, _SZ]),
    ("ibl_adjoint", ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_int, _P, ctypes.c_size_t, _D, _D, _D, _D]),
    ("ibl_linear_theory", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, _P, _P]),
    ("ibl_ensemble_workspace_size", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), _SZ]),
    ("ibl_ensemble_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), _P, ctypes.c_size_t,
                                           ctypes.POINTER(_P)]),
    ("ibl_ensemble_step", ctypes.c_int, [_P, ctypes.c_longlong]),
    ("ibl_ensemble_sync", ctypes.c_int, [_P]),
    ("ibl_ensemble_tune", ctypes.c_int, [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    ("ibl_ensemble_set_shape", ctypes.c_int, [_P, ctypes.c_int]),
    ("ibl_ensemble_shape", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    ("ibl_ensemble_destroy", None, [_P]),
    ("ibl_patch", ctypes.c_int, [_P, _I32, _I32]),
    ("ibl_velocity_set", ctypes.c_int, [_I32, _D]),
    ("ibl_profile_enable", ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    ("ibl_profile_read", ctypes.c_int, [_P, _D, ctypes.POINTER(ctypes.c_longlong)]),
    ("ibl_last_error", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libiblb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("libiblb.so is not built (%s); run __graft_entry__.build()" % path)
            L = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code: int):
    if code != IBL_OK:
        raise IblError(code, load().ibl_last_error().decode(errors="replace"))
    return code
