"""The C-ABI library builds, loads and exports every symbol include/iblb.h
declares; host-only entry points agree with the oracle.  No GPU needed (no
kernel is launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_01161_gb300 import build, _lib

    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "iblb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibl_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 28
    for n in names:
        assert hasattr(lib, n), n
    from paper_2403_01161_gb300 import _lib as L
    assert {s[0] for s in L.SIGNATURES} == set(names)


def test_velocity_set_matches_oracle(lib):
    from paper_2403_01161_gb300.sim import velocity_set

    c, w = velocity_set()
    co, wo = O.velocities(), O.weights()
    assert {tuple(v) for v in c} == {tuple(v) for v in co}
    lookup = {tuple(v): wo[i] for i, v in enumerate(co)}
    for i in range(19):
        assert w[i] == lookup[tuple(c[i])]


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_icosphere_bit_exact_against_oracle(lib, level):
    """Same mesh convention, two independent implementations: connectivity
    identical, positions equal to rounding."""
    from paper_2403_01161_gb300.sim import icosphere

    center = (15.5, 16.0, 17.25)
    r, t = icosphere(level, 7.0, center)
    ro, to = O.icosphere(level, 7.0, center)
    assert np.array_equal(t, to)
    assert np.abs(r - ro).max() < 1e-13


def test_argument_validation(lib):
    from paper_2403_01161_gb300 import _lib as L

    p = L.LbParams()
    p.version = L.IBL_ABI_VERSION
    for a in range(3):
        p.n[a] = 16
        p.bc[a] = L.BC_ZOU_HE
    p.tau = 1.0
    sz = ctypes.c_size_t()
    assert lib.ibl_lb_workspace_size(ctypes.byref(p), 3, ctypes.byref(sz)) == L.IBL_OK
    assert sz.value >= 19 * 16 ** 3 * 4 + 6 * 16 ** 3 * 4
    p.precision = L.FP64
    sz64 = ctypes.c_size_t()
    assert lib.ibl_lb_workspace_size(ctypes.byref(p), 3, ctypes.byref(sz64)) == L.IBL_OK
    assert sz64.value > sz.value
    p.n[1] = 2
    assert lib.ibl_lb_workspace_size(ctypes.byref(p), 3, ctypes.byref(sz)) == L.IBL_EINVAL
    assert b"invalid" in lib.ibl_last_error()
    p.n[1] = 16
    p.version = 99
    assert lib.ibl_lb_workspace_size(ctypes.byref(p), 3, ctypes.byref(sz)) == L.IBL_EINVAL
    nv, nt = ctypes.c_int(), ctypes.c_int()
    assert lib.ibl_icosphere_size(5, ctypes.byref(nv), ctypes.byref(nt)) == L.IBL_OK
    assert (nv.value, nt.value) == (10242, 20480)
    assert lib.ibl_icosphere_size(-1, ctypes.byref(nv), ctypes.byref(nt)) == L.IBL_EINVAL
    assert lib.ibl_set_recentring(None, 1) == L.IBL_EINVAL  # no mesh handle
    assert lib.ibl_set_viscosity_ratio(None, 2.0) == L.IBL_EINVAL
    assert lib.ibl_save(None, b"x") == L.IBL_EINVAL and lib.ibl_load(None, b"x") == L.IBL_EINVAL
    msz = ctypes.c_size_t()
    assert lib.ibl_mesh_workspace_size(2562, 5120, ctypes.byref(msz)) == L.IBL_OK
    assert msz.value > 2562 * 3 * 8 * 5
