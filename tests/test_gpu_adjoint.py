"""Discrete adjoint of the droplet trajectory: dD/dsigma, dD/dA_k and dD/dr_0
against central finite differences of the forward (the library's FP64 path
and the oracle), over ragged checkpoint segments, periodic and Zou-He axes
and both edge rules; the FP32 adjoint against FP64 differences; the state
left behind; the error paths; the autograd wrapper."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from parity import frames_ou

pytestmark = pytest.mark.gpu

N = (24, 22, 26)
R, LEVEL, SIGMA = 4.5, 2, 0.02
N_HOLD, STEPS, K = 8, 30, 7  # 4 frames; segments 7, 7, 7, 7, 2


def _frames():
    return frames_ou(31, 4, 4e-3).reshape(4, 3, 3)


def _sim(precision="fp64", sigma=SIGMA, frames=None, r0=None, bc=(0, 0, 0), rule=0):
    from paper_2403_01161_gb300.sim import Sim

    fr = _frames() if frames is None else frames
    s = Sim(N, 1.0, fr, N_HOLD, bc=bc, precision=precision, edge_rule=rule)
    c = tuple(0.5 * (k - 1) for k in N)
    if r0 is None:
        s.add_icosphere(LEVEL, R, sigma, center=c)
    else:
        _, t = O.icosphere(LEVEL, R, c)
        s.add_mesh(r0, t, sigma)
    return s


def _D(**kw):
    s = _sim(**kw)
    s.step(STEPS)
    d = s.readout()["D"]
    assert s.status() == 0
    s.close()
    return d


def _fd(f, h):
    return (f(h) - f(-h)) / (2.0 * h)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def adj64():
    s = _sim()
    out = s.adjoint(STEPS, K)
    assert s.status() == 0
    s.close()
    return out


def test_adjoint_D_matches_forward_readout(adj64):
    assert abs(adj64["D"] - _D()) < 1e-13
    assert adj64["D"] > 1e-3  # the droplet has deformed


def test_dD_dsigma_fd_fp64(adj64):
    h = 1e-4 * SIGMA
    fd = _fd(lambda e: _D(sigma=SIGMA + e), h)
    assert abs(fd) > 1e-3
    assert abs(adj64["dD_dsigma"] - fd) <= 1e-6 * abs(fd)


def test_dD_dA_every_entry_fd_fp64(adj64):
    """All 36 frame entries, each by central differences."""
    fr = _frames()
    fd = np.zeros((4, 3, 3))
    h = 1e-6
    for k in range(4):
        for a in range(3):
            for b in range(3):
                def f(e, k=k, a=a, b=b):
                    p = fr.copy()
                    p[k, a, b] += e
                    return _D(frames=p)
                fd[k, a, b] = _fd(f, h)
    g = adj64["dD_dA"]
    assert np.abs(fd).max() > 1.0
    assert _rel(g, fd) < 1e-6, (g, fd)
    # entry by entry, relative to the largest entry of the same frame
    for k in range(4):
        assert np.abs(g[k] - fd[k]).max() <= 1e-6 * np.abs(fd[k]).max() + 1e-9


def test_dD_dr0_fd_fp64(adj64):
    """Initial node positions along three random unit directions."""
    r0, _ = O.icosphere(LEVEL, R, tuple(0.5 * (k - 1) for k in N))
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(r0.shape)
        v /= np.linalg.norm(v)
        fd = _fd(lambda e: _D(r0=r0 + e * v), 1e-5)
        ad = float((adj64["dD_dr0"] * v).sum())
        assert abs(ad - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.linalg.norm(adj64["dD_dr0"]))


@pytest.mark.parametrize("bc,rule", [((1, 0, 0), 0), ((0, 1, 1), 0), ((0, 0, 0), 1)])
def test_adjoint_fd_variants_fp64(bc, rule):
    """Periodic axes (wrapped streaming and stencils) and the literal edge
    rule: sigma and four random directions in frame space."""
    s = _sim(bc=bc, rule=rule)
    g = s.adjoint(STEPS, K)
    s.close()
    fd_s = _fd(lambda e: _D(sigma=SIGMA + e, bc=bc, rule=rule), 1e-4 * SIGMA)
    assert abs(g["dD_dsigma"] - fd_s) <= 1e-6 * abs(fd_s)
    fr = _frames()
    rng = np.random.default_rng(7)
    for _ in range(4):
        v = rng.standard_normal(fr.shape)
        v /= np.linalg.norm(v)
        fd = _fd(lambda e: _D(frames=fr + e * v, bc=bc, rule=rule), 1e-6)
        ad = float((g["dD_dA"] * v).sum())
        assert abs(ad - fd) <= 1e-6 * np.abs(g["dD_dA"]).sum() + 1e-9, (ad, fd)


def test_adjoint_against_oracle_fd(adj64):
    """The oracle's own FP64 trajectory, differenced in sigma and along one
    random frame direction: the GPU adjoint differentiates the paper's
    forward, not only the library's."""
    c = tuple(0.5 * (k - 1) for k in N)
    r0, t = O.icosphere(LEVEL, R, c)
    fr = _frames()

    def D_oracle(sigma, frames):
        o = O.OracleSim(N, 1.0, frames, N_HOLD)
        o.set_mesh(r0, t, sigma)
        o.step(STEPS)
        r, _ = o.mesh()
        o.close()
        return O.observables(r, t)["D"]

    h = 1e-4 * SIGMA
    fd_s = (D_oracle(SIGMA + h, fr) - D_oracle(SIGMA - h, fr)) / (2 * h)
    assert abs(adj64["dD_dsigma"] - fd_s) <= 1e-6 * abs(fd_s)
    v = np.random.default_rng(11).standard_normal(fr.shape)
    v /= np.linalg.norm(v)
    fd_v = (D_oracle(SIGMA, fr + 1e-6 * v) - D_oracle(SIGMA, fr - 1e-6 * v)) / 2e-6
    assert abs(float((adj64["dD_dA"] * v).sum()) - fd_v) <= 1e-6 * np.abs(adj64["dD_dA"]).sum()


def test_adjoint_fp32_against_fp64_fd(adj64):
    """FP32 storage: gradients within 1e-3 of the FP64 ones (which the tests
    above pin to finite differences)."""
    s = _sim(precision="fp32")
    g = s.adjoint(STEPS, K)
    s.close()
    assert abs(g["D"] - adj64["D"]) < 1e-4 * abs(adj64["D"])
    assert abs(g["dD_dsigma"] - adj64["dD_dsigma"]) <= 1e-3 * abs(adj64["dD_dsigma"])
    assert _rel(g["dD_dA"], adj64["dD_dA"]) < 1e-3
    assert _rel(g["dD_dr0"], adj64["dD_dr0"]) < 1e-3


def test_segment_length_does_not_change_the_gradient(adj64):
    for k in (1, 30, 100):
        s = _sim()
        g = s.adjoint(STEPS, k)
        s.close()
        assert abs(g["dD_dsigma"] - adj64["dD_dsigma"]) <= 1e-11 * abs(adj64["dD_dsigma"])
        assert _rel(g["dD_dA"], adj64["dD_dA"]) < 1e-11


def test_state_after_adjoint_is_the_forward_state():
    a = _sim()
    a.adjoint(STEPS, K)
    b = _sim()
    b.step(STEPS)
    assert a.steps_done == b.steps_done == STEPS
    ra, _, _ = a.mesh()
    rb, _, _ = b.mesh()
    assert np.abs(ra - rb).max() < 1e-12
    assert np.abs(a.populations() - b.populations()).max() < 1e-13
    a.step(5)
    b.step(5)
    assert abs(a.readout()["D"] - b.readout()["D"]) < 1e-12
    a.close()
    b.close()


def test_adjoint_error_paths():
    from paper_2403_01161_gb300 import _lib as L

    s = _sim()
    s.step(1)
    with pytest.raises(L.IblError) as e:
        s.adjoint(4, 2)
    assert e.value.code == L.IBL_EINVAL
    s.close()
    s = _sim()
    s.set_regularization(every=5)
    with pytest.raises(L.IblError) as e:
        s.adjoint(4, 2)
    assert e.value.code == L.IBL_EINVAL
    s.close()
    s = _sim()
    lib = L.load()
    nb = ctypes.c_size_t()
    L.check(lib.ibl_adjoint_workspace_size(s.h, 4, 2, ctypes.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    code = lib.ibl_adjoint(s.h, 4, 2, ctypes.c_void_p(ws.data_ptr()), nb.value - 256, None, None, None, None)
    assert code == L.IBL_ENOMEM
    assert lib.ibl_adjoint(s.h, 0, 2, ctypes.c_void_p(ws.data_ptr()), nb.value, None, None, None, None) == L.IBL_EINVAL
    assert lib.ibl_adjoint(s.h, 4, 0, ctypes.c_void_p(ws.data_ptr()), nb.value, None, None, None, None) == L.IBL_EINVAL
    assert s.steps_done == 0
    s.close()


def test_autograd_function(adj64):
    from paper_2403_01161_gb300.autograd import DropletSpec, deformation

    spec = DropletSpec(n=N, tau=1.0, n_hold=N_HOLD, level=LEVEL, R=R, n_steps=STEPS, K=K, precision="fp64",
                       center=tuple(0.5 * (k - 1) for k in N))
    sigma = torch.tensor(SIGMA, dtype=torch.float64, requires_grad=True)
    frames = torch.tensor(_frames(), dtype=torch.float64, device="cuda", requires_grad=True)
    D = deformation(sigma, frames, spec)
    (3.0 * D).backward()
    assert abs(D.item() - adj64["D"]) < 1e-13
    assert abs(sigma.grad.item() - 3.0 * adj64["dD_dsigma"]) <= 1e-12 * abs(adj64["dD_dsigma"])
    assert _rel(frames.grad.cpu().numpy(), 3.0 * adj64["dD_dA"]) < 1e-12
    with torch.no_grad():
        D2 = deformation(sigma.detach(), frames.detach(), spec)
    assert abs(D2.item() - adj64["D"]) < 1e-13


def test_forward_shape_records_are_kept():
    """With shape records on, the adjoint's forward pass leaves exactly the
    records a plain run takes (the recomputations take none)."""
    a = _sim()
    a.set_readout(5)
    g = a.adjoint(STEPS, K)
    ra = a.series()
    b = _sim()
    b.set_readout(5)
    b.step(STEPS)
    rb = b.series()
    assert [r["step"] for r in ra] == [r["step"] for r in rb] == list(range(5, STEPS + 1, 5))
    for x, y in zip(ra, rb):
        assert abs(x["D"] - y["D"]) < 1e-12
    assert abs(ra[-1]["D"] - g["D"]) < 1e-12
    a.close()
    b.close()
