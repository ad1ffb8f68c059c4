"""GPU immersed-boundary path against the oracle: nodal forces, spreading,
interpolation, advection, regularisation and the shape readout, alone and
coupled to the lattice.  Connectivity is compared bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2403_01161_gb300 import inputs
from parity import frames_ou, lib_to_oracle_perm, make_pair, rel, run_both

pytestmark = pytest.mark.gpu


def _droplet_pair(n, R, level, sigma, frames, n_hold, precision, bc=(0, 0, 0), center=None):
    g, o = make_pair(n, 1.0, frames, n_hold, bc=bc, precision=precision)
    c = tuple(0.5 * (k - 1) for k in n) if center is None else center
    g.add_icosphere(level, R, sigma, center=c)
    r, t = O.icosphere(level, R, c)
    o.set_mesh(r, t, sigma)
    return g, o, t


@pytest.mark.parametrize("steps", [1, 2, 11])
def test_droplet_fp64_matches_oracle(steps):
    fr = frames_ou(21, 4, 4e-3)
    g, o, t = _droplet_pair((24, 22, 26), 4.5, 2, 0.02, fr, 4, "fp64")
    run_both(g, o, steps)
    r_g, F_g, t_g = g.mesh()
    r_o, F_o = o.mesh()
    assert np.array_equal(t_g, t)
    assert np.abs(F_g - F_o).max() < 1e-14
    assert np.abs(r_g - r_o).max() < 1e-12
    rho_g, u_g, Fe_g = g.fields()
    rho_o, u_o, Fe_o = o.fields()
    assert np.abs(Fe_g - Fe_o).max() < 1e-15
    assert np.abs(Fe_o).max() > 1e-4
    assert np.abs(u_g - u_o).max() < 1e-14
    assert np.abs(rho_g - rho_o).max() < 1e-13
    assert g.status() == 0


def test_droplet_fp32_matches_oracle():
    """FP32 deviations and FP32 Eulerian force/velocity, FP64 mesh: u within
    1e-5 relative, node positions within 1e-6 of the droplet size."""
    fr = frames_ou(22, 6, 4e-3)
    g, o, t = _droplet_pair((28, 26, 24), 5.0, 3, 0.02, fr, 10, "fp32")
    run_both(g, o, 40)
    r_g, F_g, _ = g.mesh()
    r_o, F_o = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-6 * 5.0
    assert rel(F_g, F_o) < 1e-6
    _, u_g, Fe_g = g.fields()
    _, u_o, Fe_o = o.fields()
    assert rel(u_g, u_o) < 1e-5
    assert rel(Fe_g, Fe_o) < 1e-5


def test_periodic_droplet_crossing_the_seam():
    """Periodic box with the droplet straddling the periodic seam: the
    stencils wrap, the patch wraps, results match the oracle."""
    fr = np.zeros((1, 3, 3))
    g, o, t = _droplet_pair((20, 20, 20), 4.0, 2, 0.03, fr, 1, "fp64", bc=(1, 1, 1), center=(1.3, 18.7, 9.5))
    run_both(g, o, 6)
    r_g, _, _ = g.mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-12
    rho_g, u_g, _ = g.fields()
    rho_o, u_o, _ = o.fields()
    assert np.abs(u_g - u_o).max() < 1e-14
    # exact conservation (property at any size)
    assert abs(rho_g.sum() - 8000) < 1e-10
    mom = np.array([(rho_g * u_g[k]).sum() for k in range(3)])
    assert np.abs(mom).max() < 1e-12


def test_regularize_now_matches_oracle():
    """Sec. 3.3 on a stretched, jittered icosphere: same positions, same
    iteration count, for both signs of the correction term."""
    r0, t = O.icosphere(3, 5.0, (15.5, 15.5, 15.5))
    r0 = (r0 - 15.5) * [1.5, 0.8, 0.9] + 15.5
    r0 = inputs.jitter(r0, 0.15, 3)
    for plus in (True, False):
        g, _ = make_pair((32, 32, 32), 1.0, np.zeros((1, 3, 3)), 1, precision="fp32", record=False)
        g.add_mesh(r0, t, 0.01)
        g.set_regularization(0.1, 0.51, 0.01, 100, 0, plus)
        it = g.regularize_now()
        ptr, idx = g.neighbours()
        pt, it_ = O.one_ring(t, r0.shape[0])
        assert np.array_equal(ptr, pt) and np.array_equal(idx, it_)
        x, it_o, conv = O.regularize(r0, pt, it_, 0.1, 0.51, 0.01, 100, plus)
        r_g, _, _ = g.mesh()
        assert it == it_o and conv
        assert np.abs(r_g - x).max() < 1e-12


def test_observables_match_oracle():
    """Shape record of a stretched, rotated, jittered mesh: volume, area,
    centroid, S, eigenvalues, v_max (up to sign), D and beta."""
    rng = np.random.default_rng(8)
    r0, t = O.icosphere(4, 6.0)
    Qm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    r0 = (r0 * [1.4, 1.0, 0.7]) @ Qm.T + 20.0
    r0 = inputs.jitter(r0, 0.05, 4)
    A = frames_ou(5, 1, 1e-3)
    g, _ = make_pair((40, 40, 40), 1.0, A, 1, precision="fp32", record=False)
    g.add_mesh(r0, t, 0.01)
    ob = g.readout()
    ref = O.observables(r0, t, A[0])
    assert abs(ob["V"] - ref["V"]) < 1e-10 * ref["V"]
    assert abs(ob["area"] - ref["area"]) < 1e-11 * ref["area"]
    assert np.allclose(ob["xc"], ref["xc"], atol=1e-11)
    S = ref["S"]
    assert np.allclose(ob["S6"], [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]], atol=1e-11)
    assert np.allclose(ob["lam"], ref["lam"], atol=1e-11)
    assert abs(abs(np.dot(ob["vmax"], ref["vmax"])) - 1) < 1e-11
    assert abs(ob["D"] - ref["D"]) < 1e-12
    assert abs(ob["beta"] - ref["beta"]) < 1e-11


def test_scheduled_regularization_and_series_fp64():
    """Coupled run with regularisation every 5 steps and a record every 5
    steps: positions and the recorded series match the oracle."""
    fr = frames_ou(31, 3, 6e-3)
    g, o, t = _droplet_pair((26, 26, 26), 5.0, 2, 0.01, fr, 8, "fp64")
    g.set_regularization(0.1, 0.51, 0.01, 100, 5, True)
    o.set_regularization(0.1, 0.51, 0.01, 100, 5, True)
    g.set_readout(5)
    run_both(g, o, 20)
    r_g, _, _ = g.mesh()
    r_o, _ = o.mesh()
    assert np.abs(r_g - r_o).max() < 1e-11
    ser = g.series()
    assert [s["step"] for s in ser] == [5, 10, 15, 20]
    assert ser[-1]["reg_iters"] == o.reg_iters
    ref = O.observables(r_o, t, fr[min(19 // 8, 2)])
    assert abs(ser[-1]["D"] - ref["D"]) < 1e-10
    assert abs(ser[-1]["beta"] - ref["beta"]) < 1e-9


def test_run_frames_matches_stepping():
    """The host-buffer trajectory loop equals stepping with preset frames."""
    fr = frames_ou(41, 4, 4e-3)
    a, _, _ = _droplet_pair((24, 24, 24), 4.0, 2, 0.02, fr, 5, "fp32")
    fb = np.zeros_like(fr)
    fb[0] = fr[0]  # same initial state; run_frames uploads every frame itself
    b, _, _ = _droplet_pair((24, 24, 24), 4.0, 2, 0.02, fb, 5, "fp32")
    a.set_readout(5)
    a.step(20)
    ser = a.series()
    recs = b.run_frames(fr, 5)
    assert len(recs) == 4
    for x, y in zip(ser, recs):
        assert x["step"] == y["step"] and abs(x["D"] - y["D"]) < 1e-9
    ra, _, _ = a.mesh()
    rb, _, _ = b.mesh()
    assert np.abs(ra - rb).max() < 1e-7  # FP32 atomics: summation order may differ


def test_wall_contact_is_reported():
    """A droplet whose stencil reaches a wet boundary node: the step skips
    that node's spread and advection (no out-of-box access) and the next
    synchronising call reports IBL_EWALL."""
    from paper_2403_01161_gb300 import _lib as L

    g, _ = make_pair((20, 20, 20), 1.0, np.zeros((1, 3, 3)), 1, precision="fp32", record=False)
    g.add_icosphere(2, 4.0, 0.01, center=(5.2, 10.0, 10.0))
    g.step(2)
    assert g.status() == L.IBL_EWALL


def test_graph_replay_any_phase_matches_eager_fp64():
    """With no regularisation and no readout a step's launches repeat every 6
    steps (AA parity x three patch buffers), so a chunk may start at any step:
    one captured graph per phase.  Steps 7, 100, 13, 50, 49 in turn start
    chunks at phases 1, 0 and 2; the result equals eager launches."""
    fr = frames_ou(52, 3, 5e-3)
    out = []
    for graphs in (True, False):
        g, _, t = _droplet_pair((24, 24, 24), 4.5, 2, 0.02, fr, 30, "fp64")
        g.set_graphs(graphs)
        for n in (7, 100, 13, 50, 49):
            g.step(n)
        g.sync()
        out.append((g.mesh()[0], g.steps_done, g.step_paths(), g.status()))
    (ra, na, pa, sa), (rb, nb, pb, sb) = out
    assert na == nb == 219 and sa == sb == 0
    # chunks of 48: 7 eager; 48 + 48 replayed from step 7, 4 eager; 13 eager;
    # 48 from step 120, 2 eager; 48 from step 170, 1 eager
    assert pa == (27, 192)
    assert pb == (219, 0)
    assert np.abs(ra - rb).max() < 1e-12


def test_segment_graphs_match_eager_fp64():
    """Runs shorter than a chunk replay graphs of their own: prepare(n)
    captures the graphs of the next step(n) without running a step, and a
    segment met a second time is captured on the spot.  With a record every
    20 steps and regularisation every 10 (chunk 60), steps of 25 from step 3
    start segments at phases 3, 28, 53, 18, 43, 8, ...; the trajectory, the
    shape records and the step count equal eager launches."""
    fr = frames_ou(53, 3, 5e-3)
    out = []
    for graphs in (True, False):
        g, _, t = _droplet_pair((24, 24, 24), 4.5, 2, 0.02, fr, 30, "fp64")
        g.set_graphs(graphs)
        g.set_regularization(0.1, 0.51, 0.01, 100, 10, True)
        g.set_readout(20)
        g.step(3)
        g.sync()
        p0 = g.step_paths()
        g.prepare(25)
        g.sync()
        assert g.steps_done == 3 and g.step_paths() == p0  # nothing ran
        g.step(25)  # replays the prepared segment graph
        p1 = g.step_paths()
        for _ in range(13):  # phases 28, 53, 18, 43, 8, 33, 58, 23, 48, 13, 38, 3, 28
            g.step(25)
        g.sync()
        out.append((g.mesh()[0], g.series(), g.steps_done, p0, p1, g.step_paths(), g.status()))
    (ra, sa, na, a0, a1, a2, sta), (rb, sb, nb, b0, b1, b2, stb) = out
    assert na == nb == 3 + 14 * 25 and sta == stb == 0
    assert a1[1] - a0[1] == 25 and a1[0] == a0[0]
    # phases repeat every 12 calls (60 / gcd(25, 60)): the call at phase 28
    # comes round again at the last call and is captured then; the call at
    # phase 3 follows the prepared one and replays its graph
    assert a2[1] - a1[1] == 2 * 25
    assert b2 == (3 + 14 * 25, 0)
    assert np.abs(ra - rb).max() < 1e-12
    assert [x["step"] for x in sa] == [x["step"] for x in sb]
    assert max(abs(x["D"] - y["D"]) for x, y in zip(sa, sb)) < 1e-12


def test_graph_replay_matches_eager_fp64():
    """Whole chunks replayed as a captured CUDA graph give the same result as
    eager launches (regularisation every 10 steps, a record every 20)."""
    fr = frames_ou(51, 3, 5e-3)
    out = []
    for graphs in (True, False):
        g, _, t = _droplet_pair((24, 24, 24), 4.5, 2, 0.02, fr, 30, "fp64")
        g.set_graphs(graphs)
        g.set_regularization(0.1, 0.51, 0.01, 100, 10, True)
        g.set_readout(20)
        g.step(7)
        g.step(100)  # crosses chunk boundaries: eager head, replays, eager tail
        g.step(13)
        g.sync()
        out.append((g.mesh()[0], g.series(), g.steps_done))
    (ra, sa, na), (rb, sb, nb) = out
    assert na == nb == 120
    assert np.abs(ra - rb).max() < 1e-12
    assert [x["step"] for x in sa] == [x["step"] for x in sb] == [20, 40, 60, 80, 100, 120]
    assert max(abs(x["D"] - y["D"]) for x, y in zip(sa, sb)) < 1e-12
