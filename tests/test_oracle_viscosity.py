"""Pins of the oracle's viscosity ratio (Sec. 2: droplet viscosity chi mu):
the even-odd ray indicator against two independent inside tests (the
half-space test of a convex mesh, the solid-angle winding number of a
non-convex one), chi = 1 giving the plain scheme, and the viscous droplet's
slower shape relaxation that Eq. (LT) predicts."""
import numpy as np
import pytest

import oracle as O


def _nodes(n):
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([X, Y, Z], -1).reshape(-1, 3).astype(np.float64)


@pytest.mark.parametrize("level,R,c", [(2, 4.3, (9.37, 10.11, 8.62)), (3, 6.7, (12.2, 11.9, 13.05)),
                                       (4, 5.5, (10.5, 10.5, 10.5))])
def test_indicator_of_convex_mesh_is_the_half_space_test(level, R, c):
    """A point is inside a convex, outward-oriented mesh iff it is behind
    every face plane; no node here lies within 1e-7 of a plane."""
    n = (22, 24, 26)
    r, t = O.icosphere(level, R, c)
    ind = O.indicator(n, r, t)
    P = _nodes(n)
    a, b, cc = r[t[:, 0]], r[t[:, 1]], r[t[:, 2]]
    N = np.cross(b - a, cc - a)
    d = P @ N.T - np.einsum("tk,tk->t", a, N)[None, :]
    assert np.abs(d).min() > 1e-7
    want = (d < 0).all(axis=1).reshape(n[2], n[1], n[0])
    assert np.array_equal(ind.astype(bool), want)
    assert abs(ind.sum() / (4 / 3 * np.pi * R ** 3) - 1) < 0.06


def _winding(P, r, t):
    """Generalised winding number: the signed solid angles of the triangles
    seen from each point (Van Oosterom and Strackee) over 4 pi."""
    w = np.zeros(P.shape[0])
    for k0 in range(0, t.shape[0], 256):
        tt = t[k0:k0 + 256]
        A = r[tt[:, 0]][None] - P[:, None]
        B = r[tt[:, 1]][None] - P[:, None]
        C = r[tt[:, 2]][None] - P[:, None]
        la, lb, lc = (np.linalg.norm(X, axis=-1) for X in (A, B, C))
        num = np.einsum("ptk,ptk->pt", A, np.cross(B, C))
        den = la * lb * lc + np.einsum("ptk,ptk->pt", A, B) * lc + np.einsum("ptk,ptk->pt", B, C) * la \
            + np.einsum("ptk,ptk->pt", C, A) * lb
        w += 2 * np.arctan2(num, den).sum(axis=1)
    return w / (4 * np.pi)


def test_indicator_of_non_convex_mesh_is_the_winding_number():
    """A star-shaped, non-convex droplet (three lobes around z and a waist):
    the ray parity equals the rounded winding number at every node."""
    n = (24, 22, 26)
    c = np.array([11.3, 10.6, 12.4])
    r, t = O.icosphere(3, 1.0, (0.0, 0.0, 0.0))
    th = np.arccos(np.clip(r[:, 2], -1, 1))
    ph = np.arctan2(r[:, 1], r[:, 0])
    rad = 7.0 * (1 + 0.3 * np.sin(th) ** 2 * np.cos(3 * ph) + 0.2 * np.cos(2 * th))
    x = c + rad[:, None] * r
    ind = O.indicator(n, x, t)
    wn = _winding(_nodes(n), x, t)
    assert np.abs(wn - np.round(wn)).max() < 1e-6
    want = (np.round(wn) == 1).reshape(n[2], n[1], n[0])
    assert np.array_equal(ind.astype(bool), want)
    # the mesh is not convex: the half-space test misses inside nodes here
    a, b, cc = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    N = np.cross(b - a, cc - a)
    d = _nodes(n) @ N.T - np.einsum("tk,tk->t", a, N)[None, :]
    assert ((d < 0).all(axis=1) != want.ravel()).sum() > 0


def _relaxing(chi, steps):
    """A stretched droplet (R 5, level 3) relaxing in a quiescent 24^3 box."""
    n = (24, 24, 24)
    s = O.OracleSim(n, 1.0, np.zeros((1, 3, 3)), 10 ** 9)
    c = np.array([11.5, 11.5, 11.5])
    r, t = O.icosphere(3, 5.0, tuple(c))
    r = c + (r - c) * np.array([1.15, 0.93, 0.93])
    s.set_mesh(r, t, 0.02)
    if chi != 1.0:
        s.set_viscosity_ratio(chi)
    D = []
    for _ in range(steps // 10):
        s.step(10)
        D.append(O.observables(s.mesh()[0], t)["D"])
    s.close()
    return np.array(D)


def test_viscous_droplet_relaxes_slower():
    """Eq. (LT) with no flow: S - R^2 I decays like exp(-c_r t / tau_sigma),
    c_r = 40 (chi + 1) / ((2 chi + 3)(19 chi + 16)); tau_sigma uses the
    carrier viscosity, so chi = 4 relaxes c_r(1) / c_r(4) = 2.31 times more
    slowly than chi = 1.  The immersed boundary spreads the viscosity jump
    over the stencil, so the measured ratio is looser."""
    rates = {}
    for chi in (1.0, 4.0):
        D = _relaxing(chi, 300)
        k = np.arange(D.size) * 10.0
        sel = slice(3, 20)
        rates[chi] = -np.polyfit(k[sel], np.log(D[sel]), 1)[0]
    cr = {chi: O.lt_coefficients(chi)[0] for chi in (1.0, 4.0)}
    ratio = rates[1.0] / rates[4.0]
    print("relaxation rates", rates, "ratio", ratio, "theory", cr[1.0] / cr[4.0])
    assert 1.5 < ratio < 3.0


def test_chi_one_is_the_plain_scheme_and_bad_settings():
    fr = np.zeros((1, 3, 3))
    fr[0, 0, 1] = 2e-3
    out = []
    for chi in (None, 1.0):
        s = O.OracleSim((20, 20, 20), 1.0, fr, 10 ** 9)
        s.set_mesh(*O.icosphere(2, 4.0, (9.4, 9.6, 9.5)), 0.02)
        if chi is not None:
            s.set_viscosity_ratio(chi)
        s.step(15)
        out.append((s.mesh()[0], s.fields()[1]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    s = O.OracleSim((20, 20, 20), 1.0, fr, 10, bc=(O.BC_ZOU_HE, O.BC_PERIODIC, O.BC_ZOU_HE))
    s.set_mesh(*O.icosphere(2, 4.0, (9.4, 9.6, 9.5)), 0.02)
    with pytest.raises(ValueError):
        s.set_viscosity_ratio(3.0)
    s.close()
