"""Pins of the oracle's lattice Boltzmann part against what the paper and the
mathematics fix (closed forms, invariants, special cases).  CPU only."""
import itertools

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def test_velocity_set_and_weights(golden):
    c = O.velocities()
    w = O.weights()
    assert len({tuple(v) for v in c}) == 19
    assert (c[0] == 0).all()
    g = golden["d3q19_weights"]["value"]
    c2 = (c * c).sum(1)
    assert np.allclose(w[c2 == 0], g["w0"], rtol=0, atol=1e-16)
    assert np.allclose(w[c2 == 1], g["w1_6"], rtol=0, atol=1e-16)
    assert np.allclose(w[c2 == 2], g["w7_18"], rtol=0, atol=1e-16)
    assert (c2 == 1).sum() == 6 and (c2 == 2).sum() == 12
    # lattice isotropy up to fourth order, which the equilibrium relies on
    assert abs(w.sum() - 1) < 1e-15
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * d, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_moments(seed):
    """Eq. (equilibriumLB): the hydrodynamic moments of f_eq are rho, rho u and
    rho (c_s^2 I + u u).  The quadratic term as printed (-u.u/c_s^2) fails the
    first one; the reading -u.u/(2 c_s^2) passes all three."""
    rng = np.random.default_rng(seed)
    c = O.velocities().astype(float)
    rho = 1 + 0.05 * rng.standard_normal()
    u = 0.05 * rng.standard_normal(3)
    f = O.equilibrium(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(c.T @ f, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), rho * (CS2 * np.eye(3) + np.outer(u, u)),
                       atol=1e-15)
    # the printed form would leave a mass defect of -rho u.u/(2 c_s^2)
    w = O.weights()
    cu = c @ u
    printed = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - u @ u / CS2)
    assert abs((printed.sum() - rho) - (-rho * (u @ u) / (2 * CS2))) < 1e-15


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_guo_source_moments(tau):
    """Sec. 3.1 Guo term: sum S = 0, sum c S = (1 - 1/2tau) F,
    sum c c S = (1 - 1/2tau)(u F + F u)."""
    rng = np.random.default_rng(7)
    c = O.velocities().astype(float)
    u = 0.04 * rng.standard_normal(3)
    F = 1e-3 * rng.standard_normal(3)
    S = O.guo_source(tau, u, F)
    k = 1 - 1 / (2 * tau)
    assert abs(S.sum()) < 1e-18
    assert np.allclose(c.T @ S, k * F, atol=1e-18)
    assert np.allclose(np.einsum("i,ia,ib->ab", S, c, c), k * (np.outer(u, F) + np.outer(F, u)),
                       atol=1e-18)


def test_peskin_phi_identities(golden):
    """phi of Sec. 3.1: support |x| < 2, partition of unity, even/odd sums of
    1/2 each, zero first moment and sum of squares 3/8, for any shift."""
    assert golden["peskin_phi_support"]["value"] == 2.0
    assert O.peskin_phi(0.0) == pytest.approx(0.5, abs=1e-16)
    assert O.peskin_phi(2.0) == 0.0 and O.peskin_phi(-2.5) == 0.0
    for r in np.linspace(0, 1, 37):
        j = np.arange(-3, 5)
        p = np.array([O.peskin_phi(r - jj) for jj in j])
        assert abs(p.sum() - 1) < 1e-15
        assert abs(p[j % 2 == 0].sum() - 0.5) < 1e-15
        assert abs(((r - j) * p).sum()) < 1e-15
        assert abs((p * p).sum() - 3 / 8) < 1e-15
    # continuity at |x| = 1 and |x| = 2
    assert abs(O.peskin_phi(1 - 1e-12) - O.peskin_phi(1 + 1e-12)) < 1e-9
    assert abs(O.peskin_phi(2 - 1e-12)) < 1e-5


def _faces():
    for a in range(3):
        for s in (-1, 1):
            side = [0, 0, 0]
            side[a] = s
            yield side


@pytest.mark.parametrize("side", list(_faces()))
def test_face_rule_moments_exact(side):
    """Eq. (ZH_bulk) with the Zou-He density closure: after reconstruction the
    node carries exactly the density of the closure and the momentum rho u_w,
    for non-equilibrium inputs."""
    rng = np.random.default_rng(sum((i + 2) * v for i, v in enumerate(side)) + 10)
    c = O.velocities().astype(float)
    for _ in range(5):
        uw = 0.03 * rng.standard_normal(3)
        f = O.equilibrium(1.0 + 0.01 * rng.standard_normal(), 0.03 * rng.standard_normal(3))
        f += 1e-3 * rng.standard_normal(19)
        g = O.bc_node(f, side, uw)
        a = int(np.nonzero(side)[0][0])
        s = side[a]
        known = ~((c[:, a] * s) < 0)
        assert np.array_equal(g[known], f[known])  # known populations untouched
        rho = g.sum()
        tan = c[:, a] == 0
        out = c[:, a] * s > 0
        assert abs(rho - (f[tan].sum() + 2 * f[out].sum()) / (1 + uw[a] * s)) < 1e-15
        assert np.allclose(c.T @ g, rho * uw, atol=2e-16)


@pytest.mark.parametrize("side", list(_faces()))
def test_face_rule_normal_link_is_bounce_back(side):
    """Eq. (standard BB): the link normal to the wall obeys
    f_{-i} = f_i - rho/3 (c_i . u)."""
    rng = np.random.default_rng(3)
    c = O.velocities()
    uw = 0.02 * rng.standard_normal(3)
    f = O.equilibrium(1.0, 0.01 * rng.standard_normal(3)) + 1e-4 * rng.standard_normal(19)
    g = O.bc_node(f, side, uw)
    rho = g.sum()
    a = int(np.nonzero(side)[0][0])
    n_out = np.zeros(3, int)
    n_out[a] = side[a]
    i = [k for k in range(19) if (c[k] == n_out).all()][0]
    j = [k for k in range(19) if (c[k] == -n_out).all()][0]
    assert abs(g[j] - (f[i] - rho / 3 * (n_out @ uw))) < 1e-16


def test_face_rule_reproduces_equilibrium():
    """A node already at f_eq(rho, u_w) is a fixed point of the face rule."""
    rng = np.random.default_rng(11)
    for side in _faces():
        uw = 0.03 * rng.standard_normal(3)
        f = O.equilibrium(1.02, uw)
        g = O.bc_node(f, side, uw)
        assert np.allclose(g, f, atol=1e-16)


def _edges_and_corners():
    for side in itertools.product((-1, 0, 1), repeat=3):
        if sum(1 for s in side if s) >= 2:
            yield list(side)


@pytest.mark.parametrize("rule", [O.EDGE_COUNTER_SLIP, O.EDGE_PAPER_LITERAL])
def test_edge_corner_rest_state(rule):
    """Eqs. (zh-buried-links-edges), (zh-buried-links-corners): at rest
    (f = w, u_w = 0) the buried links get 1/36 and f_0 = 12 f_b = 1/3, so the
    rest state is preserved exactly on all 12 edges and 8 corners."""
    w = O.weights()
    for side in _edges_and_corners():
        g = O.bc_node(w.copy(), side, np.zeros(3), rule)
        assert np.allclose(g, w, atol=1e-17), side


@pytest.mark.parametrize("rule", [O.EDGE_COUNTER_SLIP, O.EDGE_PAPER_LITERAL])
def test_edge_corner_structure(rule):
    """Consequences of the printed edge/corner rules: the buried links share
    one value f_b (as printed; the counter-slip reading adds to each its half
    of the moving-wall difference, so the pair's mean is f_b and its
    difference 2 w (c.u_w)/c_s^2), f_0 = 12 f_b, and an edge node carries
    rho = 36 f_b."""
    rng = np.random.default_rng(5)
    c = O.velocities()
    w = O.weights()
    for side in _edges_and_corners():
        uw = 0.02 * rng.standard_normal(3)
        f = O.equilibrium(1.0, 0.01 * rng.standard_normal(3)) + 1e-4 * rng.standard_normal(19)
        g = O.bc_node(f, side, uw, rule)
        sd = np.array(side)
        unk = np.array([any(sd[a] != 0 and c[j, a] * sd[a] < 0 for a in range(3)) for j in range(19)])
        opp = np.array([[k for k in range(19) if (c[k] == -c[j]).all()][0] for j in range(19)])
        buried = unk & unk[opp]
        nb = int((sd != 0).sum())
        assert buried.sum() == (2 if nb == 2 else 6)
        fb = g[0] / 12
        for j in np.flatnonzero(buried):
            share = w[j] * (c[j] @ uw) / CS2 if rule == O.EDGE_COUNTER_SLIP else 0.0
            assert abs(g[j] - fb - share) < 1e-17
        if nb == 2:
            assert abs(g.sum() - 36 * fb) < 1e-15


def _edge_frame(side):
    """Inward normals n1 (n2, n3) and, for an edge, the edge direction e."""
    sd = np.array(side)
    ns = [-sd[a] * np.eye(3)[a] for a in range(3) if sd[a] != 0]
    e = np.cross(ns[0], ns[1]) if len(ns) == 2 else None
    return ns, e


@pytest.mark.parametrize("uw_scale", [0.0, 0.03])
def test_edge_corner_node_carries_the_wall_momentum(uw_scale):
    """The counter-slip reading of Eqs. (ZH_edges), (zh-buried-links-edges),
    (zh-buried-links-corners): whatever populations arrive, every edge and
    corner node leaves the rebuild with momentum sum_i c_i f_i = rho0 u_w
    (rho0 = 1), the moving-wall property the face rule has with its own rho;
    at rest this is the no-slip of the wall.  A dropped wall term, a wrong
    sign of the tangential sum or a missing buried-link share each leave a
    momentum error of order u_w or of the arriving edge-line momentum."""
    rng = np.random.default_rng(21)
    c = O.velocities()
    for side in _edges_and_corners():
        for _ in range(4):
            uw = uw_scale * rng.standard_normal(3)
            f = O.equilibrium(1.0 + 0.01 * rng.standard_normal(), 0.02 * rng.standard_normal(3))
            f = f + 1e-3 * rng.standard_normal(19)
            g = O.bc_node(f, side, uw, O.EDGE_COUNTER_SLIP)
            assert np.abs(c.T @ g - uw).max() < 1e-16, (side, c.T @ g - uw)
            # the known (outgoing) populations are left as they arrived
            sd = np.array(side)
            unk = np.array([any(sd[a] != 0 and c[j, a] * sd[a] < 0 for a in range(3)) for j in range(19)])
            assert np.array_equal(g[1:][~unk[1:]], f[1:][~unk[1:]])


def test_printed_edge_sign_doubles_the_edge_line_slip():
    """Why the edge rule is read with the face rule's sign: taken as printed
    (EDGE_PAPER_LITERAL, tangential sum with a minus sign), an edge at rest
    leaves the rebuild with twice the along-edge momentum m = f_{+e} - f_{-e}
    of its edge-line pair, while the normal momenta vanish; the counter-slip
    reading leaves zero.  Worked out by hand: the four reflected links with
    a component along e each carry -/+ m/4, the bounce-back parts of the
    diagonals cancel with the outgoing ones, so the total is m + m."""
    rng = np.random.default_rng(22)
    c = O.velocities()
    for side in _edges_and_corners():
        ns, e = _edge_frame(side)
        if e is None:
            continue
        f = O.weights() + 1e-3 * rng.standard_normal(19)
        ke = [k for k in range(19) if (c[k] == e).all()][0]
        km = [k for k in range(19) if (c[k] == -e).all()][0]
        m = f[ke] - f[km]
        lit = O.bc_node(f, side, np.zeros(3), O.EDGE_PAPER_LITERAL)
        assert abs((c.T @ lit) @ e - 2 * m) < 1e-16
        for n in ns:
            assert abs((c.T @ lit) @ n) < 1e-16
        cs = O.bc_node(f, side, np.zeros(3), O.EDGE_COUNTER_SLIP)
        assert np.abs(c.T @ cs).max() < 1e-16


def test_counter_slip_reduces_to_bounce_back_off_the_edge_line():
    """Reflected edge links with no component along the edge line (t_i = 0:
    the two axis links and the diagonal n1 + n2) follow Eq. (standard BB)
    with rho0 = 1 exactly: f_{-i} = f_i - 2 w_i (c_i.u_w)/c_s^2."""
    rng = np.random.default_rng(23)
    c = O.velocities()
    w = O.weights()
    for side in _edges_and_corners():
        ns, e = _edge_frame(side)
        if e is None:
            continue
        uw = 0.03 * rng.standard_normal(3)
        f = O.equilibrium(1.0, 0.01 * rng.standard_normal(3)) + 1e-3 * rng.standard_normal(19)
        g = O.bc_node(f, side, uw, O.EDGE_COUNTER_SLIP)
        for cj in (ns[0], ns[1], ns[0] + ns[1]):
            j = [k for k in range(19) if (c[k] == cj).all()][0]
            i = [k for k in range(19) if (c[k] == -cj).all()][0]
            assert abs(g[j] - (f[i] - 2 * w[i] * (c[i] @ uw) / CS2)) < 1e-17


def _linear_field(n, A):
    x = [np.arange(k) - (k - 1) / 2 for k in n]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    L = np.stack([X, Y, Z])
    return np.einsum("ab,bzyx->azyx", A, L)


@pytest.mark.parametrize("axes", [(0, 2), (1, 0), (2, 1)])
def test_couette_exact(axes):
    """Eq. (velo_facce_cubo_da_gradiente) on Zou-He walls normal to one axis,
    periodic elsewhere: the linear shear u_a = g (l_b - L_b/2) is an exact
    steady Navier-Stokes solution and the scheme keeps it to round-off."""
    a, b = axes
    n = [4, 4, 4]
    n[b] = 16
    bc = [O.BC_PERIODIC] * 3
    bc[b] = O.BC_ZOU_HE
    A = np.zeros((3, 3))
    A[a, b] = 2e-3
    s = O.OracleSim(n, 1.0, A[None], 10 ** 9, bc=bc)
    s.step(1500)
    rho, u, _ = s.fields()
    ex = _linear_field(n, A)
    assert np.abs(u - ex).max() < 1e-12 * 2e-3 * 8
    assert np.abs(rho - 1).max() < 1e-12


@pytest.mark.parametrize("tau", [1.0, 1.5])
def test_poiseuille(tau):
    """Body-force driven channel between resting Zou-He walls: the bulk
    profile has the exact curvature -g/nu, and the whole profile matches
    u_x = g/(2 nu) z (L - z) within 1e-2 at L = 16 (Zou-He wall slip is O(g))."""
    nz, g = 17, 1e-6
    nu = (tau - 0.5) / 3
    s = O.OracleSim((3, 3, nz), tau, np.zeros((1, 3, 3)), 10 ** 9, bc=(1, 1, 0))
    s.step(int(30 * nz * nz / nu), body_force=[g, 0, 0])
    _, u, _ = s.fields()
    ux = u[0, :, 1, 1]
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    assert np.allclose(d2[1:-1], -g / nu, rtol=1e-8)
    z = np.arange(nz)
    ex = g / (2 * nu) * z * (nz - 1 - z)
    assert np.abs(ux - ex).max() / ex.max() < 1.5e-2
    assert abs(ux[0]) < 1e-15 and abs(ux[-1]) < 1e-15


def test_periodic_body_force_momentum():
    """Eq. (LBMEQ) with the Guo source: in a periodic box each step adds
    exactly sum F to the momentum; with the half-force term the moments of
    step k carry (k + 1/2) g per node; mass is conserved."""
    n = (6, 5, 4)
    g = np.array([1e-5, -2e-5, 3e-6])
    s = O.OracleSim(n, 0.9, np.zeros((1, 3, 3)), 10 ** 9, bc=(1, 1, 1))
    steps = 25
    s.step(steps, body_force=g)
    rho, u, _ = s.fields()
    N = np.prod(n)
    mom = np.array([(rho * u[k]).sum() for k in range(3)])
    assert np.allclose(mom, (steps - 0.5) * g * N, rtol=1e-12)
    assert abs(rho.sum() - N) < 1e-12 * N


@pytest.mark.parametrize("kind", ["shear", "strain"])
def test_full_box_linear_flow(kind):
    """Six Zou-He faces with the counter-slip edge and corner rules: the
    imposed linear flow (a simple shear, an exact steady Navier-Stokes
    solution; a planar strain, exact with its quadratic pressure) is kept
    across the whole box, edges and corners included.  Measured with this
    reading (600 steps, 24^3, g = 1e-3): 5.8e-4 (shear) and 4.4e-4 (strain)
    of the face velocity in the inner box |l - c| < L/4, 3.6e-3 anywhere;
    the printed sign without wall terms leaves the edges at O(1)."""
    N, g = 24, 1e-3
    A = np.zeros((3, 3))
    if kind == "shear":
        A[0, 2] = g
    else:
        A[0, 0], A[1, 1] = g, -g
    s = O.OracleSim((N, N, N), 1.0, A[None], 10 ** 9)
    s.step(600)
    _, u, _ = s.fields()
    s.close()
    ex = _linear_field((N, N, N), A)
    scale = g * (N - 1) / 2
    err = np.abs(u - ex).max(0) / scale
    x = np.arange(N) - (N - 1) / 2
    m = np.abs(x) < N / 4
    assert err[np.ix_(m, m, m)].max() < 1e-3
    assert err.max() < 5e-3
    idx = np.arange(N)
    b = (idx == 0) | (idx == N - 1)
    Z, Y, X = np.meshgrid(b, b, b, indexing="ij")
    on_edge = (X.astype(int) + Y + Z) >= 2
    assert err[on_edge].max() < 2e-3
