"""Python face of the FP64 oracle (test infrastructure only; see package doc).

Functions here cite the part of arXiv:2403.01161 they follow:

* ``icosphere``    -- the structured spherical mesh of Sec. 3.2 (a subdivided
  icosahedron; the vertex and triangle order is this project's convention).
* ``one_ring``     -- the neighbour sets of Sec. 3.3 (edge-adjacent nodes).
* ``observables``  -- Sec. 2: morphological tensor S, its largest eigenvalue
  lambda_max and eigenvector v_max, the orientation beta of Eq. (beta); S is
  read as (5/V) * second moment of the enclosed volume, so that a uniform
  ellipsoid gives eig(S) = semi-axes squared.  numpy's ``eigh`` does the
  eigen-decomposition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iblb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

BC_ZOU_HE, BC_PERIODIC = 0, 1
EDGE_COUNTER_SLIP, EDGE_PAPER_LITERAL = 0, 1
ERR_UNSTABLE, ERR_NOCONV, ERR_WALL = 1, 2, 4

_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            L.orc_velocity.argtypes = [ctypes.c_int, _I]
            L.orc_weight.argtypes = [ctypes.c_int]
            L.orc_weight.restype = ctypes.c_double
            L.orc_equilibrium.argtypes = [ctypes.c_double, _D, _D]
            L.orc_guo_source.argtypes = [ctypes.c_double, _D, _D, _D]
            L.orc_peskin_phi.argtypes = [ctypes.c_double]
            L.orc_peskin_phi.restype = ctypes.c_double
            L.orc_bc_node.argtypes = [_D, _I, _D, ctypes.c_int]
            L.orc_bc_node.restype = ctypes.c_int
            L.orc_nodal_forces.argtypes = [ctypes.c_int, _D, ctypes.c_int, _I, ctypes.c_double, _D]
            L.orc_regularize.argtypes = [ctypes.c_int, _D, _I, _I, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, _I]
            L.orc_regularize.restype = ctypes.c_int
            L.orc_enclosed_volume.argtypes = [ctypes.c_int, _D, ctypes.c_int, _I, _D, _D]
            L.orc_restore_volume.argtypes = [ctypes.c_int, _D, ctypes.c_int, _I, ctypes.c_double]
            L.orc_sim_set_regularization_volume.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_sim_set_recentring.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_sim_set_viscosity_ratio.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_sim_set_viscosity_ratio.restype = ctypes.c_int
            L.orc_sim_get_indicator.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
            L.orc_indicator.argtypes = [_I, ctypes.c_int, _D, ctypes.c_int, _I, ctypes.c_void_p]
            L.orc_sim_get_centre.argtypes = [ctypes.c_void_p, _D]
            L.orc_sim_create.argtypes = [_I, _I, ctypes.c_double, ctypes.c_int, _D, ctypes.c_int,
                                         ctypes.c_int]
            L.orc_sim_create.restype = ctypes.c_void_p
            L.orc_sim_destroy.argtypes = [ctypes.c_void_p]
            L.orc_sim_set_mesh.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_int, _I,
                                           ctypes.c_double, _I, _I]
            L.orc_sim_set_regularization.argtypes = [ctypes.c_void_p, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_sim_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.orc_sim_step.restype = ctypes.c_int
            L.orc_sim_step_body_force.argtypes = [ctypes.c_void_p, ctypes.c_long, _D]
            L.orc_sim_step_body_force.restype = ctypes.c_int
            L.orc_sim_get_step.argtypes = [ctypes.c_void_p]
            L.orc_sim_get_step.restype = ctypes.c_long
            L.orc_sim_get_error.argtypes = [ctypes.c_void_p]
            L.orc_sim_get_reg_iters.argtypes = [ctypes.c_void_p]
            L.orc_sim_get_fields.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_sim_get_mesh.argtypes = [ctypes.c_void_p, _D, _D]
            L.orc_sim_set_positions.argtypes = [ctypes.c_void_p, _D]
            L.orc_sim_get_populations.argtypes = [ctypes.c_void_p, _D]
            L.orc_sim_set_populations.argtypes = [ctypes.c_void_p, _D, ctypes.c_long]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def velocities() -> np.ndarray:
    """The oracle's D3Q19 velocity set, shape (19, 3)."""
    L = lib()
    out = np.zeros((19, 3), dtype=np.int32)
    for i in range(19):
        L.orc_velocity(i, _ip(out[i]))
    return out


def weights() -> np.ndarray:
    L = lib()
    return np.array([L.orc_weight(i) for i in range(19)])


def equilibrium(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_equilibrium(float(rho), _dp(u), _dp(out))
    return out


def guo_source(tau: float, u, F) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_guo_source(float(tau), _dp(u), _dp(F), _dp(out))
    return out


def peskin_phi(x: float) -> float:
    return lib().orc_peskin_phi(float(x))


def bc_node(f, side, uw, rule: int = EDGE_COUNTER_SLIP) -> np.ndarray:
    """Boundary reconstruction of one node's 19 populations (returns a copy)."""
    g = np.array(f, dtype=np.float64).copy()
    s = np.ascontiguousarray(side, dtype=np.int32)
    u = np.ascontiguousarray(uw, dtype=np.float64)
    lib().orc_bc_node(_dp(g), _ip(s), _dp(u), int(rule))
    return g


def nodal_forces(r, tris, sigma: float) -> np.ndarray:
    r = np.ascontiguousarray(r, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    F = np.zeros_like(r)
    lib().orc_nodal_forces(r.shape[0], _dp(r), t.shape[0], _ip(t), float(sigma), _dp(F))
    return F


def enclosed_volume(r, tris):
    """(V, volume centroid) of a closed outward-oriented mesh (signed tetrahedra)."""
    x = np.ascontiguousarray(r, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    V = np.zeros(1)
    c = np.zeros(3)
    lib().orc_enclosed_volume(x.shape[0], _dp(x), t.shape[0], _ip(t), _dp(V), _dp(c))
    return float(V[0]), c


def indicator(n, r, tris):
    """1 at the lattice nodes of an (nx, ny, nz) box that lie inside the
    closed mesh by the even-odd rule on vertical rays (see the C oracle's
    orc_indicator), as an (nz, ny, nx) uint8 array."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    nn = np.array(n, dtype=np.int32)
    out = np.zeros(int(np.prod(n)), dtype=np.uint8)
    lib().orc_indicator(_ip(nn), r.shape[0], _dp(r), t.shape[0], _ip(t), out.ctypes.data)
    return out.reshape(n[2], n[1], n[0])


def restore_volume(r, tris, V_target):
    """The mesh scaled about its volume centroid to enclose V_target."""
    x = np.ascontiguousarray(r, dtype=np.float64).copy()
    t = np.ascontiguousarray(tris, dtype=np.int32)
    lib().orc_restore_volume(x.shape[0], _dp(x), t.shape[0], _ip(t), float(V_target))
    return x


def regularize(r, nb_ptr, nb_idx, alpha=0.1, gamma=0.51, tol=0.01, max_iter=100, plus_sign=True, tris=None,
               keep_volume=False):
    """Sec. 3.3 extended Laplacian smoothing; returns (positions, iterations,
    converged).  keep_volume (needs tris): afterwards scale the mesh about its
    volume centroid back to the volume it enclosed before (an option beyond
    Sec. 3.3)."""
    x = np.ascontiguousarray(r, dtype=np.float64).copy()
    p = np.ascontiguousarray(nb_ptr, dtype=np.int32)
    q = np.ascontiguousarray(nb_idx, dtype=np.int32)
    conv = np.zeros(1, dtype=np.int32)
    V0 = enclosed_volume(x, tris)[0] if keep_volume else None
    it = lib().orc_regularize(x.shape[0], _dp(x), _ip(p), _ip(q), alpha, gamma, tol, max_iter,
                              1 if plus_sign else 0, _ip(conv))
    if keep_volume:
        x = restore_volume(x, tris, V0)
    return x, int(it), bool(conv[0])


# ----------------------------------------------------------------------------
# mesh
# ----------------------------------------------------------------------------
def _unit(v: np.ndarray) -> np.ndarray:
    n = np.sqrt(v[..., 0] * v[..., 0] + v[..., 1] * v[..., 1] + v[..., 2] * v[..., 2])
    return v / n[..., None]


def icosphere(level: int, R: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Subdivided icosahedron projected on the sphere of radius R.

    Convention (shared by every implementation in this project, written out
    independently by each):
      * base vertices, in this order, normalised to unit length:
        (-1,p,0) (1,p,0) (-1,-p,0) (1,-p,0) (0,-1,p) (0,1,p) (0,-1,-p) (0,1,-p)
        (p,0,-1) (p,0,1) (-p,0,-1) (-p,0,1), p the golden ratio;
      * base faces: every vertex triple at mutual distance 2 (before the
        normalisation), sorted lexicographically by its ascending index triple
        (a<b<c) and written (a,b,c) or (a,c,b), whichever is counter-clockwise
        seen from outside;
      * each level: faces are scanned in order; the midpoints of edges ab, bc, ca
        are created on first use (position normalise((x_a + x_b) * 0.5), appended
        in creation order) and the face is replaced by
        (a,m_ab,m_ca), (b,m_bc,m_ab), (c,m_ca,m_bc), (m_ab,m_bc,m_ca);
      * finally x = center + R * x.
    Nodes 10*4^l + 2, triangles 20*4^l.
    """
    p = (1.0 + np.sqrt(5.0)) / 2.0
    raw = np.array([[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0], [0, -1, p], [0, 1, p],
                    [0, -1, -p], [0, 1, -p], [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]],
                   dtype=np.float64)
    faces = []
    for a in range(12):
        for b in range(a + 1, 12):
            for c in range(b + 1, 12):
                dab = np.linalg.norm(raw[a] - raw[b])
                dbc = np.linalg.norm(raw[b] - raw[c])
                dca = np.linalg.norm(raw[c] - raw[a])
                if abs(dab - 2) < 1e-9 and abs(dbc - 2) < 1e-9 and abs(dca - 2) < 1e-9:
                    n = np.cross(raw[b] - raw[a], raw[c] - raw[a])
                    if np.dot(n, raw[a] + raw[b] + raw[c]) > 0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    assert len(faces) == 20
    verts = [v for v in _unit(raw)]
    for _ in range(level):
        mid = {}
        new_faces = []

        def midpoint(i, j):
            key = (min(i, j), max(i, j))
            if key not in mid:
                mid[key] = len(verts)
                verts.append(_unit((verts[i] + verts[j]) * 0.5))
            return mid[key]

        for (a, b, c) in faces:
            mab = midpoint(a, b)
            mbc = midpoint(b, c)
            mca = midpoint(c, a)
            new_faces += [(a, mab, mca), (b, mbc, mab), (c, mca, mbc), (mab, mbc, mca)]
        faces = new_faces
    r = np.array(verts, dtype=np.float64) * R + np.asarray(center, dtype=np.float64)[None, :]
    return r, np.array(faces, dtype=np.int32)


def one_ring(tris: np.ndarray, nv: int):
    """Edge-adjacent neighbours of each node as CSR (ascending indices)."""
    nbrs = [set() for _ in range(nv)]
    for (a, b, c) in np.asarray(tris):
        for (i, j) in ((a, b), (b, c), (c, a)):
            nbrs[i].add(int(j))
            nbrs[j].add(int(i))
    ptr = np.zeros(nv + 1, dtype=np.int32)
    idx = []
    for i in range(nv):
        s = sorted(nbrs[i])
        ptr[i + 1] = ptr[i] + len(s)
        idx += s
    return ptr, np.array(idx, dtype=np.int32)


def mesh_quality(r, tris) -> float:
    """Largest ratio of longest to shortest edge over the triangles (1 for an
    equilateral mesh); the degradation Sec. 3.3 regularises against shows as
    clustered nodes (short edges) and loose triangles (long edges)."""
    r = np.asarray(r, dtype=np.float64)
    t = np.asarray(tris)
    e = np.stack([np.linalg.norm(r[t[:, (k + 1) % 3]] - r[t[:, k]], axis=1) for k in range(3)], axis=1)
    return float((e.max(axis=1) / e.min(axis=1)).max())


def observables(r, tris, A=None) -> dict:
    """Volume, area, centroid, S, eigenvalues, v_max, Taylor D and beta (Sec. 2).

    Volume integrals of the closed polyhedron are sums over the signed
    tetrahedra (ref, a, b, c), ref the node mean; for a tetrahedron with one
    vertex at the origin, int x x^T dV = V_T/20 (a a^T + b b^T + c c^T + s s^T)
    with s = a + b + c.  D = (sqrt(l_max) - sqrt(l_min))/(sqrt(l_max) + sqrt(l_min)).
    beta = v.E.v / |E|_F with E = (A + A^T)/2 of the current frame; NaN if |E| = 0.
    """
    r = np.asarray(r, dtype=np.float64)
    t = np.asarray(tris)
    ref = r.mean(axis=0)
    a = r[t[:, 0]] - ref
    b = r[t[:, 1]] - ref
    c = r[t[:, 2]] - ref
    vt = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    V = vt.sum()
    s = a + b + c
    first = (vt[:, None] * s).sum(axis=0) / 4.0
    xc = first / V
    M = np.zeros((3, 3))
    for v in (a, b, c, s):
        M += np.einsum("t,ti,tj->ij", vt, v, v)
    M /= 20.0
    M -= V * np.outer(xc, xc)
    S = 5.0 * M / V
    lam, vec = np.linalg.eigh(S)
    vmax = vec[:, 2]
    area = 0.5 * np.linalg.norm(np.cross(r[t[:, 1]] - r[t[:, 0]], r[t[:, 2]] - r[t[:, 0]]), axis=1).sum()
    D = (np.sqrt(lam[2]) - np.sqrt(lam[0])) / (np.sqrt(lam[2]) + np.sqrt(lam[0]))
    beta = float("nan")
    if A is not None:
        A = np.asarray(A, dtype=np.float64).reshape(3, 3)
        E = 0.5 * (A + A.T)
        nE = np.sqrt((E * E).sum())
        if nE > 0:
            beta = float(vmax @ E @ vmax / nE)
    return {"V": V, "area": area, "xc": xc + ref, "S": S, "lam": lam, "vmax": vmax, "D": D,
            "beta": beta}


# ----------------------------------------------------------------------------
# time stepping
# ----------------------------------------------------------------------------
class OracleSim:
    """FP64 IBLB box of n = (nx, ny, nz) nodes (optional droplet mesh).

    frames: (n_frames, 3, 3) velocity gradients A[a, b] = du_a/dx_b (lattice
    units), each held n_hold steps (Sec. 3.2).  bc: per axis BC_ZOU_HE or
    BC_PERIODIC.
    """

    def __init__(self, n, tau, frames, n_hold, bc=(BC_ZOU_HE,) * 3, rule=EDGE_COUNTER_SLIP):
        self.L = lib()
        self.n = tuple(int(v) for v in n)
        self.nn = self.n[0] * self.n[1] * self.n[2]
        fr = np.ascontiguousarray(np.asarray(frames, dtype=np.float64).reshape(-1, 9))
        nn = np.array(self.n, dtype=np.int32)
        bb = np.array(bc, dtype=np.int32)
        self.h = self.L.orc_sim_create(_ip(nn), _ip(bb), float(tau), int(rule), _dp(fr), fr.shape[0],
                                       int(n_hold))
        self.nv = 0
        self.tris = None

    def close(self):
        if self.h:
            self.L.orc_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mesh(self, r, tris, sigma):
        r = np.ascontiguousarray(r, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        ptr, idx = one_ring(t, r.shape[0])
        self.nv = r.shape[0]
        self.tris = t
        self.L.orc_sim_set_mesh(self.h, r.shape[0], _dp(r), t.shape[0], _ip(t), float(sigma),
                                _ip(ptr), _ip(idx))

    def set_regularization(self, alpha=0.1, gamma=0.51, tol=0.01, max_iter=100, every=0,
                           plus_sign=True, keep_volume=False):
        self.L.orc_sim_set_regularization(self.h, alpha, gamma, tol, max_iter, every,
                                          1 if plus_sign else 0)
        self.L.orc_sim_set_regularization_volume(self.h, 1 if keep_volume else 0)

    def set_recentring(self, on=True):
        """Centre the linear boundary field of each step on the droplet's
        centre of mass (volume centroid at the start of the step) instead of
        the box centre (Sec. 3.2)."""
        self.L.orc_sim_set_recentring(self.h, 1 if on else 0)

    def set_viscosity_ratio(self, chi):
        """Droplet viscosity chi times the carrier's (Sec. 2): tau inside the
        droplet = 1/2 + chi (tau - 1/2), inside decided per node by the
        even-odd ray rule of `indicator`.  Needs the mesh and Zou-He walls on
        every axis."""
        if not self.L.orc_sim_set_viscosity_ratio(self.h, float(chi)):
            raise ValueError("viscosity ratio needs chi > 0, a mesh and Zou-He walls on every axis")

    def indicator(self):
        """Inside-the-droplet flags used by the last step, (nz, ny, nx) uint8."""
        out = np.zeros(self.nn, dtype=np.uint8)
        self.L.orc_sim_get_indicator(self.h, out.ctypes.data)
        nx, ny, nz = self.n
        return out.reshape(nz, ny, nx)

    def centre(self):
        """Centre of the boundary field used by the last step."""
        c = np.zeros(3)
        self.L.orc_sim_get_centre(self.h, _dp(c))
        return c

    def step(self, n=1, body_force=None) -> int:
        if body_force is None:
            return self.L.orc_sim_step(self.h, int(n))
        g = np.ascontiguousarray(body_force, dtype=np.float64)
        return self.L.orc_sim_step_body_force(self.h, int(n), _dp(g))

    @property
    def steps_done(self) -> int:
        return self.L.orc_sim_get_step(self.h)

    @property
    def error(self) -> int:
        return self.L.orc_sim_get_error(self.h)

    @property
    def reg_iters(self) -> int:
        return self.L.orc_sim_get_reg_iters(self.h)

    def fields(self):
        """(rho, u, F) of the last step; rho (nz,ny,nx), u and F (3,nz,ny,nx)."""
        rho = np.zeros(self.nn)
        u = np.zeros(3 * self.nn)
        F = np.zeros(3 * self.nn)
        self.L.orc_sim_get_fields(self.h, _dp(rho), _dp(u), _dp(F))
        nx, ny, nz = self.n
        return rho.reshape(nz, ny, nx), u.reshape(3, nz, ny, nx), F.reshape(3, nz, ny, nx)

    def mesh(self):
        """(positions, nodal forces of the last step), each (nv, 3)."""
        r = np.zeros((self.nv, 3))
        Fn = np.zeros((self.nv, 3))
        self.L.orc_sim_get_mesh(self.h, _dp(r), _dp(Fn))
        return r, Fn

    def set_positions(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        self.L.orc_sim_set_positions(self.h, _dp(r))

    def populations(self):
        """Pre-collision state f_t, (19, nz, ny, nx), unknown boundary slots = 0."""
        out = np.zeros(19 * self.nn)
        self.L.orc_sim_get_populations(self.h, _dp(out))
        nx, ny, nz = self.n
        return out.reshape(19, nz, ny, nx)

    def set_populations(self, f, step):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert f.size == 19 * self.nn
        self.L.orc_sim_set_populations(self.h, _dp(f), int(step))
