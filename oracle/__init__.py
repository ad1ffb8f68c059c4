"""FP64 CPU oracle of the IB-LB droplet step (arXiv:2403.01161).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  It shares no code with the CUDA path (``paper_2403_01161_gb300``),
and neither imports the other.

The lattice and immersed-boundary step is plain C (``iblb_oracle.c``, built
with gcc and loaded through ctypes); the mesh generator, the one-ring
neighbourhoods and the shape observables are plain numpy in ``oracle.py``;
the linear theory of Eq. (LT) is plain numpy in ``theory.py``.
"""
from .oracle import (  # noqa: F401
    build,
    lib,
    velocities,
    weights,
    equilibrium,
    guo_source,
    peskin_phi,
    bc_node,
    nodal_forces,
    regularize,
    icosphere,
    one_ring,
    observables,
    mesh_quality,
    enclosed_volume,
    restore_volume,
    indicator,
    OracleSim,
    BC_ZOU_HE,
    BC_PERIODIC,
    EDGE_COUNTER_SLIP,
    EDGE_PAPER_LITERAL,
    ERR_UNSTABLE,
    ERR_NOCONV,
    ERR_WALL,
)
from .theory import lt_coefficients, lt_observables, lt_propagate, lt_trajectory, strain  # noqa: F401,E402
