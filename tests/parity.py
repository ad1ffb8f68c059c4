"""Helpers shared by the GPU parity tests: run the CUDA path (through the
C-ABI binding) and the oracle on the same seeded inputs and compare."""
import numpy as np

import oracle as O


def lib_to_oracle_perm():
    """perm[k] = library index of the oracle's population k."""
    from paper_2403_01161_gb300.sim import velocity_set

    c, _ = velocity_set()
    co = O.velocities()
    return np.array([[i for i in range(19) if (c[i] == co[k]).all()][0] for k in range(19)])


def frames_ou(seed, n_frames, amp):
    from paper_2403_01161_gb300 import inputs

    return inputs.ou_gradients(seed, n_frames, 1.0, 5.0, amp)


def make_pair(n, tau, frames, n_hold, bc=(0, 0, 0), precision="fp64", rule=0, record=True):
    from paper_2403_01161_gb300.sim import Sim

    g = Sim(n, tau, frames, n_hold, bc=bc, precision=precision, edge_rule=rule, record_fields=record)
    o = O.OracleSim(n, tau, frames, n_hold, bc=bc, rule=rule)
    return g, o


def run_both(g, o, steps):
    """steps - 1 plain steps and one recording step on the GPU; steps on the oracle."""
    if steps > 1:
        g.step(steps - 1)
    g.step_record()
    g.sync()
    o.step(steps)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
