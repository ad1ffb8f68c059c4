"""Writes the FP64 oracle's reference trajectories that the full-length GPU
parity tests compare against.  Calls only the oracle (``oracle/``) and the
seeded workload definitions; nothing here comes from the CUDA path.

    python tests/golden/make_oracle_series.py NAME [NAME ...] [--threads N]

NAME is one of
  single_droplet_128    128^3, R 12, icosphere level 4, OU seed 2, rms Ca 0.2,
                        20000 steps (the trajectory loop of Sec. 3.2)
  precision_stress_256  256^3, R 24, level 5, OU seed 4, R/eta 1, rms Ca 0.5,
                        regularisation (Sec. 3.3) every 50 steps, 5000 steps
  ensemble8             the first 8 members of the 64-droplet ensemble
                        (seeds 1000-1007, boxes 48^3-96^3), 10000 steps each
  adjoint_64_fd         64^3, R 8, level 3, OU seed 500, 2000 steps: central
                        differences of the final Taylor deformation D with
                        respect to sigma and along 4 seeded unit directions
                        in the space of the gradient frames
  adjoint_64_fd_s501..s503   the same for OU seeds 501, 502 and 503
Each writes tests/golden/oracle_<NAME>.npz.

Trajectories: a shape record (Sec. 2: volume, area, centroid, eigenvalues of
S, v_max, D, beta) every 100 steps, and the state at the last record before
any sticky error (the node positions, and the velocity u of that step at a
fixed sample of lattice nodes: every `stride`-th node of the box around the
droplet, plus seeded random nodes of the whole box).  A trajectory stops at
the first record whose error bits are set (a droplet stretched until its
stencil reaches a wall, say): "last_step" is the last clean record and
"first_err_step" the first flagged one (-1 if none).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RECORD_EVERY = 100


def _used_frame(step, n_hold, n_frames):
    """Frame applied in the last completed step (the one beta refers to)."""
    return min(max(step - 1, 0) // n_hold, n_frames - 1)


def _oracle_for(w):
    import oracle as O
    from paper_2403_01161_gb300 import config

    o = O.OracleSim(w.n, w.tau, w.frames, w.n_hold)
    r0, t = O.icosphere(w.level, w.R, config.box_center(w.n))
    o.set_mesh(r0, t, w.sigma)
    if w.reg_every:
        o.set_regularization(every=w.reg_every)
    return o, t


def _u_sample(w, r, stride, n_random, seed):
    """Flat node indices [z][y][x] of the velocity sample: every stride-th
    node of the box of the droplet grown by 3 nodes, and n_random seeded
    nodes of the whole box."""
    nx, ny, nz = w.n
    lo = np.maximum(np.floor(r.min(0)).astype(int) - 3, 0)
    hi = np.minimum(np.floor(r.max(0)).astype(int) + 4, np.array(w.n) - 1)
    xs, ys, zs = (np.arange(lo[a], hi[a] + 1, stride) for a in range(3))
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    near = (X + nx * (Y + ny * Z)).ravel()
    rng = np.random.default_rng(seed)
    far = rng.integers(0, nx * ny * nz, size=n_random)
    return np.unique(np.concatenate([near, far])).astype(np.int64)


def _run_records(o, t, w, steps, log, stride=None):
    """Steps the oracle up to `steps` steps, a shape record every
    RECORD_EVERY, stopping at the first record with error bits set.  With
    `stride`, also keeps the positions and the velocity sample of the last
    clean record."""
    import oracle as O

    rec = {k: [] for k in ("step", "V", "area", "xc", "lam", "vmax", "D", "beta", "err", "reg_iters")}
    snap = {}
    t0 = time.time()
    done = 0
    first_err = -1
    while done < steps:
        k = min(RECORD_EVERY, steps - done)
        o.step(k)
        done += k
        if done % RECORD_EVERY:
            continue
        if o.error:
            first_err = done
            log("  %s: error bits %d at the record of step %d; stopping" % (w.name, o.error, done))
            break
        r, _ = o.mesh()
        A = w.frames[_used_frame(done, w.n_hold, len(w.frames))]
        ob = O.observables(r, t, A)
        rec["step"].append(done)
        rec["V"].append(ob["V"])
        rec["area"].append(ob["area"])
        rec["xc"].append(ob["xc"])
        rec["lam"].append(ob["lam"])
        rec["vmax"].append(ob["vmax"])
        rec["D"].append(ob["D"])
        rec["beta"].append(ob["beta"])
        rec["err"].append(o.error)
        rec["reg_iters"].append(o.reg_iters)
        snap["r"] = r
        if stride is not None:
            _, u, _ = o.fields()
            idx = _u_sample(w, r, stride, 4096, 12345)
            snap["u_idx"] = idx
            snap["u_sample"] = u.reshape(3, -1)[:, idx]
            snap["u_norm_all"] = np.linalg.norm(u)
        if done % (10 * RECORD_EVERY) == 0:
            log("  %s step %d D %.6f (%.0f s)" % (w.name, done, ob["D"], time.time() - t0))
    out = {k: np.asarray(v) for k, v in rec.items()}
    return out, snap, first_err


def trajectory(w, stride, log):
    o, t = _oracle_for(w)
    t0 = time.time()
    rec, snap, first_err = _run_records(o, t, w, w.steps, log, stride)
    out = {f"rec_{k}": v for k, v in rec.items()}
    out.update({"r_last": snap["r"], "tris": t, "u_idx": snap["u_idx"], "u_sample": snap["u_sample"],
                "u_norm_all": snap["u_norm_all"], "last_step": int(rec["step"][-1]), "first_err_step": first_err,
                "steps": w.steps, "oracle_seconds": time.time() - t0})
    o.close()
    return out


def single_droplet_128(log):
    from paper_2403_01161_gb300 import config

    return trajectory(config.single_droplet_128(steps=20000), 2, log)


def precision_stress_256(log):
    from paper_2403_01161_gb300 import config

    return trajectory(config.precision_stress_256(steps=5000, Ca_rms=0.5), 3, log)


def ensemble8(log):
    from paper_2403_01161_gb300 import config

    out = {}
    for k, w in enumerate(config.ensemble_workloads(8, steps=10000)):
        o, t = _oracle_for(w)
        rec, snap, first_err = _run_records(o, t, w, w.steps, log)
        for key, v in rec.items():
            out[f"m{k}_rec_{key}"] = v
        out[f"m{k}_r_last"] = snap["r"]
        out[f"m{k}_last_step"] = int(rec["step"][-1])
        out[f"m{k}_first_err_step"] = first_err
        o.close()
        log("member %d (%s) done: last clean record %d, first flagged %d" % (k, w.name, rec["step"][-1], first_err))
    out["members"] = 8
    out["steps"] = 10000
    return out


def adjoint_64_fd(log, n_dirs=4, seed=4242, member=500):
    """Central differences of D(n steps) from step 0 (fresh equilibrium of
    frame 0, as the adjoint entry point starts), FP64 oracle, for the 64^3
    droplet of OU seed `member`."""
    import oracle as O
    from paper_2403_01161_gb300 import config

    w = config.adjoint_member(member, steps=2000)

    def D_of(frames, sigma):
        o = O.OracleSim(w.n, w.tau, frames, w.n_hold)
        r0, t = O.icosphere(w.level, w.R, config.box_center(w.n))
        o.set_mesh(r0, t, sigma)
        o.step(w.steps)
        err = o.error
        r, _ = o.mesh()
        o.close()
        if err:
            raise RuntimeError("oracle error bits %d" % err)
        return O.observables(r, t)["D"]

    D0 = D_of(w.frames, w.sigma)
    hs = 1e-4 * w.sigma
    dsig = (D_of(w.frames, w.sigma + hs) - D_of(w.frames, w.sigma - hs)) / (2 * hs)
    log("D0 %.12f dD/dsigma %.9e" % (D0, dsig))
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n_dirs,) + w.frames.shape)
    V /= np.sqrt((V * V).sum(axis=(1, 2, 3)))[:, None, None, None]
    hA = 1e-7
    dV = []
    for k in range(n_dirs):
        dp = D_of(w.frames + hA * V[k], w.sigma)
        dm = D_of(w.frames - hA * V[k], w.sigma)
        dV.append((dp - dm) / (2 * hA))
        log("direction %d: dD/dV %.9e" % (k, dV[-1]))
    return {"D0": D0, "dD_dsigma": dsig, "h_sigma": hs, "V": V, "h_A": hA, "dD_dV": np.asarray(dV),
            "steps": w.steps, "seed": member}


JOBS = {"single_droplet_128": single_droplet_128, "precision_stress_256": precision_stress_256,
        "ensemble8": ensemble8, "adjoint_64_fd": adjoint_64_fd,
        "adjoint_64_fd_s501": lambda log: adjoint_64_fd(log, member=501),
        "adjoint_64_fd_s502": lambda log: adjoint_64_fd(log, member=502),
        "adjoint_64_fd_s503": lambda log: adjoint_64_fd(log, member=503)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+", choices=sorted(JOBS))
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    if args.threads > 0:
        os.environ["OMP_NUM_THREADS"] = str(args.threads)

    def log(msg):
        print(msg, flush=True)

    for name in args.names:
        t0 = time.time()
        out = JOBS[name](log)
        out["generator"] = "tests/golden/make_oracle_series.py %s" % name
        path = os.path.join(HERE, "oracle_%s.npz" % name)
        np.savez_compressed(path, **out)
        log("%s written in %.0f s -> %s" % (name, time.time() - t0, path))


if __name__ == "__main__":
    main()
