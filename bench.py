"""Benchmark of the fused IB-LB droplet step (arXiv:2403.01161) on GB300.

Workload: the single-droplet FP32 configuration -- 128^3 box with Zou-He
walls imposing seeded traceless Ornstein-Uhlenbeck velocity gradients
(correlation time 20 tau_eta, rms Ca 0.2, R/eta = 0.472), droplet R = 12
on an icosphere of level 4 (2562 nodes, 5120 triangles), tau_f = 1, a shape
record every 100 steps.  One "step" is one full IBLB time step (forces +
spread, lattice stream-collide with the box boundary, interpolation +
advection, scheduled readout).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (the droplet problems do not exchange
data); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fused LB+IB MLUPS & % HBM roofline; ensemble droplet-steps/s; adjoint/forward time"
UNIT = "MLUPS"
BYTES_PER_NODE = 152  # 19 FP32 populations read + written per lattice node update
L2_BYTES = 129 * 2 ** 20


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload():
    from paper_2403_01161_gb300 import config

    return config.single_droplet_128()


def config_dict(w, extra=None):
    d = {"workload": w.name, "box": list(w.n), "R": w.R, "icosphere_level": w.level, "mesh_nodes": 10 * 4 ** w.level + 2,
         "triangles": 20 * 4 ** w.level, "tau": w.tau, "steps_per_frame": w.n_hold, "readout_every": 100,
         "populations": "fp32 deviations, AA in place", "mesh": "fp64",
         "l2": "no flush: population array %.0f MB > %d MB L2" % (19 * 4 * w.nodes / 1e6, L2_BYTES // 2 ** 20)}
    if extra:
        d.update(extra)
    return d


def lattice_source_hash():
    """Hash of the lattice kernel's source: the kernel file up to the end of
    the lattice kernels, plus the shared device header it includes."""
    import hashlib

    src = open(os.path.join(ROOT, "paper_2403_01161_gb300", "csrc", "iblb_kernels.cu")).read()
    marker = "// ---------------------------------------------------------------------------\n// Immersed boundary."
    if marker not in src:
        return None
    hdr = open(os.path.join(ROOT, "paper_2403_01161_gb300", "csrc", "iblb_device.cuh")).read()
    return hashlib.sha256((src[: src.index(marker)] + hdr).encode()).hexdigest()


def traffic_from_profiles(name):
    """Per-launch DRAM bytes (read + write) of the far lattice kernel of the
    workload `name` from the committed ncu record, if that record was taken
    on the current lattice source; None otherwise."""
    p = os.path.join(ROOT, "profiles", "lattice_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("lattice_source_sha256") != lattice_source_hash():
        return None
    rec = d.get("workloads", {}).get(name)
    return float(rec["bytes_per_launch_full_size"]) if rec else None


CHUNK_128 = 300  # graph chunk of the single-droplet workload: lcm(6, readout period 100)


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of each rank's value (times are taken as the slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica by `steps` steps."""
    return world * nodes_per_rank * steps / seconds / 1e6


def _omp_threads(n):
    """Sets the OpenMP thread count of the calling thread's next parallel
    regions (the oracle's lattice loop) through the OpenMP runtime the
    oracle library is linked against."""
    import ctypes

    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return True
    except (OSError, AttributeError):
        return False


def cpu_baseline(w, budget_s=15.0, max_steps=400, one_core_budget_s=8.0):
    """The FP64 oracle, as it stands, on this host's cores: a bounded number
    of steps of the same workload (same box, mesh and gradients), once with
    every core and once with one core."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    import oracle as O
    from paper_2403_01161_gb300 import config

    def run(budget, cap):
        o = O.OracleSim(w.n, w.tau, w.frames, w.n_hold)
        r, t = O.icosphere(w.level, w.R, config.box_center(w.n))
        o.set_mesh(r, t, w.sigma)
        t0 = time.perf_counter()
        o.step(1)
        first = time.perf_counter() - t0
        n = max(1, min(cap, int(budget / max(first, 1e-3))))
        t0 = time.perf_counter()
        o.step(n)
        dt = time.perf_counter() - t0
        o.close()
        return n, dt

    O.lib()
    _omp_threads(cores)
    n, dt = run(budget_s, max_steps)
    out = {"value": w.nodes * n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d FP64 oracle steps of %s (steps 1..%d of the trajectory), %.1f s" % (n, w.name, n, dt)}
    if one_core_budget_s > 0 and _omp_threads(1):
        n1, dt1 = run(one_core_budget_s, max_steps)
        _omp_threads(cores)
        out["one_core"] = {"value": w.nodes * n1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                           "sample": "%d FP64 oracle steps of %s, %.1f s" % (n1, w.name, dt1)}
    return out


def ensemble_oracle_rate(budget_s=10.0, n_sample=8, steps_each=10):
    """The FP64 oracle on the 64-droplet ensemble, as it stands, on this
    host's cores: a bounded sample -- `steps_each` steps of each of the
    first `n_sample` members (seeds 1000..), after one untimed step each --
    extrapolated to all 64 members by their node counts (the oracle's cost
    per lattice-node update is the same in every box).  Returns droplet-steps
    per second of the whole ensemble, labelled as extrapolated."""
    import oracle as O
    from paper_2403_01161_gb300 import config

    ws = config.ensemble_workloads(64, steps=100)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    _omp_threads(cores)
    node_steps, seconds, used = 0, 0.0, 0
    for w in ws[:n_sample]:
        o = O.OracleSim(w.n, w.tau, w.frames, w.n_hold)
        r, t = O.icosphere(w.level, w.R, config.box_center(w.n))
        o.set_mesh(r, t, w.sigma)
        o.step(1)
        t0 = time.perf_counter()
        o.step(steps_each)
        seconds += time.perf_counter() - t0
        o.close()
        node_steps += w.nodes * steps_each
        used += 1
        if seconds > budget_s:
            break
    s_per_node = seconds / node_steps
    s_per_ensemble_step = s_per_node * sum(w.nodes for w in ws)
    return {"value": len(ws) / s_per_ensemble_step, "unit": "droplet-steps/s", "cores": cores, "kind": "oracle",
            "sample": "%d FP64 oracle steps of each of the first %d members (%.1f s), extrapolated to the 64 "
                      "members by node count" % (steps_each, used, seconds)}


def ensemble_partition(sizes, world):
    """Longest-processing-time assignment of members (by node count) to ranks."""
    load = [0] * world
    owner = [0] * len(sizes)
    for k in sorted(range(len(sizes)), key=lambda k: -sizes[k]):
        r = min(range(world), key=lambda j: load[j])
        owner[k] = r
        load[r] += sizes[k]
    return owner


def gather_member_records(records, world):
    """The union over ranks of each rank's {member id: record} (every rank
    gets it); with one rank, the rank's own records."""
    if world <= 1:
        return dict(records)
    import torch.distributed as dist

    out = [None] * world
    dist.all_gather_object(out, dict(records))
    merged = {}
    for d in out:
        merged.update(d)
    return merged


def run_member_share(workloads, rank, world, runner):
    """Runs this rank's share of the members (longest-processing-time by node
    count) through runner(workload) -> record and gathers every rank's
    records: {member index: record}."""
    owner = ensemble_partition([w.nodes for w in workloads], world)
    mine = {k: runner(w) for k, w in enumerate(workloads) if owner[k] == rank}
    return gather_member_records(mine, world)


def measure_ensemble(dev, steps, warmup, rank, world):
    """Batched ensemble of the 64 uneven droplets (boxes 48^3..96^3, R 6..10,
    own OU trajectories) against the same droplets stepped one at a time.
    Returns droplet-steps/s of both (whole job), or None on ranks without work."""
    import torch

    from paper_2403_01161_gb300 import config
    from paper_2403_01161_gb300.sim import Ensemble, Sim

    ws = config.ensemble_workloads(64, steps=warmup + 2 * steps + 80)
    owner = ensemble_partition([w.nodes for w in ws], world)
    mine = [w for k, w in enumerate(ws) if owner[k] == rank]
    sims = []
    for w in mine:
        g = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
        g.add_icosphere(w.level, w.R, w.sigma)
        g.set_readout(100)
        sims.append(g)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1) * 1e-3, world, dev)

    E = Ensemble(sims) if sims else None
    tuned = None
    if E:
        k, tms = E.tune(6)  # the autotuner's steps are steps of the members' trajectories
        tuned = {"shape": E.shape(), "ms_per_step_by_shape": [float(v) for v in tms]}
        E.step(warmup)
    t_ens = timed(lambda: E.step(steps) if E else None)
    final = {}
    if E:
        E.sync()
        E.close()
        mine_idx = [k for k in range(len(ws)) if owner[k] == rank]
        for k, g in zip(mine_idx, sims):
            ob = g.readout()
            final[k] = {"seed": ws[k].name, "step": ob["step"], "D": ob["D"], "V": ob["V"]}
    final = gather_member_records(final, world)
    for g in sims:
        g.step(warmup)
    t_seq = timed(lambda: [g.step(steps) for g in sims])
    for g in sims:
        g.sync()
        g.close()
    return {"metric": "droplet-steps/s", "value": len(ws) * steps / t_ens,
            "one_at_a_time": len(ws) * steps / t_seq, "speedup": t_seq / t_ens, "members": len(ws),
            "total_nodes": sum(w.nodes for w in ws), "steps": steps, "warmup": warmup,
            "ms_per_step": t_ens / steps * 1e3,
            "mlups": sum(w.nodes for w in ws) * steps / t_ens / 1e6,
            "members_final_D": [final[k]["D"] for k in sorted(final)] if len(final) == len(ws) else None,
            "autotuner": tuned,
            "config": "64 droplets, boxes 48^3-96^3 (seeds 1000-1063), R 6-10, icosphere level 3 or 4, "
                      "own OU gradients, FP32; baseline: the same droplets stepped one after another with "
                      "the single-droplet kernels (graph replay each)"}


def measure_adjoint(dev, rank, world, seeds=range(500, 516), steps=2000, K=100):
    """Adjoint sweep of the 64^3 droplet (R 8, level 3, own OU gradients per
    seed) against its forward run: wall time of one ibl_adjoint call (its
    forward pass with checkpoints every K steps, the recomputations and the
    reverse steps) over the wall time of the same trajectory stepped plainly
    (graph replay).  Also the same with every step's moments kept resident
    (K = steps: no recomputation).  Seeds are shared out over the ranks."""
    import numpy as np
    import torch

    from paper_2403_01161_gb300 import config
    from paper_2403_01161_gb300.sim import Sim

    def make(w):
        s = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
        s.add_icosphere(w.level, w.R, w.sigma)
        torch.cuda.synchronize(dev)
        return s

    def timed(fn):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, out

    mine = [s for k, s in enumerate(seeds) if k % world == rank]
    w0 = config.adjoint_member(seeds[0], steps)
    s = make(w0)
    s.adjoint(steps, K)  # warm-up (module load, allocator)
    s.close()
    fwd, adj, adj_all, grads = [], [], [], []
    for seed in mine:
        w = config.adjoint_member(seed, steps)
        s = make(w)
        tf, _ = timed(lambda: (s.step(steps), s.sync()))
        s.close()
        s = make(w)
        ta, g = timed(lambda: s.adjoint(steps, K))
        s.close()
        s = make(w)
        tall, _ = timed(lambda: s.adjoint(steps, steps))
        s.close()
        fwd.append(tf)
        adj.append(ta)
        adj_all.append(tall)
        grads.append((g["D"], g["dD_dsigma"], float(np.linalg.norm(g["dD_dA"]))))
    tot = [sum(fwd), sum(adj), sum(adj_all)]
    if world > 1:
        t = torch.tensor(tot, dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t)
        tot = t.tolist()
    if rank != 0:
        return None
    return {"metric": "adjoint/forward wall-time ratio", "value": tot[1] / tot[0], "unit": "x",
            "higher_is_better": False, "K": K, "steps": steps, "seeds": len(seeds),
            "forward_ms": 1e3 * tot[0] / len(seeds), "adjoint_ms": 1e3 * tot[1] / len(seeds),
            "resident_ratio": tot[2] / tot[0], "resident_adjoint_ms": 1e3 * tot[2] / len(seeds),
            "forward_us_per_step": 1e6 * tot[0] / len(seeds) / steps,
            "example_rank0_seed": {"seed": mine[0], "D": grads[0][0], "dD_dsigma": grads[0][1],
                                   "norm_dD_dA": grads[0][2]} if grads else None,
            "config": "64^3, R 8, icosphere level 3, FP32, own OU gradients per seed (seeds 500-515), "
                      "2000 steps; adjoint = one ibl_adjoint call (forward pass with checkpoints every K "
                      "steps, recomputation per segment, reverse steps); resident = every step's moments "
                      "kept in HBM (K = 2000)"}


def measure_stress_256(dev, steps, warmup=300):
    """The 256^3 precision-stress workload (R 24, icosphere level 5, OU
    gradients at R/eta 1 and rms Ca 0.5, regularisation every 50 steps, a
    shape record every 100): step time and MLUPS by CUDA events over `steps`
    graph-replayed steps after a chunk of warm-up, and the far lattice
    kernel's achieved bandwidth from event pairs on one launch in 20."""
    import numpy as np
    import torch

    from paper_2403_01161_gb300 import config
    from paper_2403_01161_gb300.sim import Sim

    w = config.precision_stress_256(steps=warmup + steps + 8)
    s = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
    s.add_icosphere(w.level, w.R, w.sigma)
    s.set_regularization(every=w.reg_every)
    s.set_readout(100)
    every = 21  # odd: both step parities
    s.profile(True, mask=1, every=every)
    s.step(warmup)
    s.sync()
    s.profile(True, mask=1, every=every)
    paths0 = s.step_paths()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    prof = s.profile_read()
    paths1 = s.step_paths()
    s.profile(False)
    st = s.status()
    _, pext = s.patch()
    patch_nodes = int(np.prod(pext + 1)) if (pext >= 0).all() else 0
    ob = s.readout()
    s.close()
    if st != 0:
        raise RuntimeError("device error status %d in the 256^3 run" % st)
    lb_ms, lb_n = prof["lattice"]
    if lb_n == 0:
        raise RuntimeError("no lattice launch was bracketed in the 256^3 run")
    t_launch = lb_ms / lb_n * 1e-3
    far = w.nodes - patch_nodes
    achieved = BYTES_PER_NODE * far / t_launch / 1e9
    peak, peak_kind = measured_peaks()
    return {"metric": "MLUPS", "value": w.nodes * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "us_per_step": 1e3 * ms / steps, "steps": steps, "warmup": warmup,
            "graph_replayed_steps": paths1[1] - paths0[1], "eager_steps": paths1[0] - paths0[0],
            "final_D": ob["D"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic_from_profiles(w.name),
                         "kernel": "lattice stream-collide, nodes outside the droplet patch",
                         "kernel_us": t_launch * 1e6, "launches_timed": lb_n, "bytes_per_launch": BYTES_PER_NODE * far,
                         "patch_nodes": patch_nodes},
            "config": "256^3, R 24, icosphere level 5 (10242 nodes, 20480 triangles), tau 1, R/eta 1, rms Ca 0.5, "
                      "OU gradients (seed 4), regularisation (alpha 0.1, gamma 0.51, tol 0.01) every 50 steps, "
                      "shape record every 100, FP32 populations; population array 1.27 GB > L2"}


PAPER_TRAJECTORY_HOURS = 3.0   # Sec. 3.2: about 3 h per trajectory on one A100
PAPER_TRAJECTORY_FRAMES = 2000  # Sec. 3.2: about 2000 gradient frames per trajectory


def measure_production(dev, steps, warmup):
    """The paper's production setup (200^3, R 19, level 5, tau_f 1.5, 496 steps
    per frame, a shape record per frame) timed with the same graph replay,
    with the Sec. 3.3 mesh regularisation after every step (the paper's
    procedure, its parameters) and without: step time, MLUPS and the
    projected time of a 2000-frame trajectory next to the paper's A100
    figure."""
    import torch

    from paper_2403_01161_gb300 import config
    from paper_2403_01161_gb300.sim import Sim

    w = config.production_200(steps=warmup + steps)
    res = {}
    for name, every in (("regularised", 1), ("plain", 0)):
        s = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
        s.add_icosphere(w.level, w.R, w.sigma)
        s.set_readout(w.n_hold)
        if every:
            s.set_regularization(every=every)
        s.step(warmup)
        s.sync()
        stream = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        st = s.status()
        D = s.readout()["D"]
        n_reg = s.regularization_stats()[0]
        s.close()
        if st != 0:
            raise RuntimeError("device error status %d in the production run" % st)
        hours = ms / steps * 1e-3 * PAPER_TRAJECTORY_FRAMES * w.n_hold / 3600.0
        res[name] = {"us_per_step": 1e3 * ms / steps, "mlups": w.nodes * steps / (ms * 1e-3) / 1e6,
                     "hours_per_trajectory": hours, "speedup_vs_paper": PAPER_TRAJECTORY_HOURS / hours,
                     "final_D": D, "regularisations": n_reg}
    r = res["regularised"]
    return {"metric": "hours per 2000-frame trajectory", "value": r["hours_per_trajectory"], "unit": "h",
            "higher_is_better": False, "paper_a100_hours": PAPER_TRAJECTORY_HOURS,
            "speedup_vs_paper": r["speedup_vs_paper"], "us_per_step": r["us_per_step"], "mlups": r["mlups"],
            "steps": steps, "warmup": warmup, "steps_per_frame": w.n_hold, "without_regularisation": res["plain"],
            "regularisations": r["regularisations"],
            "config": "200^3, R 19, icosphere level 5 (20480 triangles), tau_f 1.5, R/eta 0.472, Ca 0.2, "
                      "OU gradients (seed 6), FP32 populations, shape record per frame, regularisation "
                      "(alpha 0.1, gamma 0.51, tol 0.01) after every step"}


def measure_linear_theory(dev, n_traj=1000, n_frames=2000, Ca_values=(0.05, 0.2), seed=700):
    """The linear theory of Eq. (LT) along n_traj synthetic OU trajectories of
    n_frames frames at the production conversion (R 19 lattice units, tau_f
    1.5, R/eta 0.472, N = 496 steps per frame, chi 1): GPU time of the batched
    RK4 integration and the distributions of lambda_max/R^2 and beta (a
    synthetic analogue of the paper's ensemble statistics, first 50 frames of
    each trajectory dropped)."""
    import numpy as np
    import torch

    from paper_2403_01161_gb300 import config, inputs
    from paper_2403_01161_gb300.theory import linear_theory

    out = {"metric": "trajectory-frames/s", "trajectories": n_traj, "frames": n_frames, "substeps": 8,
           "config": "R 19, tau_f 1.5, R/eta 0.472, 496 steps per frame, chi 1, OU gradients (rms 1/tau_eta, "
                     "correlation 20 tau_eta), seed %d; quantiles 5/25/50/75/95 %% after 50 frames" % seed,
           "by_Ca": {}}
    q = [5, 25, 50, 75, 95]
    for Ca in Ca_values:
        d = config.dns_to_lbu(0.472, 19.0, 1.5, Ca)
        hold = float(round(d["N"]))
        tau_eta = d["tau_eta_lbu"]
        fr = torch.as_tensor(inputs.ou_gradients_batch(seed, n_traj, n_frames, hold, 20.0 * tau_eta, 1.0 / tau_eta),
                             device=dev)
        linear_theory(fr[:2, :8], d["tau_sigma_lbu"], 19.0, hold, 1.0, substeps=8, device=dev)  # warm-up
        stream = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        res = linear_theory(fr, d["tau_sigma_lbu"], 19.0, hold, 1.0, substeps=8, device=dev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        r = res[:, 50:].cpu().numpy()
        lam, beta = r[..., 6].ravel(), r[..., 7].ravel()
        beta = beta[np.isfinite(beta)]
        out["by_Ca"]["%g" % Ca] = {"ms": ms, "trajectory_frames_per_s": n_traj * n_frames / (ms * 1e-3),
                                   "lam_max_R2_quantiles": [float(v) for v in np.percentile(lam, q)],
                                   "beta_quantiles": [float(v) for v in np.percentile(beta, q)],
                                   "beta_mean": float(beta.mean())}
    out["value"] = min(v["trajectory_frames_per_s"] for v in out["by_Ca"].values())
    return out


def measure_iblb_statistics(dev, n_members=16, n_frames=120, Ca_values=(0.05, 0.1), skip=20):
    """The synthetic analogue of the paper's ensemble statistics (Sec. 4):
    n_members IBLB droplets (72^3, R 9, icosphere level 4, R/eta 0.472, own
    OU gradients, 213 steps per frame, regularisation every 10 steps with
    volume restoring, boundary field centred on each droplet) stepped as one
    ensemble for n_frames frames, and the linear theory (Eq. (LT)) along the
    same frames; the quantiles of lambda_max/R^2 and beta of both after
    `skip` frames, their frame-by-frame correlation and the least-squares
    factor of the IBLB excess lambda_max/R^2 - 1 over the theory's, per
    capillary number."""
    import numpy as np
    import torch

    from paper_2403_01161_gb300 import statistics

    out = {"metric": "droplet-frames/s", "members": n_members, "frames": n_frames, "skip": skip, "by_Ca": {},
           "config": "72^3 box, R 9, icosphere level 4 (2562 nodes), tau 1, R/eta 0.472 (tau_eta 2181 steps, 213 "
                     "steps per frame), OU gradients (rms 1/tau_eta, correlation 20 tau_eta, seed 900), FP32; "
                     "regularisation every 10 steps (alpha 0.1, gamma 0.51, tol 0.01) restoring the volume; "
                     "boundary field centred on each droplet; quantiles 5/25/50/75/95 % over members and frames"}
    for Ca in Ca_values:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        res = statistics.trajectories(n_members, n_frames, Ca, R=9.0, box=72, level=4, device=dev)
        dt = time.perf_counter() - t0
        qs = statistics.quantiles(res, skip)
        lam_i, lam_t = qs["iblb_lam"][2] - 1.0, qs["lt_lam"][2] - 1.0
        ex_i = res["iblb_lam"][:, skip:] - 1.0
        ex_t = res["lt_lam"][:, skip:] - 1.0
        out["by_Ca"]["%g" % Ca] = {"seconds": dt, "lam_max_R2_quantiles_iblb": qs["iblb_lam"],
                                   "lam_max_R2_quantiles_theory": qs["lt_lam"],
                                   "beta_quantiles_iblb": qs["iblb_beta"], "beta_quantiles_theory": qs["lt_beta"],
                                   "median_excess_ratio": lam_i / lam_t if lam_t > 0 else None,
                                   "excess_correlation": float(np.corrcoef(ex_i.ravel(), ex_t.ravel())[0, 1]),
                                   "excess_fit_factor": float((ex_i * ex_t).sum() / (ex_t * ex_t).sum()),
                                   "steps_per_frame": res["hold"]}
    out["value"] = n_members * n_frames * len(Ca_values) / sum(v["seconds"] for v in out["by_Ca"].values())
    return out


def regularization_study(dev, steps=50000, sample=2000):
    """Sec. 3.3 in practice: one sub-critical droplet trajectory (96^3, R 10,
    level 4, rms Ca 0.2, OU gradients changing direction every 2 tau_eta)
    without regularisation, with the paper's smoothing on fixed schedules,
    with the adaptive trigger (smooth when the longest/shortest edge ratio
    exceeds a threshold, checked every step), and with the volume-restoring
    option.  Per mode: steps run
    before a device error (or all), volume relative to the initial sphere,
    edge-ratio extremes at the samples, smoothings performed, step time."""
    import numpy as np
    import torch

    from paper_2403_01161_gb300 import config
    from paper_2403_01161_gb300.sim import Sim

    w = config.small_ou(N=96, R=10.0, level=4, seed=77, steps=steps + 10000, Ca_rms=0.2, T_over_tau_eta=2.0)
    V0 = 4.0 / 3.0 * np.pi * w.R ** 3
    # (name, schedule, trigger); "none" checks quality on the sampling schedule but never smooths
    # (name, schedule, trigger, keep volume); "none" checks quality on the
    # sampling schedule but never smooths
    modes = [("none", sample, 1e300, False), ("every50", 50, 0.0, False), ("every10", 10, 0.0, False),
             ("every1", 1, 0.0, False), ("adaptive3", 1, 3.0, False), ("every1_keep_volume", 1, 0.0, True),
             ("adaptive3_keep_volume", 1, 3.0, True), ("every10_keep_volume", 10, 0.0, True)]
    out = {"config": "96^3, R 10, icosphere level 4, FP32, rms Ca 0.2, OU seed 77 with correlation 2 tau_eta, "
                     "%d steps, samples every %d; paper parameters alpha 0.1, gamma 0.51, tol 0.01" % (steps, sample),
           "modes": {}}
    for name, every, trig, keep in modes:
        s = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
        s.add_icosphere(w.level, w.R, w.sigma)
        s.set_regularization(every=every)
        s.set_regularization_trigger(trig)
        s.set_regularization_keep_volume(keep)
        qs, vs, done, ms = [], [], 0, 0.0
        for _ in range(steps // sample):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(sample)
            e1.record()
            if s.status() != 0:
                break
            ms += e0.elapsed_time(e1)
            done += sample
            n_reg, q = s.regularization_stats()
            qs.append(q)
            vs.append(s.readout()["V"] / V0)
        out["modes"][name] = {"schedule": every, "trigger": trig if trig < 1e299 else None, "keep_volume": keep,
                              "steps_run": done,
                              "V_over_V0_final": vs[-1] if vs else None, "V_over_V0_min": min(vs) if vs else None,
                              "edge_ratio_max": max(qs) if qs else None, "edge_ratio_final": qs[-1] if qs else None,
                              "smoothings": n_reg if name != "none" else 0,
                              "us_per_step": 1e3 * ms / done if done else None,
                              "V_samples": [round(v, 4) for v in vs], "edge_ratio_samples": [round(q, 2) for q in qs]}
        s.close()
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    w = workload()
    # a step of the reference arm is a bounded sample of oracle steps
    budget = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    cb = cpu_baseline(w, budget_s=budget, one_core_budget_s=0.0)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": w.nodes / (cb["value"] * 1e6) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, {"parallelism": "replicas" if world > 1 else "single"}), "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2403_01161_gb300.sim import Sim

    w = workload()
    sim = Sim(w.n, w.tau, w.frames, w.n_hold, precision=w.precision, device=dev)
    sim.add_icosphere(w.level, w.R, w.sigma)
    sim.set_readout(100)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # event pairs around one launch in `every` of the lattice kernel (nodes
    # outside the droplet patch), eager or inside a replayed graph: an event
    # pair costs its step part of the two streams' overlap (measured in a
    # 20-step window: 56.7 us per step without pairs, 59.0 with four, 57.5
    # with two), so sampling stays sparse -- at least two launches once the
    # region has 3 steps or more; an odd stride samples both step parities
    # (the AA pattern's even and odd kernels differ)
    every = max(1, min(99, args.steps // 2)) | 1
    sim.step(args.warmup)
    sim.sync()
    sim.profile(True, mask=1, every=every)  # clears the warm-up's marks (and its graphs)
    # capture, without running them, the graphs the timed call replays: its
    # whole chunks and the runs of steps around them (a user stepping in
    # fixed increments reaches the same state after the first calls)
    sim.prepare(args.steps)
    sim.sync()
    warm = sim.steps_done
    paths0 = sim.step_paths()
    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    prof = sim.profile_read()
    paths1 = sim.step_paths()
    sim.profile(False)
    _, pext = sim.patch()
    patch_nodes = int(np.prod(pext + 1)) if (pext >= 0).all() else 0
    far_nodes = w.nodes - patch_nodes
    clk = clocks.stop()
    st = sim.status()
    if st != 0:
        raise RuntimeError("device error status %d during the timed region" % st)
    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(w.nodes, args.steps, world, ms * 1e-3)
    lb_ms, lb_n = prof["lattice"]
    if lb_n == 0:
        raise RuntimeError("no lattice launch was bracketed in the timed region")
    t_launch = lb_ms / lb_n * 1e-3
    achieved = BYTES_PER_NODE * far_nodes / t_launch / 1e9
    peak, peak_kind = measured_peaks()
    # per step: force/spread, patch update, outside update, interpolation;
    # plus one shape-record kernel every 100 steps
    launches = 4 * args.steps + (sim.steps_done // 100 - (sim.steps_done - args.steps) // 100)
    timed_path = {"graph_replayed_steps": paths1[1] - paths0[1], "eager_steps": paths1[0] - paths0[0],
                  "warmup_steps_run": warm}
    # the path a long run takes: whole graph chunks, after the timed region
    # (a reported extra; the line's value is the timed region above)
    sim.step((-sim.steps_done) % CHUNK_128 + CHUNK_128)
    sim.sync()
    e0.record(stream)
    sim.step(2 * CHUNK_128)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_graph = e0.elapsed_time(e1)
    timed_path["graph_replay_after"] = {"steps": 2 * CHUNK_128, "us_per_step": 1e3 * ms_graph / (2 * CHUNK_128),
                                        "mlups": w.nodes * 2 * CHUNK_128 / (ms_graph * 1e-3) / 1e6}
    if sim.status() != 0:
        raise RuntimeError("device error status during the graph-replay measurement")
    sim.close()

    # end to end through the C-ABI with host buffers: the Sec. 3.2 loop, per
    # frame one pinned H2D gradient copy and one D2H shape record
    n_fr = max(1, (args.steps + w.n_hold - 1) // w.n_hold)
    pinned = torch.empty((n_fr, 9), dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(np.ascontiguousarray(w.frames[1:n_fr + 1].reshape(n_fr, 9))))
    sim2 = Sim(w.n, w.tau, w.frames[:n_fr + 1], w.n_hold, precision=w.precision, device=dev)
    sim2.add_icosphere(w.level, w.R, w.sigma)
    sim2.run_frames(w.frames[:1], w.n_hold)  # warm-up frame: the chunk graphs are captured here
    sim2.prepare(w.n_hold)  # and the graphs of the next frame's steps (captured, not run)
    sim2.sync()
    barrier()
    t0 = time.perf_counter()
    recs = sim2.run_frames(pinned.numpy(), w.n_hold)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    sim2.close()
    assert len(recs) == n_fr
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e_steps = n_fr * w.n_hold
    import ctypes

    from paper_2403_01161_gb300 import _lib

    rec_bytes = ctypes.sizeof(_lib.Observables)
    e2e = {"value": job_throughput(w.nodes, e2e_steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 72.0 / w.n_hold, "d2h_bytes_per_step": rec_bytes / w.n_hold,
           "steps": e2e_steps, "api": "ibl_run_frames (host gradients in, host shape records out)"}

    stress = measure_stress_256(dev, args.stress_steps) if args.stress_steps > 0 else None
    ens = measure_ensemble(dev, args.ensemble_steps, 20, rank, world)
    adj = measure_adjoint(dev, rank, world) if args.adjoint else None
    prod = measure_production(dev, 2 * 1488, 1488) if args.production else None
    lt = measure_linear_theory(dev) if args.theory and rank == 0 else None
    lstat = measure_iblb_statistics(dev) if args.theory and rank == 0 else None

    if rank == 0:
        cb = cpu_baseline(w) if world == 1 else None
        if ens is not None and world == 1:
            ens["oracle"] = ensemble_oracle_rate()
            ens["vs_oracle"] = ens["value"] / ens["oracle"]["value"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(w, {"parallelism": "replicas" if world > 1 else "single"}),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic_from_profiles(w.name),
                             "kernel": "lattice stream-collide, nodes outside the droplet patch",
                             "peak_kind": peak_kind,
                             "kernel_us": t_launch * 1e6, "launches_timed": lb_n, "sampling_every": every,
                             "bytes_per_launch": BYTES_PER_NODE * far_nodes, "patch_nodes": patch_nodes},
                "timed_path": timed_path, "precision_stress_256": stress,
                "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches * world, "clocks": clk,
                "ensemble": ens, "adjoint": adj, "production": prod, "linear_theory": lt,
                "iblb_statistics": lstat,
                "droplet_steps_per_s": world * args.steps / (ms * 1e-3),
                "lagrangian_updates_per_s": world * (10 * 4 ** w.level + 2) * args.steps / (ms * 1e-3)}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ensemble-steps", type=int, default=200,
                    help="timed steps of the 64-droplet ensemble measurement")
    ap.add_argument("--stress-steps", type=int, default=600,
                    help="timed steps of the 256^3 precision-stress measurement (0 skips it)")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false",
                    help="skip the adjoint/forward measurement (16 seeds of the 64^3 droplet)")
    ap.add_argument("--no-production", dest="production", action="store_false",
                    help="skip the 200^3 production-setup measurement")
    ap.add_argument("--no-theory", dest="theory", action="store_false",
                    help="skip the linear-theory ensemble measurement")
    ap.add_argument("--regularization-study", action="store_true",
                    help="run only the mesh-regularisation study (Sec. 3.3) and print its JSON")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint/forward measurement and print its JSON (profiling aid)")
    ap.add_argument("--adjoint-seeds", type=int, default=16)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.steps < 1:
        ap.error("--steps must be >= 1")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ensemble_steps < 1:
        ap.error("--ensemble-steps must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    if args.regularization_study:
        import torch

        torch.cuda.set_device(0)
        print(json.dumps(regularization_study(torch.device("cuda", 0))))
        return 0
    if args.adjoint_only:
        import torch

        torch.cuda.set_device(0)
        out = measure_adjoint(torch.device("cuda", 0), 0, 1, seeds=range(500, 500 + args.adjoint_seeds),
                              steps=args.adjoint_steps)
        print(json.dumps(out))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
