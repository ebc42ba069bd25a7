#!/usr/bin/env python3
"""Benchmark of the contact step: cell-evaluations/s and ms per contact_step
at 1934 particles, with the FP32 roofline fraction of the node-sweep kernel.

Workload (headline): 1934 cuboids of edge 12 at 30 % volume fraction in a
periodic 223^3 lattice (RSA centres of volume-equivalent spheres, uniform
random orientations), sharp indicator, FP32 node tests / FP64 reductions,
swept over seeded steps of small random pose increments (dX ~ N(0, 0.05),
rotations ~ N(0, 0.01 rad)).  A "step" is one contact_step: pose -> AABB,
broad phase, work partition, node sweep, pair reduction, force law,
per-particle sums.  Secondary lines in the same JSON: the 1934-particle mixed
spheres/cubes/polytopes box, the smoothed-indicator forward + adjoint pass on
the cuboid box, and the all-FP64 one-pair-per-block form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank evaluates its own independently seeded
box (weak scaling, no data-path collective); the barrier and the max over
ranks of the timed region use torch.distributed.  --impl reference times the
CPU FP64 oracle (the test-suite's reference implementation) on the host cores.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact cell-evaluations/s and ms per contact_step at 1934 particles, % FP32 roofline"
UNIT = "cell-evals/s"
FP32_LANES_PER_SM = 128   # FP32 lanes per Blackwell SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU baseline budget")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling runs)")
    ap.add_argument("--workload", default="cubes1934", choices=sorted(WORKLOADS),
                    help="state of the main line (default: the headline, 1934 cubes)")
    ap.add_argument("--seed", type=int, default=None, help="seed of the state (default: the workload's own)")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="threads of the oracle in --impl reference (default: all host cores)")
    ap.add_argument("--backward", action="store_true",
                    help="--impl reference: each step also takes the oracle's FP64 gradient of the smoothed "
                         "workload's force/torque loss (the adjoint's CPU baseline)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def combine_ranks(ms: float, cells: float, device):
    """Whole-job numbers of a weak-scaling run: the slowest rank's timed
    milliseconds (max) and the node evaluations of all ranks (sum)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(cells)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


NARROW_REPEAT = 10   # back-to-back node-sweep runs between the timing events


def headline_state(rank: int):
    from paper_2401_10878_gb300 import workloads as W
    st = W.settling_cubes_dense(seed=4 + 1000 * rank)
    st.indicator = 0
    st.name = "cubes1934_223"
    return st


# --workload: (description, state(seed offset) -> State); the default is the headline
WORKLOADS = {
    "cubes1934": ("1934 cuboids (edge 12) at 30% volume fraction, periodic 223^3 lattice, dx = 1", None),
    "cubes1934_smooth": ("1934 cuboids (edge 12) at 30% volume fraction, periodic 223^3 lattice, dx = 1, "
                         "smoothed indicator (w = 1 cell)", "settling_cubes_dense"),
    "mixed1934": ("1934 particles (1/3 spheres d = 14.9, 1/3 cubes edge 12, 1/3 polytopes 12-20 faces) at 30% "
                  "volume fraction, periodic 223^3 lattice", "mixed_settling"),
    "cubes400": ("400 cubes (edge 12) at 10% volume fraction, periodic 190^3 lattice", "settling_cubes"),
    "mixed27": ("27 particles (14 spheres d = 15, 13 cubes edge 12) on a jittered 3x3x3 grid, periodic 64^3 "
                "lattice", "mixed_grid_27"),
}
# the resolution sweep: 500 cubes of edge e cells at 20 % (L = round(e 2500^(1/3)))
for _e, _L in ((8, 109), (12, 163), (16, 217), (24, 326)):
    WORKLOADS[f"sweep_e{_e}"] = (f"500 cubes (edge {_e}) at 20% volume fraction, periodic {_L}^3 lattice, half of them "
                                 "axis-aligned on half-integer faces", ("resolution_sweep", _e))


def workload_state(args, rank: int):
    """The main line's state: the headline unless --workload names another."""
    from paper_2401_10878_gb300 import workloads as W
    name = getattr(args, "workload", "cubes1934")
    seed = getattr(args, "seed", None)
    if name == "cubes1934":
        st = headline_state(rank) if seed is None else W.settling_cubes_dense(seed=seed + 1000 * rank)
        st.indicator = 0
        st.name = "cubes1934_223"
        return st
    spec = WORKLOADS[name][1]
    fn, pre = (getattr(W, spec), ()) if isinstance(spec, str) else (getattr(W, spec[0]), spec[1:])
    st = fn(*pre) if seed is None and rank == 0 else fn(*pre, seed=(seed if seed is not None else 0) + 1000 * rank + 1)
    st.indicator = 1 if name == "cubes1934_smooth" else 0
    if name == "cubes1934_smooth":
        st.smooth_width = 1.0
    st.name = name
    return st


def workload_config(st, extra=None, name="cubes1934"):
    cfg = {"workload": WORKLOADS[name][0],
           "particles": st.n, "lattice": list(st.n_cells), "indicator": "smoothed" if st.indicator else "sharp",
           "pose_steps": "seeded increments dX~N(0,0.05), rot~N(0,0.01 rad)",
           "l2": "flushed (1 GiB write, > 129 MB L2) before every timed step; steps enqueued 50 at a time (flush, event, step, event each), so host stalls stay outside the timed steps", "parallelism": "weak (one box per GPU)"}
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.path is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    """The CPU FP64 oracle on the host cores, same workload and metric."""
    if rank != 0:
        return
    import oracle
    from paper_2401_10878_gb300 import workloads as W
    oracle.build()
    st = workload_state(args, 0)
    pos, quat = W.pose_sequence(st, max(args.steps + args.warmup, 1))
    threads = args.cpu_threads if args.cpu_threads > 0 else oracle.max_threads()
    gf, gt = W.loss_weights(st.n)
    for s in range(args.warmup):
        oracle.contact_step(st, pos=pos[s], quat=quat[s], n_threads=threads)
    cells, secs, gsecs = 0, 0.0, 0.0
    for s in range(args.steps):
        k = args.warmup + s
        r = oracle.contact_step(st, pos=pos[k], quat=quat[k], n_threads=threads)
        cells += r.cells
        secs += r.seconds
        if args.backward:
            t0 = time.perf_counter()
            oracle.gradient(st, gf, gt, pos=pos[k], quat=quat[k], n_threads=threads)
            gsecs += time.perf_counter() - t0
    secs += gsecs
    v = cells / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(st, None, args.workload),
            "precision": "fp64 throughout (the oracle)",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} full contact steps of the workload (all pairs)"
                                       + (", each with the FP64 gradient of the force/torque loss" if args.backward
                                          else "")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.backward:
        line["gradient_ms_per_step"] = 1e3 * gsecs / args.steps
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def output_errors(st, g, r):
    """Achieved error of each output of the GPU step g against the oracle's
    step r on the same pose, over the pairs the oracle does not flag (nodes
    within 1e-5 cells of flipping, of switching the active face or the
    deepest node) and the particles only such pairs touch: V, the first
    moments about the box origin M = V (x_c - o), the normal n (absolute),
    the depth d, the pair force and the particle sums F, T (relative to the
    sum of the magnitudes they add up)."""
    aux = r.pair_aux
    gap = aux[:, 6]
    clean = ~((aux[:, 4] > 0) | (aux[:, 5] > 0) | ((gap > 0) & (gap < 4e-5)))
    go, ro = g["pair_out"], r.pair_out
    if g["n_pairs"] != r.n_pairs or not np.array_equal(g["pair_ij"], r.pair_ij):
        return {"pair_list": "differs"}
    V = ro[:, 0]
    hit = clean & (V > 0)

    def worst(x):
        return float(np.max(x, initial=0.0))

    o = r.pair_box[:, :3] * st.dx
    Mr = V[:, None] * (ro[:, 1:4] - o)
    Mg = go[:, 0:1] * (go[:, 1:4] - o)
    den = np.maximum(np.linalg.norm(Mr, axis=1), V * st.dx)
    Fs = np.linalg.norm(ro[:, 8:11], axis=1)
    fh = hit & (Fs > 0)
    dpos = hit & (ro[:, 7] > 0)
    XA = st.pos[r.pair_ij[:, 0]]
    XB = st.pos[r.pair_ij[:, 1]] - r.pair_shift * st.box
    arm = (np.linalg.norm(ro[:, 1:4] - XA, axis=1), np.linalg.norm(ro[:, 1:4] - XB, axis=1))
    sF, sT = np.zeros(st.n), np.zeros(st.n)
    dirty = np.zeros(st.n, bool)
    dirty[r.pair_ij[~clean].ravel()] = True
    for col in (0, 1):
        np.add.at(sF, r.pair_ij[:, col], Fs)
        np.add.at(sT, r.pair_ij[:, col], Fs * arm[col])
    okF, okT = ~dirty & (sF > 0), ~dirty & (sT > 0)
    return {"pair_list": "identical", "pairs_checked": int(hit.sum()), "pairs_flagged": int((~clean).sum()),
            "V_rel": worst(np.abs(go[hit, 0] - V[hit]) / V[hit]),
            "moments_rel": worst(np.linalg.norm(Mg[hit] - Mr[hit], axis=1) / den[hit]),
            "x_c_abs_cells": worst(np.linalg.norm(go[hit, 1:4] - ro[hit, 1:4], axis=1) / st.dx),
            "n_abs": worst(np.linalg.norm(go[hit, 4:7] - ro[hit, 4:7], axis=1)),
            "d_rel": worst(np.abs(go[dpos, 7] - ro[dpos, 7]) / ro[dpos, 7]),
            "F_pair_rel": worst(np.linalg.norm(go[fh, 8:11] - ro[fh, 8:11], axis=1) / Fs[fh]),
            "F_rel": worst(np.linalg.norm(g["force"][okF] - r.force[okF], axis=1) / sF[okF]),
            "T_rel": worst(np.linalg.norm(g["torque"][okT] - r.torque[okT], axis=1) / sT[okT]),
            "bounds": {"V_rel": 1e-6, "moments_rel": 1e-6, "F_pair_rel": 1e-5, "F_rel": 1e-5, "T_rel": 1e-5}}


def cpu_baseline(st, pos, quat, budget_s, gpu0=None):
    """The oracle timed on the host cores; with gpu0 (the GPU step on pose 0)
    also the achieved error of each output against the oracle's step on it."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    cells, secs, steps = 0, 0.0, 0
    errors = None
    t_end = time.perf_counter() + budget_s
    while steps < 3 or (time.perf_counter() < t_end and steps < len(pos)):
        r = oracle.contact_step(st, pos=pos[steps % len(pos)], quat=quat[steps % len(quat)])
        if steps == 0 and gpu0 is not None:
            errors = output_errors(st.with_poses(pos[0], quat[0]), gpu0, r)
        cells += r.cells
        secs += r.seconds
        steps += 1
    # one thread, a shorter sample (about a quarter of the budget)
    c1, s1, n1 = 0, 0.0, 0
    t_end = time.perf_counter() + budget_s / 4
    while n1 < 1 or (time.perf_counter() < t_end and n1 < len(pos)):
        r = oracle.contact_step(st, pos=pos[n1 % len(pos)], quat=quat[n1 % len(quat)], n_threads=1)
        c1 += r.cells
        s1 += r.seconds
        n1 += 1
    base = {"value": cells / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} full contact steps of the workload ({cells} node evaluations), "
                      f"OpenMP over pairs", "ms_per_step": 1e3 * secs / steps,
            "one_thread": {"value": c1 / s1, "ms_per_step": 1e3 * s1 / n1, "steps": n1}}
    return (base, errors) if gpu0 is not None else base


def time_forward(model, pos_d, quat_d, steps, warmup, flush, narrow=False, vel_d=None):
    """Per-step device time (events around contact_step on the context stream),
    L2 flushed before every step.  With narrow=True the model records the
    library's events around the node-sweep launch and their times are summed."""
    import torch
    s = model.stream
    tot, narrow_ms, cells, ops = 0.0, 0.0, 0, 0
    per = []
    per_pose = {}
    npose = pos_d.shape[0]
    # steps whose counters are read (each pose's first step) or whose node-sweep
    # events are read run one at a time; the others are enqueued in batches
    # (flush, event, step, event per step) and read after the batch, so that
    # the host thread never leaves the device idle inside a timed step
    batch = 1 if narrow else 50
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(batch)]
    k = 0
    while k < warmup + steps:
        n = 1 if (k % npose) not in per_pose else min(batch, warmup + steps - k)
        for b in range(n):
            idx = (k + b) % npose
            with torch.cuda.stream(s):
                flush.zero_()
            ev[b][0].record(s)
            model.step_async(pos_d[idx], quat_d[idx], None if vel_d is None else vel_d[idx])
            ev[b][1].record(s)
        ev[n - 1][1].synchronize()
        for b in range(n):
            idx = (k + b) % npose
            if idx not in per_pose:
                st = model.stats()
                per_pose[idx] = (st["cells"], st["nominal_ops"])
            if k + b >= warmup:
                ms = ev[b][0].elapsed_time(ev[b][1])
                tot += ms
                per.append(ms)
                if narrow:
                    narrow_ms += model.narrow_time_ms()
                cells += per_pose[idx][0]
                ops += per_pose[idx][1]
        k += n
    model.check()
    return dict(ms=tot, narrow_ms=narrow_ms, cells=cells, ops=ops, per=per)


def run_ours(args, ws, rank, local):
    import torch
    from paper_2401_10878_gb300 import workloads as W
    from paper_2401_10878_gb300.contact import Contact

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    st = workload_state(args, rank)
    nseq = min(100, args.steps + args.warmup)   # the seeded pose sequence is cycled
    pos, quat = W.pose_sequence(st, nseq, seed=11 + rank)
    pos_d = torch.tensor(pos, device=dev)
    quat_d = torch.tensor(quat, device=dev)
    # 1 GiB: flushes the 129 MB L2 and lasts long enough (~0.15 ms) for the
    # host to have the step enqueued before the device reaches it
    flush = torch.empty(1024 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    model = Contact.from_state(st)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        res = time_forward(model, pos_d, quat_d, args.steps, args.warmup, flush)
        # the node sweep's own time, live, from events the library records
        # around it (second contexts, same workload and steps): around
        # NARROW_REPEAT back-to-back runs of the sweep (the per-run mean, the
        # roofline's duration), and around a single run (which adds the
        # events' own overhead, reported beside it)
        nsteps = min(args.steps, 1000)
        tmodel = Contact.from_state(st, narrow_events=NARROW_REPEAT)
        tres = time_forward(tmodel, pos_d, quat_d, nsteps, args.warmup, flush, narrow=True)
        tmodel.close()
        tmodel = Contact.from_state(st, narrow_events=1)
        tres1 = time_forward(tmodel, pos_d, quat_d, nsteps, args.warmup, flush, narrow=True)
        tmodel.close()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.summary()
    t_max, total_cells = combine_ranks(res["ms"], res["cells"], dev)
    value = total_cells / (t_max * 1e-3)
    ms_per_step = t_max / args.steps
    stats = model.stats()

    # roofline of the node-sweep kernel: nominal FP32 lane-ops / its event time
    narrow_avg_s = tres["narrow_ms"] * 1e-3 / nsteps
    ops_per_launch = tres["ops"] / nsteps
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    peak = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12          # T lane-ops/s
    achieved = ops_per_launch / narrow_avg_s / 1e12
    med = clocks.get("sm_mhz")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 lane-ops/s",
                "frac": achieved / peak,
                "traffic": traffic_from_profile() if args.workload == "cubes1934" and args.seed is None else None,
                "kernel": "k_narrow32 (node sweep)", "ops_per_launch": ops_per_launch,
                "launch_ms": narrow_avg_s * 1e3,
                "launch_ms_single": tres1["narrow_ms"] / nsteps,
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {max_mhz:.0f} MHz (max SM clock)",
                "frac_at_median_clock": (achieved / (sms * FP32_LANES_PER_SM * med * 1e6 / 1e12)) if med else None,
                "cell_evals_per_s_kernel": (tres["cells"] / nsteps) / narrow_avg_s,
                "timing": f"CUDA events around {NARROW_REPEAT} back-to-back node-sweep runs per step (their mean), "
                          f"{nsteps} steps of the same workload; launch_ms_single: events around one run"}
    # the derived peak checked against this GPU's measured FFMA rate
    try:
        from paper_2401_10878_gb300.contact import fp32_ffma_rate
        ffma = fp32_ffma_rate() / 1e12
        roofline["peak_ffma_measured"] = ffma
        roofline["frac_of_measured_ffma"] = achieved / ffma
    except Exception as e:   # a measurement aid only: the line stands without it
        roofline["peak_ffma_measured"] = None
        roofline["peak_ffma_error"] = str(e)[:200]

    # end to end through the public API with host buffers
    e2e = end_to_end(model, pos, quat, args.steps, args.warmup, dev)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(st, None, args.workload),
            "precision": "fp32 node tests, fp32 tile partials, fp64 pair/particle reductions",
            "step_stats": {"pairs_per_step": stats["pairs"], "cells_per_step": res["cells"] / args.steps,
                           "overlapping_pairs": stats["overlapping"], "tiles_per_step": stats["tiles"],
                           "narrow_grid": stats["narrow_grid"]},
            "roofline": roofline, "e2e": e2e, "gpu_launches": model.kernels_per_step() * args.steps,
            "clocks": clocks,
            "ms_per_step_median": float(np.median(res["per"])),
            "ms_per_step_p10_p90": [float(np.percentile(res["per"], 10)), float(np.percentile(res["per"], 90))]}
    if rank == 0 and not args.no_cpu:
        # one checked step outside the timed region: the first pose, whose
        # oracle step the CPU leg runs first
        ref_out = model.step(pos_d[0], quat_d[0])
        gpu0 = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in ref_out.items()}
        line["cpu_baseline"], line["errors"] = cpu_baseline(st, pos, quat, args.cpu_seconds, gpu0)
    if rank == 0 and not args.no_extras:
        line["extras"] = extras(args, dev, flush, peak)
    model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def end_to_end(model, pos, quat, steps, warmup, dev):
    """The same step through the C-ABI call with HOST buffers
    (contact_step_host): page-locked host poses in, host forces and torques
    out, the transfers inside the call (the step's kernels read and write the
    mapped host buffers over the host link); wall-clock time per call."""
    import torch
    hp = torch.tensor(pos).pin_memory()
    hq = torch.tensor(quat).pin_memory()
    hf = torch.empty((model.n, 3), dtype=torch.float64).pin_memory()
    ht = torch.empty((model.n, 3), dtype=torch.float64).pin_memory()
    xp = torch.empty_like(hp[0]).pin_memory()   # the caller's input buffers, reused every step
    xq = torch.empty_like(hq[0]).pin_memory()
    tot, cells = 0.0, 0
    per_pose = {}
    per = []
    for k in range(warmup + steps):
        idx = k % hp.shape[0]
        xp.copy_(hp[idx])   # the caller fills its buffers (not timed)
        xq.copy_(hq[idx])
        t0 = time.perf_counter()
        model.step_host(xp, xq, force=hf, torque=ht)
        t1 = time.perf_counter()
        if idx not in per_pose:
            per_pose[idx] = model.stats()["cells"]
        if k >= warmup:
            tot += t1 - t0
            cells += per_pose[idx]
            per.append(t1 - t0)
    n = model.n
    return {"value": cells / tot, "unit": UNIT, "h2d_bytes_per_step": n * 7 * 8,
            "d2h_bytes_per_step": n * 6 * 8 + 4, "ms_per_step": 1e3 * tot / steps,
            "ms_per_step_median": 1e3 * float(np.median(per)),
            "ms_per_step_p10_p90": [1e3 * float(np.percentile(per, 10)), 1e3 * float(np.percentile(per, 90))],
            "timing": "wall clock around contact_step_host (pinned host buffers read and written by the step's "
                      "kernels inside the call)"}


def box_volume_percentiles(m, st, pos):
    """Pair-box volumes (nodes) of the last step, from the GPU's node ranges and
    pair list: the same box as the library's (partner image by the FP32
    position difference against L/2)."""
    import torch
    m.step(torch.tensor(pos, device=m.device), torch.tensor(st.quat, device=m.device))
    P = int(m.n_pairs.item())
    ij = m.pair_ij[:P].cpu().numpy()
    lohi = m.particle_boxes().cpu().numpy().astype(np.int64)
    X = np.asarray(pos, dtype=np.float64).astype(np.float32)
    d = X[ij[:, 1]] - X[ij[:, 0]]
    h = (0.5 * np.asarray(st.n_cells, dtype=np.float64) * st.dx).astype(np.float32)
    sft = (d > h).astype(np.int64) - (d < -h).astype(np.int64)
    n = np.asarray(st.n_cells, dtype=np.int64)
    lo = np.maximum(lohi[ij[:, 0], :3], lohi[ij[:, 1], :3] - sft * n)
    hi = np.minimum(lohi[ij[:, 0], 3:], lohi[ij[:, 1], 3:] - sft * n)
    vol = np.prod(np.maximum(hi - lo + 1, 0), axis=1)
    return [float(v) for v in np.percentile(vol, [10, 50, 90, 99])] if P else []


def extras(args, dev, flush, peak):
    """Secondary workloads, each timed like the headline (no CPU leg)."""
    import torch
    from paper_2401_10878_gb300 import workloads as W
    from paper_2401_10878_gb300.contact import Contact, FP64_PAIR

    out = {}
    steps = max(5, min(args.steps, 50))
    # mixed spheres / cubes / polytopes at 30 %
    st = W.mixed_settling()
    pos, quat = W.pose_sequence(st, steps + 3)
    m = Contact.from_state(st, narrow_events=True)
    r = time_forward(m, torch.tensor(pos, device=dev), torch.tensor(quat, device=dev), steps, 3, flush, narrow=True)
    s = m.stats()
    m.close()
    # the node sweep's roofline on this workload: the mean of back-to-back runs (as the headline's)
    m = Contact.from_state(st, narrow_events=NARROW_REPEAT)
    rr = time_forward(m, torch.tensor(pos, device=dev), torch.tensor(quat, device=dev), steps, 3, flush, narrow=True)
    achieved = rr["ops"] / (rr["narrow_ms"] * 1e-3) / 1e12
    out["mixed1934_223"] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / steps,
                            "narrow_ms_single": r["narrow_ms"] / steps, "pairs": s["pairs"],
                            "tiles_per_step": s["tiles"], "cells_per_step": r["cells"] / steps,
                            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 lane-ops/s",
                                         "frac": achieved / peak, "launch_ms": rr["narrow_ms"] / steps,
                                         "ops_per_launch": rr["ops"] / steps,
                                         "timing": f"CUDA events around {NARROW_REPEAT} back-to-back node-sweep runs"}}
    out["mixed1934_223"]["box_volume_percentiles_10_50_90_99"] = box_volume_percentiles(m, st, st.pos)
    m.close()
    m = Contact.from_state(st, precision=FP64_PAIR, narrow_events=True)
    r = time_forward(m, torch.tensor(pos, device=dev), torch.tensor(quat, device=dev), steps, 3, flush, narrow=True)
    out["mixed1934_223"]["fp64_form"] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3),
                                         "ms_per_step": r["ms"] / steps, "narrow_ms": r["narrow_ms"] / steps}
    m.close()
    # all-FP64 one-pair-per-block form on the headline workload
    st = headline_state(0)
    pos, quat = W.pose_sequence(st, steps + 3)
    m = Contact.from_state(st, precision=FP64_PAIR, narrow_events=True)
    r = time_forward(m, torch.tensor(pos, device=dev), torch.tensor(quat, device=dev), steps, 3, flush, narrow=True)
    out["cubes1934_fp64_form"] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3),
                                  "ms_per_step": r["ms"] / steps, "narrow_ms": r["narrow_ms"] / steps}
    m.close()
    # its node sweep against the FP64 pipe: the same nominal lane-ops, in FP64, over the
    # measured DFMA rate of this GPU
    try:
        from paper_2401_10878_gb300.contact import fp64_dfma_rate
        dfma = fp64_dfma_rate() / 1e12
        a64 = r["ops"] / (r["narrow_ms"] * 1e-3) / 1e12
        out["cubes1934_fp64_form"]["roofline"] = {"bound": "fp64", "achieved": a64, "peak": dfma,
                                                  "unit": "T FP64 lane-ops/s", "frac": a64 / dfma,
                                                  "peak_basis": "measured DFMA rate (contact_fp64_dfma_rate)"}
    except Exception as e:   # a measurement aid only
        out["cubes1934_fp64_form"]["roofline_error"] = str(e)[:200]
    # the headline workload with velocities: shared damping, then contact history + friction
    # (timed like the other extras, with the library's events around the node sweep; the
    # first entry, without velocities, is the same timing of the headline step)
    st = headline_state(0)
    pos, quat = W.pose_sequence(st, steps + 3)
    rng = np.random.default_rng(17)
    vel = np.concatenate([rng.normal(size=(steps + 3, st.n, 3)) * 0.05,
                          rng.normal(size=(steps + 3, st.n, 3)) * 0.01], axis=2)
    pd, qd, vd = (torch.tensor(x, device=dev) for x in (pos, quat, vel))
    law = {}
    for name, kw in (("no_velocities", dict()), ("shared_damping", dict(damping_c=0.3)),
                     ("history_friction", dict(history=True, restitution=0.5, friction=True, mu_s=0.5, mu_k=0.3,
                                               u_k=0.02))):
        m = Contact.from_state(st, narrow_events=True, **kw)
        r = time_forward(m, pd, qd, steps, 3, flush, narrow=True, vel_d=vd if kw else None)
        law[name] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / steps,
                     "narrow_ms": r["narrow_ms"] / steps, "overlapping_pairs": m.stats()["overlapping"]}
        if kw.get("history"):
            law[name]["contacts_in_history"] = int(len(m.history()[1]))
        m.close()
    out["cubes1934_velocities"] = law
    # the paper's box pipeline on the headline workload (rough detection, box
    # correction, N_c^3 samples), N_c = 8 as in the paper's runs, and 16
    boxm = {}
    for nc in (8, 16):
        st_b = dataclasses.replace(headline_state(0))
        st_b.box_mode, st_b.contact_resolution = 1, nc
        m = Contact.from_state(st_b, narrow_events=True)
        r = time_forward(m, pd, qd, steps, 3, flush, narrow=True)
        s_ = m.stats()
        # roofline of the box kernel: the nominal FP32 lane-ops of its sample
        # tests (the overlapping pairs' N_c^3 samples, the same ops per test as
        # the node sweep's) against the FP32 peak; its FP64 pipe is the busier
        # unit (ncu: 55 % of active cycles at N_c = 8)
        kern_s = r["narrow_ms"] / steps * 1e-3
        ops_per_test = s_["nominal_ops"] / max(s_["cells"], 1)
        sample_ops = s_["overlapping"] * nc ** 3 * ops_per_test
        boxm[f"nc{nc}"] = {"ms_per_step": r["ms"] / steps, "box_kernel_ms": r["narrow_ms"] / steps,
                           "pairs": s_["pairs"], "pairs_with_overlap": s_["overlapping"],
                           "samples_per_step": s_["overlapping"] * nc ** 3,
                           "roofline": {"bound": "fp64 pipe", "achieved": sample_ops / kern_s / 1e12,
                                        "peak": peak, "unit": "T FP32 lane-ops/s (sample tests)",
                                        "frac": sample_ops / kern_s / (peak * 1e12)}}
        m.close()
    # N_c = 8 with the contact history (each contact's c and its corrected box,
    # the next correction's warm start) and friction, velocities as above
    st_b = dataclasses.replace(headline_state(0))
    st_b.box_mode, st_b.contact_resolution = 1, 8
    m = Contact.from_state(st_b, narrow_events=True, history=True, restitution=0.5, friction=True, mu_s=0.5,
                           mu_k=0.3, u_k=0.02)
    r = time_forward(m, pd, qd, steps, 3, flush, narrow=True, vel_d=vd)
    s_ = m.stats()
    boxm["nc8_history_friction"] = {"ms_per_step": r["ms"] / steps, "box_kernel_ms": r["narrow_ms"] / steps,
                                    "pairs": s_["pairs"], "pairs_with_overlap": s_["overlapping"],
                                    "contacts_in_history": int(len(m.history()[1]))}
    m.close()
    out["cubes1934_box_pipeline"] = boxm
    # the headline workload between a floor and a ceiling (fixed walls, 2 of them)
    st_w = W.floor_and_ceiling(headline_state(0))
    m = Contact.from_state(st_w, narrow_events=True)
    r = time_forward(m, pd, qd, steps, 3, flush, narrow=True)
    s_ = m.stats()
    ij = m.pair_ij[:s_["pairs"]].cpu().numpy()
    out["cubes1934_floor_ceiling"] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / steps,
                                      "narrow_ms": r["narrow_ms"] / steps, "pairs": s_["pairs"],
                                      "wall_pairs": int((ij[:, 1] >= st_w.n).sum()),
                                      "cells_per_step": r["cells"] / steps}
    m.close()
    # 400 cubes at 10 %, and the resolution sweep (500 cubes at 20 %, edge 8..24), both forms
    def both_forms(st, nsteps):
        pos, quat = W.pose_sequence(st, nsteps + 3)
        pd, qd = torch.tensor(pos, device=dev), torch.tensor(quat, device=dev)
        res = {"L": int(st.n_cells[0])}
        for name, prec in (("fp32_tile", 0), ("fp64_form", FP64_PAIR)):
            m = Contact.from_state(st, precision=prec, narrow_events=True)
            r = time_forward(m, pd, qd, nsteps, 3, flush, narrow=True)
            s_ = m.stats()
            res[name] = {"cell_evals_per_s": r["cells"] / (r["ms"] * 1e-3), "ms_per_step": r["ms"] / nsteps,
                         "narrow_ms": r["narrow_ms"] / nsteps}
            if prec == 0:
                res.update(pairs=s_["pairs"], cells_per_step=r["cells"] / nsteps)
                res[name]["node_sweep_frac_of_fp32_peak"] = (r["ops"] / (r["narrow_ms"] * 1e-3)) / (peak * 1e12)
            m.close()
        return res
    out["cubes400_190"] = both_forms(W.settling_cubes(), steps)
    out["mixed27_64"] = both_forms(W.mixed_grid_27(), steps)
    out["resolution_sweep"] = {f"edge{e}": both_forms(W.resolution_sweep(e), min(steps, 20)) for e in (8, 12, 16, 24)}
    # smoothed indicator: forward + adjoint
    st = W.settling_cubes_dense()
    pos, quat = W.pose_sequence(st, steps + 3)
    m = Contact.from_state(st, narrow_events=True)
    gf, gt = W.loss_weights(st.n)
    gf, gt = torch.tensor(gf, device=dev), torch.tensor(gt, device=dev)
    gp = torch.empty((st.n, 3), dtype=torch.float64, device=dev)
    gq = torch.empty((st.n, 4), dtype=torch.float64, device=dev)
    pd, qd = torch.tensor(pos, device=dev), torch.tensor(quat, device=dev)
    fwd, bwd, cells, adj_ms, ops = 0.0, 0.0, 0, 0.0, 0
    import ctypes
    for k in range(steps + 3):
        with torch.cuda.stream(m.stream):
            flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(m.stream)
        m.step_async(pd[k], qd[k])
        e1.record(m.stream)
        rc = m.lib.contact_backward(m.ctx, ctypes.c_void_p(gf.data_ptr()), ctypes.c_void_p(gt.data_ptr()),
                                    ctypes.c_void_p(gp.data_ptr()), ctypes.c_void_p(gq.data_ptr()))
        assert rc == 0
        e2.record(m.stream)
        e2.synchronize()
        if k >= 3:
            fwd += e0.elapsed_time(e1)
            bwd += e1.elapsed_time(e2)
            st_ = m.stats()
            cells += st_["cells"]
            ops += st_["nominal_ops"]
            adj_ms += m.adjoint_time_ms()
    m.check()
    # the adjoint's cell sweep against the FP32 peak: the forward's nominal lane-ops of the
    # two distance tests per node of every pair box (it sweeps the same nodes), over its
    # event-timed duration (one launch between the events)
    aa = ops / (adj_ms * 1e-3) / 1e12
    out["cubes1934_smooth_fwd_bwd"] = {"fwd_ms": fwd / steps, "bwd_ms": bwd / steps,
                                       "cell_evals_per_s_fwd_bwd": cells / ((fwd + bwd) * 1e-3),
                                       "cells_per_step": cells / steps,
                                       "adjoint_cell_sweep": {"bound": "alu", "achieved": aa, "peak": peak,
                                                              "unit": "T FP32 lane-ops/s", "frac": aa / peak,
                                                              "launch_ms": adj_ms / steps,
                                                              "timing": "CUDA events around its launch"}}
    m.close()
    return out


def node_sweep_source_hash():
    """Hash of the sources the node-sweep kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in ("k_narrow.cu", "force_law.cuh", "contact_dev.cuh", "line_clip.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2401_10878_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile():
    """DRAM bytes per launch of the node sweep from the committed ncu summary,
    only while the kernel source is unchanged since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_narrow32_cubes1934.md")
    if not os.path.exists(path):
        return None
    h = node_sweep_source_hash()
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].rsplit(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("node sweep sources sha256[:16]") != h:
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
