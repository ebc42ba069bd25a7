"""Run a few contact steps (and optionally backwards) of a synthetic workload
on cuda:0: a short, self-contained driver for profilers and smoke checks.

    python -m paper_2401_10878_gb300.run_steps --workload cubes1934 --steps 5
    python -m paper_2401_10878_gb300.run_steps --workload cubes1934_smooth --steps 5 --backward

Workloads: cubes1934 (1934 cubes of edge 12 at 30 % in 223^3, sharp),
cubes1934_smooth (the same, smoothed indicator w = 1), mixed1934 (spheres,
cubes and polytopes at 30 % in 223^3), cubes400 (400 cubes at 10 % in 190^3),
box8 (cubes1934 with the paper's box pipeline, N_c = 8).  Seeded pose
sequence as in the benchmark; prints the pair count and the last step's
device time.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import workloads as W


def state(name: str):
    if name in ("cubes1934", "cubes1934_smooth", "box8"):
        st = W.settling_cubes_dense()
        st.indicator = 1 if name == "cubes1934_smooth" else 0
        if name == "box8":
            st.box_mode, st.contact_resolution = 1, 8
        return st
    if name == "mixed1934":
        return W.mixed_settling()
    if name == "cubes400":
        return W.settling_cubes()
    raise ValueError(f"unknown workload {name}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="cubes1934",
                    choices=["cubes1934", "cubes1934_smooth", "mixed1934", "cubes400", "box8"])
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--backward", action="store_true", help="a contact_backward after every step (smoothed)")
    args = ap.parse_args(argv)
    import torch

    from .contact import Contact
    st = state(args.workload)
    pos, quat = W.pose_sequence(st, max(args.steps, 1))
    dev = torch.device("cuda", 0)
    m = Contact.from_state(st)
    gf, gt = (torch.tensor(x, device=dev) for x in W.loss_weights(st.n))
    ms = 0.0
    for k in range(args.steps):
        p, q = torch.tensor(pos[k], device=dev), torch.tensor(quat[k], device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(m.stream)
        m.step_async(p, q)
        if args.backward:
            m.backward(gf, gt, check=False)
        e1.record(m.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
    m.check()
    print(f"{args.workload}: {m.stats()['pairs']} pairs, last step {ms * 1e3:.1f} us"
          + (" (with backward)" if args.backward else ""))
    m.close()


if __name__ == "__main__":
    main()
