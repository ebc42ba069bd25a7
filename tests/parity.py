"""Shared comparison of the CUDA contact step with the FP64 oracle.

Tolerances (north star, restated): the candidate pair list and the particle
node ranges are compared bit for bit; volume and first moments within 1e-6
relative; force and torque within 1e-5 relative (FP32-tile form).  Where
floating point decides an integer -- a node's inside/outside class, the
active face behind the normal, the deepest node -- the oracle reports the
nodes whose decision lies within BAND_EPS = 1e-5 lattice units of flipping.
Pairs with such nodes are "flagged": their volume must stay within the
flagged-node count of the oracle's, the rest is reported, not asserted.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

BAND = oracle.BAND_EPS


@dataclasses.dataclass
class Report:
    pairs: int
    cells: int
    flagged: int
    flips: int
    max_rel: dict

    def __str__(self):
        r = ", ".join(f"{k}={v:.2e}" for k, v in self.max_rel.items())
        return f"pairs={self.pairs} cells={self.cells} flagged={self.flagged} flips={self.flips} {r}"


def gpu_step(model, st, pos=None, quat=None, vel=None):
    import torch
    pos = st.pos if pos is None else pos
    quat = st.quat if quat is None else quat
    dev = model.device
    tp = torch.tensor(pos, dtype=torch.float64, device=dev).contiguous()
    tq = torch.tensor(quat, dtype=torch.float64, device=dev).contiguous()
    tv = None if vel is None else torch.tensor(vel, dtype=torch.float64, device=dev).contiguous()
    out = model.step(tp, tq, tv)
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}


def rel(a, b, scale):
    return np.abs(a - b) / np.maximum(scale, 1e-300)


def compare(st, g, r, fp64: bool, smooth: bool) -> Report:
    """Assert parity of GPU outputs g against the oracle result r."""
    assert g["n_pairs"] == r.n_pairs, (g["n_pairs"], r.n_pairs)
    assert np.array_equal(g["pair_ij"], r.pair_ij), "pair list differs"
    go, ro, aux = g["pair_out"], r.pair_out, r.pair_aux
    dx3 = st.dx ** 3
    gap = aux[:, 6]
    amb_d = (gap > 0) & (gap < 4 * BAND)
    flagged = (aux[:, 4] > 0) | (aux[:, 5] > 0) | amb_d
    if fp64:
        flagged = np.zeros_like(flagged)
    clean = ~flagged
    out = {}
    # volume: exact counts in sharp mode, 1e-6 relative otherwise
    Vs = np.maximum(np.abs(ro[:, 0]), dx3)
    vt = 1e-9 if fp64 else (0.0 if not smooth else 1e-6)
    e = rel(go[clean, 0], ro[clean, 0], Vs[clean])
    out["V"] = float(e.max(initial=0))
    assert np.all(e <= vt + 1e-12), f"volume beyond tolerance: {e.max()}"
    flips = np.rint(np.abs(go[flagged, 0] - ro[flagged, 0]) / dx3)
    if not smooth:
        assert np.all(flips <= aux[flagged, 4] + 1e-9), "classification flips outside the band"
    hit = clean & (ro[:, 0] > 0)
    # contact point: first moments / volume
    L = float(np.max(st.box))
    e = np.abs(go[hit, 1:4] - ro[hit, 1:4]).max(axis=1, initial=0) / L
    out["x_c"] = float(e.max(initial=0))
    assert np.all(e <= (1e-12 if (fp64 or not smooth) else 1e-6)), f"contact point: {e.max()}"
    # normal (unit vector): FP32 band sums
    e = np.abs(go[hit, 4:7] - ro[hit, 4:7]).max(axis=1, initial=0)
    out["n"] = float(e.max(initial=0))
    assert np.all(e <= (1e-9 if fp64 else 1e-5)), f"normal: {e.max()}"
    # depth: FP64 re-evaluation at the deepest node
    e = np.abs(go[hit, 7] - ro[hit, 7]) / st.dx
    out["d"] = float(e.max(initial=0))
    assert np.all(e <= (1e-9 if fp64 else 1e-6)), f"depth: {e.max()}"
    # force on the pair
    Fs = np.linalg.norm(ro[hit, 8:11], axis=1)
    e = np.abs(go[hit, 8:11] - ro[hit, 8:11]).max(axis=1, initial=0) / np.maximum(Fs, 1e-300)
    e[Fs == 0] = np.abs(go[hit, 8:11][Fs == 0]).max(axis=1, initial=0)
    out["F_pair"] = float(e.max(initial=0))
    assert np.all(e <= (1e-9 if fp64 else 1e-5)), f"pair force: {e.max()}"
    # zero pairs stay exactly zero
    zero = clean & (ro[:, 0] == 0)
    assert np.all(go[zero] == 0.0)
    # per-particle sums: scale = sum of |pair force| (and |torque|) touching the particle
    touched_flag = np.zeros(st.n, bool)
    touched_flag[r.pair_ij[flagged].ravel()] = True
    Fabs = np.linalg.norm(ro[:, 8:11], axis=1)
    sF = np.zeros(st.n)
    np.add.at(sF, r.pair_ij[:, 0], Fabs)
    np.add.at(sF, r.pair_ij[:, 1], Fabs)
    ok = ~touched_flag & (sF > 0)
    e = np.abs(g["force"][ok] - r.force[ok]).max(axis=1, initial=0) / sF[ok]
    out["F"] = float(e.max(initial=0))
    assert np.all(e <= (1e-9 if fp64 else 1e-5)), f"particle force: {e.max()}"
    Tabs = np.linalg.norm(r.torque, axis=1)
    XA = st.pos[r.pair_ij[:, 0]]
    xc = ro[:, 1:4]
    arm = np.linalg.norm(xc - XA, axis=1)
    sT = np.zeros(st.n)
    np.add.at(sT, r.pair_ij[:, 0], Fabs * (arm + st.dx))
    np.add.at(sT, r.pair_ij[:, 1], Fabs * (arm + st.dx))
    ok = ok & (sT > 0)
    e = np.abs(g["torque"][ok] - r.torque[ok]).max(axis=1, initial=0) / sT[ok]
    out["T"] = float(e.max(initial=0))
    assert np.all(e <= (1e-9 if fp64 else 1e-5)), f"particle torque: {e.max()}"
    del Tabs
    none = ~(sF > 0) & ~touched_flag
    assert np.all(g["force"][none] == 0.0) and np.all(g["torque"][none] == 0.0)
    return Report(r.n_pairs, r.cells, int(flagged.sum()), int(flips.sum()), out)
