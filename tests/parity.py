"""Shared comparison of the CUDA contact step with the FP64 oracle.

Tolerances: the candidate pair list and the particle
node ranges are compared bit for bit; volume and first moments within 1e-6
relative; force and torque within 1e-5 relative (FP32-tile form).

FP32 evaluates every signed distance with an absolute error below
EPS = 1e-5 lattice units (node coordinates are exact integers minus an FP32
remainder in [-1/2, 1/2]; |r| and face offsets stay below ~25 cells, so the
three FP32 roundings of a face value stay below ~8e-6).  Consequences:
  * sharp indicator: a node can change class only if |phi| < EPS.  The oracle
    reports, per pair, the nodes within EPS of flipping (and of switching the
    active face or the deepest node).  Pairs with such nodes are "flagged":
    their volume must stay within the flagged-node count, the remaining
    outputs are reported, not asserted.  Unflagged pairs: V and the moments are
    integer sums and must match exactly.
  * smoothed indicator (and the normal's band sums in both modes): outputs are
    continuous in phi, so their deviation is bounded by the oracle's
    first-order sensitivity sum_nodes |d(.)/dphi| EPS (reported per pair),
    on top of the 1e-6 / 1e-5 relative tolerances.
The all-FP64 form has no EPS: everything within 1e-9.
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
    max_err: dict            # worst err / tol ratio per check (<= 1 passes)
    rel: dict = dataclasses.field(default_factory=dict)   # achieved error per output (output_errors)

    def __str__(self):
        r = ", ".join(f"{k}={v:.2e}" for k, v in self.max_err.items())
        e = ", ".join(f"{k}={v:.2e}" for k, v in self.rel.items())
        return f"pairs={self.pairs} cells={self.cells} flagged={self.flagged} flips={self.flips} ratios: {r} | errors: {e}"


# The bounds the benchmark spec fixes for the FP32-tile form: volume and first
# moments 1e-6 relative, force and torque 1e-5 relative.
FLAT = {"V": 1e-6, "M": 1e-6, "F_pair": 1e-5, "F": 1e-5, "T": 1e-5}


def output_errors(st, g, r, clean, ro=None, r_force=None, r_torque=None) -> dict:
    """Achieved error of each output against the oracle, over the pairs in
    `clean` (unflagged) and the particles that only such pairs touch:
      V       max |dV| / V                          (pairs with V > 0)
      M       max |dM| / |M|, M = V (x_c - o) the first moments about the
              box origin o (|M| floored at V dx)
      x_c     max |dx_c| / dx                       (absolute, cells)
      n       max |dn|                              (unit vector)
      d       max |dd| / d
      F_pair  max |dF| / |F|                        (pairs with F != 0)
      F, T    per particle max |dF_p| / sum |F_pair| and |dT_p| / sum |F_pair| |arm|
              over its pairs (the scale of the sum, which may cancel)."""
    ro = r.pair_out if ro is None else ro
    r_force = r.force if r_force is None else r_force
    r_torque = r.torque if r_torque is None else r_torque
    go = g["pair_out"]
    dx = st.dx
    V = ro[:, 0]
    hit = clean & (V > 0)
    out = {}

    def worst(x):
        return float(np.max(x, initial=0.0))

    out["V"] = worst(np.abs(go[hit, 0] - V[hit]) / V[hit])
    o = r.pair_box[:, :3] * dx
    Mr = V[:, None] * (ro[:, 1:4] - o)
    Mg = go[:, 0:1] * (go[:, 1:4] - o)
    den = np.maximum(np.linalg.norm(Mr, axis=1), V * dx)
    out["M"] = worst(np.linalg.norm(Mg[hit] - Mr[hit], axis=1) / den[hit])
    out["x_c"] = worst(np.linalg.norm(go[hit, 1:4] - ro[hit, 1:4], axis=1) / dx)
    out["n"] = worst(np.linalg.norm(go[hit, 4:7] - ro[hit, 4:7], axis=1))
    dpos = hit & (ro[:, 7] > 0)
    out["d"] = worst(np.abs(go[dpos, 7] - ro[dpos, 7]) / ro[dpos, 7])
    Fs = np.linalg.norm(ro[:, 8:11], axis=1)
    fh = hit & (Fs > 0)
    out["F_pair"] = worst(np.linalg.norm(go[fh, 8:11] - ro[fh, 8:11], axis=1) / Fs[fh])
    nrow = st.n + len(getattr(st, "walls", ()))
    pos_w = np.concatenate([st.pos, np.zeros((nrow - st.n, 3))])
    XA = pos_w[r.pair_ij[:, 0]]
    XB = pos_w[r.pair_ij[:, 1]] - r.pair_shift * st.box
    armA = np.linalg.norm(ro[:, 1:4] - XA, axis=1)
    armB = np.linalg.norm(ro[:, 1:4] - XB, axis=1)
    sF = np.zeros(nrow)
    sT = np.zeros(nrow)
    dirty = np.zeros(nrow, bool)
    dirty[r.pair_ij[~clean].ravel()] = True
    for col, arm in ((0, armA), (1, armB)):
        np.add.at(sF, r.pair_ij[:, col], Fs)
        np.add.at(sT, r.pair_ij[:, col], Fs * arm)
    sF, sT, dirty = sF[:st.n], sT[:st.n], dirty[:st.n]
    okF = ~dirty & (sF > 0)
    out["F"] = worst(np.linalg.norm(g["force"][okF] - r_force[okF], axis=1) / sF[okF])
    okT = ~dirty & (sT > 0)
    out["T"] = worst(np.linalg.norm(g["torque"][okT] - r_torque[okT], axis=1) / sT[okT])
    return out


def assert_flat(rep: Report, bounds=None):
    """Assert the benchmark spec's flat relative bounds on the achieved errors."""
    bounds = FLAT if bounds is None else bounds
    for k, b in bounds.items():
        assert rep.rel[k] <= b, f"{k}: achieved error {rep.rel[k]:.3e} above the bound {b:.0e} ({rep})"


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


def _check(name, err, tol, out):
    """Record the largest err/tol ratio and assert err <= tol elementwise."""
    err = np.asarray(err, float)
    tol = np.asarray(tol, float)
    ratio = err / np.maximum(tol, 1e-300)
    out[name] = float(ratio.max(initial=0.0))
    assert np.all(err <= tol), f"{name}: err {err.max(initial=0):.3e} beyond tolerance (worst ratio {ratio.max():.2f})"


def compare(st, g, r, fp64: bool, smooth: bool, forces=None, tol_force=None, box=None) -> Report:
    """Assert parity of GPU outputs g against the oracle result r.  The
    report's numbers are the worst error / tolerance ratios (<= 1 passes).

    forces = (pair F [P,3], force [N,3], torque [N,3]) replaces r's forces
    (the oracle's contact-law extensions); tol_force(toln, tolx, tolV, told)
    then returns the per-pair force tolerance and the pairs whose forces are
    reported, not asserted (their particles' sums too, like flagged pairs).

    box = (dV [P], flag [P], ext [P]) for the box pipeline: the volume of one
    sample (counts are exact, the sample volume to FP64 rounding of the box
    corners, relative 1e-12 L / ext for the box's smallest extent ext), the
    pairs whose rough box or face correction the oracle reports within eps of
    changing."""
    assert g["n_pairs"] == r.n_pairs, (g["n_pairs"], r.n_pairs)
    assert np.array_equal(g["pair_ij"], r.pair_ij), "pair list differs"
    go, ro, aux = g["pair_out"], r.pair_out.copy(), r.pair_aux
    r_force, r_torque = r.force, r.torque
    if forces is not None:
        ro[:, 8:11] = forces[0]
        r_force, r_torque = forces[1], forces[2]
    dx, dx3 = st.dx, st.dx ** 3
    L = float(np.max(st.box))
    gap = aux[:, 6]
    flagged = (aux[:, 4] > 0) | (aux[:, 5] > 0) | ((gap > 0) & (gap < 4 * BAND))
    if fp64:
        flagged = np.zeros_like(flagged)
    unit = np.full(len(flagged), dx3)   # volume of one sample
    if box is not None:
        unit = np.where(box[0] > 0, box[0], dx3)
        flagged = flagged | box[1]
    clean = ~flagged
    out = {}
    V = ro[:, 0]
    vsens = np.zeros(len(V)) if (fp64 or not smooth) else aux[:, 8]
    msens = np.zeros(len(V)) if (fp64 or not smooth) else aux[:, 9]
    gsens = np.zeros(len(V)) if fp64 else aux[:, 10]
    Gn = np.linalg.norm(aux[:, :3], axis=1)
    rel = 1e-9 if fp64 else 1e-6
    relF = 1e-9 if fp64 else 1e-5
    # volume
    tolV = rel * np.maximum(V, dx3) + vsens
    if not smooth and not fp64:
        tolV = np.zeros_like(V) if box is None else 1e-12 * V * (1 + L / np.maximum(box[2], 1e-300))
    _check("V", np.abs(go[clean, 0] - V[clean]), tolV[clean], out)
    flips = np.rint(np.abs(go[flagged, 0] - V[flagged]) / unit[flagged])
    if not smooth:
        assert np.all(flips <= aux[flagged, 4] + 1e-9), "classification flips outside the band"
    hit = clean & (V > 0)
    # contact point x_c = o + M / V
    o = r.pair_box[:, :3] * dx
    arm_o = np.linalg.norm(ro[:, 1:4] - o, axis=1)
    # FP32 moments are summed in box coordinates: their rounding scales with the pair box, not the lattice
    ext = (r.pair_box[:, 3:6] - r.pair_box[:, :3] + 1).max(axis=1) * dx
    tolx = np.where(V > 0, (msens + arm_o * vsens) / np.maximum(V, 1e-300), 0) + rel * ext
    if not smooth and not fp64:
        tolx = np.full(len(V), 1e-12 * L)
    _check("x_c", np.abs(go[hit, 1:4] - ro[hit, 1:4]).max(axis=1, initial=0), tolx[hit], out)
    # normal n = G / |G| (FP32 band sums)
    toln = relF + 2.0 * gsens / np.maximum(Gn, 1e-300)
    _check("n", np.abs(go[hit, 4:7] - ro[hit, 4:7]).max(axis=1, initial=0), toln[hit], out)
    # depth: FP64 re-evaluation at the deepest node
    told = (1e-9 if fp64 else 1e-6) * dx
    _check("d", np.abs(go[hit, 7] - ro[hit, 7]), np.full(hit.sum(), told), out)
    # pair force: |F| ~ sqrt(V d) |n|
    Fs = np.linalg.norm(ro[:, 8:11], axis=1)
    d = np.maximum(ro[:, 7], 1e-300)
    tolFrel = relF + 0.5 * tolV / np.maximum(V, 1e-300) + 0.5 * told / d + toln
    tolF = tolFrel * Fs
    tolF[Fs == 0] = 0.0
    skipF = np.zeros(len(V), bool)
    if tol_force is not None:
        tolF, skipF = tol_force(toln, tolx, tolV, told, flagged)
    hitF = hit & ~skipF
    _check("F_pair", np.abs(go[hitF, 8:11] - ro[hitF, 8:11]).max(axis=1, initial=0), tolF[hitF], out)
    zero = clean & (V == 0)
    assert np.all(go[zero] == 0.0), "pairs with no overlap must be exactly zero"
    # per-particle sums: tolerance = sum of the pair tolerances touching it
    # rows n .. n + walls - 1 stand for the walls (partner indices j >= n; no sums)
    nrow = st.n + len(getattr(st, "walls", ()))
    touched_flag = np.zeros(nrow, bool)
    touched_flag[r.pair_ij[flagged | skipF].ravel()] = True
    sF = np.zeros(nrow)
    tF = np.zeros(nrow)
    for col in (0, 1):
        np.add.at(sF, r.pair_ij[:, col], Fs)
        np.add.at(tF, r.pair_ij[:, col], tolF)
    touched_flag, sF, tF = touched_flag[:st.n], sF[:st.n], tF[:st.n]
    ok = ~touched_flag & ((sF > 0) | (tF > 0))
    _check("F", np.abs(g["force"][ok] - r_force[ok]).max(axis=1, initial=0), tF[ok] + 1e-12 * sF[ok], out)
    pos_w = np.concatenate([st.pos, np.zeros((nrow - st.n, 3))])   # a wall sits at the origin
    XA = pos_w[r.pair_ij[:, 0]]
    XB = pos_w[r.pair_ij[:, 1]] - r.pair_shift * st.box
    armA = np.linalg.norm(ro[:, 1:4] - XA, axis=1)
    armB = np.linalg.norm(ro[:, 1:4] - XB, axis=1)
    tT = np.zeros(nrow)
    np.add.at(tT, r.pair_ij[:, 0], tolF * armA + Fs * tolx)
    np.add.at(tT, r.pair_ij[:, 1], tolF * armB + Fs * tolx)
    sT = np.zeros(nrow)
    np.add.at(sT, r.pair_ij[:, 0], Fs * armA)
    np.add.at(sT, r.pair_ij[:, 1], Fs * armB)
    tT, sT = tT[:st.n], sT[:st.n]
    _check("T", np.abs(g["torque"][ok] - r_torque[ok]).max(axis=1, initial=0), tT[ok] + 1e-12 * sT[ok], out)
    none = ~ok & ~touched_flag
    assert np.all(g["force"][none] == 0.0) and np.all(g["torque"][none] == 0.0)
    rel = output_errors(st, g, r, clean & ~skipF, ro, r_force, r_torque)
    return Report(r.n_pairs, r.cells, int(flagged.sum()), int(flips.sum()), out, rel)
