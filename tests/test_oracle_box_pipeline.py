"""Pins of the oracle's box pipeline (Sec. 3.3.1 as restated: rough on-lattice
detection with the half-cell-diagonal threshold, correction of the box by
lines cast inward from its faces, N_c^3 sample points over the corrected box).

Checked against geometry: for two face-aligned boxes the corrected box is the
exact overlap box and the sampled volume, contact point, depth and normal are
exact; for two spheres the corrected box lies inside the lens's bounding box
and tends to it, and the volume to the lens volume; the rough box equals a
brute-force node scan; a pair within the rough threshold but apart keeps its
rough box and gets zero outputs; a cube on a floor gives the exact slab.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import lens_volume, state


def boxed(st, nc=8):
    st.box_mode, st.contact_resolution = 1, nc
    return st


def test_face_aligned_boxes_exact():
    """A (half extents 4) and B (4, 10, 10) overlapping by 0.8 along x, B
    centred on A across: the corrected box is A's cross-section times the
    x-overlap, V its volume, x_c its centre, d = 0.8, n = +x."""
    XA = np.array([30.3, 31.7, 29.2])
    XB = XA + [7.2, 0.0, 0.0]
    st = boxed(state([1, 1], [[4, 4, 4], [4, 10, 10]], [XA, XB], n=80))
    rough, box, flags = oracle.box_pipeline(st)
    lo = [XB[0] - 4, XA[1] - 4, XA[2] - 4]
    hi = [XA[0] + 4, XA[1] + 4, XA[2] + 4]
    assert np.allclose(box[0, :3], lo, atol=1e-12) and np.allclose(box[0, 3:], hi, atol=1e-12)
    r = oracle.contact_step(st)
    o = r.pair_out[0]
    assert o[0] == pytest.approx(0.8 * 8 * 8, rel=1e-12)
    assert np.allclose(o[1:4], (np.array(lo) + hi) / 2, atol=1e-11)
    assert o[7] == pytest.approx(0.8, abs=1e-12)
    assert np.allclose(o[4:7], [1, 0, 0], atol=1e-12)


@pytest.mark.parametrize("nc", [8, 16, 32])
def test_sphere_lens_box_inside_and_volume(nc):
    r1, r2, D = 6.0, 5.0, 9.7
    XA = np.array([30.25, 31.5, 29.75])
    XB = XA + [D, 0.0, 0.0]
    st = boxed(state([0, 0], [[r1, 0, 0], [r2, 0, 0]], [XA, XB]), nc)
    rough, box, flags = oracle.box_pipeline(st)
    xp = (D * D + r1 * r1 - r2 * r2) / (2 * D)          # lens plane, from A's centre
    a = math.sqrt(r1 * r1 - xp * xp)                     # lens circle radius
    exact_lo = XA + [D - r2, -a, -a]
    exact_hi = XA + [r1, a, a]
    # inside the lens's bounding box (lines cannot see beyond the lens) ...
    assert np.all(box[0, :3] >= exact_lo - 1e-9) and np.all(box[0, 3:] <= exact_hi + 1e-9)
    # ... and closer to it the finer the lines (the lens apex lies on the centre line)
    spacing = (exact_hi - exact_lo).max() / nc + 2 * math.sqrt(0.75)
    assert np.abs(box[0, [0, 3]] - [exact_lo[0], exact_hi[0]]).max() < 0.05 * spacing
    assert np.abs(box[0, 1:3] - exact_lo[1:]).max() < 2 * spacing ** 2 / a
    V = oracle.contact_step(st).pair_out[0, 0]
    Vx = lens_volume(r1, r2, D)
    assert abs(V - Vx) / Vx < {8: 0.1, 16: 0.05, 32: 0.025}[nc], (V, Vx)


def _sdf_np(kind, prm, X, R, x):
    r = (x - X) @ R
    if kind == 0:
        return np.linalg.norm(x - X, axis=1) - prm[0]
    return np.max(np.abs(r) - prm, axis=1)


def test_rough_box_equals_brute_force_scan():
    rng = np.random.default_rng(9)
    s = math.sqrt(0.75)
    for trial in range(6):
        types = rng.integers(0, 2, size=2)
        prm = np.where(types[:, None] == 0, [[5.5, 0, 0]], [[3.5, 4.0, 4.5]])
        q = W.random_quaternions(rng, 2)
        XA = np.array([30.0, 31.0, 32.0]) + rng.random(3)
        XB = XA + rng.normal(size=3) * 2 + [8.5, 0, 0]
        st = boxed(state(types, prm, [XA, XB], q))
        rough, box, flags = oracle.box_pipeline(st)
        R = W.rotation_matrices(q)
        k = np.stack(np.meshgrid(*[np.arange(16, 52)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
        inside = (_sdf_np(types[0], prm[0], XA, R[0], k) < s) & (_sdf_np(types[1], prm[1], XB, R[1], k) < s)
        if not inside.any():
            continue
        assert rough[0].tolist() == [*k[inside].min(axis=0).astype(int), *k[inside].max(axis=0).astype(int)]


def test_rough_contact_without_overlap_gives_zero():
    """Spheres 0.3 apart: nodes within half a cell diagonal of both exist,
    but no line enters both shapes: the box stays and V = 0."""
    XA = np.array([30.0, 31.0, 32.0])
    st = boxed(state([0, 0], [[5.0, 0, 0], [5.0, 0, 0]], [XA, XA + [10.3, 0, 0]]))
    rough, box, flags = oracle.box_pipeline(st)
    assert rough[0, 3] >= rough[0, 0]
    r = oracle.contact_step(st)
    assert np.all(r.pair_out[0] == 0.0)


def test_cube_on_floor_exact_slab():
    X = np.array([30.3, 31.7, 20.6])
    st = boxed(W.with_walls(state([1], [[4, 4, 4]], [X]), [[0, 0, 1, 17.3]]))
    r = oracle.contact_step(st)
    o = r.pair_out[0]
    assert r.pair_ij[0].tolist() == [0, 1]
    assert o[0] == pytest.approx(64 * (17.3 - 16.6), rel=1e-12)
    assert np.allclose(o[1:4], [30.3, 31.7, (16.6 + 17.3) / 2], atol=1e-11)
    assert o[7] == pytest.approx(0.7, abs=1e-12)
    assert np.allclose(o[4:7], [0, 0, -1], atol=1e-12)


def test_box_mode_has_no_gradient():
    st = boxed(state([0, 0], [[5.0, 0, 0], [5.0, 0, 0]], [[30.0, 31.0, 32.0], [39.0, 31.0, 32.0]]))
    st.indicator = 1
    with pytest.raises(oracle.OracleError):
        oracle.gradient(st, np.zeros((2, 3)), np.zeros((2, 3)))


# --- warm start of the box correction (Sec. 4.3.3, with the contact history) ---

LAW_H = oracle.ContactLaw(restitution=1.0, history=True)


def lens_aabb(XA, r1, XB, r2):
    """Axis-aligned bounding box of the intersection of two balls: per axis and
    side, the ball's extreme point if it lies in the other ball, else the
    extreme of the intersection circle."""
    d = XB - XA
    D = np.linalg.norm(d)
    u = d / D
    xp = (D * D + r1 * r1 - r2 * r2) / (2 * D)
    a = math.sqrt(r1 * r1 - xp * xp)
    c0 = XA + xp * u
    lo, hi = np.zeros(3), np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        for sgn in (1.0, -1.0):
            cand = [c0[k] + sgn * a * math.sqrt(max(0.0, 1.0 - u[k] ** 2))]
            if np.linalg.norm(XA + sgn * r1 * e - XB) <= r2:
                cand.append(XA[k] + sgn * r1)
            if np.linalg.norm(XB + sgn * r2 * e - XA) <= r1:
                cand.append(XB[k] + sgn * r2)
            if sgn > 0:
                hi[k] = max(cand)
            else:
                lo[k] = min(cand)
    return lo, hi


def warm_steps(st, k):
    """k history steps at a fixed pose; returns the first (cold) and the last result."""
    r0 = oracle.contact_step_ext(st, LAW_H)
    r = r0
    for _ in range(k):
        r = oracle.contact_step_ext(st, LAW_H, hist=(r.hist_ij, r.hist_c, r.hist_box))
    return r0, r


@pytest.mark.parametrize("nc", [4, 8])
def test_warm_start_tightens_the_box_inside_the_lens(nc):
    """Random lens orientations and sub-cell offsets: the warm-started box stays
    inside the exact lens box (lines cannot see past the overlap), and on
    average its faces lie much closer to it than the cold box's."""
    rng = np.random.default_rng(0)
    r1, r2, D = 7.5, 6.0, 12.6
    gap_cold, gap_warm = [], []
    for _ in range(16):
        XA = np.array([30.0, 30.0, 30.0]) + rng.random(3)
        u = rng.normal(size=3)
        XB = XA + D * u / np.linalg.norm(u)
        st = boxed(state([0, 0], [[r1, 0, 0], [r2, 0, 0]], [XA, XB]), nc)
        lo, hi = lens_aabb(XA, r1, XB, r2)
        r0, r = warm_steps(st, 3)
        bc, bw = r0.hist_box[0] + np.tile(XA, 2), r.hist_box[0] + np.tile(XA, 2)
        for b in (bc, bw):
            assert np.all(b[:3] >= lo - 1e-9) and np.all(b[3:] <= hi + 1e-9)
        gap_cold.append(np.sum(bc[:3] - lo) + np.sum(hi - bc[3:]))
        gap_warm.append(np.sum(bw[:3] - lo) + np.sum(hi - bw[3:]))
    print(nc, "mean face gap cold", np.mean(gap_cold), "warm", np.mean(gap_warm))
    assert np.mean(gap_warm) < 0.8 * np.mean(gap_cold)


def _lens_state(nc=8):
    XA = np.array([30.25, 31.5, 29.75])
    return boxed(state([0, 0], [[6.0, 0, 0], [5.0, 0, 0]], [XA, XA + [9.5, 1.25, -0.5]]), nc), XA


def test_stored_box_bounds_the_correction():
    """A stored box is taken relative to X_i and widened by sqrt(0.75) dx: the
    corrected box lies inside it; a stored box apart from B0 on every axis
    leaves the cold result unchanged."""
    st, XA = _lens_state()
    r0 = oracle.contact_step_ext(st, LAW_H)
    lo, hi = lens_aabb(XA, 6.0, st.pos[1], 5.0)
    c = 0.5 * (lo + hi)
    rel = np.concatenate([c - 0.3, c + 0.3]) - np.tile(XA, 2)
    r = oracle.contact_step_ext(st, LAW_H, hist=(r0.hist_ij, r0.hist_c, rel[None]))
    s = math.sqrt(0.75)
    b = r.hist_box[0] + np.tile(XA, 2)
    assert np.all(b[:3] >= c - 0.3 - s - 1e-12) and np.all(b[3:] <= c + 0.3 + s + 1e-12)
    # across the lens (which reaches far past it) the stored box is widened by s
    assert np.all(b[1:3] <= c[1:3] - 0.3 - 0.5 * s) and np.all(b[4:6] >= c[1:3] + 0.3 + 0.5 * s)
    cold = r0.hist_box[0] + np.tile(XA, 2)
    assert np.all(b[1:3] > cold[1:3]) and np.all(b[4:6] < cold[4:6])   # cut across the lens (y, z)
    far = rel + 40.0
    rf = oracle.contact_step_ext(st, LAW_H, hist=(r0.hist_ij, r0.hist_c, far[None]))
    assert np.array_equal(rf.pair_out, r0.pair_out) and np.array_equal(rf.hist_box, r0.hist_box)


@pytest.mark.parametrize("offset, t, who", [(0.6875, 33.0, 0), (0.1875, 24.0, 1)])
def test_warm_start_follows_particle_i_across_the_periodic_boundary(offset, t, who):
    """Two steps (both spheres moved by 1/8 along x in between) of the lens and
    of the same lens translated by t nodes, where particle i (who = 0) or its
    partner j (who = 1, so the pair's image changes) crosses the boundary at
    the second step: the same outputs and stored boxes (to rounding), and the
    second step differs from a cold one."""
    runs = []
    for shift in (0.0, t):
        st, XA = _lens_state()
        pos1 = st.pos + [shift + offset, 0.0, 0.0]
        pos2 = pos1 + [0.125, 0.0, 0.0]
        L = st.n_cells[0] * st.dx
        pos1[:, 0] = np.mod(pos1[:, 0], L)
        pos2[:, 0] = np.mod(pos2[:, 0], L)
        r1 = oracle.contact_step_ext(st, LAW_H, pos=pos1)
        r2 = oracle.contact_step_ext(st, LAW_H, pos=pos2, hist=(r1.hist_ij, r1.hist_c, r1.hist_box))
        cold = oracle.contact_step_ext(st, LAW_H, pos=pos2)
        runs.append((pos1, pos2, r2, cold))
    (p1a, p2a, ra, ca), (p1b, p2b, rb, cb) = runs
    assert p1b[who, 0] > 63.0 and p2b[who, 0] < 1.0   # the particle wrapped
    assert p1a[:, 0].max() < 63.0 and p2a[:, 0].max() < 63.0
    for k in (0, 4, 5, 6, 7, 8, 9, 10):
        assert ra.pair_out[0, k] == pytest.approx(rb.pair_out[0, k], rel=1e-11, abs=1e-12)
    assert np.allclose(ra.hist_box, rb.hist_box, rtol=0, atol=1e-11)
    assert abs(ra.pair_out[0, 0] - ca.pair_out[0, 0]) > 1e-6 * ca.pair_out[0, 0]


def test_warm_start_keeps_face_aligned_boxes_exact():
    XA = np.array([30.3, 31.7, 29.2])
    st = boxed(state([1, 1], [[4, 4, 4], [4, 10, 10]], [XA, XA + [7.2, 0.0, 0.0]], n=80))
    r0, r = warm_steps(st, 2)
    o = r.pair_out[0]
    assert o[0] == pytest.approx(0.8 * 8 * 8, rel=1e-12) and o[7] == pytest.approx(0.8, abs=1e-12)
    assert np.allclose(r.hist_box, r0.hist_box, atol=1e-12)


def test_box_pipeline_history_keeps_c_and_friction_opposes_sliding():
    """With the history, a contact's c from its first step is kept at the next
    one; with friction, the tangential force on B points along A's sliding."""
    st, XA = _lens_state()
    vel = np.zeros((2, 6))
    vel[0, :3] = [0.05, 0.02, 0.0]   # A approaches B and slides along y
    law = oracle.ContactLaw(restitution=0.5, history=True, friction=True, mu_s=0.5, mu_k=0.3, u_k=0.01)
    r1 = oracle.contact_step_ext(st, law, vel=vel)
    assert r1.pair_c[0] > 0.0
    vel2 = vel.copy()
    vel2[0, :3] *= 3.0
    r2 = oracle.contact_step_ext(st, law, vel=vel2, hist=(r1.hist_ij, r1.hist_c, r1.hist_box))
    assert r2.pair_c[0] == r1.pair_c[0]
    n = r2.pair_out[0, 4:7]
    Ft = r2.pair_out[0, 8:11] - np.dot(r2.pair_out[0, 8:11], n) * n
    ut = vel2[0, :3] - np.dot(vel2[0, :3], n) * n
    assert np.dot(Ft, ut) > 0.99 * np.linalg.norm(Ft) * np.linalg.norm(ut)
