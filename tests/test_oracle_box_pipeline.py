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
