"""Pins of the FP64 oracle against what the paper and geometry fix.

Each test states the passage or closed form it pins.  None re-types the
oracle's own formula; they check closed forms, invariants, special cases and a
brute-force whole-lattice scan, chosen so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import (IDENTITY, cap_centroid_offset, cube_planes, lens_volume, quat_axis_angle,
                           state)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "force_law.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


# ---------------------------------------------------------------- rotations

def test_rotation_known_quaternions():
    assert np.array_equal(oracle.rotation([1, 0, 0, 0]), np.eye(3))
    # 90 degrees about z maps x to y and y to -x
    R = oracle.rotation(quat_axis_angle([0, 0, 1], np.pi / 2))
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    assert np.allclose(R @ [0, 1, 0], [-1, 0, 0], atol=1e-15)
    # 120 degrees about (1,1,1) permutes the axes x -> y -> z
    R = oracle.rotation(quat_axis_angle([1, 1, 1], 2 * np.pi / 3))
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_rotation_orthonormal_and_scale_free():
    rng = np.random.default_rng(0)
    for q in rng.normal(size=(20, 4)):
        R = oracle.rotation(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.allclose(oracle.rotation(3.7 * q), R, atol=1e-15)


# ------------------------------------------------------------ shape prep

def test_polytope_vertices_cube_and_octahedron():
    v = oracle.polytope_vertices(cube_planes([1.0, 2.0, 3.0]))
    uniq = np.unique(np.round(v, 12), axis=0)
    assert len(uniq) == 8
    assert np.allclose(np.sort(np.abs(uniq), axis=0), np.tile([1.0, 2.0, 3.0], (8, 1)))
    v = oracle.polytope_vertices(cube_planes(1.0), delta=0.5)
    assert np.allclose(np.unique(np.abs(np.round(v, 12))), [1.5])
    s = 1 / np.sqrt(3)
    octa = np.array([[a * s, b * s, c * s, s * 2.0] for a in (1, -1) for b in (1, -1) for c in (1, -1)])
    v = np.unique(np.round(oracle.polytope_vertices(octa), 12), axis=0)
    assert len(v) == 6 and np.allclose(np.sort(np.abs(v).max(axis=1)), 2.0)


def test_unbounded_polytope_rejected():
    half = cube_planes(1.0)[[0, 2, 3, 4, 5]]   # no -x face: unbounded
    with pytest.raises(oracle.OracleError):
        oracle.polytope_vertices(half)


# ------------------------------------------------------------- force law

def test_normal_force_worked_value():
    """Eq. (contact_force_normal), prefactor 4/(3 pi) as printed."""
    g = golden()
    F = oracle.normal_force(1.0, 11 * np.pi / 3, 1.0)
    assert F == pytest.approx(g["normal_force_Estar1_V11pi3_d1"], rel=1e-14)
    # sqrt(V d) scaling and linearity in E*
    assert oracle.normal_force(2.0, 4 * 11 * np.pi / 3, 1.0) == pytest.approx(4 * F, rel=1e-14)
    assert oracle.normal_force(1.0, 0.0, 1.0) == 0.0
    # (1 + c ddot) factor, clamped at zero (no adhesion)
    assert oracle.normal_force(1.0, 11 * np.pi / 3, 1.0, 0.5, 1.0) == pytest.approx(1.5 * F, rel=1e-14)
    assert oracle.normal_force(1.0, 11 * np.pi / 3, 1.0, 1.0, -3.0) == 0.0


def test_effective_modulus_special_cases():
    """Sec. 2.3: E* = ((1 - nu_A^2)/E_A + (1 - nu_B^2)/E_B)^-1."""
    assert oracle.effective_modulus(10.0, 0.0, 10.0, 0.0) == pytest.approx(5.0, rel=1e-15)
    assert oracle.effective_modulus(10.0, 0.5, 10.0, 0.5) == pytest.approx(10.0 / 1.5, rel=1e-15)
    # a rigid partner leaves E/(1 - nu^2)
    assert oracle.effective_modulus(3.0, 0.6, 1e300, 0.0) == pytest.approx(3.0 / 0.64, rel=1e-12)
    assert oracle.effective_modulus(3.0, 0.2, 7.0, 0.4) == oracle.effective_modulus(7.0, 0.4, 3.0, 0.2)


def test_damping_factor():
    """Eq. (damping_factor) (Carvalho-Martins): worked values, e = 1 is elastic, u0 <= 0 gives 0."""
    g = golden()
    assert oracle.damping_factor(0.926, 1.0) == pytest.approx(g["damping_c_e0.926_u0_1"], rel=1e-14)
    assert oracle.damping_factor(0.0, 1.0) == pytest.approx(g["damping_c_e0_u0_1"], rel=1e-15)
    assert oracle.damping_factor(1.0, 2.0) == 0.0
    assert oracle.damping_factor(0.5, 0.0) == 0.0 and oracle.damping_factor(0.5, -1.0) == 0.0
    assert oracle.damping_factor(0.5, 4.0) == pytest.approx(oracle.damping_factor(0.5, 1.0) / 4, rel=1e-15)


# ---------------------------------------------------------- sphere lenses

def _sphere_pair(r1, r2, c1, c2, dx=1.0, L=64.0, **kw):
    return state([0, 0], [[r1, 0, 0], [r2, 0, 0]], [c1, c2], n=int(round(L / dx)), dx=dx, **kw)


def test_lens_volume_converges_linearly():
    """Overlap volume -> analytic lens volume under refinement, EOC >= 1
    (the paper reports linear convergence of the method, Sec. 5.2)."""
    r1, r2, D = 7.5, 6.0, 10.0
    Vex = lens_volume(r1, r2, D)
    rng = np.random.default_rng(0)
    dxs = [1.0, 0.5, 0.25]
    err = []
    for dx in dxs:
        e = []
        for _ in range(6):
            c = np.array([32.0, 32.0, 32.0]) + rng.random(3)
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            r = oracle.contact_step(_sphere_pair(r1, r2, c, c + D * u, dx=dx))
            assert r.n_pairs == 1
            e.append(abs(r.pair_out[0, 0] - Vex) / Vex)
        err.append(np.mean(e))
    eoc = np.polyfit(np.log(dxs), np.log(err), 1)[0]
    assert eoc >= 1.0, (err, eoc)
    assert err[-1] < 2e-3


def test_lens_worked_example_force_and_depth():
    """r = 7.5, D = 14: lens volume 11 pi / 3; centres on a lattice line give
    d = r1 + r2 - D = 1 exactly (Sec. 3.3.1 outputs), |F| -> 1.4405 with E* = 1."""
    g = golden()
    dx = 0.125
    c1 = np.array([20.0, 32.0, 32.0])
    r = oracle.contact_step(_sphere_pair(7.5, 7.5, c1, c1 + [14.0, 0, 0], dx=dx))
    V, d = r.pair_out[0, 0], r.pair_out[0, 7]
    assert V == pytest.approx(g["lens_volume_r7.5_D14"], rel=5e-3)
    assert d == pytest.approx(1.0, abs=1e-12)
    Fmag = np.linalg.norm(r.pair_out[0, 8:11])
    assert Fmag == pytest.approx(g["normal_force_Estar1_V11pi3_d1"] * math.sqrt(V / (11 * math.pi / 3)),
                                 rel=1e-12)
    assert Fmag == pytest.approx(g["normal_force_Estar1_V11pi3_d1"], rel=3e-3)
    # normal exactly along the centre line, pointing from the lower to the higher ID
    assert np.allclose(r.pair_out[0, 4:7], [1, 0, 0], atol=1e-14)


def test_depth_of_a_deep_sphere_pair():
    """Spheres r1 = 6, r2 = 4 with centres 3 apart on a lattice line: on the
    segment between the centres -phi_A - phi_B = r1 + r2 - D = 7, its maximum,
    so d = 7 (one body's depth alone would give 6)."""
    XA = np.array([30.0, 31.0, 29.0])
    st = state([0, 0], [[6, 0, 0], [4, 0, 0]], [XA, XA + [3.0, 0.0, 0.0]])
    r = oracle.contact_step(st)
    assert r.n_pairs == 1 and r.pair_out[0, 7] == pytest.approx(7.0, abs=1e-12)


def test_lens_centroid_and_normal():
    """Contact point -> volume-weighted mean of the two cap centroids on the centre line."""
    r1, r2, D = 7.5, 6.0, 10.0
    h1 = (r2 - r1 + D) * (r2 + r1 - D) / (2 * D)
    h2 = (r1 - r2 + D) * (r1 + r2 - D) / (2 * D)
    v1 = np.pi * h1 * h1 * (3 * r1 - h1) / 3
    v2 = np.pi * h2 * h2 * (3 * r2 - h2) / 3
    x1 = cap_centroid_offset(r1, h1)   # cap of ball 1 faces ball 2
    x2 = D - cap_centroid_offset(r2, h2)
    xc_exact = (v1 * x1 + v2 * x2) / (v1 + v2)
    c1 = np.array([20.0, 32.0, 32.0])
    errs = []
    for dx in (0.5, 0.25):
        r = oracle.contact_step(_sphere_pair(r1, r2, c1, c1 + [0, 0, D], dx=dx))
        xc = r.pair_out[0, 1:4] - c1
        errs.append(abs(xc[2] - xc_exact))
        assert np.allclose(xc[:2], 0, atol=1e-12)
        assert np.allclose(r.pair_out[0, 4:7], [0, 0, 1], atol=1e-14)
    assert errs[1] < errs[0] and errs[1] < 0.02


# ----------------------------------------------------- face-aligned boxes

def test_face_aligned_cuboids_exact_box_volume():
    """Axis-aligned boxes with faces on half-integer node coordinates: the
    lattice volume is the exact product of interval overlaps, the contact point
    the exact centre of the intersection box, d the penetration."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        h = rng.integers(2, 7, size=(2, 3)).astype(float)
        cA = np.array([30.5, 31.5, 29.5])
        pen = float(rng.integers(1, 3))
        lat = rng.integers(-1, 2, size=2).astype(float)
        cB = cA + [h[0, 0] + h[1, 0] - pen, lat[0], lat[1]]
        r = oracle.contact_step(state([1, 1], h, [cA, cB]))
        lo = np.maximum(cA - h[0], cB - h[1])
        hi = np.minimum(cA + h[0], cB + h[1])
        assert r.pair_out[0, 0] == np.prod(hi - lo)
        assert np.array_equal(r.pair_out[0, 1:4], (lo + hi) / 2)
        assert r.pair_out[0, 7] == pen
        # faces on half-integer offsets sit at the edges of the smoothed
        # derivative's support, so the band normal G vanishes and the
        # centre-line fallback applies
        assert np.abs(r.pair_aux[0, :3]).max() == 0.0
        u = (cB - cA) / np.linalg.norm(cB - cA)
        assert np.allclose(r.pair_out[0, 4:7], u, atol=1e-15)


def test_cube_as_polytope_matches_cuboid_bitwise():
    """Sec. 3.3.1 signed distance of a box = max over its 6 face planes."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        h = rng.uniform(3, 6, size=3)
        q = W.random_quaternions(rng, 2)
        cA = np.array([30.0, 30.0, 30.0]) + rng.random(3)
        cB = cA + rng.normal(size=3) * 3 + [8, 0, 0]
        a = oracle.contact_step(state([1, 1], [h, [5, 5, 5]], [cA, cB], q))
        b = oracle.contact_step(state([2, 1], [[0, 0, 0], [5, 5, 5]], [cA, cB], q,
                                      planes=[cube_planes(h), None]))
        assert np.array_equal(a.pair_ij, b.pair_ij)
        assert np.array_equal(a.pair_out, b.pair_out)


# --------------------------------------------------------------- invariants

def test_separated_candidates_give_zero():
    """Boxes overlap but shapes do not: V = 0 and F = 0 exactly (sharp)."""
    c = np.array([30.0, 30.0, 30.0])
    r = oracle.contact_step(_sphere_pair(6.0, 6.0, c, c + [9.0, 9.0, 0.0]))
    assert r.n_pairs == 1
    assert np.all(r.pair_out[0] == 0.0)
    assert np.all(r.force == 0.0)


def test_swap_labels_flips_normal_and_force():
    rng = np.random.default_rng(5)
    q = W.random_quaternions(rng, 2)
    pA, pB = np.array([30.2, 31.1, 29.7]), np.array([39.0, 33.0, 31.0])
    a = oracle.contact_step(state([1, 0], [[6, 6, 6], [7.5, 0, 0]], [pA, pB], q))
    b = oracle.contact_step(state([0, 1], [[7.5, 0, 0], [6, 6, 6]], [pB, pA], q[::-1]))
    assert a.pair_out[0, 0] > 0
    assert a.pair_out[0, 0] == b.pair_out[0, 0] and a.pair_out[0, 7] == b.pair_out[0, 7]
    assert np.array_equal(a.pair_out[0, 1:4], b.pair_out[0, 1:4])
    assert np.array_equal(a.pair_out[0, 4:7], -b.pair_out[0, 4:7])
    assert np.array_equal(a.pair_out[0, 8:11], -b.pair_out[0, 8:11])
    assert np.array_equal(a.force, b.force[::-1])


def test_integer_translation_and_lattice_rotation():
    st = W.mixed_grid_27()
    base = oracle.contact_step(st)
    t = np.array([3.0, -5.0, 7.0])
    moved = oracle.contact_step(st.with_poses(np.mod(st.pos + t, st.box), st.quat))
    assert np.array_equal(base.pair_ij, moved.pair_ij)
    assert np.array_equal(base.pair_out[:, 0], moved.pair_out[:, 0])
    for k in (4, 5, 6, 7, 8, 9, 10):
        assert np.allclose(base.pair_out[:, k], moved.pair_out[:, k], rtol=1e-9, atol=1e-9)
    # 90 degrees about z through the origin node: (x, y, z) -> (-y, x, z)
    Rz = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1.0]])
    pos = np.mod(st.pos @ Rz.T, st.box)
    quat = W.quat_mul(np.tile(quat_axis_angle([0, 0, 1], np.pi / 2), (st.n, 1)), st.quat)
    rot = oracle.contact_step(st.with_poses(pos, quat))
    assert np.array_equal(base.pair_ij, rot.pair_ij)
    assert np.array_equal(base.pair_out[:, 0], rot.pair_out[:, 0])
    assert np.allclose(base.pair_out[:, 4:7] @ Rz.T, rot.pair_out[:, 4:7], atol=1e-9)
    assert np.allclose(base.force @ Rz.T, rot.force, rtol=1e-9, atol=1e-9)


def test_momentum_balance():
    """Equal and opposite forces per pair; sum_p F_p = 0 and sum_p (T_p + X_p x F_p) = 0
    in the unwrapped frame of each pair."""
    st = W.mixed_settling(n=300, L=120)
    r = oracle.contact_step(st)
    scale = np.abs(r.pair_out[:, 8:11]).sum()
    assert scale > 0
    assert np.abs(r.force.sum(axis=0)).max() < 1e-12 * scale
    XA = st.pos[r.pair_ij[:, 0]]
    XB = st.pos[r.pair_ij[:, 1]] - r.pair_shift * st.box
    F = r.pair_out[:, 8:11]
    xc = r.pair_out[:, 1:4]
    TA = np.cross(xc - XA, -F)
    TB = np.cross(xc - XB, F)
    L = TA + np.cross(XA, -F) + TB + np.cross(XB, F)
    assert np.abs(L).max() < 1e-10 * max(1.0, np.abs(TA).max())
    # torques in the per-particle sums are exactly the per-pair ones
    T = np.zeros_like(r.torque)
    np.add.at(T, r.pair_ij[:, 0], TA)
    np.add.at(T, r.pair_ij[:, 1], TB)
    assert np.allclose(T, r.torque, rtol=1e-12, atol=1e-9)


def _sdf_sphere_or_box(t, prm, X, R, x):
    if t == 0:
        return np.linalg.norm(x - X, axis=-1) - prm[0]
    y = (x - X) @ R
    return np.max(np.abs(y) - prm, axis=-1)


def test_contact_point_inside_both_shapes():
    """The centroid of a convex node set lies in the convex intersection."""
    st = W.mixed_grid_27()
    r = oracle.contact_step(st)
    R = W.rotation_matrices(st.quat)
    hit = r.pair_out[:, 0] > 0
    assert hit.sum() > 10
    for p in np.nonzero(hit)[0]:
        i, j = r.pair_ij[p]
        XB = st.pos[j] - r.pair_shift[p] * st.box
        xc = r.pair_out[p, 1:4]
        assert _sdf_sphere_or_box(st.shape_type[i], st.shape_param[i], st.pos[i], R[i], xc) <= 1e-9
        assert _sdf_sphere_or_box(st.shape_type[j], st.shape_param[j], XB, R[j], xc) <= 1e-9


# ---------------------------------------------------------- periodic images

def test_periodic_pairs_across_faces_edges_corners():
    """Sec. 3.3.2: a pair straddling a periodic face, edge or corner gives the
    same V, d, n, F as the same pair in the interior; x_c is reported in the
    lower-ID particle's frame (shifted by whole periods)."""
    rng = np.random.default_rng(6)
    q = W.random_quaternions(rng, 2)
    L = 48.0
    pA = np.array([20.3, 21.6, 22.1])
    d = np.array([7.7, 3.1, -2.2])
    ref = oracle.contact_step(state([1, 0], [[6, 6, 6], [7.5, 0, 0]], [pA, pA + d], q, n=48))
    assert ref.pair_out[0, 0] > 0
    for corner in ([1, 0, 0], [1, 1, 0], [1, 1, 1], [0, 1, 1]):
        shift = np.round(np.array([47.0, 46.0, 45.0]) - pA) * corner   # integer node shift
        a, b = np.mod(pA + shift, L), np.mod(pA + d + shift, L)
        for swap in (False, True):
            if swap:
                r = oracle.contact_step(state([0, 1], [[7.5, 0, 0], [6, 6, 6]], [b, a], q[::-1], n=48))
                sgn, ref_xc_origin = -1.0, b
            else:
                r = oracle.contact_step(state([1, 0], [[6, 6, 6], [7.5, 0, 0]], [a, b], q, n=48))
                sgn, ref_xc_origin = 1.0, a
            assert r.n_pairs == 1
            assert r.pair_out[0, 0] == ref.pair_out[0, 0]
            assert r.pair_out[0, 7] == pytest.approx(ref.pair_out[0, 7], abs=1e-12)
            assert np.allclose(sgn * r.pair_out[0, 4:7], ref.pair_out[0, 4:7], atol=1e-12)
            # x_c relative to the lower-ID particle is the same up to whole periods
            rel = r.pair_out[0, 1:4] - ref_xc_origin
            rel_ref = ref.pair_out[0, 1:4] - (pA if not swap else pA + d)
            assert np.allclose(rel, rel_ref, atol=1e-9)


def test_brute_force_whole_lattice_scan():
    """On a tiny periodic lattice, a scan of every node against all 27 images
    of the partner equals the oracle's box-restricted sums (pins the AABB node
    ranges, the minimum image and the pair box)."""
    rng = np.random.default_rng(7)
    n = 32
    k = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
    hits = 0
    for trial in range(6):
        types = rng.integers(0, 2, size=2)
        prm = np.where(types[:, None] == 0, [[5.5, 0, 0]], [[3.5, 4.0, 4.5]])
        q = W.random_quaternions(rng, 2)
        pA = rng.random(3) * n
        pB = np.mod(pA + rng.normal(size=3) * 3 + [7, 0, 0], n)
        st = state(types, prm, [pA, pB], q, n=n)
        r = oracle.contact_step(st)
        R = W.rotation_matrices(q)
        # brute force: node sums over the whole periodic lattice, A in its own
        # image nearest each node, B in every image
        inA = _sdf_sphere_or_box(types[0], prm[0], pA, R[0], k) <= 0
        total = 0
        for s in np.stack(np.meshgrid(*[[-1, 0, 1]] * 3, indexing="ij"), -1).reshape(-1, 3):
            for sa in np.stack(np.meshgrid(*[[-1, 0, 1]] * 3, indexing="ij"), -1).reshape(-1, 3):
                a = _sdf_sphere_or_box(types[0], prm[0], pA + sa * n, R[0], k) <= 0
                b = _sdf_sphere_or_box(types[1], prm[1], pB + s * n, R[1], k) <= 0
                total += int(np.sum(a & b))
        V = r.pair_out[0, 0] if r.n_pairs else 0.0
        assert V == total, (trial, V, total)
        hits += V > 0
        del inA
    assert hits >= 4


# ------------------------------------------------------------ smoothed mode

def test_smoothed_indicator_limits():
    """H_w -> sharp H as w -> 0; smoothed V is continuous in the pose while the
    sharp V jumps by whole cells."""
    st = W.mixed_grid_27()
    sharp = oracle.contact_step(st)
    thin = st.with_poses(st.pos, st.quat)
    thin.indicator, thin.smooth_width = 1, 1e-4
    sm = oracle.contact_step(thin)
    both = np.isin(sm.pair_ij.view([("a", np.int32), ("b", np.int32)]),
                   sharp.pair_ij.view([("a", np.int32), ("b", np.int32)])).ravel()
    assert np.allclose(sm.pair_out[both, 0], sharp.pair_out[:, 0], atol=1e-9)
    c = np.array([30.0, 30.0, 30.0])
    vs = []
    for e in (0.0, 1e-7, 2e-7):
        a = oracle.contact_step(_sphere_pair(7.5, 6.0, c, c + [10.0 + e, 0.3, 0.1], indicator=1))
        vs.append(a.pair_out[0, 0])
    assert abs(vs[1] - vs[0]) < 1e-5 and abs(vs[2] - vs[1]) < 1e-5 and vs[0] != vs[1]


def test_smoothed_band_weights_of_mirrored_faces_sum_to_sharp():
    """S(t) + S(1 - t) = 1: a box whose only face inside the band sits at
    offset delta or 1 - delta from a node row (its other faces on half-integer
    nodes, where w = 1 leaves no node in the band), inside a large box, has
    smoothed volumes that add up to the two sharp volumes exactly."""
    def vol(delta, indicator):
        lo_x, hi_x = 20.5, 30.0 + delta
        A = [(hi_x - lo_x) / 2, 4.0, 4.0]
        XA = [(hi_x + lo_x) / 2, 30.5, 30.5]
        st = state([1, 1], [A, [8.0, 8.0, 8.0]], [XA, [25.5, 30.5, 30.5]], indicator=indicator, w=1.0)
        return oracle.contact_step(st).pair_out[0, 0]
    for delta in (0.2, 0.35):
        smooth = vol(delta, 1) + vol(1 - delta, 1)
        sharp = vol(delta, 0) + vol(1 - delta, 0)
        assert smooth == pytest.approx(sharp, rel=1e-13), (delta, smooth, sharp)
        assert vol(delta, 1) != vol(delta, 0)   # the face's band node is weighted


# ---------------------------------------------------------------- gradient

def _fd_check(st, gf, gt, h_pos=1e-4, h_q=1e-4):
    gp, gq = oracle.gradient(st, gf, gt)

    def loss(pos, quat):
        r = oracle.contact_step(st, pos=pos, quat=quat)
        return float(np.sum(gf * r.force) + np.sum(gt * r.torque))

    fd_p = np.zeros_like(gp)
    fd_q = np.zeros_like(gq)
    for p in range(st.n):
        for k in range(3):
            a, b = st.pos.copy(), st.pos.copy()
            a[p, k] += h_pos
            b[p, k] -= h_pos
            fd_p[p, k] = (loss(a, st.quat) - loss(b, st.quat)) / (2 * h_pos)
        for k in range(4):
            a, b = st.quat.copy(), st.quat.copy()
            a[p, k] += h_q
            b[p, k] -= h_q
            fd_q[p, k] = (loss(st.pos, a) - loss(st.pos, b)) / (2 * h_q)
    return gp, gq, fd_p, fd_q


def test_dual_gradient_matches_central_differences():
    """The oracle's forward-mode gradient equals central differences of the
    oracle's own forward map (smoothed indicator, w = 1 cell)."""
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width = 1, 1.0
    gf, gt = W.loss_weights(st.n)
    gp, gq, fp, fq = _fd_check(st, gf, gt)
    g = np.concatenate([gp.ravel(), gq.ravel()])
    f = np.concatenate([fp.ravel(), fq.ravel()])
    scale = np.abs(g).max()
    assert scale > 0
    err = np.abs(g - f) / scale
    # kinks of the max-of-planes SDF and of the depth argmax can fall inside
    # a +-h stencil; allow at most 2 % of the components to see one
    assert np.mean(err < 1e-4) >= 0.98, np.sort(err)[-10:]
    assert np.median(err) < 1e-6
    # the gradient w.r.t. the raw quaternion is orthogonal to the quaternion
    assert np.abs(np.einsum("ij,ij->i", gq, st.quat)).max() < 1e-9 * scale


# ---------------------------------------------------------------- errors

def test_invalid_inputs_rejected():
    c = np.array([30.0, 30.0, 30.0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.contact_step(_sphere_pair(6, 6, c, [70.0, 30.0, 30.0]))   # outside [0, L)
    assert e.value.code == 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.contact_step(_sphere_pair(6, 6, c, c + 5, L=24.0))         # two images could overlap
    assert e.value.code == 5
    st = _sphere_pair(6, 6, c, c + 5)
    st.quat[0] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.contact_step(st)
