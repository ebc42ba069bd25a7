"""Pins of the oracle's per-pair diagnostics, the numbers that decide which
pairs the GPU parity checks assert and how loosely.

The diagnostics are not outputs of the method (Sec. 3.3.1 defines none of
them); they measure how close the FP64 result sits to a decision that a
1e-5-cell perturbation of the signed distances could change:
  * n_band: nodes whose sharp overlap classification flips within +-eps;
  * n_gtie: nodes with a band term of the normal whose active face (or, in
    sharp mode, the partner's classification) is within eps of a tie;
  * d_gap: the gap between the deepest and the second deepest overlap node;
  * v_sens, m_sens, g_sens: the first-order change of V, of the moments and
    of G when every distance moves by eps;
  * n_rough_band (box pipeline): nodes within eps of the rough threshold
    sqrt(0.75) dx; n_face_tie: box faces whose two nearest lines are within
    1e-4 dx without being equal.
Each is checked on a hand-built configuration whose value follows in closed
form from the geometry (face-aligned cubes with faces on node planes or half
way between them, spheres about a lattice line), with a nearby configuration
that moves the value in a known way.
"""
import math

import numpy as np
import pytest

import oracle
from tests.helpers import quat_axis_angle, state

EPS = oracle.BAND_EPS
S075 = math.sqrt(0.75)


def aux_of(st):
    r = oracle.contact_step(st)
    assert r.n_pairs == 1
    a = r.pair_aux[0]
    return dict(G=a[0:3], cells=a[3], n_band=a[4], n_gtie=a[5], d_gap=a[6], v_sens=a[8], m_sens=a[9],
                g_sens=a[10], V=r.pair_out[0, 0], d=r.pair_out[0, 7])


def test_band_count_face_on_a_node_plane():
    """Cube A (half extent 3) about (10, 10, 10) has its +x, +y and +z faces
    on the node planes 13; cube B about (15.5, 10.25, 10.25) covers the 6 x 6
    nodes x = 13, y, z = 8..13 of A's +x face, each with phi_A = 0 exactly and
    phi_B <= -0.25: all 36 are band nodes, and all count in the sharp volume.
    Moving A by +2e-5 along every axis puts them 2e-5 inside: none is in the
    band, the volume stays 36."""
    a = aux_of(state([1, 1], [[3, 3, 3], [3, 3, 3]], [[10, 10, 10], [15.5, 10.25, 10.25]], n=40))
    assert a["n_band"] == 36 and a["V"] == 36
    s = 2e-5
    a = aux_of(state([1, 1], [[3, 3, 3], [3, 3, 3]], [[10 + s, 10 + s, 10 + s], [15.5, 10.25, 10.25]], n=40))
    assert a["n_band"] == 0 and a["V"] == 36


def test_band_count_nodes_just_outside_a_sphere():
    """Sphere A about (10, 10, 10) with radius sqrt(10): the four nodes
    (13, 10 +- 1, 10), (13, 10, 10 +- 1) lie on its surface and deep inside
    cube B (about (15.5, 10.5, 10.5)): four band nodes, counted in V with
    (13, 10, 10).  Radius sqrt(10) - 2e-5 puts them 2e-5 outside, beyond eps:
    no band node, V = 1.  Radius sqrt(10) + 2e-5: 2e-5 inside, V = 5."""
    r0 = math.sqrt(10.0)
    for dr, band, V in ((0.0, 4, 5), (-2e-5, 0, 1), (2e-5, 0, 5)):
        a = aux_of(state([0, 1], [[r0 + dr, 0, 0], [3, 3, 3]], [[10, 10, 10], [15.5, 10.5, 10.5]], n=40))
        assert (a["n_band"], a["V"]) == (band, V), (dr, a)


def test_face_tie_count_on_a_cube_edge():
    """Cube A about (10, 10, 10) (half extent 3), cuboid B about (15.5, 15.5,
    10) with half extents (3, 3, 2.5): B holds A's edge nodes (13, 13, z),
    z = 8..12, where |y_x| = |y_y| = 3 (the +x and +y faces tie, phi_A = 0,
    the normal's band term is on) and B's own distances are -0.5 (no band
    term, no tie): five face ties.  Moving A by 0.3 along y leaves phi_A = 0
    on those nodes but opens a gap of 0.3 between the two faces: no tie."""
    a = aux_of(state([1, 1], [[3, 3, 3], [3, 3, 2.5]], [[10, 10, 10], [15.5, 15.5, 10]], n=40))
    assert a["n_gtie"] == 5 and a["V"] == 5
    a = aux_of(state([1, 1], [[3, 3, 3], [3, 3, 2.5]], [[10, 10.3, 10], [15.5, 15.5, 10]], n=40))
    assert a["n_gtie"] == 0 and a["V"] == 5


def test_depth_gap_closed_form_and_symmetric_tie():
    """Spheres of radii 3.2 and 3 about (10, 10, 10) and (15.5, 10, 10): the
    overlap nodes are (13, 10, 10), at depth (3.2 - 3) + (3 - 2.5) = 0.7, and
    its four neighbours across the centre line, at depth (3.2 - sqrt(10)) +
    (3 - sqrt(7.25)): the gap is sqrt(10) + sqrt(7.25) - 5.5.  Two cubes
    overlapping in a slab one node thick have equal depth at all 36 nodes:
    gap 0."""
    a = aux_of(state([0, 0], [[3.2, 0, 0], [3, 0, 0]], [[10, 10, 10], [15.5, 10, 10]], n=40))
    assert a["V"] == 5
    assert a["d"] == pytest.approx(0.7, abs=1e-12)
    assert a["d_gap"] == pytest.approx(math.sqrt(10) + math.sqrt(7.25) - 5.5, abs=1e-12)
    a = aux_of(state([1, 1], [[3, 3, 3], [3, 3, 3]], [[10.2, 10.5, 10.5], [15.9, 10.5, 10.5]], n=40))
    assert a["V"] == 36 and a["d"] == pytest.approx(0.3, abs=1e-12)
    assert a["d_gap"] == 0.0


# The smoothed slab: cubes A about (10.2, 10.5, 10.5) and B about (15.7, 10.5,
# 10.5), both half extent 3, so their y and z faces lie half way between node
# planes (every node there has |phi| >= 1/2: no band term) and only the nodes
# x = 13, y, z = 8..13 see both x faces inside the band: phi_A = -0.2 and
# phi_B = -0.3, i.e. t_A = 0.7 and t_B = 0.8 with t = 1/2 - phi (w = 1).
T_A, T_B = 0.7, 0.8
H_A, H_B = T_A * T_A * (3 - 2 * T_A), T_B * T_B * (3 - 2 * T_B)     # smoothstep
HP_A, HP_B = 6 * T_A * (1 - T_A), 6 * T_B * (1 - T_B)                # |dH/dphi|
DHP_A, DHP_B = 6 * abs(1 - 2 * T_A), 6 * abs(1 - 2 * T_B)            # |d^2H/dphi^2|
SLAB = ([1, 1], [[3, 3, 3], [3, 3, 3]], [[10.2, 10.5, 10.5], [15.7, 10.5, 10.5]])


def test_sensitivities_of_a_smoothed_slab():
    """V = 36 H_A H_B; G = 1/2 sum(-H_A' grad phi_A H_B + H_A H_B' grad phi_B)
    with grad phi_A = +x and grad phi_B = -x; a shift eps of every phi moves W
    by (|H_A'| H_B + H_A |H_B'|) eps at each node, so v_sens is 36 times that;
    m_sens weights it by the node's distance from the box origin (13, 7, 7)
    (offsets (0, i, j), i, j = 1..6); g_sens bounds the change of each band
    term, 1/2 (|H_A''| H_B + 2 |H_A'| |H_B'| + H_A |H_B''|) eps per node."""
    a = aux_of(state(*SLAB, n=40, indicator=1))
    dw = HP_A * H_B + H_A * HP_B
    assert a["V"] == pytest.approx(36 * H_A * H_B, rel=1e-12)
    assert np.allclose(a["G"], [18 * (HP_A * H_B + H_A * HP_B), 0, 0], rtol=1e-12, atol=1e-12)
    assert a["v_sens"] == pytest.approx(36 * dw * EPS, rel=1e-9)
    radii = sum(math.hypot(i, j) for i in range(1, 7) for j in range(1, 7))
    assert a["m_sens"] == pytest.approx(dw * EPS * radii, rel=1e-9)
    assert a["g_sens"] == pytest.approx(18 * (DHP_A * H_B + 2 * HP_A * HP_B + H_A * DHP_B) * EPS, rel=1e-9)


def test_sensitivities_of_a_sharp_slab():
    """The same slab with the sharp indicator: V = 36 (H = 1 on both sides),
    the normal's band terms use the smoothed derivative with H = 1, so
    G = 18 (|H_A'| + |H_B'|) along +x and g_sens = 18 (|H_A''| + |H_B''|) eps;
    v_sens and m_sens are not defined for the step indicator (zero), and no
    node lies within eps of flipping."""
    a = aux_of(state(*SLAB, n=40, indicator=0))
    assert a["V"] == 36 and a["n_band"] == 0
    assert np.allclose(a["G"], [18 * (HP_A + HP_B), 0, 0], rtol=1e-12, atol=1e-12)
    assert a["v_sens"] == 0.0 and a["m_sens"] == 0.0
    assert a["g_sens"] == pytest.approx(18 * (DHP_A + DHP_B) * EPS, rel=1e-9)


def boxed(st, nc=8):
    st.box_mode, st.contact_resolution = 1, nc
    return st


def test_rough_band_nodes_at_the_half_diagonal():
    """Cube A about (10 - sqrt(0.75), 10.5, 10.5) puts its +x face
    sqrt(0.75) below the node plane 13, so the 8 x 8 nodes x = 13, y, z =
    7..14 lie exactly at the rough threshold from A (their y, z distances are
    at most 1/2) while cube B about (15, 10.5, 10.5) holds them at phi_B <= 1/2:
    64 rough-band nodes.  Moving A by -2e-5 or +2e-5 along x puts them beyond
    eps on either side: none, and the rough box loses or keeps x = 13."""
    for dx, band, hi_x in ((0.0, 64, None), (-2e-5, 0, 12), (2e-5, 0, 13)):
        st = boxed(state([1, 1], [[3, 3, 3], [3, 3, 3]], [[10 - S075 + dx, 10.5, 10.5], [15, 10.5, 10.5]], n=40))
        rough, _, flags = oracle.box_pipeline(st)
        assert flags[0, 0] == band, (dx, flags)
        assert list(rough[0, [0, 1, 2, 4, 5]]) == [12, 7, 7, 14, 14]
        if hi_x is not None:
            assert rough[0, 3] == hi_x


def test_rough_band_nodes_around_a_sphere():
    """Sphere A about (10, 10, 10) with radius sqrt(10) - sqrt(0.75): the
    nodes at distance sqrt(10) from its centre lie exactly at the rough
    threshold.  Cube B about (15.5, 10.5, 10.5) (half extent 3) holds four of
    them, (13, 10 +- 1, 10) and (13, 10, 10 +- 1), at phi_B = -1/2 (the other
    such nodes lie 1.5 or more outside B): four rough-band nodes.  Radius
    -+2e-5 puts them beyond eps outside or inside: none."""
    r0 = math.sqrt(10.0) - S075
    for dr, band in ((0.0, 4), (-2e-5, 0), (2e-5, 0)):
        st = boxed(state([0, 1], [[r0 + dr, 0, 0], [3, 3, 3]], [[10, 10, 10], [15.5, 10.5, 10.5]], n=40))
        _, _, flags = oracle.box_pipeline(st)
        assert flags[0, 0] == band, (dr, flags)


def test_face_ties_of_face_aligned_boxes_are_exact():
    """Face-aligned boxes: every line of a face that meets the overlap enters
    it at the same plane, with the same FP64 arithmetic, so the two nearest
    lines tie exactly and no face counts as a near tie."""
    XA = np.array([30.3, 31.7, 29.2])
    st = boxed(state([1, 1], [[4, 4, 4], [4, 10, 10]], [XA, XA + [7.2, 0.0, 0.0]], n=80))
    _, _, flags = oracle.box_pipeline(st)
    assert flags[0, 1] == 0


def test_face_ties_of_slightly_tilted_boxes():
    """The same boxes, each turned by theta about a generic axis: every face
    of B0 is now met by its lines at an affine function of the line's
    position with slopes O(theta), so on each of the six faces the nearest
    and the second nearest line differ by about theta times the line spacing
    (0.5 to 1.3 cells here), never exactly.  theta = 1e-5: below 1e-4 dx on
    every face, six near ties.  theta = 3e-3: above it on every face, none."""
    XA = np.array([30.3, 31.7, 29.2])
    for theta, ties in ((1e-5, 6), (3e-3, 0)):
        q = [quat_axis_angle([1, 2, 3], theta), quat_axis_angle([-2, 1, 0.5], theta)]
        st = boxed(state([1, 1], [[4, 4, 4], [4, 10, 10]], [XA, XA + [7.2, 0.0, 0.0]], quat=q, n=80))
        _, _, flags = oracle.box_pipeline(st)
        assert flags[0, 1] == ties, (theta, flags)
