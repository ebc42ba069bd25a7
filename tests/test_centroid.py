"""The centre-of-mass convention (Sec. 2.2: poses refer to the centre of
mass): polytope volume centroids, by the oracle (face pyramids) against
closed forms and by the library (tetrahedra) against the oracle; a polytope
whose body origin is off its centroid is moved there, by both sides (the
last test needs a GB300)."""

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import cube_planes, state


def box_planes(lo, hi):
    rows = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        rows.append([*e, hi[k]])
        rows.append([*(-e), -lo[k]])
    return np.array(rows)


def planes_from_vertices(verts):
    """Face planes (outward unit normal, offset) of a convex hull."""
    from scipy.spatial import ConvexHull
    hull = ConvexHull(verts)
    _, first = np.unique(np.round(hull.equations, 9), axis=0, return_index=True)   # coplanar facets: one row
    eq = hull.equations[np.sort(first)]
    return np.concatenate([eq[:, :3], -eq[:, 3:]], axis=1)


def test_box_centroid_is_its_centre():
    lo, hi = np.array([-1.0, -2.0, -0.5]), np.array([3.0, 2.0, 1.5])
    assert np.allclose(oracle.polytope_centroid(box_planes(lo, hi)), (lo + hi) / 2, atol=1e-14)


def test_tetrahedron_centroid_is_the_vertex_mean():
    v = np.array([[2.0, -1.0, -1.0], [-1.0, 2.5, -1.0], [-1.2, -1.0, 2.0], [-0.5, -0.7, -1.5]])
    c = oracle.polytope_centroid(planes_from_vertices(v))
    assert np.allclose(c, v.mean(axis=0), atol=1e-13)


def test_pyramid_centroid_at_a_quarter_height():
    """Square pyramid, base z = -0.6 (side 2), apex z = 3.4: the centroid a
    quarter of the height above the base, z = 0.4 (off the origin, so a wrong
    weight of the face pyramids shows)."""
    v = np.array([[-1, -1, -0.6], [1, -1, -0.6], [1, 1, -0.6], [-1, 1, -0.6], [0, 0, 3.4]])
    assert np.allclose(oracle.polytope_centroid(planes_from_vertices(v)), [0.0, 0.0, 0.4], atol=1e-13)


def test_library_centroid_matches_oracle():
    from paper_2401_10878_gb300.contact import load_library
    lib = load_library()
    rng = np.random.default_rng(3)
    for f in (6, 9, 14, 20, 32):
        pl = W.random_polytope(rng, f, 7.0)[0]
        pl[:, 3] += pl[:, :3] @ rng.normal(size=3) * 0.5   # move the origin off the centroid
        c_lib = np.zeros(3)
        assert lib.contact_polytope_centroid(np.ascontiguousarray(pl).ctypes.data, len(pl), c_lib.ctypes.data) == 0
        assert np.allclose(c_lib, oracle.polytope_centroid(pl), atol=1e-11)
    # a cube's planes: the origin
    c = np.zeros(3)
    assert lib.contact_polytope_centroid(np.ascontiguousarray(cube_planes(2.0)).ctypes.data, 6, c.ctypes.data) == 0
    assert np.abs(c).max() < 1e-14


def test_off_centre_polytope_moved_to_its_centroid():
    """An off-centre box is moved to its centroid (1, 0, 0.5): the step equals
    that of the box given about its centroid at the same position, and the
    shift is reported; centred polytopes are not moved."""
    pl = box_planes(np.array([-1.0, -2.0, -0.5]), np.array([3.0, 2.0, 1.5]))
    pos = [[20.3, 20.1, 20.2], [25.0, 21.4, 20.9]]
    cube = cube_planes(3.0)
    st = state([2, 2], np.zeros((2, 3)), pos, planes=[pl, cube])
    assert np.array_equal(oracle.polytope_shift(st), [[1.0, 0.0, 0.5], [0.0, 0.0, 0.0]])
    pl2 = pl.copy()
    pl2[:, 3] -= pl[:, :3] @ np.array([1.0, 0.0, 0.5])   # axis normals: exact
    r1 = oracle.contact_step(st)
    r2 = oracle.contact_step(state([2, 2], np.zeros((2, 3)), pos, planes=[pl2, cube]))
    assert r1.n_pairs == 1 and r1.pair_out[0, 0] > 0
    assert np.array_equal(r1.pair_out, r2.pair_out) and np.array_equal(r1.force, r2.force)
    rng = np.random.default_rng(5)
    centred = state([2, 2], np.zeros((2, 3)), pos, planes=[W.random_polytope(rng, f, 5.0)[0] for f in (12, 20)])
    assert not oracle.polytope_shift(centred).any()


def off_centre_polytopes():
    rng = np.random.default_rng(11)
    polys = []
    for f in (14, 20, 16, 24):
        pl = W.random_polytope(rng, f, 8.0)[0]
        u = rng.normal(size=3)
        pl[:, 3] += pl[:, :3] @ (u / np.linalg.norm(u) * 0.4 * pl[:, 3].min())   # the origin moved off the centroid
        polys.append(pl)
    pos = [[20, 20, 20], [29, 21, 19], [20, 29, 21], [29, 29, 20]]
    return state([2, 2, 2, 2], np.zeros((4, 3)), pos, W.random_quaternions(rng, 4), planes=polys)


def test_off_centre_state_needs_a_shift():
    st = off_centre_polytopes()
    sh = oracle.polytope_shift(st)
    assert (np.linalg.norm(sh, axis=1) > 0.05).all()
    assert oracle.contact_step(st).n_pairs >= 3


@pytest.mark.gpu
def test_library_moves_polytopes_like_the_oracle():
    pytest.importorskip("torch")
    from paper_2401_10878_gb300.contact import Contact
    from tests.parity import compare, gpu_step
    st = off_centre_polytopes()
    m = Contact.from_state(st)
    assert np.allclose(m.polytope_shift(), oracle.polytope_shift(st), rtol=0, atol=1e-11)
    g = gpu_step(m, st)
    r = oracle.contact_step(st)
    print("off-centre polytopes", compare(st, g, r, fp64=False, smooth=False))
    assert np.array_equal(m.particle_boxes().cpu().numpy(), oracle.aabb(st))
    m.close()
