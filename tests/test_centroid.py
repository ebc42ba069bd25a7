"""The centre-of-mass convention (Sec. 2.2: poses refer to the centre of
mass): polytope volume centroids, by the oracle (face pyramids) against
closed forms, by the library (tetrahedra) against the oracle, and the
refusal of a polytope whose body origin is not its centroid (CPU only; the
library's check runs before any device work)."""
import ctypes

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
    """Square pyramid, base z = -1 (side 2), apex z = 3: centroid at z = 0."""
    v = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [0, 0, 3.0]])
    assert np.allclose(oracle.polytope_centroid(planes_from_vertices(v)), 0.0, atol=1e-13)


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


def test_off_centre_polytope_refused():
    from paper_2401_10878_gb300 import contact as C
    lib = C.load_library()
    pl = box_planes(np.array([-1.0, -2.0, -0.5]), np.array([3.0, 2.0, 1.5]))   # centroid (1, 0, 0.5)
    st = state([2], [[0, 0, 0]], [[30.0, 30.0, 30.0]], planes=[pl])
    with pytest.raises(oracle.OracleError):
        oracle.contact_step(st)
    cfg = C.Config()
    n_cells = (ctypes.c_int32 * 3)(*st.n_cells)
    lib.contact_config_default(ctypes.byref(cfg), st.n, n_cells, st.dx)
    arrs = [np.ascontiguousarray(a) for a in (st.shape_type, st.shape_param, st.face_offset, st.planes, st.young,
                                              st.poisson)]
    ctx = ctypes.c_void_p()
    rc = lib.contact_init(ctypes.byref(cfg), *[a.ctypes.data for a in arrs], None, ctypes.byref(ctx))
    assert rc == C.EINVAL and not ctx.value
    # re-centred planes are accepted by the oracle
    c = oracle.polytope_centroid(pl)
    pl2 = pl.copy()
    pl2[:, 3] -= pl[:, :3] @ c
    oracle.contact_step(state([2], [[0, 0, 0]], [[30.0, 30.0, 30.0]], planes=[pl2]))
