"""Small hand-built particle states for the tests (no contact arithmetic here)."""
import numpy as np

from paper_2401_10878_gb300 import workloads as W

IDENTITY = [1.0, 0.0, 0.0, 0.0]


def state(types, params, pos, quat=None, n=64, dx=1.0, planes=None, indicator=0, w=1.0,
          young=2.0, poisson=0.0, inflate=0.0, damping_c=0.0):
    """A state with the given particles; planes is a list (one entry per
    particle, None for non-polytopes) of [F,4] arrays."""
    k = len(types)
    quat = [IDENTITY] * k if quat is None else quat
    offs, pl = [0], []
    for p in range(k):
        if planes is not None and planes[p] is not None:
            pl.append(np.asarray(planes[p], float))
            offs.append(offs[-1] + len(planes[p]))
        else:
            offs.append(offs[-1])
    n_cells = (n, n, n) if np.isscalar(n) else tuple(n)
    return W.State("test", n_cells, float(dx), np.asarray(types, np.int32),
                   np.asarray(params, float).reshape(k, 3), np.asarray(offs, np.int32),
                   np.concatenate(pl) if pl else np.zeros((0, 4)), np.full(k, float(young)),
                   np.full(k, float(poisson)), np.asarray(pos, float).reshape(k, 3),
                   np.asarray(quat, float).reshape(k, 4), indicator=indicator, smooth_width=w,
                   inflate=inflate, damping_c=damping_c)


def cube_planes(h):
    """The 6 face planes (+x, -x, +y, -y, +z, -z) of a box with half extents h."""
    h = np.broadcast_to(np.asarray(h, float), (3,))
    rows = []
    for k in range(3):
        for s in (1.0, -1.0):
            nrm = np.zeros(3)
            nrm[k] = s
            rows.append([*nrm, h[k]])
    return np.array(rows)


def quat_axis_angle(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def lens_volume(r1, r2, D):
    """Volume of the intersection of two balls (radii r1, r2, centre distance D)."""
    return np.pi * (r1 + r2 - D) ** 2 * (D * D + 2 * D * r2 - 3 * r2 * r2 + 2 * D * r1 + 6 * r1 * r2
                                         - 3 * r1 * r1) / (12 * D)


def cap_centroid_offset(r, h):
    """Distance of the centroid of a spherical cap of height h from the ball centre."""
    return 3 * (2 * r - h) ** 2 / (4 * (3 * r - h))
