"""Seeded synthetic particle states shaped like the paper's hindered-settling runs.

The paper (Sec. 5.1, Sec. 5.4, Sec. 5.5) simulates periodic settling boxes of
spheres and cubes at 10-30 % volume fraction, up to 1934 particles at
L = 15 D_s; no dataset is involved.  These generators stand in for those
states: shapes, sizes, volume fractions and orientation statistics follow the
paper, positions come from random sequential addition (RSA).

This module holds no arithmetic of the contact method itself (no signed
distances, no lattice sweeps, no force law).  It only places shapes; the
overlap tests it uses for placement are the separating axis test and the
closest-point test of a sphere and a box.  Both the CUDA library and the oracle consume its output.

Every generator is deterministic in its seed.  Units are lattice units
(dx = 1 unless stated).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPHERE, CUBOID, POLYTOPE = 0, 1, 2

# Paper Sec. 5.1: E = 5 kPa for stable settling runs; the Poisson ratio is not
# given, 0.3 is used throughout.
YOUNG = 5.0e3
POISSON = 0.3


@dataclasses.dataclass
class State:
    """A particle state: shapes, material, poses and the lattice."""

    name: str
    n_cells: tuple
    dx: float
    shape_type: np.ndarray      # [N] int32
    shape_param: np.ndarray     # [N,3] f64 (sphere radius | cuboid half extents)
    face_offset: np.ndarray     # [N+1] int32 into planes
    planes: np.ndarray          # [F,4] f64, body frame n.y <= d, unit n
    young: np.ndarray           # [N] f64
    poisson: np.ndarray         # [N] f64
    pos: np.ndarray             # [N,3] f64 in [0, L)
    quat: np.ndarray            # [N,4] f64 (w, x, y, z)
    indicator: int = 0          # 0 sharp, 1 smoothed
    smooth_width: float = 1.0
    inflate: float = 0.0
    damping_c: float = 0.0
    info: dict = dataclasses.field(default_factory=dict)
    # fixed walls (Sec. 4.3): half-spaces m . x <= h, one (m, h) row each, not periodic
    walls: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 4)))
    wall_young: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    wall_poisson: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    # sample set: 0 every lattice node of the pair box; 1 the paper's box pipeline
    # (rough detection, box correction, contact_resolution^3 points; Sec. 3.3.1)
    box_mode: int = 0
    contact_resolution: int = 8

    @property
    def n(self) -> int:
        return int(self.shape_type.shape[0])

    @property
    def box(self) -> np.ndarray:
        return np.asarray(self.n_cells, dtype=np.float64) * self.dx

    def with_poses(self, pos, quat) -> "State":
        return dataclasses.replace(self, pos=np.ascontiguousarray(pos, dtype=np.float64),
                                   quat=np.ascontiguousarray(quat, dtype=np.float64))

    def subset(self, idx) -> "State":
        """The particles idx (in that order) in the same lattice."""
        idx = np.asarray(idx, dtype=np.int64)
        planes, offs = [], [0]
        for p in idx:
            pl = self.planes[self.face_offset[p]:self.face_offset[p + 1]]
            planes.append(pl)
            offs.append(offs[-1] + len(pl))
        planes = np.concatenate(planes) if planes else np.zeros((0, 4))
        return dataclasses.replace(
            self, shape_type=self.shape_type[idx].copy(), shape_param=self.shape_param[idx].copy(),
            face_offset=np.asarray(offs, dtype=np.int32), planes=np.ascontiguousarray(planes),
            young=self.young[idx].copy(), poisson=self.poisson[idx].copy(),
            pos=self.pos[idx].copy(), quat=self.quat[idx].copy(), info=dict(self.info))


# ----------------------------------------------------------------------------
# orientation and shape helpers

def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake's subgroup algorithm), (w,x,y,z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    return np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                     a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)


def rotation_matrices(q: np.ndarray) -> np.ndarray:
    """Body->world rotation matrices of quaternions (w,x,y,z) (placement only)."""
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw], -1)


def random_polytope(rng: np.random.Generator, n_faces: int, circumradius: float):
    """Convex polytope from n_faces random unit normals tangent to the unit
    sphere, origin moved to the volume centroid, scaled to the circumradius.

    Returns (planes [F,4] with unit normals, vertices [V,3]) in the body frame.
    """
    from scipy.spatial import ConvexHull, HalfspaceIntersection

    while True:
        nrm = rng.normal(size=(n_faces, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        hull = ConvexHull(nrm)
        if np.all(hull.equations[:, 3] < -0.05):   # origin well inside conv(normals): bounded
            break
    d = np.ones(n_faces)
    hs = np.concatenate([nrm, -d[:, None]], axis=1)
    verts = HalfspaceIntersection(hs, np.zeros(3)).intersections
    poly = ConvexHull(verts)
    # volume centroid from tetrahedra (interior point, facet triangle)
    inner = verts.mean(axis=0)
    vol, cen = 0.0, np.zeros(3)
    for simplex in poly.simplices:
        a, b, c = verts[simplex]
        v = abs(np.dot(a - inner, np.cross(b - inner, c - inner))) / 6.0
        vol += v
        cen += v * (inner + a + b + c) / 4.0
    cen /= vol
    d = d - nrm @ cen
    verts = verts - cen
    scale = circumradius / np.max(np.linalg.norm(verts, axis=1))
    return np.concatenate([nrm, (d * scale)[:, None]], axis=1), verts * scale


def cubes_intersect(c1, R1, h1, c2, R2, h2) -> bool:
    """Separating axis test of two oriented boxes (placement only)."""
    t = c2 - c1
    axes = [R1[:, k] for k in range(3)] + [R2[:, k] for k in range(3)]
    for a in range(3):
        for b in range(3):
            ax = np.cross(R1[:, a], R2[:, b])
            if np.linalg.norm(ax) > 1e-9:
                axes.append(ax / np.linalg.norm(ax))
    for ax in axes:
        r1 = np.sum(np.abs(R1.T @ ax) * h1)
        r2 = np.sum(np.abs(R2.T @ ax) * h2)
        if abs(np.dot(t, ax)) > r1 + r2:
            return False
    return True


def min_image(d: np.ndarray, L: np.ndarray) -> np.ndarray:
    return d - L * np.round(d / L)


def rsa_spheres(rng: np.random.Generator, n: int, diameter: float, L: float, batch: int = 4096):
    """Random sequential addition of n non-overlapping spheres in a periodic cube."""
    from scipy.spatial import cKDTree

    pts = np.zeros((0, 3))
    attempts = 0
    while len(pts) < n:
        cand = rng.random((batch, 3)) * L
        attempts += batch
        if len(pts):
            tree = cKDTree(pts, boxsize=L)
            dist, _ = tree.query(cand, k=1, distance_upper_bound=diameter)
            cand = cand[~np.isfinite(dist) | (dist >= diameter)]
        acc = []
        for c in cand:
            if acc:
                dd = min_image(np.asarray(acc) - c, np.full(3, L))
                if np.min(np.einsum("ij,ij->i", dd, dd)) < diameter * diameter:
                    continue
            acc.append(c)
            if len(pts) + len(acc) == n:
                break
        if acc:
            pts = np.concatenate([pts, np.asarray(acc)])
        if attempts > 200 * n * 50:
            raise RuntimeError("RSA did not reach the requested count")
    return np.mod(pts, L)


def _assemble(name, n_cells, dx, types, params, polys, pos, quat, **kw) -> State:
    planes, offs = [], [0]
    for p, t in enumerate(types):
        if t == POLYTOPE:
            planes.append(polys[p][0])
            offs.append(offs[-1] + len(polys[p][0]))
        else:
            offs.append(offs[-1])
    planes = np.concatenate(planes) if planes else np.zeros((0, 4))
    n = len(types)
    L = np.asarray(n_cells, dtype=np.float64) * dx
    return State(name=name, n_cells=tuple(int(v) for v in n_cells), dx=float(dx),
                 shape_type=np.asarray(types, dtype=np.int32),
                 shape_param=np.ascontiguousarray(params, dtype=np.float64),
                 face_offset=np.asarray(offs, dtype=np.int32), planes=np.ascontiguousarray(planes),
                 young=np.full(n, YOUNG), poisson=np.full(n, POISSON),
                 pos=np.ascontiguousarray(np.mod(pos, L)), quat=np.ascontiguousarray(quat), **kw)


# ----------------------------------------------------------------------------
# the five workloads

def shapes_intersect(ti, hi_, Ri, ci, tj, hj_, Rj, cj) -> bool:
    """Exact intersection test of two spheres/oriented boxes (placement only)."""
    if ti == SPHERE and tj == SPHERE:
        return float(np.linalg.norm(cj - ci)) <= hi_[0] + hj_[0]
    if ti == CUBOID and tj == CUBOID:
        return cubes_intersect(ci, Ri, hi_, cj, Rj, hj_)
    if ti == SPHERE:
        ti, hi_, Ri, ci, tj, hj_, Rj, cj = tj, hj_, Rj, cj, ti, hi_, Ri, ci
    y = Ri.T @ (cj - ci)                      # sphere centre in the box frame
    return float(np.linalg.norm(y - np.clip(y, -hi_, hi_))) <= hj_[0]


def _touch_offset(st_i, st_j, ci, base, direction, lo, hi):
    """Largest s in [lo, hi] with the shapes at ci and base + s*direction still
    intersecting (bisection; lo must intersect, hi must not)."""
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if shapes_intersect(*st_i, ci, *st_j, base + mid * direction):
            lo = mid
        else:
            hi = mid
    return lo


def mixed_grid_27(seed: int = 1, cuboid_half=(6.0, 6.0, 6.0)) -> State:
    """27 particles (14 spheres of diameter 15, 13 cubes of edge 12, or
    cuboids of the given half extents) on a jittered 3x3x3 grid in a periodic
    64^3 lattice.  Along every periodic grid line two of the three neighbour
    gaps are closed (the same open gap for all lines of one axis): the partner
    moves along the axis to first touch and then on by a penetration drawn
    from U(0, 1.5)."""
    rng = np.random.default_rng(seed)
    n, L = 27, 64.0
    types = np.array([SPHERE] * 14 + [CUBOID] * 13)[rng.permutation(27)]
    params = np.where(types[:, None] == SPHERE, [[7.5, 7.5, 7.5]], [list(cuboid_half)]).astype(np.float64)
    a = L / 3
    g = np.stack(np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij"), -1).reshape(-1, 3)
    pos = (g + 0.5) * a + rng.uniform(-1, 1, size=(n, 3))
    quat = random_quaternions(rng, n)
    R = rotation_matrices(quat)
    Lv = np.full(3, L)
    idx = lambda c: int(c[0] * 9 + c[1] * 3 + c[2])
    for ax in range(3):
        others = [k for k in range(3) if k != ax]
        start = int(rng.integers(3))
        for u in range(3):
            for v in range(3):
                line = []
                for t in range(3):
                    c = [0, 0, 0]
                    c[ax] = (start + t) % 3
                    c[others[0]], c[others[1]] = u, v
                    line.append(idx(c))
                for t in range(2):
                    i, j = line[t], line[t + 1]
                    e = np.zeros(3)
                    e[ax] = 1.0
                    ci = pos[i]
                    base = ci + min_image(pos[j] - ci, Lv)
                    base[ax] = ci[ax]
                    s = _touch_offset((types[i], params[i], R[i]), (types[j], params[j], R[j]),
                                      ci, base, e, 0.0, 30.0)
                    pos[j, ax] = ci[ax] + s - rng.uniform(0.0, 1.5)
    return _assemble("mixed27_64", (64, 64, 64), 1.0, types, params, {}, pos, quat)


def settling_cubes(seed: int = 2, n: int = 400, edge: float = 12.0, phi: float = 0.10,
                   touch_frac: float = 0.15, max_pen: float = 1.0) -> State:
    """n cubes of the given edge at volume fraction phi by RSA with an exact
    box-box overlap test; then touch_frac of the particles are moved towards
    their nearest neighbour to a support overlap of U(0, max_pen)."""
    rng = np.random.default_rng(seed)
    Lf = (n * edge ** 3 / phi) ** (1.0 / 3.0)
    L = float(round(Lf))
    Lv = np.full(3, L)
    h = np.full(3, edge / 2)
    quat = random_quaternions(rng, n)
    R = rotation_matrices(quat)
    pos = np.zeros((n, 3))
    circ = float(np.linalg.norm(h))
    placed = 0
    while placed < n:
        c = rng.random(3) * L
        ok = True
        if placed:
            d = min_image(pos[:placed] - c, Lv)
            near = np.nonzero(np.einsum("ij,ij->i", d, d) < (2 * circ) ** 2)[0]
            for k in near:
                if cubes_intersect(c, R[placed], h, c + d[k], R[k], h):
                    ok = False
                    break
        if ok:
            pos[placed] = c
            placed += 1
    params = np.tile(h, (n, 1))
    movers = rng.choice(n, size=int(round(touch_frac * n)), replace=False)
    for j in movers:
        d = min_image(pos - pos[j], Lv)
        dist = np.einsum("ij,ij->i", d, d)
        dist[j] = np.inf
        i = int(np.argmin(dist))
        dv = min_image(pos[j] - pos[i], Lv)
        u = dv / np.linalg.norm(dv)
        s = _touch_offset((CUBOID, h, R[i]), (CUBOID, h, R[j]), pos[i], pos[i], u, 0.0, 4 * circ)
        pos[j] = pos[i] + u * (s - rng.uniform(0.0, max_pen))
    st = _assemble(f"cubes{n}_{int(L)}", (int(L),) * 3, 1.0, [CUBOID] * n, params, {}, pos, quat)
    st.info["phi"] = n * edge ** 3 / L ** 3
    return st


def mixed_settling(seed: int = 3, n: int = 1934, L: int = 223, d_sphere: float = 14.9,
                   phi_rsa: float = None, kinds=(SPHERE, CUBOID, POLYTOPE)) -> State:
    """Settling box of n particles: RSA positions of volume-equivalent spheres
    (diameter d_sphere), then 1/len(kinds) each of spheres (d_sphere), cubes of
    edge 12 and convex polytopes (12-20 random faces, circumradius U(8, 11))
    placed at those centres with uniform random orientations."""
    rng = np.random.default_rng(seed)
    pos = rsa_spheres(rng, n, d_sphere, float(L))
    kinds = list(kinds)
    types = np.array([kinds[k % len(kinds)] for k in range(n)])[rng.permutation(n)]
    quat = random_quaternions(rng, n)
    params = np.zeros((n, 3))
    polys = {}
    for p in range(n):
        if types[p] == SPHERE:
            params[p] = [d_sphere / 2, 0, 0]
        elif types[p] == CUBOID:
            params[p] = [6.0, 6.0, 6.0]
        else:
            polys[p] = random_polytope(rng, int(rng.integers(12, 21)), float(rng.uniform(8.0, 11.0)))
    st = _assemble(f"mixed{n}_{L}", (L, L, L), 1.0, types, params, polys, pos, quat)
    st.info["phi_spheres"] = n * math.pi / 6 * d_sphere ** 3 / L ** 3
    return st


def settling_cubes_dense(seed: int = 4, n: int = 1934, L: int = 223) -> State:
    """n cubes of edge 12 at the RSA centres of volume-equivalent spheres
    (phi = n 12^3 / L^3 = 0.301 at n = 1934, L = 223), smoothed indicator w = 1."""
    st = mixed_settling(seed=seed, n=n, L=L, kinds=(CUBOID,))
    st.name = f"cubes{n}_{L}_smooth"
    st.indicator = 1
    st.smooth_width = 1.0
    st.info["phi"] = n * 12.0 ** 3 / L ** 3
    return st


def resolution_sweep(edge: int, seed: int = 5, n: int = 500, phi: float = 0.20,
                     aligned_frac: float = 0.5, face_pairs_frac: float = 0.15) -> State:
    """n cubes of edge `edge` at volume fraction phi in L = round(edge 2500^(1/3)).
    A fraction of the cubes is axis-aligned with faces on half-integer node
    coordinates (exact lattice box volumes); some of those are moved into
    face-aligned contact with an integer penetration of 1 or 2 cells."""
    rng = np.random.default_rng(seed)
    L = int(round(edge * (n / phi) ** (1.0 / 3.0)))
    d_eq = edge * (6.0 / math.pi) ** (1.0 / 3.0)
    pos = rsa_spheres(rng, n, d_eq, float(L))
    quat = random_quaternions(rng, n)
    aligned = rng.random(n) < aligned_frac
    quat[aligned] = [1.0, 0.0, 0.0, 0.0]
    half = edge / 2.0
    off = 0.5 if edge % 2 == 0 else 0.0
    pos[aligned] = np.floor(pos[aligned]) + off
    Lv = np.full(3, float(L))
    al = np.nonzero(aligned)[0]
    moved = set()
    for j in rng.permutation(al)[: int(face_pairs_frac * len(al))]:
        if j in moved:
            continue
        d = min_image(pos[al] - pos[j], Lv)
        dist = np.einsum("ij,ij->i", d, d)
        dist[al == j] = np.inf
        i = int(al[np.argmin(dist)])
        dv = min_image(pos[j] - pos[i], Lv)
        ax = int(np.argmax(np.abs(dv)))
        sgn = 1.0 if dv[ax] >= 0 else -1.0
        new = pos[i].copy()
        new[ax] += sgn * (2 * half - rng.integers(1, 3))
        for k in range(3):
            if k != ax:
                new[k] = pos[i][k] + np.clip(np.round(dv[k]), -(edge - 2), edge - 2)
        pos[j] = new
        moved.add(j)
        moved.add(i)
    params = np.full((n, 3), half)
    st = _assemble(f"cubes{n}_e{edge}_{L}", (L, L, L), 1.0, [CUBOID] * n, params, {}, pos, quat)
    st.info["phi"] = n * edge ** 3 / L ** 3
    st.info["aligned"] = aligned
    return st


def with_walls(state: State, walls, young=None, poisson=None) -> State:
    """The state with fixed walls (rows (m, h): the half-space m . x <= h, unit m
    out of the wall), of the particles' material unless given."""
    st = dataclasses.replace(state)
    st.walls = np.asarray(walls, float).reshape(-1, 4).copy()
    st.walls[:, :3] /= np.linalg.norm(st.walls[:, :3], axis=1, keepdims=True)
    w = len(st.walls)
    st.wall_young = np.full(w, float(state.young[0] if young is None else young))
    st.wall_poisson = np.full(w, float(state.poisson[0] if poisson is None else poisson))
    return st


def floor_and_ceiling(state: State, gap: float = 2.0) -> State:
    """A floor below the lowest centre and a ceiling above the highest, each
    `gap` from it, so the particles near them press into the walls."""
    z = state.pos[:, 2]
    return with_walls(state, [[0.0, 0.0, 1.0, z.min() - gap], [0.0, 0.0, -1.0, -(z.max() + gap)]])


def pose_sequence(state: State, steps: int, seed: int = 11, sigma_x: float = 0.05,
                  sigma_rot: float = 0.01):
    """`steps` poses after small random increments: dX ~ N(0, sigma_x) per
    axis, a rotation by N(0, sigma_rot) rad about a uniform random axis."""
    rng = np.random.default_rng(seed)
    L = state.box
    pos = np.empty((steps, state.n, 3))
    quat = np.empty((steps, state.n, 4))
    p, q = state.pos.copy(), state.quat.copy()
    for s in range(steps):
        pos[s], quat[s] = p, q
        p = np.mod(p + rng.normal(0.0, sigma_x, size=p.shape), L)
        p[p >= L] = 0.0
        axis = rng.normal(size=(state.n, 3))
        axis /= np.linalg.norm(axis, axis=1, keepdims=True)
        ang = rng.normal(0.0, sigma_rot, size=state.n)
        dq = np.concatenate([np.cos(ang / 2)[:, None], np.sin(ang / 2)[:, None] * axis], axis=1)
        q = quat_mul(dq, q)
        q /= np.linalg.norm(q, axis=1, keepdims=True)
    return pos, quat


def loss_weights(n: int, seed: int = 7):
    """Random FP32 weights w_f, w_t ~ U(-1, 1) for the loss sum_p w_f.F_p + w_t.T_p."""
    rng = np.random.default_rng(seed)
    wf = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32).astype(np.float64)
    wt = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32).astype(np.float64)
    return wf, wt


WORKLOADS = {
    "mixed27_64": mixed_grid_27,
    "cubes400_191": settling_cubes,
    "mixed1934_223": mixed_settling,
    "cubes1934_223_smooth": settling_cubes_dense,
}
