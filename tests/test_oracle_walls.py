"""Pins of the oracle's particle-wall contacts (CPU only).

Sec. 4.3 treats a contact with a fixed wall like a particle pair; the wall
here is the half-space m . x <= h (unit m pointing out of the wall), not
periodic, and the pair is (i, N + w).  The pins: exact slab volumes, contact
point and depth for face-aligned cubes, the spherical-cap volume with its
convergence, the normal by symmetry, a brute-force scan of every node near an
oblique wall (pins the clipped box), integer translations, the wall's
non-periodicity, damping and friction signs, and the gradient against central
differences.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import state


def with_walls(st, walls, young=2.0, poisson=0.0):
    st.walls = np.asarray(walls, float).reshape(-1, 4)
    st.wall_young = np.full(len(st.walls), float(young))
    st.wall_poisson = np.full(len(st.walls), float(poisson))
    return st


def floor(h):
    return [0.0, 0.0, 1.0, h]   # solid z <= h


def wall_rows(r, n):
    return np.nonzero(r.pair_ij[:, 1] >= n)[0]


@pytest.mark.parametrize("h,layers", [(17.5, 1), (19.5, 3)])
def test_face_aligned_cube_on_floor_exact(h, layers):
    """Cube (half extent 4, faces on half-integer nodes, bottom at z = 16.5)
    on the floor z <= h: V = 8 x 8 x layers nodes, x_c the slab centre,
    d = h - 16.5, n = -m, no torque."""
    X = np.array([30.5, 31.5, 20.5])
    st = with_walls(state([1], [[4, 4, 4]], [X]), [floor(h)])
    r = oracle.contact_step(st)
    rows = wall_rows(r, 1)
    assert r.pair_ij[rows].tolist() == [[0, 1]]
    o = r.pair_out[rows[0]]
    assert o[0] == 64 * layers
    assert np.array_equal(o[1:4], [30.5, 31.5, 17 + (layers - 1) / 2])
    assert o[4:7].tolist() == [0.0, 0.0, -1.0]
    assert o[7] == h - 16.5
    # the force on the cube points out of the wall; the torque vanishes
    assert np.allclose(r.force[0] / np.linalg.norm(r.force[0]), [0, 0, 1], atol=1e-15)
    assert np.abs(r.torque[0]).max() == 0.0


def test_sphere_cap_volume():
    """Sphere of radius r cut by the floor at depth t: averaged over a 4 x 4 x 4
    grid of sub-cell shifts of the whole configuration, the volume approaches
    the cap volume pi t^2 (3 r - t) / 3 at first order in dx."""
    r_phys, t = 6.0, 1.7
    exact = math.pi * t * t * (3 * r_phys - t) / 3
    errs = []
    for dx in (1.0, 0.5):
        n = int(round(40 / dx))
        vs = []
        for s in itertools.product(range(4), repeat=3):
            X = np.array([20.0, 20.0, 12.3]) + (np.array(s) + 0.37) / 4 * dx
            h = X[2] - (r_phys - t)
            st = with_walls(state([0], [[r_phys, 0, 0]], [X], n=n, dx=dx), [floor(h)])
            res = oracle.contact_step(st)
            vs.append(res.pair_out[wall_rows(res, 1)[0], 0])
        errs.append(abs(np.mean(vs) - exact) / exact)
    assert errs[1] < 0.025 and math.log2(errs[0] / errs[1]) > 0.9, errs


def test_sphere_on_floor_normal_and_contact_point_by_symmetry():
    """Centre on a lattice column: the normal is -m and x_c on the column."""
    X = np.array([20.0, 21.0, 12.3])
    st = with_walls(state([0], [[6.0, 0, 0]], [X]), [floor(7.9)])
    r = oracle.contact_step(st)
    o = r.pair_out[wall_rows(r, 1)[0]]
    assert o[0] > 0
    assert np.allclose(o[4:7], [0, 0, -1], atol=1e-12)
    assert abs(o[1] - 20.0) < 1e-12 and abs(o[2] - 21.0) < 1e-12
    assert 12.3 - 6.0 < o[3] < 7.9   # inside the cap


def _sdf_np(kind, prm, X, R, planes, x):
    r = (x - X) @ R          # body coordinates
    if kind == 0:
        return np.linalg.norm(x - X, axis=1) - prm[0]
    if kind == 1:
        return np.max(np.abs(r) - prm, axis=1)
    return np.max(r @ planes[:, :3].T - planes[:, 3], axis=1)


def test_brute_force_scan_near_oblique_walls():
    """Every node in a window around the particle (no box): the count of nodes
    inside both the particle and the oblique wall, and their first moments,
    equal the oracle's clipped-box sums (pins the candidate test and the clip)."""
    rng = np.random.default_rng(11)
    hits = 0
    for trial in range(8):
        kind = trial % 3
        prm = [[5.5, 0, 0], [3.5, 4.0, 4.5], [0, 0, 0]][kind]
        pl = W.random_polytope(rng, 12, 6.0)[0] if kind == 2 else None
        q = W.random_quaternions(rng, 1)
        X = np.array([30.0, 31.0, 32.0]) + rng.random(3)
        m = rng.normal(size=3)
        m /= np.linalg.norm(m)
        h = float(m @ X) - rng.uniform(2.0, 6.5)    # the wall reaches into the particle
        st = with_walls(state([kind], [prm], [X], q, planes=[pl]), [[*m, h]])
        r = oracle.contact_step(st)
        rows = wall_rows(r, 1)
        R = W.rotation_matrices(q)[0]
        k = np.stack(np.meshgrid(*[np.arange(16, 48)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
        inside = (_sdf_np(kind, np.asarray(prm, float), X, R, pl, k) <= 0) & (k @ m - h <= 0)
        V = r.pair_out[rows[0], 0] if len(rows) else 0.0
        assert V == inside.sum(), (trial, V, inside.sum())
        if V > 0:
            hits += 1
            assert np.allclose(r.pair_out[rows[0], 1:4], k[inside].mean(axis=0), atol=1e-12)
    assert hits >= 6
    # grazing: axis-aligned walls entering a sphere by 0.9 cells, where the
    # candidate test decides near its threshold
    grazing = 0
    for trial in range(6):
        X = np.array([30.0, 31.0, 32.0]) + rng.random(3)
        m = np.zeros(3)
        m[trial % 3] = 1.0 if trial < 3 else -1.0
        h = float(m @ X) - 5.5 + 0.9
        st = with_walls(state([0], [[5.5, 0, 0]], [X]), [[*m, h]])
        r = oracle.contact_step(st)
        rows = wall_rows(r, 1)
        k = np.stack(np.meshgrid(*[np.arange(16, 48)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(float)
        inside = (np.linalg.norm(k - X, axis=1) - 5.5 <= 0) & (k @ m - h <= 0)
        V = r.pair_out[rows[0], 0] if len(rows) else 0.0
        assert V == inside.sum(), (trial, V, inside.sum())
        grazing += inside.sum() > 0
    assert grazing >= 4


def test_integer_translation_of_particle_and_wall():
    rng = np.random.default_rng(3)
    q = W.random_quaternions(rng, 1)
    m = np.array([0.3, -0.5, 0.8])
    m /= np.linalg.norm(m)
    X = np.array([30.2, 29.7, 31.4])
    h = float(m @ X) - 2.5
    a = oracle.contact_step(with_walls(state([1], [[3.5, 4.0, 4.5]], [X], q), [[*m, h]]))
    t = np.array([3.0, -2.0, 5.0])
    b = oracle.contact_step(with_walls(state([1], [[3.5, 4.0, 4.5]], [X + t], q), [[*m, h + m @ t]]))
    oa, ob = a.pair_out[wall_rows(a, 1)[0]], b.pair_out[wall_rows(b, 1)[0]]
    assert oa[0] > 0 and oa[0] == ob[0]
    assert np.allclose(ob[1:4], oa[1:4] + t, atol=1e-11)
    assert np.allclose(ob[4:11], oa[4:11], atol=1e-11)


def test_wall_is_not_periodic_and_far_particles_have_no_pair():
    # solid x <= 2: a cube at x = 61 touches it only through the periodic image
    st = with_walls(state([1, 1], [[4, 4, 4]] * 2, [[61.0, 20.0, 20.0], [30.0, 40.0, 40.0]]),
                    [[1.0, 0.0, 0.0, 2.0]])
    r = oracle.contact_step(st)
    assert len(wall_rows(r, 2)) == 0
    # a candidate whose box reaches only the wall's band: a pair with zero outputs
    st = with_walls(state([1], [[4, 4, 4]], [[30.5, 30.5, 30.5]], indicator=1, w=1.0), [floor(26.2)])
    r = oracle.contact_step(st)
    rows = wall_rows(r, 1)
    assert len(rows) == 1 and r.pair_out[rows[0], 0] == 0.0 and np.all(r.pair_out[rows[0]] == 0.0)


def test_wall_damping_and_friction_signs():
    """A cube moving into the floor is damped more than one moving away; a
    cube sliding along +x receives friction along -x, opposing its slip."""
    X = np.array([30.5, 31.5, 20.5])
    st = with_walls(state([1], [[4, 4, 4]], [X]), [floor(17.5)])
    law = oracle.ContactLaw(restitution=0.5, history=True)
    down = oracle.contact_step_ext(st, law, vel=np.array([[0, 0, -0.2, 0, 0, 0]]))
    base = oracle.contact_step(st)
    Fb = base.force[0, 2]
    assert down.force[0, 2] == pytest.approx(Fb * (1 + oracle.damping_factor(0.5, 1.0)), rel=1e-13)
    c = down.hist_c[0]
    up = oracle.contact_step_ext(st, law, vel=np.array([[0, 0, 0.1, 0, 0, 0]]), hist=(down.hist_ij, down.hist_c))
    assert up.force[0, 2] == pytest.approx(Fb * (1 - 0.1 * c), rel=1e-13)
    fr = oracle.ContactLaw(friction=True, mu_s=0.5, mu_k=0.3, u_k=1e-3)
    slide = oracle.contact_step_ext(st, fr, vel=np.array([[0.5, 0, 0, 0, 0, 0]]))
    assert slide.force[0, 0] < 0 and slide.force[0, 0] == pytest.approx(-0.3 * Fb, rel=1e-4)   # a = 500


def test_gradient_with_walls_matches_central_differences():
    """Particles pressed into a floor and an oblique wall (smoothed
    indicator): the forward-mode gradient equals central differences on every
    component whose stencil is smooth (FD with h and h/2 agree; the rest
    straddle a switch of the deepest node or the active face)."""
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width = 1, 1.0
    m = np.array([0.6, 0.0, -0.8])
    with_walls(st, [[0, 0, 1.0, float(st.pos[:, 2].min()) - 3.0], [*m, float((st.pos @ m).min()) - 3.0]])
    r = oracle.contact_step(st)
    rows = wall_rows(r, st.n)
    assert len(rows) >= 4 and np.count_nonzero(r.pair_out[rows, 0]) >= 4
    gf, gt = W.loss_weights(st.n)
    gp, gq = oracle.gradient(st, gf, gt)

    def loss(pos, quat):
        rr = oracle.contact_step(st, pos=pos, quat=quat)
        return float(np.sum(gf * rr.force) + np.sum(gt * rr.torque))

    def fd(p, k, h, on_pos):
        a, b = (st.pos.copy(), st.pos.copy()) if on_pos else (st.quat.copy(), st.quat.copy())
        a[p, k] += h
        b[p, k] -= h
        return ((loss(a, st.quat) - loss(b, st.quat)) if on_pos else (loss(st.pos, a) - loss(st.pos, b))) / (2 * h)

    scale = max(np.abs(gp).max(), np.abs(gq).max())
    smooth, err = [], []
    for p in np.unique(r.pair_ij[rows, 0]):
        for on_pos, nk, g in ((True, 3, gp), (False, 4, gq)):
            for k in range(nk):
                f1, f2 = fd(p, k, 1e-4, on_pos), fd(p, k, 5e-5, on_pos)
                smooth.append(abs(f1 - f2) < 1e-6 * scale)
                err.append(abs(f2 - g[p, k]) / scale)
    smooth, err = np.array(smooth), np.array(err)
    assert smooth.mean() >= 0.8, smooth.mean()
    assert np.all(err[smooth] < 1e-5), np.sort(err[smooth])[-5:]
