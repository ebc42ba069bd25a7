"""CUDA particle-wall contacts vs the oracle (needs a GB300): fixed walls
(Sec. 4.3) as half-spaces, pairs (i, N + w), in every node-sweep variant
(cubes, spheres and cuboids, all kinds), both forms, the smoothed indicator
with the adjoint, and the contact law (history and friction) with walls.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.helpers import state
from tests.law_parity import LawTracker
from tests.parity import compare, gpu_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def model_for(st, **kw):
    from paper_2401_10878_gb300.contact import Contact
    return Contact.from_state(st, **kw)


def run(st, precision=0, **kw):
    m = model_for(st, precision=precision, **kw)
    g = gpu_step(m, st)
    r = oracle.contact_step(st)
    rep = compare(st, g, r, fp64=precision == 1, smooth=st.indicator == 1)
    walls = int((r.pair_ij[:, 1] >= st.n).sum())
    m.close()
    return rep, walls


def oblique(st, gap=2.0):
    """Floor, ceiling and one oblique wall below the particles' lowest point along it."""
    m = np.array([0.48, -0.36, 0.8])
    m /= np.linalg.norm(m)
    fc = W.floor_and_ceiling(st, gap)
    return W.with_walls(st, np.concatenate([fc.walls, [[*m, float((st.pos @ m).min()) - gap]]]))


@pytest.mark.parametrize("precision", [0, 1])
def test_cubes1934_floor_ceiling_oblique(precision):
    rep, walls = run(oblique(W.settling_cubes_dense()), precision)
    print("cubes1934 + walls", precision, rep, "wall pairs", walls)
    assert walls > 100


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed1934_walls(precision):
    rep, walls = run(oblique(W.mixed_settling()), precision)
    print("mixed1934 + walls", precision, rep, "wall pairs", walls)
    assert walls > 80


def test_spheres_and_cuboids_walls():
    st = W.mixed_grid_27()
    keep = st.shape_type != 2
    assert keep.all()   # spheres and cubes only: the sphere/cuboid variant
    rep, walls = run(oblique(st, gap=1.0))
    print("mixed27 + walls", rep, "wall pairs", walls)
    assert walls >= 6


@pytest.mark.parametrize("precision", [0, 1])
def test_elongated_cuboids_walls(precision):
    """Cuboids of unequal half extents (7, 5, 4) and spheres against a floor,
    a ceiling and an oblique wall: the wall-cuboid evaluator pair."""
    rep, walls = run(oblique(W.mixed_grid_27(cuboid_half=(7.0, 5.0, 4.0)), gap=1.0), precision)
    print("mixed27 cuboids + walls", precision, rep, "wall pairs", walls)
    assert walls >= 6


def test_face_aligned_cube_on_floor_exact():
    X = np.array([30.5, 31.5, 20.5])
    st = W.with_walls(state([1], [[4, 4, 4]], [X]), [[0, 0, 1, 19.5]])
    m = model_for(st, precision=0)
    g = gpu_step(m, st)
    assert g["pair_ij"].tolist() == [[0, 1]]
    o = g["pair_out"][0]
    assert o[0] == 192 and np.array_equal(o[1:4], [30.5, 31.5, 18.0]) and o[4:7].tolist() == [0.0, 0.0, -1.0]
    assert o[7] == pytest.approx(3.0, abs=1e-12)
    r = oracle.contact_step(st)
    assert np.allclose(g["force"], r.force, rtol=1e-12, atol=0) and np.abs(g["torque"]).max() == 0.0
    m.close()


def test_smoothed_walls_and_adjoint():
    st = oblique(W.settling_cubes())
    st.indicator, st.smooth_width = 1, 1.0
    rep, walls = run(st)
    print("cubes400 smooth + walls", rep, "wall pairs", walls)
    m = model_for(st)
    pos = torch.tensor(st.pos, device="cuda")
    quat = torch.tensor(st.quat, device="cuda")
    m.step(pos, quat)
    gf, gt = W.loss_weights(st.n)
    gp, gq = m.backward(torch.tensor(gf, device="cuda"), torch.tensor(gt, device="cuda"))
    rp, rq = oracle.gradient(st, gf, gt)
    s = max(np.abs(rp).max(), np.abs(rq).max())
    err = max(np.abs(gp.cpu().numpy() - rp).max(), np.abs(gq.cpu().numpy() - rq).max()) / s
    print("adjoint with walls: max |diff| / max |grad|", err)
    assert err <= 1e-4
    m.close()


def test_walls_with_history_and_friction():
    law = oracle.ContactLaw(restitution=0.5, history=True, friction=True, mu_s=0.5, mu_k=0.3, u_k=0.02)
    st = oblique(W.settling_cubes())
    m = model_for(st, precision=0, history=True, restitution=law.restitution, friction=True, mu_s=law.mu_s,
                  mu_k=law.mu_k, u_k=law.u_k)
    pos, quat = W.pose_sequence(st, 3, seed=3, sigma_x=0.3, sigma_rot=0.02)
    rng = np.random.default_rng(4)
    tr = LawTracker(law, fp64=False)
    hist = None
    for s in range(3):
        vel = np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
        sts = dataclasses.replace(st, pos=pos[s], quat=quat[s])
        g = gpu_step(m, sts, vel=vel)
        rb = oracle.contact_step(sts)
        rx = oracle.contact_step_ext(sts, law, vel=vel, hist=hist)
        forces, tol = tr.step(sts, pos[s], vel, rb, rx, rb)
        print("walls + law", s, compare(sts, g, rb, fp64=False, smooth=False, forces=forces, tol_force=tol))
        hist = (rx.hist_ij, rx.hist_c)
        gij, gc = m.history()
        assert (gij[:, 1] >= st.n).sum() > 10   # wall contacts kept in the history
    # a checkpoint with wall contacts restores into a fresh context
    m2 = model_for(st, precision=0, history=True, restitution=law.restitution, friction=True, mu_s=law.mu_s,
                   mu_k=law.mu_k, u_k=law.u_k)
    m2.set_history(gij, gc)
    hij, hc = m2.history()
    assert np.array_equal(hij, gij) and np.array_equal(hc, gc)
    m2.close()
    m.close()


def test_invalid_walls_refused():
    from paper_2401_10878_gb300.contact import ContactError
    st = W.mixed_grid_27()
    with pytest.raises(ContactError):
        model_for(st, walls=np.array([[0, 0, 2.0, 5.0]]), wall_young=[1.0], wall_poisson=[0.3])   # not unit
    with pytest.raises(ContactError):
        model_for(st, walls=np.array([[0, 0, 1.0, 5.0]]), wall_young=[-1.0], wall_poisson=[0.3])
