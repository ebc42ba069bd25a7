"""CUDA box pipeline (the paper's rough detection, box correction and N_c^3
sampling, Sec. 3.3.1) vs the oracle's (needs a GB300).

The rough box and the corrected box are reproduced exactly unless the oracle
reports a node within eps of the rough threshold or two nearest lines of a
face within 1e-4 dx (those pairs are flagged); the sample counts are then
exact and the sample volume agrees to FP64 rounding, so the tolerances are
the lattice path's (tests/parity.py) with the sample volume as the unit.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.parity import compare, gpu_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def boxed(st, nc=8):
    st = dataclasses.replace(st)
    st.box_mode, st.contact_resolution = 1, nc
    return st


def run(st, vel=None):
    from paper_2401_10878_gb300.contact import Contact
    m = Contact.from_state(st)
    g = gpu_step(m, st, vel=vel)
    r = oracle.contact_step(st, vel=vel)
    rough, box, flags = oracle.box_pipeline(st)
    nc = st.contact_resolution
    dV = np.prod((box[:, 3:] - box[:, :3]) / nc, axis=1)
    ext = (box[:, 3:] - box[:, :3]).min(axis=1)
    rep = compare(st, g, r, fp64=False, smooth=st.indicator == 1,
                  box=(dV, (flags[:, 0] > 0) | (flags[:, 1] > 0), ext))
    m.close()
    return rep, r


@pytest.mark.parametrize("nc", [4, 8, 16])
def test_mixed27_box_pipeline(nc):
    rep, r = run(boxed(W.mixed_grid_27(), nc))
    print("mixed27 box", nc, rep)
    assert np.count_nonzero(r.pair_out[:, 0]) > 20


def test_elongated_cuboids_box_pipeline():
    """Cuboids of unequal half extents (7, 5, 4) with spheres: the pair
    builder's cut of two boxes' node box and the FP64 re-clip with per-axis
    extents."""
    rep, r = run(boxed(W.mixed_grid_27(cuboid_half=(7.0, 5.0, 4.0))))
    print("mixed27 cuboids box", rep)
    assert rep.pairs > 40


def test_cubes400_box_pipeline():
    rep, _ = run(boxed(W.settling_cubes()))
    print("cubes400 box", rep)


def test_mixed1934_box_pipeline_full_size():
    rep, r = run(boxed(W.mixed_settling()))
    print("mixed1934 box", rep)
    assert np.count_nonzero(r.pair_out[:, 0]) > 300


def test_cubes1934_walls_box_pipeline():
    st = boxed(W.floor_and_ceiling(W.settling_cubes_dense()))
    rep, r = run(st)
    print("cubes1934 + walls box", rep)
    assert (r.pair_ij[:, 1] >= st.n).sum() > 50


def test_smoothed_box_pipeline_with_damping():
    st = boxed(W.mixed_grid_27())
    st.indicator, st.smooth_width, st.damping_c = 1, 1.0, 0.3
    rng = np.random.default_rng(2)
    vel = np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
    rep, _ = run(st, vel)
    print("mixed27 smooth box + damping", rep)


def test_box_pipeline_refuses_backward():
    from paper_2401_10878_gb300.contact import ESTATE, Contact, ContactError
    st = boxed(W.mixed_grid_27())
    st.indicator = 1
    m = Contact.from_state(st)
    gpu_step(m, st)
    z = torch.zeros((st.n, 3), dtype=torch.float64, device=m.device)
    with pytest.raises(ContactError) as e:
        m.backward(z, z)
    assert e.value.code == ESTATE
    m.close()


def test_box_pipeline_history_friction_and_warm_start():
    """Four steps of cubes400 between a floor and a ceiling with the box
    pipeline, the contact history (each contact's c and its corrected box as
    the next correction's warm start, Sec. 4.3.3) and friction: geometry,
    forces, the contact list, each c and each stored box against the oracle;
    a pair the oracle flags at one step may take another box on the GPU, so
    it is reported, not asserted, for as long as the contact lasts.  Then a
    checkpoint (contacts, c, boxes) restored into a fresh context steps
    exactly like the original."""
    from paper_2401_10878_gb300.contact import Contact
    from tests.law_parity import LawTracker
    from tests.test_gpu_contact_law import check_history
    law = oracle.ContactLaw(restitution=0.5, history=True, friction=True, mu_s=0.5, mu_k=0.3, u_k=0.02)
    st = boxed(W.floor_and_ceiling(W.settling_cubes()))
    kw = dict(history=True, restitution=law.restitution, friction=True, mu_s=law.mu_s, mu_k=law.mu_k, u_k=law.u_k)
    m = Contact.from_state(st, **kw)
    steps = 4
    pos, quat = W.pose_sequence(st, steps + 1, seed=5, sigma_x=0.3, sigma_rot=0.02)
    rng = np.random.default_rng(6)
    vels = [np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
            for _ in range(steps + 1)]
    tr = LawTracker(law, fp64=False)
    hist = None
    warm = 0
    for s in range(steps):
        sts = dataclasses.replace(st, pos=pos[s], quat=quat[s])
        g = gpu_step(m, sts, vel=vels[s])
        rb = oracle.contact_step(sts, hist=hist)
        rx = oracle.contact_step_ext(sts, law, vel=vels[s], hist=hist)
        _, box, flags = oracle.box_pipeline(sts, hist=hist)
        keys = [tuple(k) for k in rb.pair_ij.tolist()]
        carried = np.array([k in tr.tainted for k in keys], bool)
        nc = st.contact_resolution
        dV = np.prod((box[:, 3:] - box[:, :3]) / nc, axis=1)
        ext = (box[:, 3:] - box[:, :3]).min(axis=1)
        flag = (flags[:, 0] > 0) | (flags[:, 1] > 0) | carried
        forces, tol_force = tr.step(sts, pos[s], vels[s], rb, rx, rb)
        rep = compare(sts, g, rb, fp64=False, smooth=False, forces=forces, tol_force=tol_force,
                      box=(dV, flag, ext))
        print("cubes400 + walls box, history, friction", s, rep, "carried", int(carried.sum()))
        if hist is not None:
            warm += len(set(map(tuple, hist[0].tolist())) & set(keys))
        hist = (rx.hist_ij, rx.hist_c, rx.hist_box)
        check_history(m, rx, tr)
        gij, gc, gbox = m.history(boxes=True)
        ob = {tuple(k): b for k, b in zip(rx.hist_ij.tolist(), rx.hist_box)}
        for k, b in zip(gij.tolist(), gbox):
            if tuple(k) in ob and tuple(k) not in tr.tainted:
                assert np.allclose(b, ob[tuple(k)], rtol=0, atol=1e-9), (k, b, ob[tuple(k)])
        assert (gij[:, 1] >= st.n).sum() > 5   # wall contacts in the history
    assert warm > 100   # contacts that went through a warm start
    # checkpoint: a fresh context with the saved contacts steps like the original
    gij, gc, gbox = m.history(boxes=True)
    m2 = Contact.from_state(st, **kw)
    m2.set_history(gij, gc, gbox)
    sts = dataclasses.replace(st, pos=pos[steps], quat=quat[steps])
    g1 = gpu_step(m, sts, vel=vels[steps])
    g2 = gpu_step(m2, sts, vel=vels[steps])
    for key in ("pair_ij", "pair_out", "force", "torque"):
        assert np.array_equal(g1[key], g2[key]), key
    with pytest.raises(Exception):
        m2.set_history(gij, gc)   # the box pipeline's history needs the boxes
    m2.close()
    m.close()
