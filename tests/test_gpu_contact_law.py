"""CUDA contact law extensions vs the oracle (needs a GB300): friction of
Eq. (contact_force_tangential) and the contact history of Sec. 4.3.3 (each
contact keeps the damping factor of Eq. (damping_factor) from its first
step), over sequences of steps in which contacts begin and end; the history
API (read, checkpoint restore, reset); the adjoint with damping, friction
and each contact's c held fixed, against the oracle's dual-number gradient.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2401_10878_gb300 import workloads as W
from tests.law_parity import LawTracker
from tests.parity import compare, gpu_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAW = oracle.ContactLaw(restitution=0.5, history=True, friction=True, mu_s=0.5, mu_k=0.3, u_k=0.02)


def model_for(st, law, precision):
    from paper_2401_10878_gb300.contact import Contact
    return Contact.from_state(st, precision=precision, history=law.history, restitution=law.restitution,
                              friction=law.friction, mu_s=law.mu_s, mu_k=law.mu_k, u_k=law.u_k)


def velocities(rng, n, v=0.05, w=0.01):
    return np.concatenate([rng.normal(size=(n, 3)) * v, rng.normal(size=(n, 3)) * w], axis=1)


def run_sequence(st, law, precision, steps, sigma_x, seed=5):
    m = model_for(st, law, precision)
    pos, quat = W.pose_sequence(st, steps, seed=seed, sigma_x=sigma_x, sigma_rot=0.02)
    rng = np.random.default_rng(seed + 1)
    tr = LawTracker(law, fp64=precision == 1)
    hist = None
    reps = []
    for s in range(steps):
        vel = velocities(rng, st.n)
        sts = dataclasses.replace(st, pos=pos[s], quat=quat[s])
        g = gpu_step(m, sts, vel=vel)
        rb = oracle.contact_step(sts)                       # geometry; undamped forces
        rx = oracle.contact_step_ext(sts, law, vel=vel, hist=hist)
        forces, tol_force = tr.step(sts, pos[s], vel, rb, rx, rb)
        reps.append(compare(sts, g, rb, fp64=precision == 1, smooth=st.indicator == 1, forces=forces,
                            tol_force=tol_force))
        hist = (rx.hist_ij, rx.hist_c)
        if law.history:
            check_history(m, rx, tr)
    m.close()
    return reps, tr


def check_history(m, rx, tr):
    """The context's contact list equals the oracle's (up to contacts the
    comparison skips), each c within its carried relative uncertainty."""
    gij, gc = m.history()
    g = {tuple(k): c for k, c in zip(gij.tolist(), gc)}
    o = {tuple(k): c for k, c in zip(rx.hist_ij.tolist(), rx.hist_c)}
    for k in set(g) ^ set(o):
        assert k in tr.tainted, f"contact {k} on one side only"
    for k in set(g) & set(o):
        if k in tr.tainted:
            continue
        tol = (2.0 * tr.rho_c.get(k, 0.0) + 1e-12) * abs(o[k])
        assert abs(g[k] - o[k]) <= tol, (k, g[k], o[k], tol)
    key = gij[:, 0].astype(np.int64) * (1 << 31) + gij[:, 1]
    assert np.all(np.diff(key) > 0), "history rows not sorted"


@pytest.mark.parametrize("precision", [1, 0])
def test_mixed27_history_and_friction_sequence(precision):
    reps, tr = run_sequence(W.mixed_grid_27(), LAW, precision, steps=8, sigma_x=0.4)
    for r in reps:
        print("mixed27", precision, r)


@pytest.mark.parametrize("precision", [0, 1])
def test_cubes400_history_and_friction_sequence(precision):
    reps, _ = run_sequence(W.settling_cubes(), LAW, precision, steps=4, sigma_x=0.3)
    for r in reps:
        print("cubes400", precision, r)


def test_mixed1934_full_size_sequence():
    reps, tr = run_sequence(W.mixed_settling(), LAW, 0, steps=3, sigma_x=0.2)
    for r in reps:
        print("mixed1934", r)
    print("skipped contacts", len(tr.tainted))


def test_cubes1934_smoothed_sequence():
    st = W.settling_cubes_dense()
    st.indicator, st.smooth_width = 1, 1.0
    reps, _ = run_sequence(st, LAW, 0, steps=2, sigma_x=0.2)
    for r in reps:
        print("cubes1934 smooth", r)


def test_friction_only_with_shared_damping():
    st = W.mixed_grid_27()
    st.damping_c = 0.3
    law = dataclasses.replace(LAW, history=False)
    reps, _ = run_sequence(st, law, 1, steps=3, sigma_x=0.4)
    for r in reps:
        print("friction only", r)


def test_history_only_without_velocities():
    """No velocities: no damping and no friction; the contacts are still
    recorded (with c = 0) and the forces equal the plain step's."""
    st = W.mixed_grid_27()
    m = model_for(st, LAW, 1)
    g = gpu_step(m, st)
    r = oracle.contact_step(st)
    print("no vel", compare(st, g, r, fp64=True, smooth=False))
    ij, c = m.history()
    rx = oracle.contact_step_ext(st, LAW)
    assert np.array_equal(ij, rx.hist_ij) and np.all(c == 0.0)
    m.close()


def test_history_checkpoint_restore_and_reset():
    """A context resumed from another's history gives the same step bit for
    bit; after a reset every contact is new again."""
    st = W.mixed_grid_27()
    pos, quat = W.pose_sequence(st, 3, seed=8, sigma_x=0.3)
    rng = np.random.default_rng(9)
    vels = [velocities(rng, st.n) for _ in range(3)]
    a = model_for(st, LAW, 0)
    for s in range(2):
        gpu_step(a, dataclasses.replace(st, pos=pos[s], quat=quat[s]), vel=vels[s])
    ij, c = a.history()
    assert len(c) > 10 and np.count_nonzero(c) > 3
    b = model_for(st, LAW, 0)
    b.set_history(ij, c)
    s2 = dataclasses.replace(st, pos=pos[2], quat=quat[2])
    ga = gpu_step(a, s2, vel=vels[2])
    gb = gpu_step(b, s2, vel=vels[2])
    for k in ("pair_out", "force", "torque"):
        assert np.array_equal(ga[k], gb[k]), k
    # reset: the step equals the oracle's with no previous contacts
    b.reset_history()
    g = gpu_step(b, s2, vel=vels[2])
    rx = oracle.contact_step_ext(s2, LAW, vel=vels[2])
    rb = oracle.contact_step(s2)
    forces, tol = LawTracker(LAW, fp64=False).step(s2, pos[2], vels[2], rb, rx, rb)
    print("after reset", compare(s2, g, rb, fp64=False, smooth=False, forces=forces, tol_force=tol))
    # invalid rows are refused
    from paper_2401_10878_gb300.contact import ContactError
    with pytest.raises(ContactError):
        b.set_history(np.array([[3, 2]]), np.array([0.1]))
    with pytest.raises(ContactError):
        b.set_history(np.array([[1, 2], [1, 2]]), np.array([0.1, 0.2]))
    a.close()
    b.close()


def adjoint_case(law, damping_c=0.0, seed=12):
    """Two steps (the second's contacts partly ongoing), then the backward;
    returns the GPU gradient, the oracle's (the step's own contact list as
    the table of fixed c), and its scale."""
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width, st.damping_c = 1, 1.0, damping_c
    m = model_for(st, law, 0)
    rng = np.random.default_rng(seed)
    pos, quat = W.pose_sequence(st, 2, seed=seed + 1, sigma_x=0.3)
    vels = [velocities(rng, st.n) for _ in range(2)]
    hist = None
    dev = m.device
    for s in range(2):
        sts = dataclasses.replace(st, pos=pos[s], quat=quat[s])
        # the step's inputs stay alive until the backward (it reads them)
        inputs = [torch.tensor(x, dtype=torch.float64, device=dev) for x in (pos[s], quat[s], vels[s])]
        m.step(*inputs)
        rx = oracle.contact_step_ext(sts, law, vel=vels[s], hist=hist)
        hist = (rx.hist_ij, rx.hist_c)
    gf, gt = W.loss_weights(st.n)
    gp, gq = m.backward(torch.tensor(gf, device=dev), torch.tensor(gt, device=dev))
    op, oq = oracle.gradient_ext(sts, law, gf, gt, vel=vels[1], table=hist)
    m.close()
    scale = max(np.abs(op).max(), np.abs(oq).max())
    err = max(np.abs(gp.cpu().numpy() - op).max(), np.abs(gq.cpu().numpy() - oq).max()) / scale
    other = oracle.gradient(sts, gf, gt, vel=vels[1])   # shared c, no friction
    diff = np.abs(other[0] - op).max() / scale
    return err, diff


def test_adjoint_with_shared_damping():
    err, _ = adjoint_case(dataclasses.replace(LAW, history=False, friction=False), damping_c=0.3)
    print("adjoint, shared damping: max err / scale", err)
    assert err <= 1e-4   # the adjoint's tolerance without velocities (FP32 node sweep)


def test_adjoint_with_history_holds_c_fixed():
    err, diff = adjoint_case(dataclasses.replace(LAW, friction=False))
    print("adjoint with history: max err / scale", err, "| shared-c gradient differs by", diff)
    assert err <= 1e-4
    assert diff > 1e-2   # the per-contact c matters


def test_adjoint_with_friction_and_history():
    err, diff = adjoint_case(LAW)
    print("adjoint with friction and history: max err / scale", err, "| without friction differs by", diff)
    assert err <= 1e-4
    assert diff > 1e-2
