"""The checked build (libcontact_checks.so, -DCONTACT_CHECKS; needs a GB300).

Every index the kernels read from a device list (bin, candidate, partner,
pair, tile and overlap-list entries) is tested against its array in that
build; a failure sets the sticky error word to CONTACT_EBOUNDS and the access
is skipped.  Here the checked build runs every kernel variant -- the node
sweep's three kind sets in both indicators, the force law with and without
velocities, the particle sums, the adjoint, the all-FP64 form, the box
pipeline, walls and the contact history -- and must (a) report no error and
(b) give the outputs of the normal build bit for bit (the checks add no
arithmetic).  The self-test entry point shows that a failed check reaches
contact_check as CONTACT_EBOUNDS in the checked build and compiles away in the
normal one.
"""
import numpy as np
import pytest

from paper_2401_10878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(st, checks, steps=2, vel=None, backward=False, **kw):
    from paper_2401_10878_gb300.contact import Contact
    m = Contact.from_state(st, checks=checks, **kw)
    seq_p, seq_q = W.pose_sequence(st, steps)
    outs = []
    for k in range(steps):
        pos = torch.tensor(seq_p[k], device="cuda")
        quat = torch.tensor(seq_q[k], device="cuda")
        v = None if vel is None else torch.tensor(vel, device="cuda")
        r = m.step(pos, quat, v)
        o = {key: r[key].cpu().numpy() for key in ("pair_ij", "pair_out", "force", "torque")}
        if backward:
            gf, gt = W.loss_weights(st.n)
            gp, gq = m.backward(torch.tensor(gf, device="cuda"), torch.tensor(gt, device="cuda"))
            o["gpos"], o["gquat"] = gp.cpu().numpy(), gq.cpu().numpy()
        outs.append(o)
    assert m.lib.contact_check(m.ctx) == 0, m.lib.contact_last_error(m.ctx).decode()
    m.close()
    return outs


def _cases():
    c = {}
    st = W.mixed_grid_27()
    st.indicator = 0
    c["mixed27_sharp"] = (st, {})
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width = 1, 1.0
    c["mixed27_smooth_backward"] = (st, dict(backward=True))
    st = W.settling_cubes_dense()
    st.indicator = 0
    c["cubes1934_sharp"] = (st, {})
    st = W.settling_cubes_dense()
    st.indicator, st.smooth_width = 1, 1.0
    c["cubes1934_smooth_backward"] = (st, dict(backward=True))
    st = W.mixed_settling()
    st.indicator = 0
    c["mixed1934_sharp"] = (st, {})
    st = W.mixed_grid_27()
    st.indicator = 0
    c["mixed27_fp64_form"] = (st, dict(precision=1))
    st = W.mixed_grid_27(cuboid_half=(7.0, 5.0, 4.0))
    st.indicator = 0
    c["mixed27_elongated_cuboids"] = (st, {})
    st = W.settling_cubes()
    st.indicator = 0
    st.box_mode, st.contact_resolution = 1, 8
    c["cubes400_box_pipeline"] = (st, {})
    st = W.floor_and_ceiling(W.settling_cubes())
    st.indicator = 0
    c["cubes400_walls"] = (st, {})
    st = W.mixed_grid_27()
    st.indicator = 0
    rng = np.random.default_rng(3)
    vel = np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
    c["mixed27_history_friction"] = (st, dict(vel=vel, history=True, restitution=0.5, friction=True, mu_s=0.5,
                                              mu_k=0.3, u_k=0.02))
    return c


CASES = _cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_checked_build_reports_nothing_and_matches(name):
    st, kw = CASES[name]
    ref = _run(st, False, **kw)
    chk = _run(st, True, **kw)
    for a, b in zip(ref, chk):
        assert a.keys() == b.keys()
        for key in a:
            assert np.array_equal(a[key], b[key]), (name, key)


def test_failed_check_reaches_contact_check():
    from paper_2401_10878_gb300.contact import EBOUNDS, Contact
    st = W.mixed_grid_27()
    for checks, expect in ((False, 0), (True, EBOUNDS)):
        m = Contact.from_state(st, checks=checks)
        assert m.lib.contact_bounds_selftest(m.ctx) == expect
        assert m.lib.contact_check(m.ctx) == expect   # sticky
        m.lib.contact_clear_error(m.ctx)
        assert m.lib.contact_check(m.ctx) == 0
        # the context stays usable
        out = m.step(torch.tensor(st.pos, device="cuda"), torch.tensor(st.quat, device="cuda"))
        assert out["n_pairs"] > 0
        m.close()
