"""Pins of the oracle's contact-law extensions (CPU only): the friction of
Eq. (contact_force_tangential) and the contact history of Sec. 4.3.3 (each
contact keeps the damping factor of Eq. (damping_factor) computed from its
approach speed at its first step).

A pair of axis-aligned cubes touching along x with faces on half-integer
nodes has an exactly known overlap (V, d) and normal n = +x, so the forces
can be pinned by limits and ratios that do not restate the formulas."""
import os

import numpy as np
import pytest

import oracle
from tests.helpers import state

H = [4.0, 4.0, 4.0]
CA = np.array([30.5, 31.5, 29.5])
CB = CA + [2 * H[0] - 1.0, 0.0, 0.0]   # penetration 1 along x, no lateral offset


def pair(cb=CB):
    return state([1, 1], [H, H], [CA, cb])


def vel(uA=(0, 0, 0), wA=(0, 0, 0), uB=(0, 0, 0), wB=(0, 0, 0)):
    return np.array([[*uA, *wA], [*uB, *wB]], dtype=float)


def friction(mu_s=0.4, mu_k=0.3, u_k=1e-3):
    return oracle.ContactLaw(mu_s=mu_s, mu_k=mu_k, u_k=u_k, friction=True)


def ft_over_fn(r):
    """(tangential force on B along y) / (normal force on B), pair 0."""
    F = r.pair_out[0, 8:11]
    return F[1] / F[0]


def test_no_extension_matches_base_step():
    st = pair()
    v = vel(uA=(0.1, 0.2, 0.0))
    a = oracle.contact_step(st, vel=v)
    b = oracle.contact_step_ext(st, oracle.ContactLaw(), vel=v)
    assert np.array_equal(a.pair_out, b.pair_out) and np.array_equal(a.force, b.force)


def test_shared_damping_clamped_when_separating_fast():
    """Eq. (contact_force_normal) with (1 + c ddot_n) below zero (A leaving B
    faster than 1/c) gives no force at all, not an attraction; at half the
    threshold speed the force is half the undamped one."""
    st = pair()
    st.damping_c = 0.5
    r0 = oracle.contact_step(st)
    fast = oracle.contact_step(st, vel=vel(uA=(-3.0, 0, 0)))   # 1 + 0.5 (-3) < 0
    half = oracle.contact_step(st, vel=vel(uA=(-1.0, 0, 0)))   # 1 + 0.5 (-1) = 0.5
    assert fast.pair_out[0, 0] > 0 and np.all(fast.pair_out[0, 8:11] == 0.0)
    assert half.pair_out[0, 8] == pytest.approx(0.5 * r0.pair_out[0, 8], rel=1e-14)


def test_friction_kinetic_limit():
    """|u_t| >> u_k: the friction coefficient tends to mu_k."""
    r = oracle.contact_step_ext(pair(), friction(u_k=1e-3), vel=vel(uA=(0, 1e3, 0)))   # a = 1e6
    assert r.pair_out[0, 4:7] == pytest.approx([1, 0, 0], abs=1e-15)
    assert ft_over_fn(r) == pytest.approx(0.3, rel=1e-10)


def test_friction_static_peak_without_kinetic_friction():
    """mu_k = 0 and |u_t| = u_k: the coefficient is exactly mu_s."""
    r = oracle.contact_step_ext(pair(), friction(mu_s=0.25, mu_k=0.0, u_k=0.5), vel=vel(uA=(0, 0.5, 0)))
    assert ft_over_fn(r) == pytest.approx(0.25, rel=1e-14)


def golden():
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "friction_law.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_friction_worked_values():
    """|F_t| / |F_n| at a = 1 and a = 2 for mu_s = 0.4, mu_k = 0.3 (hand-worked values)."""
    g = golden()
    for a, key in ((1.0, "friction_coef_mus0.4_muk0.3_a1"), (2.0, "friction_coef_mus0.4_muk0.3_a2")):
        r = oracle.contact_step_ext(pair(), friction(mu_s=0.4, mu_k=0.3, u_k=0.25), vel=vel(uA=(0, 0.25 * a, 0)))
        assert ft_over_fn(r) == pytest.approx(g[key], rel=1e-13)


def test_friction_vanishes_without_slip():
    r = oracle.contact_step_ext(pair(), friction(u_k=1.0), vel=vel(uA=(0, 1e-6, 0)))   # a = 1e-6
    assert abs(ft_over_fn(r)) < 1e-10
    r = oracle.contact_step_ext(pair(), friction(), vel=vel(uA=(0.2, 0, 0)))   # pure normal approach
    assert r.pair_out[0, 9] == 0.0 and r.pair_out[0, 10] == 0.0


def test_friction_opposes_sliding_and_dissipates():
    """A slides along +y (and spins) relative to B: the friction force on A points
    against A's sliding, B is dragged along; the frictional power is negative."""
    st = pair()
    v = vel(uA=(0, 0.02, 0.01), wA=(0, 0, 0.003), uB=(0, -0.01, 0))
    r = oracle.contact_step_ext(st, friction(), vel=v)
    xc = r.pair_out[0, 1:4]
    F_B = r.pair_out[0, 8:11]
    F_A = -F_B
    uA = v[0, :3] + np.cross(v[0, 3:], xc - CA)
    uB = v[1, :3] + np.cross(v[1, 3:], xc - CB)
    n = r.pair_out[0, 4:7]
    u_t = (uA - uB) - np.dot(uA - uB, n) * n
    ft_A = F_A - np.dot(F_A, n) * n
    assert np.dot(ft_A, u_t) < 0.0
    assert np.allclose(np.cross(ft_A, u_t), 0.0, atol=1e-12 * np.linalg.norm(ft_A) * np.linalg.norm(u_t))
    assert np.dot(F_A, uA - np.dot(uA, n) * n) + np.dot(F_B, uB - np.dot(uB, n) * n) < 0.0


def test_friction_momentum_balance():
    """With friction and spin: sum of forces and of (torque + X x force) vanish."""
    st = pair()
    v = vel(uA=(0.01, 0.03, -0.02), wA=(0.002, -0.001, 0.004), uB=(-0.01, 0.0, 0.01), wB=(0, 0.003, 0))
    r = oracle.contact_step_ext(st, friction(), vel=v)
    assert np.abs(r.force[0] + r.force[1]).max() <= 1e-13 * np.abs(r.force).max()
    X = np.array([CA, CB])
    L = r.torque + np.cross(X, r.force)
    assert np.abs(L.sum(axis=0)).max() <= 1e-12 * np.abs(np.cross(X, r.force)).max()


def _ratio(law, v, hist=None, cb=CB):
    """Normal force with the law over the undamped normal force; the new history."""
    st = pair(cb)
    r = oracle.contact_step_ext(st, law, vel=v, hist=hist)
    r0 = oracle.contact_step_ext(st, oracle.ContactLaw(), vel=v)
    if r0.n_pairs == 0 or r0.pair_out[0, 0] == 0.0:
        return None, (r.hist_ij, r.hist_c)
    return r.pair_out[0, 8] / r0.pair_out[0, 8], (r.hist_ij, r.hist_c)


def test_history_first_step_damping_is_independent_of_u0():
    """At a contact's first step c = c(e, u0) and the damping multiplier is
    1 + c u0 = 1 + c(e, 1) for every approach speed u0 (Eq. damping_factor scales as 1/u0)."""
    e = 0.926
    law = oracle.ContactLaw(restitution=e, history=True)
    k1 = oracle.damping_factor(e, 1.0)
    for u0 in (0.05, 0.3, 2.0):
        ratio, (hij, hc) = _ratio(law, vel(uA=(u0, 0, 0)))
        assert ratio == pytest.approx(1.0 + k1, rel=1e-13)
        assert hij.tolist() == [[0, 1]] and hc[0] == pytest.approx(oracle.damping_factor(e, u0), rel=1e-14)


def test_history_keeps_c_until_the_contact_ends():
    e = 0.5
    law = oracle.ContactLaw(restitution=e, history=True)
    u0, u1, u2 = 0.2, 0.05, 0.7
    ratio0, h = _ratio(law, vel(uA=(u0, 0, 0)))
    c0 = h[1][0]
    # next step, another approach speed: the contact keeps c0
    ratio1, h = _ratio(law, vel(uA=(u1, 0, 0)), hist=h)
    assert ratio1 == pytest.approx(1.0 + c0 * u1, rel=1e-13) and h[1][0] == c0
    # the cubes separate: the contact ends
    ratio2, h = _ratio(law, vel(uA=(u1, 0, 0)), hist=h, cb=CB + [3.0, 0, 0])
    assert ratio2 is None and len(h[0]) == 0
    # a new contact takes c from its own approach speed
    ratio3, h = _ratio(law, vel(uA=(u2, 0, 0)), hist=h)
    assert ratio3 == pytest.approx(1.0 + oracle.damping_factor(e, 1.0), rel=1e-13)
    assert h[1][0] == pytest.approx(oracle.damping_factor(e, u2), rel=1e-14)


def test_history_contact_starting_apart_keeps_no_damping():
    """u0 <= 0 at the first step gives c = 0, kept while the contact lasts."""
    law = oracle.ContactLaw(restitution=0.3, history=True)
    ratio0, h = _ratio(law, vel(uA=(-0.1, 0, 0)))
    assert ratio0 == 1.0 and h[1][0] == 0.0
    ratio1, h = _ratio(law, vel(uA=(0.4, 0, 0)), hist=h)
    assert ratio1 == 1.0 and h[1][0] == 0.0


def test_gradient_ext_without_extensions_is_the_base_gradient():
    from paper_2401_10878_gb300 import workloads as W
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width = 1, 1.0
    gf, gt = W.loss_weights(st.n)
    a = oracle.gradient(st, gf, gt)
    b = oracle.gradient_ext(st, oracle.ContactLaw(), gf, gt)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_gradient_ext_friction_and_fixed_c_match_central_differences():
    """Friction and each contact's c held fixed (every contact found in the
    table): the forward-mode gradient equals central differences of the
    oracle's forward map with that table as the previous step's contacts."""
    from paper_2401_10878_gb300 import workloads as W
    st = W.mixed_grid_27()
    st.indicator, st.smooth_width = 1, 1.0
    rng = np.random.default_rng(21)
    v = np.concatenate([rng.normal(size=(st.n, 3)) * 0.05, rng.normal(size=(st.n, 3)) * 0.01], axis=1)
    law = oracle.ContactLaw(restitution=0.5, history=True, friction=True, mu_s=0.5, mu_k=0.3, u_k=0.05)
    r0 = oracle.contact_step_ext(st, law, vel=v)
    table = (r0.hist_ij, r0.hist_c)
    assert len(table[1]) > 20 and np.count_nonzero(table[1]) > 5
    gf, gt = W.loss_weights(st.n)
    gp, gq = oracle.gradient_ext(st, law, gf, gt, vel=v, table=table)

    def loss(pos, quat):
        r = oracle.contact_step_ext(st, law, pos=pos, quat=quat, vel=v, hist=table)
        return float(np.sum(gf * r.force) + np.sum(gt * r.torque))

    h = 1e-4
    fp = np.zeros_like(gp)
    fq = np.zeros_like(gq)
    for p in range(st.n):
        for k in range(3):
            a, b = st.pos.copy(), st.pos.copy()
            a[p, k] += h
            b[p, k] -= h
            fp[p, k] = (loss(a, st.quat) - loss(b, st.quat)) / (2 * h)
        for k in range(4):
            a, b = st.quat.copy(), st.quat.copy()
            a[p, k] += h
            b[p, k] -= h
            fq[p, k] = (loss(st.pos, a) - loss(st.pos, b)) / (2 * h)
    g = np.concatenate([gp.ravel(), gq.ravel()])
    f = np.concatenate([fp.ravel(), fq.ravel()])
    scale = np.abs(g).max()
    assert scale > 0
    err = np.abs(g - f) / scale
    assert np.mean(err < 1e-4) >= 0.98, np.sort(err)[-10:]
    assert np.median(err) < 1e-6
    # friction changes the gradient (the test is not blind to it)
    g0 = oracle.gradient_ext(st, oracle.ContactLaw(restitution=0.5, history=True), gf, gt, vel=v, table=table)
    assert np.abs(g0[0] - gp).max() > 1e-3 * scale
