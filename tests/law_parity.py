"""Force tolerances of the contact-law extensions (friction of Eq.
(contact_force_tangential), contact history with the damping factor of Eq.
(damping_factor)) for the CUDA-vs-oracle comparison.

The geometry (V, x_c, n, d) carries the tolerances of tests/parity.py; the
law maps them to the force with a sensitivity that the oracle's own values
bound, pair by pair:
  * u_AB, the relative velocity at x_c, moves by |w_A - w_B| dx_c; its normal
    part ddot_n by |u_AB| dn + that; its tangential part u_t by 2 |u_AB| dn +
    that.
  * damping 1 + c ddot_n: c is a constant of the contact, known to the
    relative accuracy of the approach speed u0 it came from; at a contact's
    first step c ddot_n = K exactly (no sensitivity).  A contact that began
    with |u0| within ten times its uncertainty may take c = 0 on one side and
    K / u0 on the other: it is skipped (reported, not asserted) for as long as
    it lasts.
  * friction |F_t| = f(a) |F_n| t, a = |u_t| / u_k: the direction t moves by
    du_t / |u_t| (at most 2), f by its largest slope over a +- da.
"""
from __future__ import annotations

import numpy as np

import oracle


def friction_coef(a, mu_s, mu_k):
    ms = mu_s * (1.0 - 0.09 * (mu_k / mu_s) ** 4)
    a2 = a * a
    return (2 * ms - mu_k) * a2 / (a2 * a2 + 1) + mu_k - mu_k / (a2 + 1)


def friction_slope_bound(a, da, mu_s, mu_k):
    """max |f'| over [a - da, a + da] (sampled finely; f' is smooth)."""
    ms = mu_s * (1.0 - 0.09 * (mu_k / mu_s) ** 4)
    A = 2 * ms - mu_k
    lo = np.maximum(a - da, 0.0)
    hi = a + da
    t = np.linspace(0.0, 1.0, 65)[None, :]
    x = lo[:, None] + (hi - lo)[:, None] * t
    fp = A * 2 * x * (1 - x ** 4) / (x ** 4 + 1) ** 2 + 2 * mu_k * x / (x * x + 1) ** 2
    return np.abs(fp).max(axis=1) * 1.05


class LawTracker:
    """Carries, across steps, each contact's relative uncertainty of c and
    the contacts to skip; builds each step's force tolerance."""

    def __init__(self, law: oracle.ContactLaw, fp64: bool):
        self.law = law
        self.rel = 1e-9 if fp64 else 1e-5
        self.rho_c = {}      # (i, j) -> relative uncertainty of the contact's c
        self.tainted = set()
        self.K = oracle.damping_factor(law.restitution, 1.0) if law.history else 0.0

    def step(self, st, pos, vel, r_base, r_ext, r_undamped):
        """(forces, tol_force) for tests.parity.compare; tol_force returns the
        per-pair tolerance and the pairs to report without asserting."""
        law = self.law
        ij = r_ext.pair_ij
        P = len(ij)
        o = r_ext.pair_out
        V, xc, n, d = o[:, 0], o[:, 1:4], o[:, 4:7], o[:, 7]
        F = o[:, 8:11]
        Fn = np.linalg.norm(F, axis=1)
        fmag0 = np.linalg.norm(r_undamped.pair_out[:, 8:11], axis=1)   # undamped, no friction
        nw = len(getattr(st, "walls", ()))   # partners j >= n are walls: at the origin, at rest
        pos_w = np.concatenate([pos, np.zeros((nw, 3))])
        vel_w = np.concatenate([vel, np.zeros((nw, 6))])
        XA = pos_w[ij[:, 0]]
        XB = pos_w[ij[:, 1]] - r_base.pair_shift * st.box
        vA, vB = vel_w[ij[:, 0]], vel_w[ij[:, 1]]
        uab = (vA[:, :3] + np.cross(vA[:, 3:], xc - XA)) - (vB[:, :3] + np.cross(vB[:, 3:], xc - XB))
        wrel = np.linalg.norm(vA[:, 3:] - vB[:, 3:], axis=1)
        ddot = np.einsum("pk,pk->p", uab, n)
        utn = np.linalg.norm(uab - ddot[:, None] * n, axis=1)
        uabn = np.linalg.norm(uab, axis=1)
        c = r_ext.pair_c
        keys = [(int(a), int(b)) for a, b in ij]
        contact = V > 0
        new = np.array([law.history and contact[p] and keys[p] not in self.rho_c for p in range(P)], bool)
        rho_c = np.array([self.rho_c.get(k, 0.0) for k in keys])

        def tol_force(toln, tolx, tolV, told, flagged):
            dn = np.sqrt(3.0) * toln
            dxc = np.sqrt(3.0) * tolx
            duab = wrel * dxc
            dddot = uabn * dn + duab
            # damping 1 + c ddot_n, clamped at 0; at a contact's first step c ddot_n = K
            damp = np.maximum(0.0, 1.0 + c * ddot)
            ddamp = np.where(new, 1e-13 * (1.0 + np.abs(c * ddot)), np.abs(c) * (dddot + rho_c * np.abs(ddot)))
            geom = self.rel + 0.5 * tolV / np.maximum(V, 1e-300) + 0.5 * told / np.maximum(d, 1e-300)
            fmag = fmag0 * damp
            dfmag = fmag0 * (damp * geom + ddamp)
            tol = dfmag + (fmag + dfmag) * dn + self.rel * Fn
            if law.friction:
                a = utn / law.u_k
                dut = duab + 2.0 * uabn * dn
                coef = friction_coef(a, law.mu_s, law.mu_k)
                dcoef = friction_slope_bound(a, dut / law.u_k, law.mu_s, law.mu_k) * dut / law.u_k
                dt = np.where(utn > 0, np.minimum(2.0, dut / np.maximum(utn, 1e-300)), 2.0)
                tol = tol + coef * dfmag + (fmag + dfmag) * (dcoef + coef * dt)
            tol = np.where(fmag0 > 0, tol, 0.0)
            # a contact that began with |u0| within ten times its uncertainty
            # may take c = 0 on one side and K / u0 on the other
            if self.K > 0:
                for p in np.nonzero(new & (np.abs(ddot) < 10.0 * dddot))[0]:
                    self.tainted.add(keys[p])
            # a flagged pair may be a contact (V > 0) on one side only, so the
            # two histories may differ for it from here on
            if law.history:
                for p in np.nonzero(flagged)[0]:
                    self.tainted.add(keys[p])
            skip = np.array([k in self.tainted for k in keys], bool) & contact
            rho = {}
            for p in np.nonzero(contact)[0]:
                if law.history:
                    rho[keys[p]] = dddot[p] / max(abs(ddot[p]), 1e-300) if new[p] else rho_c[p]
            self.rho_c = rho
            self.tainted &= set(rho) | {keys[p] for p in np.nonzero(flagged)[0]}
            return tol, skip

        return (F, r_ext.force, r_ext.torque), tol_force
