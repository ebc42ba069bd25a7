// FP64 force law of one overlapping pair (Sec. 2.3 Eq. (contact_force_normal),
// Sec. 2.2 torques, Sec. 3.3.1 contact point, normal and indentation depth),
// run by a node-sweep warp for up to eight overlapping pairs it has completed.
//
// Every FP64 warp instruction occupies a sub-partition's FP64 pipe for ~64
// cycles however many lanes are active, so each pair's chain is split over
// four lanes (component k = 0..2 on lanes 0..2, lane 3 for the fourth
// reciprocal square root) and eight pairs share one pass.  Lanes of unused
// slots run the same instructions on pair 0 and store nothing.
#pragma once

#include "contact_dev.cuh"

namespace gbc {

// Everything the force law reads or writes, as plain pointers and scalars.
struct ForceArgs {
  const double* X;
  const double* R;
  const int* type;
  const double* param;
  const int* face_off;
  const double* planes;
  const double* compl_;
  const double* vel;
  double* pair_out;
  double* ft;
  double* tape;
  double L[3];
  double dx, dx3, gscale, g_min2, inflate, damping_c;
  int n;                 // particles: a partner j >= n is wall j - n (at rest, fallback normal -m)
  const double* rest6;   // [6] zeros, the velocity of a wall
  // contact history (Sec. 4.3.3): last step's contacts of each particle i
  // (partner j, damping factor c) are read from *_rd, this step's go to *_wr
  int history, friction, hist_cap;
  const int* hn_rd;
  const int* hj_rd;
  const double* hc_rd;
  int* hn_wr;
  int* hj_wr;
  double* hc_wr;
  double damp_K;                    // c = damp_K / u0 for a contact's first step
  double mu_s_star, mu_k, inv_u_k;  // friction law of Eq. (contact_force_tangential)
};

namespace fl {

constexpr unsigned kFull = 0xffffffffu;

// 1/sqrt(a) for a > 0: FP32 seed (the double's leading 24 bits, rsqrt.approx)
// and two Newton-Raphson steps y <- y + y (1 - a y^2) / 2 in FP64 (each step
// squares the relative error: 2^-22 -> ~1e-13 -> FP64 rounding).  Arguments
// outside the FP32 exponent range take the library square root.
__device__ __forceinline__ double nr_rsqrt(double a) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(a));
  const unsigned lo = static_cast<unsigned>(__double2loint(a));
  const int e = static_cast<int>((hi >> 20) & 0x7ffu) - 896;
  if (e < 1 || e > 254 || (hi >> 31)) return 1.0 / sqrt(a);
  const float af = __uint_as_float((static_cast<unsigned>(e) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  float yf;
  asm("rsqrt.approx.f32 %0, %1;" : "=f"(yf) : "f"(af));
  double y = widen(yf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double h = a * y;
    const double r = fma(-h, y, 1.0);
    y = fma(0.5 * y, r, y);
  }
  return y;
}

// max of two doubles by their order-preserving integer keys (no FP64 instruction)
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dmax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }

// Exact int -> FP64 conversion with integer operations (|v| < 2^31).
__device__ __forceinline__ double int_to_double(int v) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ULL << 63) : 0ULL;
  const unsigned a = v < 0 ? 0u - static_cast<unsigned>(v) : static_cast<unsigned>(v);
  const int lz = __clz(a);
  const unsigned long long frac = (static_cast<unsigned long long>(a) << (lz + 21)) & ((1ULL << 52) - 1ULL);
  return __longlong_as_double(static_cast<long long>(sgn | (static_cast<unsigned long long>(1054 - lz) << 52) | frac));
}

// SET 2 (cubes only) compiles out every type but the cuboid (walls are
// one-plane polytopes, so the other kind sets keep every branch).
template <int SET>
__device__ __forceinline__ double shape_value(int type, double prm0, double prmk, const double* planes, int nf, int k,
                                              const double r[3], const double y[3], double yk) {
  if (SET != 2 && type == 0) {   // sphere: |r| - radius (the same on the pair's lanes)
    const double rr = fma(r[2], r[2], fma(r[1], r[1], r[0] * r[0]));
    const double nr = __double_as_longlong(rr) > 0 ? rr * nr_rsqrt(rr) : 0.0;
    return nr - prm0;
  }
  if (SET == 2 || type == 1) return fabs(yk) - prmk;   // cuboid: this lane's face pair
  double best = -1e300;                          // polytope: faces k, k + 3, ... (loads 4 faces at a time)
  const double2* pl = reinterpret_cast<const double2*>(planes);
  for (int f0 = k; f0 < nf; f0 += 12) {
    double2 e01[4], e23[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int f = min(f0 + 3 * u, nf - 1);
      e01[u] = pl[2 * f];
      e23[u] = pl[2 * f + 1];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (f0 + 3 * u < nf)
        best = dmax(best, fma(e23[u].x, y[2], fma(e01[u].y, y[1], e01[u].x * y[0])) - e23[u].y);
  }
  return best;
}

}  // namespace fl

constexpr int kForcePairsPerPass = 8;   // pairs one call handles (four lanes each)

// The whole warp calls this for the n <= 8 pairs e[0..n) (shared memory).
// SET: the context's kind set (as shape_value).  LAW: false when the step has
// no contact history, no friction and no velocity-driven damping (the
// relative-velocity, history and friction code is then compiled out).
template <int SET, bool LAW>
__device__ __forceinline__ void pair_force_law(ForceArgs a, const OvlRec* e, int n) {
  using namespace fl;
  const int lane = threadIdx.x & 31;
  const int slot = lane >> 2, k = lane & 3, kc = k < 3 ? k : 0, b0 = lane & ~3;
  {
    const bool act = slot < n;
    const OvlRec& er = e[act ? slot : 0];
    const int q = er.q;
    const int i = er.i, j = er.j;
    const int lok = er.lo[kc], d0 = er.dim[0], d1 = er.dim[1], d2 = er.dim[2], sh = er.shift[kc];
    // one round of global loads: both particles' state and shape data
    const double XA = a.X[3 * i + kc];
    const double Xj = a.X[3 * j + kc];
    const double* RA = a.R + 9 * i;
    const double* RB = a.R + 9 * j;
    const double ra0 = RA[kc], ra1 = RA[3 + kc], ra2 = RA[6 + kc];
    const double rb0 = RB[kc], rb1 = RB[3 + kc], rb2 = RB[6 + kc];
    const int ta = a.type[i], tb = a.type[j];
    const double pa0 = a.param[3 * i], pak = a.param[3 * i + kc];
    const double pb0 = a.param[3 * j], pbk = a.param[3 * j + kc];
    const int fa0 = a.face_off[i], fa1 = a.face_off[i + 1], fb0 = a.face_off[j], fb1 = a.face_off[j + 1];
    const double cc = a.compl_[i] + a.compl_[j];
    const double* sm = er.s;
    const double Lk = kc == 0 ? a.L[0] : (kc == 1 ? a.L[1] : a.L[2]);
    const double Lsel = sh == 0 ? 0.0 : (sh > 0 ? Lk : -Lk);
    const double XB = Xj - Lsel;   // X_j - s L, s in {-1, 0, 1}
    const double s0 = sm[0];
    const double V = a.dx3 * s0;
    const double Gk = a.gscale * sm[4 + kc];
    const double G0 = __shfl_sync(kFull, Gk, b0), G1 = __shfl_sync(kFull, Gk, b0 + 1),
                   G2 = __shfl_sync(kFull, Gk, b0 + 2);
    const double gn2 = fma(G2, G2, fma(G1, G1, G0 * G0));
    const bool gok = __double_as_longlong(gn2) > __double_as_longlong(a.g_min2);
    // indentation depth: FP64 re-evaluation at the deepest node
    const int idx = min(max(er.idx, 0), d0 * d1 * d2 - 1);
    const int ck = kc == 0 ? idx % d0 : (kc == 1 ? (idx / d0) % d1 : idx / (d0 * d1));
    const double xk = int_to_double(lok + ck) * a.dx;
    const double rAk = xk - XA, rBk = xk - XB;
    double rA[3], rB[3], yA[3], yB[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rA[c] = __shfl_sync(kFull, rAk, b0 + c);
      rB[c] = __shfl_sync(kFull, rBk, b0 + c);
    }
    const double yAk = fma(ra2, rA[2], fma(ra1, rA[1], ra0 * rA[0]));
    const double yBk = fma(rb2, rB[2], fma(rb1, rB[1], rb0 * rB[0]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      yA[c] = __shfl_sync(kFull, yAk, b0 + c);
      yB[c] = __shfl_sync(kFull, yBk, b0 + c);
    }
    double vA = k < 3 ? shape_value<SET>(ta, pa0, pak, a.planes + 4 * fa0, fa1 - fa0, kc, rA, yA, yAk) : -1e300;
    double vB = k < 3 ? shape_value<SET>(tb, pb0, pbk, a.planes + 4 * fb0, fb1 - fb0, kc, rB, yB, yBk) : -1e300;
    vA = dmax(vA, __shfl_xor_sync(kFull, vA, 1));
    vA = dmax(vA, __shfl_xor_sync(kFull, vA, 2));
    vB = dmax(vB, __shfl_xor_sync(kFull, vB, 1));
    vB = dmax(vB, __shfl_xor_sync(kFull, vB, 2));
    const double fa = vA - a.inflate, fb = vB - a.inflate;
    const double d = dmax(0.0, -(fa + fb));
    const double vd = V * d;
    const bool vok = __double_as_longlong(vd) > 0;
    // four reciprocal square roots, one per lane: s0, E*'s compliance sum, |G|^2, V d
    const double arg = k == 0 ? s0 : (k == 1 ? cc : (k == 2 ? (gok ? gn2 : 1.0) : (vok ? vd : 1.0)));
    const double y = nr_rsqrt(arg);
    const double y0 = __shfl_sync(kFull, y, b0), y1 = __shfl_sync(kFull, y, b0 + 1),
                   y2 = __shfl_sync(kFull, y, b0 + 2), y3 = __shfl_sync(kFull, y, b0 + 3);
    const double inv_s0 = y0 * y0;
    const double estar = y1 * y1;
    const double xck = fma(sm[1 + kc], inv_s0, int_to_double(lok)) * a.dx;
    double nk = Gk * y2;
    double fallback = 0.0;
    if (__any_sync(kFull, act && !gok)) {   // centre-line fallback normal (a wall: -m)
      const double dXk = XB - XA;
      const double e0v = __shfl_sync(kFull, dXk, b0), e1v = __shfl_sync(kFull, dXk, b0 + 1),
                     e2v = __shfl_sync(kFull, dXk, b0 + 2);
      if (!gok) {
        fallback = 1.0;
        const double nd2 = fma(e2v, e2v, fma(e1v, e1v, e0v * e0v));
        nk = __double_as_longlong(nd2) > 0 ? dXk * nr_rsqrt(nd2) : 0.0;
        if (j >= a.n) nk = -a.planes[4 * fb0 + kc];
      }
    }
    const double gn = gok ? gn2 * y2 : 0.0;
    const double rak = xck - XA, rbk = xck - XB;
    // components k1 = k+1, k2 = k+2 (mod 3) of the lever arms, for the cross products
    const int k1 = kc == 2 ? 0 : kc + 1, k2 = kc == 0 ? 2 : kc - 1;
    const double ra1v = __shfl_sync(kFull, rak, b0 + k1), ra2v = __shfl_sync(kFull, rak, b0 + k2);
    const double rb1v = __shfl_sync(kFull, rbk, b0 + k1), rb2v = __shfl_sync(kFull, rbk, b0 + k2);
    // velocity of A relative to B at x_c, u_AB = (v_A + w_A x r_A) - (v_B + w_B x r_B),
    // and its normal part ddot_n (> 0 when approaching)
    double uabk = 0.0, ddot = 0.0;
    if (LAW && a.vel != nullptr && (a.damping_c != 0.0 || a.history || a.friction)) {
      const double* va = a.vel + 6 * i;
      const double* vb = j < a.n ? a.vel + 6 * j : a.rest6;
      const double wak = fma(va[3 + k1], ra2v, -va[3 + k2] * ra1v);
      const double wbk = fma(vb[3 + k1], rb2v, -vb[3 + k2] * rb1v);
      uabk = (va[kc] + wak) - (vb[kc] + wbk);
      const double uk = uabk * nk;
      const double u0 = __shfl_sync(kFull, uk, b0), u1 = __shfl_sync(kFull, uk, b0 + 1),
                     u2 = __shfl_sync(kFull, uk, b0 + 2);
      ddot = (u0 + u1) + u2;
    }
    // tangential part u_t = u_AB - ddot_n n, for the friction law
    double utk = 0.0, utn2 = 0.0;
    if (LAW && a.friction && a.vel != nullptr) {
      utk = fma(-ddot, nk, uabk);
      const double t2 = utk * utk;
      const double t0 = __shfl_sync(kFull, t2, b0), t1 = __shfl_sync(kFull, t2, b0 + 1),
                     t2b = __shfl_sync(kFull, t2, b0 + 2);
      utn2 = (t0 + t1) + t2b;
    }
    // two more reciprocal square roots: of ddot_n (lane 0, a new contact's
    // c = damp_K / ddot_n) and of |u_t|^2 (lane 1)
    double inv_ddot = 0.0, inv_utn = 0.0;
    const bool dpos = __double_as_longlong(ddot) > 0, upos = __double_as_longlong(utn2) > 0;
    if (LAW && (a.history || a.friction)) {
      const double y5 = nr_rsqrt(k == 0 ? (dpos ? ddot : 1.0) : (upos ? utn2 : 1.0));
      const double ya = __shfl_sync(kFull, y5, b0), yb = __shfl_sync(kFull, y5, b0 + 1);
      inv_ddot = dpos ? ya * ya : 0.0;
      inv_utn = upos ? yb : 0.0;
    }
    double cdamp = a.damping_c;   // c of Eq. (damping_factor) for this pair
    if (LAW && a.history) {
      // an ongoing contact (i, j) keeps its c; a new one takes c from u0 = ddot_n
      // (0 without velocities or for u0 <= 0).  Lane k of the pair checks the
      // entries k, k + 4, ... of i's list; the first 8 are loaded before the count.
      const size_t base = static_cast<size_t>(i) * a.hist_cap;
      const int cnt = min(a.hn_rd[i], a.hist_cap);
      int hit = -1;
      double ch = 0.0;
      {
        const int m0 = k, m1 = k + 4;
        const int j0 = m0 < a.hist_cap ? a.hj_rd[base + m0] : -1;
        const int j1 = m1 < a.hist_cap ? a.hj_rd[base + m1] : -1;
        const double c0 = m0 < a.hist_cap ? a.hc_rd[base + m0] : 0.0;
        const double c1 = m1 < a.hist_cap ? a.hc_rd[base + m1] : 0.0;
        if (m0 < cnt && j0 == j) { hit = m0; ch = c0; }
        if (m1 < cnt && j1 == j) { hit = m1; ch = c1; }
      }
      const int cmax = __reduce_max_sync(kFull, act ? cnt : 0);
      for (int m0 = 8; m0 < cmax; m0 += 4) {
        const int m = m0 + k;
        if (m < cnt && a.hj_rd[base + m] == j) { hit = m; ch = a.hc_rd[base + m]; }
      }
      // the pair's lane with the hit (if any) supplies c
      int src = hit >= 0 ? lane : -1;
      src = max(src, __shfl_xor_sync(kFull, src, 1));
      src = max(src, __shfl_xor_sync(kFull, src, 2));
      ch = __shfl_sync(kFull, ch, src >= 0 ? src : b0);
      cdamp = src >= 0 ? ch : a.damp_K * inv_ddot;
    }
    double damp = 1.0;
    if (LAW && a.vel != nullptr && cdamp != 0.0) damp = dmax(0.0, fma(cdamp, ddot, 1.0));
    const double fmag = vok ? (4.0 / (3.0 * 3.14159265358979323846)) * estar * (vd * y3) * damp : 0.0;
    double Fk = fmag * nk;
    if (LAW && a.friction && __double_as_longlong(fmag) > 0 && upos) {
      // Eq. (contact_force_tangential): B receives +f(a) |F_n| t, a = |u_t| / u_k,
      // f = (2 mu_s* - mu_k) a^2 / (a^4 + 1) + mu_k a^2 / (a^2 + 1)
      const double sa = utn2 * inv_utn * a.inv_u_k;
      const double a2 = sa * sa;
      double coef = a.mu_k;
      if (a2 < 1e30) {
        const double den1 = fma(a2, a2, 1.0), den2 = a2 + 1.0;
        coef = a2 * fma(2.0 * a.mu_s_star - a.mu_k, den2, a.mu_k * den1) / (den1 * den2);
      }
      Fk = fma(coef * fmag, utk * inv_utn, Fk);
    }
    const double F1 = __shfl_sync(kFull, Fk, b0 + k1), F2 = __shfl_sync(kFull, Fk, b0 + k2);
    // T_A = r_A x (-F), T_B = r_B x F
    const double TAk = fma(ra2v, F1, -ra1v * F2);
    const double TBk = fma(rb1v, F2, -rb2v * F1);
    if (act) {
      double* o = a.pair_out + static_cast<size_t>(q) * 11;
      double* f = a.ft + static_cast<size_t>(q) * kFtDoubles;
      double* tp = a.tape + static_cast<size_t>(q) * kTapeDoubles;
      if (k < 3) {
        o[1 + k] = xck; o[4 + k] = nk; o[8 + k] = Fk;
        f[k] = Fk; f[3 + k] = TAk; f[6 + k] = TBk;
        tp[1 + k] = xck; tp[4 + k] = nk;
      }
      if (k == 0) {
        o[0] = V; o[7] = d;
        tp[0] = s0; tp[7] = d; tp[8] = gn; tp[9] = fallback;
      } else if (k == 3) {
        tp[10] = estar; tp[11] = damp; tp[12] = fmag; tp[13] = int_to_double(idx);
        tp[14] = cdamp; tp[15] = 0.0;
      }
      if (LAW && a.history && k == 0) {   // this step's contact list of i
        const int slot = atomicAdd(a.hn_wr + i, 1);
        if (slot < a.hist_cap) {
          a.hj_wr[static_cast<size_t>(i) * a.hist_cap + slot] = j;
          a.hc_wr[static_cast<size_t>(i) * a.hist_cap + slot] = cdamp;
        }
      }
    }
  }
}

}  // namespace gbc
