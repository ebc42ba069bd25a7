// Adjoint of the contact step (smoothed indicator): gradient of
//   L = sum_p (gF_p . F_p + gT_p . T_p)
// with respect to positions and raw quaternions.
//
// Forward map per pair (lattice sums over the pair box, lattice units):
//   S0 = sum W, S1 = sum W c, Sg = sum (mA grad phiA - mB grad phiB),
//   W = H(phiA) H(phiB), H = S(t), t = clamp(1/2 - phi/w, 0, 1), m = t(1-t) H_other,
//   V = dx^3 S0, x_c = (lo + S1/S0) dx, G = 1/2 dx^2 (6/w) Sg, n = G/|G|,
//   d = -phiA(x*) - phiB(x*) at the deepest node x*,
//   F = 4/(3 pi) E* sqrt(V d)(1 + c ddot_n) n  (Eq. contact_force_normal),
//   T_A = (x_c - X_A) x (-F), T_B = (x_c - X_B') x F.
// k_adj_pre: FP64 chain rule from (gF, gT) to seeds dL/dS0, dL/dS1, dL/dSg
//   and the explicit pose terms (torque arms, damping, fallback normal).
// k_adj_cells: persistent tile sweep (the forward's tiles, warp w taking
//   tiles w, w + W, ...); each line clipped to the nodes where both phi < w/2
//   (line_clip.cuh), every other node's terms being exact zeros, the clipped
//   nodes spread one per lane; per node
//   dL/dphi and dL/d(grad phi) pulled back to the 12 pose directions of the
//   pair (translation and infinitesimal world rotation of each particle):
//     dphi/dX = -grad phi,  dphi/domega = grad phi x r,
//     sphere: d(grad phi)/dX = -(I - g g^T)/|r|; faces: d(grad phi) = omega x grad phi.
//   The warp completing a pair's last tile sums the tile partials in FP64
//   and adds them, in physical units, to the pair's pose gradient (which
//   k_adj_pre starts with the explicit and the depth terms).
// k_adj_scatter: per particle in the forward order; the rotation gradient tau
//   becomes dL/dq = (2/|q|) (-v.tau, w tau + tau x v) for q/|q| = (w, v).
#include <cfloat>
#include <cstddef>

#include "contact_dev.cuh"
#include "force_law.cuh"
#include "line_clip.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
// Warps per block and blocks per SM of the cell sweep, per kind set: the
// cubes-only and sphere/cuboid variants at three blocks (a warp per tile at a
// settling box's size, a few spilled registers: 16.0 -> 15.0 us on the 1934
// cubes), the variant with every kind at two (three spill too much there:
// 23.5 -> 28.5 us on the mixed box).
constexpr int kAdjWarps = 8;
template <int SET>
__host__ __device__ constexpr int adj_blocks() { return SET == 0 ? 2 : 3; }
constexpr int kAdjPartial = 12;
constexpr int kSeedFloats = 8;
constexpr int kPairGrad = 16;

struct AdjBufs {
  float* partial;  // [max_tiles, 12]
  float* seeds;    // [max_pairs, 8]
  double* pgrad;   // [max_pairs, 16]
  int* done;       // [max_pairs] tiles of the pair swept so far (pairs of several tiles)
};


__device__ __forceinline__ void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------- pair level
// The depth term of d = -phiA(x*) - phiB(x*) at the pair's deepest node x*
// (the tape's node index), seeded with gd = dL/dd: d(-phi)/dX = grad phi and
// d(-phi)/domega = r x grad phi (world frame; the face of the maximum, first
// index on ties), component kc on lanes 0..2 of the pair's four (the layout
// of k_adj_pre).  Called by the whole warp; `want` selects the pairs that
// need it (the others get zeros).
__device__ __forceinline__ void adj_depth_term(const Params& P, const Shapes& S, const Parts& D, const PairRec& pr,
                                               const double* tp, double gd, bool want, double& dA, double& dcA,
                                               double& dB, double& dcB) {
  const int lane = threadIdx.x & 31;
  const int k = lane & 3, kc = k < 3 ? k : 0, b0 = lane & ~3;
  const int k1 = kc == 2 ? 0 : kc + 1, k2 = kc == 0 ? 2 : kc - 1;
  dA = dcA = dB = dcB = 0.0;
  if (__any_sync(kFull, want)) {
    const int i = pr.i, j = pr.j;
    const int d0 = pr.dim[0], d1 = pr.dim[1], d2 = pr.dim[2];
    const int idx = min(max(static_cast<int>(tp[13]), 0), d0 * d1 * d2 - 1);
    const int ck = kc == 0 ? idx % d0 : (kc == 1 ? (idx / d0) % d1 : idx / (d0 * d1));
    const int lok = kc == 0 ? pr.lo[0] : (kc == 1 ? pr.lo[1] : pr.lo[2]);
    const int sh = kc == 0 ? pr.shift[0] : (kc == 1 ? pr.shift[1] : pr.shift[2]);
    const double Lk = kc == 0 ? P.L[0] : (kc == 1 ? P.L[1] : P.L[2]);
    const double xk = static_cast<double>(lok + ck) * P.dx;
    const double XA = D.X[3 * i + kc];
    const double XB = D.X[3 * j + kc] - (sh == 0 ? 0.0 : (sh > 0 ? Lk : -Lk));
    const double rAk = xk - XA, rBk = xk - XB;
    double rA[3], rB[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rA[c] = __shfl_sync(kFull, rAk, b0 + c);
      rB[c] = __shfl_sync(kFull, rBk, b0 + c);
    }
    // world gradient component kc of one particle's phi at x* (r = x* - X, scalars;
    // shp: the image shift of this lane's component, 0 for particle i)
    auto grad_k = [&](int pid, double r0, double r1, double r2, int shp) -> double {
      const double* R = D.R + 9 * pid;
      const int type = S.type[pid];
      const double yk = R[kc] * r0 + R[3 + kc] * r1 + R[6 + kc] * r2;   // y = R^T r
      const double y0 = __shfl_sync(kFull, yk, b0), y1 = __shfl_sync(kFull, yk, b0 + 1),
                   y2 = __shfl_sync(kFull, yk, b0 + 2);
      // this lane's candidate: value and index of its faces (cuboid: face pair kc; polytope: kc, kc + 3, ...)
      double best = -1e300;
      int bidx = 0x7fffffff;
      // polytopes: an FP32 prefilter over the world planes (lattice units,
      // inflate included: the FP64 values up to a constant shift and scale,
      // so the same order of faces).  Each lane keeps its best face and the
      // value of its second; the FP64 value of a lane's best face is formed
      // when it lies within the margin of the pair's FP32 maximum, and every
      // face is formed in FP64 when a second face of a lane lies within it
      // too.  The margin is far above the FP32 rounding (~1e-6 of the terms),
      // so the faces left out lie below the FP64 maximum.  The shuffles run on
      // every lane (other types carry no faces).
      const bool poly = type == 2;
      const int f0 = poly ? S.face_off[pid] : 0, nf = poly ? S.face_off[pid + 1] - f0 : 0;
      float rl = 0.f;
      if (poly) {
        const float ncell = static_cast<float>(kc == 0 ? P.ncell[0] : (kc == 1 ? P.ncell[1] : P.ncell[2]));
        rl = (static_cast<float>((lok + ck) - D.kX[3 * pid + kc]) + static_cast<float>(shp) * ncell) -
             D.fX[3 * pid + kc];
      }
      const float rl0 = __shfl_sync(kFull, rl, b0), rl1 = __shfl_sync(kFull, rl, b0 + 1),
                  rl2 = __shfl_sync(kFull, rl, b0 + 2);
      float v1 = -FLT_MAX, v2 = -FLT_MAX, wmax = 0.f;
      int i1 = kc;
      for (int f = kc; f < nf && k < 3; f += 3) {
        const float4 e = D.wplane[f0 + f];
        const float v = fmaf(e.x, rl0, fmaf(e.y, rl1, fmaf(e.z, rl2, -e.w)));
        wmax = fmaxf(wmax, fabsf(e.w));
        if (v > v1) {
          v2 = v1;
          v1 = v;
          i1 = f;
        } else {
          v2 = fmaxf(v2, v);
        }
      }
      float m32 = fmaxf(v1, __shfl_xor_sync(kFull, v1, 1));
      m32 = fmaxf(m32, __shfl_xor_sync(kFull, m32, 2));
      wmax = fmaxf(wmax, __shfl_xor_sync(kFull, wmax, 1));
      wmax = fmaxf(wmax, __shfl_xor_sync(kFull, wmax, 2));
      const float margin = 1e-5f * (1.f + fabsf(rl0) + fabsf(rl1) + fabsf(rl2) + wmax);
      const bool all_faces = __any_sync(kFull, poly && k < 3 && v2 >= m32 - margin);
      if (type == 1) {
        best = fabs(yk) - S.param[3 * pid + kc];
        bidx = kc;
      } else if (poly && all_faces) {
        for (int f = kc; f < nf; f += 3) {
          const double* pl = S.planes + 4 * (f0 + f);
          const double a = (pl[0] * y0 + pl[1] * y1 + pl[2] * y2) - pl[3];
          if (a > best) { best = a; bidx = f; }
        }
      } else if (poly && k < 3 && i1 < nf && v1 >= m32 - margin) {
        const double* pl = S.planes + 4 * (f0 + i1);
        best = (pl[0] * y0 + pl[1] * y1 + pl[2] * y2) - pl[3];
        bidx = i1;
      }
      if (k == 3) { best = -1e300; bidx = 0x7fffffff; }
      // first maximal face over the pair's three lanes
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        const double ob = __shfl_xor_sync(kFull, best, o);
        const int oi = __shfl_xor_sync(kFull, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
      }
      // sphere r / |r|; cuboid R e_kk sign(y_kk); polytope R n_f
      if (type == 0) {   // r / |r| by a Newton-Raphson reciprocal square root
        const double rr = r0 * r0 + r1 * r1 + r2 * r2;
        return rr > 0.0 ? (kc == 0 ? r0 : (kc == 1 ? r1 : r2)) * fl::nr_rsqrt(rr) : 0.0;
      }
      if (type == 1) {
        const int bb = min(max(bidx, 0), 2);
        const double ykk = bb == 0 ? y0 : (bb == 1 ? y1 : y2);
        return R[3 * kc + bb] * (ykk < 0.0 ? -1.0 : 1.0);
      }
      const double* pl = S.planes + 4 * (f0 + min(max(bidx, 0), nf - 1));   // (a face always: nf >= 1 here)
      return R[3 * kc] * pl[0] + R[3 * kc + 1] * pl[1] + R[3 * kc + 2] * pl[2];
    };
    const double g[2] = {grad_k(i, rA[0], rA[1], rA[2], 0), grad_k(j, rB[0], rB[1], rB[2], sh)};
    // r x grad phi, component kc
    const double gA1 = __shfl_sync(kFull, g[0], b0 + k1), gA2 = __shfl_sync(kFull, g[0], b0 + k2);
    const double gB1 = __shfl_sync(kFull, g[1], b0 + k1), gB2 = __shfl_sync(kFull, g[1], b0 + k2);
    const double rA1 = kc == 0 ? rA[1] : (kc == 1 ? rA[2] : rA[0]), rA2 = kc == 0 ? rA[2] : (kc == 1 ? rA[0] : rA[1]);
    const double rB1 = kc == 0 ? rB[1] : (kc == 1 ? rB[2] : rB[0]), rB2 = kc == 0 ? rB[2] : (kc == 1 ? rB[0] : rB[1]);
    if (want) {
      dA = gd * g[0];
      dcA = gd * (rA1 * gA2 - rA2 * gA1);
      dB = gd * g[1];
      dcB = gd * (rB1 * gB2 - rB2 * gB1);
    }
  }
}

// The pair-level chain rule, four lanes per pair and eight pairs per warp pass:
// component k = 0..2 of every 3-vector on lanes 0..2 of the pair (cross and dot
// products by shuffles), lane 3 for the third reciprocal square root and the
// scalar stores.  Every FP64 warp instruction holds a sub-partition's FP64 pipe
// ~40 ns however many lanes are active, so splitting each pair's vectors over
// lanes shortens the chain about threefold.  Per-pair conditions are taken by
// selects (or branches without shuffles); a branch with shuffles is entered
// by the whole warp when any of its pairs needs it.
__global__ void __launch_bounds__(32) k_adj_pre(Params P, Shapes S, Parts D, Lists W, AdjBufs B,
                                                 const double* __restrict__ vel, const double* __restrict__ gF,
                                                 const double* __restrict__ gT) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int slot = lane >> 2, k = lane & 3, kc = k < 3 ? k : 0, b0 = lane & ~3;
  const int k1 = kc == 2 ? 0 : kc + 1, k2 = kc == 0 ? 2 : kc - 1;
  const int np = min(W.counters[0], P.max_pairs);
  const int nw = gridDim.x * static_cast<int>(blockDim.x >> 5);
  const int gw = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  // component c of the pair's vector held as v (component k on lane b0 + k)
  auto at = [&](double v, int c) { return __shfl_sync(kFull, v, b0 + c); };
  auto sum3 = [&](double v) { return (at(v, 0) + at(v, 1)) + at(v, 2); };
  // component kc of a x b
  auto cross = [&](double a, double b) { return at(a, k1) * at(b, k2) - at(a, k2) * at(b, k1); };
  for (int q0 = 8 * gw; q0 < np; q0 += 8 * nw) {
    const int p = q0 + slot;
    const bool inr = p < np;
    const int pc = inr ? p : q0;
    const double* tp = W.tape + static_cast<size_t>(pc) * kTapeDoubles;
    const PairRec& pr = W.pairs[pc];
    const double S0 = tp[0];
    const double fmag = tp[12];
    const bool act = inr && S0 > 0.0 && record_in_bounds(P, W.err, pr, false);
    const int i = act ? pr.i : 0, j = act ? pr.j : 0;
    const bool wallj = j >= P.n;   // a wall has no output and no velocity
    const double dx = P.dx;
    const double Lk = kc == 0 ? P.L[0] : (kc == 1 ? P.L[1] : P.L[2]);
    const double XA = D.X[3 * i + kc];
    const double XB = D.X[3 * j + kc] - pr.shift[kc] * Lk;
    const double xc = tp[1 + kc], nk = tp[4 + kc];
    double Fk = fmag * nk;
    const double rA = xc - XA, rB = xc - XB;
    const double gFi = gF[3 * i + kc], gFj = wallj ? 0.0 : gF[3 * j + kc];
    const double gTi = gT[3 * i + kc], gTj = wallj ? 0.0 : gT[3 * j + kc];
    const double d = tp[7], gnorm = tp[8], damp = tp[11], fb = tp[9];
    // c of Eq. (damping_factor) as the forward used it (the shared one, or the
    // contact's own with contact history, held fixed like every per-contact constant)
    const double cdamp = tp[14];
    // relative velocity u_AB = (v_A + w_A x r_A) - (v_B + w_B x r_B) at x_c, ddot_n = u_AB . n
    double uab = 0.0, ddot = 0.0;
    const double* va = vel != nullptr ? vel + 6 * i : nullptr;
    const double* vb = vel != nullptr ? (wallj ? D.rest6 : vel + 6 * j) : nullptr;
    if (vel != nullptr) {
      const double wa = va[3 + k1] * at(rA, k2) - va[3 + k2] * at(rA, k1);
      const double wb = vb[3 + k1] * at(rB, k2) - vb[3 + k2] * at(rB, k1);
      const double u = (va[kc] + wa) - (vb[kc] + wb);
      const double dd = sum3(u * nk);
      const bool vlaw = fmag > 0.0 && (cdamp != 0.0 || P.friction);
      uab = vlaw ? u : 0.0;
      ddot = vlaw ? dd : 0.0;
    }
    // friction, Eq. (contact_force_tangential): F = fmag (n + f(a) t), t = u_t / |u_t|,
    // u_t = u_AB - ddot_n n, a = |u_t| / u_k
    bool fric = false;
    double tdir = 0.0, coef = 0.0, dcoef = 0.0, utn = 0.0;
    if (P.friction && vel != nullptr) {
      const double ut = uab - ddot * nk;
      const double utn2 = sum3(ut * ut);
      fric = fmag > 0.0 && utn2 > 0.0;
      if (fric) {
        utn = sqrt(utn2);
        tdir = ut / utn;
        const double a = utn * P.inv_u_k, a2 = a * a;
        const double A = 2.0 * P.mu_s_star - P.mu_k;
        coef = P.mu_k;
        if (a2 < 1e30) {
          const double den1 = a2 * a2 + 1.0, den2 = a2 + 1.0;
          coef = a2 * (A * den2 + P.mu_k * den1) / (den1 * den2);
          // f'(a) = 2a [A (1 - a^4) / (a^4 + 1)^2 + mu_k / (a^2 + 1)^2]
          dcoef = 2.0 * a * (A * (1.0 - a2 * a2) / (den1 * den1) + P.mu_k / (den2 * den2));
        }
        Fk += fmag * coef * tdir;
      }
    }
    // dL/dF = Lambda, dL/dx_c, explicit dL/dX_A, dL/dX_B'
    const double c1 = cross(gTi, rA), c2 = cross(gTj, rB);
    const double Lam = gFj - gFi - c1 + c2;
    const double dT = gTj - gTi;
    double gxc = cross(Fk, dT);
    double gXA = cross(Fk, gTi);
    double gXB = cross(gTj, Fk);
    const double Ln = sum3(Lam * nk);
    const double Lt = sum3(Lam * tdir);
    const double Lm = Ln + coef * Lt;   // dL/dfmag
    double gn = fmag * Lam;
    double guab = 0.0;   // dL/du_AB
    if (__any_sync(kFull, fric)) {
      // through t (projected on its normal plane) and through f(a)
      const double s_dir = fric ? fmag * coef / utn : 0.0, s_mag = fmag * Lt * dcoef * P.inv_u_k;
      const double gut = s_dir * (Lam - Lt * tdir) + s_mag * tdir;
      const double gun = sum3(gut * nk);
      if (fric) {
        guab += gut - gun * nk;
        gn -= uab * gun + ddot * gut;
      }
    }
    // reciprocal square roots by Newton-Raphson from an FP32 seed (no FP64
    // division sequence): lane 0 of S0, lane 1 of d, lane 2 of |G|^2
    const double rarg = k == 0 ? S0 : (k == 1 ? d : (k == 2 ? gnorm : 1.0));
    const double rr = fl::nr_rsqrt(rarg > 0.0 ? rarg : 1.0);
    const double yS = at(rr, 0), yd = at(rr, 1), yg = at(rr, 2);
    const double inv_S0 = yS * yS;
    double gV = 0.0, gd = 0.0;
    if (fmag > 0.0) {
      const double half_lf = 0.5 * Lm * fmag;
      gV = half_lf * inv_S0 * (P.inv_dx * P.inv_dx * P.inv_dx);
      gd = half_lf * (yd * yd);
      if (vel != nullptr && cdamp != 0.0 && damp > 0.0) {
        const double gdd = Lm * fmag * cdamp / damp;   // dL/d(ddot_n)
        gn += gdd * uab;
        guab += gdd * nk;
      }
    }
    if (vel != nullptr) {
      // u_AB depends on x_c, X_A and X_B' through the angular velocities
      const double ga = at(guab, k1) * va[3 + k2] - at(guab, k2) * va[3 + k1];
      const double gb = at(guab, k1) * vb[3 + k2] - at(guab, k2) * vb[3 + k1];
      if (fric || cdamp != 0.0) {
        gxc += ga - gb;
        gXA -= ga;
        gXB += gb;
      }
    }
    // normal: n = G / |G| with G = kappa Sg, or the centre-line fallback
    const double kappa = P.gscale;
    const double gnn = sum3(gn * nk);
    double sg = 0.0;
    if (fb == 0.0) sg = (kappa * (yg * yg)) * (gn - gnn * nk);
    if (__any_sync(kFull, act && fb != 0.0)) {
      const double e = XB - XA;
      const double dl = sqrt(sum3(e * e));
      if (fb != 0.0 && dl > 0.0) {
        const double g = (gn - gnn * nk) / dl;
        gXB += g;
        gXA -= g;
      }
    }
    // the depth term at the deepest node (independent of the cell sums, so formed here)
    double dA, dcA, dB, dcB;
    adj_depth_term(P, S, D, pr, tp, gd, act && gd != 0.0 && d > 0.0, dA, dcA, dB, dcB);
    gXA += dA;
    gXB += dB;
    // x_c = (lo + S1/S0) dx ; V = dx^3 S0
    const double s1 = gxc * dx * inv_S0;
    const double s0t = gxc * (xc - pr.lo[kc] * dx) * inv_S0;
    const double s0 = ((gV * dx * dx * dx - at(s0t, 0)) - at(s0t, 1)) - at(s0t, 2);
    if (inr) {
      float* sd = B.seeds + static_cast<size_t>(p) * kSeedFloats;
      double* pg = B.pgrad + static_cast<size_t>(p) * kPairGrad;
      if (k < 3) {
        sd[1 + k] = act ? static_cast<float>(s1) : 0.f;
        sd[4 + k] = act ? static_cast<float>(sg) : 0.f;
        pg[k] = act ? gXA : 0.0;
        pg[3 + k] = act ? dcA : 0.0;
        pg[6 + k] = act ? gXB : 0.0;
        pg[9 + k] = act ? dcB : 0.0;
      } else {
        sd[0] = act ? static_cast<float>(s0) : 0.f;
        sd[7] = 0.f;
        pg[12] = act ? gd : 0.0;
        pg[13] = 0.0;
        pg[14] = 0.0;
        pg[15] = 0.0;
        B.done[p] = 0;
      }
    }
  }
}

// ---------------------------------------------------------------- node level
struct AdjGeom {
  int type, nf;
  float c[3];    // centre relative to the box origin (lattice units)
  float rt[9];   // R^T (row k = body axis k in world)
  float size[3];
  const float4* sp;  // world planes (x, y, z, offset) in shared memory
};

// Component k of (a, b, c) by selects (no runtime-indexed array).
__device__ __forceinline__ float sel3(float a, float b, float c, int k) { return k == 0 ? a : (k == 1 ? b : c); }


// phi (lattice units, inflate included), unit world gradient, |r| (spheres).
// SET is the context's kind set (2: cubes only, 1: spheres, cuboids and
// walls, 0: every kind): the types a set cannot hold are compiled out.
template <int SET>
__device__ __forceinline__ float adj_eval(const AdjGeom& g, const float r[3], float gr[3], float* rn) {
  if (SET != 2 && g.type == 0) {
    const float q = fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]));
    const float nr = sqrtf(q);
    const float inv = nr > 0.f ? 1.f / nr : 0.f;
    for (int k = 0; k < 3; ++k) gr[k] = r[k] * inv;
    *rn = nr;
    return nr - g.size[0];
  }
  *rn = 0.f;
  if (SET != 2 && g.type == 3) {   // wall
    for (int k = 0; k < 3; ++k) gr[k] = g.rt[k];
    return fmaf(g.rt[0], r[0], fmaf(g.rt[1], r[1], fmaf(g.rt[2], r[2], g.size[0])));
  }
  if (SET != 0 || g.type == 1) {
    float y[3], a[3];
    for (int k = 0; k < 3; ++k) {
      y[k] = fmaf(g.rt[3 * k], r[0], fmaf(g.rt[3 * k + 1], r[1], g.rt[3 * k + 2] * r[2]));
      a[k] = fabsf(y[k]) - g.size[k];
    }
    const int kk = (a[0] >= a[1] && a[0] >= a[2]) ? 0 : (a[1] >= a[2] ? 1 : 2);
    const float yk = kk == 0 ? y[0] : (kk == 1 ? y[1] : y[2]);
    const float sgn = yk < 0.f ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) gr[k] = sgn * (kk == 0 ? g.rt[k] : (kk == 1 ? g.rt[3 + k] : g.rt[6 + k]));
    return kk == 0 ? a[0] : (kk == 1 ? a[1] : a[2]);
  }
  int kk = 0;
  float best = -FLT_MAX;
  for (int f = 0; f < g.nf; ++f) {
    const float4 e = g.sp[f];
    const float v = fmaf(e.x, r[0], fmaf(e.y, r[1], fmaf(e.z, r[2], -e.w)));
    if (v > best) { best = v; kk = f; }
  }
  const float4 e = g.sp[kk];
  gr[0] = e.x; gr[1] = e.y; gr[2] = e.z;
  return best;
}

// phi alone (the same arithmetic as adj_eval, without the gradient): the band test
template <int SET>
__device__ __forceinline__ float adj_phi(const AdjGeom& g, const float r[3]) {
  if (SET != 2 && g.type == 0) return sqrtf(fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2]))) - g.size[0];
  if (SET != 2 && g.type == 3) return fmaf(g.rt[0], r[0], fmaf(g.rt[1], r[1], fmaf(g.rt[2], r[2], g.size[0])));
  if (SET != 0 || g.type == 1) {
    float best = -FLT_MAX;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float y = fmaf(g.rt[3 * k], r[0], fmaf(g.rt[3 * k + 1], r[1], g.rt[3 * k + 2] * r[2]));
      best = fmaxf(best, fabsf(y) - g.size[k]);
    }
    return best;
  }
  float best = -FLT_MAX;
  for (int f = 0; f < g.nf; ++f) {
    const float4 e = g.sp[f];
    best = fmaxf(best, fmaf(e.x, r[0], fmaf(e.y, r[1], fmaf(e.z, r[2], -e.w))));
  }
  return best;
}

// [lo, hi] (box coordinates along au) cut to where phi < T on the node line
// with box coordinates cv, cw along av, aw; ci, cf: the particle centre
// relative to the box origin as nearest node + remainder (r = (c - ci) - cf).
template <int SET>
__device__ __forceinline__ void adj_clip(const AdjGeom& g, int au, int av, int aw, int cv, int cw, const int* ci,
                                         const float* cf, float T, float& lo, float& hi) {
  const int iu = ci[0] * (au == 0) + ci[1] * (au == 1) + ci[2] * (au == 2);
  const int iv = ci[0] * (av == 0) + ci[1] * (av == 1) + ci[2] * (av == 2);
  const int iw = ci[0] * (aw == 0) + ci[1] * (aw == 1) + ci[2] * (aw == 2);
  const float fu = sel3(cf[0], cf[1], cf[2], au);
  const float rv = static_cast<float>(cv - iv) - sel3(cf[0], cf[1], cf[2], av);
  const float rw = static_cast<float>(cw - iw) - sel3(cf[0], cf[1], cf[2], aw);
  const float o = static_cast<float>(iu);
  float l = lo - o, h = hi - o;   // node counter c = cu - iu, r_u = c - fu
  if (SET != 2 && g.type == 0) {
    clip_ball(fu, fmaf(rv, rv, rw * rw), g.size[0], T, l, h);
  } else if (SET != 2 && g.type == 3) {
    const float mu = sel3(g.rt[0], g.rt[1], g.rt[2], au);
    const float p = fmaf(sel3(g.rt[0], g.rt[1], g.rt[2], av), rv,
                         fmaf(sel3(g.rt[0], g.rt[1], g.rt[2], aw), rw, fmaf(-mu, fu, g.size[0])));
    clip_half(mu, clip_inv(mu), p, T, l, h);
  } else if (SET != 0 || g.type == 1) {
    // constants staged by adj_prep_clip: slab k is the node-counter interval
    // centred at fu - sv_k rv - sw_k rw with half-width hd_k
    const float4 a = g.sp[0], b = g.sp[1], c = g.sp[2];
    if (__float_as_int(c.y) == 0) {
      const float x0 = fmaf(-a.x, rv, fmaf(-b.x, rw, fu));
      const float x1 = fmaf(-a.y, rv, fmaf(-b.y, rw, fu));
      const float x2 = fmaf(-a.z, rv, fmaf(-b.z, rw, fu));
      l = fmaxf(l, fmaxf(fmaxf(x0 - a.w, x1 - b.w), x2 - c.x));
      h = fminf(h, fminf(fminf(x0 + a.w, x1 + b.w), x2 + c.x));
    } else {   // a slab parallel to the line
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float* t = g.rt + 3 * k;
        const float tu = sel3(t[0], t[1], t[2], au);
        const float p = fmaf(sel3(t[0], t[1], t[2], av), rv, fmaf(sel3(t[0], t[1], t[2], aw), rw, -tu * fu));
        clip_slab(tu, clip_inv(tu), p, g.size[k] + T, l, h);
      }
    }
  } else {
    const float* inv = reinterpret_cast<const float*>(g.sp + kMaxFaces);
    for (int f = 0; f < g.nf; ++f) {
      const float4 e = g.sp[f];
      const float eu = sel3(e.x, e.y, e.z, au);
      const float p = fmaf(sel3(e.x, e.y, e.z, av), rv, fmaf(sel3(e.x, e.y, e.z, aw), rw, fmaf(-eu, fu, -e.w)));
      clip_half(eu, inv[f], p, T, l, h);
    }
  }
  lo = l + o;
  hi = h + o;
}

// Per-tile constants of a cuboid's line clip along au (sweep axis) in
// g.sp[0 .. 3): (sv_k, hd_0), (sw_k, hd_1), (hd_2, flat) with sv_k = tv_k / tu_k,
// sw_k = tw_k / tu_k, hd_k = (size_k + T) / |tu_k| (tu, tv, tw: body axis k's
// components along au, av, aw); flat: a slab parallel to the lines.
__device__ __forceinline__ void adj_prep_clip(AdjGeom& g, int au, int av, int aw, float T) {
  float4 a, b, c;
  float* pa = &a.x;
  float* pb = &b.x;
  bool flat = false;
  float hd[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float* t = g.rt + 3 * k;
    const float tu = sel3(t[0], t[1], t[2], au);
    flat = flat || !(fabsf(tu) > kClipFlat);
    const float it = clip_inv(tu);
    pa[k] = sel3(t[0], t[1], t[2], av) * it;
    pb[k] = sel3(t[0], t[1], t[2], aw) * it;
    hd[k] = (g.size[k] + T) * fabsf(it);
  }
  a.w = hd[0];
  b.w = hd[1];
  c = make_float4(hd[2], __int_as_float(flat ? 1 : 0), 0.f, 0.f);
  float4* sm = const_cast<float4*>(g.sp);
  if ((threadIdx.x & 31) == 0) {
    sm[0] = a;
    sm[1] = b;
    sm[2] = c;
  }
  __syncwarp();
}

__device__ __forceinline__ void cross3f(const float a[3], const float b[3], float c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}


// The geometry of particle i (second = false) or j of a staged pair record:
// centre, R^T rows and sizes as the forward's sweep reads them, the type from
// the record's kinds; a polytope's planes and their inverse slopes along the
// sweep axis au go to sm (planes at sm[0 .. nf), slopes after sm[kMaxFaces]).
__device__ __forceinline__ void adj_load_rec(const PairRec& r, bool second, const Shapes& S, const Parts& D,
                                             float4* sm, AdjGeom& g, int au) {
  const int lane = threadIdx.x & 31;
  const int kind = second ? (r.kinds >> 8) : (r.kinds & 0xff);
  const int* ci = second ? r.bi : r.ai;
  const float* cf = second ? r.bf : r.af;
  const float* rt = second ? r.rtb : r.rta;
  const float* sz = second ? r.szb : r.sza;
#pragma unroll
  for (int k = 0; k < 9; ++k) g.rt[k] = rt[k];
  g.nf = 0;
  g.sp = sm;
  if (kind == KIND_WALL) {   // phi = m . c + p0 at box-relative node c (p0 in the size slot)
    g.type = 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g.c[k] = 0.f;
      g.size[k] = sz[0];
    }
    return;
  }
  g.type = kind == KIND_SPHERE ? 0 : (kind == KIND_POLY ? 2 : 1);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g.c[k] = static_cast<float>(ci[k]) + cf[k];
    g.size[k] = sz[k];
  }
  if (g.type == 2) {
    const int pid = second ? r.j : r.i;
    const int f0 = S.face_off[pid];
    g.nf = S.face_off[pid + 1] - f0;
    if (lane < g.nf) {
      const float4 e = D.wplane[f0 + lane];
      sm[lane] = e;
      reinterpret_cast<float*>(sm + kMaxFaces)[lane] = clip_inv(sel3(e.x, e.y, e.z, au));
    }
    __syncwarp();
  }
}

// The warp copies a 224-byte pair record with 14 lanes x 16 bytes.
__device__ __forceinline__ int4 adj_rec_part(const PairRec* src, int lane) {
  return lane < kPairRecWords / 4 ? reinterpret_cast<const int4*>(src)[lane] : make_int4(0, 0, 0, 0);
}
// The pair index of a record held as adj_rec_part pieces (every lane gets it).
constexpr int kPairWord = static_cast<int>(offsetof(PairRec, pair) / 4);
__device__ __forceinline__ int adj_rec_pair(const int4& v) {
  constexpr int c = kPairWord & 3;
  const int w = c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
  return __shfl_sync(kFull, w, kPairWord >> 2);
}
// The seeds of pair p: lanes 0..6 hold s0, s1 and sg (all zero: the pair's
// cells add nothing, its explicit and depth terms came from k_adj_pre).
__device__ __forceinline__ float adj_seed(const AdjBufs& B, int p, int lane) {
  return lane < 7 ? B.seeds[static_cast<size_t>(p) * kSeedFloats + lane] : 0.f;
}

// Sum of acc[0 .. 12) over the warp by halving exchanges (14 shuffles): lane
// c < 12 returns the sum of component c.
__device__ __forceinline__ float adj_warp_sum12(const float acc[12]) {
  const int lane = threadIdx.x & 31;
  const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
  float h6[6];   // components 6 b4 + (0 .. 6)
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float send = b4 ? acc[k] : acc[6 + k];
    h6[k] = (b4 ? acc[6 + k] : acc[k]) + __shfl_xor_sync(kFull, send, 16);
  }
  float h4[4];   // components 6 b4 + 3 b3 + (0 .. 3), the fourth a zero pad
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float send = b3 ? h6[k] : h6[3 + k];
    h4[k] = (b3 ? h6[3 + k] : h6[k]) + __shfl_xor_sync(kFull, send, 8);
  }
  h4[3] = 0.f;
  float h2[2];   // ... + 2 b2 + (0 .. 2)
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b2 ? h4[k] : h4[2 + k];
    h2[k] = (b2 ? h4[2 + k] : h4[k]) + __shfl_xor_sync(kFull, send, 4);
  }
  float h1 = (b1 ? h2[1] : h2[0]) + __shfl_xor_sync(kFull, b1 ? h2[0] : h2[1], 2);   // ... + b1
  h1 += __shfl_xor_sync(kFull, h1, 1);
  // lane c < 12 reads the lane holding component c = 6 b4 + 3 b3 + 2 b2 + b1
  const int c = lane < 12 ? lane : 0;
  const int c4 = c >= 6, r4 = c - 6 * c4, c3 = r4 >= 3, r3 = r4 - 3 * c3;
  return __shfl_sync(kFull, h1, (c4 << 4) | (c3 << 3) | ((r3 >> 1) << 2) | ((r3 & 1) << 1));
}

template <int SET>
__global__ void __launch_bounds__(kAdjWarps * 32, adj_blocks<SET>()) k_adj_cells(Params P, Shapes S, Parts D,
                                                                               Lists W, AdjBufs B) {
  __shared__ float4 s_pl[kAdjWarps][2][kMaxFaces + kMaxFaces / 4];   // planes, then their inverse slopes
  __shared__ __align__(16) PairRec s_rec[kAdjWarps][2];
  __shared__ unsigned s_pk[SET == 0 ? kAdjWarps : 1][kTileItemsPerLane * 32];   // clipped ranges (rolled sweep)
  __shared__ int4 s_own[kAdjWarps][64];   // the lanes with clipped nodes of the current tile
  constexpr bool ROLL = SET == 0;   // every kind: rolled slot loops (code size)
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ntiles = min(W.counters[1], P.max_tiles);
  const float inv_w = P.inv_w, hw = 0.5f * P.wdx_l, T = hw + kClipMargin;
  unsigned* spk = s_pk[ROLL ? wid : 0];
  // tiles w, w + W, ... of the forward's list (W warps): each record is staged
  // in shared memory, the next record and its pair's seeds are fetched while
  // a tile runs
  const int nwarps = gridDim.x * kAdjWarps;
  int qpos = blockIdx.x * kAdjWarps + wid;
  float seed = 0.f;
  if (qpos < ntiles) {
    const int4 v = adj_rec_part(W.tiles + qpos, lane);
    if (lane < kPairRecWords / 4) reinterpret_cast<int4*>(&s_rec[wid][0])[lane] = v;
    seed = adj_seed(B, checked_index(W.err, adj_rec_pair(v), P.max_pairs, 0), lane);
  }
  __syncwarp();
  int buf = 0;
  while (qpos < ntiles) {
    const int qn = qpos + nwarps;
    int4 next = make_int4(0, 0, 0, 0);
    float seed_n = 0.f;
    if (qn < ntiles) {
      next = adj_rec_part(W.tiles + qn, lane);
      seed_n = adj_seed(B, checked_index(W.err, adj_rec_pair(next), P.max_pairs, 0), lane);
    }
    const PairRec& r = s_rec[wid][buf];
    const bool valid = record_in_bounds(P, W.err, r, true);
    const bool active = valid && __any_sync(kFull, lane < 7 && seed != 0.f);
    const int p = r.pair;
    const int t = r.tile0 + r.tile;   // the tile's index (its partial slot)
    // the pair's pose gradient so far (explicit and depth terms), lane c < 12:
    // component c, read now for the sum added at the pair's end
    const double pgv = (active && lane < 12) ? B.pgrad[static_cast<size_t>(p) * kPairGrad + lane] : 0.0;
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.f;
    if (active) {
      const float s0 = __shfl_sync(kFull, seed, 0);
      const float s1[3] = {__shfl_sync(kFull, seed, 1), __shfl_sync(kFull, seed, 2), __shfl_sync(kFull, seed, 3)};
      const float sg[3] = {__shfl_sync(kFull, seed, 4), __shfl_sync(kFull, seed, 5), __shfl_sync(kFull, seed, 6)};
      int ai[3], bi[3];
      float af[3], bf[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ai[k] = r.ai[k]; bi[k] = r.bi[k];
        af[k] = r.af[k]; bf[k] = r.bf[k];
      }
      const int ax0 = r.axis, ax1 = ax0 == 2 ? 0 : ax0 + 1, ax2 = ax1 == 2 ? 0 : ax1 + 1;
      AdjGeom A, Bg;
      adj_load_rec(r, false, S, D, s_pl[wid][0], A, ax0);
      adj_load_rec(r, true, S, D, s_pl[wid][1], Bg, ax0);
      const float Tc = hw + kClipMargin;
      if (SET == 2 || A.type == 1) adj_prep_clip(A, ax0, ax1, ax2, Tc);
      if (SET == 2 || Bg.type == 1) adj_prep_clip(Bg, ax0, ax1, ax2, Tc);
      const int dm0 = r.dim[0], dm1 = r.dim[1], dm2 = r.dim[2];
      const int du = ax0 == 0 ? dm0 : (ax0 == 1 ? dm1 : dm2);
      const int dv = ax0 == 0 ? dm1 : (ax0 == 1 ? dm2 : dm0);   // side along (ax0 + 1) mod 3
      const float inv_dv = __fdividef(1.f, static_cast<float>(dv));
      const int nitems = r.nitems;
      // (A) lane l clips its lines it0 + 32 s + l; (B) the tile's clipped
      // nodes, numbered lane by lane by a scan of the counts, one per lane
      // (owner lane by a binary search over the scan, slot by the owner's
      // counts): the same node set as a walk of every line
      auto node = [&](int cu, int l1, int l2) {
        // node coordinates in box axes x, y, z (selects: no runtime-indexed array)
        int c[3];
        c[0] = ax0 == 0 ? cu : (ax0 == 1 ? l2 : l1);
        c[1] = ax0 == 1 ? cu : (ax0 == 2 ? l2 : l1);
        c[2] = ax0 == 2 ? cu : (ax0 == 0 ? l2 : l1);
        float ra[3], rb[3], ga[3], gb[3], na, nb;
        for (int k = 0; k < 3; ++k) {
          ra[k] = static_cast<float>(c[k] - ai[k]) - af[k];
          rb[k] = static_cast<float>(c[k] - bi[k]) - bf[k];
        }
        // every term below needs both phi inside the upper half of the band
        if (fmaxf(adj_phi<SET>(A, ra), adj_phi<SET>(Bg, rb)) >= hw) return;
        const float fa = adj_eval<SET>(A, ra, ga, &na);
        const float fb = adj_eval<SET>(Bg, rb, gb, &nb);
        const float ta = fminf(fmaxf(fmaf(fa, -inv_w, 0.5f), 0.f), 1.f);
        const float tb = fminf(fmaxf(fmaf(fb, -inv_w, 0.5f), 0.f), 1.f);
        const bool ina = ta > 0.f && ta < 1.f, inb = tb > 0.f && tb < 1.f;
        const float Ha = ta * ta * (3.f - 2.f * ta), Hb = tb * tb * (3.f - 2.f * tb);
        const float ha = ta * (1.f - ta), hb = tb * (1.f - tb);
        // derivatives with respect to phi (lattice units); zero outside the band
        const float dHa = ina ? -6.f * ha * inv_w : 0.f, dHb = inb ? -6.f * hb * inv_w : 0.f;
        const float dha = ina ? -(1.f - 2.f * ta) * inv_w : 0.f, dhb = inb ? -(1.f - 2.f * tb) * inv_w : 0.f;
        if (Ha * Hb == 0.f && ha * Hb == 0.f && Ha * hb == 0.f && dHa * Hb == 0.f && Ha * dHb == 0.f) return;
        const float sw = fmaf(s1[0], static_cast<float>(c[0]),
                              fmaf(s1[1], static_cast<float>(c[1]), fmaf(s1[2], static_cast<float>(c[2]), s0)));
        const float gma = sg[0] * ga[0] + sg[1] * ga[1] + sg[2] * ga[2];
        const float gmb = sg[0] * gb[0] + sg[1] * gb[1] + sg[2] * gb[2];
        const float ka = sw * dHa * Hb + dha * Hb * gma - dHa * hb * gmb;
        const float kb = sw * Ha * dHb + ha * dHb * gma - Ha * dhb * gmb;
        float xa[3], xb[3];
        cross3f(ga, ra, xa);
        cross3f(gb, rb, xb);
        for (int k = 0; k < 3; ++k) {
          acc[k] -= ka * ga[k];
          acc[3 + k] += ka * xa[k];
          acc[6 + k] -= kb * gb[k];
          acc[9 + k] += kb * xb[k];
        }
        const float wa = ha * Hb, wb = Ha * hb;
        if (SET != 2 && A.type == 0) {
          if (na > 0.f)
            for (int k = 0; k < 3; ++k) acc[k] -= wa * (sg[k] - gma * ga[k]) / na;
        } else {
          float cr[3];
          cross3f(ga, sg, cr);
          for (int k = 0; k < 3; ++k) acc[3 + k] += wa * cr[k];
        }
        if (SET != 2 && Bg.type == 0) {
          if (nb > 0.f)
            for (int k = 0; k < 3; ++k) acc[6 + k] += wb * (sg[k] - gmb * gb[k]) / nb;
        } else {
          float cr[3];
          cross3f(gb, sg, cr);
          for (int k = 0; k < 3; ++k) acc[9 + k] -= wb * cr[k];
        }
      };
      const int it0 = r.tile * 32 * kTileItemsPerLane;
      const int ns = min(kTileItemsPerLane, (nitems - it0 + 31) >> 5);
      unsigned pk[kTileItemsPerLane];
      int nl = 0;
#pragma unroll(ROLL ? 1 : kTileItemsPerLane)
      for (int s = 0; s < kTileItemsPerLane; ++s) {
        if (!ROLL) pk[s] = 0u;
        if (s < ns) {
          const int it = it0 + s * 32 + lane;
          int l1;
          const int l2 = div_small(it, dv, inv_dv, &l1);   // coordinates along axes ax1, ax2
          const int u1 = it < nitems ? du : 0;
          float clo = 0.f, chi = static_cast<float>(u1 - 1);
          adj_clip<SET>(A, ax0, ax1, ax2, l1, l2, ai, af, T, clo, chi);
          adj_clip<SET>(Bg, ax0, ax1, ax2, l1, l2, bi, bf, T, clo, chi);
          int ub;
          const int nk = clip_nodes(clo, chi, 0, u1, &ub);
          const unsigned v = static_cast<unsigned>(ub) | (static_cast<unsigned>(nk) << 16);
          if constexpr (ROLL) spk[s * 32 + lane] = v;
          else pk[s] = v;
          nl += nk;
        }
      }
      if (ROLL) __syncwarp();
      int incl = nl;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += v;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      const int excl = incl - nl;
      // the lanes with nodes in lane order: entry k of own holds the k-th
      // one's lane, first node and clipped ranges
      const bool has = nl > 0;
      int4* own = s_own[wid];
      if (total > 0) {
        const int rank = __popc(__ballot_sync(kFull, has) & ((1u << lane) - 1u));
        if (has) {
          if constexpr (ROLL) {
            own[rank] = make_int4(lane, excl, 0, 0);
          } else {
            static_assert(kTileItemsPerLane == 4, "own holds four clipped ranges per lane");
            own[rank] = make_int4(lane, excl, static_cast<int>(pk[0]), static_cast<int>(pk[1]));
            own[32 + rank] = make_int4(static_cast<int>(pk[2]), static_cast<int>(pk[3]), 0, 0);
          }
        }
        __syncwarp();
      }
      for (int base = 0; base < total; base += 32) {
        const int g = base + lane;
        // owner: the last lane with nodes whose first node is <= g
        const unsigned before = __ballot_sync(kFull, has && excl < base);
        const unsigned inside =
            __reduce_or_sync(kFull, (has && excl >= base && excl - base < 32) ? 1u << (excl - base) : 0u);
        const int cnt_le = __popc(before) + __popc(inside & (lane == 31 ? 0xffffffffu : (2u << lane) - 1u));
        const int ie = min(max(cnt_le - 1, 0), 31);
        const int4 e = own[ie];
        const int o = e.x;
        int k = g - e.y;   // the node's rank among the owner's
        int4 e2 = make_int4(0, 0, 0, 0);
        if (!ROLL) e2 = own[32 + ie];
        int os = 0, cu = 0;
#pragma unroll(ROLL ? 1 : kTileItemsPerLane)
        for (int s = 0; s < kTileItemsPerLane; ++s) {
          if (s < ns) {
            unsigned q;
            if constexpr (ROLL) q = spk[s * 32 + o];
            else q = static_cast<unsigned>(s == 0 ? e.z : (s == 1 ? e.w : (s == 2 ? e2.x : e2.y)));
            const int n = static_cast<int>(q >> 16);
            if (k >= 0 && k < n) {
              os = s;
              cu = static_cast<int>(q & 0xffffu) + k;
            }
            k -= n;
          }
        }
        int ol1;
        const int ol2 = div_small(it0 + os * 32 + o, dv, inv_dv, &ol1);
        if (g < total) node(cu, ol1, ol2);
      }
      if (ROLL) __syncwarp();   // spk is rewritten by the next tile
    }
    const float x = adj_warp_sum12(acc);   // lane c < 12: component c
    if (active) {
      // end of the pair: one tile -> its sums directly; several -> the warp
      // completing the last tile sums all partials in FP64 (fixed order)
      bool complete = true;
      double sum = 0.0;   // lane c < 12: component c
      const int ntp = r.ntiles, tile0 = r.tile0;
      if (ntp == 1) {
        sum = widen(x);
      } else {
        if (lane < 12) B.partial[static_cast<size_t>(t) * kAdjPartial + lane] = x;
        __threadfence();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(&B.done[p], 1);
        prev = __shfl_sync(kFull, prev, 0);
        complete = prev == ntp - 1;
        if (complete) {
          __threadfence();
          const int slot = lane >> 4, c = lane & 15;   // component c < 12 of tiles slot, slot + 2, ...
          for (int tb = 0; tb < ntp; tb += 16) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int tt = tb + slot + 2 * u;
              v[u] = (tt < ntp && c < 12) ? __ldcg(B.partial + static_cast<size_t>(tile0 + tt) * kAdjPartial + c) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += widen(v[u]);
          }
          sum += __shfl_xor_sync(kFull, sum, 16);
        }
      }
      if (complete && lane < 12) {   // cell sums in lattice units -> physical (positions / dx)
        const bool pos_part = lane < 3 || (lane >= 6 && lane < 9);
        B.pgrad[static_cast<size_t>(p) * kPairGrad + lane] = pgv + (pos_part ? sum * P.inv_dx : sum);
      }
    }
    __syncwarp();
    if (qn < ntiles && lane < kPairRecWords / 4) reinterpret_cast<int4*>(&s_rec[wid][buf ^ 1])[lane] = next;
    __syncwarp();
    buf ^= 1;
    qpos = qn;
    seed = seed_n;
  }
}

// Per particle and component (eight lanes per particle, six used), FP64 adds
// in the forward order: the pairs where the particle is j (by i), then the
// pairs where it is i (by j); lane 0 of each group then maps the rotation
// gradient to the raw quaternion.
__global__ void __launch_bounds__(32) k_adj_scatter(Params P, Parts D, Lists W, AdjBufs B,
                                                    double* __restrict__ gpos, double* __restrict__ gquat) {
  pdl_begin();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, g0 = lane & ~7;
  const int p0 = t >> 3, c = t & 7;
  const bool ok = p0 < P.n;
  const int p = ok ? p0 : P.n - 1;
  const int np = min(W.counters[0], P.max_pairs);
  double acc = 0.0;
  if (ok && c < 6) {
    // contributions in order (j side, then i side), eight loads in flight at a time
    const int* dp = W.dn_pair + static_cast<size_t>(p) * P.max_nbr;
    const int nd = W.dn_count[p], r0 = W.row_off[p], nu = W.up_count[p];
    const int total = nd + nu;
    for (int base = 0; base < total; base += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = base + u;
        const bool isj = e < nd;   // p is the pair's j: columns 6..11; else its i: columns 0..5
        int q = isj ? dp[e] : (e < total ? r0 + (e - nd) : np);
        if (e < total) q = checked_index(W.err, q, np, -1);
        v[u] = (q >= 0 && q < np) ? B.pgrad[static_cast<size_t>(q) * kPairGrad + (isj ? 6 + c : c)] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (base + u < total) acc += v[u];
    }
  }
  double tau[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) tau[k] = __shfl_sync(kFull, acc, g0 + 3 + k);
  if (!ok) return;
  if (c < 3) gpos[3 * p + c] = acc;
  if (c == 0) {
    const double* qr = D.qhat + 4 * p;
    const double iq = fl::nr_rsqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
    const double w = qr[0] * iq, v[3] = {qr[1] * iq, qr[2] * iq, qr[3] * iq};
    const double s2 = 2.0 * iq;
    double tv[3];
    cross3(tau, v, tv);
    gquat[4 * p] = -s2 * (v[0] * tau[0] + v[1] * tau[1] + v[2] * tau[2]);
    for (int k = 0; k < 3; ++k) gquat[4 * p + 1 + k] = s2 * (w * tau[k] + tv[k]);
  }
}

}  // namespace

size_t adjoint_scratch_doubles(int max_pairs, int max_tiles) {
  return static_cast<size_t>(max_tiles) * kAdjPartial / 2 + static_cast<size_t>(max_pairs) * kSeedFloats / 2 +
         static_cast<size_t>(max_pairs) * kPairGrad + static_cast<size_t>(max_pairs) / 2 + 16;
}

// ev0 / ev1 (nullable): events recorded around the cell sweep's launch.
void launch_adjoint(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                    const double* gF, const double* gT, double* gpos, double* gquat, double* scratch, int grid,
                    cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
  AdjBufs B;
  B.partial = reinterpret_cast<float*>(scratch);
  B.seeds = B.partial + static_cast<size_t>(P.max_tiles) * kAdjPartial;
  B.pgrad = reinterpret_cast<double*>(B.seeds + static_cast<size_t>(P.max_pairs) * kSeedFloats + 8);
  B.done = reinterpret_cast<int*>(B.pgrad + static_cast<size_t>(P.max_pairs) * kPairGrad);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int wneed0 = (P.max_pairs + 7) / 8;   // pre: eight pairs per warp pass
  const int wgrid0 = wneed0 < 8 * sms ? (wneed0 > 0 ? wneed0 : 1) : 8 * sms;
  launch_pdl(k_adj_pre, dim3(wgrid0), dim3(32), 0, st, P, S, D, W, B, vel, gF, gT);
  // compiled per kind set, as the node sweep (2 cubes only, 1 spheres / cuboids / walls, 0 every kind)
  auto cells = P.kind_set == 2 ? k_adj_cells<2> : (P.kind_set == 1 ? k_adj_cells<1> : k_adj_cells<0>);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cells, kAdjWarps * 32, 0);
  const int cgrid = (per_sm > 0 ? per_sm : 1) * sms;   // persistent: every resident slot pulls tiles
  (void)grid;
  if (ev0 != nullptr) cudaEventRecord(ev0, st);
  launch_pdl(cells, dim3(cgrid), dim3(kAdjWarps * 32), 0, st, P, S, D, W, B);
  if (ev1 != nullptr) cudaEventRecord(ev1, st);
  launch_pdl(k_adj_scatter, dim3((8 * P.n + 31) / 32), dim3(32), 0, st, P, D, W, B, gpos, gquat);
}

}  // namespace gbc
