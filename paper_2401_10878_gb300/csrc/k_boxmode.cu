// The paper's own box pipeline (Sec. 3.3.1 of arXiv:2401.10878): rough
// contact detection on the lattice, correction of the bounding box, and the
// final sweep of N_c points per direction over the corrected box.
//
//   1. rough detection: the lattice nodes where both signed distances are
//      below half the cell diagonal, sqrt(0.75) dx; their node-index bounds
//      form the rough box (none: no contact).  The node ranges of this mode
//      are widened by that threshold, so the pair box holds all such nodes.
//   2. correction: the rough box widened by sqrt(0.75) dx (every point inside
//      both shapes lies within that distance of such a node) is B0; on each of
//      its six faces an N_c x N_c grid of points (the face's cell centres)
//      casts lines along the inward normal; a line's entry into the overlap
//      (the line clipped exactly against both shapes) is its distance to the
//      contact, and the face moves inward by the smallest one (a face whose
//      lines all miss stays; an axis left empty keeps B0's extent).
//   3. the N_c^3 cell centres of the corrected box are the sample points of
//      the overlap volume, contact point, normal and depth (the lattice
//      path's estimators, each sample weighing its cell's volume), then the
//      force law of Eq. (contact_force_normal).
//
// One warp per pair, pulled from a queue over the pairs the pair builder
// keeps: pairs whose regions at the rough threshold are apart (separating
// axes of two boxes, the distance tests of balls) have no rough-contact node
// and get their zero outputs there, and two boxes' node box is cut to the
// bounding box of their regions' intersection.  The node tests, the line
// clipping and the sample sweep run in FP32 relative to the particle centres
// (offsets formed in FP64); each face's nearest line is re-clipped in FP64,
// so the corrected box carries no FP32 error; the pair sums, the depth at the
// deepest sample and the force law are FP64.
#include <cfloat>
#include <climits>

#include "contact_dev.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBoxWarps = 8;

// One shape of the pair in FP32, lattice units: centre relative to the pair
// box origin, R^T rows, sizes (inflate included), world planes (polytope),
// plane value at the box origin (wall).
struct ShapeF {
  int kind;
  float c[3];
  float rt[9];
  float sz[3];
  const float4* pl;
  int nf;
};

__device__ __forceinline__ void load_shape(const PairRec& r, bool second, const Shapes& S, const Parts& D, int pid,
                                           float4* sm, ShapeF& s) {
  const int lane = threadIdx.x & 31;
  s.kind = second ? (r.kinds >> 8) : (r.kinds & 0xff);
  const int* ci = second ? r.bi : r.ai;
  const float* cf = second ? r.bf : r.af;
  const float* rt = second ? r.rtb : r.rta;
  const float* sz = second ? r.szb : r.sza;
  for (int k = 0; k < 3; ++k) {
    s.c[k] = static_cast<float>(ci[k]) + cf[k];
    s.sz[k] = sz[k];
  }
  for (int k = 0; k < 9; ++k) s.rt[k] = rt[k];
  s.nf = 0;
  s.pl = sm;
  if (s.kind == KIND_POLY) {
    const int f0 = S.face_off[pid];
    s.nf = S.face_off[pid + 1] - f0;
    if (lane < s.nf) sm[lane] = D.wplane[f0 + lane];
    __syncwarp();
  }
}

// Signed distance (lattice units) at q = point - centre, and the world
// gradient of the active branch (first maximal face).  SET is the context's
// kind set (2: cubes only, 1: spheres, cuboids and walls, 0: every kind): the
// kinds a set cannot hold are compiled out.
template <int SET>
__device__ __forceinline__ float phi_f(const ShapeF& s, const float q[3], float g[3]) {
  if (SET != 2 && s.kind == KIND_SPHERE) {
    const float n2 = fmaf(q[0], q[0], fmaf(q[1], q[1], q[2] * q[2]));
    const float nr = sqrtf(n2);
    const float inv = nr > 0.f ? 1.f / nr : 0.f;
    for (int k = 0; k < 3; ++k) g[k] = q[k] * inv;
    return nr - s.sz[0];
  }
  if (SET != 2 && s.kind == KIND_WALL) {   // q = box-relative point; sz[0] = value at the box origin
    for (int k = 0; k < 3; ++k) g[k] = s.rt[k];
    return fmaf(s.rt[0], q[0], fmaf(s.rt[1], q[1], fmaf(s.rt[2], q[2], s.sz[0])));
  }
  if (SET != 0 || s.kind == KIND_CUBOID || s.kind == KIND_CUBE) {
    float best = -FLT_MAX;
    int kk = 0;
    float sg = 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float y = fmaf(s.rt[3 * k], q[0], fmaf(s.rt[3 * k + 1], q[1], s.rt[3 * k + 2] * q[2]));
      const float a = fabsf(y) - s.sz[k];
      if (a > best) { best = a; kk = k; sg = y < 0.f ? -1.f : 1.f; }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = sg * (kk == 0 ? s.rt[k] : (kk == 1 ? s.rt[3 + k] : s.rt[6 + k]));
    return best;
  }
  float best = -FLT_MAX;
  int kk = 0;
  for (int f = 0; f < s.nf; ++f) {
    const float4 e = s.pl[f];
    const float v = fmaf(e.x, q[0], fmaf(e.y, q[1], fmaf(e.z, q[2], -e.w)));
    if (v > best) { best = v; kk = f; }
  }
  const float4 e = s.pl[kk];
  g[0] = e.x; g[1] = e.y; g[2] = e.z;
  return best;
}

// Interval [t0, t1] of the line q + t e (q = start - centre, e = +-axis k)
// inside the shape, FP32 (empty: t0 > t1); SET as for phi_f.
template <int SET>
__device__ __forceinline__ void clip_f(const ShapeF& s, const float q[3], int k, float sgn, float* t0, float* t1) {
  *t0 = -FLT_MAX;
  *t1 = FLT_MAX;
  auto plane = [&](float n0, float n1, float n2, float off) {
    const float a = fmaf(n0, q[0], fmaf(n1, q[1], fmaf(n2, q[2], -off)));
    const float b = sgn * (k == 0 ? n0 : (k == 1 ? n1 : n2));
    if (b > 0.f) *t1 = fminf(*t1, -a / b);
    else if (b < 0.f) *t0 = fmaxf(*t0, -a / b);
    else if (a > 0.f) { *t0 = FLT_MAX; *t1 = -FLT_MAX; }
  };
  if (SET != 2 && s.kind == KIND_SPHERE) {
    const float b = sgn * (k == 0 ? q[0] : (k == 1 ? q[1] : q[2]));
    const float c = fmaf(q[0], q[0], fmaf(q[1], q[1], q[2] * q[2])) - s.sz[0] * s.sz[0];
    const float disc = b * b - c;
    if (disc < 0.f) { *t0 = FLT_MAX; *t1 = -FLT_MAX; return; }
    const float sq = sqrtf(disc);
    *t0 = -b - sq;
    *t1 = -b + sq;
    return;
  }
  if (SET != 2 && s.kind == KIND_WALL) {
    plane(s.rt[0], s.rt[1], s.rt[2], -s.sz[0]);
    return;
  }
  if (SET != 0 || s.kind == KIND_CUBOID || s.kind == KIND_CUBE) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      plane(s.rt[3 * a], s.rt[3 * a + 1], s.rt[3 * a + 2], s.sz[a]);
      plane(-s.rt[3 * a], -s.rt[3 * a + 1], -s.rt[3 * a + 2], s.sz[a]);
    }
    return;
  }
  for (int f = 0; f < s.nf; ++f) {
    const float4 e = s.pl[f];
    plane(e.x, e.y, e.z, e.w);
  }
}

// FP64 interval of the line p + t e (physical units) inside particle / wall
// `pid`, the same clipping as the FP32 form; used for each face's nearest
// line.  The bounds -a/b of the face planes are compared as fractions (b
// carries the sign), so only the two winning ones are divided.
__device__ void clip_d(const Params& P, const Shapes& S, const Parts& D, int pid, const double X[3], const double p[3],
                       int k, double sgn, double* t0, double* t1) {
  const int type = S.type[pid];
  const double* R = D.R + 9 * static_cast<size_t>(pid);
  if (type == 0) {   // sphere
    const double r = S.param[3 * pid] + P.inflate;
    const double q0 = p[0] - X[0], q1 = p[1] - X[1], q2 = p[2] - X[2];
    const double b = sgn * (k == 0 ? q0 : (k == 1 ? q1 : q2));
    const double c = (q0 * q0 + q1 * q1 + q2 * q2) - r * r;
    const double disc = b * b - c;
    if (disc < 0.0) { *t0 = DBL_MAX; *t1 = -DBL_MAX; return; }
    const double sq = sqrt(disc);
    *t0 = -b - sq;
    *t1 = -b + sq;
    return;
  }
  // lower bound -a0/b0 (b0 < 0), upper bound -a1/b1 (b1 > 0); none yet: b = 0
  double a0 = 0.0, b0 = 0.0, a1 = 0.0, b1 = 0.0;
  bool empty = false;
  // the half-line a + b t <= 0 of one face along the line
  auto bound = [&](double a, double b) {
    if (b > 0.0) {   // t <= -a/b: keep the smaller, -a/b < -a1/b1  <=>  a b1 > a1 b
      if (b1 == 0.0 || a * b1 > a1 * b) { a1 = a; b1 = b; }
    } else if (b < 0.0) {   // t >= -a/b: keep the larger, -a/b > -a0/b0  <=>  a b0 < a0 b (b b0 > 0)
      if (b0 == 0.0 || a * b0 < a0 * b) { a0 = a; b0 = b; }
    } else if (a > 0.0) {
      empty = true;
    }
  };
  auto plane = [&](double n0, double n1, double n2, double off) {
    bound(((n0 * p[0] + n1 * p[1]) + n2 * p[2]) - off, sgn * (k == 0 ? n0 : (k == 1 ? n1 : n2)));
  };
  if (type == 1) {   // cuboid: faces +-R e_a share n = R e_a and d = n . (p - X)
    const double q0 = p[0] - X[0], q1 = p[1] - X[1], q2 = p[2] - X[2];
    for (int a = 0; a < 3; ++a) {
      const double n0 = R[a], n1 = R[3 + a], n2 = R[6 + a];
      const double d = (n0 * q0 + n1 * q1) + n2 * q2;
      const double h = S.param[3 * pid + a] + P.inflate;
      const double b = sgn * (k == 0 ? n0 : (k == 1 ? n1 : n2));
      bound(d - h, b);     // n . (x - X) <= h
      bound(-d - h, -b);   // -n . (x - X) <= h
    }
  } else {   // polytope, or a wall's single plane
    const int f0 = S.face_off[pid], nf = S.face_off[pid + 1] - f0;
    for (int f = 0; f < nf; ++f) {
      const double* b = S.planes + 4 * (f0 + f);
      const double n0 = (R[0] * b[0] + R[1] * b[1]) + R[2] * b[2];
      const double n1 = (R[3] * b[0] + R[4] * b[1]) + R[5] * b[2];
      const double n2 = (R[6] * b[0] + R[7] * b[1]) + R[8] * b[2];
      plane(n0, n1, n2, ((n0 * X[0] + n1 * X[1]) + n2 * X[2]) + b[3] + P.inflate);
    }
  }
  if (empty) { *t0 = DBL_MAX; *t1 = -DBL_MAX; return; }
  *t0 = b0 != 0.0 ? -a0 / b0 : -DBL_MAX;
  *t1 = b1 != 0.0 ? -a1 / b1 : DBL_MAX;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ void zero_pair(const Lists& W, double* pair_out, int q) {
  const int lane = threadIdx.x & 31;
  if (lane < 11) pair_out[static_cast<size_t>(q) * 11 + lane] = 0.0;
  if (lane < kFtDoubles) W.ft[static_cast<size_t>(q) * kFtDoubles + lane] = 0.0;
  if (lane < kTapeDoubles) W.tape[static_cast<size_t>(q) * kTapeDoubles + lane] = 0.0;
}

template <int SET>
__global__ void __launch_bounds__(kBoxWarps * 32, 2) k_box_pairs(Params P, Shapes S, Parts D, Lists W,
                                                              const double* __restrict__ vel,
                                                              double* __restrict__ pair_out) {
  __shared__ float4 s_pl[kBoxWarps][2][kMaxFaces];
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the pairs the pair builder kept (one entry of the tile list each; the
  // others are apart at the rough threshold and have their zero outputs)
  const int ntl = W.counters[1];
  if (ntl > P.max_tiles) return;   // capacity exceeded: the step reports ECAPACITY
  const int Nc = P.box_res;
  const float srough = kRoughT;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&W.counters[2], 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= ntl) break;
    const PairRec& r = W.tiles[t];
    if (!record_in_bounds(P, W.err, r, true)) continue;   // warp-uniform (checked build only)
    const int q = r.pair;
    const int i = r.i, j = r.j;
    const int d0 = r.dim[0], d1 = r.dim[1], d2 = r.dim[2];
    ShapeF A, B;
    load_shape(r, false, S, D, i, s_pl[wid][0], A);
    load_shape(r, true, S, D, j, s_pl[wid][1], B);
    // 1. rough detection over the pair box's nodes (box-relative node c)
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    const int vol = d0 * d1 * d2;
    for (int n0 = 0; n0 < vol; n0 += 32) {
      const int n = n0 + lane;
      if (n < vol) {
        const int c[3] = {n % d0, (n / d0) % d1, n / (d0 * d1)};
        float qa[3], qb[3], g[3];
        for (int k = 0; k < 3; ++k) {
          qa[k] = static_cast<float>(c[k] - r.ai[k]) - r.af[k];
          qb[k] = B.kind == KIND_WALL ? static_cast<float>(c[k]) : static_cast<float>(c[k] - r.bi[k]) - r.bf[k];
        }
        if (phi_f<SET>(A, qa, g) < srough && phi_f<SET>(B, qb, g) < srough)
          for (int k = 0; k < 3; ++k) {
            mn[k] = min(mn[k], c[k]);
            mx[k] = max(mx[k], c[k]);
          }
      }
    }
    for (int k = 0; k < 3; ++k) {
      mn[k] = __reduce_min_sync(kFull, mn[k]);
      mx[k] = __reduce_max_sync(kFull, mx[k]);
    }
    if (mn[0] > mx[0]) {
      zero_pair(W, pair_out, q);
      continue;
    }
    // 2. B0 (physical, as the rough box's nodes +- sqrt(0.75) dx), then the lines
    const double s64 = sqrt(0.75) * P.dx;
    double b0lo[3], b0hi[3];
    for (int k = 0; k < 3; ++k) {
      b0lo[k] = (r.lo[k] + mn[k]) * P.dx - s64;
      b0hi[k] = (r.lo[k] + mx[k]) * P.dx + s64;
    }
    double XA[3], XB[3];
    for (int k = 0; k < 3; ++k) {
      XA[k] = D.X[3 * i + k];
      XB[k] = D.X[3 * j + k] - r.shift[k] * P.L[k];
    }
    // contact history (Sec. 4.3.3): is (i, j) an ongoing contact?  Its c, and
    // its last corrected box (relative to X_i) as the warm start: moved with
    // particle i and widened by sqrt(0.75) dx, it cuts B0 down per axis
    // (unless the cut leaves nothing)
    size_t hslot = 0;
    int hit = -1;
    double c_hist = 0.0;
    if (P.history) {
      const int rd = W.counters[kStepCounter] & 1;
      const size_t base = (static_cast<size_t>(rd) * P.n + i) * P.max_nbr;
      const int cnt = min(W.hist_n[static_cast<size_t>(rd) * P.n + i], P.max_nbr);
      for (int m = lane; m < cnt; m += 32)
        if (W.hist_j[base + m] == j) hit = m;
      hit = __reduce_max_sync(kFull, hit);
      if (hit >= 0) {
        hslot = base + hit;
        c_hist = W.hist_c[hslot];
        const double* wb = W.hist_box + 6 * hslot;
        for (int k = 0; k < 3; ++k) {
          const double wl = __dsub_rn(__dadd_rn(XA[k], wb[k]), s64), wh = __dadd_rn(__dadd_rn(XA[k], wb[3 + k]), s64);
          const double l = fmax(b0lo[k], wl), h = fmin(b0hi[k], wh);
          if (l < h) {
            b0lo[k] = l;
            b0hi[k] = h;
          }
        }
      }
    }
    // per face: the FP32 nearest line (line starts as FP32 offsets from each
    // centre: the face corner formed in FP64, plus the line's position on the
    // face), then lane f re-clips face f's nearest line in FP64
    const int nl = Nc * Nc;
    const double inv_nc = 1.0 / Nc;
    unsigned my_key = 0xffffffffu;
    int my_line = 0;
    auto sel = [](const double* a, int c) { return c == 0 ? a[0] : (c == 1 ? a[1] : a[2]); };
    // each face's line geometry in FP64 once, face f on lane f (the FP64 pipe
    // takes a warp instruction's time however few lanes it has): the corner's
    // offsets from both centres, the line spacings and the line length, as FP32
    float fca[3] = {0.f, 0.f, 0.f}, fcb[3] = {0.f, 0.f, 0.f}, fdu = 0.f, fdv = 0.f, flen = 0.f;
    if (lane < 6) {
      const int k = lane >> 1, side = lane & 1;
      const int u = k == 0 ? 1 : 0, v = k == 2 ? 1 : 2;
      const double corner[3] = {k == 0 ? (side == 0 ? b0lo[0] : b0hi[0]) : b0lo[0],
                                k == 1 ? (side == 0 ? b0lo[1] : b0hi[1]) : b0lo[1],
                                k == 2 ? (side == 0 ? b0lo[2] : b0hi[2]) : b0lo[2]};
      for (int c = 0; c < 3; ++c) {
        fca[c] = static_cast<float>((corner[c] - XA[c]) * P.inv_dx);
        fcb[c] = B.kind == KIND_WALL ? static_cast<float>(corner[c] * P.inv_dx - r.lo[c])
                                     : static_cast<float>((corner[c] - XB[c]) * P.inv_dx);
      }
      fdu = static_cast<float>((sel(b0hi, u) - sel(b0lo, u)) * (P.inv_dx * inv_nc));
      fdv = static_cast<float>((sel(b0hi, v) - sel(b0lo, v)) * (P.inv_dx * inv_nc));
      flen = static_cast<float>((sel(b0hi, k) - sel(b0lo, k)) * P.inv_dx);
    }
    for (int f = 0; f < 6; ++f) {
      const int k = f >> 1, side = f & 1;
      const float sgn = side == 0 ? 1.f : -1.f;
      const float ca[3] = {__shfl_sync(kFull, fca[0], f), __shfl_sync(kFull, fca[1], f), __shfl_sync(kFull, fca[2], f)};
      const float cb[3] = {__shfl_sync(kFull, fcb[0], f), __shfl_sync(kFull, fcb[1], f), __shfl_sync(kFull, fcb[2], f)};
      const float du = __shfl_sync(kFull, fdu, f), dv = __shfl_sync(kFull, fdv, f);
      const float lenl = __shfl_sync(kFull, flen, f);
      const int u = k == 0 ? 1 : 0, v = k == 2 ? 1 : 2;
      float best = FLT_MAX;
      int bestl = 0x7fffffff;
      for (int l0 = 0; l0 < nl; l0 += 32) {
        const int l = l0 + lane;
        if (l < nl) {
          const int a = l / Nc, b = l - a * Nc;
          const float ou = (static_cast<float>(a) + 0.5f) * du, ov = (static_cast<float>(b) + 0.5f) * dv;
          // (selects, not a runtime index: the arrays stay in registers)
          const float o0 = u == 0 ? ou : (v == 0 ? ov : 0.f), o1 = u == 1 ? ou : (v == 1 ? ov : 0.f);
          const float o2 = u == 2 ? ou : (v == 2 ? ov : 0.f);
          const float qa[3] = {ca[0] + o0, ca[1] + o1, ca[2] + o2}, qb[3] = {cb[0] + o0, cb[1] + o1, cb[2] + o2};
          float a0, a1, c0, c1;
          clip_f<SET>(A, qa, k, sgn, &a0, &a1);
          clip_f<SET>(B, qb, k, sgn, &c0, &c1);
          const float tin = fmaxf(fmaxf(a0, c0), 0.f);
          const float tout = fminf(fminf(a1, c1), lenl);
          if (tin <= tout && tin < best) { best = tin; bestl = l; }
        }
      }
      // the face's nearest line (first index on ties): t >= 0, so the bits order as the values
      const unsigned key = best < FLT_MAX ? __float_as_uint(best) : 0xffffffffu;
      const unsigned kmin = __reduce_min_sync(kFull, key);
      const int lmin = __reduce_min_sync(kFull, key == kmin ? bestl : 0x7fffffff);
      if (lane == f) {
        my_key = kmin;
        my_line = lmin;
      }
    }
    double my_shift = 0.0;
    if (lane < 6 && my_key != 0xffffffffu) {
      const int f = lane, k = f >> 1, side = f & 1;
      const int u = k == 0 ? 1 : 0, v = k == 2 ? 1 : 2;
      const int a = my_line / Nc, b = my_line - a * Nc;
      double p[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double ic = c == u ? a + 0.5 : b + 0.5;
        p[c] = c == k ? (side == 0 ? b0lo[c] : b0hi[c]) : b0lo[c] + ic * (b0hi[c] - b0lo[c]) * inv_nc;
      }
      double a0, a1, c0, c1;
      clip_d(P, S, D, i, XA, p, k, side == 0 ? 1.0 : -1.0, &a0, &a1);
      clip_d(P, S, D, j, XB, p, k, side == 0 ? 1.0 : -1.0, &c0, &c1);
      const double len = sel(b0hi, k) - sel(b0lo, k);
      const double tin = fmax(fmax(a0, c0), 0.0);
      const double tout = fmin(fmin(a1, c1), len);
      my_shift = tin <= tout ? tin : static_cast<double>(__uint_as_float(my_key)) * P.dx;
    }
    double shift_face[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) shift_face[f] = __shfl_sync(kFull, my_shift, f);
    double lo1[3], hi1[3], step[3];
    for (int k = 0; k < 3; ++k) {
      double l = b0lo[k] + shift_face[2 * k], h = b0hi[k] - shift_face[2 * k + 1];
      if (!(l <= h)) {
        l = b0lo[k];
        h = b0hi[k];
      }
      lo1[k] = l;
      hi1[k] = h;
      step[k] = (h - l) * inv_nc;
    }
    // 3. the N_c^3 sample points: offsets from each centre (and the box origin) in FP64, rounded once
    // (component k on lane k, then shared)
    float loA = 0.f, loB = 0.f, lst = 0.f;
    if (lane < 3) {
      const double lk = sel(lo1, lane), sk = sel(step, lane), xa = sel(XA, lane), xb = sel(XB, lane);
      const int rlo = lane == 0 ? r.lo[0] : (lane == 1 ? r.lo[1] : r.lo[2]);
      const double c0 = lk + 0.5 * sk;
      loA = static_cast<float>((c0 - xa) * P.inv_dx);
      loB = B.kind == KIND_WALL ? static_cast<float>(c0 * P.inv_dx - rlo) : static_cast<float>((c0 - xb) * P.inv_dx);
      lst = static_cast<float>(sk * P.inv_dx);
    }
    float oA[3], oB[3], st[3];
    for (int k = 0; k < 3; ++k) {
      oA[k] = __shfl_sync(kFull, loA, k);
      oB[k] = __shfl_sync(kFull, loB, k);
      st[k] = __shfl_sync(kFull, lst, k);
    }
    const float inv_w = P.inv_w, hw = 0.5f * P.wdx_l;
    float cnt = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, bestf = -FLT_MAX;
    int bestidx = 0x7fffffff;
    const int ns = Nc * Nc * Nc;
    for (int s0 = 0; s0 < ns; s0 += 32) {
      const int sidx = s0 + lane;
      if (sidx >= ns) continue;
      const int ix = sidx % Nc, iy = (sidx / Nc) % Nc, iz = sidx / (Nc * Nc);
      const float t[3] = {static_cast<float>(ix), static_cast<float>(iy), static_cast<float>(iz)};
      float qa[3], qb[3], ga[3], gb[3];
      for (int k = 0; k < 3; ++k) {
        qa[k] = fmaf(t[k], st[k], oA[k]);
        qb[k] = fmaf(t[k], st[k], oB[k]);
      }
      const float fa = phi_f<SET>(A, qa, ga), fb = phi_f<SET>(B, qb, gb);
      if (fmaxf(fa, fb) >= hw) continue;   // no weight and no band term
      const float ta = __saturatef(fmaf(fa, -inv_w, 0.5f)), tb = __saturatef(fmaf(fb, -inv_w, 0.5f));
      float w, ma, mb;
      if (P.smooth) {
        const float ha = ta * ta * fmaf(-2.f, ta, 3.f), hb = tb * tb * fmaf(-2.f, tb, 3.f);
        w = ha * hb;
        ma = fmaf(-ta, ta, ta) * hb;
        mb = ha * fmaf(-tb, tb, tb);
      } else {
        w = (fa <= 0.f && fb <= 0.f) ? 1.f : 0.f;
        ma = fb <= 0.f ? fmaf(-ta, ta, ta) : 0.f;
        mb = fa <= 0.f ? fmaf(-tb, tb, tb) : 0.f;
      }
      cnt += w;   // moments of the sample indices (exact integers in sharp mode)
      m0 = fmaf(w, t[0], m0);
      m1 = fmaf(w, t[1], m1);
      m2 = fmaf(w, t[2], m2);
      g0 += ma * ga[0] - mb * gb[0];
      g1 += ma * ga[1] - mb * gb[1];
      g2 += ma * ga[2] - mb * gb[2];
      const float f = -(fa + fb);
      if (w > 0.f && (f > bestf || (f == bestf && sidx < bestidx))) { bestf = f; bestidx = sidx; }
    }
    cnt = warp_sum_f(cnt);
    m0 = warp_sum_f(m0); m1 = warp_sum_f(m1); m2 = warp_sum_f(m2);
    g0 = warp_sum_f(g0); g1 = warp_sum_f(g1); g2 = warp_sum_f(g2);
    {
      const int bk = __float_as_int(bestf);   // order-preserving key (-FLT_MAX: no sample, the lowest)
      const int key = bk >= 0 ? bk : (bk ^ 0x7fffffff);
      const int kmax = __reduce_max_sync(kFull, key);
      bestidx = __reduce_min_sync(kFull, key == kmax ? bestidx : 0x7fffffff);
    }
    if (!(cnt > 0.f)) {
      zero_pair(W, pair_out, q);
      continue;
    }
    // 4. FP64 pair results and the force law: component k of every vector on
    // lane k < 3 (cross and dot products by shuffles; every FP64 warp
    // instruction costs the same however few lanes it has), the distances of
    // A and B at the deepest sample on lanes 0 and 1; the scalars on every lane
    {
      const int kc = lane < 3 ? lane : 0;
      const int k1 = kc == 2 ? 0 : kc + 1, k2 = k1 == 2 ? 0 : k1 + 1;
      auto at = [&](double v, int c) { return __shfl_sync(kFull, v, c); };
      const double dV = step[0] * step[1] * step[2];
      const double V = dV * cnt;
      const double gscale = 0.5 * dV * 6.0 / P.wdx;
      const double inv_cnt = 1.0 / static_cast<double>(cnt);
      const double stk = sel(step, kc), lok = sel(lo1, kc), xak = sel(XA, kc), xbk = sel(XB, kc);
      const double Mk = kc == 0 ? m0 : (kc == 1 ? m1 : m2);
      const double Gsk = kc == 0 ? g0 : (kc == 1 ? g1 : g2);
      const double xck = lok + (Mk * inv_cnt + 0.5) * stk;
      const double Gk = gscale * Gsk;
      const double G0 = at(Gk, 0), G1 = at(Gk, 1), G2 = at(Gk, 2);
      const double gn = sqrt(G0 * G0 + G1 * G1 + G2 * G2);
      const double ddk = xbk - xak;
      const double dd0 = at(ddk, 0), dd1 = at(ddk, 1), dd2 = at(ddk, 2);
      double nk;
      if (gn > 1e-12 * P.dx * P.dx) {
        const double ig = 1.0 / gn;
        nk = Gk * ig;
      } else if (j >= P.n) {
        nk = -S.planes[4 * S.face_off[j] + kc];
      } else {
        const double dn = sqrt(dd0 * dd0 + dd1 * dd1 + dd2 * dd2);
        nk = dn > 0.0 ? ddk / dn : 0.0;
      }
      // depth at the deepest sample, FP64: A's distance on lane 0, B's on lane 1
      const int bi = min(max(bestidx, 0), ns - 1);
      const int bx = bi % Nc, by = (bi / Nc) % Nc, bz = bi / (Nc * Nc);
      const double xs[3] = {lo1[0] + (bx + 0.5) * step[0], lo1[1] + (by + 0.5) * step[1],
                            lo1[2] + (bz + 0.5) * step[2]};
      double pv = 0.0;
      if (lane < 2) {
        const bool sb = lane == 1;
        const int pid = sb ? j : i;
        const double Xp[3] = {sb ? XB[0] : XA[0], sb ? XB[1] : XA[1], sb ? XB[2] : XA[2]};
        const int f0 = S.face_off[pid];
        double gdummy[3];
        pv = sdf64(S.type[pid], S.param + 3 * pid, S.planes + 4 * f0, S.face_off[pid + 1] - f0, Xp, D.R + 9 * pid,
                   xs, P.inflate, gdummy);
      }
      const double pa = at(pv, 0), pb = at(pv, 1);
      const double d = fmax(0.0, -(pa + pb));
      const double estar = 1.0 / (S.compl_[i] + S.compl_[j]);
      double damp = 1.0;
      const double rak = xck - xak, rbk = xck - xbk;
      const double n0 = at(nk, 0), n1 = at(nk, 1), n2 = at(nk, 2);
      // u_AB = (v_A + w_A x r_A) - (v_B + w_B x r_B) at x_c, ddot_n = u_AB . n
      double uabk = 0.0, ddot = 0.0;
      if (vel != nullptr && (P.damping_c != 0.0 || P.history || P.friction)) {
        const double* va = vel + 6 * i;
        const double* vb = j < P.n ? vel + 6 * j : D.rest6;
        const double ra1 = at(rak, k1), ra2 = at(rak, k2), rb1 = at(rbk, k1), rb2 = at(rbk, k2);
        const double uak = va[kc] + (va[3 + k1] * ra2 - va[3 + k2] * ra1);
        const double ubk = vb[kc] + (vb[3 + k1] * rb2 - vb[3 + k2] * rb1);
        uabk = uak - ubk;
        ddot = at(uabk, 0) * n0 + at(uabk, 1) * n1 + at(uabk, 2) * n2;
      }
      // c: the shared one, or with the history the contact's own (a new
      // contact's from u0 = ddot_n, Eq. damping_factor; 0 for u0 <= 0)
      double cdamp = P.damping_c;
      if (P.history) cdamp = hit >= 0 ? c_hist : (ddot > 0.0 ? P.damp_K / ddot : 0.0);
      if (vel != nullptr && cdamp != 0.0) damp = fmax(0.0, 1.0 + cdamp * ddot);
      const double vd = V * d;
      const double fmag = vd > 0.0 ? (4.0 / (3.0 * 3.14159265358979323846)) * estar * sqrt(vd) * damp : 0.0;
      double Fk = fmag * nk;
      if (P.friction && vel != nullptr && fmag > 0.0) {
        // Eq. (contact_force_tangential): B receives +f(a) |F_n| t, t = u_t / |u_t|
        const double utk = uabk - ddot * nk;
        const double u0 = at(utk, 0), u1 = at(utk, 1), u2 = at(utk, 2);
        const double utn = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        if (utn > 0.0) {
          const double a = utn * P.inv_u_k, a2 = a * a;
          double coef = P.mu_k;
          if (a2 < 1e30) {
            const double den1 = a2 * a2 + 1.0, den2 = a2 + 1.0;
            coef = a2 * ((2.0 * P.mu_s_star - P.mu_k) * den2 + P.mu_k * den1) / (den1 * den2);
          }
          Fk += coef * fmag * utk / utn;
        }
      }
      const double F1 = at(Fk, k1), F2 = at(Fk, k2);
      const double TAk = -(at(rak, k1) * F2 - at(rak, k2) * F1);
      const double TBk = at(rbk, k1) * F2 - at(rbk, k2) * F1;
      double* o = pair_out + static_cast<size_t>(q) * 11;
      double* ft = W.ft + static_cast<size_t>(q) * kFtDoubles;
      if (lane < 3) {
        o[1 + lane] = xck; o[4 + lane] = nk; o[8 + lane] = Fk;
        ft[lane] = Fk; ft[3 + lane] = TAk; ft[6 + lane] = TBk;
      }
      if (lane == 0) {
        o[0] = V;
        o[7] = d;
        atomicAdd(&W.counters[5], 1);
      }
      if (lane < kTapeDoubles) W.tape[static_cast<size_t>(q) * kTapeDoubles + lane] = 0.0;
      if (P.history) {   // this step's contact: j, c and the corrected box minus X_i
        const int wr = (W.counters[kStepCounter] & 1) ^ 1;
        int slot = 0;
        if (lane == 0) slot = atomicAdd(W.hist_n + static_cast<size_t>(wr) * P.n + i, 1);
        slot = __shfl_sync(kFull, slot, 0);
        if (slot < P.max_nbr) {
          const size_t e = (static_cast<size_t>(wr) * P.n + i) * P.max_nbr + slot;
          if (lane == 0) {
            W.hist_j[e] = j;
            W.hist_c[e] = cdamp;
          }
          if (lane < 3) {
            W.hist_box[6 * e + lane] = __dsub_rn(lok, xak);
            W.hist_box[6 * e + 3 + lane] = __dsub_rn(sel(hi1, kc), xak);
          }
        }
      }
    }
  }
}

}  // namespace

void launch_box(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel, double* pair_out,
                int grid, cudaStream_t st) {
  // the node sweep's kind set: 2 cubes only, 1 spheres / cuboids / walls, 0 every kind;
  // persistent: as many blocks as are resident (the kernel's own occupancy)
  auto kern = P.kind_set == 2 ? k_box_pairs<2> : (P.kind_set == 1 ? k_box_pairs<1> : k_box_pairs<0>);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBoxWarps * 32, 0);
  const int g = sms > 0 && per_sm > 0 ? sms * per_sm : grid;
  launch_pdl(kern, dim3(g), dim3(kBoxWarps * 32), 0, st, P, S, D, W, vel, pair_out);
}

}  // namespace gbc
