// Narrow phase of the contact step: every lattice node of every candidate
// pair's box is tested against both particles' signed distance functions and
// reduced to the overlap volume, its first moments, the band sum behind the
// contact normal and the deepest node (Sec. 3.3.1 of arXiv:2401.10878: "iterate
// over the entire overlap region to determine the overlap volume, the contact
// point, the contact normal, the indentation depth").
//
// k_narrow32 (FP32 node tests, FP32 tile partials):
//   * persistent grid, one warp per tile; warp w takes tiles w, w + W, ...
//     of the cost-ordered tile list (W warps; no queue atomics), the next
//     tile's record fetched while the current one runs; pairs whose distance
//     regions are apart never reach the list (the pair builder's test);
//   * a pair's box is cut into node lines along its longest axis; a tile is
//     32 lanes x 4 lines of one pair;
//   * each lane clips its line to the interval where both signed distances
//     lie below w/2 (line_clip.cuh: one bound per face plane, the sphere's
//     quadratic) and evaluates only the nodes inside it: every node outside
//     adds exact zeros to every sum, and ~99 % of a settling box's pair-box
//     nodes lie outside;
//   * along a line only the sweep coordinate changes, so the per-line part of
//     each face value is computed once and a node costs one FMA per face;
//   * node coordinates relative to each particle are exact integers minus an
//     FP32 remainder in [-1/2, 1/2] (no large-offset cancellation);
//   * polytope faces (and their inverse slopes along the line) are staged
//     in shared memory;
//   * the volume/moment/depth update and the normal-band update run only when
//     some lane of the warp needs them (warp-uniform branches);
//   * warp-shuffle reduction per tile (skipped when no lane met a node to
//     evaluate); a pair of one tile is finished from the warp's registers,
//     otherwise the partials go to HBM and the warp that completes the pair's
//     last tile sums them in FP64 in tile order (deterministic).
// k_narrow64: all-FP64 comparison form, one thread block per pair.
#include <cfloat>
#include <type_traits>

#include "contact_dev.cuh"
#include "force_law.cuh"
#include "line_clip.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;  // warps per block of the persistent kernel

// Local sweep axes (u = along the lines, v, w across) and the node-index
// stride of each (the node index is x-fastest over the pair box).
struct Local {
  int u, v, w;
  int su, sv, sw;
};

__device__ __forceinline__ Local make_local(const PairRec& r) {
  Local L;
  L.u = r.axis;
  L.v = L.u == 2 ? 0 : L.u + 1;
  L.w = L.v == 2 ? 0 : L.v + 1;
  const int s1 = r.dim[0], s2 = r.dim[0] * r.dim[1];
  L.su = L.u == 0 ? 1 : (L.u == 1 ? s1 : s2);
  L.sv = L.v == 0 ? 1 : (L.v == 1 ? s1 : s2);
  L.sw = L.w == 0 ? 1 : (L.w == 1 ? s1 : s2);
  return L;
}

// (a_u, a_v, a_w) in local axes -> component c of the world vector
__device__ __forceinline__ float world_comp(int c, const Local& L, float au, float av, float aw) {
  return c == L.u ? au : (c == L.v ? av : aw);
}


// ---------------------------------------------------------------- evaluators
// Each evaluator holds one particle's geometry for the current tile, in
// lattice units, relative to the pair box origin; it reads the pair record
// from shared memory (second = the record's particle j).

struct SphereEval {
  int iu, iv, iw;
  float fu, fv, fw, rad;
  float cnt_u, rv, rw, rho2, ru, q;
  float gu, gv, gw, gl;
  __device__ void load(const PairRec& r, bool second, const Shapes&, const Parts&, const Local& L, float4*) {
    const int* ci = second ? r.bi : r.ai;
    const float* cf = second ? r.bf : r.af;
    iu = ci[L.u]; iv = ci[L.v]; iw = ci[L.w];
    fu = cf[L.u]; fv = cf[L.v]; fw = cf[L.w];
    rad = second ? r.szb[0] : r.sza[0];
    gu = gv = gw = 0.f;
  }
  __device__ __forceinline__ void begin_line(int cv, int cw, int u0) {
    rv = static_cast<float>(cv - iv) - fv;
    rw = static_cast<float>(cw - iw) - fw;
    rho2 = fmaf(rv, rv, rw * rw);
    gl = 0.f;
    cnt_u = static_cast<float>(u0 - iu) - 1.f;
  }
  // [lo, hi] (line coordinates) cut to where phi < T on the current line
  __device__ __forceinline__ void clip(float T, float& lo, float& hi) const {
    const float o = static_cast<float>(iu);
    float l = lo - o, h = hi - o;
    clip_ball(fu, rho2, rad, T, l, h);
    lo = l + o;
    hi = h + o;
  }
  __device__ __forceinline__ float phi() {
    cnt_u += 1.f;
    ru = cnt_u - fu;
    q = fmaf(ru, ru, rho2);
    return sqrtf(q) - rad;
  }
  __device__ __forceinline__ void grad(float m) {
    const float mi = m * (q > 0.f ? rsqrtf(q) : 0.f);
    gu = fmaf(mi, ru, gu);
    gl += mi;
  }
  __device__ __forceinline__ void end_line() {
    gv = fmaf(gl, rv, gv);
    gw = fmaf(gl, rw, gw);
  }
  __device__ float world(int c, const Local& L, const PairRec&, bool) const { return world_comp(c, L, gu, gv, gw); }
};

struct CuboidEval {
  int iu, iv, iw;
  float fu, fv, fw;
  float tu[3], tv[3], tw[3], h[3], itu[3];
  float cnt_u, p[3], y[3], a[3];
  float gb[3];
  __device__ void load(const PairRec& r, bool second, const Shapes&, const Parts&, const Local& L, float4*) {
    const int* ci = second ? r.bi : r.ai;
    const float* cf = second ? r.bf : r.af;
    const float* rt = second ? r.rtb : r.rta;
    const float* sz = second ? r.szb : r.sza;
    iu = ci[L.u]; iv = ci[L.v]; iw = ci[L.w];
    fu = cf[L.u]; fv = cf[L.v]; fw = cf[L.w];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      tu[k] = rt[3 * k + L.u];
      tv[k] = rt[3 * k + L.v];
      tw[k] = rt[3 * k + L.w];
      h[k] = sz[k];
      itu[k] = clip_inv(tu[k]);
      gb[k] = 0.f;
    }
  }
  __device__ __forceinline__ void begin_line(int cv, int cw, int u0) {
    const float rv = static_cast<float>(cv - iv) - fv;
    const float rw = static_cast<float>(cw - iw) - fw;
    // y_k = tu_k (m - fu) + tv_k rv + tw_k rw with m = cu - iu: the constant
    // part is folded once per line, a node costs one FMA per axis
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = fmaf(-tu[k], fu, fmaf(tv[k], rv, tw[k] * rw));
    cnt_u = static_cast<float>(u0 - iu) - 1.f;
  }
  __device__ __forceinline__ void clip(float T, float& lo, float& hi) const {
    const float o = static_cast<float>(iu);
    float l = lo - o, hh = hi - o;
#pragma unroll
    for (int k = 0; k < 3; ++k) clip_slab(tu[k], itu[k], p[k], h[k] + T, l, hh);
    lo = l + o;
    hi = hh + o;
  }
  __device__ __forceinline__ float phi() {
    cnt_u += 1.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      y[k] = fmaf(tu[k], cnt_u, p[k]);
      a[k] = fabsf(y[k]) - h[k];
    }
    return fmaxf(a[0], fmaxf(a[1], a[2]));
  }
  __device__ __forceinline__ void grad(float m) {
    // active face: first maximal axis; gradient sign(y_k) e_k (body frame)
    const bool s0 = a[0] >= a[1] && a[0] >= a[2];
    const bool s1 = !s0 && a[1] >= a[2];
    gb[0] += s0 ? copysignf(m, y[0]) : 0.f;
    gb[1] += s1 ? copysignf(m, y[1]) : 0.f;
    gb[2] += (!s0 && !s1) ? copysignf(m, y[2]) : 0.f;
  }
  __device__ __forceinline__ void end_line() {}
  // world component c of R gb, R^T row k = body axis k in world
  __device__ float world(int c, const Local&, const PairRec& r, bool second) const {
    const float* rt = second ? r.rtb : r.rta;
    return rt[c] * gb[0] + rt[3 + c] * gb[1] + rt[6 + c] * gb[2];
  }
};

// Cube (equal half extents h): phi = max_k |y_k| - h.  Only what the node
// loop needs stays in registers; the cross-axis terms are re-read from the
// shared-memory pair record at each line start.  The line clip reads per-tile
// constants from shared memory (prep_clip): along the line, slab k of
// |y_k| < h + T is the node-counter interval centred at
// c_k = fu - (tv_k rv + tw_k rw) / tu_k with half-width (h + T) / |tu_k|.
struct CubeEval {
  int iu;
  float fu, tu0, tu1, tu2, h, itu0, itu1, itu2;
  bool flat;   // a slab parallel to the lines (|tu_k| <= kClipFlat): the general clip
  float cnt_u, p0, p1, p2, y0, y1, y2;
  float gb0, gb1, gb2;
  // the geometry comes with the staged constants (prep_clip, then fetch)
  __device__ void load(const PairRec&, bool, const Shapes&, const Parts&, const Local&, float4*) {
    gb0 = gb1 = gb2 = 0.f;
  }
  __device__ __forceinline__ void begin_line_rec(const PairRec& r, bool second, const Local& L, int cv, int cw,
                                                 int u0) {
    const int* ci = second ? r.bi : r.ai;
    const float* cf = second ? r.bf : r.af;
    const float* rt = second ? r.rtb : r.rta;
    const float rv = static_cast<float>(cv - ci[L.v]) - cf[L.v];
    const float rw = static_cast<float>(cw - ci[L.w]) - cf[L.w];
    p0 = fmaf(-tu0, fu, fmaf(rt[L.v], rv, rt[L.w] * rw));
    p1 = fmaf(-tu1, fu, fmaf(rt[3 + L.v], rv, rt[3 + L.w] * rw));
    p2 = fmaf(-tu2, fu, fmaf(rt[6 + L.v], rv, rt[6 + L.w] * rw));
    cnt_u = static_cast<float>(u0 - iu) - 1.f;
  }
  __device__ __forceinline__ void clip(float T, float& lo, float& hi) const {
    const float o = static_cast<float>(iu), ht = h + T;
    float l = lo - o, hh = hi - o;
    clip_slab(tu0, itu0, p0, ht, l, hh);
    clip_slab(tu1, itu1, p1, ht, l, hh);
    clip_slab(tu2, itu2, p2, ht, l, hh);
    lo = l + o;
    hi = hh + o;
  }
  // per-tile constants in cs[0 .. 8): (sv_k, hd_0), (sw_k, hd_1),
  // (hd_2, iv + fv, iw + fw, fu + iu), (iv, iw, iu, fu), (tv_k, fv),
  // (tw_k, fw), (tu_k, h), (1 / tu_k, -) with sv_k = tv_k / tu_k,
  // sw_k = tw_k / tu_k, hd_k = (h + T) / |tu_k| (the line clip reads the
  // first three, the node start the next three).  Lane k < 3 forms axis k's entries, lane 3 the
  // centre and size (two cubes: lanes 4 .. 7 form B's in the same pass); the
  // caller syncs the warp once for both evaluators and every lane then
  // fetches its registers.
  __device__ __forceinline__ void prep_clip(const PairRec& r, bool second, const Local& L, float T, float4* cs) {
    prep_lanes(r, second, L, T, cs, threadIdx.x & 31);
  }
  // the stores of lane q of the group that forms the constants (q < 3: axis
  // q's entries, q = 3: the centre and size, q > 3: none)
  static __device__ __forceinline__ void prep_lanes(const PairRec& r, bool second, const Local& L, float T,
                                                    float4* cs, int q) {
    const int* ci = second ? r.bi : r.ai;
    const float* cf = second ? r.bf : r.af;
    const float* rt = second ? r.rtb : r.rta;
    const float hh = second ? r.szb[0] : r.sza[0];
    const int k = q < 3 ? q : 0;
    const float tu = rt[3 * k + L.u], tv = rt[3 * k + L.v], tw = rt[3 * k + L.w];
    const float itu = clip_inv(tu);
    float* f = reinterpret_cast<float*>(cs);
    if (q < 3) {
      f[k] = tv * itu;
      f[4 + k] = tw * itu;
      f[k == 0 ? 3 : (k == 1 ? 7 : 8)] = (hh + T) * fabsf(itu);
      f[16 + k] = tv;
      f[20 + k] = tw;
      f[24 + k] = tu;
      f[28 + k] = itu;
    } else if (q == 3) {
      const int iu = ci[L.u], iv = ci[L.v], iw = ci[L.w];
      const float fu = cf[L.u], fv = cf[L.v], fw = cf[L.w];
      f[9] = static_cast<float>(iv) + fv;
      f[10] = static_cast<float>(iw) + fw;
      f[11] = fu + static_cast<float>(iu);
      cs[3] = make_float4(__int_as_float(iv), __int_as_float(iw), __int_as_float(iu), fu);
      f[19] = fv;
      f[23] = fw;
      f[27] = hh;
    }
  }
  __device__ __forceinline__ void fetch(const float4* cs) {
    const float4 a = cs[6], b = cs[7], d = cs[3];
    tu0 = a.x; tu1 = a.y; tu2 = a.z; h = a.w;
    itu0 = b.x; itu1 = b.y; itu2 = b.z;
    fu = d.w;
    iu = __float_as_int(d.z);
    flat = !(fabsf(tu0) > kClipFlat && fabsf(tu1) > kClipFlat && fabsf(tu2) > kClipFlat);
  }
  // begin_line_rec from the staged constants (the same operands, the same arithmetic)
  __device__ __forceinline__ void begin_node(const float4* cs, int cv, int cw, int u0) {
    const float4 d = cs[3], tv = cs[4], tw = cs[5];
    const float rv = static_cast<float>(cv - __float_as_int(d.x)) - tv.w;
    const float rw = static_cast<float>(cw - __float_as_int(d.y)) - tw.w;
    p0 = fmaf(-tu0, fu, fmaf(tv.x, rv, tw.x * rw));
    p1 = fmaf(-tu1, fu, fmaf(tv.y, rv, tw.y * rw));
    p2 = fmaf(-tu2, fu, fmaf(tv.z, rv, tw.z * rw));
    cnt_u = static_cast<float>(u0 - iu) - 1.f;
  }
  // [lo, hi] cut to the nodes of line (cv, cw) inside all three slabs
  __device__ __forceinline__ void clip_line(const PairRec& r, bool second, const Local& L, const float4* cs, int cv,
                                            int cw, float T, float& lo, float& hi) {
    const float4 a = cs[0], b = cs[1], c = cs[2];
    if (flat) {
      begin_line_rec(r, second, L, cv, cw, 0);
      clip(T, lo, hi);
      return;
    }
    // in box nodes: the centre's offsets (iv + fv, iw + fw) and fu + iu formed
    // once per tile (their rounding, ~1e-5 cells, stays far inside the margin)
    const float rv = static_cast<float>(cv) - c.y;
    const float rw = static_cast<float>(cw) - c.z;
    const float x0 = fmaf(-a.x, rv, fmaf(-b.x, rw, c.w));
    const float x1 = fmaf(-a.y, rv, fmaf(-b.y, rw, c.w));
    const float x2 = fmaf(-a.z, rv, fmaf(-b.z, rw, c.w));
    lo = fmaxf(lo, max3f(x0 - a.w, x1 - b.w, x2 - c.x));
    hi = fminf(hi, min3f(x0 + a.w, x1 + b.w, x2 + c.x));
  }
  __device__ __forceinline__ float phi() {
    cnt_u += 1.f;
    y0 = fmaf(tu0, cnt_u, p0);
    y1 = fmaf(tu1, cnt_u, p1);
    y2 = fmaf(tu2, cnt_u, p2);
    return fmaxf(fabsf(y0), fmaxf(fabsf(y1), fabsf(y2))) - h;
  }
  __device__ __forceinline__ void grad(float m) {
    const float a0 = fabsf(y0), a1 = fabsf(y1), a2 = fabsf(y2);
    const bool s0 = a0 >= a1 && a0 >= a2;
    const bool s1 = !s0 && a1 >= a2;
    gb0 += s0 ? copysignf(m, y0) : 0.f;
    gb1 += s1 ? copysignf(m, y1) : 0.f;
    gb2 += (!s0 && !s1) ? copysignf(m, y2) : 0.f;
  }
  __device__ __forceinline__ void end_line() {}
  __device__ float world(int c, const Local&, const PairRec& r, bool second) const {
    const float* rt = second ? r.rtb : r.rta;
    return rt[c] * gb0 + rt[3 + c] * gb1 + rt[6 + c] * gb2;
  }
};

// Stage a polytope's world planes in local axes (u, v, w, offset) into shared
// memory, and each face's inverse slope along u (the line clip) after them;
// faces beyond nf are padded so that they never win the maximum (and are
// constant along the line, below any threshold).
__device__ __forceinline__ int stage_planes(const Shapes& S, const Parts& D, int pid, const Local& L,
                                            float4* sm, int npad) {
  const int lane = threadIdx.x & 31;
  const int f0 = S.face_off[pid];
  const int nf = S.face_off[pid + 1] - f0;
  if (lane < npad) {
    float4 e = make_float4(0.f, 0.f, 0.f, 1e30f);
    if (lane < nf) {
      const float4 w = D.wplane[f0 + lane];
      e = make_float4(L.u == 0 ? w.x : (L.u == 1 ? w.y : w.z), L.v == 0 ? w.x : (L.v == 1 ? w.y : w.z),
                      L.w == 0 ? w.x : (L.w == 1 ? w.y : w.z), w.w);
    }
    sm[lane] = e;
  }
  __syncwarp();
  return nf;
}

// Polytopes: planes read from shared memory (sp[0 .. nf)); phi keeps the index
// of the first maximal face for the gradient.  The line clip reads per-tile
// half-line bounds (prep_clip) from sp[kMaxFaces ..): along the line, face f
// of slope m = e.x bounds the node counter c - iu by
// C_f - sy_f rv - sz_f rw (above for m > 0, below for m < 0) with
// sy_f = e.y / m, sz_f = e.z / m, C_f = (T + e.w) / m + fu; a face parallel
// to the line (|m| <= kClipFlat) keeps or empties the whole line.
struct PolyEval {
  int iu, iv, iw, nf, nup, ndn, kbest;
  float fu, fv, fw;
  const float4* sp;
  float cnt_u, ru, rv, rw;
  float gu, gv, gw;
  __device__ void load(const PairRec& r, bool second, const Shapes& S, const Parts& D, const Local& L,
                       float4* sm) {
    const int* ci = second ? r.bi : r.ai;
    const float* cf = second ? r.bf : r.af;
    iu = ci[L.u]; iv = ci[L.v]; iw = ci[L.w];
    fu = cf[L.u]; fv = cf[L.v]; fw = cf[L.w];
    nf = stage_planes(S, D, second ? r.j : r.i, L, sm, kMaxFaces);
    sp = sm;
    gu = gv = gw = 0.f;
  }
  __device__ __forceinline__ void begin_line(int cv, int cw, int u0) {
    rv = static_cast<float>(cv - iv) - fv;
    rw = static_cast<float>(cw - iw) - fw;
    cnt_u = static_cast<float>(u0 - iu) - 1.f;
  }
  // the half-line bounds of the tile's faces in sp[kMaxFaces ..): faces
  // bounding from above, then from below, then parallel ones (their planes)
  __device__ __forceinline__ void prep_clip(const PairRec&, bool, const Local&, float T, float4* cs) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < nf;
    const float4 e = sp[act ? lane : 0];
    const bool up = act && e.x > kClipFlat, dn = act && e.x < -kClipFlat, par = act && !up && !dn;
    const unsigned bu = __ballot_sync(kFull, up), bd = __ballot_sync(kFull, dn), bp = __ballot_sync(kFull, par);
    nup = __popc(bu);
    ndn = __popc(bd);
    const unsigned lt = (1u << lane) - 1u;
    const int pos = up ? __popc(bu & lt) : (dn ? nup + __popc(bd & lt) : nup + ndn + __popc(bp & lt));
    if (act) {
      float4 c = e;
      if (!par) {
        const float im = __fdividef(1.f, e.x);
        c = make_float4(e.y * im, e.z * im, fmaf(T + e.w, im, fu), 0.f);
      }
      cs[kMaxFaces + pos] = c;
    }
    __syncwarp();
  }
  __device__ __forceinline__ void clip_line(const PairRec&, bool, const Local&, const float4*, int cv, int cw,
                                            float T, float& lo, float& hi) const {
    const float lrv = static_cast<float>(cv - iv) - fv, lrw = static_cast<float>(cw - iw) - fw;
    const float o = static_cast<float>(iu);
    const float4* cl = sp + kMaxFaces;
    float l = lo - o, h = hi - o;
    int f = 0;
    for (; f < nup; ++f) {
      const float4 c = cl[f];
      h = fminf(h, fmaf(-c.x, lrv, fmaf(-c.y, lrw, c.z)));
    }
    for (; f < nup + ndn; ++f) {
      const float4 c = cl[f];
      l = fmaxf(l, fmaf(-c.x, lrv, fmaf(-c.y, lrw, c.z)));
    }
    for (; f < nf; ++f) {
      const float4 e = cl[f];
      if (!(fmaf(-e.x, fu, fmaf(e.y, lrv, fmaf(e.z, lrw, -e.w))) < T)) l = kClipEmpty;
    }
    lo = l + o;
    hi = h + o;
  }
  __device__ __forceinline__ float value(int f) const {
    const float4 e = sp[f];
    return fmaf(e.x, ru, fmaf(e.y, rv, fmaf(e.z, rw, -e.w)));
  }
  __device__ __forceinline__ float phi() {
    cnt_u += 1.f;
    ru = cnt_u - fu;
    int k = 0;
    float best = value(0);
    for (int f = 1; f < nf; ++f) {
      const float v = value(f);
      if (v > best) { best = v; k = f; }
    }
    kbest = k;
    return best;
  }
  __device__ __forceinline__ void grad(float m) {
    const float4 e = sp[kbest];
    gu = fmaf(m, e.x, gu);
    gv = fmaf(m, e.y, gv);
    gw = fmaf(m, e.z, gw);
  }
  __device__ __forceinline__ void end_line() {}
  __device__ float world(int c, const Local& L, const PairRec&, bool) const { return world_comp(c, L, gu, gv, gw); }
};

// Fixed wall m . x <= h: phi = m . c + p0 at box-relative node c (lattice
// units; p0 = the value at the box origin, inflate included, computed in
// FP64 by the pair builder and kept in the record's size slot; the record's
// centre of a wall is the box origin).  Box-relative values stay small, so
// FP32 keeps them to ~1e-6.
struct WallEval {
  float mu_, mv_, mw_, p0, imu_;
  float base, cnt_u, g;
  __device__ void load(const PairRec& r, bool second, const Shapes&, const Parts&, const Local& L, float4*) {
    const float* rt = second ? r.rtb : r.rta;   // row 0: the wall normal m (world)
    mu_ = rt[L.u]; mv_ = rt[L.v]; mw_ = rt[L.w];
    imu_ = clip_inv(mu_);
    p0 = second ? r.szb[0] : r.sza[0];
    g = 0.f;
  }
  __device__ __forceinline__ void begin_line(int cv, int cw, int u0) {
    base = fmaf(mv_, static_cast<float>(cv), fmaf(mw_, static_cast<float>(cw), p0));
    cnt_u = static_cast<float>(u0) - 1.f;
  }
  __device__ __forceinline__ void clip(float T, float& lo, float& hi) const { clip_half(mu_, imu_, base, T, lo, hi); }
  __device__ __forceinline__ float phi() {
    cnt_u += 1.f;
    return fmaf(mu_, cnt_u, base);
  }
  __device__ __forceinline__ void grad(float m) { g += m; }
  __device__ __forceinline__ void end_line() {}
  __device__ float world(int c, const Local&, const PairRec& r, bool second) const {
    return (second ? r.rtb : r.rta)[c] * g;
  }
};

// Line start of an evaluator: from the shared-memory record when the
// evaluator re-reads its cross-axis terms there, else from its registers.
template <class E>
__device__ __forceinline__ auto begin_line_of(E& e, const PairRec& r, bool second, const Local& L, int cv, int cw,
                                              int u0, int) -> decltype(e.begin_line_rec(r, second, L, cv, cw, u0)) {
  e.begin_line_rec(r, second, L, cv, cw, u0);
}
template <class E>
__device__ __forceinline__ void begin_line_of(E& e, const PairRec&, bool, const Local&, int cv, int cw, int u0, long) {
  e.begin_line(cv, cw, u0);
}

// Line clip of an evaluator: its own clip_line (per-tile constants staged by
// prep_clip) where it has one, else the line start and the general clip.
template <class E>
__device__ __forceinline__ auto prep_clip_of(E& e, const PairRec& r, bool second, const Local& L, float T, float4* cs,
                                             int) -> decltype(e.prep_clip(r, second, L, T, cs)) {
  e.prep_clip(r, second, L, T, cs);
}
template <class E>
__device__ __forceinline__ void prep_clip_of(E&, const PairRec&, bool, const Local&, float, float4*, long) {}
// Registers from the staged constants (after the warp's sync), where the evaluator keeps them there.
template <class E>
__device__ __forceinline__ auto fetch_of(E& e, const float4* cs, int) -> decltype(e.fetch(cs)) {
  e.fetch(cs);
}
template <class E>
__device__ __forceinline__ void fetch_of(E&, const float4*, long) {}
template <class E>
__device__ __forceinline__ auto clip_line_of(E& e, const PairRec& r, bool second, const Local& L, const float4* cs,
                                             int cv, int cw, float T, float& lo, float& hi, int)
    -> decltype(e.clip_line(r, second, L, cs, cv, cw, T, lo, hi)) {
  e.clip_line(r, second, L, cs, cv, cw, T, lo, hi);
}
template <class E>
__device__ __forceinline__ void clip_line_of(E& e, const PairRec& r, bool second, const Local& L, const float4*, int cv,
                                             int cw, float T, float& lo, float& hi, long) {
  begin_line_of(e, r, second, L, cv, cw, 0, 0);
  e.clip(T, lo, hi);
}

template <class E>
__device__ __forceinline__ auto node_line_of(E& e, const PairRec&, bool, const Local&, const float4* cs, int cv, int cw,
                                             int u0, int) -> decltype(e.begin_node(cs, cv, cw, u0)) {
  e.begin_node(cs, cv, cw, u0);
}
template <class E>
__device__ __forceinline__ void node_line_of(E& e, const PairRec& r, bool second, const Local& L, const float4*,
                                             int cv, int cw, int u0, long) {
  begin_line_of(e, r, second, L, cv, cw, u0, 0);
}

// ---------------------------------------------------------------- tile sweep
// Per-lane partials of a tile: node count and first moments (exact integers
// in sharp mode), the band sum of the normal, and the deepest node.
struct Partial {
  float cnt, mx, my, mz, gx, gy, gz, bestf;
  int bestidx;
  bool touched;   // warp-uniform: some lane evaluated a node (else every sum is zero)
};

// Order-preserving map of FP32 values to signed ints (for integer max).
__device__ __forceinline__ int float_key(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : (b ^ 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : (k ^ 0x7fffffff)); }

// Two phases per tile.  (A) Lane l clips its lines it0 + 32 s + l (s <
// kTileItemsPerLane) to the nodes where both distances lie below w/2 (+ the
// clip margin) and keeps each clipped range's first node and count.  (B) The
// tile's clipped nodes, typically a few dozen spread over a few lines, are
// numbered lane by lane (a scan of the lanes' counts), each lane's in slot
// order, and each lane evaluates one of them: the owning lane from a table
// of the lanes with nodes, the slot by the owner's counts, and the evaluators
// start that node's line at the node itself, so the node gets exactly the
// arithmetic of a node walk (the same FP32 distances, bit for bit).
// ROLL (the kernel with every kind, nine kind pairs): the slot loops stay
// rolled, with the slots' clipped ranges in shared memory, to keep the
// kernel's code small; otherwise they are unrolled over registers.
template <bool SMOOTH, bool ROLL, class EA, class EB>
__device__ __forceinline__ Partial sweep_tile(const Params& P, const Shapes& S, const Parts& D, const PairRec& r,
                                              bool swap, int tl, float4* smA, float4* smB, unsigned* spk,
                                              int4* own) {
  const int lane = threadIdx.x & 31;
  const Local L = make_local(r);
  EA A;
  EB B;
  A.load(r, swap, S, D, L, smA);
  B.load(r, !swap, S, D, L, smB);
  const int du = r.dim[L.u], dv = r.dim[L.v];
  const float inv_dv = __fdividef(1.f, static_cast<float>(dv));
  const float inv_w = P.inv_w, hw = 0.5f * P.wdx_l, T = hw + kClipMargin;
  // evaluators with a staged line clip keep its constants in their (otherwise
  // unused) plane buffer
  if constexpr (std::is_same<EA, CubeEval>::value && std::is_same<EB, CubeEval>::value) {
    // two cubes in one pass: lanes 0 .. 3 form A's constants, lanes 4 .. 7 B's
    const bool isb = (lane & 4) != 0;
    CubeEval::prep_lanes(r, isb ? !swap : swap, L, T, isb ? smB : smA, lane < 8 ? (lane & 3) : 4);
  } else {
    prep_clip_of(A, r, swap, L, T, smA, 0);
    prep_clip_of(B, r, !swap, L, T, smB, 0);
  }
  __syncwarp();
  fetch_of(A, smA, 0);
  fetch_of(B, smB, 0);
  const float4* csA = smA;
  const float4* csB = smB;
  float cnt = 0.f, mu = 0.f, mv = 0.f, mw = 0.f, bestf = -FLT_MAX;
  int bestidx = 0x7fffffff;
  const int it0 = tl * 32 * kTileItemsPerLane;
  const int ns = min(kTileItemsPerLane, (r.nitems - it0 + 31) >> 5);   // slots of this tile (warp-uniform)
  // (A) per slot: first clipped node (low 16 bits) and count (high 16 bits);
  // a pair box is below 2^16 nodes along an axis
  unsigned pk[kTileItemsPerLane];
  int nl = 0;
  // line it0 + 32 s + lane as (cv, cw) = its remainder and quotient by dv:
  // unrolled, one division for slot 0, then steps of 32 = q32 dv + r32; the
  // rolled loop divides per slot (fewer live registers)
  int cv = 0, r32 = 0, q32 = 0;
  int cw = 0;
  if constexpr (!ROLL) {
    cw = div_small(it0 + lane, dv, inv_dv, &cv);
    q32 = div_small(32, dv, inv_dv, &r32);
  }
#pragma unroll(ROLL ? 1 : kTileItemsPerLane)
  for (int s = 0; s < kTileItemsPerLane; ++s) {
    if (!ROLL) pk[s] = 0u;
    if (s < ns) {
      const int it = it0 + s * 32 + lane;
      if constexpr (ROLL) cw = div_small(it, dv, inv_dv, &cv);
      const int len = it < r.nitems ? du : 0;
      float clo = 0.f, chi = static_cast<float>(len - 1);
      clip_line_of(A, r, swap, L, csA, cv, cw, T, clo, chi, 0);
      clip_line_of(B, r, !swap, L, csB, cv, cw, T, clo, chi, 0);
      int ub;
      const int nk = clip_nodes(clo, chi, 0, len, &ub);
      const unsigned v = static_cast<unsigned>(ub) | (static_cast<unsigned>(nk) << 16);
      if constexpr (ROLL) spk[s * 32 + lane] = v;
      else pk[s] = v;
      nl += nk;
    }
    if constexpr (!ROLL) {
      cv += r32;
      cw += q32;
      if (cv >= dv) {
        cv -= dv;
        ++cw;
      }
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
  // the lanes with nodes, in lane order (their first nodes strictly
  // increase): entry k of own holds the k-th one's lane, first node and
  // clipped ranges
  const bool has = nl > 0;
  if (total > 0) {
    const int rank = __popc(__ballot_sync(kFull, has) & ((1u << lane) - 1u));
    if (has) {
      if constexpr (ROLL) {
        own[rank] = make_int4(lane, excl, 0, 0);
      } else {
        static_assert(kTileItemsPerLane == 4, "own holds four clipped ranges per lane");
        // and the lane's node counts before slots 2 and 3
        const int c2 = static_cast<int>(pk[0] >> 16) + static_cast<int>(pk[1] >> 16);
        own[rank] = make_int4(lane, excl, static_cast<int>(pk[0]), static_cast<int>(pk[1]));
        own[32 + rank] = make_int4(static_cast<int>(pk[2]), static_cast<int>(pk[3]), c2,
                                   c2 + static_cast<int>(pk[2] >> 16));
      }
    }
    __syncwarp();
  }
  // (B) node g of the tile's clipped nodes on lane g mod 32; its owner is the
  // last lane with nodes whose first node is <= g, i.e. entry (number of such
  // lanes) - 1 of own, counted from the lanes that start before the pass and
  // a mask of the first nodes inside it
  for (int base = 0; base < total; base += 32) {
    const int g = base + lane;
    const unsigned before = __ballot_sync(kFull, has && excl < base);
    const unsigned inside =
        __reduce_or_sync(kFull, (has && excl >= base && excl - base < 32) ? 1u << (excl - base) : 0u);
    const int cnt_le = __popc(before) + __popc(inside & (lane == 31 ? 0xffffffffu : (2u << lane) - 1u));
    const int4 e = own[min(max(cnt_le - 1, 0), 31)];
    const int o = e.x;
    int k = g - e.y;   // the node's rank among the owner's
    int4 e2 = make_int4(0, 0, 0, 0);
    if (!ROLL) e2 = own[32 + min(max(cnt_le - 1, 0), 31)];
    int os = 0, u = 0;
    if constexpr (ROLL) {
#pragma unroll 1
      for (int s = 0; s < kTileItemsPerLane; ++s) {
        if (s < ns) {
          const unsigned q = spk[s * 32 + o];
          const int n = static_cast<int>(q >> 16);
          if (k >= 0 && k < n) {
            os = s;
            u = static_cast<int>(q & 0xffffu) + k;
          }
          k -= n;
        }
      }
    } else {
      // the slot: how many of the owner's slot boundaries (node counts before
      // slots 1, 2, 3; empty slots repeat a boundary) lie at or below k
      const int c1 = static_cast<int>(static_cast<unsigned>(e.z) >> 16), c2 = e2.z, c3 = e2.w;
      os = (k >= c1 ? 1 : 0) + (k >= c2 ? 1 : 0) + (k >= c3 ? 1 : 0);
      const unsigned q = static_cast<unsigned>(os == 0 ? e.z : (os == 1 ? e.w : (os == 2 ? e2.x : e2.y)));
      u = static_cast<int>(q & 0xffffu) + k - (os == 0 ? 0 : (os == 1 ? c1 : (os == 2 ? c2 : c3)));
    }
    int ocv;
    const int ocw = div_small(it0 + os * 32 + o, dv, inv_dv, &ocv);
    node_line_of(A, r, swap, L, csA, ocv, ocw, u, 0);
    node_line_of(B, r, !swap, L, csB, ocv, ocw, u, 0);
    const float fa = A.phi();
    const float fb = B.phi();
    // W > 0, or a band term of the normal: max < w/2 and (sharp) min <= 0
    const bool any = g < total && fmaxf(fa, fb) < hw && (SMOOTH || fminf(fa, fb) <= 0.f);
    const float ta = __saturatef(fmaf(fa, -inv_w, 0.5f));
    const float tb = __saturatef(fmaf(fb, -inv_w, 0.5f));
    float w, ma, mb;
    if (SMOOTH) {
      const float ha = ta * ta * fmaf(-2.f, ta, 3.f);
      const float hb = tb * tb * fmaf(-2.f, tb, 3.f);
      w = any ? ha * hb : 0.f;
      ma = any ? fmaf(-ta, ta, ta) * hb : 0.f;
      mb = any ? ha * fmaf(-tb, tb, tb) : 0.f;
    } else {
      w = (any && fmaxf(fa, fb) <= 0.f) ? 1.f : 0.f;
      ma = (any && fb <= 0.f) ? fmaf(-ta, ta, ta) : 0.f;
      mb = (any && fa <= 0.f) ? fmaf(-tb, tb, tb) : 0.f;
    }
    cnt += w;
    mu = fmaf(w, static_cast<float>(u), mu);
    mv = fmaf(w, static_cast<float>(ocv), mv);
    mw = fmaf(w, static_cast<float>(ocw), mw);
    const float f = -(fa + fb);
    const int idx = u * L.su + ocv * L.sv + ocw * L.sw;
    if (w > 0.f && (f > bestf || (f == bestf && idx < bestidx))) {
      bestf = f;
      bestidx = idx;
    }
    A.grad(ma);
    B.grad(mb);
    A.end_line();
    B.end_line();
  }
  Partial o;
  o.cnt = cnt;
  o.mx = world_comp(0, L, mu, mv, mw);
  o.my = world_comp(1, L, mu, mv, mw);
  o.mz = world_comp(2, L, mu, mv, mw);
  o.gx = A.world(0, L, r, swap) - B.world(0, L, r, !swap);
  o.gy = A.world(1, L, r, swap) - B.world(1, L, r, !swap);
  o.gz = A.world(2, L, r, swap) - B.world(2, L, r, !swap);
  o.bestf = bestf;
  o.bestidx = bestidx;
  o.touched = total > 0;
  return o;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
  return v;
}

// Warp sums of (a, b, c) by halving exchanges (7 shuffles): lanes 4, 5, 6
// return the sums of a, b, c (other lanes: partial values).
__device__ __forceinline__ float warp_sum3_to_456(float a, float b, float c) {
  const int lane = threadIdx.x & 31;
  const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1;
  // (a, b) on lanes with bit 4 clear, (c, 0) on the others
  const float h0 = (b4 ? c : a) + __shfl_xor_sync(kFull, b4 ? a : c, 16);
  const float h1 = (b4 ? 0.f : b) + __shfl_xor_sync(kFull, b4 ? b : 0.f, 16);
  // component 2 b4 + b3
  float h = (b3 ? h1 : h0) + __shfl_xor_sync(kFull, b3 ? h0 : h1, 8);
  h += __shfl_xor_sync(kFull, h, 4);
  h += __shfl_xor_sync(kFull, h, 2);
  h += __shfl_xor_sync(kFull, h, 1);
  // lane 4 + c reads the lane holding component c (c = 0: lane 0, 1: lane 8, 2: lane 16)
  const int c3 = lane - 4;
  return __shfl_sync(kFull, h, (c3 >= 0 && c3 < 3) ? 8 * c3 : 0);
}

// Tile reduction.  Sharp mode: counts and moments are exact integers, summed
// with integer warp reductions; the deepest node via an integer max of an
// order-preserving key and an integer min of the node index among the ties.
template <bool SMOOTH>
__device__ __forceinline__ float reduce_tile(const Partial& o) {
  const int lane = threadIdx.x & 31;
  float c, x, y, z;
  if (SMOOTH) {
    c = warp_sum(o.cnt); x = warp_sum(o.mx); y = warp_sum(o.my); z = warp_sum(o.mz);
  } else {
    c = static_cast<float>(__reduce_add_sync(kFull, __float2int_rn(o.cnt)));
    x = static_cast<float>(__reduce_add_sync(kFull, __float2int_rn(o.mx)));
    y = static_cast<float>(__reduce_add_sync(kFull, __float2int_rn(o.my)));
    z = static_cast<float>(__reduce_add_sync(kFull, __float2int_rn(o.mz)));
  }
  const float g = warp_sum3_to_456(o.gx, o.gy, o.gz);   // lanes 4, 5, 6
  const int key = __reduce_max_sync(kFull, float_key(o.bestf));
  const int idx = __reduce_min_sync(kFull, float_key(o.bestf) == key ? o.bestidx : 0x7fffffff);
  float v = c;
  v = lane == 1 ? x : v;
  v = lane == 2 ? y : v;
  v = lane == 3 ? z : v;
  v = (lane >= 4 && lane < 7) ? g : v;
  v = lane == 7 ? key_float(key) : v;
  v = lane == 8 ? __int_as_float(idx) : v;
  return v;   // lane c < 9: component c of the tile partial
}

// The partial of a tile in which no node was evaluated: zero sums, no deepest node.
__device__ __forceinline__ float empty_partial() {
  const int lane = threadIdx.x & 31;
  return lane == 7 ? -FLT_MAX : (lane == 8 ? __int_as_float(0x7fffffff) : 0.f);
}

// The force law of the n <= 8 overlapping pairs staged in ov (whole warp).
template <int SET, bool LAW>
__device__ __forceinline__ void flush_overlaps(const Params& P, const Shapes& S, const Parts& D, const Lists& W,
                                               const double* vel, double* pair_out, OvlRec* ov, int nov) {
  if (nov == 0) return;
  __syncwarp();
  ForceArgs a;
  a.X = D.X; a.R = D.R;
  a.type = S.type; a.param = S.param; a.face_off = S.face_off; a.planes = S.planes; a.compl_ = S.compl_;
  a.vel = vel; a.pair_out = pair_out; a.ft = W.ft; a.tape = W.tape;
  for (int k = 0; k < 3; ++k) a.L[k] = P.L[k];
  a.dx = P.dx; a.dx3 = P.dx3; a.gscale = P.gscale; a.g_min2 = P.g_min2; a.inflate = P.inflate;
  a.damping_c = P.damping_c;
  a.history = P.history; a.friction = P.friction; a.hist_cap = P.max_nbr;
  a.n = P.n; a.rest6 = D.rest6;
  a.damp_K = P.damp_K; a.mu_s_star = P.mu_s_star; a.mu_k = P.mu_k; a.inv_u_k = P.inv_u_k;
  if (P.history) {   // buffer (steps & 1) holds the previous step's contacts
    const int rd = W.counters[kStepCounter] & 1;
    const size_t nn = static_cast<size_t>(P.n);
    a.hn_rd = W.hist_n + rd * nn; a.hn_wr = W.hist_n + (rd ^ 1) * nn;
    a.hj_rd = W.hist_j + rd * nn * P.max_nbr; a.hj_wr = W.hist_j + (rd ^ 1) * nn * P.max_nbr;
    a.hc_rd = W.hist_c + rd * nn * P.max_nbr; a.hc_wr = W.hist_c + (rd ^ 1) * nn * P.max_nbr;
  } else {
    a.hn_rd = a.hj_rd = nullptr; a.hc_rd = nullptr; a.hn_wr = a.hj_wr = nullptr; a.hc_wr = nullptr;
  }
  pair_force_law<SET, LAW>(a, ov, nov);
  __syncwarp();
}

// End of a pair (called by the whole warp once all its nodes are summed):
// lanes c < 7 hold the FP64 sum of component c, every lane the deepest node.
// A pair without overlap gets its zero outputs; an overlapping pair's sums go
// to its entry of the overlap list, flagged for the force law (the next
// kernel gathers the flagged entries, eight pairs per warp pass).
__device__ __forceinline__ void pair_done(const Params& P, const Lists& W, const PairRec& r, double* pair_out,
                                          double sv, int idx) {
  const int lane = threadIdx.x & 31;
  const int q = r.pair;
  const double s0 = __shfl_sync(kFull, sv, 0);
  const bool hit = __double_as_longlong(s0) > 0;   // V > 0
  if (lane == 31) W.oflag[q] = hit ? 1 : 0;
  if (hit) {
    OvlRec* e = W.olist + q;
    if (lane < 7) e->s[lane] = sv;
    if (lane == 7) e->q = q;
    if (lane == 8) e->idx = idx;
    if (lane >= 9 && lane < 20) (&e->i)[lane - 9] = reinterpret_cast<const int*>(&r)[lane - 9];   // i, j, lo, dim, shift
  } else {
    if (lane < 11) pair_out[static_cast<size_t>(q) * 11 + lane] = 0.0;
    if (lane < kFtDoubles) W.ft[static_cast<size_t>(q) * kFtDoubles + lane] = 0.0;
    if (lane < kTapeDoubles) W.tape[static_cast<size_t>(q) * kTapeDoubles + lane] = 0.0;
  }
}

// After a tile: a pair of one tile is finished at once from the warp's
// registers; otherwise the partial is stored, and the warp that completes the
// pair's last tile sums all of them in FP64 in a fixed order (4 tile slots x
// 8 components per lane pattern, slots combined pairwise), whichever warp
// that is.
__device__ __forceinline__ void tile_done(const Params& P, const Lists& W, const PairRec& r, double* pair_out,
                                          float v) {
  const int lane = threadIdx.x & 31;
  if (r.ntiles == 1) {
    const int idx = __shfl_sync(kFull, __float_as_int(v), 8);
    // (the hardware conversion: one issue slot on the node sweep's otherwise idle FP64 pipe)
    pair_done(P, W, r, pair_out, lane < 7 ? static_cast<double>(v) : 0.0, idx);
    return;
  }
  const size_t t0 = static_cast<size_t>(r.tile0);
  if (lane < 9) W.partial[(t0 + r.tile) * kPartialFloats + lane] = v;
  __threadfence();
  int prev = 0;
  if (lane == 0) prev = atomicAdd(&W.pdone[r.pair], 1);
  prev = __shfl_sync(kFull, prev, 0);
  if (prev != r.ntiles - 1) return;
  __threadfence();
  const int nt = r.ntiles, slot = lane >> 3, c = lane & 7;
  double acc = 0.0;
  float bf = -FLT_MAX;
  int bi = 0x7fffffff;
  for (int tb = 0; tb < nt; tb += 32) {   // batches of 32 tiles, all loads in flight at once
    float x[8];
    int ix[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = tb + slot + 4 * u;
      const float* q = W.partial + (t0 + (t < nt ? t : 0)) * kPartialFloats;
      x[u] = t < nt ? __ldcg(q + c) : 0.0f;
      ix[u] = (t < nt && c == 7) ? __float_as_int(__ldcg(q + 8)) : 0x7fffffff;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = tb + slot + 4 * u;
      if (t < nt) {
        if (c < 7) {
          const double w = static_cast<double>(x[u]);
          acc = t == slot ? w : acc + w;
        } else if (x[u] > bf || (x[u] == bf && ix[u] < bi)) {
          bf = x[u];
          bi = ix[u];
        }
      }
    }
  }
  acc += __shfl_xor_sync(kFull, acc, 8);    // (s0 + s1) + (s2 + s3): the same on every lane
  acc += __shfl_xor_sync(kFull, acc, 16);
  for (int o = 8; o <= 16; o <<= 1) {
    const float ob = __shfl_xor_sync(kFull, bf, o);
    const int oi = __shfl_xor_sync(kFull, bi, o);
    if (ob > bf || (ob == bf && oi < bi)) { bf = ob; bi = oi; }
  }
  if (lane == 0) W.pdone[r.pair] = 0;   // ready for a repeated sweep of the same tiles
  pair_done(P, W, r, pair_out, acc, __shfl_sync(kFull, bi, 7));
}

// Kernel variants: the full set of pair kinds, or spheres and cuboids only
// (chosen at init when no polytope is present; fewer registers, no spills).
enum KindSet : int { SET_ALL = 0, SET_SC = 1, SET_CUBE = 2 };

template <bool SMOOTH, int SET>
__device__ __forceinline__ Partial dispatch(const Params& P, const Shapes& S, const Parts& D, const PairRec& r,
                                            int tl, float4* smA, float4* smB, unsigned* spk, int4* own) {
  int ka = r.kinds & 0xff, kb = r.kinds >> 8;
  // evaluate the cheaper kind as A (G's sign flips back below); two cubes keep the record's order
  const bool swap = SET == SET_CUBE ? false : sweep_swap(ka, kb);
  if (swap) {
    const int t = ka; ka = kb; kb = t;
  }
  if (SET == SET_ALL) {   // the full variant sweeps cubes as cuboids
    ka = ka == KIND_CUBE ? KIND_CUBOID : ka;
    kb = kb == KIND_CUBE ? KIND_CUBOID : kb;
  }
  Partial o{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -FLT_MAX, 0x7fffffff, false};
#define GBC_CASE(KA, KB, TA, TB)                                                  \
  case (KA) * 8 + (KB):                                                          \
    o = sweep_tile<SMOOTH, SET == SET_ALL, TA, TB>(P, S, D, r, swap, tl, smA, smB, spk, own); \
    break;
  if constexpr (SET == SET_CUBE) {
    o = sweep_tile<SMOOTH, false, CubeEval, CubeEval>(P, S, D, r, swap, tl, smA, smB, spk, own);
  } else if constexpr (SET == SET_SC) {
    switch (ka * 8 + kb) {
      GBC_CASE(0, 0, SphereEval, SphereEval)
      GBC_CASE(0, 4, SphereEval, CubeEval)
      GBC_CASE(0, 1, SphereEval, CuboidEval)
      GBC_CASE(4, 4, CubeEval, CubeEval)
      GBC_CASE(4, 1, CubeEval, CuboidEval)
      GBC_CASE(1, 1, CuboidEval, CuboidEval)
      GBC_CASE(5, 0, WallEval, SphereEval)
      GBC_CASE(5, 4, WallEval, CubeEval)
      GBC_CASE(5, 1, WallEval, CuboidEval)
      default:
        break;
    }
  } else {
    switch (ka * 8 + kb) {
      GBC_CASE(0, 0, SphereEval, SphereEval)
      GBC_CASE(0, 1, SphereEval, CuboidEval)
      GBC_CASE(0, 3, SphereEval, PolyEval)
      GBC_CASE(1, 1, CuboidEval, CuboidEval)
      GBC_CASE(1, 3, CuboidEval, PolyEval)
      GBC_CASE(3, 3, PolyEval, PolyEval)
      GBC_CASE(5, 0, WallEval, SphereEval)
      GBC_CASE(5, 1, WallEval, CuboidEval)
      GBC_CASE(5, 3, WallEval, PolyEval)
      default:
        break;
    }
  }
#undef GBC_CASE
  if (swap) {
    o.gx = -o.gx; o.gy = -o.gy; o.gz = -o.gz;
  }
  return o;
}

// The warp copies a 224-byte pair record with 14 lanes x 16 bytes.
__device__ __forceinline__ int4 load_rec_part(const PairRec* src, int lane) {
  return lane < kPairRecWords / 4 ? reinterpret_cast<const int4*>(src)[lane] : make_int4(0, 0, 0, 0);
}
__device__ __forceinline__ void store_rec_part(PairRec* dst, int lane, int4 v) {
  if (lane < kPairRecWords / 4) reinterpret_cast<int4*>(dst)[lane] = v;
}

// Blocks per SM: 3 for the sphere/cuboid/cube variants (<= 85 registers, so
// 24 warps per SM: about one tile per warp at a settling box's size), 2 for
// the variant with every kind (measured faster than 3, which spills more).
// Warps per block and blocks per SM of the node sweep (compiled per kind set).
constexpr int kNarrowWarps = 8, kNarrowBlocks = 3;
template <int SET>
__host__ __device__ constexpr int narrow_warps() { return SET == SET_ALL ? 8 : kNarrowWarps; }
template <int SET>
__host__ __device__ constexpr int narrow_blocks() { return SET == SET_ALL ? 2 : kNarrowBlocks; }

template <bool SMOOTH, int SET>
__global__ void __launch_bounds__(narrow_warps<SET>() * 32, narrow_blocks<SET>()) k_narrow32(Params P, Shapes S,
                                                                                             Parts D, Lists W,
                                                                                             const double* vel,
                                                                                             double* pair_out) {
  constexpr int NW = narrow_warps<SET>();
  __shared__ __align__(16) PairRec s_rec[NW][2];
  // per evaluator: a polytope's planes, then its line clip's constants (a cube: the clip constants)
  __shared__ float4 s_planes[NW][2][SET == SET_CUBE ? 8 : 2 * kMaxFaces];
  __shared__ unsigned s_pk[SET == SET_ALL ? NW : 1][kTileItemsPerLane * 32];   // clipped ranges (rolled sweep)
  __shared__ int4 s_own[NW][64];   // the lanes with clipped nodes (sweep_tile)
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int ntiles = W.counters[1];
  // tiles w, w + W, ... of the list (W warps); the first record is fetched
  // with the tile count, the next one while a tile runs
  const int nwarps = gridDim.x * NW;
  int t = blockIdx.x * NW + wid;
  const int4 first = t < P.max_tiles ? load_rec_part(W.tiles + t, lane) : make_int4(0, 0, 0, 0);
  if (ntiles > P.max_tiles) return;   // capacity exceeded: the step reports ECAPACITY
  if (t < ntiles) store_rec_part(&s_rec[wid][0], lane, first);
  __syncwarp();
  int buf = 0;
  while (t < ntiles) {
    const int tn = t + nwarps;
    const int4 next = tn < ntiles ? load_rec_part(W.tiles + tn, lane) : make_int4(0, 0, 0, 0);
    const PairRec& r = s_rec[wid][buf];
    if (record_in_bounds(P, W.err, r, true)) {
      const Partial o = dispatch<SMOOTH, SET>(P, S, D, r, r.tile, s_planes[wid][0], s_planes[wid][1],
                                              s_pk[SET == SET_ALL ? wid : 0], s_own[wid]);
      tile_done(P, W, r, pair_out, o.touched ? reduce_tile<SMOOTH>(o) : empty_partial());
    }
    __syncwarp();
    if (tn < ntiles) store_rec_part(&s_rec[wid][buf ^ 1], lane, next);
    __syncwarp();
    buf ^= 1;
    t = tn;
  }
  (void)vel;   // the velocities enter with the force law (next kernel)
}

// The force law of the step's overlapping pairs, up to eight per warp pass
// (four lanes each).  Warp w of block b takes chunk c = b + grid * w (then
// c + grid * 8, ...) of 16 consecutive pairs: their overlap flags and, in the
// same round of loads, all 16 entries of the overlap list (the flagged ones
// are kept, in pair order), so one memory round trip precedes the pass.  With
// one block per SM the chunks of a step land on different sub-partitions, so
// the FP64 passes (the pipe serialises one warp instruction per ~64 cycles)
// run side by side.  Each warp adds its count of overlapping pairs to
// counters[5] (reported by contact_stats).
constexpr int kForceChunk = 16;

template <int SET, bool LAW>
__global__ void __launch_bounds__(kWarps * 32, 1) k_force(Params P, Shapes S, Parts D, Lists W, const double* vel,
                                                       double* pair_out) {
  __shared__ __align__(16) OvlRec s_ovl[kWarps][kForceChunk];
  pdl_begin();
  if (W.counters[1] > P.max_tiles) return;   // the node sweep did not run (ECAPACITY)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int np = min(W.counters[0], P.max_pairs);
  const int nchunk = (np + kForceChunk - 1) / kForceChunk;
  constexpr int kPieces = static_cast<int>(sizeof(OvlRec) / 16);          // 16-byte pieces per entry
  constexpr int kPerLane = kForceChunk * kPieces / 32;                    // pieces per lane
  int nov = 0;
  for (int c = blockIdx.x + gridDim.x * wid; c < nchunk; c += gridDim.x * kWarps) {
    const int q0 = kForceChunk * c;
    const int q = q0 + lane;
    const bool flag = lane < kForceChunk && q < np && W.oflag[q] != 0;
    int4 piece[kPerLane];
#pragma unroll
    for (int u = 0; u < kPerLane; ++u) {   // entry e / kPieces, part e % kPieces of the chunk
      const int e = lane + 32 * u;
      const int qe = q0 + e / kPieces;
      piece[u] = qe < np ? reinterpret_cast<const int4*>(W.olist + qe)[e % kPieces] : make_int4(0, 0, 0, 0);
    }
    unsigned mask = __ballot_sync(kFull, flag);
    nov += __popc(mask);
    while (mask != 0u) {
      const int n = min(__popc(mask), kForcePairsPerPass);
      // keep the next n flagged entries, packed in pair order
      unsigned take = mask;   // the lowest n flagged entries (all of them but in a rare 9th+)
      if (n < __popc(mask)) take = mask & ((1u << __fns(mask, 0, n + 1)) - 1u);   // below the (n+1)-th
      int4* dst = reinterpret_cast<int4*>(s_ovl[wid]);
#pragma unroll
      for (int u = 0; u < kPerLane; ++u) {
        const int e = lane + 32 * u, r = e / kPieces;
        if ((take >> r) & 1u) dst[__popc(take & ((1u << r) - 1u)) * kPieces + e % kPieces] = piece[u];
      }
      mask &= ~take;
      __syncwarp();
#ifdef CONTACT_CHECKS
      if (lane < n) {   // the staged entries' pair and particles
        OvlRec& e = s_ovl[wid][lane];
        e.q = checked_index(W.err, e.q, P.max_pairs, 0);
        e.i = checked_index(W.err, e.i, P.n, 0);
        e.j = checked_index(W.err, e.j, P.n + P.nwall, 0);
      }
      __syncwarp();
#endif
      flush_overlaps<SET, LAW>(P, S, D, W, vel, pair_out, s_ovl[wid], n);
    }
  }
  if (lane == 0 && nov > 0) atomicAdd(&W.counters[5], nov);
}

// ---------------------------------------------------------------- FP64 form
template <bool SMOOTH>
__global__ void __launch_bounds__(256) k_narrow64(Params P, Shapes S, Parts D, Lists W, const double* vel,
                                                  double* pair_out) {
  __shared__ double s_red[8][8];
  __shared__ double s_bf[8];
  __shared__ int s_bi[8];
  pdl_begin();
  const int np = min(W.counters[0], P.max_pairs);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int p = blockIdx.x; p < np; p += gridDim.x) {
    const PairRec pr = W.pairs[p];
    if (!record_in_bounds(P, W.err, pr, false)) continue;   // block-uniform (checked build only)
    const int i = pr.i, j = pr.j;
    double XA[3], XB[3], RA[9], RB[9];
    for (int k = 0; k < 3; ++k) {
      XA[k] = D.X[3 * i + k];
      XB[k] = D.X[3 * j + k] - pr.shift[k] * P.L[k];
    }
    for (int k = 0; k < 9; ++k) { RA[k] = D.R[9 * i + k]; RB[k] = D.R[9 * j + k]; }
    const int ta = S.type[i], tb = S.type[j];
    const double* pla = S.planes + 4 * S.face_off[i];
    const double* plb = S.planes + 4 * S.face_off[j];
    const int nfa = S.face_off[i + 1] - S.face_off[i], nfb = S.face_off[j + 1] - S.face_off[j];
    const int vol = pr.dim[0] * pr.dim[1] * pr.dim[2];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    double bf = -DBL_MAX;
    int bi = 0x7fffffff;
    for (int c = threadIdx.x; c < vol; c += blockDim.x) {
      const int cx = c % pr.dim[0], cy = (c / pr.dim[0]) % pr.dim[1], cz = c / (pr.dim[0] * pr.dim[1]);
      const double x[3] = {(pr.lo[0] + cx) * P.dx, (pr.lo[1] + cy) * P.dx, (pr.lo[2] + cz) * P.dx};
      double gA[3], gB[3];
      const double fa = sdf64(ta, S.param + 3 * i, pla, nfa, XA, RA, x, P.inflate, gA);
      const double fb = sdf64(tb, S.param + 3 * j, plb, nfb, XB, RB, x, P.inflate, gB);
      const double tA = fmin(fmax(0.5 - fa / P.wdx, 0.0), 1.0);
      const double tB = fmin(fmax(0.5 - fb / P.wdx, 0.0), 1.0);
      double hA, hB;
      if (SMOOTH) {
        hA = tA * tA * (3.0 - 2.0 * tA);
        hB = tB * tB * (3.0 - 2.0 * tB);
      } else {
        hA = fa <= 0.0 ? 1.0 : 0.0;
        hB = fb <= 0.0 ? 1.0 : 0.0;
      }
      const double w = hA * hB;
      const double ma = tA * (1.0 - tA) * hB, mb = hA * tB * (1.0 - tB);
      acc[0] += w;
      acc[1] += w * cx; acc[2] += w * cy; acc[3] += w * cz;
      for (int k = 0; k < 3; ++k) acc[4 + k] += ma * gA[k] - mb * gB[k];
      if (w > 0.0) {
        const double f = -(fa + fb) * P.inv_dx;
        if (f > bf || (f == bf && c < bi)) { bf = f; bi = c; }
      }
    }
    // block reduction
    for (int off = 16; off > 0; off >>= 1) {
      for (int k = 0; k < 7; ++k) acc[k] += __shfl_xor_sync(kFull, acc[k], off);
      const double of = __shfl_xor_sync(kFull, bf, off);
      const int oi = __shfl_xor_sync(kFull, bi, off);
      if (of > bf || (of == bf && oi < bi)) { bf = of; bi = oi; }
    }
    if (lane == 0) {
      for (int k = 0; k < 7; ++k) s_red[wid][k] = acc[k];
      s_bf[wid] = bf;
      s_bi[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {   // lanes c < 7: component c summed over the warps in order
      double tot = 0.0;
      double b = -DBL_MAX;
      int bidx = 0x7fffffff;
      for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
        if (lane < 7) tot += s_red[w][lane];
        if (s_bf[w] > b || (s_bf[w] == b && s_bi[w] < bidx)) { b = s_bf[w]; bidx = s_bi[w]; }
      }
      pair_done(P, W, W.pairs[p], pair_out, tot, bidx);
    }
    __syncthreads();
  }
}

}  // namespace

template <bool SMOOTH, int SET>
int blocks_per_sm() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow32<SMOOTH, SET>, narrow_warps<SET>() * 32, 0);
  return per_sm > 0 ? per_sm : 1;
}

int narrow_grid(const Params& P) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (P.precision == 1) return sms * 4;
  int per_sm = 1;
  if (P.smooth) {
    per_sm = P.kind_set == SET_CUBE ? blocks_per_sm<true, SET_CUBE>()
             : P.kind_set == SET_SC ? blocks_per_sm<true, SET_SC>() : blocks_per_sm<true, SET_ALL>();
  } else {
    per_sm = P.kind_set == SET_CUBE ? blocks_per_sm<false, SET_CUBE>()
             : P.kind_set == SET_SC ? blocks_per_sm<false, SET_SC>() : blocks_per_sm<false, SET_ALL>();
  }
  return sms * per_sm;
}

void launch_force(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel, double* pair_out,
                  cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // compiled per kind set (cubes only, or any) and with or without the
  // velocity-dependent law (damping from velocities, contact history, friction)
  const bool law = P.history || P.friction || (vel != nullptr && P.damping_c != 0.0);
  auto kern = P.kind_set == 2 ? (law ? k_force<2, true> : k_force<2, false>)
                              : (law ? k_force<0, true> : k_force<0, false>);
  launch_pdl(kern, dim3(sms > 0 ? sms : 1), dim3(kWarps * 32), 0, st, P, S, D, W, vel, pair_out);
}

void launch_narrow(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                   double* pair_out, int grid, cudaStream_t st) {
  if (P.box_mode == 1) {   // the paper's box pipeline instead of every node of the pair box
    launch_box(P, S, D, W, vel, pair_out, grid, st);
    return;
  }
  if (P.precision == 1) {
    if (P.smooth)
      launch_pdl(k_narrow64<true>, dim3(grid), dim3(256), 0, st, P, S, D, W, vel, pair_out);
    else
      launch_pdl(k_narrow64<false>, dim3(grid), dim3(256), 0, st, P, S, D, W, vel, pair_out);
    return;
  }
  const dim3 bc(narrow_warps<SET_CUBE>() * 32), bs(narrow_warps<SET_SC>() * 32), ba(narrow_warps<SET_ALL>() * 32);
  if (P.smooth) {
    if (P.kind_set == SET_CUBE) launch_pdl(k_narrow32<true, SET_CUBE>, dim3(grid), bc, 0, st, P, S, D, W, vel, pair_out);
    else if (P.kind_set == SET_SC) launch_pdl(k_narrow32<true, SET_SC>, dim3(grid), bs, 0, st, P, S, D, W, vel, pair_out);
    else launch_pdl(k_narrow32<true, SET_ALL>, dim3(grid), ba, 0, st, P, S, D, W, vel, pair_out);
  } else {
    if (P.kind_set == SET_CUBE) launch_pdl(k_narrow32<false, SET_CUBE>, dim3(grid), bc, 0, st, P, S, D, W, vel, pair_out);
    else if (P.kind_set == SET_SC) launch_pdl(k_narrow32<false, SET_SC>, dim3(grid), bs, 0, st, P, S, D, W, vel, pair_out);
    else launch_pdl(k_narrow32<false, SET_ALL>, dim3(grid), ba, 0, st, P, S, D, W, vel, pair_out);
  }
}

}  // namespace gbc
