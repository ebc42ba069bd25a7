// CPU FP64 oracle for the discrete contact model's per-pair overlap evaluation.
//
// TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header,
// table or helper with the CUDA library; it is the plain, slow, direct
// definition that the CUDA path is checked against.
//
// Paper: Marquardt, Hafen, Krause, "A novel model for direct numerical
// simulation of suspension dynamics with arbitrarily shaped convex particles"
// (arXiv:2401.10878).
//   * Sec. 2.2: poses refer to the centre of mass X_p (torque reference).
//   * Sec. 2.3, Eq. (contact_force_normal): F_n = 4/(3 pi) n_c E* sqrt(V_c d)(1 + c ddot_n);
//     E* = ((1-nu_A^2)/E_A + (1-nu_B^2)/E_B)^-1; Eq. (damping_factor) for c.
//   * Sec. 3.3.1: contact = sweep over the sample points of the overlap region,
//     giving overlap volume, contact point, contact normal, indentation depth, force.
//     A node belongs to a particle by the sign of its signed distance.
//   * Sec. 3.3.2: across a periodic boundary the contact lives on the side of
//     the lower-ID particle; the higher-ID particle is shifted there.
//   * Sec. 5.1: contact enlargement of the particles (inflate parameter).
//   * Sec. 4.3: particle-wall contacts; walls do not move.  A wall is the
//     half-space m . x <= h (unit m pointing out of the wall), not periodic;
//     its contacts are pairs (i, N + w) evaluated like particle pairs.
//
// Readings where the paper is silent (each is restated in the design notes):
//   sample set = lattice nodes k*dx of the intersection of the two particles'
//   node-range AABBs; sharp indicator H = [phi <= 0]; polytope/cuboid SDF =
//   max over face planes; smoothed indicator H_w(phi) = S(clamp(1/2 - phi/(w dx),0,1)),
//   S(t) = 3t^2 - 2t^3; contact normal from G = 1/2 (dV/dX_A - dV/dX_B) in its
//   band form; indentation depth d = max over overlap nodes of (-phi_A - phi_B);
//   prefactor 4/(3 pi) as printed; one damping factor c for all contacts, or
//   with the contact history each contact's own (from its first step's
//   approach speed) and, in the box pipeline, its last corrected box (relative
//   to X_i, widened by sqrt(0.75) dx) as the warm start that cuts the next
//   correction's starting box down (Sec. 4.3.3); a polytope whose volume
//   centroid is off its body origin is moved there (Sec. 2.2).
//
// The per-pair evaluation is a template over the scalar type so that the same
// code, run with forward-mode dual numbers, yields the oracle's own FP64
// gradient of sum_p (gF_p . F_p + gT_p . T_p) with respect to the poses.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared [-fopenmp].
// Contraction must stay off: the AABB node ranges are compared bit for bit.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ----------------------------------------------------------------------------
// status codes (same numbering as the public C-ABI, written independently)
enum { OR_OK = 0, OR_EINVAL = 1, OR_EDOMAIN = 5 };
enum { SH_SPHERE = 0, SH_CUBOID = 1, SH_POLYTOPE = 2, SH_WALL = 3 };

// ----------------------------------------------------------------------------
// forward-mode dual number with NT tangent directions
constexpr int NT = 14;

struct Dual {
  double v;
  double g[NT];
  Dual() : v(0.0) { for (double& x : g) x = 0.0; }
  Dual(double a) : v(a) { for (double& x : g) x = 0.0; }  // NOLINT (implicit by design)
};

inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v + b.v; for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] + b.g[i]; return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v - b.v; for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] - b.g[i]; return r;
}
inline Dual operator-(const Dual& a) {
  Dual r; r.v = -a.v; for (int i = 0; i < NT; ++i) r.g[i] = -a.g[i]; return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v * b.v;
  for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r; r.v = a.v / b.v;
  for (int i = 0; i < NT; ++i) r.g[i] = (a.g[i] * b.v - a.v * b.g[i]) / (b.v * b.v);
  return r;
}
inline Dual operator+(const Dual& a, double b) { Dual r = a; r.v += b; return r; }
inline Dual operator+(double a, const Dual& b) { Dual r = b; r.v += a; return r; }
inline Dual operator-(const Dual& a, double b) { Dual r = a; r.v -= b; return r; }
inline Dual operator-(double a, const Dual& b) { Dual r = -b; r.v += a; return r; }
inline Dual operator*(const Dual& a, double b) {
  Dual r; r.v = a.v * b; for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * b; return r;
}
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) {
  Dual r; r.v = a.v / b; for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] / b; return r;
}
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual sqrt(const Dual& a) {
  Dual r; r.v = std::sqrt(a.v);
  for (int i = 0; i < NT; ++i) r.g[i] = (r.v > 0.0) ? a.g[i] / (2.0 * r.v) : 0.0;
  return r;
}
inline Dual fabs(const Dual& a) { return (a.v < 0.0) ? -a : a; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double sqrt_s(double x) { return std::sqrt(x); }
inline Dual sqrt_s(const Dual& x) { return sqrt(x); }
inline double fabs_s(double x) { return std::fabs(x); }
inline Dual fabs_s(const Dual& x) { return fabs(x); }

// ----------------------------------------------------------------------------
struct Config {
  int32_t n_cells[3];
  double dx;
  int32_t indicator;     // 0 sharp, 1 smoothed
  double smooth_width;   // w in lattice cells
  double inflate;        // physical length, subtracted from every SDF (Sec. 5.1)
  double damping_c;      // c of Eq. (damping_factor), shared by all contacts
  double band_eps;       // classification band in lattice units (diagnostics only)
  int32_t n_walls;       // fixed walls: half-spaces m . x <= h, (m, h) per row of `walls`
  const double* walls;   // [n_walls, 4]
  const double* wall_young;
  const double* wall_poisson;
  int32_t box_mode;      // 0: every lattice node of the pair box; 1: the paper's box pipeline
  int32_t contact_resolution;   // N_c of the box pipeline (points per direction)
};

struct Shape {
  int type = SH_SPHERE;
  double p[3] = {0, 0, 0};         // sphere: radius; cuboid: half extents
  std::vector<double> planes;      // polytope: (n0, n1, n2, d) per face, n.y <= d; wall: (m, h), world frame
  std::vector<double> verts;       // vertices of the offset shape used for the AABB
};

// Rotation matrix of the normalised quaternion (w, x, y, z), Hamilton
// convention, body -> world, row-major, in homogeneous form: with
// s = 2 / |q|^2 the products of the raw components give R of q / |q|.  The
// operation order is fixed (and contraction is off) because the AABB node
// ranges are compared bit for bit.
template <class S>
void quat_to_rot(const S q_in[4], S R[9]) {
  const S w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];
  const S nn = ((w * w + x * x) + y * y) + z * z;
  const S s = 2.0 / nn;
  R[0] = 1.0 - s * (y * y + z * z);
  R[1] = s * (x * y - w * z);
  R[2] = s * (x * z + w * y);
  R[3] = s * (x * y + w * z);
  R[4] = 1.0 - s * (x * x + z * z);
  R[5] = s * (y * z - w * x);
  R[6] = s * (x * z - w * y);
  R[7] = s * (y * z + w * x);
  R[8] = 1.0 - s * (x * x + y * y);
}

// Vertices of the convex polytope {y : n_i . y <= d_i + delta}: every plane
// triple solved by Cramer's rule, kept when it satisfies all half-spaces.
std::vector<double> polytope_vertices(const std::vector<double>& pl, double delta) {
  std::vector<double> out;
  const int F = static_cast<int>(pl.size() / 4);
  double dmax = 1.0;
  for (int i = 0; i < F; ++i) dmax = std::max(dmax, std::fabs(pl[4 * i + 3] + delta));
  const double tol = 1e-9 * dmax;
  for (int i = 0; i < F; ++i)
    for (int j = i + 1; j < F; ++j)
      for (int k = j + 1; k < F; ++k) {
        const double* a = &pl[4 * i];
        const double* b = &pl[4 * j];
        const double* c = &pl[4 * k];
        const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
        const double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
        const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
        if (std::fabs(det) < 1e-12) continue;
        const double da = a[3] + delta, db = b[3] + delta, dc = c[3] + delta;
        double v[3];
        for (int t = 0; t < 3; ++t) v[t] = (da * bc[t] + db * ca[t] + dc * ab[t]) / det;
        bool inside = true;
        for (int m = 0; m < F && inside; ++m) {
          const double* e = &pl[4 * m];
          if (e[0] * v[0] + e[1] * v[1] + e[2] * v[2] - (e[3] + delta) > tol) inside = false;
        }
        if (inside) out.insert(out.end(), v, v + 3);
      }
  return out;
}

// A polyhedron {n_i . y <= d_i} with all d_i > 0 is bounded iff no direction u
// has n_i . u <= 0 for all i.  Extreme rays of the recession cone lie on
// intersections of two plane boundaries, so testing +-(n_i x n_j) suffices.
// Volume and centroid of the polytope {y : n_f . y <= d_f} with the origin
// inside, as pyramids from the origin over its faces: a face of area A at
// distance d has volume d A / 3 and its centroid 3/4 of the way from the
// origin to the face's area centroid (triangles of the face polygon, its
// vertices ordered around their mean).
bool polytope_centroid(const std::vector<double>& pl, double c[3]) {
  const std::vector<double> v = polytope_vertices(pl, 0.0);
  const int F = static_cast<int>(pl.size() / 4), nv = static_cast<int>(v.size() / 3);
  double V = 0.0, mom[3] = {0.0, 0.0, 0.0};
  for (int f = 0; f < F; ++f) {
    const double* e = &pl[4 * f];
    std::vector<const double*> pts;
    for (int i = 0; i < nv; ++i) {
      const double* w = &v[3 * i];
      if (std::fabs(e[0] * w[0] + e[1] * w[1] + e[2] * w[2] - e[3]) <= 1e-9 * std::max(1.0, std::fabs(e[3])))
        pts.push_back(w);
    }
    if (pts.size() < 3) continue;
    double ctr[3] = {0.0, 0.0, 0.0};
    for (const double* w : pts)
      for (int k = 0; k < 3; ++k) ctr[k] += w[k];
    for (int k = 0; k < 3; ++k) ctr[k] /= static_cast<double>(pts.size());
    // order around ctr by the angle in the face plane (reference direction: the first point)
    const double ref[3] = {pts[0][0] - ctr[0], pts[0][1] - ctr[1], pts[0][2] - ctr[2]};
    std::vector<std::pair<double, const double*>> order;
    for (const double* w : pts) {
      const double r[3] = {w[0] - ctr[0], w[1] - ctr[1], w[2] - ctr[2]};
      const double cx[3] = {ref[1] * r[2] - ref[2] * r[1], ref[2] * r[0] - ref[0] * r[2], ref[0] * r[1] - ref[1] * r[0]};
      const double sn = cx[0] * e[0] + cx[1] * e[1] + cx[2] * e[2];
      const double cs = ref[0] * r[0] + ref[1] * r[1] + ref[2] * r[2];
      order.push_back({std::atan2(sn, cs), w});
    }
    std::sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    double area = 0.0, ac[3] = {0.0, 0.0, 0.0};
    for (size_t t = 0; t < order.size(); ++t) {
      const double* p = order[t].second;
      const double* q = order[(t + 1) % order.size()].second;
      const double u[3] = {p[0] - ctr[0], p[1] - ctr[1], p[2] - ctr[2]};
      const double w[3] = {q[0] - ctr[0], q[1] - ctr[1], q[2] - ctr[2]};
      const double cx[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
      const double a = 0.5 * std::sqrt(cx[0] * cx[0] + cx[1] * cx[1] + cx[2] * cx[2]);
      area += a;
      for (int k = 0; k < 3; ++k) ac[k] += a * (ctr[k] + p[k] + q[k]) / 3.0;
    }
    if (!(area > 0.0)) continue;
    const double vf = e[3] * area / 3.0;
    V += vf;
    for (int k = 0; k < 3; ++k) mom[k] += vf * 0.75 * (ac[k] / area);
  }
  if (!(V > 0.0)) return false;
  for (int k = 0; k < 3; ++k) c[k] = mom[k] / V;
  return true;
}

bool polytope_bounded(const std::vector<double>& pl) {
  const int F = static_cast<int>(pl.size() / 4);
  if (F < 4) return false;
  for (int i = 0; i < F; ++i)
    for (int j = i + 1; j < F; ++j) {
      const double* a = &pl[4 * i];
      const double* b = &pl[4 * j];
      double u[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      const double nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      if (nu < 1e-12) continue;
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        bool ray = true;
        for (int m = 0; m < F && ray; ++m) {
          const double* e = &pl[4 * m];
          if (sgn * (e[0] * u[0] + e[1] * u[1] + e[2] * u[2]) / nu > 1e-12) ray = false;
        }
        if (ray) return false;
      }
    }
  return true;
}

// Signed distance of a shape at world point x (physical units), reduced by
// `inflate`; also the world gradient of the active branch and, for ties, the
// gap between the largest and second-largest face value (inf for a sphere).
template <class S>
S sdf(const Shape& sh, const S X[3], const S R[9], const double x[3], double inflate, S grad[3],
      double* gap) {
  if (sh.type == SH_WALL) {   // fixed half-space m . x <= h (world frame)
    const double* e = sh.planes.data();
    for (int k = 0; k < 3; ++k) grad[k] = S(e[k]);
    *gap = std::numeric_limits<double>::infinity();
    return S(((e[0] * x[0] + e[1] * x[1]) + e[2] * x[2]) - e[3] - inflate);
  }
  S r[3] = {x[0] - X[0], x[1] - X[1], x[2] - X[2]};
  if (sh.type == SH_SPHERE) {
    S nr = sqrt_s(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (val(nr) > 0.0) {
      for (int k = 0; k < 3; ++k) grad[k] = r[k] / nr;
    } else {
      for (int k = 0; k < 3; ++k) grad[k] = S(0.0);
    }
    *gap = std::numeric_limits<double>::infinity();
    return nr - sh.p[0] - inflate;
  }
  // body coordinates y = R^T r
  S y[3];
  for (int k = 0; k < 3; ++k) y[k] = R[0 * 3 + k] * r[0] + R[1 * 3 + k] * r[1] + R[2 * 3 + k] * r[2];
  S best(0.0);
  double gb[3] = {0, 0, 0};
  double bestv = -std::numeric_limits<double>::infinity();
  double second = -std::numeric_limits<double>::infinity();
  if (sh.type == SH_CUBOID) {
    for (int k = 0; k < 3; ++k) {
      S a = fabs_s(y[k]) - sh.p[k];
      if (val(a) > bestv) {
        second = bestv;
        bestv = val(a);
        best = a;
        gb[0] = gb[1] = gb[2] = 0.0;
        gb[k] = (val(y[k]) < 0.0) ? -1.0 : 1.0;
      } else if (val(a) > second) {
        second = val(a);
      }
    }
  } else {
    const int F = static_cast<int>(sh.planes.size() / 4);
    for (int i = 0; i < F; ++i) {
      const double* e = &sh.planes[4 * i];
      S a = (e[0] * y[0] + e[1] * y[1] + e[2] * y[2]) - e[3];
      if (val(a) > bestv) {
        second = bestv;
        bestv = val(a);
        best = a;
        gb[0] = e[0]; gb[1] = e[1]; gb[2] = e[2];
      } else if (val(a) > second) {
        second = val(a);
      }
    }
  }
  for (int k = 0; k < 3; ++k) grad[k] = R[k * 3 + 0] * gb[0] + R[k * 3 + 1] * gb[1] + R[k * 3 + 2] * gb[2];
  *gap = bestv - second;
  return best - inflate;
}

// Indicator H(phi) and the derivative of the smoothed profile dH_w/dphi.
// Sharp mode: H = [phi <= 0]; the derivative (used by the normal) is always
// the smoothed one.  Smoothed mode: H = S(t), t = clamp(1/2 - phi/wdx, 0, 1).
template <class S>
void indicator(bool smooth, double wdx, const S& phi, S* H, S* Hp) {
  S t = 0.5 - phi / wdx;
  if (val(t) <= 0.0) {
    *Hp = S(0.0);
    if (smooth) *H = S(0.0);
  } else if (val(t) >= 1.0) {
    *Hp = S(0.0);
    if (smooth) *H = S(1.0);
  } else {
    *Hp = -6.0 * t * (1.0 - t) / wdx;
    if (smooth) *H = t * t * (3.0 - 2.0 * t);
  }
  if (!smooth) *H = S(val(phi) <= 0.0 ? 1.0 : 0.0);
}

struct PairGeom {
  int i, j;
  int shift[3];   // image index s: X_j' = X_j - s * L
  int lo[3], hi[3];
};

template <class S>
struct PairResult {
  S V, xc[3], n[3], d, F[3], TA[3], TB[3];
  double G[3];
  double box_cells, n_band, n_gtie, d_gap, estar;
  double v_sens, m_sens, g_sens;  // first-order change of V, M, G for a perturbation eps of every phi
  double c_used;                  // damping factor the force law used
  // box pipeline: rough box (node indices), corrected box (physical), and
  // the nodes / faces whose outcome is within eps of changing
  int rough[6];
  double box[6];
  double n_rough_band, n_face_tie;
};

// Eq. (damping_factor): c from the coefficient of restitution e and the
// relative speed u0 at the initial contact (0 for u0 <= 0).
inline double damping_factor(double e, double u0) {
  if (!(u0 > 0.0)) return 0.0;
  return 1.5 * (1.0 - e) * (11.0 - e) / ((1.0 + 9.0 * e) * u0);
}

// The contact law of one pair: its damping factor c (of an ongoing contact,
// or the shared one), or, for a contact that begins at this step with the
// contact history on, c from this step's approach speed u0 = ddot_n
// (Eq. damping_factor); and the friction law of Eq. (contact_force_tangential).
struct ContactLaw {
  double c = 0.0;
  bool new_contact = false;
  double restitution = 1.0;
  bool friction = false;
  double mu_s = 0.0, mu_k = 0.0, u_k = 1.0;
  // box pipeline with the contact history (Sec. 4.3.3): the ongoing
  // contact's corrected box of the previous step, relative to X_i (or null)
  const double* warm_box = nullptr;
};

// Parameter interval [t0, t1] of the line p + t e inside a shape reduced by
// `inflate` (empty: t0 > t1): a sphere by its quadratic, a cuboid / polytope /
// wall by clipping against each face plane (world frame).
void line_interval(const Shape& sh, const double X[3], const double R[9], const double p[3], const double e[3],
                   double inflate, double* t0, double* t1) {
  const double inf = std::numeric_limits<double>::infinity();
  *t0 = -inf;
  *t1 = inf;
  if (sh.type == SH_SPHERE) {
    const double r = sh.p[0] + inflate;
    const double q[3] = {p[0] - X[0], p[1] - X[1], p[2] - X[2]};
    const double b = q[0] * e[0] + q[1] * e[1] + q[2] * e[2];   // |e| = 1
    const double c = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] - r * r;
    const double disc = b * b - c;
    if (disc < 0.0) {
      *t0 = inf;
      *t1 = -inf;
      return;
    }
    const double sq = std::sqrt(disc);
    *t0 = -b - sq;
    *t1 = -b + sq;
    return;
  }
  // faces (n_w, offset) with n_w . x <= offset along the line: a + t b <= 0
  auto clip = [&](const double nw[3], double off) {
    const double a = (nw[0] * p[0] + nw[1] * p[1] + nw[2] * p[2]) - off;
    const double b = nw[0] * e[0] + nw[1] * e[1] + nw[2] * e[2];
    if (b > 0.0) {
      *t1 = std::min(*t1, -a / b);
    } else if (b < 0.0) {
      *t0 = std::max(*t0, -a / b);
    } else if (a > 0.0) {
      *t0 = inf;
      *t1 = -inf;
    }
  };
  if (sh.type == SH_WALL) {
    clip(sh.planes.data(), sh.planes[3] + inflate);
    return;
  }
  if (sh.type == SH_CUBOID) {
    for (int k = 0; k < 3; ++k)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const double nw[3] = {sgn * R[0 * 3 + k], sgn * R[1 * 3 + k], sgn * R[2 * 3 + k]};   // +-R e_k
        clip(nw, (nw[0] * X[0] + nw[1] * X[1] + nw[2] * X[2]) + sh.p[k] + inflate);
      }
    return;
  }
  const int F = static_cast<int>(sh.planes.size() / 4);
  for (int f = 0; f < F; ++f) {
    const double* b = &sh.planes[4 * f];
    const double nw[3] = {R[0] * b[0] + R[1] * b[1] + R[2] * b[2], R[3] * b[0] + R[4] * b[1] + R[5] * b[2],
                          R[6] * b[0] + R[7] * b[1] + R[8] * b[2]};
    clip(nw, (nw[0] * X[0] + nw[1] * X[1] + nw[2] * X[2]) + b[3] + inflate);
  }
}

// The paper's box pipeline (Sec. 3.3.1), restated:
//  1. rough detection: the lattice nodes where both signed distances are
//     below half the cell diagonal, sqrt(0.75) dx (all inside the pair box,
//     whose node ranges are widened by that much); their node-index bounds are
//     the rough box (none: no contact);
//  2. correction: the rough box widened by sqrt(0.75) dx (every point inside
//     both shapes lies within that distance of such a node) is B0; on each of
//     its six faces an N_c x N_c grid of points (cell centres of the face)
//     casts lines along the inward normal; each line's entry into the overlap
//     (both shapes, the line clipped exactly) is its distance to the contact,
//     and the face moves inward by the smallest such distance (a face whose
//     lines all miss stays; an axis left empty keeps B0's extent);
//  3. the N_c^3 cell centres of the corrected box are the sample points.
// Fills the sample box (lo, spacing) or returns false when no node is rough-in.
template <class S>
bool box_pipeline(const Config& cfg, const Shape& A, const Shape& B, const PairGeom& pg, const double XA[3],
                  const double RA[9], const double XB[3], const double RB[9], PairResult<S>& res, double lo[3],
                  double step[3], const double* warm = nullptr) {
  const double dx = cfg.dx;
  const int Nc = cfg.contact_resolution;
  const double srough = std::sqrt(0.75) * dx;
  const double eps = cfg.band_eps * dx;
  int mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  double n_rough_band = 0;
  // (the node ranges of the box pipeline are widened by sqrt(0.75) dx, so
  // the pair box holds every node where both distances are below it)
  for (int kz = pg.lo[2]; kz <= pg.hi[2]; ++kz)
    for (int ky = pg.lo[1]; ky <= pg.hi[1]; ++ky)
      for (int kx = pg.lo[0]; kx <= pg.hi[0]; ++kx) {
        const double x[3] = {kx * dx, ky * dx, kz * dx};
        double gA[3], gB[3], gapA, gapB;
        const double pa = sdf(A, XA, RA, x, cfg.inflate, gA, &gapA);
        const double pb = sdf(B, XB, RB, x, cfg.inflate, gB, &gapB);
        if (pa < srough && pb < srough) {
          const int k[3] = {kx, ky, kz};
          for (int a = 0; a < 3; ++a) {
            mn[a] = std::min(mn[a], k[a]);
            mx[a] = std::max(mx[a], k[a]);
          }
        }
        const bool loose = pa < srough + eps && pb < srough + eps;
        const bool strict = pa < srough - eps && pb < srough - eps;
        if (loose && !strict) n_rough_band += 1;
      }
  res.n_rough_band = n_rough_band;
  if (mn[0] > mx[0]) return false;
  double b0lo[3], b0hi[3];
  for (int a = 0; a < 3; ++a) {
    res.rough[a] = mn[a];
    res.rough[3 + a] = mx[a];
    b0lo[a] = mn[a] * dx - srough;
    b0hi[a] = mx[a] * dx + srough;
  }
  // warm start (Sec. 4.3.3): an ongoing contact's corrected box of the last
  // step, moved with particle i and widened by the same sqrt(0.75) dx, cuts
  // B0 down (per axis, unless the cut leaves nothing)
  if (warm != nullptr)
    for (int a = 0; a < 3; ++a) {
      const double wl = (XA[a] + warm[a]) - srough, wh = (XA[a] + warm[3 + a]) + srough;
      const double l = std::max(b0lo[a], wl), h = std::min(b0hi[a], wh);
      if (l < h) {
        b0lo[a] = l;
        b0hi[a] = h;
      }
    }
  // correction: face (axis k, lower / upper), lines along the inward normal
  double shift[3][2];
  double n_face_tie = 0;
  for (int k = 0; k < 3; ++k)
    for (int side = 0; side < 2; ++side) {
      const int u = k == 0 ? 1 : 0, v = k == 2 ? 1 : 2;
      const double len = b0hi[k] - b0lo[k];
      double best = std::numeric_limits<double>::infinity(), second = best;
      for (int a = 0; a < Nc; ++a)
        for (int b = 0; b < Nc; ++b) {
          double p[3], e[3] = {0.0, 0.0, 0.0};
          p[u] = b0lo[u] + (a + 0.5) * (b0hi[u] - b0lo[u]) / Nc;
          p[v] = b0lo[v] + (b + 0.5) * (b0hi[v] - b0lo[v]) / Nc;
          p[k] = side == 0 ? b0lo[k] : b0hi[k];
          e[k] = side == 0 ? 1.0 : -1.0;
          double a0, a1, c0, c1;
          line_interval(A, XA, RA, p, e, cfg.inflate, &a0, &a1);
          line_interval(B, XB, RB, p, e, cfg.inflate, &c0, &c1);
          const double tin = std::max(std::max(a0, c0), 0.0);
          const double tout = std::min(std::min(a1, c1), len);
          if (tin <= tout) {
            if (tin < best) {
              second = best;
              best = tin;
            } else if (tin < second) {
              second = tin;
            }
          }
        }
      shift[k][side] = std::isfinite(best) ? best : 0.0;
      if (std::isfinite(second) && second - best < 1e-4 * dx && second != best) n_face_tie += 1;
    }
  res.n_face_tie = n_face_tie;
  for (int k = 0; k < 3; ++k) {
    double l = b0lo[k] + shift[k][0], h = b0hi[k] - shift[k][1];
    if (!(l <= h)) {
      l = b0lo[k];
      h = b0hi[k];
    }
    lo[k] = l;
    step[k] = (h - l) / Nc;
    res.box[k] = l;
    res.box[3 + k] = h;
  }
  return true;
}

// Sweep of every lattice node of the pair box (Sec. 3.3.1) and the force law
// of Eq. (contact_force_normal).  XA, qA, XB (already the image X_j'), qB are
// the poses; vel (nullable) holds (u, omega) per particle.
template <class S>
PairResult<S> eval_pair(const Config& cfg, const Shape& A, const Shape& B, const PairGeom& pg,
                        const S XA[3], const S qA[4], const S XB[3], const S qB[4], const double* velA,
                        const double* velB, double estar, const ContactLaw& law) {
  const double dx = cfg.dx;
  const bool smooth = cfg.indicator == 1;
  const double wdx = cfg.smooth_width * dx;
  const double eps = cfg.band_eps * dx;
  S RA[9], RB[9];
  quat_to_rot(qA, RA);
  quat_to_rot(qB, RB);

  S SW(0.0), SM[3] = {S(0.0), S(0.0), S(0.0)}, SG[3] = {S(0.0), S(0.0), S(0.0)};
  S dbest(0.0);
  double top1 = -std::numeric_limits<double>::infinity(), top2 = top1;
  double n_band = 0, n_gtie = 0, v_sens = 0, m_sens = 0, g_sens = 0;
  const double o[3] = {pg.lo[0] * dx, pg.lo[1] * dx, pg.lo[2] * dx};
  // sample set: every node of the pair box, or the box pipeline's N_c^3 points
  const bool boxed = cfg.box_mode == 1;
  int cnt[3] = {pg.hi[0] - pg.lo[0] + 1, pg.hi[1] - pg.lo[1] + 1, pg.hi[2] - pg.lo[2] + 1};
  double s_lo[3] = {o[0], o[1], o[2]}, s_step[3] = {dx, dx, dx};
  PairResult<S> res;
  for (int k = 0; k < 6; ++k) { res.rough[k] = 0; res.box[k] = 0.0; }
  res.n_rough_band = res.n_face_tie = 0.0;
  if (boxed) {
    double XAd[3], XBd[3], RAd[9], RBd[9];
    for (int k = 0; k < 3; ++k) { XAd[k] = val(XA[k]); XBd[k] = val(XB[k]); }
    for (int k = 0; k < 9; ++k) { RAd[k] = val(RA[k]); RBd[k] = val(RB[k]); }
    if (box_pipeline(cfg, A, B, pg, XAd, RAd, XBd, RBd, res, s_lo, s_step, law.warm_box)) {
      for (int k = 0; k < 3; ++k) {
        cnt[k] = cfg.contact_resolution;
        s_lo[k] += 0.5 * s_step[k];   // cell centres
      }
    } else {
      cnt[0] = cnt[1] = cnt[2] = 0;
    }
  }
  for (int iz = 0; iz < cnt[2]; ++iz)
    for (int iy = 0; iy < cnt[1]; ++iy)
      for (int ix = 0; ix < cnt[0]; ++ix) {
        const double x[3] = {boxed ? s_lo[0] + ix * s_step[0] : (pg.lo[0] + ix) * dx,
                             boxed ? s_lo[1] + iy * s_step[1] : (pg.lo[1] + iy) * dx,
                             boxed ? s_lo[2] + iz * s_step[2] : (pg.lo[2] + iz) * dx};
        const double c[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
        S gA[3], gB[3];
        double gapA, gapB;
        S phA = sdf(A, XA, RA, x, cfg.inflate, gA, &gapA);
        S phB = sdf(B, XB, RB, x, cfg.inflate, gB, &gapB);
        S HA, HpA, HB, HpB;
        indicator(smooth, wdx, phA, &HA, &HpA);
        indicator(smooth, wdx, phB, &HB, &HpB);
        S W = HA * HB;
        SW = SW + W;
        for (int k = 0; k < 3; ++k) SM[k] = SM[k] + W * c[k];
        for (int k = 0; k < 3; ++k) SG[k] = SG[k] + (-(HpA * HB)) * gA[k] + (HA * HpB) * gB[k];
        if (val(W) > 0.0) {
          S f = -phA - phB;
          const double fv = val(f);
          if (fv > top1) {
            top2 = top1;
            top1 = fv;
            dbest = f;
          } else if (fv > top2) {
            top2 = fv;
          }
        }
        // diagnostics: cells whose classification or active face is ambiguous
        // at the eps level (reported, never used in the result)
        const double pa = val(phA), pb = val(phB);
        if (!smooth) {
          const bool loose = pa <= eps && pb <= eps;
          const bool strict = pa <= -eps && pb <= -eps;
          if (loose && !strict) n_band += 1;
        }
        const bool gA_on = val(HpA) != 0.0 && (smooth ? val(HB) > 0.0 : pb <= eps);
        const bool gB_on = val(HpB) != 0.0 && (smooth ? val(HA) > 0.0 : pa <= eps);
        const bool tieA = gapA < eps || (!smooth && std::fabs(pb) <= eps);
        const bool tieB = gapB < eps || (!smooth && std::fabs(pa) <= eps);
        if ((gA_on && tieA) || (gB_on && tieB)) n_gtie += 1;
        // sensitivities (diagnostics): |dW/dphi| eps, |dW/dphi| eps |c|, and the
        // change of the normal's band terms; smoothed H only (sharp H is a step)
        const double hpa = std::fabs(val(HpA)), hpb = std::fabs(val(HpB));
        const double ta = std::min(std::max(0.5 - pa / wdx, 0.0), 1.0);
        const double tb = std::min(std::max(0.5 - pb / wdx, 0.0), 1.0);
        const double dhpa = (ta > 0.0 && ta < 1.0) ? 6.0 * std::fabs(1.0 - 2.0 * ta) / (wdx * wdx) : 0.0;
        const double dhpb = (tb > 0.0 && tb < 1.0) ? 6.0 * std::fabs(1.0 - 2.0 * tb) / (wdx * wdx) : 0.0;
        const double ha = val(HA), hb = val(HB);
        if (smooth) {
          const double dw = hpa * hb + ha * hpb;
          v_sens += dw * eps;
          m_sens += dw * eps * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
          g_sens += (dhpa * hb + 2.0 * hpa * hpb + ha * dhpb) * eps;
        } else {
          g_sens += (dhpa * hb + ha * dhpb) * eps;
        }
      }

  // volume of one sample: dx^3 on the lattice, the sample cell in the box pipeline
  const double dx3 = boxed ? s_step[0] * s_step[1] * s_step[2] : dx * dx * dx;
  res.box_cells = double(cnt[0]) * double(cnt[1]) * double(cnt[2]);
  res.n_band = n_band;
  res.n_gtie = n_gtie;
  res.d_gap = (top2 > -std::numeric_limits<double>::infinity()) ? (top1 - top2) / dx
                                                                : std::numeric_limits<double>::infinity();
  res.estar = estar;
  res.v_sens = dx3 * v_sens;
  res.m_sens = dx3 * m_sens;
  res.g_sens = 0.5 * dx3 * g_sens;
  S G[3];
  for (int k = 0; k < 3; ++k) {
    G[k] = 0.5 * dx3 * SG[k];
    res.G[k] = val(G[k]);
  }
  S V = dx3 * SW;
  res.V = V;
  for (int k = 0; k < 3; ++k) {
    res.xc[k] = S(0.0); res.n[k] = S(0.0); res.F[k] = S(0.0); res.TA[k] = S(0.0); res.TB[k] = S(0.0);
  }
  res.d = S(0.0);
  if (!(val(V) > 0.0)) {
    res.V = S(0.0);
    return res;
  }
  for (int k = 0; k < 3; ++k) res.xc[k] = o[k] + (dx3 * SM[k]) / V;
  S gn = sqrt_s(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
  if (val(gn) > 1e-12 * dx * dx) {
    for (int k = 0; k < 3; ++k) res.n[k] = G[k] / gn;
  } else if (B.type == SH_WALL) {   // into the wall: -m
    for (int k = 0; k < 3; ++k) res.n[k] = S(-B.planes[k]);
  } else {
    S dX[3] = {XB[0] - XA[0], XB[1] - XA[1], XB[2] - XA[2]};
    S dn = sqrt_s(dX[0] * dX[0] + dX[1] * dX[1] + dX[2] * dX[2]);
    if (val(dn) > 0.0)
      for (int k = 0; k < 3; ++k) res.n[k] = dX[k] / dn;
  }
  S d = (top1 > 0.0) ? dbest : S(0.0);
  res.d = d;
  // velocity of A relative to B at the contact point; its normal part ddot_n
  // is positive when approaching (n points from A to B)
  const bool have_vel = velA != nullptr && velB != nullptr;
  S uab[3] = {S(0.0), S(0.0), S(0.0)};
  S ddot(0.0);
  if (have_vel) {
    S ra[3] = {res.xc[0] - XA[0], res.xc[1] - XA[1], res.xc[2] - XA[2]};
    S rb[3] = {res.xc[0] - XB[0], res.xc[1] - XB[1], res.xc[2] - XB[2]};
    const double* wa = velA + 3;
    const double* wb = velB + 3;
    S ua[3] = {velA[0] + (wa[1] * ra[2] - wa[2] * ra[1]), velA[1] + (wa[2] * ra[0] - wa[0] * ra[2]),
               velA[2] + (wa[0] * ra[1] - wa[1] * ra[0])};
    S ub[3] = {velB[0] + (wb[1] * rb[2] - wb[2] * rb[1]), velB[1] + (wb[2] * rb[0] - wb[0] * rb[2]),
               velB[2] + (wb[0] * rb[1] - wb[1] * rb[0])};
    for (int k = 0; k < 3; ++k) uab[k] = ua[k] - ub[k];
    ddot = uab[0] * res.n[0] + uab[1] * res.n[1] + uab[2] * res.n[2];
  }
  // damping factor: the contact's own, or from u0 = ddot_n at the start of the contact
  const double c = law.new_contact ? damping_factor(law.restitution, have_vel ? val(ddot) : 0.0) : law.c;
  res.c_used = c;
  S damp(1.0);
  if (have_vel && c != 0.0) {
    damp = 1.0 + c * ddot;
    if (val(damp) < 0.0) damp = S(0.0);
  }
  S vd = V * d;
  S fmag(0.0);
  if (val(vd) > 0.0) fmag = (4.0 / (3.0 * M_PI)) * estar * sqrt_s(vd) * damp;
  for (int k = 0; k < 3; ++k) res.F[k] = fmag * res.n[k];
  // friction, Eq. (contact_force_tangential): the force on A opposes A's
  // tangential velocity relative to B, so B receives +coef |F_n| t
  if (law.friction && have_vel && val(fmag) > 0.0) {
    S ut[3];
    for (int k = 0; k < 3; ++k) ut[k] = uab[k] - ddot * res.n[k];
    const S utn = sqrt_s(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    if (val(utn) > 0.0) {
      const S a = utn / law.u_k;
      const double ratio = law.mu_k / law.mu_s;
      const double mus_star = law.mu_s * (1.0 - 0.09 * ratio * ratio * ratio * ratio);
      const S a2 = a * a;
      const S coef = (2.0 * mus_star - law.mu_k) * a2 / (a2 * a2 + 1.0) + law.mu_k - law.mu_k / (a2 + 1.0);
      for (int k = 0; k < 3; ++k) res.F[k] = res.F[k] + coef * fmag * ut[k] / utn;
    }
  }
  // F acts on B, -F on A; torques about each particle's centre of mass (Sec. 2.2)
  S ra[3] = {res.xc[0] - XA[0], res.xc[1] - XA[1], res.xc[2] - XA[2]};
  S rb[3] = {res.xc[0] - XB[0], res.xc[1] - XB[1], res.xc[2] - XB[2]};
  S FA[3] = {-res.F[0], -res.F[1], -res.F[2]};
  res.TA[0] = ra[1] * FA[2] - ra[2] * FA[1];
  res.TA[1] = ra[2] * FA[0] - ra[0] * FA[2];
  res.TA[2] = ra[0] * FA[1] - ra[1] * FA[0];
  res.TB[0] = rb[1] * res.F[2] - rb[2] * res.F[1];
  res.TB[1] = rb[2] * res.F[0] - rb[0] * res.F[2];
  res.TB[2] = rb[0] * res.F[1] - rb[1] * res.F[0];
  return res;
}

// ----------------------------------------------------------------------------
struct Problem {
  Config cfg;
  int n = 0;        // particles; shapes/young/poisson hold them, then the walls
  std::vector<Shape> shapes;
  std::vector<double> young, poisson;
  std::vector<int> lo, hi;   // node ranges [n,3]
  std::vector<double> shift; // [n,3]: body origin moved to the centroid by this (polytopes)
  std::vector<PairGeom> pairs;
};

// Node box of particle range [lo, hi] against the wall m . x <= h widened by
// delta: empty (false) when even the range's lowest corner in m has
// m . x > h + delta; else the range clipped, per axis with m_k != 0, to the
// nodes that some node of the range with that coordinate keeps inside (and
// false if rounding leaves no node).  Plain FP64 operations in this order,
// no contraction: the box is compared bit for bit.
bool wall_box(const Config& c, const double* e, double delta, const int* lo_in, const int* hi_in, int lo[3],
              int hi[3]) {
  const double H = e[3] + delta;
  double t[3];
  for (int k = 0; k < 3; ++k) {
    const int ck = e[k] > 0.0 ? lo_in[k] : hi_in[k];
    t[k] = e[k] * (ck * c.dx);
    lo[k] = lo_in[k];
    hi[k] = hi_in[k];
  }
  if (!(((t[0] + t[1]) + t[2]) <= H)) return false;
  for (int k = 0; k < 3; ++k) {
    if (e[k] == 0.0) continue;
    const double rest = k == 0 ? t[1] + t[2] : (k == 1 ? t[0] + t[2] : t[0] + t[1]);
    const double b = ((H - rest) / e[k]) / c.dx;
    if (e[k] > 0.0) {
      if (b < hi[k]) hi[k] = static_cast<int>(std::floor(b));
    } else {
      if (b > lo[k]) lo[k] = static_cast<int>(std::ceil(b));
    }
  }
  return lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2];   // rounding may leave no node
}

int build_problem(Problem& pb, const Config* cfg, int32_t n, const int32_t* shape_type,
                  const double* shape_param, const int32_t* face_offset, const double* planes,
                  const double* young, const double* poisson, const double* pos, const double* quat) {
  pb.cfg = *cfg;
  pb.n = n;
  const Config& c = pb.cfg;
  if (n < 0 || !(c.dx > 0.0) || !std::isfinite(c.dx)) return OR_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (c.n_cells[k] < 1) return OR_EINVAL;
  if (c.indicator != 0 && c.indicator != 1) return OR_EINVAL;
  if (c.box_mode != 0 && c.box_mode != 1) return OR_EINVAL;
  if (c.box_mode == 1 && (c.contact_resolution < 1 || c.contact_resolution > 64)) return OR_EINVAL;
  if (!(c.smooth_width > 0.0)) return OR_EINVAL;
  if (!(c.inflate >= 0.0) || !(c.damping_c >= 0.0)) return OR_EINVAL;
  // offset used for the AABB: inflation plus, in smoothed mode, half the band
  // offset of the node ranges: inflation plus, in smoothed mode, half the band;
  // the box pipeline widens them to its rough-detection threshold sqrt(0.75) dx
  double band = (c.indicator == 1) ? (0.5 * c.smooth_width) * c.dx : 0.0;
  if (c.box_mode == 1) band = std::max(band, std::sqrt(0.75) * c.dx);
  const double delta = c.inflate + band;
  pb.shapes.resize(n);
  pb.shift.assign(3 * static_cast<size_t>(std::max(n, 0)), 0.0);
  pb.young.assign(young, young + n);
  pb.poisson.assign(poisson, poisson + n);
  double rmax = 0.0;
  for (int p = 0; p < n; ++p) {
    Shape& s = pb.shapes[p];
    s.type = shape_type[p];
    for (int k = 0; k < 3; ++k) s.p[k] = shape_param[3 * p + k];
    if (!(young[p] > 0.0) || !(poisson[p] >= 0.0) || !(poisson[p] < 1.0)) return OR_EINVAL;
    double circ = 0.0;
    if (s.type == SH_SPHERE) {
      if (!(s.p[0] > 0.0)) return OR_EINVAL;
      circ = s.p[0] + delta;
    } else if (s.type == SH_CUBOID) {
      for (int k = 0; k < 3; ++k)
        if (!(s.p[k] > 0.0)) return OR_EINVAL;
      const double e[3] = {s.p[0] + delta, s.p[1] + delta, s.p[2] + delta};
      circ = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    } else if (s.type == SH_POLYTOPE) {
      const int f0 = face_offset[p], f1 = face_offset[p + 1];
      if (f1 - f0 < 4) return OR_EINVAL;
      s.planes.assign(planes + 4 * f0, planes + 4 * f1);
      for (int f = 0; f < f1 - f0; ++f) {
        double* e = &s.planes[4 * f];
        const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        if (std::fabs(nn - 1.0) > 1e-9) return OR_EINVAL;  // unit normals required
        if (!(e[3] > 0.0)) return OR_EINVAL;                // origin strictly inside
      }
      if (!polytope_bounded(s.planes)) return OR_EINVAL;
      // poses refer to the centre of mass (Sec. 2.2): a body origin further than
      // 1e-6 x (smallest d) from the volume centroid is moved there, d_f -= n_f . c
      double cm[3], dmin = std::numeric_limits<double>::infinity();
      if (!polytope_centroid(s.planes, cm)) return OR_EINVAL;
      for (int f = 0; f < f1 - f0; ++f) dmin = std::min(dmin, s.planes[4 * f + 3]);
      if (std::sqrt(cm[0] * cm[0] + cm[1] * cm[1] + cm[2] * cm[2]) > 1e-6 * dmin) {
        for (int f = 0; f < f1 - f0; ++f) {
          double* e = &s.planes[4 * f];
          e[3] -= e[0] * cm[0] + e[1] * cm[1] + e[2] * cm[2];
          if (!(e[3] > 0.0)) return OR_EINVAL;
        }
        for (int k = 0; k < 3; ++k) pb.shift[3 * p + k] = cm[k];
      }
      s.verts = polytope_vertices(s.planes, delta);
      if (s.verts.size() < 12) return OR_EINVAL;
      for (size_t v = 0; v < s.verts.size(); v += 3) {
        const double* w = &s.verts[v];
        circ = std::max(circ, std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
      }
    } else {
      return OR_EINVAL;
    }
    rmax = std::max(rmax, circ);
  }
  // walls: shapes N + w, unit normals, materials
  if (c.n_walls < 0 || (c.n_walls > 0 && (c.walls == nullptr || c.wall_young == nullptr || c.wall_poisson == nullptr)))
    return OR_EINVAL;
  for (int w = 0; w < c.n_walls; ++w) {
    const double* e = c.walls + 4 * w;
    const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (std::fabs(nn - 1.0) > 1e-9 || !std::isfinite(e[3])) return OR_EINVAL;
    if (!(c.wall_young[w] > 0.0) || !(c.wall_poisson[w] >= 0.0) || !(c.wall_poisson[w] < 1.0)) return OR_EINVAL;
    Shape s;
    s.type = SH_WALL;
    s.planes.assign(e, e + 4);
    pb.shapes.push_back(s);
    pb.young.push_back(c.wall_young[w]);
    pb.poisson.push_back(c.wall_poisson[w]);
  }
  // at most one periodic image of a partner can overlap (Sec. 3.3.2 reading)
  for (int k = 0; k < 3; ++k)
    if (n > 0 && !(c.n_cells[k] * c.dx > 4.0 * rmax + 2.0 * c.dx)) return OR_EDOMAIN;

  pb.lo.assign(3 * n, 0);
  pb.hi.assign(3 * n, 0);
  for (int p = 0; p < n; ++p) {
    const double* X = pos + 3 * p;
    const double* q = quat + 4 * p;
    for (int k = 0; k < 3; ++k) {
      const double L = c.n_cells[k] * c.dx;
      if (!(X[k] >= 0.0) || !(X[k] < L)) return OR_EINVAL;
    }
    const double qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(qn > 1e-24) || !std::isfinite(qn)) return OR_EINVAL;
    double R[9];
    quat_to_rot(q, R);
    const Shape& s = pb.shapes[p];
    double mn[3], mx[3];
    if (s.type == SH_SPHERE) {
      const double rad = s.p[0] + delta;
      for (int k = 0; k < 3; ++k) { mn[k] = X[k] - rad; mx[k] = X[k] + rad; }
    } else if (s.type == SH_CUBOID) {
      const double e0 = s.p[0] + delta, e1 = s.p[1] + delta, e2 = s.p[2] + delta;
      for (int k = 0; k < 3; ++k) {
        const double ext = std::fabs(R[3 * k + 0]) * e0 + std::fabs(R[3 * k + 1]) * e1 +
                           std::fabs(R[3 * k + 2]) * e2;
        mn[k] = X[k] - ext;
        mx[k] = X[k] + ext;
      }
    } else {
      double wmn[3] = {std::numeric_limits<double>::infinity(), std::numeric_limits<double>::infinity(),
                       std::numeric_limits<double>::infinity()};
      double wmx[3] = {-wmn[0], -wmn[1], -wmn[2]};
      for (size_t v = 0; v < s.verts.size(); v += 3) {
        const double* w = &s.verts[v];
        for (int k = 0; k < 3; ++k) {
          const double t = R[3 * k + 0] * w[0] + R[3 * k + 1] * w[1] + R[3 * k + 2] * w[2];
          wmn[k] = std::min(wmn[k], t);
          wmx[k] = std::max(wmx[k], t);
        }
      }
      for (int k = 0; k < 3; ++k) { mn[k] = X[k] + wmn[k]; mx[k] = X[k] + wmx[k]; }
    }
    for (int k = 0; k < 3; ++k) {
      pb.lo[3 * p + k] = static_cast<int>(std::ceil(mn[k] / c.dx));
      pb.hi[3 * p + k] = static_cast<int>(std::floor(mx[k] / c.dx));
    }
  }
  // O(N^2) candidate test with the image of j nearest to i (Sec. 3.3.2)
  pb.pairs.clear();
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      PairGeom g;
      g.i = i;
      g.j = j;
      bool hit = true;
      for (int k = 0; k < 3 && hit; ++k) {
        const double L = c.n_cells[k] * c.dx;
        const int s = static_cast<int>(std::nearbyint((pos[3 * j + k] - pos[3 * i + k]) / L));
        g.shift[k] = s;
        g.lo[k] = std::max(pb.lo[3 * i + k], pb.lo[3 * j + k] - s * c.n_cells[k]);
        g.hi[k] = std::min(pb.hi[3 * i + k], pb.hi[3 * j + k] - s * c.n_cells[k]);
        if (g.lo[k] > g.hi[k]) hit = false;
      }
      if (hit) pb.pairs.push_back(g);
    }
    // particle-wall candidates: nodes of i's range with m . x <= h + delta
    // (the wall's band-widened half-space); the box is i's range clipped to it
    for (int w = 0; w < c.n_walls; ++w) {
      PairGeom g;
      if (wall_box(c, c.walls + 4 * w, delta, &pb.lo[3 * i], &pb.hi[3 * i], g.lo, g.hi)) {
        g.i = i;
        g.j = n + w;
        g.shift[0] = g.shift[1] = g.shift[2] = 0;
        pb.pairs.push_back(g);
      }
    }
  }
  return OR_OK;
}

double effective_modulus(double EA, double nuA, double EB, double nuB) {
  return 1.0 / ((1.0 - nuA * nuA) / EA + (1.0 - nuB * nuB) / EB);
}

// Pose of the pair's partner j: its image position, or for a wall the
// origin with the identity rotation; its velocity (a wall is at rest).
void image_pos(const Problem& pb, const PairGeom& g, const double* pos, double XB[3]) {
  for (int k = 0; k < 3; ++k)
    XB[k] = g.j < pb.n ? pos[3 * g.j + k] - g.shift[k] * (pb.cfg.n_cells[k] * pb.cfg.dx) : 0.0;
}
const double kIdentityQuat[4] = {1.0, 0.0, 0.0, 0.0};
const double kRest[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
const double* partner_quat(const Problem& pb, const PairGeom& g, const double* quat) {
  return g.j < pb.n ? quat + 4 * g.j : kIdentityQuat;
}
const double* partner_vel(const Problem& pb, const PairGeom& g, const double* vel) {
  if (vel == nullptr) return nullptr;
  return g.j < pb.n ? vel + 6 * g.j : kRest;
}

void set_threads(int32_t n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
}

}  // namespace

// ============================================================================
// C interface
extern "C" {

typedef struct {
  int32_t n_cells[3];
  double dx;
  int32_t indicator;
  double smooth_width;
  double inflate;
  double damping_c;
  double band_eps;
  int32_t n_walls;
  const double* walls;
  const double* wall_young;
  const double* wall_poisson;
  int32_t box_mode;
  int32_t contact_resolution;
} oracle_config;

// Volume centroid of a polytope given by n_faces rows (n, d) (origin inside).
// Returns 0, or 1 for a polytope the centroid cannot be formed for.
int32_t oracle_polytope_centroid(const double* planes, int32_t n_faces, double* centroid) {
  std::vector<double> pl(planes, planes + 4 * static_cast<size_t>(n_faces));
  if (n_faces < 4 || !polytope_bounded(pl)) return OR_EINVAL;
  return polytope_centroid(pl, centroid) ? OR_OK : OR_EINVAL;
}

int32_t oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_rotation(const double* q, double* R) { quat_to_rot(q, R); }

double oracle_effective_modulus(double EA, double nuA, double EB, double nuB) {
  return effective_modulus(EA, nuA, EB, nuB);
}

// Eq. (damping_factor): c from the coefficient of restitution e and the
// relative speed u0 at first contact.
double oracle_damping_factor(double e, double u0) {
  if (!(u0 > 0.0)) return 0.0;
  return 1.5 * (1.0 - e) * (11.0 - e) / ((1.0 + 9.0 * e) * u0);
}

// Normal force magnitude of Eq. (contact_force_normal).
double oracle_normal_force(double estar, double V, double d, double c, double ddot) {
  double damp = 1.0 + c * ddot;
  if (damp < 0.0) damp = 0.0;
  if (!(V * d > 0.0)) return 0.0;
  return (4.0 / (3.0 * M_PI)) * estar * std::sqrt(V * d) * damp;
}

int32_t oracle_polytope_vertices(int32_t n_planes, const double* planes, double delta, int32_t max_verts,
                                 double* verts) {
  std::vector<double> pl(planes, planes + 4 * n_planes);
  if (!polytope_bounded(pl)) return -1;
  std::vector<double> v = polytope_vertices(pl, delta);
  const int nv = static_cast<int>(v.size() / 3);
  for (int i = 0; i < std::min(nv, static_cast<int>(max_verts)); ++i)
    for (int k = 0; k < 3; ++k) verts[3 * i + k] = v[3 * i + k];
  return nv;
}

// Particle node ranges (lo, hi) per axis [n,6].  Returns a status code.
int32_t oracle_aabb(const oracle_config* cfg, int32_t n, const int32_t* shape_type, const double* shape_param,
                    const int32_t* face_offset, const double* planes, const double* young,
                    const double* poisson, const double* pos, const double* quat, int32_t* lo_hi) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return st;
  for (int p = 0; p < n; ++p)
    for (int k = 0; k < 3; ++k) {
      lo_hi[6 * p + k] = pb.lo[3 * p + k];
      lo_hi[6 * p + 3 + k] = pb.hi[3 * p + k];
    }
  return OR_OK;
}

// Per particle [n,3]: the centroid offset by which a polytope's body origin
// was moved (zero for spheres, cuboids and polytopes given about their
// centroid).  Returns a status code.
int32_t oracle_polytope_shift(const oracle_config* cfg, int32_t n, const int32_t* shape_type,
                              const double* shape_param, const int32_t* face_offset, const double* planes,
                              const double* young, const double* poisson, const double* pos,
                              const double* quat, double* shift) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return st;
  std::copy(pb.shift.begin(), pb.shift.end(), shift);
  return OR_OK;
}

// Row of contact (i, j) in a history table sorted by (i, j), or -1.
static int64_t hist_find(int64_t n_hist, const int32_t* hist_ij, int i, int j) {
  int64_t a = 0, b = n_hist;
  while (a < b) {
    const int64_t m = (a + b) / 2;
    const bool less = hist_ij[2 * m] < i || (hist_ij[2 * m] == i && hist_ij[2 * m + 1] < j);
    if (less) a = m + 1; else b = m;
  }
  return (a < n_hist && hist_ij[2 * a] == i && hist_ij[2 * a + 1] == j) ? a : -1;
}

// Full contact evaluation.  Returns the number of candidate pairs P (>= 0;
// only the first max_pairs rows are written when P > max_pairs) or a negative
// status code.  Per pair: pair_ij [P,2], pair_shift [P,3], pair_box [P,6]
// (lo, hi), pair_out [P,11] = V, x_c[3], n[3], d, F[3] (force on the
// higher-ID particle j), pair_aux [P,11] = G[3], box cells, ambiguous cells,
// ambiguous normal cells, depth gap (lattice units), E*, and the first-order
// change of V, of the first moments and of G when every signed distance moves
// by band_eps (smoothed indicator; G's also in sharp mode).  force/torque [n,3].
int64_t oracle_contact_step(const oracle_config* cfg, int32_t n, const int32_t* shape_type,
                            const double* shape_param, const int32_t* face_offset, const double* planes,
                            const double* young, const double* poisson, const double* pos,
                            const double* quat, const double* vel, int64_t max_pairs, int32_t* pair_ij,
                            int32_t* pair_shift, int32_t* pair_box, double* pair_out, double* pair_aux,
                            double* force, double* torque, int64_t n_hist, const int32_t* hist_ij,
                            const double* hist_box, int32_t n_threads) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return -st;
  const int64_t P = static_cast<int64_t>(pb.pairs.size());
  std::vector<PairResult<double>> res(P);
  set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    double XB[3];
    image_pos(pb, g, pos, XB);
    const double es = effective_modulus(pb.young[g.i], pb.poisson[g.i], pb.young[g.j], pb.poisson[g.j]);
    ContactLaw law;
    law.c = pb.cfg.damping_c;
    if (pb.cfg.box_mode == 1 && hist_box != nullptr) {   // warm starts of the ongoing contacts
      const int64_t row = hist_find(n_hist, hist_ij, g.i, g.j);
      if (row >= 0) law.warm_box = hist_box + 6 * row;
    }
    res[p] = eval_pair<double>(pb.cfg, pb.shapes[g.i], pb.shapes[g.j], g, pos + 3 * g.i, quat + 4 * g.i, XB,
                               partner_quat(pb, g, quat), vel ? vel + 6 * g.i : nullptr, partner_vel(pb, g, vel), es, law);
  }
  if (force) std::memset(force, 0, sizeof(double) * 3 * n);
  if (torque) std::memset(torque, 0, sizeof(double) * 3 * n);
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    const PairResult<double>& r = res[p];
    if (force && torque)
      for (int k = 0; k < 3; ++k) {
        force[3 * g.i + k] -= r.F[k];
        torque[3 * g.i + k] += r.TA[k];
        if (g.j < n) {   // a wall takes no sum
          force[3 * g.j + k] += r.F[k];
          torque[3 * g.j + k] += r.TB[k];
        }
      }
    if (p >= max_pairs) continue;
    if (pair_ij) { pair_ij[2 * p] = g.i; pair_ij[2 * p + 1] = g.j; }
    if (pair_shift)
      for (int k = 0; k < 3; ++k) pair_shift[3 * p + k] = g.shift[k];
    if (pair_box)
      for (int k = 0; k < 3; ++k) { pair_box[6 * p + k] = g.lo[k]; pair_box[6 * p + 3 + k] = g.hi[k]; }
    if (pair_out) {
      double* o = pair_out + 11 * p;
      o[0] = r.V;
      for (int k = 0; k < 3; ++k) { o[1 + k] = r.xc[k]; o[4 + k] = r.n[k]; o[8 + k] = r.F[k]; }
      o[7] = r.d;
    }
    if (pair_aux) {
      double* a = pair_aux + 11 * p;
      a[0] = r.G[0]; a[1] = r.G[1]; a[2] = r.G[2];
      a[3] = r.box_cells; a[4] = r.n_band; a[5] = r.n_gtie; a[6] = r.d_gap; a[7] = r.estar;
      a[8] = r.v_sens; a[9] = r.m_sens; a[10] = r.g_sens;
    }
  }
  return P;
}

typedef struct {
  double restitution;   // e of Eq. (damping_factor) (contact history)
  double mu_s, mu_k;    // coefficients of static and kinetic friction
  double u_k;           // transition speed of Eq. (contact_force_tangential)
  int32_t history;      // 1: every contact keeps the c of its first step
  int32_t friction;     // 1: tangential force of Eq. (contact_force_tangential)
} oracle_contact_law;

// The contact step with the contact law's extensions: friction, and the
// contact history of Sec. 4.3.3 (a contact keeps the damping factor computed
// from its approach speed at the first step with V > 0; it ends with the
// first step without overlap).  hist_ij [n_hist,2] / hist_c [n_hist] are the
// contacts of the previous step sorted by (i, j); the contacts of this step
// (pairs with V > 0, in pair order) go to hist_ij_out / hist_c_out (up to
// max_hist rows; *n_hist_out receives their count).  pair_c [P] (nullable)
// receives the damping factor each pair used.  With the box pipeline,
// hist_box [n_hist,6] (nullable) holds each contact's corrected box of the
// previous step relative to X_i (lo, hi), the warm start of its box
// correction, and hist_box_out [max_hist,6] (nullable) receives this step's.
// Other arguments and the return value as oracle_contact_step.
int64_t oracle_contact_step_ext(const oracle_config* cfg, const oracle_contact_law* law_in, int32_t n,
                                const int32_t* shape_type, const double* shape_param, const int32_t* face_offset,
                                const double* planes, const double* young, const double* poisson,
                                const double* pos, const double* quat, const double* vel, int64_t max_pairs,
                                int32_t* pair_ij, double* pair_out, double* pair_c, double* force, double* torque,
                                int64_t n_hist, const int32_t* hist_ij, const double* hist_c, const double* hist_box,
                                int64_t max_hist, int32_t* hist_ij_out, double* hist_c_out, double* hist_box_out,
                                int64_t* n_hist_out, int32_t n_threads) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return -st;
  if (law_in->friction && (!(law_in->mu_s > 0.0) || !(law_in->mu_k >= 0.0) || !(law_in->u_k > 0.0)))
    return -OR_EINVAL;
  const int64_t P = static_cast<int64_t>(pb.pairs.size());
  std::vector<PairResult<double>> res(P);
  set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    double XB[3];
    image_pos(pb, g, pos, XB);
    const double es = effective_modulus(pb.young[g.i], pb.poisson[g.i], pb.young[g.j], pb.poisson[g.j]);
    ContactLaw law;
    law.c = pb.cfg.damping_c;
    law.restitution = law_in->restitution;
    law.friction = law_in->friction != 0;
    law.mu_s = law_in->mu_s;
    law.mu_k = law_in->mu_k;
    law.u_k = law_in->u_k;
    if (law_in->history) {   // an ongoing contact keeps its c; a new one takes c from u0
      const int64_t row = hist_find(n_hist, hist_ij, g.i, g.j);
      if (row >= 0) {
        law.c = hist_c[row];
        if (pb.cfg.box_mode == 1 && hist_box != nullptr) law.warm_box = hist_box + 6 * row;
      } else {
        law.new_contact = true;
      }
    }
    res[p] = eval_pair<double>(pb.cfg, pb.shapes[g.i], pb.shapes[g.j], g, pos + 3 * g.i, quat + 4 * g.i, XB,
                               partner_quat(pb, g, quat), vel ? vel + 6 * g.i : nullptr, partner_vel(pb, g, vel), es, law);
  }
  if (force) std::memset(force, 0, sizeof(double) * 3 * n);
  if (torque) std::memset(torque, 0, sizeof(double) * 3 * n);
  int64_t nh = 0;
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    const PairResult<double>& r = res[p];
    if (force && torque)
      for (int k = 0; k < 3; ++k) {
        force[3 * g.i + k] -= r.F[k];
        torque[3 * g.i + k] += r.TA[k];
        if (g.j < n) {   // a wall takes no sum
          force[3 * g.j + k] += r.F[k];
          torque[3 * g.j + k] += r.TB[k];
        }
      }
    if (r.V > 0.0) {
      if (nh < max_hist) {
        hist_ij_out[2 * nh] = g.i;
        hist_ij_out[2 * nh + 1] = g.j;
        hist_c_out[nh] = r.c_used;
        if (hist_box_out != nullptr)
          for (int k = 0; k < 6; ++k)
            hist_box_out[6 * nh + k] = pb.cfg.box_mode == 1 ? r.box[k] - pos[3 * g.i + k % 3] : 0.0;
      }
      ++nh;
    }
    if (p >= max_pairs) continue;
    if (pair_ij) { pair_ij[2 * p] = g.i; pair_ij[2 * p + 1] = g.j; }
    if (pair_out) {
      double* o = pair_out + 11 * p;
      o[0] = r.V;
      for (int k = 0; k < 3; ++k) { o[1 + k] = r.xc[k]; o[4 + k] = r.n[k]; o[8 + k] = r.F[k]; }
      o[7] = r.d;
    }
    if (pair_c) pair_c[p] = r.V > 0.0 ? r.c_used : 0.0;
  }
  *n_hist_out = nh;
  return P;
}

}  // extern "C"

// Gradient of L = sum_p (grad_force_p . F_p + grad_torque_p . T_p) with
// respect to positions [n,3] and raw (unnormalised) quaternions [n,4], by
// forward-mode dual numbers through the same per-pair code as above.  With a
// contact law (nullable), each contact's damping factor c is looked up in the
// table (hist_ij, hist_c) and held fixed: c is a constant of the contact
// (Eq. damping_factor, Sec. 4.3.3); pairs missing from it take c = 0.
static int64_t gradient_impl(const oracle_config* cfg, const oracle_contact_law* law_in, int32_t n,
                             const int32_t* shape_type, const double* shape_param, const int32_t* face_offset,
                             const double* planes, const double* young, const double* poisson,
                             const double* pos, const double* quat, const double* vel, int64_t n_hist,
                             const int32_t* hist_ij, const double* hist_c, const double* grad_force,
                             const double* grad_torque, double* grad_pos, double* grad_quat, int32_t n_threads) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return -st;
  if (pb.cfg.box_mode != 0) return -OR_EINVAL;   // the box pipeline's samples move with the box: no gradient
  const int64_t P = static_cast<int64_t>(pb.pairs.size());
  std::vector<double> pg(static_cast<size_t>(P) * NT, 0.0);
  set_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    double XBd[3];
    image_pos(pb, g, pos, XBd);
    Dual XA[3], qA[4], XB[3], qB[4];
    for (int k = 0; k < 3; ++k) { XA[k] = Dual(pos[3 * g.i + k]); XA[k].g[k] = 1.0; }
    for (int k = 0; k < 4; ++k) { qA[k] = Dual(quat[4 * g.i + k]); qA[k].g[3 + k] = 1.0; }
    for (int k = 0; k < 3; ++k) { XB[k] = Dual(XBd[k]); XB[k].g[7 + k] = 1.0; }
    const double* qj = partner_quat(pb, g, quat);
    for (int k = 0; k < 4; ++k) { qB[k] = Dual(qj[k]); qB[k].g[10 + k] = 1.0; }
    const double es = effective_modulus(pb.young[g.i], pb.poisson[g.i], pb.young[g.j], pb.poisson[g.j]);
    ContactLaw law;
    law.c = pb.cfg.damping_c;
    if (law_in != nullptr) {
      law.friction = law_in->friction != 0;
      law.mu_s = law_in->mu_s;
      law.mu_k = law_in->mu_k;
      law.u_k = law_in->u_k;
      if (law_in->history) {
        const int64_t row = hist_find(n_hist, hist_ij, g.i, g.j);
        law.c = row >= 0 ? hist_c[row] : 0.0;
      }
    }
    PairResult<Dual> r = eval_pair<Dual>(pb.cfg, pb.shapes[g.i], pb.shapes[g.j], g, XA, qA, XB, qB,
                                         vel ? vel + 6 * g.i : nullptr, partner_vel(pb, g, vel), es, law);
    Dual L(0.0);
    for (int k = 0; k < 3; ++k) {
      L = L + grad_force[3 * g.i + k] * (-r.F[k]) + grad_torque[3 * g.i + k] * r.TA[k];
      if (g.j < n) L = L + grad_force[3 * g.j + k] * r.F[k] + grad_torque[3 * g.j + k] * r.TB[k];
    }
    for (int t = 0; t < NT; ++t) pg[static_cast<size_t>(p) * NT + t] = L.g[t];
  }
  std::memset(grad_pos, 0, sizeof(double) * 3 * n);
  std::memset(grad_quat, 0, sizeof(double) * 4 * n);
  for (int64_t p = 0; p < P; ++p) {
    const PairGeom& g = pb.pairs[p];
    const double* t = &pg[static_cast<size_t>(p) * NT];
    for (int k = 0; k < 3; ++k) grad_pos[3 * g.i + k] += t[k];
    for (int k = 0; k < 4; ++k) grad_quat[4 * g.i + k] += t[3 + k];
    if (g.j >= n) continue;   // walls do not move
    for (int k = 0; k < 3; ++k) grad_pos[3 * g.j + k] += t[7 + k];
    for (int k = 0; k < 4; ++k) grad_quat[4 * g.j + k] += t[10 + k];
  }
  return P;
}

extern "C" {

int64_t oracle_gradient(const oracle_config* cfg, int32_t n, const int32_t* shape_type, const double* shape_param,
                        const int32_t* face_offset, const double* planes, const double* young,
                        const double* poisson, const double* pos, const double* quat, const double* vel,
                        const double* grad_force, const double* grad_torque, double* grad_pos,
                        double* grad_quat, int32_t n_threads) {
  return gradient_impl(cfg, nullptr, n, shape_type, shape_param, face_offset, planes, young, poisson, pos, quat,
                       vel, 0, nullptr, nullptr, grad_force, grad_torque, grad_pos, grad_quat, n_threads);
}

// The gradient with the contact law's extensions: friction, and the damping
// factor of each contact from the table (hist_ij [n_hist,2] sorted by (i, j),
// hist_c [n_hist]: the c every contact of the step used), held fixed.
int64_t oracle_gradient_ext(const oracle_config* cfg, const oracle_contact_law* law, int32_t n,
                            const int32_t* shape_type, const double* shape_param, const int32_t* face_offset,
                            const double* planes, const double* young, const double* poisson, const double* pos,
                            const double* quat, const double* vel, int64_t n_hist, const int32_t* hist_ij,
                            const double* hist_c, const double* grad_force, const double* grad_torque,
                            double* grad_pos, double* grad_quat, int32_t n_threads) {
  if (law == nullptr) return -OR_EINVAL;
  if (law->friction && (!(law->mu_s > 0.0) || !(law->mu_k >= 0.0) || !(law->u_k > 0.0))) return -OR_EINVAL;
  return gradient_impl(cfg, law, n, shape_type, shape_param, face_offset, planes, young, poisson, pos, quat, vel,
                       n_hist, hist_ij, hist_c, grad_force, grad_torque, grad_pos, grad_quat, n_threads);
}

// The box pipeline's boxes per candidate pair (cfg.box_mode must be 1):
// rough [P,6] node-index bounds (0 when no node is rough-in), box [P,6] the
// corrected box (physical), flags [P,2] = rough-detection nodes within
// band_eps of the threshold, faces whose two smallest line distances lie
// within 1e-4 dx.  hist_ij [n_hist,2] (sorted by (i, j)) and hist_box
// [n_hist,6] (nullable) are the ongoing contacts and their warm-start boxes
// relative to X_i, as for oracle_contact_step_ext.  Returns P or a negative
// status.
int64_t oracle_box_pipeline(const oracle_config* cfg, int32_t n, const int32_t* shape_type,
                            const double* shape_param, const int32_t* face_offset, const double* planes,
                            const double* young, const double* poisson, const double* pos, const double* quat,
                            int64_t n_hist, const int32_t* hist_ij, const double* hist_box, int64_t max_pairs,
                            int32_t* rough, double* box, double* flags) {
  Problem pb;
  const int st = build_problem(pb, reinterpret_cast<const Config*>(cfg), n, shape_type, shape_param,
                               face_offset, planes, young, poisson, pos, quat);
  if (st != OR_OK) return -st;
  if (pb.cfg.box_mode != 1) return -OR_EINVAL;
  const int64_t P = static_cast<int64_t>(pb.pairs.size());
  for (int64_t p = 0; p < std::min(P, max_pairs); ++p) {
    const PairGeom& g = pb.pairs[p];
    double XB[3], RA[9], RB[9];
    image_pos(pb, g, pos, XB);
    quat_to_rot(quat + 4 * g.i, RA);
    quat_to_rot(partner_quat(pb, g, quat), RB);
    PairResult<double> r;
    for (int k = 0; k < 6; ++k) { r.rough[k] = 0; r.box[k] = 0.0; }
    double lo[3], step[3];
    r.n_face_tie = 0.0;
    const int64_t row = hist_box != nullptr ? hist_find(n_hist, hist_ij, g.i, g.j) : -1;
    box_pipeline(pb.cfg, pb.shapes[g.i], pb.shapes[g.j], g, pos + 3 * g.i, RA, XB, RB, r, lo, step,
                 row >= 0 ? hist_box + 6 * row : nullptr);
    for (int k = 0; k < 6; ++k) {
      rough[6 * p + k] = r.rough[k];
      box[6 * p + k] = r.box[k];
    }
    flags[2 * p] = r.n_rough_band;
    flags[2 * p + 1] = r.n_face_tie;
  }
  return P;
}

}  // extern "C"
