// Host side of libcontact: context, shape preparation, validation, buffer
// allocation, launch sequencing, CUDA-graph replay and error reporting.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/contact.h"
#include "contact_dev.cuh"
#include "line_clip.cuh"

using namespace gbc;

struct contact_ctx {
  contact_config cfg{};
  Params P{};
  Shapes S{};
  Parts D{};
  Lists W{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int grid_narrow = 0;
  int grid_adjoint = 0;
  std::vector<void*> dev_allocs;
  int* err_host = nullptr;        // mapped pinned words: the error mirror and the step tokens (Lists::err_host)
  int host_token = 0;             // the last token contact_step_host gave a step
  bool hzero = false;             // the captured host-buffer graph writes the results in place (no copies)
  bool step_unwaited = false;     // contact_step enqueued a step nobody has waited for through this context
  double* adj_scratch = nullptr;  // adjoint tile partials, pair seeds and pair gradients
  std::string last_error = "no error";
  // graph cache
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[9] = {};
  std::vector<double> shift;   // [N,3]: polytope body origins moved to the centroid by this
  int last_replay = 0;   // 0 instantiated (or no graph), 1 replayed, 2 replayed after an in-place update
  cudaEvent_t ev_narrow[2] = {nullptr, nullptr};
  cudaEvent_t ev_adj[2] = {nullptr, nullptr};
  bool have_backward = false;
  // contact_step_host: device staging buffers and their own graph cache
  double *hs_pos = nullptr, *hs_quat = nullptr, *hs_vel = nullptr, *hs_force = nullptr, *hs_torque = nullptr;
  double* hs_pair_out = nullptr;
  int32_t *hs_pair_ij = nullptr, *hs_npairs = nullptr;
  cudaGraphExec_t hexec = nullptr;
  const void* hkey[7] = {};
  // tape of the last step (for contact_backward)
  bool have_step = false;
  const double* last_vel = nullptr;
};

namespace {

// NVTX range around a public call (host side: a profiler's timeline shows each
// call with the kernels and copies it enqueued; without a tool attached it
// costs a function-pointer call)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

contact_status fail(contact_ctx* c, contact_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

contact_status cuda_fail(contact_ctx* c, cudaError_t e, const char* what) {
  return fail(c, CONTACT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace gbc {
// Slots per cell-list bin: at most n, else twice the bin volume over the
// smallest inscribed-ball volume plus 8 (particles overlap only by their
// contact indentation, so far fewer centres fit in a bin), at least 16, and
// at most max_entries / nbins.  A fuller bin is reported as ECAPACITY.
int bin_capacity(int n, const double binw[3], double rin_min, long long nbins, long long max_entries) {
  const double vmin = 4.0 / 3.0 * 3.14159265358979323846 * rin_min * rin_min * rin_min;
  const double bound = 2.0 * binw[0] * binw[1] * binw[2] / vmin + 8.0;
  long long cap = bound < static_cast<double>(n) ? static_cast<long long>(std::ceil(bound)) : n;
  cap = std::max<long long>(std::min<long long>(cap, n), std::min<long long>(16, n));
  cap = std::min<long long>(cap, std::max<long long>(1, max_entries / std::max<long long>(1, nbins)));
  return static_cast<int>(cap);
}

// contact_bounds_selftest: the index n checked against an array of n entries
__global__ void k_bounds_selftest(int* err, int n) { (void)checked_index(err, n, n, 0); }
}  // namespace gbc

namespace {

template <class T>
cudaError_t dev_alloc(contact_ctx* c, T** p, size_t count) {
  void* ptr = nullptr;
  const cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) {
    c->dev_allocs.push_back(ptr);
    *p = static_cast<T*>(ptr);
  }
  return e;
}

template <class T>
cudaError_t upload(contact_ctx* c, T** p, const std::vector<T>& v) {
  cudaError_t e = dev_alloc(c, p, v.size());
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Vertices of {y : n_i . y <= d_i + delta}: every plane triple solved by
// Cramer's rule (cross products, determinant, then the weighted sum divided
// by the determinant), kept when no half-space is violated by more than
// 1e-9 max(1, |d + delta|).  The AABB node ranges derived from these vertices
// must match an independent CPU evaluation bit for bit, so the formula and
// its operation order are fixed; contraction is off for this file.
std::vector<double> offset_vertices(const double* pl, int F, double delta) {
  std::vector<double> out;
  double dmax = 1.0;
  for (int i = 0; i < F; ++i) dmax = std::max(dmax, std::fabs(pl[4 * i + 3] + delta));
  const double tol = 1e-9 * dmax;
  for (int i = 0; i < F; ++i)
    for (int j = i + 1; j < F; ++j)
      for (int k = j + 1; k < F; ++k) {
        const double* a = pl + 4 * i;
        const double* b = pl + 4 * j;
        const double* c = pl + 4 * k;
        const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
        const double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
        const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        const double det = a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2];
        if (std::fabs(det) < 1e-12) continue;
        const double da = a[3] + delta, db = b[3] + delta, dc = c[3] + delta;
        double v[3];
        for (int t = 0; t < 3; ++t) v[t] = (da * bc[t] + db * ca[t] + dc * ab[t]) / det;
        bool ok = true;
        for (int m = 0; m < F && ok; ++m) {
          const double* e = pl + 4 * m;
          ok = !(e[0] * v[0] + e[1] * v[1] + e[2] * v[2] - (e[3] + delta) > tol);
        }
        if (ok) out.insert(out.end(), v, v + 3);
      }
  return out;
}

// smallest face offset: the radius of a ball about the origin inside the polytope
double rin_poly(const double* pl, int F) {
  double r = DBL_MAX;
  for (int f = 0; f < F; ++f) r = std::min(r, pl[4 * f + 3]);
  return r;
}
constexpr double kCentroidTol = 1e-6;   // |centroid| allowed, relative to rin_poly

// Volume centroid of the polytope {y : n_f . y <= d_f} (origin inside): each
// face's vertices ordered by angle around their mean, fanned from it into
// triangles, and each triangle closed to a tetrahedron with the origin.
// Returns false when a face has fewer than three vertices.
bool polytope_centroid(const double* pl, int F, double c[3]) {
  const std::vector<double> v = offset_vertices(pl, F, 0.0);
  const int nv = static_cast<int>(v.size() / 3);
  double dmax = 1.0;
  for (int f = 0; f < F; ++f) dmax = std::max(dmax, std::fabs(pl[4 * f + 3]));
  const double tol = 1e-9 * dmax;
  double vol = 0.0, acc[3] = {0.0, 0.0, 0.0};
  for (int f = 0; f < F; ++f) {
    const double* e = pl + 4 * f;
    std::vector<int> on;
    for (int i = 0; i < nv; ++i) {
      const double* w = &v[3 * i];
      if (std::fabs(e[0] * w[0] + e[1] * w[1] + e[2] * w[2] - e[3]) <= tol) on.push_back(i);
    }
    if (on.size() < 3) continue;   // a redundant plane touching at an edge or vertex
    double m[3] = {0.0, 0.0, 0.0};
    for (int i : on)
      for (int k = 0; k < 3; ++k) m[k] += v[3 * i + k] / on.size();
    // in-plane basis (a, b) of the face
    double a[3] = {v[3 * on[0]] - m[0], v[3 * on[0] + 1] - m[1], v[3 * on[0] + 2] - m[2]};
    const double na = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(na > 0.0)) continue;
    for (double& x : a) x /= na;
    const double b[3] = {e[1] * a[2] - e[2] * a[1], e[2] * a[0] - e[0] * a[2], e[0] * a[1] - e[1] * a[0]};
    std::vector<std::pair<double, int>> ang;
    for (int i : on) {
      const double r[3] = {v[3 * i] - m[0], v[3 * i + 1] - m[1], v[3 * i + 2] - m[2]};
      ang.push_back({std::atan2(r[0] * b[0] + r[1] * b[1] + r[2] * b[2], r[0] * a[0] + r[1] * a[1] + r[2] * a[2]), i});
    }
    std::sort(ang.begin(), ang.end());
    for (size_t t = 0; t < ang.size(); ++t) {
      const double* p1 = &v[3 * ang[t].second];
      const double* p2 = &v[3 * ang[(t + 1) % ang.size()].second];
      const double cr[3] = {p1[1] * p2[2] - p1[2] * p2[1], p1[2] * p2[0] - p1[0] * p2[2], p1[0] * p2[1] - p1[1] * p2[0]};
      const double tv = std::fabs(m[0] * cr[0] + m[1] * cr[1] + m[2] * cr[2]) / 6.0;   // tetrahedron (0, m, p1, p2)
      vol += tv;
      for (int k = 0; k < 3; ++k) acc[k] += tv * (m[k] + p1[k] + p2[k]) / 4.0;
    }
  }
  if (!(vol > 0.0)) return false;
  for (int k = 0; k < 3; ++k) c[k] = acc[k] / vol;
  return true;
}

// Bounded iff no direction u has n_i . u <= 0 for every face; candidate
// extreme rays of the recession cone are +-(n_i x n_j).
bool bounded(const double* pl, int F) {
  for (int i = 0; i < F; ++i)
    for (int j = i + 1; j < F; ++j) {
      const double* a = pl + 4 * i;
      const double* b = pl + 4 * j;
      const double u[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      const double nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      if (nu < 1e-12) continue;
      for (int sg = -1; sg <= 1; sg += 2) {
        bool ray = true;
        for (int m = 0; m < F && ray; ++m) {
          const double* e = pl + 4 * m;
          ray = !(sg * (e[0] * u[0] + e[1] * u[1] + e[2] * u[2]) / nu > 1e-12);
        }
        if (ray) return false;
      }
    }
  return true;
}

contact_status check_sticky(contact_ctx* c) {
  const int e = *reinterpret_cast<volatile int*>(c->err_host);
  if (e != 0) {
    return fail(c, static_cast<contact_status>(e),
                e == CONTACT_ECAPACITY ? "device: capacity exceeded (pairs, neighbours or tiles)"
                : e == CONTACT_EBOUNDS ? "device: an index read from a device list is out of range (checked build)"
                                       : "device: invalid pose (position outside [0, L), zero or non-finite quaternion)");
  }
  return CONTACT_OK;
}

// `capturing`: the stream is being captured (ours or the caller's), so the
// timing events must become event-record nodes of the graph.
// publish: the step reads the host's token and publishes it when done (a
// host-buffer step whose results are written in place)
void enqueue_step(contact_ctx* c, bool capturing, const double* pos, const double* quat, const double* vel,
                  int32_t* pair_ij, double* pair_out, int32_t* n_pairs, double* force, double* torque,
                  bool publish = false) {
  const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  Lists W = c->W;
  W.publish = publish ? 1 : 0;
  // bin counts are zero: contact_init clears them, every step's last kernel clears them again
  launch_pose(c->P, c->S, c->D, W, pos, quat, c->stream);
  launch_broad(c->P, c->D, W, c->stream);
  launch_plan(c->P, c->S, c->D, W, pair_ij, n_pairs, pair_out, c->stream);
  if (c->cfg.narrow_events) cudaEventRecordWithFlags(c->ev_narrow[0], c->stream, ev_flags);
  launch_narrow(c->P, c->S, c->D, W, vel, pair_out, c->grid_narrow, c->stream);
  // narrow_events = K > 1: K - 1 more launches of the node sweep, each
  // recomputing the same outputs from the same tiles (the timing's average)
  for (int k = 1; k < c->cfg.narrow_events; ++k)
    launch_narrow(c->P, c->S, c->D, W, vel, pair_out, c->grid_narrow, c->stream);
  if (c->cfg.narrow_events) cudaEventRecordWithFlags(c->ev_narrow[1], c->stream, ev_flags);
  if (c->P.box_mode == 0) launch_force(c->P, c->S, c->D, W, vel, pair_out, c->stream);
  launch_particle_sum(c->P, c->D, W, force, torque, c->stream);
}

}  // namespace

extern "C" {

void contact_config_default(contact_config* cfg, int32_t n_particles, const int32_t n_cells[3], double dx) {
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n_particles = n_particles;
  for (int k = 0; k < 3; ++k) cfg->n_cells[k] = n_cells[k];
  cfg->dx = dx;
  cfg->indicator = CONTACT_INDICATOR_SHARP;
  cfg->smooth_width = 1.0;
  cfg->inflate = 0.0;
  cfg->damping_c = 0.0;
  cfg->precision = CONTACT_PRECISION_FP32_TILE;
  cfg->max_pairs = std::max(64, 16 * n_particles);
  cfg->max_neighbors = 64;
  cfg->max_tiles = 0;
  cfg->use_graph = 1;
  cfg->narrow_events = 0;
  cfg->history = 0;
  cfg->friction = 0;
  cfg->restitution = 1.0;
  cfg->mu_s = 0.0;
  cfg->mu_k = 0.0;
  cfg->u_k = 1.0;
  cfg->n_walls = 0;
  cfg->reserved = 0;
  cfg->walls = nullptr;
  cfg->wall_young = nullptr;
  cfg->wall_poisson = nullptr;
  cfg->box_mode = 0;
  cfg->contact_resolution = 8;
}

contact_status contact_polytope_centroid(const double* planes, int32_t n_faces, double* centroid) {
  if (planes == nullptr || centroid == nullptr || n_faces < 4) return CONTACT_EINVAL;
  for (int f = 0; f < n_faces; ++f) {
    const double* e = planes + 4 * f;
    const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (!(std::fabs(nn - 1.0) <= 1e-9) || !(e[3] > 0.0) || !std::isfinite(e[3])) return CONTACT_EINVAL;
  }
  if (!bounded(planes, n_faces)) return CONTACT_EINVAL;
  return polytope_centroid(planes, n_faces, centroid) ? CONTACT_OK : CONTACT_EINVAL;
}

double contact_damping_factor(double e, double u0) {
  if (!(u0 > 0.0)) return 0.0;
  return 1.5 * (1.0 - e) * (11.0 - e) / ((1.0 + 9.0 * e) * u0);
}

contact_status contact_polytope_shift(const contact_ctx* ctx, double* shift) {
  if (ctx == nullptr || shift == nullptr) return CONTACT_EINVAL;
  std::copy(ctx->shift.begin(), ctx->shift.end(), shift);
  return CONTACT_OK;
}

contact_status contact_init(const contact_config* cfg, const int32_t* shape_type, const double* shape_param,
                            const int32_t* face_offset, const double* planes, const double* young,
                            const double* poisson, void* stream, contact_ctx** out) {
  if (out == nullptr) return CONTACT_EINVAL;
  *out = nullptr;
  if (cfg == nullptr || shape_type == nullptr || shape_param == nullptr || face_offset == nullptr ||
      young == nullptr || poisson == nullptr)
    return CONTACT_EINVAL;
  const contact_config& C = *cfg;
  const int n = C.n_particles;
  if (n < 1 || !(C.dx > 0.0) || !std::isfinite(C.dx) || C.max_pairs < 1) return CONTACT_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (C.n_cells[k] < 1) return CONTACT_EINVAL;
  if (C.indicator != 0 && C.indicator != 1) return CONTACT_EINVAL;
  if (C.precision != 0 && C.precision != 1) return CONTACT_EINVAL;
  if (!(C.smooth_width > 0.0) || !(C.inflate >= 0.0) || !(C.damping_c >= 0.0)) return CONTACT_EINVAL;
  if (C.max_neighbors < 0 || C.max_neighbors > 512 || C.max_tiles < 0) return CONTACT_EINVAL;
  if (C.history != 0 && C.history != 1) return CONTACT_EINVAL;
  if (C.history && !(C.restitution >= 0.0 && C.restitution <= 1.0)) return CONTACT_EINVAL;
  if (C.friction != 0 && C.friction != 1) return CONTACT_EINVAL;
  if (C.friction && (!(C.mu_s > 0.0) || !(C.mu_k >= 0.0) || !(C.u_k > 0.0) || !std::isfinite(C.mu_s) ||
                     !std::isfinite(C.mu_k) || !std::isfinite(C.u_k)))
    return CONTACT_EINVAL;
  if (C.box_mode != 0 && C.box_mode != 1) return CONTACT_EINVAL;
  // repeated node sweeps (timing) recompute the same outputs only without the
  // box pipeline, whose kernel keeps the contact history and a work queue
  if (C.narrow_events < 0 || C.narrow_events > 64 || (C.narrow_events > 1 && C.box_mode != 0)) return CONTACT_EINVAL;
  if (C.box_mode == 1 && (C.contact_resolution < 1 || C.contact_resolution > 64)) return CONTACT_EINVAL;
  const int nw = C.n_walls;
  if (nw < 0 || nw > CONTACT_MAX_WALLS) return CONTACT_EINVAL;
  if (nw > 0 && (C.walls == nullptr || C.wall_young == nullptr || C.wall_poisson == nullptr)) return CONTACT_EINVAL;
  for (int w = 0; w < nw; ++w) {
    const double* e = C.walls + 4 * w;
    const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (!(std::fabs(nn - 1.0) <= 1e-9) || !std::isfinite(e[3])) return CONTACT_EINVAL;
    if (!(C.wall_young[w] > 0.0) || !(C.wall_poisson[w] >= 0.0) || !(C.wall_poisson[w] < 1.0))
      return CONTACT_EINVAL;
  }
  const int max_nbr = C.max_neighbors > 0 ? C.max_neighbors : 64;
  const long long max_tiles_ll = C.max_tiles > 0 ? C.max_tiles : 8LL * C.max_pairs;
  if (max_tiles_ll > (1LL << 30)) return CONTACT_EINVAL;

  // offset of the node ranges: inflation plus, in smoothed mode, half the band;
  // the box pipeline widens them to its rough-detection threshold sqrt(0.75) dx
  double band = (C.indicator == 1) ? (0.5 * C.smooth_width) * C.dx : 0.0;
  if (C.box_mode == 1) band = std::max(band, std::sqrt(0.75) * C.dx);
  const double delta = C.inflate + band;
  std::vector<int> type(n), kind(n), vert_off(n + 1, 0);
  std::vector<double> param(3 * static_cast<size_t>(n)), verts, ext(3 * static_cast<size_t>(n), 0.0);
  std::vector<float> size_l(3 * static_cast<size_t>(n));
  // nominal FP32 lane-ops of one signed-distance test (roofline accounting):
  // sphere 7, cuboid 15, polytope with F faces 4F
  std::vector<int> nomops(n);
  const int nfaces = face_offset[n];
  if (face_offset[0] != 0 || nfaces < 0 || (nfaces > 0 && planes == nullptr)) return CONTACT_EINVAL;
  // the library's own copy of the planes: polytopes off their centroid are shifted in it
  std::vector<double> pl_in(planes ? planes : nullptr, planes ? planes + 4 * static_cast<size_t>(nfaces) : nullptr);
  std::vector<double> shift(3 * static_cast<size_t>(n), 0.0);
  double rmax = 0.0;
  double rin_min = DBL_MAX;   // smallest inscribed-ball radius (bounds how many particles one bin holds)
  for (int p = 0; p < n; ++p) {
    type[p] = shape_type[p];
    for (int k = 0; k < 3; ++k) param[3 * p + k] = shape_param[3 * p + k];
    if (!(young[p] > 0.0) || !(poisson[p] >= 0.0) || !(poisson[p] < 1.0)) return CONTACT_EINVAL;
    const int f0 = face_offset[p], f1 = face_offset[p + 1];
    if (f1 < f0) return CONTACT_EINVAL;
    double circ = 0.0;
    if (type[p] == CONTACT_SHAPE_SPHERE) {
      if (!(param[3 * p] > 0.0) || f1 != f0) return CONTACT_EINVAL;
      circ = param[3 * p] + delta;
      rin_min = std::min(rin_min, param[3 * p]);
      ext[3 * p] = param[3 * p] + delta;
      kind[p] = KIND_SPHERE;
      nomops[p] = 7;
      size_l[3 * p] = static_cast<float>((param[3 * p] + C.inflate) / C.dx);
    } else if (type[p] == CONTACT_SHAPE_CUBOID) {
      if (f1 != f0) return CONTACT_EINVAL;
      double e2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        if (!(param[3 * p + k] > 0.0)) return CONTACT_EINVAL;
        e2 += (param[3 * p + k] + delta) * (param[3 * p + k] + delta);
        ext[3 * p + k] = param[3 * p + k] + delta;
        size_l[3 * p + k] = static_cast<float>((param[3 * p + k] + C.inflate) / C.dx);
      }
      circ = std::sqrt(e2);
      rin_min = std::min(rin_min, std::min(param[3 * p], std::min(param[3 * p + 1], param[3 * p + 2])));
      kind[p] = (param[3 * p] == param[3 * p + 1] && param[3 * p] == param[3 * p + 2]) ? KIND_CUBE : KIND_CUBOID;
      nomops[p] = 15;
    } else if (type[p] == CONTACT_SHAPE_POLYTOPE) {
      const int F = f1 - f0;
      if (F < 4 || F > kMaxFaces) return CONTACT_EINVAL;
      double* pl = pl_in.data() + 4 * f0;
      for (int f = 0; f < F; ++f) {
        const double* e = pl + 4 * f;
        const double nn = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        if (!(std::fabs(nn - 1.0) <= 1e-9) || !(e[3] > 0.0) || !std::isfinite(e[3])) return CONTACT_EINVAL;
      }
      if (!bounded(pl, F)) return CONTACT_EINVAL;
      // poses refer to the centre of mass (the torque reference, Sec. 2.2): an
      // origin off the volume centroid is moved there, d_f -= n_f . c
      double cm[3];
      if (!polytope_centroid(pl, F, cm)) return CONTACT_EINVAL;
      if (std::sqrt(cm[0] * cm[0] + cm[1] * cm[1] + cm[2] * cm[2]) > kCentroidTol * rin_poly(pl, F)) {
        for (int f = 0; f < F; ++f) {
          double* e = pl + 4 * f;
          e[3] -= e[0] * cm[0] + e[1] * cm[1] + e[2] * cm[2];
          if (!(e[3] > 0.0)) return CONTACT_EINVAL;
        }
        for (int k = 0; k < 3; ++k) shift[3 * p + k] = cm[k];
      }
      rin_min = std::min(rin_min, rin_poly(pl, F));   // unit normals, origin inside: the ball of radius min d fits
      std::vector<double> v = offset_vertices(pl, F, delta);
      if (v.size() < 12) return CONTACT_EINVAL;
      for (size_t t = 0; t < v.size(); t += 3)
        circ = std::max(circ, std::sqrt(v[t] * v[t] + v[t + 1] * v[t + 1] + v[t + 2] * v[t + 2]));
      // the node sweep's pair test bounds a polytope by balls (lattice units,
      // rounded up): its region {phi <= 0} (offset inflate) in size slot 0, its
      // region {phi < w/2 + the clip margin} in slot 1
      const double tcut = (0.5 * C.smooth_width + static_cast<double>(kClipMargin)) * C.dx;
      for (int s = 0; s < 2; ++s) {
        const std::vector<double> vs = offset_vertices(pl, F, C.inflate + (s == 0 ? 0.0 : tcut));
        double r = 0.0;
        for (size_t t = 0; t < vs.size(); t += 3)
          r = std::max(r, std::sqrt(vs[t] * vs[t] + vs[t + 1] * vs[t + 1] + vs[t + 2] * vs[t + 2]));
        size_l[3 * p + s] = std::nextafter(static_cast<float>(r / C.dx), 3.0e38f);
      }
      verts.insert(verts.end(), v.begin(), v.end());
      kind[p] = KIND_POLY;
      nomops[p] = 4 * F;
    } else {
      return CONTACT_EINVAL;
    }
    vert_off[p + 1] = static_cast<int>(verts.size() / 3);
    rmax = std::max(rmax, circ);
  }
  // walls: rows n .. n + nw - 1 of the shape tables, one world-frame plane each
  for (int w = 0; w < nw; ++w) {
    type.push_back(CONTACT_SHAPE_POLYTOPE);
    kind.push_back(KIND_WALL);
    for (int k = 0; k < 3; ++k) {
      param.push_back(0.0);
      ext.push_back(0.0);
      size_l.push_back(0.f);
    }
    nomops.push_back(4);   // one plane
    vert_off.push_back(vert_off.back());
  }
  double L[3];
  for (int k = 0; k < 3; ++k) {
    L[k] = C.n_cells[k] * C.dx;
    if (!(L[k] > 4.0 * rmax + 2.0 * C.dx)) return CONTACT_EDOMAIN;
  }
  // a pair box spans below 2^16 nodes along every axis (the node sweep packs node offsets in 16 bits)
  if (!(2.0 * rmax / C.dx + 4.0 < 65535.0)) return CONTACT_EDOMAIN;

  contact_ctx* c = new contact_ctx();
  c->cfg = C;
  c->shift = std::move(shift);
  c->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&c->device);
  Params& P = c->P;
  P.n = n;
  for (int k = 0; k < 3; ++k) {
    P.ncell[k] = C.n_cells[k];
    P.L[k] = L[k];
    // bins at least 2 R_max + 2 dx wide: intersecting AABBs sit in adjacent bins
    int nb = static_cast<int>(std::floor(L[k] / (2.0 * rmax + 2.0 * C.dx)));
    if (nb < 3) nb = 1;
    nb = std::min(nb, 256);
    P.nbin[k] = nb;
    P.binw[k] = L[k] / nb;
    P.inv_binw_f[k] = static_cast<float>(nb / L[k]);
  }
  P.bin_cap = bin_capacity(n, P.binw, rin_min, static_cast<long long>(P.nbin[0]) * P.nbin[1] * P.nbin[2], 1LL << 26);
  P.dx = C.dx;
  P.inv_dx = 1.0 / C.dx;
  {
    int ex = 0;
    P.dx_pow2 = std::frexp(C.dx, &ex) == 0.5 ? 1 : 0;
  }
  P.delta = delta;
  P.inflate = C.inflate;
  P.wdx = C.smooth_width * C.dx;
  P.dx3 = C.dx * C.dx * C.dx;
  P.gscale = 0.5 * C.dx * C.dx * 6.0 / (P.wdx / C.dx);
  P.g_min2 = 1e-24 * C.dx * C.dx * C.dx * C.dx;
  P.smooth = C.indicator;
  P.precision = C.precision;
  // node-sweep variant from the particle kinds; walls need a variant with the wall evaluator
  P.kind_set = std::all_of(kind.begin(), kind.begin() + n, [](int k) { return k == KIND_CUBE; }) ? 2
               : std::all_of(kind.begin(), kind.begin() + n,
                             [](int k) { return k == KIND_SPHERE || k == KIND_CUBOID || k == KIND_CUBE; }) ? 1 : 0;
  if (nw > 0 && P.kind_set == 2) P.kind_set = 1;
  P.nwall = nw;
  P.box_mode = C.box_mode;
  P.box_res = C.box_mode == 1 ? C.contact_resolution : 0;
  P.damping_c = C.damping_c;
  P.history = C.history;
  P.friction = C.friction;
  // Eq. (damping_factor) as c = K / u0 with K = 1.5 (1 - e)(11 - e) / (1 + 9 e)
  P.damp_K = C.history ? 1.5 * (1.0 - C.restitution) * (11.0 - C.restitution) / (1.0 + 9.0 * C.restitution) : 0.0;
  P.mu_k = C.mu_k;
  P.mu_s_star = C.friction ? C.mu_s * (1.0 - 0.09 * std::pow(C.mu_k / C.mu_s, 4)) : 0.0;
  P.inv_u_k = C.friction ? 1.0 / C.u_k : 0.0;
  P.max_pairs = C.max_pairs;
  P.max_nbr = max_nbr;
  P.max_tiles = static_cast<int>(max_tiles_ll);
  P.inflate_l = static_cast<float>(C.inflate / C.dx);
  P.inv_w = static_cast<float>(1.0 / C.smooth_width);
  P.neg6_over_w = static_cast<float>(-6.0 / C.smooth_width);
  P.wdx_l = static_cast<float>(C.smooth_width);

  cudaError_t e = cudaSuccess;
  std::vector<double> pl_vec(std::move(pl_in));
  std::vector<int> foff(face_offset, face_offset + n + 1);
  std::vector<double> yv(young, young + n), pv(poisson, poisson + n), cv(n);
  for (int p = 0; p < n; ++p) cv[p] = (1.0 - poisson[p] * poisson[p]) / young[p];
  std::vector<double> wall_tab(C.walls ? C.walls : nullptr, C.walls ? C.walls + 4 * static_cast<size_t>(nw) : nullptr);
  for (int w = 0; w < nw; ++w) {
    pl_vec.insert(pl_vec.end(), C.walls + 4 * w, C.walls + 4 * w + 4);
    foff.push_back(foff.back() + 1);
    yv.push_back(C.wall_young[w]);
    pv.push_back(C.wall_poisson[w]);
    cv.push_back((1.0 - C.wall_poisson[w] * C.wall_poisson[w]) / C.wall_young[w]);
  }
  const int nrows = n + nw;             // particle rows, then wall rows
  const int nplanes = nfaces + nw;      // particle faces, then one plane per wall
  int *d_type, *d_foff, *d_voff, *d_kind;
  double *d_param, *d_planes, *d_verts, *d_young, *d_pois;
  float* d_size;
  int* d_nomops;
  double* d_compl;
#define GBC_TRY(x)                                              \
  do {                                                          \
    e = (x);                                                    \
    if (e != cudaSuccess) {                                     \
      contact_destroy(c);                                       \
      return e == cudaErrorMemoryAllocation ? CONTACT_ENOMEM : CONTACT_ECUDA; \
    }                                                           \
  } while (0)
  GBC_TRY(upload(c, &d_type, type));
  GBC_TRY(upload(c, &d_kind, kind));
  GBC_TRY(upload(c, &d_param, param));
  GBC_TRY(upload(c, &d_foff, foff));
  GBC_TRY(upload(c, &d_planes, pl_vec));
  GBC_TRY(upload(c, &d_voff, vert_off));
  GBC_TRY(upload(c, &d_verts, verts));
  GBC_TRY(upload(c, &d_young, yv));
  GBC_TRY(upload(c, &d_pois, pv));
  GBC_TRY(upload(c, &d_size, size_l));
  GBC_TRY(upload(c, &d_nomops, nomops));
  GBC_TRY(upload(c, &d_compl, cv));
  std::vector<float> verts32(verts.begin(), verts.end()), off32(static_cast<size_t>(std::max(nplanes, 1)), 0.f);
  for (int f = 0; f < nplanes; ++f) off32[f] = static_cast<float>((pl_vec[4 * f + 3] + C.inflate) / C.dx);
  double* d_ext;
  float *d_verts32, *d_off32;
  GBC_TRY(upload(c, &d_ext, ext));
  GBC_TRY(upload(c, &d_verts32, verts32));
  GBC_TRY(upload(c, &d_off32, off32));
  std::vector<int> poly_ids;
  for (int p = 0; p < n; ++p)
    if (type[p] == CONTACT_SHAPE_POLYTOPE) poly_ids.push_back(p);
  if (poly_ids.empty()) poly_ids.push_back(0);   // (a non-empty allocation; npoly stays 0)
  P.npoly = static_cast<int>(std::count(type.begin(), type.begin() + n, static_cast<int>(CONTACT_SHAPE_POLYTOPE)));
  int* d_poly;
  GBC_TRY(upload(c, &d_poly, poly_ids));
  c->S = Shapes{d_type, d_param, d_foff, d_planes, d_voff, d_verts, d_young, d_pois, d_size, d_nomops, d_compl,
                d_ext, d_verts32, d_off32, d_poly};

  Parts& D = c->D;
  GBC_TRY(dev_alloc(c, &D.X, 3 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.qhat, 4 * static_cast<size_t>(n)));
  GBC_TRY(dev_alloc(c, &D.R, 9 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.lohi, 6 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.bin, static_cast<size_t>(n)));
  GBC_TRY(dev_alloc(c, &D.Rt, 9 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.wplane, static_cast<size_t>(std::max(nplanes, 1))));
  GBC_TRY(dev_alloc(c, &D.Xf, 3 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.kX, 3 * static_cast<size_t>(nrows)));
  GBC_TRY(dev_alloc(c, &D.fX, 3 * static_cast<size_t>(nrows)));
  {
    double* rest = nullptr;
    GBC_TRY(dev_alloc(c, &rest, 8));
    GBC_TRY(cudaMemset(rest, 0, 8 * sizeof(double)));
    D.rest6 = rest;
  }
  if (nw > 0) {   // wall rows: at the origin, identity rotation, Rt row 0 = m, world plane
    std::vector<double> X0(3 * static_cast<size_t>(nw), 0.0), R0(9 * static_cast<size_t>(nw), 0.0);
    std::vector<float> Rt0(9 * static_cast<size_t>(nw), 0.f), f0(3 * static_cast<size_t>(nw), 0.f);
    std::vector<int> k0(3 * static_cast<size_t>(nw), 0), lohi0(6 * static_cast<size_t>(nw), 0);
    std::vector<float4> wp(nw);
    for (int w = 0; w < nw; ++w) {
      R0[9 * w] = R0[9 * w + 4] = R0[9 * w + 8] = 1.0;
      for (int k = 0; k < 3; ++k) Rt0[9 * w + k] = static_cast<float>(C.walls[4 * w + k]);
      wp[w] = make_float4(static_cast<float>(C.walls[4 * w]), static_cast<float>(C.walls[4 * w + 1]),
                          static_cast<float>(C.walls[4 * w + 2]), off32[nfaces + w]);
    }
    const size_t o3 = 3 * static_cast<size_t>(n), o9 = 9 * static_cast<size_t>(n);
    GBC_TRY(cudaMemcpy(D.X + o3, X0.data(), sizeof(double) * X0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.R + o9, R0.data(), sizeof(double) * R0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.Rt + o9, Rt0.data(), sizeof(float) * Rt0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.Xf + o3, f0.data(), sizeof(float) * f0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.fX + o3, f0.data(), sizeof(float) * f0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.kX + o3, k0.data(), sizeof(int) * k0.size(), cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.lohi + 6 * static_cast<size_t>(n), lohi0.data(), sizeof(int) * lohi0.size(),
                       cudaMemcpyHostToDevice));
    GBC_TRY(cudaMemcpy(D.wplane + nfaces, wp.data(), sizeof(float4) * wp.size(), cudaMemcpyHostToDevice));
    double* d_wall = nullptr;
    GBC_TRY(upload(c, &d_wall, wall_tab));
    P.wall = d_wall;
  }

  Lists& W = c->W;
  const size_t nbins = static_cast<size_t>(P.nbin[0]) * P.nbin[1] * P.nbin[2];
  const size_t mp = static_cast<size_t>(C.max_pairs), mt = static_cast<size_t>(P.max_tiles);
  GBC_TRY(dev_alloc(c, &W.bin_count, nbins));
  GBC_TRY(dev_alloc(c, &W.bin_items, nbins * static_cast<size_t>(P.bin_cap)));
  GBC_TRY(dev_alloc(c, &W.up_count, static_cast<size_t>(n)));
  GBC_TRY(dev_alloc(c, &W.up_list, static_cast<size_t>(n) * max_nbr));
  GBC_TRY(dev_alloc(c, &W.dn_count, static_cast<size_t>(n)));
  GBC_TRY(dev_alloc(c, &W.dn_list, static_cast<size_t>(n) * max_nbr));
  GBC_TRY(dev_alloc(c, &W.dn_pair, static_cast<size_t>(n) * max_nbr));
  GBC_TRY(dev_alloc(c, &W.row_off, static_cast<size_t>(n) + 1));
  GBC_TRY(dev_alloc(c, &W.grp_sum, static_cast<size_t>((n + kRowGroup - 1) / kRowGroup)));
  // contact history: two buffers (read the previous step's, write this step's)
  if (C.history) {
    GBC_TRY(dev_alloc(c, &W.hist_j, 2 * static_cast<size_t>(n) * max_nbr));
    GBC_TRY(dev_alloc(c, &W.hist_c, 2 * static_cast<size_t>(n) * max_nbr));
    GBC_TRY(dev_alloc(c, &W.hist_n, 2 * static_cast<size_t>(n)));
    // the box pipeline's warm start: each contact's corrected box relative to X_i
    if (C.box_mode == 1) GBC_TRY(dev_alloc(c, &W.hist_box, 2 * static_cast<size_t>(n) * max_nbr * 6));
  }
  GBC_TRY(dev_alloc(c, &W.pairs, mp));
  GBC_TRY(dev_alloc(c, &W.olist, mp));
  GBC_TRY(dev_alloc(c, &W.oflag, mp));
  GBC_TRY(dev_alloc(c, &W.tile_pair, mt));
  GBC_TRY(dev_alloc(c, &W.tiles, mt));
  GBC_TRY(dev_alloc(c, &W.partial, mt * kPartialFloats));
  GBC_TRY(dev_alloc(c, &W.pdone, mp));
  GBC_TRY(dev_alloc(c, &W.tape, mp * kTapeDoubles));
  GBC_TRY(dev_alloc(c, &W.ft, mp * kFtDoubles));
  GBC_TRY(dev_alloc(c, &W.counters, 16));
  GBC_TRY(dev_alloc(c, &W.u64, 4));
  GBC_TRY(dev_alloc(c, &W.err, 1));
  GBC_TRY(dev_alloc(c, &c->adj_scratch, adjoint_scratch_doubles(C.max_pairs, P.max_tiles)));
  W.kind = d_kind;
  GBC_TRY(cudaMemset(W.counters, 0, 16 * sizeof(int)));
  GBC_TRY(cudaMemset(W.u64, 0, 4 * sizeof(unsigned long long)));
  GBC_TRY(cudaMemset(W.err, 0, sizeof(int)));
  GBC_TRY(cudaMemset(W.up_count, 0, sizeof(int) * n));
  GBC_TRY(cudaMemset(W.bin_count, 0, sizeof(int) * nbins));
  GBC_TRY(cudaMemset(W.dn_count, 0, sizeof(int) * n));
  if (C.history) GBC_TRY(cudaMemset(W.hist_n, 0, sizeof(int) * 2 * n));
  GBC_TRY(cudaEventCreate(&c->ev_narrow[0]));
  GBC_TRY(cudaEventCreate(&c->ev_narrow[1]));
  GBC_TRY(cudaEventCreate(&c->ev_adj[0]));
  GBC_TRY(cudaEventCreate(&c->ev_adj[1]));
  GBC_TRY(cudaHostAlloc(reinterpret_cast<void**>(&c->err_host), 3 * sizeof(int), cudaHostAllocMapped));
  c->err_host[0] = c->err_host[1] = c->err_host[2] = 0;
  int* err_dev_view = nullptr;
  GBC_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&err_dev_view), c->err_host, 0));
  W.err_host = err_dev_view;
#undef GBC_TRY
  c->grid_narrow = narrow_grid(P);
  c->grid_adjoint = c->grid_narrow;
  *out = c;
  return CONTACT_OK;
}

contact_status contact_set_stream(contact_ctx* c, void* stream) {
  if (c == nullptr) return CONTACT_EINVAL;
  c->stream = static_cast<cudaStream_t>(stream);
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return CONTACT_OK;
}

contact_status contact_step(contact_ctx* c, const double* pos, const double* quat, const double* vel,
                            int32_t* pair_ij, double* pair_out, int32_t* n_pairs, double* force,
                            double* torque) {
  const NvtxRange range("contact_step");
  if (c == nullptr) return CONTACT_EINVAL;
  if (pos == nullptr || quat == nullptr || pair_ij == nullptr || pair_out == nullptr || n_pairs == nullptr ||
      force == nullptr || torque == nullptr)
    return fail(c, CONTACT_EINVAL, "contact_step: null buffer");
  const contact_status sticky = check_sticky(c);
  if (sticky != CONTACT_OK) return sticky;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cap);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamIsCapturing");
  const void* key[9] = {pos, quat, vel, pair_ij, pair_out, n_pairs, force, torque, c->stream};
  c->last_replay = 0;
  if (cap == cudaStreamCaptureStatusNone && c->cfg.use_graph && c->stream != nullptr) {
    if (c->gexec == nullptr || std::memcmp(key, c->gkey, sizeof(key)) != 0) {
      // capture the step; new buffers on the same stream only change kernel
      // arguments, so the executable graph is updated in place (no
      // re-instantiation); otherwise it is instantiated anew
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
      enqueue_step(c, true, pos, quat, vel, pair_ij, pair_out, n_pairs, force, torque);
      e = cudaStreamEndCapture(c->stream, &g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      bool updated = false;
      if (c->gexec != nullptr && c->gkey[8] == c->stream) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(c->gexec, g, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();   // clear the update failure; instantiate below
      }
      if (!updated) {
        if (c->gexec) {
          cudaGraphExecDestroy(c->gexec);
          c->gexec = nullptr;
        }
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (e != cudaSuccess) {
          cudaGraphDestroy(g);
          c->gexec = nullptr;
          return cuda_fail(c, e, "cudaGraphInstantiate");
        }
      } else {
        c->last_replay = 2;
      }
      cudaGraphDestroy(g);
      std::memcpy(c->gkey, key, sizeof(key));
    } else {
      c->last_replay = 1;
    }
    e = cudaGraphLaunch(c->gexec, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  } else {
    enqueue_step(c, cap != cudaStreamCaptureStatusNone, pos, quat, vel, pair_ij, pair_out, n_pairs, force,
                 torque);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  }
  c->step_unwaited = true;
  c->have_step = true;
  c->last_vel = vel;
  return CONTACT_OK;
}

contact_status contact_check(contact_ctx* c) {
  if (c == nullptr) return CONTACT_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  int err = 0;
  e = cudaMemcpy(&err, c->W.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
  *c->err_host = err;
  return check_sticky(c);
}

contact_status contact_bounds_selftest(contact_ctx* c) {
  if (c == nullptr) return CONTACT_EINVAL;
  k_bounds_selftest<<<1, 1, 0, c->stream>>>(c->W.err, 1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "bounds self-test launch");
  return contact_check(c);
}

void contact_clear_error(contact_ctx* c) {
  if (c == nullptr) return;
  cudaStreamSynchronize(c->stream);
  cudaMemset(c->W.err, 0, sizeof(int));
  cudaMemset(c->W.bin_count, 0, sizeof(int) * c->P.nbin[0] * c->P.nbin[1] * c->P.nbin[2]);
  *c->err_host = 0;
  c->last_error = "no error";
}

const char* contact_last_error(contact_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

contact_status contact_stats(contact_ctx* c, int64_t* stats) {
  if (c == nullptr || stats == nullptr) return CONTACT_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  int h[16];
  unsigned long long u[4];
  e = cudaMemcpy(h, c->W.counters, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(u, c->W.u64, sizeof(u), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
  stats[0] = h[0];
  stats[1] = static_cast<int64_t>(u[0]);
  stats[2] = h[1];
  stats[3] = h[5];
  stats[4] = contact_kernels_per_step(c);
  stats[5] = c->grid_narrow;
  stats[6] = c->P.nbin[0];
  stats[7] = c->last_replay;
  stats[8] = static_cast<int64_t>(u[1]);
  stats[9] = c->P.max_tiles;
  return CONTACT_OK;
}

contact_status contact_particle_boxes(contact_ctx* c, int32_t* lo_hi) {
  if (c == nullptr || lo_hi == nullptr) return CONTACT_EINVAL;
  const cudaError_t e =
      cudaMemcpyAsync(lo_hi, c->D.lohi, sizeof(int) * 6 * c->P.n, cudaMemcpyDeviceToDevice, c->stream);
  return e == cudaSuccess ? CONTACT_OK : cuda_fail(c, e, "cudaMemcpyAsync");
}

contact_status contact_narrow_time(contact_ctx* c, float* ms) {
  if (c == nullptr || ms == nullptr) return CONTACT_EINVAL;
  if (!c->have_step) return fail(c, CONTACT_ESTATE, "contact_narrow_time: no step yet");
  if (!c->cfg.narrow_events) return fail(c, CONTACT_ESTATE, "contact_narrow_time: narrow_events is off");
  cudaError_t e = cudaEventSynchronize(c->ev_narrow[1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  e = cudaEventElapsedTime(ms, c->ev_narrow[0], c->ev_narrow[1]);
  if (e == cudaSuccess && c->cfg.narrow_events > 1) *ms /= static_cast<float>(c->cfg.narrow_events);
  return e == cudaSuccess ? CONTACT_OK : cuda_fail(c, e, "cudaEventElapsedTime");
}

namespace {
// The contact-history buffer the next step reads (after the stream's work).
contact_status history_buffer(contact_ctx* c, int* buf) {
  if (!c->P.history) return fail(c, CONTACT_ESTATE, "contact history is off");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  int steps = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(&steps, c->W.counters + kStepCounter, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "contact history");
  *buf = steps & 1;
  return CONTACT_OK;
}
}  // namespace

contact_status contact_history_get(contact_ctx* c, int64_t max_rows, int32_t* ij, double* cv, double* box,
                                   int64_t* n) {
  if (c == nullptr || n == nullptr || max_rows < 0 || (max_rows > 0 && (ij == nullptr || cv == nullptr)))
    return CONTACT_EINVAL;
  int b = 0;
  const contact_status hs = history_buffer(c, &b);
  if (hs != CONTACT_OK) return hs;
  const size_t np = static_cast<size_t>(c->P.n), cap = static_cast<size_t>(c->P.max_nbr);
  std::vector<int> cnt(np), hj(np * cap);
  std::vector<double> hc(np * cap), hb(c->W.hist_box != nullptr ? np * cap * 6 : 0);
  cudaError_t e = cudaMemcpy(cnt.data(), c->W.hist_n + b * np, sizeof(int) * np, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(hj.data(), c->W.hist_j + b * np * cap, sizeof(int) * np * cap, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(hc.data(), c->W.hist_c + b * np * cap, sizeof(double) * np * cap, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && !hb.empty())
    e = cudaMemcpy(hb.data(), c->W.hist_box + b * np * cap * 6, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "contact_history_get");
  std::vector<std::pair<std::pair<int, int>, size_t>> rows;   // (i, j), slot
  for (size_t i = 0; i < np; ++i)
    for (int m = 0; m < std::min(cnt[i], c->P.max_nbr); ++m)
      rows.push_back({{static_cast<int>(i), hj[i * cap + m]}, i * cap + m});
  std::sort(rows.begin(), rows.end());
  *n = static_cast<int64_t>(rows.size());
  for (int64_t r = 0; r < std::min<int64_t>(max_rows, *n); ++r) {
    ij[2 * r] = rows[r].first.first;
    ij[2 * r + 1] = rows[r].first.second;
    cv[r] = hc[rows[r].second];
    if (box != nullptr)
      for (int k = 0; k < 6; ++k) box[6 * r + k] = hb.empty() ? 0.0 : hb[6 * rows[r].second + k];
  }
  return CONTACT_OK;
}

contact_status contact_history_set(contact_ctx* c, int64_t n_rows, const int32_t* ij, const double* cv,
                                   const double* box) {
  if (c == nullptr || n_rows < 0 || (n_rows > 0 && (ij == nullptr || cv == nullptr))) return CONTACT_EINVAL;
  int b = 0;
  const contact_status hs = history_buffer(c, &b);
  if (hs != CONTACT_OK) return hs;
  const size_t np = static_cast<size_t>(c->P.n), cap = static_cast<size_t>(c->P.max_nbr);
  std::vector<int> cnt(np, 0), hj(np * cap, -1);
  std::vector<double> hc(np * cap, 0.0), hb(c->W.hist_box != nullptr ? np * cap * 6 : 0, 0.0);
  if (!hb.empty() && n_rows > 0 && box == nullptr)
    return fail(c, CONTACT_EINVAL, "contact_history_set: the box pipeline's history needs the boxes");
  for (int64_t r = 0; r < n_rows; ++r) {
    const int i = ij[2 * r], j = ij[2 * r + 1];
    if (i < 0 || i >= c->P.n || j <= i || j >= c->P.n + c->P.nwall)   // j >= N: a wall
      return fail(c, CONTACT_EINVAL, "contact_history_set: bad (i, j)");
    if (cnt[i] >= c->P.max_nbr) return fail(c, CONTACT_EINVAL, "contact_history_set: more rows of i than max_neighbors");
    for (int m = 0; m < cnt[i]; ++m)
      if (hj[i * cap + m] == j) return fail(c, CONTACT_EINVAL, "contact_history_set: repeated (i, j)");
    hj[i * cap + cnt[i]] = j;
    hc[i * cap + cnt[i]] = cv[r];
    if (!hb.empty()) {
      for (int k = 0; k < 3; ++k)
        if (!(box[6 * r + k] <= box[6 * r + 3 + k]) || !std::isfinite(box[6 * r + k]) || !std::isfinite(box[6 * r + 3 + k]))
          return fail(c, CONTACT_EINVAL, "contact_history_set: bad box");
      for (int k = 0; k < 6; ++k) hb[6 * (i * cap + cnt[i]) + k] = box[6 * r + k];
    }
    ++cnt[i];
  }
  cudaError_t e = cudaMemcpy(c->W.hist_n + b * np, cnt.data(), sizeof(int) * np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->W.hist_j + b * np * cap, hj.data(), sizeof(int) * np * cap, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->W.hist_c + b * np * cap, hc.data(), sizeof(double) * np * cap, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hb.empty())
    e = cudaMemcpy(c->W.hist_box + b * np * cap * 6, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? CONTACT_OK : cuda_fail(c, e, "contact_history_set");
}

contact_status contact_history_reset(contact_ctx* c) {
  if (c == nullptr) return CONTACT_EINVAL;
  if (!c->P.history) return fail(c, CONTACT_ESTATE, "contact history is off");
  const cudaError_t e = cudaMemsetAsync(c->W.hist_n, 0, sizeof(int) * 2 * c->P.n, c->stream);
  return e == cudaSuccess ? CONTACT_OK : cuda_fail(c, e, "cudaMemsetAsync");
}

int32_t contact_kernels_per_step(const contact_ctx* c) {
  if (c == nullptr) return 0;
  return 5 + (c->P.npoly > 0 ? 1 : 0) + (c->P.box_mode == 0 ? 1 : 0);   // + polytope pose, + force law
}
int32_t contact_kernels_per_backward(const contact_ctx*) { return 3; }

contact_status contact_backward(contact_ctx* c, const double* grad_force, const double* grad_torque,
                                double* grad_pos, double* grad_quat) {
  const NvtxRange range("contact_backward");
  if (c == nullptr) return CONTACT_EINVAL;
  if (grad_force == nullptr || grad_torque == nullptr || grad_pos == nullptr || grad_quat == nullptr)
    return fail(c, CONTACT_EINVAL, "contact_backward: null buffer");
  if (!c->have_step) return fail(c, CONTACT_ESTATE, "contact_backward: no contact_step before");
  if (c->P.smooth != 1) return fail(c, CONTACT_ESTATE, "contact_backward: needs the smoothed indicator");
  if (c->P.box_mode != 0)
    return fail(c, CONTACT_ESTATE, "contact_backward: the box pipeline's samples move with the box (no adjoint)");
  const contact_status sticky = check_sticky(c);
  if (sticky != CONTACT_OK) return sticky;
  launch_adjoint(c->P, c->S, c->D, c->W, c->last_vel, grad_force, grad_torque, grad_pos, grad_quat,
                 c->adj_scratch, c->grid_adjoint, c->stream, c->cfg.narrow_events ? c->ev_adj[0] : nullptr,
                 c->cfg.narrow_events ? c->ev_adj[1] : nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  c->have_backward = true;
  return CONTACT_OK;
}

contact_status contact_adjoint_time(contact_ctx* c, float* ms) {
  if (c == nullptr || ms == nullptr) return CONTACT_EINVAL;
  if (!c->have_backward) return fail(c, CONTACT_ESTATE, "contact_adjoint_time: no backward yet");
  if (!c->cfg.narrow_events) return fail(c, CONTACT_ESTATE, "contact_adjoint_time: narrow_events is off");
  cudaError_t e = cudaEventSynchronize(c->ev_adj[1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  e = cudaEventElapsedTime(ms, c->ev_adj[0], c->ev_adj[1]);
  return e == cudaSuccess ? CONTACT_OK : cuda_fail(c, e, "cudaEventElapsedTime");
}

contact_status contact_step_host(contact_ctx* c, const double* pos, const double* quat, const double* vel,
                                 int32_t* n_pairs, double* force, double* torque, int32_t* pair_ij,
                                 double* pair_out) {
  const NvtxRange range("contact_step_host");
  if (c == nullptr) return CONTACT_EINVAL;
  if (pos == nullptr || quat == nullptr || n_pairs == nullptr || force == nullptr || torque == nullptr)
    return fail(c, CONTACT_EINVAL, "contact_step_host: null buffer");
  const contact_status sticky = check_sticky(c);
  if (sticky != CONTACT_OK) return sticky;
  const size_t n = static_cast<size_t>(c->P.n), mp = static_cast<size_t>(c->P.max_pairs);
  cudaError_t e = cudaSuccess;
  if (c->hs_pos == nullptr) {   // first call: the device side of the host buffers
    if ((e = dev_alloc(c, &c->hs_pos, 3 * n)) != cudaSuccess || (e = dev_alloc(c, &c->hs_quat, 4 * n)) != cudaSuccess ||
        (e = dev_alloc(c, &c->hs_vel, 6 * n)) != cudaSuccess || (e = dev_alloc(c, &c->hs_force, 3 * n)) != cudaSuccess ||
        (e = dev_alloc(c, &c->hs_torque, 3 * n)) != cudaSuccess ||
        (e = dev_alloc(c, &c->hs_pair_ij, 2 * mp)) != cudaSuccess ||
        (e = dev_alloc(c, &c->hs_pair_out, 11 * mp)) != cudaSuccess ||
        (e = dev_alloc(c, &c->hs_npairs, 1)) != cudaSuccess) {
      c->hs_pos = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(c, CONTACT_ENOMEM, "contact_step_host: device buffers")
                                            : cuda_fail(c, e, "cudaMalloc");
    }
  }
  // page-locked host memory (all of it): copies inside the captured graph
  auto pinned = [](const void* p) {
    if (p == nullptr) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeHost;
  };
  const void* key[7] = {pos, quat, vel, n_pairs, force, torque, c->stream};
  const bool same = c->hexec != nullptr && std::memcmp(key, c->hkey, sizeof(key)) == 0;   // replay: pinned before
  const bool all_pinned = same || (pinned(pos) && pinned(quat) && pinned(vel) && pinned(n_pairs) && pinned(force) &&
                                   pinned(torque));
  double* dvel = vel != nullptr ? c->hs_vel : nullptr;
  // Page-locked host memory is mapped into the device's address space (and on
  // Grace-Blackwell reached coherently over NVLink-C2C): when every buffer
  // has a device address, the pose kernels read the poses and the particle
  // sums write the forces and torques there directly, with no copy nodes.
  // The velocities, read per pair by the force law, are still copied.
  auto mapped = [](const void* p) -> void* {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  };
  const double *zpos = nullptr, *zquat = nullptr;
  double *zforce = nullptr, *ztorque = nullptr;
  int32_t* znp = nullptr;
  bool zero_copy = false;
  if (!same && all_pinned) {
    zpos = static_cast<const double*>(mapped(pos));
    zquat = static_cast<const double*>(mapped(quat));
    zforce = static_cast<double*>(mapped(force));
    ztorque = static_cast<double*>(mapped(torque));
    znp = static_cast<int32_t*>(mapped(n_pairs));
    zero_copy = zpos && zquat && zforce && ztorque && znp;
  }
  auto enqueue_all = [&](bool capturing) {
    if (zero_copy) {
      if (vel != nullptr) cudaMemcpyAsync(c->hs_vel, vel, 6 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
      enqueue_step(c, capturing, zpos, zquat, dvel, c->hs_pair_ij, c->hs_pair_out, znp, zforce, ztorque, true);
      return;
    }
    cudaMemcpyAsync(c->hs_pos, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->hs_quat, quat, 4 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (vel != nullptr) cudaMemcpyAsync(c->hs_vel, vel, 6 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    enqueue_step(c, capturing, c->hs_pos, c->hs_quat, dvel, c->hs_pair_ij, c->hs_pair_out, c->hs_npairs,
                 c->hs_force, c->hs_torque);
    cudaMemcpyAsync(force, c->hs_force, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(torque, c->hs_torque, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(n_pairs, c->hs_npairs, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
  };
  // When the kernels write the results in place (no copies after the last
  // kernel) and no step of contact_step may still be queued, the step gets a
  // fresh token (read by its first kernel, published by its last block once
  // the results are stored) and the call waits for that token instead of
  // synchronising the stream; a queued step could carry the token, so after
  // contact_step, as with copies, it synchronises (and later calls use tokens
  // again).
  const bool in_place = same ? c->hzero : zero_copy;
  const bool idle = in_place && !c->step_unwaited;
  int token = 0;
  if (idle) {
    token = c->host_token = c->host_token == 0x7fffffff ? 1 : c->host_token + 1;
    reinterpret_cast<volatile int*>(c->err_host)[2] = token;
  }
  if (all_pinned && c->cfg.use_graph && c->stream != nullptr) {
    if (!same) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
      enqueue_all(true);
      e = cudaStreamEndCapture(c->stream, &g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      bool updated = false;
      if (c->hexec != nullptr && c->hkey[6] == c->stream) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(c->hexec, g, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();
      }
      if (!updated) {
        if (c->hexec) cudaGraphExecDestroy(c->hexec);
        c->hexec = nullptr;
        e = cudaGraphInstantiate(&c->hexec, g, 0);
        if (e != cudaSuccess) {
          cudaGraphDestroy(g);
          c->hexec = nullptr;
          return cuda_fail(c, e, "cudaGraphInstantiate");
        }
      }
      cudaGraphDestroy(g);
      std::memcpy(c->hkey, key, sizeof(key));
      c->hzero = zero_copy;
    }
    e = cudaGraphLaunch(c->hexec, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  } else {
    enqueue_all(false);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "contact_step_host");
  }
  c->have_step = true;
  c->last_vel = dvel;
  bool done = false;
  if (idle) {   // bounded wait for the token (a step that fails to finish is reported by the synchronisation)
    const volatile int* published = c->err_host + 1;
    for (long it = 0; it < (1L << 26) && !done; ++it) done = *published == token;
  }
  if (!done) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  }
  c->step_unwaited = false;
  const contact_status st = check_sticky(c);
  if (st != CONTACT_OK) return st;
  if (pair_ij != nullptr || pair_out != nullptr) {
    const size_t P = static_cast<size_t>(std::min<int32_t>(std::max<int32_t>(*n_pairs, 0), c->P.max_pairs));
    if (P > 0 && pair_ij != nullptr)
      e = cudaMemcpy(pair_ij, c->hs_pair_ij, 2 * P * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && P > 0 && pair_out != nullptr)
      e = cudaMemcpy(pair_out, c->hs_pair_out, 11 * P * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
  }
  return CONTACT_OK;
}

void contact_destroy(contact_ctx* c) {
  if (c == nullptr) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->hexec) cudaGraphExecDestroy(c->hexec);
  cudaDeviceSynchronize();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (cudaEvent_t ev : c->ev_narrow)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : c->ev_adj)
    if (ev) cudaEventDestroy(ev);
  for (void* p : c->dev_allocs) cudaFree(p);
  if (c->err_host) cudaFreeHost(c->err_host);
  delete c;
}

}  // extern "C"
