// Internal layouts and device helpers of libcontact (not part of the C-ABI).
//
// Memory layout in HBM (all buffers allocated once by contact_init):
//   shape tables (read-only): type/kind per particle, FP64 body parameters,
//     body planes, offset-shape vertices (for the AABB), E and nu;
//   per-step particle records: FP64 pose copy (the adjoint's tape), FP64
//     rotation, node ranges, bins, FP32 geometry for the node sweep
//     (R^T rows, effective sizes, world-frame polytope planes);
//   pair list: PairRec per candidate pair, tile -> pair map, FP32 tile
//     partials, FP64 per-pair sums and results.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gbc {

// Sweep kinds: polytopes (up to 32 faces) read their planes from shared
// memory; cubes (equal half extents) have their own kind: max|y| - h needs no
// per-axis offset.  (Kind 2 is not used.)
enum Kind : int { KIND_SPHERE = 0, KIND_CUBOID = 1, KIND_POLY = 3, KIND_CUBE = 4, KIND_WALL = 5 };

// Evaluator order of a pair in the node sweep: the cheaper kind is A (wall <
// sphere < cube < cuboid < polytope; kind 2 is unused); true when the
// record's particle j is A.
__device__ __forceinline__ bool sweep_swap(int ka, int kb) {
  // ranks 1, 3, 6, 5, 2, 0 of kinds 0 .. 5 in nibbles (an indexed array would live in local memory)
  constexpr unsigned kRank = 0x025631u;
  return ((kRank >> (4 * ka)) & 15u) > ((kRank >> (4 * kb)) & 15u);
}

// Half the cell diagonal, sqrt(0.75), in lattice units: the box pipeline's
// rough-detection threshold (Sec. 3.3.1).
constexpr float kRoughT = 0.8660254037844386f;

constexpr int kMaxFaces = 32;         // faces of one polytope
constexpr int kTileItemsPerLane = 4;  // node lines per lane per tile
constexpr int kPartialFloats = 12;    // FP32 partial sums per tile
constexpr int kTapeDoubles = 16;      // FP64 per-pair values kept for the adjoint
constexpr int kStepCounter = 12;      // counters[] slot of the completed-step count
constexpr int kDoneCounter = 13;      // counters[] slot: particle-sum blocks finished (the last resets it)
constexpr int kTokenCounter = 14;     // counters[] slot: the host's token of this step
constexpr int kFtDoubles = 9;         // per-pair F, T_A, T_B

// Error codes written by kernels (same numbering as contact_status).
constexpr int kErrInval = 1;
constexpr int kErrCapacity = 4;
constexpr int kErrBounds = 8;

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Index checks of the checked build (-DCONTACT_CHECKS): an index read from a
// device list (a partner, a pair, a tile, a bin) that lies outside [0, n)
// sets the sticky error word to kErrBounds and is replaced by `safe` (an
// index that is in range, or a value the caller already treats as "none"),
// so the access it feeds stays inside its array and no lane leaves its warp.
// In the normal build the index passes through unchanged and the check
// compiles away.
__device__ __forceinline__ int checked_index(int* err, int i, long long n, int safe) {
#ifdef CONTACT_CHECKS
  if (i >= 0 && static_cast<long long>(i) < n) return i;
  set_error(err, kErrBounds);
  return safe;
#else
  (void)err; (void)n; (void)safe;
  return i;
#endif
}

// floor(a / b) and the remainder for small non-negative ints via an FP32
// reciprocal, corrected by one step (exact for a < 2^22)
__device__ __forceinline__ int div_small(int a, int b, float inv_b, int* rem) {
  int q = static_cast<int>((static_cast<float>(a) + 0.5f) * inv_b);
  int r = a - q * b;
  if (r < 0) { --q; r += b; }
  if (r >= b) { ++q; r -= b; }
  *rem = r;
  return q;
}

// --------------------------------------------------------------------------
// Constant per-context parameters, passed to every kernel by value.
struct Params {
  int n;                 // particles
  int ncell[3];          // lattice nodes per axis
  double dx, inv_dx;
  double L[3];           // n_cells * dx
  double delta;          // AABB offset: inflate (+ w dx / 2 in smoothed mode)
  double inflate;        // physical
  double wdx;            // smoothing width, physical
  double dx3;            // dx^3 (volume of a node)
  double gscale;         // 1/2 dx^2 * 6 / w: band sum -> G
  double g_min2;         // (1e-12 dx^2)^2: |G|^2 below it takes the centre-line normal
  int smooth;            // 1: smoothed indicator
  int precision;         // 0: FP32 tiles, 1: FP64 per pair
  int kind_set;          // node-sweep variant: 0 all kinds, 1 spheres and cuboids, 2 cubes only
  int dx_pow2;           // 1: dx is a power of two, so x / dx == x * inv_dx exactly
  double damping_c;
  int box_mode, box_res; // 1: the paper's box pipeline with box_res (N_c) points per direction
  int npoly;             // polytope particles (one pose warp each)
  int nwall;             // fixed walls: partner indices n .. n + nwall - 1
  const double* wall;    // [nwall,4] (m, h): the half-space m . x <= h
  int history, friction;  // contact history; tangential force
  double damp_K;         // history: c = damp_K / u0 at a contact's first step (u0 > 0)
  double mu_s_star, mu_k, inv_u_k;   // friction law
  int nbin[3];           // bins per axis
  int bin_cap;           // particles one bin can hold (bin_items row length)
  double binw[3];        // bin width (physical)
  float inv_binw_f[3];   // FP32 reciprocal of the bin width
  int max_pairs, max_nbr, max_tiles;
  // FP32 copies for the node sweep (lattice units)
  float inflate_l, inv_w, neg6_over_w, wdx_l;   // wdx_l: smoothing width in cells
};

// Shape tables (read-only after contact_init); rows N .. N + nwall - 1 are
// the walls, one-plane polytopes (the plane in the world frame).
struct Shapes {
  const int* type;         // [N] CONTACT_SHAPE_*
  const double* param;     // [N,3]
  const int* face_off;     // [N+1]
  const double* planes;    // [F,4] body frame
  const int* vert_off;     // [N+1]
  const double* verts;     // [V,3] vertices of the offset shape (AABB)
  const double* young;     // [N]
  const double* poisson;   // [N]
  const float* size_l;     // [N,3] lattice units incl. inflate: sphere r', cuboid h'
  const int* nomops;       // [N] nominal FP32 lane-ops of one signed-distance test
  const double* compl_;    // [N] (1 - nu^2) / E, so that E* = 1 / (compl_i + compl_j)
  const double* ext;       // [N,3] sphere: r + delta; cuboid: h_k + delta (AABB half sizes in the body frame)
  const float* verts32;    // [V,3] FP32 copy of the offset-shape vertices (prefilter of the extremes)
  const float* off32;      // [F] (d + inflate) / dx per face, FP32
  const int* poly_ids;     // [npoly] the polytope particles (the pose kernel's polytope warps)
};

// Per-step particle records; rows N .. N + nwall - 1 are the walls (set once:
// X = 0, R = I, Rt row 0 = the wall normal m, kX = fX = 0).
struct Parts {
  double* X;       // [N,3] copy of the positions of the step
  double* qhat;    // [N,4] the step's quaternion as given (normalised by the adjoint)
  double* R;       // [N,9] FP64 rotation, row-major, body -> world
  int* lohi;       // [N,6]
  int* bin;        // [N]
  float* Rt;       // [N,9] FP32 R^T (row k = body axis k in world)
  float4* wplane;  // [F] FP32 world normal, offset (lattice units, incl. inflate)
  float* Xf;       // [N,3] FP32 positions (periodic image choice only)
  int* kX;         // [N,3] nearest node of X / dx
  float* fX;       // [N,3] X / dx - kX, in [-1/2, 1/2] (FP64 difference, rounded once)
  const double* rest6;   // [6] zeros: the velocity of a wall
};

// One candidate pair (i < j).
struct __align__(16) PairRec {   // 16-byte aligned: records are copied with 16-byte accesses
  int i, j;
  int lo[3];       // lower node of the pair box (i's frame)
  int dim[3];      // nodes per axis
  int shift[3];    // image index s of j: X_j' = X_j - s L
  int axis;        // sweep axis (the box's longest)
  int seglen;      // nodes per line segment (the whole line)
  int nseg;        // segments per line (1)
  int nitems;      // lines * nseg
  int tile0;       // first tile of the pair
  int ntiles;
  int kinds;       // kind of i | kind of j << 8 (set by the planner)
  // particle centres relative to lo in lattice units, split into the nearest
  // integer and an FP32 remainder in [-1/2, 1/2] so that node offsets stay exact
  int ai[3], bi[3];
  float af[3], bf[3];
  // FP32 sweep geometry of both particles: R^T rows and sizes (lattice units)
  float rta[9], rtb[9];
  float sza[3], szb[3];
  int tile;        // in a tile record: the tile's index within its pair
  int pair;        // in a tile record: the pair index
};
constexpr int kPairRecWords = sizeof(PairRec) / 4;
static_assert(sizeof(PairRec) % 16 == 0, "PairRec is staged with 16-byte copies");

// Node box of particle node range [lo_in, hi_in] against the wall m . x <= h
// widened by delta (e = (m, h)): false when even the range's lowest corner in
// m lies beyond h + delta, or when the clip leaves no node; else the range
// clipped, per axis with m_k != 0, to the nodes that some node of the range
// with that coordinate keeps inside.  Rounded FP64 operations in a fixed
// order (no contraction), so that the box is reproducible bit for bit.
__device__ __forceinline__ bool wall_box(const double* e, double delta, double dx, const int* lo_in,
                                         const int* hi_in, int lo[3], int hi[3]) {
  const double H = __dadd_rn(e[3], delta);
  double t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int ck = e[k] > 0.0 ? lo_in[k] : hi_in[k];
    t[k] = __dmul_rn(e[k], __dmul_rn(static_cast<double>(ck), dx));
    lo[k] = lo_in[k];
    hi[k] = hi_in[k];
  }
  if (!(__dadd_rn(__dadd_rn(t[0], t[1]), t[2]) <= H)) return false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (e[k] == 0.0) continue;
    const double rest = k == 0 ? __dadd_rn(t[1], t[2]) : (k == 1 ? __dadd_rn(t[0], t[2]) : __dadd_rn(t[0], t[1]));
    const double b = __ddiv_rn(__ddiv_rn(__dsub_rn(H, rest), e[k]), dx);
    if (e[k] > 0.0) {
      if (b < hi[k]) hi[k] = static_cast<int>(floor(b));
    } else {
      if (b > lo[k]) lo[k] = static_cast<int>(ceil(b));
    }
  }
  return lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2];
}

// Checked build: a pair or tile record read from a device list names a pair,
// two particles (j may be a wall) and tiles inside their arrays; otherwise the
// sticky error word gets kErrBounds and the caller skips the record (its
// value is warp-uniform, so the whole warp skips it).  Always true, and
// compiled away, in the normal build.
__device__ __forceinline__ bool record_in_bounds(const Params& P, int* err, const PairRec& r, bool tile_rec) {
#ifdef CONTACT_CHECKS
  bool ok = r.i >= 0 && r.i < P.n && r.j >= 0 && r.j < P.n + P.nwall && r.ntiles >= 0 && r.tile0 >= 0 &&
            static_cast<long long>(r.tile0) + r.ntiles <= P.max_tiles;
  if (tile_rec) ok = ok && r.pair >= 0 && r.pair < P.max_pairs && r.tile >= 0 && r.tile < r.ntiles;
  if (!ok) set_error(err, kErrBounds);
  return ok;
#else
  (void)P; (void)err; (void)r; (void)tile_rec;
  return true;
#endif
}

// Work lists shared by the step's kernels.
// One overlapping pair for the force law (appended to the step's overlap list
// by the warp that completes it): its FP64 sums (count, first moments, band
// terms of G), its deepest node, and the pair record's geometry.
struct OvlRec {
  double s[7];     // sum of H, of H x (x, y, z) in box coordinates, of the band terms (x, y, z)
  int q;           // pair index
  int idx;         // deepest node (linear index in the pair box)
  int i, j;        // particles
  int lo[3];       // pair box origin (nodes)
  int dim[3];      // pair box nodes per axis
  int shift[3];    // image index of j
  int pad[5];
};
static_assert(sizeof(OvlRec) == 128, "one overlap record per 128-byte line");

struct Lists {
  int* bin_count;   // [nbins]
  int* bin_items;   // [nbins, bin_cap] particles of each bin, in arrival order
  int* up_count;    // [N] partners j > p
  int* up_list;     // [N, max_nbr]
  int* dn_count;    // [N] partners i < p
  int* dn_list;     // [N, max_nbr]
  int* dn_pair;     // [N, max_nbr] pair index of (dn_list[p][r], p)
  int* row_off;     // [N + 1] first pair of particle i
  int* grp_sum;     // [ceil(N / 256)] partners above, summed over groups of 256 particles
  int* hist_j;      // [2, N, max_nbr] contact history: partner j > i of each ongoing contact of i
  double* hist_c;   // [2, N, max_nbr] its damping factor
  int* hist_n;      // [2, N] contacts per particle; buffer (steps & 1) is read, the other written
  double* hist_box; // [2, N, max_nbr, 6] box pipeline: each contact's corrected box relative to X_i (or null)
  PairRec* pairs;   // [max_pairs]
  OvlRec* olist;    // [max_pairs] entry q: pair q's sums when it overlaps (oflag[q] = 1): the force law's work
  int* oflag;       // [max_pairs] 1 when pair q overlaps (V > 0), else 0 (written by the node sweep or the
                    // pair builder's separation test)
  int* tile_pair;   // [max_tiles] pair of each tile
  PairRec* tiles;   // [max_tiles] one record per tile (the pair's record with tile and pair set), the
                    // node sweep's list: a pair's tiles contiguous from its tile0
  float* partial;   // [max_tiles, kPartialFloats]
  int* pdone;       // [max_pairs] tiles of the pair swept so far (pairs of several tiles)
  double* tape;     // [max_pairs, kTapeDoubles]
  double* ft;       // [max_pairs, kFtDoubles]
  const int* kind;  // [N] sweep kind of each particle (Kind, polytopes by face bucket)
  int* counters;    // [16]: 0 pairs, 1 tiles, 2 box pipeline queue, 5 overlapping pairs, kStepCounter
                    // steps completed (its parity selects the contact-history buffer)
  unsigned long long* u64;  // [4]: 0 node evaluations, 1 nominal lane-ops of the node sweep
  int* err;         // [1] sticky device error
  int* err_host;    // [3] mapped host words: 0 mirrors err; 1 the token of the last completed step
                    // (written by the step's last block); 2 the token the host gave the step being
                    // launched (read by k_pose into counters[kTokenCounter])
  int publish;      // 1 in a host-buffer step that returns on its token: k_pose reads the token, the
                    // particle sums' last block mirrors err and publishes it (0: err mirrored at the
                    // start of the particle sums, no token)
};

// --------------------------------------------------------------------------
// FP64 helpers with explicit rounding (no contraction): the node ranges must
// agree bit for bit with an independent CPU evaluation of the same formulas.
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Row k of the rotation of q / |q| (w, x, y, z), body -> world, in homogeneous
// form with s = 2 / |q|^2 (2 RN(1/nn) == RN(2/nn): scaling by 2 is exact).
__device__ inline void rotation_row_rn(const double q[4], double s, int k, double r[3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  if (k == 0) {
    r[0] = dsub(1.0, dmul(s, dadd(dmul(y, y), dmul(z, z))));
    r[1] = dmul(s, dsub(dmul(x, y), dmul(w, z)));
    r[2] = dmul(s, dadd(dmul(x, z), dmul(w, y)));
  } else if (k == 1) {
    r[0] = dmul(s, dadd(dmul(x, y), dmul(w, z)));
    r[1] = dsub(1.0, dmul(s, dadd(dmul(x, x), dmul(z, z))));
    r[2] = dmul(s, dsub(dmul(y, z), dmul(w, x)));
  } else {
    r[0] = dmul(s, dsub(dmul(x, z), dmul(w, y)));
    r[1] = dmul(s, dadd(dmul(y, z), dmul(w, x)));
    r[2] = dsub(1.0, dmul(s, dadd(dmul(x, x), dmul(y, y))));
  }
}

// Rotation of the normalised quaternion (w, x, y, z), body -> world, row-major.
__device__ inline void rotation_rn(const double q[4], double* qh, double* qn, double R[9]) {
  const double nrm = __dsqrt_rn(dadd(dadd(dadd(dmul(q[0], q[0]), dmul(q[1], q[1])), dmul(q[2], q[2])),
                                     dmul(q[3], q[3])));
  const double w = __ddiv_rn(q[0], nrm), x = __ddiv_rn(q[1], nrm), y = __ddiv_rn(q[2], nrm),
               z = __ddiv_rn(q[3], nrm);
  qh[0] = w; qh[1] = x; qh[2] = y; qh[3] = z;
  *qn = nrm;
  R[0] = dsub(1.0, dmul(2.0, dadd(dmul(y, y), dmul(z, z))));
  R[1] = dmul(2.0, dsub(dmul(x, y), dmul(w, z)));
  R[2] = dmul(2.0, dadd(dmul(x, z), dmul(w, y)));
  R[3] = dmul(2.0, dadd(dmul(x, y), dmul(w, z)));
  R[4] = dsub(1.0, dmul(2.0, dadd(dmul(x, x), dmul(z, z))));
  R[5] = dmul(2.0, dsub(dmul(y, z), dmul(w, x)));
  R[6] = dmul(2.0, dsub(dmul(x, z), dmul(w, y)));
  R[7] = dmul(2.0, dadd(dmul(y, z), dmul(w, x)));
  R[8] = dsub(1.0, dmul(2.0, dadd(dmul(x, x), dmul(y, y))));
}

// FP64 signed distance (physical units, reduced by inflate) at world point x
// for a particle at X with rotation R; writes the world gradient of the
// active branch (first maximal face on ties).
__device__ inline double sdf64(int type, const double* prm, const double* planes, int nf, const double X[3],
                               const double R[9], const double x[3], double inflate, double g[3]) {
  const double r[3] = {x[0] - X[0], x[1] - X[1], x[2] - X[2]};
  if (type == 0) {
    const double nr = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int k = 0; k < 3; ++k) g[k] = nr > 0.0 ? r[k] / nr : 0.0;
    return nr - prm[0] - inflate;
  }
  double y[3];
  for (int k = 0; k < 3; ++k) y[k] = R[k] * r[0] + R[3 + k] * r[1] + R[6 + k] * r[2];
  double best = -1e300, gb[3] = {0.0, 0.0, 0.0};
  if (type == 1) {
    for (int k = 0; k < 3; ++k) {
      const double a = fabs(y[k]) - prm[k];
      if (a > best) {
        best = a;
        gb[0] = gb[1] = gb[2] = 0.0;
        gb[k] = y[k] < 0.0 ? -1.0 : 1.0;
      }
    }
  } else {
    for (int f = 0; f < nf; ++f) {
      const double* e = planes + 4 * f;
      const double a = (e[0] * y[0] + e[1] * y[1] + e[2] * y[2]) - e[3];
      if (a > best) {
        best = a;
        gb[0] = e[0]; gb[1] = e[1]; gb[2] = e[2];
      }
    }
  }
  for (int k = 0; k < 3; ++k) g[k] = R[3 * k] * gb[0] + R[3 * k + 1] * gb[1] + R[3 * k + 2] * gb[2];
  return best - inflate;
}


// Exact FP32 -> FP64 conversion with integer operations (IEEE 754: sign kept,
// exponent rebiased by 1023 - 127, fraction widened by 29 bits; subnormals
// normalised): no FP64 instruction, for kernels whose FP64 pipe is the limit.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sgn = u & 0x80000000u;
  int e = static_cast<int>((u >> 23) & 0xffu);
  unsigned m = u & 0x7fffffu;
  if (e == 0xff) return static_cast<double>(f);   // inf / NaN: not produced by the sweep
  if (e == 0) {
    if (m == 0) return __hiloint2double(static_cast<int>(sgn), 0);
    const int lz = __clz(m) - 8;                   // moves the leading 1 to the implicit bit
    m = (m << lz) & 0x7fffffu;
    e = 1 - lz;
  }
  const unsigned hi = sgn | (static_cast<unsigned>(e + 896) << 20) | (m >> 3);
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(m << 29));
}

// Programmatic dependent launch: every kernel of a step lets the next one
// launch at its start, and waits for the previous one (completion and memory
// visibility) before it reads that kernel's results.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch with the programmatic-stream-serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// --------------------------------------------------------------------------
// Launch wrappers (defined in the kernel translation units).
void launch_pose(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* pos,
                 const double* quat, cudaStream_t st);
void launch_broad(const Params& P, const Parts& D, const Lists& W, cudaStream_t st);
void launch_plan(const Params& P, const Shapes& S, const Parts& D, const Lists& W, int32_t* pair_ij, int32_t* n_pairs,
                 double* pair_out, cudaStream_t st);
constexpr int kRowGroup = 256;   // particles per group sum of the pair-row offsets
int bin_capacity(int n, const double binw[3], double rin_min, long long nbins, long long max_entries);
void launch_narrow(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                   double* pair_out, int grid, cudaStream_t st);
int narrow_grid(const Params& P);
void launch_box(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel, double* pair_out,
                int grid, cudaStream_t st);
void launch_force(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel, double* pair_out,
                  cudaStream_t st);
void launch_particle_sum(const Params& P, const Parts& D, const Lists& W, double* force, double* torque,
                         cudaStream_t st);
size_t adjoint_scratch_doubles(int max_pairs, int max_tiles);
void launch_adjoint(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                    const double* gF, const double* gT, double* gpos, double* gquat, double* scratch,
                    int grid, cudaStream_t st, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);

}  // namespace gbc
