/*
 * contact.h -- C-ABI of the GB300 discrete-contact library (libcontact.so).
 *
 * The library evaluates the discrete contact model of Marquardt, Hafen and
 * Krause, "A novel model for direct numerical simulation of suspension
 * dynamics with arbitrarily shaped convex particles" (arXiv:2401.10878), for
 * spheres, cuboids and convex polytopes in a periodic lattice:
 *
 *   broad phase      -> candidate pairs, periodic image of the higher-ID
 *                       particle moved to the lower-ID side (Sec. 3.3.2)
 *   overlap sweep    -> every lattice node of each pair's bounding box is tested
 *                       against both signed distance functions; the nodes are
 *                       reduced to overlap volume, contact point, contact
 *                       normal and indentation depth (Sec. 3.3.1)
 *   force law        -> F = 4/(3 pi) n E* sqrt(V d)(1 + c ddot_n),
 *                       E* = ((1-nu_A^2)/E_A + (1-nu_B^2)/E_B)^-1 (Sec. 2.3,
 *                       Eq. contact_force_normal), torques about each centre
 *                       of mass (Sec. 2.2)
 *   adjoint          -> gradient of sum_p (gF_p . F_p + gT_p . T_p) with
 *                       respect to positions and quaternions (smoothed indicator)
 *
 * Conventions (all calls):
 *   - Lattice node k in Z^3 sits at x = k dx; the periodic box is L = n_cells * dx.
 *   - A pose is a centre of mass X (Sec. 2.2) and a quaternion (w, x, y, z),
 *     Hamilton convention, body -> world, normalised inside the library.
 *   - Shapes are given in their body frame with the origin at the centre of
 *     mass: a sphere by its radius, a cuboid by its half extents, a polytope
 *     by half-spaces n . y <= d with unit n and d > 0 (bounded).
 *   - "dev" pointers are device memory of the context's GPU, "host" pointers
 *     are host memory.  The caller owns every buffer it passes; the context
 *     owns its scratch, allocated once in contact_init.
 *   - Calls that take dev pointers enqueue work on the context stream and
 *     return without synchronising.  contact_step and contact_backward
 *     allocate nothing.
 *   - Errors found on the host return at once.  Errors found on the device
 *     (inputs out of range, capacity overflow) are sticky: they are returned by
 *     the next call once the device has written them, and by contact_check.
 */
#ifndef GB300_CONTACT_H
#define GB300_CONTACT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct contact_ctx contact_ctx; /* opaque, owned by the library */

typedef enum {
  CONTACT_OK = 0,
  CONTACT_EINVAL = 1,    /* invalid argument or input value                   */
  CONTACT_ENOMEM = 2,    /* device or host allocation failed (contact_init)   */
  CONTACT_ECUDA = 3,     /* a CUDA runtime call failed                        */
  CONTACT_ECAPACITY = 4, /* more pairs / neighbours / tiles than configured,
                            or more particle centres in one cell-list bin than
                            its capacity (twice the bin volume over the
                            smallest inscribed ball, plus 8)                   */
  CONTACT_EDOMAIN = 5,   /* periodic box too small for the largest particle   */
  CONTACT_ETIMEOUT = 6,  /* a bounded device wait ran out                     */
  CONTACT_ESTATE = 7,    /* call out of order (e.g. backward before a step)   */
  CONTACT_EBOUNDS = 8    /* a device index check failed: only the checked
                            build (compiled with -DCONTACT_CHECKS) tests the
                            indices it reads from device lists; the access is
                            skipped and the step's outputs are invalid       */
} contact_status;

enum { CONTACT_SHAPE_SPHERE = 0, CONTACT_SHAPE_CUBOID = 1, CONTACT_SHAPE_POLYTOPE = 2 };
enum { CONTACT_INDICATOR_SHARP = 0, CONTACT_INDICATOR_SMOOTH = 1 };
enum { CONTACT_PRECISION_FP32_TILE = 0, CONTACT_PRECISION_FP64_PAIR = 1 };

/* Width of one row of pair_out. */
#define CONTACT_PAIR_OUT_COLS 11

typedef struct {
  int32_t n_particles;
  int32_t n_cells[3];       /* periodic lattice, L = n_cells * dx                   */
  double dx;                /* lattice spacing (> 0)                                 */
  int32_t indicator;        /* CONTACT_INDICATOR_SHARP: H = [phi <= 0];
                               CONTACT_INDICATOR_SMOOTH: H_w(phi) = S(clamp(1/2 -
                               phi/(w dx), 0, 1)), S(t) = 3t^2 - 2t^3              */
  double smooth_width;      /* w in lattice cells (> 0); also the width of the band
                               used for the contact normal in sharp mode           */
  double inflate;           /* enlargement subtracted from every signed distance,
                               physical units (the paper uses dx/5, Sec. 5.1)      */
  double damping_c;         /* damping factor c of Eq. (contact_force_normal),
                               applied to every contact when velocities are given;
                               contact_damping_factor computes it (>= 0)           */
  int32_t precision;        /* CONTACT_PRECISION_FP32_TILE: FP32 node tests, FP32
                               tile partials, FP64 per-pair reduction;
                               CONTACT_PRECISION_FP64_PAIR: everything in FP64,
                               one thread block per pair                           */
  int32_t max_pairs;        /* capacity of the pair list (> 0)                       */
  int32_t max_neighbors;    /* capacity of one particle's candidate list (0: 64)    */
  int32_t max_tiles;        /* capacity of the node-tile list (0: 8 * max_pairs)    */
  int32_t use_graph;        /* 1: contact_step captures its launches in a CUDA graph
                               on first use and replays it while the buffers are
                               the same (not while the stream is being captured)   */
  int32_t narrow_events;    /* 1: record CUDA events around the node-sweep launch
                               (read with contact_narrow_time); K in 2..64: the
                               node sweep runs K times back to back between the
                               events (the later runs recompute the same outputs)
                               and contact_narrow_time returns the time per run,
                               without the events' own overhead (not with
                               box_mode 1: EINVAL); 0: none, so that consecutive
                               kernels overlap their launch                       */
  int32_t history;          /* 1: contact history (Sec. 4.3.3): a contact (a pair
                               with V > 0) keeps the damping factor of Eq.
                               (damping_factor) computed with `restitution` from
                               its approach speed ddot_n at its first step (u0 <= 0
                               gives 0) until the first step without overlap;
                               damping_c is then unused.  Needs velocities.        */
  int32_t friction;         /* 1: tangential force of Eq. (contact_force_tangential)
                               added to F: B receives +f(a) |F_n| t, A the
                               opposite, t the direction of A's velocity relative to
                               B at x_c minus its normal part, a = |u_t| / u_k,
                               f(a) = (2 mu_s* - mu_k) a^2/(a^4+1) + mu_k -
                               mu_k/(a^2+1), mu_s* = mu_s (1 - 0.09 (mu_k/mu_s)^4).
                               Needs velocities.                                  */
  double restitution;       /* coefficient of restitution e in [0, 1] (history)   */
  double mu_s, mu_k;        /* friction coefficients (mu_s > 0, mu_k >= 0)        */
  double u_k;               /* transition speed of the friction law (> 0), in the
                               caller's velocity units (the paper: 0.001 m/s)     */
  int32_t n_walls;          /* fixed walls (Sec. 4.3), 0..CONTACT_MAX_WALLS: wall w
                               is the half-space m . x <= h, not periodic (it is
                               tested in the frame where the particle's centre lies
                               in [0, L)); its contacts are pairs (i, N + w) and
                               are evaluated like particle pairs, the wall at rest
                               with the identity pose at the origin.  Forces and
                               torques are reported for the particles only.       */
  int32_t reserved;
  const double* walls;      /* [n_walls,4] host, (m, h) with unit m pointing out of
                               the wall; read by contact_init only                */
  const double* wall_young; /* [n_walls] host, E of each wall (> 0)               */
  const double* wall_poisson; /* [n_walls] host, nu of each wall (0 <= nu < 1)    */
  int32_t box_mode;         /* 0: the sample set is every lattice node of the pair
                               box (default); 1: the paper's box pipeline (Sec.
                               3.3.1): rough detection at the nodes where both
                               signed distances are below sqrt(0.75) dx (node
                               ranges widened by that much), the box widened by
                               it and each face moved inward to the nearest entry
                               of contact_resolution^2 axis-parallel lines into the
                               overlap, then contact_resolution^3 cell-centre
                               samples; no contact_backward.  With the history, an
                               ongoing contact's corrected box of the last step
                               (kept relative to X_i), widened by sqrt(0.75) dx,
                               cuts the widened rough box down per axis before
                               the correction (the warm start of Sec. 4.3.3)      */
  int32_t contact_resolution; /* N_c of box_mode 1, 1..64 (the paper uses 8)      */
} contact_config;

enum { CONTACT_MAX_WALLS = 64 };

/* Fills *cfg with defaults (sharp indicator, w = 1, no inflation, FP32 tiles,
 * no contact history (restitution 1), no friction (mu_s = mu_k = 0, u_k = 1),
 * max_pairs = 16 n, graphs on) for n particles in an n_cells lattice of
 * spacing dx. */
void contact_config_default(contact_config* cfg, int32_t n_particles, const int32_t n_cells[3], double dx);

/* Creates a context on the current CUDA device.
 *   shape_type  [N]      host, CONTACT_SHAPE_*
 *   shape_param [N,3]    host, sphere: (r, -, -); cuboid: half extents (hx, hy, hz)
 *   face_offset [N+1]    host, polytope p owns planes[face_offset[p] .. face_offset[p+1])
 *                        (non-polytopes own none; 4 <= faces <= 32)
 *   planes      [F,4]    host, (n0, n1, n2, d) body frame, n . y <= d, |n| = 1, d > 0
 *   young, poisson [N]   host, E > 0 and 0 <= nu < 1 per particle (Sec. 2.3)
 *   stream               cudaStream_t (NULL: default stream); changeable with
 *                        contact_set_stream
 * Returns CONTACT_EINVAL for an invalid shape or configuration,
 * CONTACT_EDOMAIN when L <= 4 R_max + 2 dx on some axis (R_max = the largest
 * circumradius after inflation), so that at most one periodic image of a
 * partner can overlap a particle, or when 2 R_max / dx + 4 >= 65535 (a pair's
 * node box spans fewer than 2^16 nodes along every axis).  *out is NULL on
 * failure. */
contact_status contact_init(const contact_config* cfg, const int32_t* shape_type, const double* shape_param,
                            const int32_t* face_offset, const double* planes, const double* young,
                            const double* poisson, void* stream, contact_ctx** out);

/* One contact evaluation (Sec. 3.3.1 / 3.3.2 / Eq. contact_force_normal).
 *   pos   [N,3] dev f64  centres of mass, 0 <= X < L on every axis
 *   quat  [N,4] dev f64  (w, x, y, z), any non-zero norm
 *   vel   [N,6] dev f64  (u, omega) per particle, or NULL (then ddot_n = 0)
 * Outputs (dev, written on the context stream):
 *   pair_ij  [max_pairs,2] i32   candidate pairs (i < j) sorted by (i, j); j >= N
 *                                is wall j - N
 *   pair_out [max_pairs,11] f64  per pair: V, x_c[3], n[3], d, F[3]; F is the
 *                                force on j (-F acts on i), n points from i to
 *                                j, x_c is in i's frame (not wrapped)
 *   n_pairs  [1] i32             number of candidate pairs P
 *   force, torque [N,3] f64      per-particle sums over the pairs, in the order
 *                                (pairs where the particle is j, by i), then
 *                                (pairs where it is i, by j)
 * Pairs whose shapes do not overlap on any node have V = x_c = n = d = F = 0.
 * Positions outside [0, L), zero quaternions and non-finite values set the
 * sticky CONTACT_EINVAL; more than max_pairs candidates sets
 * CONTACT_ECAPACITY (n_pairs then holds the count that was needed). */
contact_status contact_step(contact_ctx* ctx, const double* pos, const double* quat, const double* vel,
                            int32_t* pair_ij, double* pair_out, int32_t* n_pairs, double* force,
                            double* torque);

/* contact_step with HOST buffers, end to end: copies pos [N,3], quat [N,4]
 * and vel [N,6] (or NULL) from host memory into context-owned device buffers,
 * runs the step, copies force and torque [N,3] and the pair count back to host
 * memory (n_pairs, force, torque must not be NULL), and returns when the
 * copies are complete.  When pair_ij / pair_out are not NULL the first
 * min(P, max_pairs) rows of the pair outputs are copied to them as well (as
 * laid out by contact_step).  When pos, quat, n_pairs, force and torque are
 * all page-locked and mapped into the device's address space (as cudaHostAlloc
 * and cudaHostRegister memory is with unified addressing), the step's kernels
 * read the poses and write the pair count, forces and torques there directly
 * (coherent over NVLink-C2C on Grace-Blackwell), with vel copied, all in one
 * captured graph; other page-locked buffers are copied inside that graph,
 * pageable ones with ordinary copies around the step.  The device buffers are allocated at the first call and owned by
 * the context.  Completion: with the results written in place and no step of
 * contact_step still unwaited on this context, the call waits (spinning on a
 * mapped host word, bounded, then falling back to a synchronisation) for a
 * token its step publishes after the forces and torques are stored, so it may
 * return while the step's last kernel is still retiring; otherwise it
 * synchronises the context stream.  Either way the outputs are complete on
 * return.  Errors: those of contact_step, reported by this call;
 * CONTACT_ENOMEM if the buffers cannot be allocated.  A later
 * contact_backward differentiates this step. */
contact_status contact_step_host(contact_ctx* ctx, const double* pos, const double* quat, const double* vel,
                                 int32_t* n_pairs, double* force, double* torque, int32_t* pair_ij,
                                 double* pair_out);

/* Gradient of L = sum_p (grad_force_p . force_p + grad_torque_p . torque_p)
 * of the last contact_step with respect to its positions and raw quaternions
 * (the quaternion gradient is orthogonal to the quaternion).  Needs the
 * smoothed indicator (CONTACT_ESTATE otherwise) and uses the step's tape, so
 * the step's pos/quat/vel must still hold the same values (the buffers are
 * read again).  Covers damping and friction; each contact's damping factor c
 * (the shared one, or with the contact history the contact's own) is held
 * fixed, a constant of the contact.
 *   grad_force, grad_torque [N,3] dev f64 ; grad_pos [N,3], grad_quat [N,4] dev f64 */
contact_status contact_backward(contact_ctx* ctx, const double* grad_force, const double* grad_torque,
                                double* grad_pos, double* grad_quat);

/* Synchronises the context stream and returns the sticky device error (the
 * error stays set; contact_clear_error resets it). */
contact_status contact_check(contact_ctx* ctx);
void contact_clear_error(contact_ctx* ctx);

/* Human-readable description of the last error of the context (never NULL). */
const char* contact_last_error(contact_ctx* ctx);

/* Makes later calls enqueue on another stream (drops cached graphs). */
contact_status contact_set_stream(contact_ctx* ctx, void* stream);

/* Synchronises, then fills stats[0..9] (host) with the last step's pair count,
 * node evaluations (sum of box volumes), node tiles, pairs with V > 0,
 * kernels launched per step, narrow-phase grid size, bins per axis (x),
 * whether the last step replayed a graph (0: instantiated it, or no graph;
 * 1: replayed; 2: replayed after updating it in place for new buffers on the
 * same stream), the nominal FP32 lane-operations of
 * the node sweep (sum over pairs of box volume x (ops_i + ops_j), with 7 per
 * sphere test, 15 per cuboid test and 4F per polytope test), and the tile
 * capacity. */
contact_status contact_stats(contact_ctx* ctx, int64_t* stats);

/* Synchronises, then writes the device time in milliseconds of the last
 * step's narrow-phase kernel (the node sweep), measured with CUDA events that
 * contact_step records on the context stream around that launch (also when
 * the step replays a graph) when cfg.narrow_events is on; with
 * narrow_events = K > 1 the events enclose K back-to-back runs and the time
 * is their mean.  CONTACT_ESTATE before the first step or with narrow_events
 * off. */
contact_status contact_narrow_time(contact_ctx* ctx, float* ms);

/* Synchronises, then writes the device time in milliseconds of the last
 * contact_backward's node-level kernel (the adjoint's cell sweep), measured
 * with CUDA events recorded around that launch when cfg.narrow_events is on.
 * CONTACT_ESTATE before the first backward or with narrow_events off. */
contact_status contact_adjoint_time(contact_ctx* ctx, float* ms);

/* Per-particle node ranges (lo[3], hi[3]) [N,6] i32 dev of the last step. */
contact_status contact_particle_boxes(contact_ctx* ctx, int32_t* lo_hi);

/* Contact history (cfg.history = 1; Sec. 4.3.3): the contacts of the last
 * completed step (pairs (i, j), i < j, with V > 0), the damping factor c
 * each keeps and, with box_mode 1, its corrected box (lo[3], hi[3]) minus
 * X_i, the warm start of the next correction; the next step reads them.
 * All three return CONTACT_ESTATE with the history off.
 * contact_history_get synchronises, then writes the first min(*n, max_rows)
 * contacts, sorted by (i, j), to ij [max_rows,2] i32 host, c [max_rows] f64
 * host and box [max_rows,6] f64 host (nullable; zeros with box_mode 0); *n
 * receives the number of contacts (which may exceed max_rows).
 * contact_history_set replaces them with the n_rows given (host arrays, as
 * a checkpoint to resume from; box is read with box_mode 1 only, where it is
 * required): CONTACT_EINVAL for a row with i >= j, i outside [0, N), j
 * outside [0, N + n_walls) (j >= N: a wall), a repeated (i, j), more than
 * max_neighbors rows of one i, or a box with lo > hi or a non-finite bound.
 * contact_history_reset forgets every contact (asynchronous, on the context
 * stream). */
contact_status contact_history_get(contact_ctx* ctx, int64_t max_rows, int32_t* ij, double* c, double* box,
                                   int64_t* n);
contact_status contact_history_set(contact_ctx* ctx, int64_t n_rows, const int32_t* ij, const double* c,
                                   const double* box);
contact_status contact_history_reset(contact_ctx* ctx);

/* Volume centroid (host) of the polytope {y : n_f . y <= d_f} given by
 * n_faces >= 4 rows (n, d) with unit n and d > 0 (origin inside), bounded.
 *   planes [n_faces,4] host; centroid [3] host out.  CONTACT_EINVAL on
 *   invalid planes. */
contact_status contact_polytope_centroid(const double* planes, int32_t n_faces, double* centroid);

/* Poses refer to the centre of mass (Sec. 2.2: the torque reference).
 * contact_init moves the body origin of every polytope whose volume centroid
 * c lies more than 1e-6 x (its smallest d) from it to c, by d_f -= n_f . c in
 * its own copy of the planes; positions passed to contact_step then name the
 * centroid (a caller holding the origin's position X_o passes X_o + R c).
 * Polytopes given about their centroid are used unchanged, bit for bit.
 * contact_polytope_shift writes c per particle, shift [N,3] f64 host (zero
 * for spheres, cuboids and unmoved polytopes).  CONTACT_EINVAL for a null
 * argument. */
contact_status contact_polytope_shift(const contact_ctx* ctx, double* shift);

/* Eq. (damping_factor): c = 1.5 (1-e)(11-e) / ((1+9e) u0) for u0 > 0, else 0,
 * from the coefficient of restitution e and the relative speed u0 at first
 * contact (Carvalho-Martins, as used in Sec. 2.3). */
double contact_damping_factor(double restitution, double u0);

/* Number of kernel launches one contact_step / contact_backward issues (a
 * step has one more when polytopes are present). */
int32_t contact_kernels_per_step(const contact_ctx* ctx);
int32_t contact_kernels_per_backward(const contact_ctx* ctx);

void contact_destroy(contact_ctx* ctx);

/* Fixed capacity of contact_step_noalloc: the size of its scratch array in
 * MiB, the largest particle count and pair capacity it accepts, the node-tile
 * budget per pair (max_tiles 0 means CONTACT_NOALLOC_TILES_PER_PAIR x
 * max_pairs; a tile holds up to 128 node lines of one pair, so this covers
 * pair boxes of up to 256 lines on average), and the cell list's limits (at
 * most CONTACT_NOALLOC_MAX_BINS bins per axis, and bins x bin capacity at
 * most CONTACT_NOALLOC_MAX_BIN_ENTRIES).  contact_init allows 8 tiles per
 * pair, 256 bins per axis and 2^26 bin entries. */
#define CONTACT_NOALLOC_SCRATCH_MIB 32
#define CONTACT_NOALLOC_MAX_PARTICLES 2048
#define CONTACT_NOALLOC_MAX_PAIRS 8192
#define CONTACT_NOALLOC_TILES_PER_PAIR 2
#define CONTACT_NOALLOC_MAX_BINS 32
#define CONTACT_NOALLOC_MAX_BIN_ENTRIES (1 << 20)

/* contact_step for callers that cannot allocate device memory (no
 * counterpart in the paper: it is an interface for such callers, e.g. a host
 * program whose own pool owns all device memory, or a loop that may not call
 * the driver's allocator).  No context is created and nothing is allocated:
 * the step's intermediate buffers live in one static device array of
 * CONTACT_NOALLOC_SCRATCH_MIB MiB, which every GPU that loads the library
 * holds until the process exits.
 *   cfg, shape_type, shape_param, young, poisson   host, as for contact_init;
 *                     spheres and cuboids only, n_particles <=
 *                     CONTACT_NOALLOC_MAX_PARTICLES, max_pairs <=
 *                     CONTACT_NOALLOC_MAX_PAIRS, max_neighbors 0 or 64,
 *                     precision CONTACT_PRECISION_FP32_TILE; use_graph ignored
 *   pos, quat, pair_ij, pair_out, n_pairs, force, torque   dev, as for contact_step
 *   stream            cudaStream_t for all work (NULL: default stream)
 * Larger sizes, polytopes or other settings return CONTACT_EINVAL before any
 * work is enqueued.  The call waits for its stream and returns the device's
 * error (CONTACT_EINVAL for a bad pose, CONTACT_ECAPACITY) directly; velocities
 * are not taken (ddot_n = 0).  More pairs than max_pairs, more tiles than the
 * tile budget or a fuller bin than the cell list holds return
 * CONTACT_ECAPACITY (n_pairs then holds the pair count needed).  The first
 * call on a device, and the first after its primary context was recreated
 * (cudaDeviceReset), looks up the array's device address, so make that call
 * before any stream capture.  All
 * calls share the one array and the set-up clears what must start at zero:
 * calls whose work overlaps on the GPU (from other threads or streams) race
 * and must be serialised by the caller. */
contact_status contact_step_noalloc(const contact_config* cfg, const int32_t* shape_type, const double* shape_param,
                                    const double* young, const double* poisson, const double* pos,
                                    const double* quat, int32_t* pair_ij, double* pair_out, int32_t* n_pairs,
                                    double* force, double* torque, void* stream);

/* Measurement utility (no counterpart in the paper): the FP32 FFMA rate of
 * the current device, the measured counterpart of the node sweep's roofline
 * peak (SMs x 128 FP32 lanes x clock).  One warm-up and one timed launch of
 * eight independent FFMA chains per thread, iters x 128 FFMAs each, on eight
 * 256-thread blocks per SM (~1 ms at iters = 2000); synchronous, on the
 * default stream, with its own 1.2 MB scratch allocation.
 *   iters        1 .. 2^20
 *   ffma_per_s   host out: FFMA lane-operations per second
 * CONTACT_EINVAL for a bad argument, CONTACT_ENOMEM / CONTACT_ECUDA on a CUDA
 * failure. */
contact_status contact_fp32_ffma_rate(int32_t iters, double* ffma_per_s);

/* Measurement utility (no counterpart in the paper): the FP64 DFMA rate of
 * the current device, the measured peak of the all-FP64 comparison form.
 * The same launch shape as contact_fp32_ffma_rate with FP64 chains (GB300's
 * FP64 pipe is narrow: iters = 50 takes ~2 ms); synchronous, default stream,
 * its own 2.5 MB scratch allocation.
 *   iters        1 .. 2^20
 *   dfma_per_s   host out: DFMA lane-operations per second
 * CONTACT_EINVAL for a bad argument, CONTACT_ENOMEM / CONTACT_ECUDA on a CUDA
 * failure. */
contact_status contact_fp64_dfma_rate(int32_t iters, double* dfma_per_s);

/* Self-test of the device index checks (no counterpart in the paper).
 * Enqueues on the context stream one kernel that passes the index n to the
 * check for an array of n entries (one past its end; nothing is accessed),
 * then synchronises and reads the sticky error word like contact_check.  The
 * checked build (libcontact_checks.so, compiled with -DCONTACT_CHECKS)
 * returns CONTACT_EBOUNDS and keeps it sticky until contact_clear_error; the
 * normal build compiles the check away and returns CONTACT_OK.
 * CONTACT_EINVAL for a null context. */
contact_status contact_bounds_selftest(contact_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GB300_CONTACT_H */
