// contact_step_noalloc: the contact step without any device allocation.
//
// Some callers cannot call cudaMalloc: a host program that hands all device
// memory to its own pool allocator and forbids libraries from allocating, a
// real-time loop that must not touch the driver's allocator between steps, or
// an embedding that may not create a context-owned object.  contact_init
// allocates its scratch, so those callers cannot create a context.  This entry
// point needs no context: the caller passes its inputs and outputs, and every
// intermediate buffer of the step lives in one file-scope __device__ array of
// fixed size (below), which every GPU that loads the library holds until the
// process exits.
//
// The scratch is shared by all calls, and keeps the contents of the last call;
// the set-up kernel clears everything that must start at zero.  Two calls
// whose work overlaps on the GPU (other threads, other streams) race on it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>   // CUcontext (types only; cuCtxGetCurrent is reached through the runtime)

#include "../../include/contact.h"
#include "contact_dev.cuh"

using namespace gbc;

namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(CONTACT_NOALLOC_SCRATCH_MIB) << 20;
constexpr int kMaxNbr = 64;
constexpr int kMaxTilesPerPair = CONTACT_NOALLOC_TILES_PER_PAIR;
constexpr int kMaxBinsPerAxis = CONTACT_NOALLOC_MAX_BINS;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device address of g_scratch (host code may not use the symbol itself),
// with the context it belongs to: a device reset destroys the primary
// context and the module with it, and the next call, in a new context,
// looks the address up again.
std::mutex g_mutex;
unsigned char* g_addr[64] = {};
CUcontext g_ctx[64] = {};

using CtxGetCurrent = CUresult (*)(CUcontext*);

CUcontext current_context() {
  static const CtxGetCurrent fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<CtxGetCurrent>(nullptr);
    return reinterpret_cast<CtxGetCurrent>(p);
  }();
  CUcontext c = nullptr;
  if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

contact_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 64) return CONTACT_ECUDA;
  // the device's primary context, current (cudaSetDevice initialises it)
  if (cudaSetDevice(dev) != cudaSuccess) return CONTACT_ECUDA;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_addr[dev] == nullptr || ctx == nullptr || ctx != g_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return CONTACT_ECUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
    g_ctx[dev] = ctx;
  }
  *out = g_addr[dev];
  return CONTACT_OK;
}

// Bump carving of the scratch array into 256-byte aligned regions.
struct Carver {
  unsigned char* base;
  size_t used = 0;
  bool overflow = false;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (std::max<size_t>(count, 1) * sizeof(T) + 255) & ~static_cast<size_t>(255);
    if (used + bytes > kScratchBytes) {
      overflow = true;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// Derived per-particle tables and the zero-initialised words of the step.
__global__ void k_noalloc_prep(Params P, int* type, int* kind, double* param, float* size_l, int* nomops,
                               const double* young, const double* poisson, double* compl_, double* ext,
                               int* face_off, int* vert_off, Lists W, int nbins) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P.n) {
    const int ty = type[t];
    // the same rounded operations as contact_init's host code (no contraction)
    compl_[t] = __ddiv_rn(__dsub_rn(1.0, __dmul_rn(poisson[t], poisson[t])), young[t]);
    for (int k = 0; k < 3; ++k) ext[3 * t + k] = (ty == 0 && k > 0) ? 0.0 : __dadd_rn(param[3 * t + k], P.delta);
    const double* q = param + 3 * t;
    kind[t] = ty == 0 ? KIND_SPHERE : ((q[0] == q[1] && q[0] == q[2]) ? KIND_CUBE : KIND_CUBOID);
    nomops[t] = ty == 0 ? 7 : 15;
    for (int k = 0; k < 3; ++k)
      size_l[3 * t + k] = static_cast<float>(__ddiv_rn(__dadd_rn(param[3 * t + k], P.inflate), P.dx));
  }
  if (t <= P.n) {
    face_off[t] = 0;
    vert_off[t] = 0;
  }
  for (int b = t; b < nbins; b += gridDim.x * blockDim.x) W.bin_count[b] = 0;
  if (t < 16) W.counters[t] = 0;
  if (t < 4) W.u64[t] = 0;
  if (t == 0) *W.err = 0;
  if (t < 4) W.err_host[t] = 0;
}

}  // namespace

extern "C" contact_status contact_step_noalloc(const contact_config* cfg, const int32_t* shape_type,
                                               const double* shape_param, const double* young,
                                               const double* poisson, const double* pos, const double* quat,
                                               int32_t* pair_ij, double* pair_out, int32_t* n_pairs,
                                               double* force, double* torque, void* stream) {
  if (cfg == nullptr || shape_type == nullptr || shape_param == nullptr || young == nullptr ||
      poisson == nullptr || pos == nullptr || quat == nullptr || pair_ij == nullptr || pair_out == nullptr ||
      n_pairs == nullptr || force == nullptr || torque == nullptr)
    return CONTACT_EINVAL;
  const contact_config& C = *cfg;
  const int n = C.n_particles;
  // sizes beyond the scratch array's fixed capacity are rejected up front
  if (n < 1 || n > CONTACT_NOALLOC_MAX_PARTICLES) return CONTACT_EINVAL;
  if (C.max_pairs < 1 || C.max_pairs > CONTACT_NOALLOC_MAX_PAIRS) return CONTACT_EINVAL;
  if (C.max_neighbors != 0 && C.max_neighbors != kMaxNbr) return CONTACT_EINVAL;
  if (C.max_tiles != 0 && C.max_tiles > kMaxTilesPerPair * CONTACT_NOALLOC_MAX_PAIRS) return CONTACT_EINVAL;
  if (C.precision != CONTACT_PRECISION_FP32_TILE) return CONTACT_EINVAL;
  if (C.history != 0 || C.friction != 0 || C.n_walls != 0 || C.box_mode != 0)
    return CONTACT_EINVAL;   // contact history, friction, walls: the context path
  if (!(C.dx > 0.0) || !std::isfinite(C.dx) || (C.indicator != 0 && C.indicator != 1)) return CONTACT_EINVAL;
  if (!(C.smooth_width > 0.0) || !(C.inflate >= 0.0) || !(C.damping_c >= 0.0)) return CONTACT_EINVAL;
  for (int k = 0; k < 3; ++k)
    if (C.n_cells[k] < 1) return CONTACT_EINVAL;
  const double band = (C.indicator == 1) ? (0.5 * C.smooth_width) * C.dx : 0.0;
  const double delta = C.inflate + band;
  double rmax = 0.0, rin_min = 1e300;
  for (int p = 0; p < n; ++p) {
    const double* prm = shape_param + 3 * p;
    if (!(young[p] > 0.0) || !(poisson[p] >= 0.0) || !(poisson[p] < 1.0)) return CONTACT_EINVAL;
    if (shape_type[p] == CONTACT_SHAPE_SPHERE) {
      if (!(prm[0] > 0.0)) return CONTACT_EINVAL;
      rmax = std::max(rmax, prm[0] + delta);
      rin_min = std::min(rin_min, prm[0]);
    } else if (shape_type[p] == CONTACT_SHAPE_CUBOID) {
      double e2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        if (!(prm[k] > 0.0)) return CONTACT_EINVAL;
        e2 += (prm[k] + delta) * (prm[k] + delta);
      }
      rmax = std::max(rmax, std::sqrt(e2));
      rin_min = std::min(rin_min, std::min(prm[0], std::min(prm[1], prm[2])));
    } else {
      return CONTACT_EINVAL;  // polytopes need the context path
    }
  }
  Params P{};
  P.n = n;
  for (int k = 0; k < 3; ++k) {
    P.ncell[k] = C.n_cells[k];
    P.L[k] = C.n_cells[k] * C.dx;
    if (!(P.L[k] > 4.0 * rmax + 2.0 * C.dx)) return CONTACT_EDOMAIN;
    if (!(2.0 * rmax / C.dx + 4.0 < 65535.0)) return CONTACT_EDOMAIN;
    int nb = static_cast<int>(std::floor(P.L[k] / (2.0 * rmax + 2.0 * C.dx)));
    if (nb < 3) nb = 1;
    P.nbin[k] = std::min(nb, kMaxBinsPerAxis);
    P.binw[k] = P.L[k] / P.nbin[k];
    P.inv_binw_f[k] = static_cast<float>(P.nbin[k] / P.L[k]);
  }
  P.bin_cap = bin_capacity(n, P.binw, rin_min, static_cast<long long>(P.nbin[0]) * P.nbin[1] * P.nbin[2],
                           CONTACT_NOALLOC_MAX_BIN_ENTRIES);
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
  P.precision = CONTACT_PRECISION_FP32_TILE;
  P.kind_set = 1;
  P.damping_c = C.damping_c;
  P.max_pairs = C.max_pairs;
  P.max_nbr = kMaxNbr;
  P.max_tiles = C.max_tiles > 0 ? C.max_tiles : kMaxTilesPerPair * C.max_pairs;
  P.inflate_l = static_cast<float>(C.inflate / C.dx);
  P.inv_w = static_cast<float>(1.0 / C.smooth_width);
  P.neg6_over_w = static_cast<float>(-6.0 / C.smooth_width);
  P.wdx_l = static_cast<float>(C.smooth_width);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CONTACT_ECUDA;
  unsigned char* base = nullptr;
  const contact_status st = scratch_address(dev, &base);
  if (st != CONTACT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // carve the scratch array
  Carver cv{base};
  const size_t N = static_cast<size_t>(n), MP = static_cast<size_t>(P.max_pairs),
               MT = static_cast<size_t>(P.max_tiles);
  const int nbins = P.nbin[0] * P.nbin[1] * P.nbin[2];
  int* type = cv.take<int>(N);
  int* kind = cv.take<int>(N);
  double* param = cv.take<double>(3 * N);
  double* yv = cv.take<double>(N);
  double* pv = cv.take<double>(N);
  float* size_l = cv.take<float>(3 * N);
  int* nomops = cv.take<int>(N);
  double* compl_ = cv.take<double>(N);
  double* ext = cv.take<double>(3 * N);
  float* verts32 = cv.take<float>(3);
  float* off32 = cv.take<float>(1);
  int* face_off = cv.take<int>(N + 1);
  int* vert_off = cv.take<int>(N + 1);
  double* planes = cv.take<double>(4);
  double* verts = cv.take<double>(3);
  Shapes S{type, param, face_off, planes, vert_off, verts, yv, pv, size_l, nomops, compl_, ext, verts32, off32};
  Parts D{};
  D.X = cv.take<double>(3 * N);
  D.qhat = cv.take<double>(4 * N);
  D.R = cv.take<double>(9 * N);
  D.lohi = cv.take<int>(6 * N);
  D.bin = cv.take<int>(N);
  D.Rt = cv.take<float>(9 * N);
  D.wplane = cv.take<float4>(1);
  D.Xf = cv.take<float>(3 * N);
  D.kX = cv.take<int>(3 * N);
  D.fX = cv.take<float>(3 * N);
  Lists W{};
  W.bin_count = cv.take<int>(nbins);
  W.bin_items = cv.take<int>(static_cast<size_t>(nbins) * P.bin_cap);
  W.up_count = cv.take<int>(N);
  W.up_list = cv.take<int>(N * kMaxNbr);
  W.dn_count = cv.take<int>(N);
  W.dn_list = cv.take<int>(N * kMaxNbr);
  W.dn_pair = cv.take<int>(N * kMaxNbr);
  W.row_off = cv.take<int>(N + 1);
  W.grp_sum = cv.take<int>((N + kRowGroup - 1) / kRowGroup);
  W.pairs = cv.take<PairRec>(MP);
  W.olist = cv.take<OvlRec>(MP);
  W.oflag = cv.take<int>(MP);
  W.tile_pair = cv.take<int>(MT);
  W.tiles = cv.take<PairRec>(MT);
  W.partial = cv.take<float>(MT * kPartialFloats);
  W.pdone = cv.take<int>(MP);
  W.tape = cv.take<double>(MP * kTapeDoubles);
  W.ft = cv.take<double>(MP * kFtDoubles);
  W.kind = kind;
  W.counters = cv.take<int>(16);
  W.u64 = cv.take<unsigned long long>(4);
  W.err = cv.take<int>(1);
  W.err_host = cv.take<int>(4);   // the mapped-host words of the context path, here on the device
  if (cv.overflow) return CONTACT_EINVAL;

  // inputs into the scratch array (copies, no allocation)
  cudaError_t e = cudaSuccess;
  e = cudaMemcpyAsync(type, shape_type, N * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(param, shape_param, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(yv, young, N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pv, poisson, N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return CONTACT_ECUDA;
  const int threads = 256, blocks = (n + 1 + threads - 1) / threads;
  k_noalloc_prep<<<blocks, threads, 0, s>>>(P, type, kind, param, size_l, nomops, yv, pv, compl_, ext, face_off,
                                            vert_off, W, nbins);
  // the step's kernels, unchanged, on the scratch array
  launch_pose(P, S, D, W, pos, quat, s);
  launch_broad(P, D, W, s);
  launch_plan(P, S, D, W, pair_ij, n_pairs, pair_out, s);
  launch_narrow(P, S, D, W, nullptr, pair_out, narrow_grid(P), s);
  launch_force(P, S, D, W, nullptr, pair_out, s);
  launch_particle_sum(P, D, W, force, torque, s);
  if (cudaGetLastError() != cudaSuccess) return CONTACT_ECUDA;
  // synchronous: the device error word is read back before returning
  int err = 0;
  if (cudaMemcpyAsync(&err, W.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CONTACT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CONTACT_ECUDA;
  return static_cast<contact_status>(err);
}
