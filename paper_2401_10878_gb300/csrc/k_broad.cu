// Pose -> AABB, cell-list broad phase and pair planning of the contact step.
//
// Paper (arXiv:2401.10878): Sec. 3.3.1 (a contact is swept over the region
// where both particles may overlap), Sec. 3.3.2 (periodic boundaries: the
// higher-ID particle is moved to the side of the lower-ID one), Sec. 4.1
// (the neighbourhood radius is the largest circumradius).
#include <cfloat>

#include "contact_dev.cuh"
#include "line_clip.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int clamp_node(double v) {
  // node indices stay far inside int range even for garbage input
  v = fmin(fmax(v, -1.0e9), 1.0e9);
  return static_cast<int>(v);
}

// ---------------------------------------------------------------------------
// K1: one thread per (particle p, axis k): row k of the rotation, the node
// range along k, the FP32 sweep geometry and, on axis 0, the bin slot.  FP64
// is kept to what the bit-exact node range needs (every FP64 instruction
// costs ~64 cycles per warp on this GPU), and spread over three threads.
// Polytope p by one warp: the node range along each axis (the extreme
// projections of the offset-shape vertices: an FP32 prefilter over the
// vertices on all lanes, FP64 for the at most two candidates per side, all
// vertices in FP64 when more lie within the prefilter's window) and the
// FP32 world planes (faces on lanes).  The FP64 arithmetic is the per-axis
// thread's, operation for operation, so the node range is the same bit for bit.
__device__ void pose_polytope(const Params& P, const Shapes& S, const Parts& D, int p, const double* __restrict__ pos,
                              const double* __restrict__ quat) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  double q[4];
  for (int c = 0; c < 4; ++c) q[c] = quat[4 * p + c];
  bool bad = false;
  double Xv[3];
  for (int c = 0; c < 3; ++c) {
    const double v = pos[3 * p + c];
    long long b = __double_as_longlong(v);
    if (b == static_cast<long long>(0x8000000000000000ULL)) b = 0;
    const bool ok = b >= 0 && b < __double_as_longlong(P.L[c]);
    bad = bad || !ok;
    Xv[c] = ok ? __longlong_as_double(b) : 0.0;
  }
  const double nn = dadd(dadd(dadd(dmul(q[0], q[0]), dmul(q[1], q[1])), dmul(q[2], q[2])), dmul(q[3], q[3]));
  if (!(nn > 1e-24) || !(nn < 1e300)) {
    bad = true;
    q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
  }
  const double s = bad ? 2.0 : dmul(2.0, __drcp_rn(nn));
  // rotation rows: lane k < 3 computes row k, then every lane holds all nine
  double rk[3] = {0.0, 0.0, 0.0};
  if (lane < 3) rotation_row_rn(q, s, lane, rk);
  double R[3][3];
  float R32[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R[k][c] = __shfl_sync(full, rk[c], k);
      R32[k][c] = static_cast<float>(R[k][c]);
    }
  const int v0 = S.vert_off[p], v1 = S.vert_off[p + 1];
  // FP32 prefilter: extremes per axis and the largest |w|_1
  float lo32[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi32[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX}, wmax = 0.f;
  for (int vb = v0; vb < v1; vb += 32) {
    const int v = vb + lane;
    if (v < v1) {
      const float* w = S.verts32 + 3 * v;
      const float x0 = w[0], x1 = w[1], x2 = w[2];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float tv = fmaf(R32[k][0], x0, fmaf(R32[k][1], x1, R32[k][2] * x2));
        lo32[k] = fminf(lo32[k], tv);
        hi32[k] = fmaxf(hi32[k], tv);
      }
      wmax = fmaxf(wmax, fabsf(x0) + fabsf(x1) + fabsf(x2));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      lo32[k] = fminf(lo32[k], __shfl_xor_sync(full, lo32[k], o));
      hi32[k] = fmaxf(hi32[k], __shfl_xor_sync(full, hi32[k], o));
    }
    wmax = fmaxf(wmax, __shfl_xor_sync(full, wmax, o));
  }
  const float tol = 1e-5f * wmax + 1e-30f;
  // candidates within tol of the FP32 extremes, the first two in vertex order
  int lc[3][2], hc[3][2], nlo[3] = {0, 0, 0}, nhi[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < 3; ++k) lc[k][0] = lc[k][1] = hc[k][0] = hc[k][1] = v0;
  for (int vb = v0; vb < v1; vb += 32) {
    const int v = vb + lane;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (v < v1) {
      const float* w = S.verts32 + 3 * v;
      x0 = w[0]; x1 = w[1]; x2 = w[2];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float tv = fmaf(R32[k][0], x0, fmaf(R32[k][1], x1, R32[k][2] * x2));
      unsigned bl = __ballot_sync(full, v < v1 && tv <= lo32[k] + tol);
      unsigned bh = __ballot_sync(full, v < v1 && tv >= hi32[k] - tol);
      while (bl) {
        const int l = __ffs(bl) - 1;
        if (nlo[k] == 0) lc[k][0] = vb + l;
        else if (nlo[k] == 1) lc[k][1] = vb + l;
        ++nlo[k];
        bl &= bl - 1;
      }
      while (bh) {
        const int l = __ffs(bh) - 1;
        if (nhi[k] == 0) hc[k][0] = vb + l;
        else if (nhi[k] == 1) hc[k][1] = vb + l;
        ++nhi[k];
        bh &= bh - 1;
      }
    }
  }
  // exact FP64 projections of the candidates: lane k < 3 takes axis k
  auto proj3 = [&](double r0, double r1, double r2, int v) {
    const double* w = S.verts + 3 * v;
    return dadd(dadd(dmul(r0, w[0]), dmul(r1, w[1])), dmul(r2, w[2]));
  };
  double lo = 0.0, hi = 0.0;
  if (lane < 3) {
    const int k = lane;
    const int a0 = k == 0 ? lc[0][0] : (k == 1 ? lc[1][0] : lc[2][0]);
    const int a1 = k == 0 ? lc[0][1] : (k == 1 ? lc[1][1] : lc[2][1]);
    const int b0 = k == 0 ? hc[0][0] : (k == 1 ? hc[1][0] : hc[2][0]);
    const int b1 = k == 0 ? hc[0][1] : (k == 1 ? hc[1][1] : hc[2][1]);
    const int nl = k == 0 ? nlo[0] : (k == 1 ? nlo[1] : nlo[2]);
    const int nh = k == 0 ? nhi[0] : (k == 1 ? nhi[1] : nhi[2]);
    const double r0 = k == 0 ? R[0][0] : (k == 1 ? R[1][0] : R[2][0]);
    const double r1 = k == 0 ? R[0][1] : (k == 1 ? R[1][1] : R[2][1]);
    const double r2 = k == 0 ? R[0][2] : (k == 1 ? R[1][2] : R[2][2]);
    lo = proj3(r0, r1, r2, a0);
    hi = proj3(r0, r1, r2, b0);
    if (nl > 1) lo = fmin(lo, proj3(r0, r1, r2, a1));
    if (nh > 1) hi = fmax(hi, proj3(r0, r1, r2, b1));
  }
  // rare: more than two vertices at an extreme -> every vertex in FP64 (lanes over vertices)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (nlo[k] > 2 || nhi[k] > 2) {
      double l = DBL_MAX, h = -DBL_MAX;
      for (int v = v0 + lane; v < v1; v += 32) {
        const double tt = proj3(R[k][0], R[k][1], R[k][2], v);
        l = fmin(l, tt);
        h = fmax(h, tt);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        l = fmin(l, __shfl_xor_sync(full, l, o));
        h = fmax(h, __shfl_xor_sync(full, h, o));
      }
      if (lane == k) {
        lo = fmin(lo, l);
        hi = fmax(hi, h);
      }
    }
  }
  if (lane < 3) {
    const int k = lane;
    const double Xk = k == 0 ? Xv[0] : (k == 1 ? Xv[1] : Xv[2]);
    const double mn = dadd(Xk, lo), mx = dadd(Xk, hi);
    const double a = P.dx_pow2 ? dmul(mn, P.inv_dx) : __ddiv_rn(mn, P.dx);
    const double c = P.dx_pow2 ? dmul(mx, P.inv_dx) : __ddiv_rn(mx, P.dx);
    D.lohi[6 * p + k] = clamp_node(ceil(a));
    D.lohi[6 * p + 3 + k] = clamp_node(floor(c));
  }
  // world planes: face f on lane f (FP64 product per component, one rounding to FP32)
  const int f0 = S.face_off[p], f1 = S.face_off[p + 1];
  for (int f = f0 + lane; f < f1; f += 32) {
    const double2* e = reinterpret_cast<const double2*>(S.planes + 4 * f);
    const double2 e01 = e[0], e2x = e[1];
    float4 o;
    o.x = static_cast<float>(fma(R[0][0], e01.x, fma(R[0][1], e01.y, R[0][2] * e2x.x)));
    o.y = static_cast<float>(fma(R[1][0], e01.x, fma(R[1][1], e01.y, R[1][2] * e2x.x)));
    o.z = static_cast<float>(fma(R[2][0], e01.x, fma(R[2][1], e01.y, R[2][2] * e2x.x)));
    o.w = S.off32[f];
    D.wplane[f] = o;
  }
}

// K1b: one warp per polytope (node range and world planes), its own kernel so
// that the per-axis kernel's code stays as lean as it is without polytopes.
__global__ void k_pose_poly(Params P, Shapes S, Parts D, const double* __restrict__ pos, const double* __restrict__ quat) {
  pdl_begin();
  pose_polytope(P, S, D, S.poly_ids[blockIdx.x], pos, quat);
}

__global__ void k_pose(Params P, Shapes S, Parts D, Lists W, const double* __restrict__ pos,
                       const double* __restrict__ quat) {
  pdl_begin();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // the host's token of this step (mapped host memory: read here, stored at the end)
  const int token = (t == 0 && W.publish) ? *reinterpret_cast<const volatile int*>(W.err_host + 2) : 0;
  // the step's counters start at zero (the previous step has completed)
  if (t == 0) {
    W.counters[0] = 0;   // pairs (written by the pair builder)
    W.counters[1] = 0;   // tiles allocated
    W.counters[2] = 0;   // box pipeline queue head
    W.counters[5] = 0;   // pairs with V > 0
    W.u64[0] = 0;        // node evaluations
    W.u64[1] = 0;        // nominal lane-ops
  }
  if (t < (P.n + kRowGroup - 1) / kRowGroup) W.grp_sum[t] = 0;
  // contact history: this step's lists (the buffer not read) start empty
  if (P.history && t < P.n) W.hist_n[static_cast<size_t>(((W.counters[kStepCounter] & 1) ^ 1)) * P.n + t] = 0;
  if (t >= 3 * P.n) return;
  const int p = t / 3, k = t - 3 * p;
  double q[4];
  for (int c = 0; c < 4; ++c) q[c] = quat[4 * p + c];
  // position check by bit patterns: 0 <= X < L (NaN and negatives fail; -0.0 counts as 0)
  bool bad = false;
  float xs[3];
  double Xk = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double v = pos[3 * p + c];
    long long b = __double_as_longlong(v);
    if (b == static_cast<long long>(0x8000000000000000ULL)) b = 0;
    const bool ok = b >= 0 && b < __double_as_longlong(P.L[c]);
    bad = bad || !ok;
    const double vv = ok ? __longlong_as_double(b) : 0.0;
    xs[c] = static_cast<float>(vv);
    if (c == k) Xk = vv;
  }
  const double nn = dadd(dadd(dadd(dmul(q[0], q[0]), dmul(q[1], q[1])), dmul(q[2], q[2])), dmul(q[3], q[3]));
  if (!(nn > 1e-24) || !(nn < 1e300)) {
    bad = true;
    q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
  }
  if (bad && k == 0) set_error(W.err, kErrInval);
  const double s = bad ? 2.0 : dmul(2.0, __drcp_rn(nn));
  double r[3];
  rotation_row_rn(q, s, k, r);
  D.X[3 * p + k] = Xk;
  if (k == 0)
    for (int c = 0; c < 4; ++c) D.qhat[4 * p + c] = q[c];   // raw quaternion of the step (adjoint tape)
  for (int c = 0; c < 3; ++c) D.R[9 * p + 3 * k + c] = r[c];
  float r32[3];
  for (int c = 0; c < 3; ++c) {
    r32[c] = static_cast<float>(r[c]);
    D.Rt[9 * p + 3 * c + k] = r32[c];   // R^T row c, column k
  }
  // extent along k of the offset shape {phi <= delta} (explicit rounding: compared bit for bit)
  const int type = S.type[p];
  double mn, mx;
  if (type == 0) {
    const double rad = S.ext[3 * p];
    mn = dsub(Xk, rad);
    mx = dadd(Xk, rad);
  } else if (type == 1) {
    const double* e = S.ext + 3 * p;
    const double ext = dadd(dadd(dmul(fabs(r[0]), e[0]), dmul(fabs(r[1]), e[1])), dmul(fabs(r[2]), e[2]));
    mn = dsub(Xk, ext);
    mx = dadd(Xk, ext);
  } else {
    mn = mx = 0.0;   // polytope: node range and world planes by the polytope warps below
  }
  const double a = P.dx_pow2 ? dmul(mn, P.inv_dx) : __ddiv_rn(mn, P.dx);
  const double c = P.dx_pow2 ? dmul(mx, P.inv_dx) : __ddiv_rn(mx, P.dx);
  if (type != 2) {
    D.lohi[6 * p + k] = clamp_node(ceil(a));
    D.lohi[6 * p + 3 + k] = clamp_node(floor(c));
  }
  D.Xf[3 * p + k] = xs[k];
  const double xl = Xk * P.inv_dx;
  const double kx = rint(xl);
  D.kX[3 * p + k] = static_cast<int>(kx);
  D.fX[3 * p + k] = static_cast<float>(xl - kx);
  if (k == 0) {
    int b[3];
    for (int cc = 0; cc < 3; ++cc) b[cc] = min(max(static_cast<int>(xs[cc] * P.inv_binw_f[cc]), 0), P.nbin[cc] - 1);
    const int bin = checked_index(W.err, b[0] + P.nbin[0] * (b[1] + P.nbin[1] * b[2]),
                                  static_cast<long long>(P.nbin[0]) * P.nbin[1] * P.nbin[2], 0);
    D.bin[p] = bin;
    const int slot = atomicAdd(&W.bin_count[bin], 1);
    if (slot < P.bin_cap) W.bin_items[static_cast<size_t>(bin) * P.bin_cap + slot] = p;
    else set_error(W.err, kErrCapacity);
  }
  if (t == 0 && W.publish) W.counters[kTokenCounter] = token;
}

// Node box of pair (p, q) with q's image nearest p; returns false if empty.
// The image index s = rint((X_q - X_p) / L) is taken by comparing the FP32
// position difference with L/2 (positions lie in [0, L), so s is -1, 0 or 1).
// It can differ from the exact choice only when |X_q - X_p| is within FP32
// rounding of L/2; such a pair is no candidate in any image, because every
// image lies at least L/2 - 1e-3 > 2 R_max away on that axis (L > 4 R_max + 2 dx).
__device__ __forceinline__ bool pair_box(const Params& P, const Parts& D, int p, int q, int s[3], int lo[3],
                                         int hi[3]) {
  bool hit = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float d = D.Xf[3 * q + k] - D.Xf[3 * p + k];
    const float h = 0.5f * static_cast<float>(P.L[k]);
    s[k] = (d > h) ? 1 : ((d < -h) ? -1 : 0);
    lo[k] = max(D.lohi[6 * p + k], D.lohi[6 * q + k] - s[k] * P.ncell[k]);
    hi[k] = min(D.lohi[6 * p + 3 + k], D.lohi[6 * q + 3 + k] - s[k] * P.ncell[k]);
    hit = hit && lo[k] <= hi[k];
  }
  return hit;
}

// K3: one warp per particle p.  Lane b < 27 owns neighbour bin b of the
// fixed-capacity cell list; the candidates are read four per lane at a time
// (their particle data loaded together), tested against p's node range, and
// compacted with warp ballots into partners above (j > p) and below (j < p);
// each list is then sorted by rank.
__global__ void __launch_bounds__(256) k_broad(Params P, Parts D, Lists W) {
  extern __shared__ int s_buf[];
  // the block's partner count (its particles share one row group), added
  // to the group sum by the block's last warp to finish: one global atomic per block
  __shared__ int s_gsum, s_gdone;
  if (threadIdx.x == 0) {
    s_gsum = 0;
    s_gdone = 0;
  }
  __syncthreads();
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = blockIdx.x * (blockDim.x >> 5) + wid;
  const int nw = static_cast<int>(blockDim.x >> 5);
  auto group_sum = [&](int nup) {
    if (lane == 0) {
      if (nup > 0) atomicAdd_block(&s_gsum, nup);
      __threadfence_block();
      if (atomicAdd_block(&s_gdone, 1) == nw - 1) {   // every warp's count is in
        __threadfence_block();
        const int tot = atomicAdd_block(&s_gsum, 0);
        if (tot > 0) atomicAdd(&W.grp_sum[(blockIdx.x * nw) / kRowGroup], tot);
      }
    }
  };
  if (p >= P.n) {
    group_sum(0);
    return;
  }
  const int cap = P.max_nbr;
  int* up = s_buf + wid * 2 * cap;
  int* dn = up + cap;
  const int bin = D.bin[p];
  float xp[3];
  int plo[3], phi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xp[k] = D.Xf[3 * p + k];
    plo[k] = D.lohi[6 * p + k];
    phi[k] = D.lohi[6 * p + 3 + k];
  }
  const int b[3] = {bin % P.nbin[0], (bin / P.nbin[0]) % P.nbin[1], bin / (P.nbin[0] * P.nbin[1])};
  int cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) cnt[k] = P.nbin[k] >= 3 ? 3 : P.nbin[k];
  const int nnb = cnt[0] * cnt[1] * cnt[2];
  int num = 0;
  const int* items = W.bin_items;
  int pre[4] = {-1, -1, -1, -1};   // the bin's next four entries (the first ones fetched with its count)
  if (lane < nnb) {
    int o[3] = {lane % cnt[0], (lane / cnt[0]) % cnt[1], lane / (cnt[0] * cnt[1])};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = P.nbin[k] >= 3 ? b[k] + o[k] - 1 : o[k];
      o[k] = (c + P.nbin[k]) % P.nbin[k];
    }
    const int q = checked_index(W.err, o[0] + P.nbin[0] * (o[1] + P.nbin[1] * o[2]),
                                static_cast<long long>(P.nbin[0]) * P.nbin[1] * P.nbin[2], bin);
    items += static_cast<size_t>(q) * P.bin_cap;
    // (entries past the count are stale and unused)
#pragma unroll
    for (int u = 0; u < 4; ++u) pre[u] = u < P.bin_cap ? items[u] : -1;
    num = min(W.bin_count[q], P.bin_cap);
  }
  const int maxn = __reduce_max_sync(kFull, num);
  int nup = 0, ndn = 0;
  const unsigned below = (1u << lane) - 1u;
  for (int t0 = 0; t0 < maxn; t0 += 4) {
    int jj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) jj[u] = t0 + u < num ? checked_index(W.err, pre[u], P.n, -1) : -1;
    // the next four entries, fetched with this round's candidate data
#pragma unroll
    for (int u = 0; u < 4; ++u) pre[u] = t0 + 4 + u < num ? items[t0 + 4 + u] : -1;
    float xj[4][3];
    int jlo[4][3], jhi[4][3];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jj[u] >= 0 ? jj[u] : p;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        xj[u][k] = D.Xf[3 * j + k];
        jlo[u][k] = D.lohi[6 * j + k];
        jhi[u][k] = D.lohi[6 * j + 3 + k];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jj[u];
      // node ranges intersect, the partner moved by the image shift (as in pair_box)
      bool hit = j >= 0 && j != p;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float d = xj[u][k] - xp[k];
        const float h = 0.5f * static_cast<float>(P.L[k]);
        const int sk = (d > h) ? 1 : ((d < -h) ? -1 : 0);
        const int lo = max(plo[k], jlo[u][k] - sk * P.ncell[k]);
        const int hi = min(phi[k], jhi[u][k] - sk * P.ncell[k]);
        hit = hit && lo <= hi;
      }
      const unsigned bu = __ballot_sync(kFull, hit && j > p);
      const unsigned bd = __ballot_sync(kFull, hit && j < p);
      if (hit && j > p) {
        const int at = nup + __popc(bu & below);
        if (at < cap) up[at] = j;
      }
      if (hit && j < p) {
        const int at = ndn + __popc(bd & below);
        if (at < cap) dn[at] = j;
      }
      nup += __popc(bu);
      ndn += __popc(bd);
    }
  }
  // walls (partners n + w, after every particle): lane w tests wall w with an
  // FP32 prefilter, then exactly in FP64 (the node box must be non-empty)
  for (int w0 = 0; w0 < P.nwall; w0 += 32) {
    const int w = w0 + lane;
    bool hit = false;
    if (w < P.nwall) {
      const double* e = P.wall + 4 * w;
      const float m0 = static_cast<float>(e[0]), m1 = static_cast<float>(e[1]), m2 = static_cast<float>(e[2]);
      const float dxf = static_cast<float>(P.dx);
      const float t0 = m0 * static_cast<float>(m0 > 0.f ? plo[0] : phi[0]);
      const float t1 = m1 * static_cast<float>(m1 > 0.f ? plo[1] : phi[1]);
      const float t2 = m2 * static_cast<float>(m2 > 0.f ? plo[2] : phi[2]);
      const float lowest = (t0 + t1 + t2) * dxf;
      const float H = static_cast<float>(e[3] + P.delta);
      // the FP32 error of `lowest` is below 1e-6 of its terms' magnitudes:
      // walls beyond 1e-4 of them skip the exact FP64 test
      const float mag = (fabsf(t0) + fabsf(t1) + fabsf(t2)) * dxf + fabsf(H) + dxf;
      if (lowest <= H + 1e-4f * mag) {
        int lo[3], hi[3];
        hit = wall_box(e, P.delta, P.dx, plo, phi, lo, hi);
      }
    }
    const unsigned bw = __ballot_sync(kFull, hit);
    if (hit) {
      const int at = nup + __popc(bw & below);
      if (at < cap) up[at] = P.n + w;
    }
    nup += __popc(bw);
  }
  if (nup > cap || ndn > cap) {
    if (lane == 0) set_error(W.err, kErrCapacity);
    nup = min(nup, cap);
    ndn = min(ndn, cap);
  }
  __syncwarp();
  // rank sort (lists are short and keys unique)
  for (int e = lane; e < nup; e += 32) {
    const int v = up[e];
    int r = 0;
    for (int t = 0; t < nup; ++t) r += up[t] < v;
    W.up_list[p * cap + r] = v;
  }
  for (int e = lane; e < ndn; e += 32) {
    const int v = dn[e];
    int r = 0;
    for (int t = 0; t < ndn; ++t) r += dn[t] < v;
    W.dn_list[p * cap + r] = v;
  }
  if (lane == 0) {
    W.up_count[p] = nup;
    W.dn_count[p] = ndn;
  }
  group_sum(nup);
}


// K4: one warp per particle row i, one lane per partner slot r: the pair
// record of pair row_off[i] + r, its sweep layout and its node tiles.  Tiles
// are allocated with one atomic per warp round; a pair's tiles are
// contiguous, and its partial sums do not depend on where they land, so the
// results are deterministic.  No FP64: centres come as integer node + FP32
// remainder from the pose kernel.
constexpr int kBuildWarps = 8;   // particle rows per block of the pair builder

// Store a pair record (with its tile index) as fourteen 16-byte stores from
// registers, field by field (an aggregate copy would stage it in local memory).
__device__ __forceinline__ void store_pair_rec(PairRec* dst, const PairRec& r, int tile) {
  int4* d = reinterpret_cast<int4*>(dst);
  const auto f = [](float x) { return __float_as_int(x); };
  d[0] = make_int4(r.i, r.j, r.lo[0], r.lo[1]);
  d[1] = make_int4(r.lo[2], r.dim[0], r.dim[1], r.dim[2]);
  d[2] = make_int4(r.shift[0], r.shift[1], r.shift[2], r.axis);
  d[3] = make_int4(r.seglen, r.nseg, r.nitems, r.tile0);
  d[4] = make_int4(r.ntiles, r.kinds, r.ai[0], r.ai[1]);
  d[5] = make_int4(r.ai[2], r.bi[0], r.bi[1], r.bi[2]);
  d[6] = make_int4(f(r.af[0]), f(r.af[1]), f(r.af[2]), f(r.bf[0]));
  d[7] = make_int4(f(r.bf[1]), f(r.bf[2]), f(r.rta[0]), f(r.rta[1]));
  d[8] = make_int4(f(r.rta[2]), f(r.rta[3]), f(r.rta[4]), f(r.rta[5]));
  d[9] = make_int4(f(r.rta[6]), f(r.rta[7]), f(r.rta[8]), f(r.rtb[0]));
  d[10] = make_int4(f(r.rtb[1]), f(r.rtb[2]), f(r.rtb[3]), f(r.rtb[4]));
  d[11] = make_int4(f(r.rtb[5]), f(r.rtb[6]), f(r.rtb[7]), f(r.rtb[8]));
  d[12] = make_int4(f(r.sza[0]), f(r.sza[1]), f(r.sza[2]), f(r.szb[0]));
  d[13] = make_int4(f(r.szb[1]), f(r.szb[2]), tile, r.pair);
}
static_assert(offsetof(PairRec, rta) == 30 * 4 && offsetof(PairRec, szb) == 51 * 4 &&
                  offsetof(PairRec, pair) == 55 * 4 && sizeof(PairRec) == 14 * 16,
              "store_pair_rec follows the PairRec layout");

// Whether the regions {phi_A < Ta} and {phi_B < Tb} of the pair are
// disjoint (by more than kCullMargin cells).  A node adds to the node sweep's
// sums only when both distances lie below w/2 and, with the sharp indicator,
// one of them is <= 0; so with T = w/2 (+ the clip margin) a pair apart for
// (T, T) (smoothed), or for both (0, T) and (T, 0) (sharp), has zero
// outputs and is not queued.  Spheres, cubes, cuboids and polytopes (their
// regions are balls and boxes of half extents size + T; a polytope is bounded
// by a ball, its circumradius at each threshold from the shape tables):
// box-box by the 15 separating axes (faces of either box, edge cross
// products), ball-box by the box's closest point, ball-ball by the centre
// distance; walls are never skipped.  FP32 in lattice units: the centres
// differ by an exact integer plus the FP32 difference of two remainders, and
// every rounding is far below the margin.
constexpr float kCullMargin = 1e-3f;

__device__ __forceinline__ float dot3(const float* a, const float* b) { return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2])); }

// The three threshold pairs of the test, from one set of projections: bit 0
// (T, T), bit 1 (0, T), bit 2 (T, 0) set when the regions are apart.  On an
// axis the reach of a box's region is R0 + T S (R0 its reach at 0, S the sum
// of its axes' projections), of a ball r + T or its tabulated radius.
struct Apart {
  unsigned bits = 0;
  __device__ __forceinline__ void axis(float proj, float ra0, float sa, float rb0, float sb, float T) {
    const float base = proj - kCullMargin - ra0 - rb0;
    bits |= (base > T * (sa + sb) ? 1u : 0u) | (base > T * sb ? 2u : 0u) | (base > T * sa ? 4u : 0u);
  }
};

__device__ unsigned pair_apart(const PairRec& r, float T) {
  const int ka = r.kinds & 0xff, kb = r.kinds >> 8;
  const bool pa = ka == KIND_POLY, pb = kb == KIND_POLY;
  const bool sa = ka == KIND_SPHERE || pa, sb = kb == KIND_SPHERE || pb;   // balls
  const bool ba = ka == KIND_CUBOID || ka == KIND_CUBE, bb = kb == KIND_CUBOID || kb == KIND_CUBE;
  if (!((sa || ba) && (sb || bb))) return 0u;
  float d[3];   // centre of B minus centre of A (lattice units)
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = static_cast<float>(r.bi[k] - r.ai[k]) + (r.bf[k] - r.af[k]);
  Apart ap;
  if (sa && sb) {
    // ball radii at 0 and at T: a sphere's r and r + T, a polytope's two tabulated radii
    const float a0 = r.sza[0], aT = pa ? r.sza[1] : r.sza[0] + T;
    const float b0 = r.szb[0], bT = pb ? r.szb[1] : r.szb[0] + T;
    const float dist = sqrtf(dot3(d, d));
    ap.axis(dist, a0, (aT - a0) / T, b0, (bT - b0) / T, T);
    return ap.bits;
  }
  if (sa || sb) {   // a ball and a box: the distance from the ball's centre to the box at each threshold
    // (element-wise selects: a runtime-chosen pointer into the record would put it in local memory)
    const bool pol = sa ? pa : pb;
    const float r0 = sa ? r.sza[0] : r.szb[0];
    const float rT = pol ? (sa ? r.sza[1] : r.szb[1]) : r0 + T;
    float y[3], sz[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {   // |ball centre - box centre| in the box frame
      const float t0 = sa ? r.rtb[3 * k] : r.rta[3 * k], t1 = sa ? r.rtb[3 * k + 1] : r.rta[3 * k + 1],
                  t2 = sa ? r.rtb[3 * k + 2] : r.rta[3 * k + 2];
      y[k] = fabsf(fmaf(t0, d[0], fmaf(t1, d[1], t2 * d[2])));
      sz[k] = sa ? r.szb[k] : r.sza[k];
    }
    // the box at 0 and at T, the ball at 0 and at T: bits as (A, B) thresholds
    float dist[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      float d2 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float o = fmaxf(y[k] - (sz[k] + (t ? T : 0.f)), 0.f);
        d2 = fmaf(o, o, d2);
      }
      dist[t] = sqrtf(d2) - kCullMargin;
    }
    // (T, T): box T, ball T; (0, T) and (T, 0) with the ball on side A or B
    const bool tt = dist[1] > rT, box0_ballT = dist[0] > rT, boxT_ball0 = dist[1] > r0;
    ap.bits = (tt ? 1u : 0u) | ((sa ? boxT_ball0 : box0_ballT) ? 2u : 0u) | ((sa ? box0_ballT : boxT_ball0) ? 4u : 0u);
    return ap.bits;
  }
  // two boxes: R[i][j] = a_i . b_j, t = d in A's frame; 15 axes
  float R[3][3], AR[3][3], t[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    t[i] = dot3(r.rta + 3 * i, d);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R[i][j] = dot3(r.rta + 3 * i, r.rtb + 3 * j);
      AR[i][j] = fabsf(R[i][j]) + 1e-6f;
    }
  }
  const float ea[3] = {r.sza[0], r.sza[1], r.sza[2]}, eb[3] = {r.szb[0], r.szb[1], r.szb[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i) {   // A's faces
    const float sbi = AR[i][0] + AR[i][1] + AR[i][2];
    ap.axis(fabsf(t[i]), ea[i], 1.f, fmaf(eb[0], AR[i][0], fmaf(eb[1], AR[i][1], eb[2] * AR[i][2])), sbi, T);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {   // B's faces
    const float tb = fmaf(t[0], R[0][j], fmaf(t[1], R[1][j], t[2] * R[2][j]));
    const float saj = AR[0][j] + AR[1][j] + AR[2][j];
    ap.axis(fabsf(tb), fmaf(ea[0], AR[0][j], fmaf(ea[1], AR[1][j], ea[2] * AR[2][j])), saj, eb[j], 1.f, T);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {   // edge pairs a_i x b_j
    const int i1 = i == 2 ? 0 : i + 1, i2 = i1 == 2 ? 0 : i1 + 1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = j == 2 ? 0 : j + 1, j2 = j1 == 2 ? 0 : j1 + 1;
      const float ra0 = fmaf(ea[i1], AR[i2][j], ea[i2] * AR[i1][j]);
      const float rb0 = fmaf(eb[j1], AR[i][j2], eb[j2] * AR[i][j1]);
      ap.axis(fabsf(fmaf(t[i2], R[i1][j], -t[i1] * R[i2][j])), ra0, AR[i2][j] + AR[i1][j], rb0,
              AR[i][j2] + AR[i][j1], T);
    }
  }
  return ap.bits;
}

// The node range of a pair of boxes (cubes, cuboids) where both distances lie
// below T (the box pipeline's rough-detection threshold).  A node outside
// {phi_A < T} or {phi_B < T} is no rough-contact node, so the pair's node box
// shrinks to the bounding box of the intersection of the two boxes grown by T
// (half extents size + T).  The vertices of that intersection are end points
// of the edges of either box clipped to the other one, so lane e < 24 clips
// edge e (A's twelve, then B's) to the other box, grown by kCutSlack more, and
// the bounds of the end points, widened by kCutSlack, are reduced over the
// warp.  FP32 in box-relative lattice units: the rounding (~1e-5 cells) stays
// far inside the slack, so every node with both distances below T is kept.
// The whole warp calls this with the record in shared memory; false: the
// intersection is empty.
constexpr float kCutSlack = 1e-2f;

__device__ __forceinline__ bool cut_box(const PairRec& sr, float T, int nlo[3], int nhi[3]) {
  const int lane = threadIdx.x & 31;
  const bool onb = lane >= 12;
  const int q = onb ? lane - 12 : lane;
  const int m = min(q >> 2, 2), m1 = m == 2 ? 0 : m + 1, m2 = m1 == 2 ? 0 : m1 + 1;
  const float s1 = (q & 1) ? 1.f : -1.f, s2 = (q & 2) ? 1.f : -1.f;
  const float* ro = onb ? sr.rtb : sr.rta;   // the edge's box: body axis k = row k
  const float* rx = onb ? sr.rta : sr.rtb;   // the other box
  const float* eo = onb ? sr.szb : sr.sza;
  const float* ex = onb ? sr.sza : sr.szb;
  const int* io = onb ? sr.bi : sr.ai;
  const int* ix = onb ? sr.ai : sr.bi;
  const float* fo = onb ? sr.bf : sr.af;
  const float* fx = onb ? sr.af : sr.bf;
  const float e0 = eo[m] + T, e1 = eo[m1] + T, e2 = eo[m2] + T;
  // edge p0 + t dv, t in [-1, 1]; rel = p0 minus the other box's centre
  float p0[3], dv[3], rel[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float co = static_cast<float>(io[c]) + fo[c], cx = static_cast<float>(ix[c]) + fx[c];
    p0[c] = fmaf(s2 * e2, ro[3 * m2 + c], fmaf(s1 * e1, ro[3 * m1 + c], co));
    dv[c] = e0 * ro[3 * m + c];
    rel[c] = p0[c] - cx;
  }
  float t0 = -1.f, t1 = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float base = dot3(rx + 3 * k, rel), sl = dot3(rx + 3 * k, dv);
    const float E = ex[k] + T + kCutSlack;
    if (fabsf(sl) > 1e-6f) {
      const float is = __fdividef(1.f, sl);
      const float a = (-E - base) * is, b = (E - base) * is;
      t0 = fmaxf(t0, fminf(a, b));
      t1 = fminf(t1, fmaxf(a, b));
    } else if (!(fabsf(base) <= E)) {
      t1 = -2.f;
    }
  }
  const bool ok = lane < 24 && t0 <= t1;
  bool any = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float a = t0 * dv[c], b = t1 * dv[c];
    const int lo = ok ? static_cast<int>(ceilf(p0[c] + fminf(a, b) - kCutSlack)) : 0x7fffffff;
    const int hi = ok ? static_cast<int>(floorf(p0[c] + fmaxf(a, b) + kCutSlack)) : -0x7fffffff;
    nlo[c] = __reduce_min_sync(kFull, lo);
    nhi[c] = __reduce_max_sync(kFull, hi);
    any = any && nlo[c] <= nhi[c];
  }
  return any;
}

// BOXM: the box pipeline's variant (its separation test at the rough threshold,
// the cut node boxes of two boxes, one list entry per kept pair).
template <bool BOXM>
__global__ void __launch_bounds__(kBuildWarps * 32) k_build_pairs(Params P, Shapes S, Parts D, Lists W,
                                                                  int32_t* __restrict__ pair_ij,
                                                                  int32_t* __restrict__ n_pairs_out,
                                                                  double* __restrict__ pair_out) {
  // per warp: tiles (exclusive prefix after the block scan)
  __shared__ int s_w[kBuildWarps];
  __shared__ int s_base;
  __shared__ unsigned long long s_u64[kBuildWarps][2];
  __shared__ __align__(16) PairRec s_pr[BOXM ? kBuildWarps : 1];   // a record being cut (cut_box)
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kBuildWarps + wid;
  const bool row_ok = i0 < P.n;
  const int i = row_ok ? i0 : P.n - 1;   // rows past the end take part in the block's barriers only
  const int cap = P.max_nbr;
  // first pair of row i: the group sums before i's group plus the counts of
  // the earlier particles of its group (both sets of loads in flight at once)
  const int g = i / kRowGroup;
  int acc = 0;
  for (int base = 0; base < g; base += 8 * 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + 32 * u + lane;
      acc += e < g ? W.grp_sum[e] : 0;
    }
  }
#pragma unroll
  for (int u = 0; u < kRowGroup / 32; ++u) {
    const int e = g * kRowGroup + 32 * u + lane;
    acc += e < i ? W.up_count[e] : 0;
  }
  const int cnt = row_ok ? W.up_count[i] : 0;
  // the first 32 partners, fetched before the count is known (stale beyond it, unused)
  const int jpre = lane < cap ? W.up_list[static_cast<size_t>(i) * cap + lane] : 0;
  const int row = __reduce_add_sync(kFull, acc);
  if (lane == 0 && row_ok) {
    W.row_off[i] = row;
    if (i == P.n - 1) {   // the pair count: the last row's offset plus its partners
      const int total = row + cnt;
      W.counters[0] = total;
      W.row_off[P.n] = total;
      *n_pairs_out = total;
      if (total > P.max_pairs) set_error(W.err, kErrCapacity);
    }
  }
  for (int base = 0; __syncthreads_or(base < cnt); base += 32) {   // block-uniform rounds of 32 partners
    const int r = base + lane;
    const bool active = r < cnt && (row + r) < P.max_pairs;
    PairRec pr;
    int pi = 0, ntiles = 0;
    bool skip = false, cut = false;
    unsigned long long vol = 0, ops = 0;
    if (active) {
      pi = row + r;
      const int j = checked_index(W.err, base == 0 ? jpre : W.up_list[static_cast<size_t>(i) * cap + r],
                                  P.n + P.nwall, i);
      // j's lower-partner list, fetched with j's particle data (slot of this pair below);
      // a wall (j >= n) has none
      const bool wall = j >= P.n;
      const int* dl = W.dn_list + static_cast<size_t>(wall ? 0 : j) * cap;
      const int dc = wall ? 0 : checked_index(W.err, W.dn_count[j], cap + 1, 0);
      int dpre[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) dpre[u] = u < cap ? dl[u] : 0;
      int lo[3], hi[3];
      int shift[3] = {0, 0, 0};
      if (wall) {
        int plo[3], phi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          plo[k] = D.lohi[6 * i + k];
          phi[k] = D.lohi[6 * i + 3 + k];
        }
        wall_box(P.wall + 4 * (j - P.n), P.delta, P.dx, plo, phi, lo, hi);   // non-empty (tested by the broad phase)
      } else {
        pair_box(P, D, i, j, shift, lo, hi);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) pr.shift[k] = shift[k];
      pr.i = i;
      pr.j = j;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        pr.lo[k] = lo[k];
        pr.dim[k] = hi[k] - lo[k] + 1;
      }
      // the candidate box's nodes (the cell evaluations and nominal lane-ops
      // of the step), whatever the node sweep later skips
      const long long volp = static_cast<long long>(pr.dim[0]) * pr.dim[1] * pr.dim[2];
      pr.kinds = W.kind[i] | (W.kind[j] << 8);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // X_i / dx - lo and X_j' / dx - lo = (X_j / dx - s n) - lo
        pr.ai[k] = D.kX[3 * i + k] - lo[k];
        pr.af[k] = D.fX[3 * i + k];
        pr.bi[k] = D.kX[3 * j + k] - pr.shift[k] * P.ncell[k] - lo[k];
        pr.bf[k] = D.fX[3 * j + k];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        pr.rta[k] = D.Rt[9 * i + k];
        pr.rtb[k] = D.Rt[9 * j + k];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        pr.sza[k] = S.size_l[3 * i + k];
        pr.szb[k] = S.size_l[3 * j + k];
      }
      if (wall) {   // the wall's value at the box origin, m . lo - (h + inflate) / dx (lattice
                    // units), and its origin at the box origin (node offsets are box-relative)
        const double* e = P.wall + 4 * (j - P.n);
        const double p0 = ((e[0] * lo[0] + e[1] * lo[1]) + e[2] * lo[2]) - (e[3] + P.inflate) * P.inv_dx;
        pr.szb[0] = static_cast<float>(p0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          pr.bi[k] = 0;
          pr.bf[k] = 0.f;
        }
      }
      // the FP32 node sweep skips pairs whose distance regions are apart, and
      // so does the box pipeline (regions at its rough-detection threshold;
      // a polytope's tabulated radii belong to the node sweep's threshold, so
      // pairs with one are kept there); the skipped pairs' zero outputs are
      // written below.  In the box pipeline two boxes' node box is also cut to
      // their regions' intersection (after the record is complete).
      const int ka = pr.kinds & 0xff, kb = pr.kinds >> 8;
      constexpr bool boxm = BOXM;
      const bool test = (P.precision == 0 && !boxm) || (boxm && ka != KIND_POLY && kb != KIND_POLY);
      const unsigned apart = test ? pair_apart(pr, boxm ? kRoughT : 0.5f * P.wdx_l + kClipMargin) : 0u;
      skip = (P.smooth || boxm) ? (apart & 1u) != 0u : (apart & 6u) == 6u;
      cut = boxm && !skip && (ka == KIND_CUBE || ka == KIND_CUBOID) && (kb == KIND_CUBE || kb == KIND_CUBOID);
      pr.tile = 0;
      pr.pair = pi;
      W.pdone[pi] = 0;
      vol = static_cast<unsigned long long>(volp);
      ops = vol * static_cast<unsigned long long>(S.nomops[i] + S.nomops[j]);
      pair_ij[2 * pi] = i;
      pair_ij[2 * pi + 1] = j;
      // slot of this pair in j's (sorted) list of lower partners: the number of entries below i
      int a0 = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) a0 += (u < dc && dpre[u] < i) ? 1 : 0;
      for (int b = 8; b < dc; ++b) a0 += dl[b] < i ? 1 : 0;
      if (!wall) W.dn_pair[static_cast<size_t>(j) * cap + checked_index(W.err, a0, cap, 0)] = pi;
    }
    // the box pipeline's cut node boxes, one pair at a time for the whole
    // warp (the record passes through shared memory); the box, the centres'
    // integer parts and nothing else change, so every node keeps its FP32
    // distances
    for (unsigned todo = BOXM ? __ballot_sync(kFull, cut) : 0u; todo != 0u; todo &= todo - 1u) {
      const int src = __ffs(todo) - 1;
      if (lane == src) store_pair_rec(&s_pr[wid], pr, 0);
      __syncwarp();
      int nlo[3], nhi[3];
      const bool any = cut_box(s_pr[wid], kRoughT, nlo, nhi);
      if (lane == src) {
        int a[3], b[3];
        bool keep = any;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a[k] = max(nlo[k], 0);
          b[k] = min(nhi[k], pr.dim[k] - 1);
          keep = keep && a[k] <= b[k];
        }
        if (keep) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            pr.lo[k] += a[k];
            pr.dim[k] = b[k] - a[k] + 1;
            pr.ai[k] -= a[k];
            pr.bi[k] -= a[k];
          }
        } else {
          skip = true;   // no rough-contact node: zero outputs
        }
      }
      __syncwarp();
    }
    if (active) {
      // sweep layout: whole node lines along the box's longest axis (the
      // fewest lines).  The node sweeps clip every line to the few nodes near
      // both surfaces, so a line costs about the same whatever its length
      // (selects, not a runtime index into pr.dim: that would put pr in local memory).
      const int lines_of[3] = {pr.dim[1] * pr.dim[2], pr.dim[0] * pr.dim[2], pr.dim[0] * pr.dim[1]};
      {
        const int a = pr.dim[1] > pr.dim[0] ? (pr.dim[2] > pr.dim[1] ? 2 : 1) : (pr.dim[2] > pr.dim[0] ? 2 : 0);
        pr.axis = a;
        pr.nseg = 1;
        pr.seglen = a == 0 ? pr.dim[0] : (a == 1 ? pr.dim[1] : pr.dim[2]);
      }
      pr.nitems = pr.axis == 0 ? lines_of[0] : (pr.axis == 1 ? lines_of[1] : lines_of[2]);
      // the box pipeline takes each kept pair as one entry of the tile list
      ntiles = skip ? 0 : (BOXM ? 1 : (pr.nitems + 32 * kTileItemsPerLane - 1) / (32 * kTileItemsPerLane));
      pr.ntiles = ntiles;
      // a skipped pair's outputs, as the node sweep or the box pipeline would write them (zeros)
      if (skip) {
        double* po = pair_out + static_cast<size_t>(pi) * 11;
        double* pf = W.ft + static_cast<size_t>(pi) * kFtDoubles;
        double* pt = W.tape + static_cast<size_t>(pi) * kTapeDoubles;
#pragma unroll
        for (int k = 0; k < 11; ++k) po[k] = 0.0;
#pragma unroll
        for (int k = 0; k < kFtDoubles; ++k) pf[k] = 0.0;
#pragma unroll
        for (int k = 0; k < kTapeDoubles; ++k) pt[k] = 0.0;
        W.oflag[pi] = 0;
      }
    }
    // allocations aggregated over the block (one atomic per counter and
    // block, all in flight together): the pairs' tiles, contiguous per pair;
    // tile k of a pair is entry tile0 + k of the node sweep's tile list
    int incl = ntiles;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += v;
    }
    unsigned long long wv = vol, wo = ops;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      wv += __shfl_xor_sync(kFull, wv, d);
      wo += __shfl_xor_sync(kFull, wo, d);
    }
    const int wtiles = __shfl_sync(kFull, incl, 31);
    if (lane == 0) {
      s_w[wid] = wtiles;
      s_u64[wid][0] = wv;
      s_u64[wid][1] = wo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive prefix over the warps, one atomic
      int run = 0;
      for (int w = 0; w < kBuildWarps; ++w) {
        const int v = s_w[w];
        s_w[w] = run;
        run += v;
      }
      s_base = run > 0 ? atomicAdd(&W.counters[1], run) : 0;
    } else if (threadIdx.x == 32) {
      unsigned long long a = 0, b = 0;
      for (int w = 0; w < kBuildWarps; ++w) { a += s_u64[w][0]; b += s_u64[w][1]; }
      if (a > 0) {
        atomicAdd(&W.u64[0], a);
        atomicAdd(&W.u64[1], b);
      }
    }
    __syncthreads();
    const int tbase = s_base + s_w[wid];
    if (active) {
      pr.tile0 = tbase + incl - ntiles;
      store_pair_rec(W.pairs + pi, pr, 0);
      // the tile records (beyond the tile capacity the step fails with
      // ECAPACITY and the node sweep does not run)
      for (int k = 0; k < ntiles; ++k) {
        if (pr.tile0 + k < P.max_tiles) {
          W.tile_pair[pr.tile0 + k] = pi;
          store_pair_rec(W.tiles + pr.tile0 + k, pr, k);
        } else {
          set_error(W.err, kErrCapacity);
        }
      }
    }
  }
}

}  // namespace

void launch_pose(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* pos,
                 const double* quat, cudaStream_t st) {
  // one-warp blocks: the FP64 chains of different warps land on different sub-partitions
  // (then one block per polytope for its vertices and faces)
  const int nb = (3 * P.n + 31) / 32;
  if (nb > 0) launch_pdl(k_pose, dim3(nb), dim3(32), 0, st, P, S, D, W, pos, quat);
  if (P.npoly > 0) launch_pdl(k_pose_poly, dim3(P.npoly), dim3(32), 0, st, P, S, D, pos, quat);
}


void launch_broad(const Params& P, const Parts& D, const Lists& W, cudaStream_t st) {
  const int warps = 8;
  const int nb = (P.n + warps - 1) / warps;
  const size_t smem = static_cast<size_t>(warps) * 2 * P.max_nbr * sizeof(int);
  if (nb > 0) launch_pdl(k_broad, dim3(nb), dim3(warps * 32), smem, st, P, D, W);
}

void launch_plan(const Params& P, const Shapes& S, const Parts& D, const Lists& W, int32_t* pair_ij, int32_t* n_pairs,
                 double* pair_out, cudaStream_t st) {
  const int nb = (P.n + kBuildWarps - 1) / kBuildWarps;   // one particle row per warp
  launch_pdl(P.box_mode == 1 ? k_build_pairs<true> : k_build_pairs<false>, dim3(nb > 0 ? nb : 1),
             dim3(kBuildWarps * 32), 0, st, P, S, D, W, pair_ij, n_pairs, pair_out);
}

}  // namespace gbc
