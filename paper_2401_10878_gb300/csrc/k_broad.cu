// Pose -> AABB, cell-list broad phase and pair planning of the contact step.
//
// Paper (arXiv:2401.10878): Sec. 3.3.1 (a contact is swept over the region
// where both particles may overlap), Sec. 3.3.2 (periodic boundaries: the
// higher-ID particle is moved to the side of the lower-ID one), Sec. 4.1
// (the neighbourhood radius is the largest circumradius).
#include <cfloat>

#include "contact_dev.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int clamp_node(double v) {
  // node indices stay far inside int range even for garbage input
  v = fmin(fmax(v, -1.0e9), 1.0e9);
  return static_cast<int>(v);
}

// ---------------------------------------------------------------------------
// K1: per particle rotation, node ranges, FP32 sweep geometry and bin slot.
__global__ void k_pose(Params P, Shapes S, Parts D, Lists W, const double* __restrict__ pos,
                       const double* __restrict__ quat) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.n) return;
  double X[3], q[4];
  bool bad = false;
  for (int k = 0; k < 3; ++k) {
    X[k] = pos[3 * p + k];
    if (!(X[k] >= 0.0) || !(X[k] < P.L[k])) {  // also catches NaN
      bad = true;
      X[k] = 0.0;
    }
  }
  for (int k = 0; k < 4; ++k) q[k] = quat[4 * p + k];
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  if (!(qq > 1e-24) || !(qq < 1e300)) {
    bad = true;
    q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
  }
  if (bad) set_error(W.err, kErrInval);
  double qh[4], qn, R[9];
  rotation_rn(q, qh, &qn, R);
  for (int k = 0; k < 3; ++k) D.X[3 * p + k] = X[k];
  for (int k = 0; k < 4; ++k) D.qhat[4 * p + k] = qh[k];
  D.qnorm[p] = qn;
  for (int k = 0; k < 9; ++k) D.R[9 * p + k] = R[k];

  // AABB of the offset shape {phi <= delta} (explicit rounding: compared bit for bit)
  const int type = S.type[p];
  const double* prm = S.param + 3 * p;
  double mn[3], mx[3];
  if (type == 0) {
    const double rad = dadd(prm[0], P.delta);
    for (int k = 0; k < 3; ++k) { mn[k] = dsub(X[k], rad); mx[k] = dadd(X[k], rad); }
  } else if (type == 1) {
    const double e0 = dadd(prm[0], P.delta), e1 = dadd(prm[1], P.delta), e2 = dadd(prm[2], P.delta);
    for (int k = 0; k < 3; ++k) {
      const double ext = dadd(dadd(dmul(fabs(R[3 * k]), e0), dmul(fabs(R[3 * k + 1]), e1)),
                              dmul(fabs(R[3 * k + 2]), e2));
      mn[k] = dsub(X[k], ext);
      mx[k] = dadd(X[k], ext);
    }
  } else {
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int v = S.vert_off[p]; v < S.vert_off[p + 1]; ++v) {
      const double* w = S.verts + 3 * v;
      for (int k = 0; k < 3; ++k) {
        const double t = dadd(dadd(dmul(R[3 * k], w[0]), dmul(R[3 * k + 1], w[1])), dmul(R[3 * k + 2], w[2]));
        lo[k] = fmin(lo[k], t);
        hi[k] = fmax(hi[k], t);
      }
    }
    for (int k = 0; k < 3; ++k) { mn[k] = dadd(X[k], lo[k]); mx[k] = dadd(X[k], hi[k]); }
  }
  int b[3];
  for (int k = 0; k < 3; ++k) {
    // x / dx, exactly as an IEEE division (a multiply when dx is a power of two)
    const double a = P.dx_pow2 ? dmul(mn[k], P.inv_dx) : __ddiv_rn(mn[k], P.dx);
    const double c = P.dx_pow2 ? dmul(mx[k], P.inv_dx) : __ddiv_rn(mx[k], P.dx);
    D.lohi[6 * p + k] = clamp_node(ceil(a));
    D.lohi[6 * p + 3 + k] = clamp_node(floor(c));
    const float xf = static_cast<float>(X[k]);
    D.Xf[3 * p + k] = xf;
    b[k] = min(max(static_cast<int>(xf * P.inv_binw_f[k]), 0), P.nbin[k] - 1);
    const double xl = X[k] * P.inv_dx;
    const double kx = rint(xl);
    D.kX[3 * p + k] = static_cast<int>(kx);
    D.fX[3 * p + k] = static_cast<float>(xl - kx);
  }
  // FP32 geometry of the node sweep (lattice units)
  for (int k = 0; k < 3; ++k)
    for (int j = 0; j < 3; ++j) D.Rt[9 * p + 3 * k + j] = static_cast<float>(R[3 * j + k]);
  if (type == 2) {
    for (int f = S.face_off[p]; f < S.face_off[p + 1]; ++f) {
      const double* e = S.planes + 4 * f;
      const double m0 = R[0] * e[0] + R[1] * e[1] + R[2] * e[2];
      const double m1 = R[3] * e[0] + R[4] * e[1] + R[5] * e[2];
      const double m2 = R[6] * e[0] + R[7] * e[1] + R[8] * e[2];
      D.wplane[f] = make_float4(static_cast<float>(m0), static_cast<float>(m1), static_cast<float>(m2),
                                static_cast<float>((e[3] + P.inflate) * P.inv_dx));
    }
  }
  const int bin = b[0] + P.nbin[0] * (b[1] + P.nbin[1] * b[2]);
  D.bin[p] = bin;
  D.slot[p] = atomicAdd(&W.bin_count[bin], 1);
}

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of n ints in global memory (one CTA of 1024
// threads, each scanning a contiguous chunk).  Returns the total.
__device__ long long block_scan_excl(int* data, int n, long long* s_tmp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int chunk = (n + nt - 1) / nt;
  const int b = min(n, tid * chunk), e = min(n, b + chunk);
  long long s = 0;
  for (int i = b; i < e; ++i) s += data[i];
  s_tmp[tid] = s;
  __syncthreads();
  // Hillis-Steele over the 1024 chunk sums
  for (int off = 1; off < nt; off <<= 1) {
    const long long v = (tid >= off) ? s_tmp[tid - off] : 0;
    __syncthreads();
    s_tmp[tid] += v;
    __syncthreads();
  }
  const long long total = s_tmp[nt - 1];
  long long run = s_tmp[tid] - s;
  for (int i = b; i < e; ++i) {
    const int v = data[i];
    data[i] = static_cast<int>(run);
    run += v;
  }
  __syncthreads();
  return total;
}

// K2: bin offsets and particle ids grouped by bin (single CTA).
__global__ void __launch_bounds__(1024) k_bin_scatter(Params P, Parts D, Lists W) {
  __shared__ long long s_tmp[1024];
  pdl_begin();
  const int nbins = P.nbin[0] * P.nbin[1] * P.nbin[2];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) W.bin_start[i] = W.bin_count[i];
  __syncthreads();
  const long long total = block_scan_excl(W.bin_start, nbins, s_tmp);
  if (threadIdx.x == 0) W.bin_start[nbins] = static_cast<int>(total);
  __syncthreads();
  for (int p = threadIdx.x; p < P.n; p += blockDim.x) W.bin_items[W.bin_start[D.bin[p]] + D.slot[p]] = p;
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

// K3: one warp per particle.  Lanes 0..26 fetch the ranges of the 27
// neighbour bins at once; the candidates of all bins are then swept as one
// flat list, 32 per round, and compacted with warp ballots into partners
// above (j > p) and below (j < p); each list is sorted by rank.
__global__ void __launch_bounds__(256) k_broad(Params P, Parts D, Lists W) {
  extern __shared__ int s_buf[];
  pdl_begin();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = blockIdx.x * (blockDim.x >> 5) + wid;
  if (p >= P.n) return;
  const int cap = P.max_nbr;
  int* up = s_buf + wid * 2 * cap;
  int* dn = up + cap;
  const int bin = D.bin[p];
  const int b[3] = {bin % P.nbin[0], (bin / P.nbin[0]) % P.nbin[1], bin / (P.nbin[0] * P.nbin[1])};
  int cnt[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) cnt[k] = P.nbin[k] >= 3 ? 3 : P.nbin[k];
  const int nnb = cnt[0] * cnt[1] * cnt[2];
  int beg = 0, num = 0;
  if (lane < nnb) {
    int o[3] = {lane % cnt[0], (lane / cnt[0]) % cnt[1], lane / (cnt[0] * cnt[1])};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = P.nbin[k] >= 3 ? b[k] + o[k] - 1 : o[k];
      o[k] = (c + P.nbin[k]) % P.nbin[k];
    }
    const int q = o[0] + P.nbin[0] * (o[1] + P.nbin[1] * o[2]);
    beg = W.bin_start[q];
    num = W.bin_start[q + 1] - beg;
  }
  // exclusive prefix of the bin sizes over the lanes
  int off = num;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int v = __shfl_up_sync(kFull, off, d);
    if (lane >= d) off += v;
  }
  const int total = __shfl_sync(kFull, off, 31);
  off -= num;
  int nup = 0, ndn = 0;
  const unsigned below = (1u << lane) - 1u;
  for (int base = 0; base < total; base += 32) {
    const int e = base + lane;
    // bin of flat candidate e: the last lane whose offset is <= e
    int src = 0;
    for (int t = 1; t < nnb; ++t) src = (e >= __shfl_sync(kFull, off, t)) ? t : src;
    const int bb = __shfl_sync(kFull, beg, src), bo = __shfl_sync(kFull, off, src);
    const int j = (e < total) ? W.bin_items[bb + e - bo] : -1;
    bool hit = false;
    if (j >= 0 && j != p) {
      int s[3], lo[3], hi[3];
      hit = pair_box(P, D, p, j, s, lo, hi);
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
}

// K4a: first pair of every particle row (exclusive scan of the partner
// counts, one CTA) and reset of the step's counters.
__global__ void __launch_bounds__(1024) k_rows(Params P, Lists W, int32_t* __restrict__ n_pairs_out) {
  __shared__ long long s_tmp[1024];
  pdl_begin();
  const int n = P.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) W.row_off[i] = W.up_count[i];
  __syncthreads();
  const long long total_pairs = block_scan_excl(W.row_off, n, s_tmp);
  if (threadIdx.x == 0) {
    W.row_off[n] = static_cast<int>(total_pairs);
    W.counters[0] = static_cast<int>(total_pairs);
    W.counters[1] = 0;   // tiles allocated
    W.counters[2] = 0;   // node-sweep queue head
    W.counters[5] = 0;   // pairs with V > 0
    for (int b = 0; b < kCostBuckets; ++b) W.counters[8 + b] = 0;
    W.u64[0] = 0;        // node evaluations
    W.u64[1] = 0;        // nominal lane-ops
    *n_pairs_out = static_cast<int>(total_pairs);
    if (total_pairs > P.max_pairs) set_error(W.err, kErrCapacity);
  }
}

// K4b: one warp per particle row i, one lane per partner slot r: the pair
// record of pair row_off[i] + r, its sweep layout and its node tiles.  Tiles
// are allocated with one atomic per warp round; a pair's tiles are
// contiguous, and its partial sums do not depend on where they land, so the
// results are deterministic.  No FP64: centres come as integer node + FP32
// remainder from the pose kernel.
__global__ void __launch_bounds__(128) k_build_pairs(Params P, Shapes S, Parts D, Lists W,
                                                     int32_t* __restrict__ pair_ij) {
  pdl_begin();
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= P.n) return;
  const int cap = P.max_nbr;
  const int cnt = W.up_count[i], row = W.row_off[i];
  for (int base = 0; base < cnt; base += 32) {
    const int r = base + lane;
    const bool active = r < cnt && (row + r) < P.max_pairs;
    PairRec pr;
    int pi = 0, ntiles = 0;
    unsigned long long vol = 0, ops = 0;
    if (active) {
      pi = row + r;
      const int j = W.up_list[i * cap + r];
      int lo[3], hi[3];
      pair_box(P, D, i, j, pr.shift, lo, hi);
      pr.i = i;
      pr.j = j;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        pr.lo[k] = lo[k];
        pr.dim[k] = hi[k] - lo[k] + 1;
      }
      // sweep layout: lines along one axis, lines cut into nseg segments; the
      // choice minimises warp slots x (segment length + 2 node-equivalents
      // for the line set-up)
      const long long volp = static_cast<long long>(pr.dim[0]) * pr.dim[1] * pr.dim[2];
      long long best = -1;
      for (int a = 0; a < 3; ++a) {
        const int du = pr.dim[a];
        const long long lines = volp / du;
        for (int ns = 1; ns <= 8 && ns <= du; ++ns) {
          const int sl = (du + ns - 1) / ns;
          if (sl > kSegMax) continue;
          const long long slots = (lines * ns + 31) / 32;
          const long long cost = slots * (sl + 2);
          if (best < 0 || cost < best) {
            best = cost;
            pr.axis = a;
            pr.nseg = ns;
            pr.seglen = sl;
          }
        }
      }
      if (best < 0) {   // a box longer than 8 * kSegMax nodes: longest axis, more segments
        int a = 0;
        for (int k = 1; k < 3; ++k) a = pr.dim[k] > pr.dim[a] ? k : a;
        pr.axis = a;
        pr.nseg = (pr.dim[a] + kSegMax - 1) / kSegMax;
        pr.seglen = (pr.dim[a] + pr.nseg - 1) / pr.nseg;
      }
      pr.nitems = static_cast<int>(volp / pr.dim[pr.axis]) * pr.nseg;
      ntiles = (pr.nitems + 32 * kTileItemsPerLane - 1) / (32 * kTileItemsPerLane);
      pr.ntiles = ntiles;
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
      pr.tile = 0;
      pr.pair = pi;
      vol = static_cast<unsigned long long>(volp);
      ops = vol * static_cast<unsigned long long>(S.nomops[i] + S.nomops[j]);
      pair_ij[2 * pi] = i;
      pair_ij[2 * pi + 1] = j;
      // slot of this pair in j's list of lower partners
      const int* dl = W.dn_list + static_cast<size_t>(j) * cap;
      int a0 = 0, a1 = W.dn_count[j];
      while (a0 < a1) {
        const int mid = (a0 + a1) >> 1;
        if (dl[mid] < i) a0 = mid + 1; else a1 = mid;
      }
      W.dn_pair[static_cast<size_t>(j) * cap + a0] = pi;
    }
    // warp-aggregated tile allocation and counters
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
    int tbase = 0;
    if (lane == 31 && incl > 0) tbase = atomicAdd(&W.counters[1], incl);
    if (lane == 0 && wv > 0) {
      atomicAdd(&W.u64[0], wv);
      atomicAdd(&W.u64[1], wo);
    }
    tbase = __shfl_sync(kFull, tbase, 31);
    if (active) {
      pr.tile0 = tbase + incl - ntiles;
      W.pairs[pi] = pr;
      for (int k = 0; k < ntiles; ++k) {
        if (pr.tile0 + k < P.max_tiles) W.tile_pair[pr.tile0 + k] = pi;
        else set_error(W.err, kErrCapacity);
      }
    }
    // queue records, grouped by estimated cost: slots x (segment + 2), scaled
    // by the pair's nominal ops per node (warp-aggregated atomics per bucket)
    int maxt = ntiles;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) maxt = max(maxt, __shfl_xor_sync(kFull, maxt, d));
    const int slots_total = active ? (pr.nitems + 31) / 32 : 0;
    const int weight = active ? (S.nomops[pr.i] + S.nomops[pr.j]) : 0;
    for (int k = 0; k < maxt; ++k) {
      const bool has = active && k < ntiles && pr.tile0 + k < P.max_tiles;
      int bucket = kCostBuckets;   // none
      if (has) {
        const int slots = min(kTileItemsPerLane, slots_total - k * kTileItemsPerLane);
        const int cost = slots * (pr.seglen + 2) * weight;   // ~ warp instructions
        bucket = cost >= 2400 ? 0 : (cost >= 1200 ? 1 : (cost >= 600 ? 2 : 3));
      }
      const unsigned grp = __match_any_sync(kFull, bucket);
      const int leader = __ffs(grp) - 1;
      int pos = 0;
      if (has && lane == leader) pos = atomicAdd(&W.counters[8 + bucket], __popc(grp));
      pos = __shfl_sync(kFull, pos, leader) + __popc(grp & ((1u << lane) - 1u));
      if (has) {
        pr.tile = k;
        W.tiles[static_cast<size_t>(bucket) * P.max_tiles + pos] = pr;
      }
    }
  }
}

}  // namespace

void launch_pose(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* pos,
                 const double* quat, cudaStream_t st) {
  const int nb = (P.n + 31) / 32;   // few threads per SM: the FP64 pipe is narrow
  if (nb > 0) launch_pdl(k_pose, dim3(nb), dim3(32), 0, st, P, S, D, W, pos, quat);
}

void launch_bin_scatter(const Params& P, const Parts& D, const Lists& W, cudaStream_t st) {
  launch_pdl(k_bin_scatter, dim3(1), dim3(1024), 0, st, P, D, W);
}

void launch_broad(const Params& P, const Parts& D, const Lists& W, cudaStream_t st) {
  const int warps = 8;
  const int nb = (P.n + warps - 1) / warps;
  const size_t smem = static_cast<size_t>(warps) * 2 * P.max_nbr * sizeof(int);
  if (nb > 0) launch_pdl(k_broad, dim3(nb), dim3(warps * 32), smem, st, P, D, W);
}

void launch_plan(const Params& P, const Shapes& S, const Parts& D, const Lists& W, int32_t* pair_ij, int32_t* n_pairs,
                 cudaStream_t st) {
  launch_pdl(k_rows, dim3(1), dim3(1024), 0, st, P, W, n_pairs);
  const int nb = (P.n + 3) / 4;   // four particle rows (warps) per block
  launch_pdl(k_build_pairs, dim3(nb > 0 ? nb : 1), dim3(128), 0, st, P, S, D, W, pair_ij);
}

}  // namespace gbc
