// Per-pair reduction, force law and per-particle sums of the contact step.
//
// Paper (arXiv:2401.10878):
//   Sec. 3.3.1  overlap volume, contact point, contact normal, indentation depth;
//   Sec. 2.3    Eq. (contact_force_normal) F = 4/(3 pi) n E* sqrt(V d)(1 + c ddot_n),
//               E* = ((1-nu_A^2)/E_A + (1-nu_B^2)/E_B)^-1;
//   Sec. 2.2    torques about the centres of mass;
//   Sec. 4.3.3  contact forces and torques are delivered to both particles.
#include <cfloat>

#include "contact_dev.cuh"

namespace gbc {

namespace {

__device__ __forceinline__ void cross(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// K6: FP64 per-pair reduction and force law.  Every lane first sums its
// pair's tile partials in FP64 (tile order) and writes zeros for pairs without
// overlap; the overlapping pairs of the block are then compacted so that the
// FP64-heavy part (on GB300 every FP64 warp instruction occupies the SM's
// narrow FP64 pipe, however many lanes are active) runs with full warps.
constexpr int kFinBlock = 64;

__global__ void __launch_bounds__(kFinBlock) k_finalize(Params P, Shapes S, Parts D, Lists W,
                                                        const double* __restrict__ vel,
                                                        double* __restrict__ pair_out) {
  __shared__ double s_sum[kFinBlock][9];
  __shared__ int s_pair[kFinBlock];
  __shared__ int s_count;
  pdl_begin();
  const int np = min(W.counters[0], P.max_pairs);
  const bool tiles_ok = P.precision == 1 || W.counters[1] <= P.max_tiles;
  const int tid = threadIdx.x;
  for (int base = blockIdx.x * kFinBlock; base < np; base += gridDim.x * kFinBlock) {
    if (tid == 0) s_count = 0;
    __syncthreads();
    const int p = base + tid;
    if (p < np) {
      double s[9] = {0, 0, 0, 0, 0, 0, 0, -DBL_MAX, 0};
      if (P.precision == 1) {
        const double* q = W.sums + static_cast<size_t>(p) * kSumDoubles;
        for (int k = 0; k < 9; ++k) s[k] = q[k];
      } else if (tiles_ok) {
        const PairRec& pr = W.pairs[p];
        const int t0 = pr.tile0, t1 = pr.tile0 + pr.ntiles;
        int bi = 0x7fffffff;
        float bf = -FLT_MAX;
        for (int t = t0; t < t1; ++t) {
          const float* q = W.partial + static_cast<size_t>(t) * kPartialFloats;
          for (int k = 0; k < 7; ++k) s[k] += static_cast<double>(q[k]);
          const int qi = __float_as_int(q[8]);
          if (q[7] > bf || (q[7] == bf && qi < bi)) { bf = q[7]; bi = qi; }
        }
        s[7] = bf;
        s[8] = static_cast<double>(bi);
      }
      if (s[0] > 0.0 && s[7] > -DBL_MAX) {
        const int at = atomicAdd(&s_count, 1);
        s_pair[at] = p;
        for (int k = 0; k < 9; ++k) s_sum[at][k] = s[k];
      } else {
        double* o = pair_out + static_cast<size_t>(p) * 11;
        for (int k = 0; k < 11; ++k) o[k] = 0.0;
        double* f = W.ft + static_cast<size_t>(p) * kFtDoubles;
        for (int k = 0; k < kFtDoubles; ++k) f[k] = 0.0;
        double* tp = W.tape + static_cast<size_t>(p) * kTapeDoubles;
        for (int k = 0; k < kTapeDoubles; ++k) tp[k] = 0.0;
      }
    }
    __syncthreads();
    if (tid < s_count) {
      const int q = s_pair[tid];
      double s[9];
      for (int k = 0; k < 9; ++k) s[k] = s_sum[tid][k];
      const PairRec& pr = W.pairs[q];
      const int i = pr.i, j = pr.j;
      double XA[3], XB[3];
      for (int k = 0; k < 3; ++k) {
        XA[k] = D.X[3 * i + k];
        XB[k] = D.X[3 * j + k] - pr.shift[k] * P.L[k];
      }
      const double dx = P.dx;
      const double V = dx * dx * dx * s[0];
      const double inv_s0 = 1.0 / s[0];
      double xc[3], G[3], n[3];
      for (int k = 0; k < 3; ++k) xc[k] = (pr.lo[k] + s[1 + k] * inv_s0) * dx;
      const double gscale = 0.5 * dx * dx * 6.0 / (P.wdx / dx);
      for (int k = 0; k < 3; ++k) G[k] = gscale * s[4 + k];
      const double gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
      double fallback = 0.0;
      if (gn > 1e-12 * dx * dx) {
        const double inv = 1.0 / gn;
        for (int k = 0; k < 3; ++k) n[k] = G[k] * inv;
      } else {
        fallback = 1.0;
        const double dX[3] = {XB[0] - XA[0], XB[1] - XA[1], XB[2] - XA[2]};
        const double nd = sqrt(dX[0] * dX[0] + dX[1] * dX[1] + dX[2] * dX[2]);
        const double inv = nd > 0.0 ? 1.0 / nd : 0.0;
        for (int k = 0; k < 3; ++k) n[k] = dX[k] * inv;
      }
      // indentation depth: FP64 re-evaluation at the deepest node
      const int vol = pr.dim[0] * pr.dim[1] * pr.dim[2];
      const int idx = min(max(static_cast<int>(s[8]), 0), vol - 1);
      const int c[3] = {idx % pr.dim[0], (idx / pr.dim[0]) % pr.dim[1], idx / (pr.dim[0] * pr.dim[1])};
      const double x[3] = {(pr.lo[0] + c[0]) * dx, (pr.lo[1] + c[1]) * dx, (pr.lo[2] + c[2]) * dx};
      double gA[3], gB[3];
      const double fa = sdf64(S.type[i], S.param + 3 * i, S.planes + 4 * S.face_off[i],
                              S.face_off[i + 1] - S.face_off[i], XA, D.R + 9 * i, x, P.inflate, gA);
      const double fb = sdf64(S.type[j], S.param + 3 * j, S.planes + 4 * S.face_off[j],
                              S.face_off[j + 1] - S.face_off[j], XB, D.R + 9 * j, x, P.inflate, gB);
      const double d = fmax(0.0, -(fa + fb));
      const double estar = 1.0 / (S.compl_[i] + S.compl_[j]);
      double damp = 1.0;
      double ra[3], rb[3];
      for (int k = 0; k < 3; ++k) {
        ra[k] = xc[k] - XA[k];
        rb[k] = xc[k] - XB[k];
      }
      if (vel != nullptr && P.damping_c != 0.0) {
        const double* va = vel + 6 * i;
        const double* vb = vel + 6 * j;
        double wa[3], wb[3];
        cross(va + 3, ra, wa);
        cross(vb + 3, rb, wb);
        double ddot = 0.0;
        for (int k = 0; k < 3; ++k) ddot += ((va[k] + wa[k]) - (vb[k] + wb[k])) * n[k];
        damp = fmax(0.0, 1.0 + P.damping_c * ddot);
      }
      const double vd = V * d;
      const double fmag = vd > 0.0 ? (4.0 / (3.0 * 3.14159265358979323846)) * estar * sqrt(vd) * damp : 0.0;
      double F[3], FA[3], TA[3], TB[3];
      for (int k = 0; k < 3; ++k) {
        F[k] = fmag * n[k];
        FA[k] = -F[k];
      }
      cross(ra, FA, TA);
      cross(rb, F, TB);
      double* o = pair_out + static_cast<size_t>(q) * 11;
      o[0] = V;
      for (int k = 0; k < 3; ++k) {
        o[1 + k] = xc[k];
        o[4 + k] = n[k];
        o[8 + k] = F[k];
      }
      o[7] = d;
      double* f = W.ft + static_cast<size_t>(q) * kFtDoubles;
      for (int k = 0; k < 3; ++k) {
        f[k] = F[k];
        f[3 + k] = TA[k];
        f[6 + k] = TB[k];
      }
      double* tp = W.tape + static_cast<size_t>(q) * kTapeDoubles;
      tp[0] = s[0];
      for (int k = 0; k < 3; ++k) { tp[1 + k] = xc[k]; tp[4 + k] = n[k]; }
      tp[7] = d;
      tp[8] = gn;
      tp[9] = fallback;
      tp[10] = estar;
      tp[11] = damp;
      tp[12] = fmag;
      tp[13] = s[8];
      tp[14] = 0.0;
      tp[15] = 0.0;
    }
    if (tid == 0 && s_count > 0) atomicAdd(&W.counters[5], s_count);
    __syncthreads();
  }
}

// K7: one lane per particle (FP64 adds in full warps).  Its contributions are
// added in this order: the pairs where it is j (by i), then the pairs where it
// is i (by j).
__global__ void __launch_bounds__(128) k_particle_sum(Params P, Parts D, Lists W, double* __restrict__ force,
                                                      double* __restrict__ torque) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) *W.err_host = *W.err;
  // the cell list's bin counts start the next step at zero
  const int nbins = P.nbin[0] * P.nbin[1] * P.nbin[2];
  for (int b = p; b < nbins; b += gridDim.x * blockDim.x) W.bin_count[b] = 0;
  if (p >= P.n) return;
  const int np = min(W.counters[0], P.max_pairs);
  const int nd = W.dn_count[p], nu = W.up_count[p], r0 = W.row_off[p];
  const int* dp = W.dn_pair + static_cast<size_t>(p) * P.max_nbr;
  double f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
  for (int r = 0; r < nd; ++r) {
    const int q = dp[r];
    if (q >= np) continue;
    const double* x = W.ft + static_cast<size_t>(q) * kFtDoubles;
    f0 += x[0]; f1 += x[1]; f2 += x[2];
    t0 += x[6]; t1 += x[7]; t2 += x[8];
  }
  for (int r = 0; r < nu; ++r) {
    const int q = r0 + r;
    if (q >= np) break;
    const double* x = W.ft + static_cast<size_t>(q) * kFtDoubles;
    f0 -= x[0]; f1 -= x[1]; f2 -= x[2];
    t0 += x[3]; t1 += x[4]; t2 += x[5];
  }
  force[3 * p] = f0; force[3 * p + 1] = f1; force[3 * p + 2] = f2;
  torque[3 * p] = t0; torque[3 * p + 1] = t1; torque[3 * p + 2] = t2;
}

}  // namespace

void launch_finalize(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                     double* pair_out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (P.max_pairs + kFinBlock - 1) / kFinBlock;
  const int grid = need < 4 * sms ? (need > 0 ? need : 1) : 4 * sms;
  launch_pdl(k_finalize, dim3(grid), dim3(kFinBlock), 0, st, P, S, D, W, vel, pair_out);
}

void launch_particle_sum(const Params& P, const Parts& D, const Lists& W, double* force, double* torque,
                         cudaStream_t st) {
  const int nb = (P.n + 31) / 32;
  launch_pdl(k_particle_sum, dim3(nb > 0 ? nb : 1), dim3(32), 0, st, P, D, W, force, torque);
}

}  // namespace gbc
