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

// K6: one thread per pair.  FP64 sums of the tile partials in tile order (or
// the FP64 kernel's sums), then contact point, normal, depth, force, torques.
__global__ void __launch_bounds__(64) k_finalize(Params P, Shapes S, Parts D, Lists W,
                                                  const double* __restrict__ vel, double* __restrict__ pair_out) {
  const int np = min(W.counters[0], P.max_pairs);
  const bool tiles_ok = P.precision == 1 || W.counters[1] <= P.max_tiles;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const PairRec pr = W.pairs[p];
    double s[9] = {0, 0, 0, 0, 0, 0, 0, -DBL_MAX, 0};
    if (P.precision == 1) {
      const double* q = W.sums + static_cast<size_t>(p) * kSumDoubles;
      for (int k = 0; k < 9; ++k) s[k] = q[k];
    } else if (tiles_ok) {
      int bi = 0x7fffffff;
      float bf = -FLT_MAX;
      for (int t = pr.tile0; t < pr.tile0 + pr.ntiles; ++t) {
        const float* q = W.partial + static_cast<size_t>(t) * kPartialFloats;
        for (int k = 0; k < 7; ++k) s[k] += static_cast<double>(q[k]);
        const int qi = __float_as_int(q[8]);
        if (q[7] > bf || (q[7] == bf && qi < bi)) { bf = q[7]; bi = qi; }
      }
      s[7] = bf;
      s[8] = static_cast<double>(bi);
    }
    const int i = pr.i, j = pr.j;
    double XA[3], XB[3];
    for (int k = 0; k < 3; ++k) {
      XA[k] = D.X[3 * i + k];
      XB[k] = D.X[3 * j + k] - pr.shift[k] * P.L[k];
    }
    const double dx = P.dx;
    const double V = dx * dx * dx * s[0];
    double out[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double ft[kFtDoubles] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double tape[kTapeDoubles] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (V > 0.0 && s[7] > -DBL_MAX) {
      double xc[3], G[3], n[3];
      for (int k = 0; k < 3; ++k) xc[k] = (pr.lo[k] + s[1 + k] / s[0]) * dx;
      const double gscale = 0.5 * dx * dx * 6.0 / (P.wdx / dx);
      for (int k = 0; k < 3; ++k) G[k] = gscale * s[4 + k];
      const double gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
      double fallback = 0.0;
      if (gn > 1e-12 * dx * dx) {
        for (int k = 0; k < 3; ++k) n[k] = G[k] / gn;
      } else {
        fallback = 1.0;
        const double dX[3] = {XB[0] - XA[0], XB[1] - XA[1], XB[2] - XA[2]};
        const double nd = sqrt(dX[0] * dX[0] + dX[1] * dX[1] + dX[2] * dX[2]);
        for (int k = 0; k < 3; ++k) n[k] = nd > 0.0 ? dX[k] / nd : 0.0;
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
      const double EA = S.young[i], EB = S.young[j], nuA = S.poisson[i], nuB = S.poisson[j];
      const double estar = 1.0 / ((1.0 - nuA * nuA) / EA + (1.0 - nuB * nuB) / EB);
      double damp = 1.0;
      if (vel != nullptr && P.damping_c != 0.0) {
        const double* va = vel + 6 * i;
        const double* vb = vel + 6 * j;
        const double ra[3] = {xc[0] - XA[0], xc[1] - XA[1], xc[2] - XA[2]};
        const double rb[3] = {xc[0] - XB[0], xc[1] - XB[1], xc[2] - XB[2]};
        double wa[3], wb[3];
        cross(va + 3, ra, wa);
        cross(vb + 3, rb, wb);
        double ddot = 0.0;
        for (int k = 0; k < 3; ++k) ddot += ((va[k] + wa[k]) - (vb[k] + wb[k])) * n[k];
        damp = fmax(0.0, 1.0 + P.damping_c * ddot);
      }
      const double vd = V * d;
      const double fmag = vd > 0.0 ? (4.0 / (3.0 * 3.14159265358979323846)) * estar * sqrt(vd) * damp : 0.0;
      double F[3], FA[3], ra[3], rb[3], TA[3], TB[3];
      for (int k = 0; k < 3; ++k) {
        F[k] = fmag * n[k];
        FA[k] = -F[k];
        ra[k] = xc[k] - XA[k];
        rb[k] = xc[k] - XB[k];
      }
      cross(ra, FA, TA);
      cross(rb, F, TB);
      out[0] = V;
      for (int k = 0; k < 3; ++k) {
        out[1 + k] = xc[k];
        out[4 + k] = n[k];
        out[8 + k] = F[k];
        ft[k] = F[k];
        ft[3 + k] = TA[k];
        ft[6 + k] = TB[k];
      }
      out[7] = d;
      tape[0] = s[0];
      for (int k = 0; k < 3; ++k) { tape[1 + k] = xc[k]; tape[4 + k] = n[k]; }
      tape[7] = d;
      tape[8] = gn;
      tape[9] = fallback;
      tape[10] = estar;
      tape[11] = damp;
      tape[12] = fmag;
      tape[13] = s[8];
      atomicAdd(&W.counters[5], 1);
    }
    double* o = pair_out + static_cast<size_t>(p) * 11;
    for (int k = 0; k < 11; ++k) o[k] = out[k];
    double* f = W.ft + static_cast<size_t>(p) * kFtDoubles;
    for (int k = 0; k < kFtDoubles; ++k) f[k] = ft[k];
    double* tp = W.tape + static_cast<size_t>(p) * kTapeDoubles;
    for (int k = 0; k < kTapeDoubles; ++k) tp[k] = tape[k];
  }
}

// K7: one warp per particle.  Its contributions are, in this order, the
// pairs where it is j (by i) and the pairs where it is i (by j); lanes fetch
// them 32 at a time, lane 0 adds them up in that order (FP64).
__global__ void __launch_bounds__(128) k_particle_sum(Params P, Parts D, Lists W, double* __restrict__ force,
                                                      double* __restrict__ torque) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p == 0 && lane == 0) *W.err_host = *W.err;
  if (p >= P.n) return;
  const int np = min(W.counters[0], P.max_pairs);
  const int nd = W.dn_count[p], nu = W.up_count[p], r0 = W.row_off[p];
  const size_t slot = static_cast<size_t>(p) * P.max_nbr;
  double f[3] = {0, 0, 0}, t[3] = {0, 0, 0};
  for (int base = 0; base < nd + nu; base += 32) {
    const int e = base + lane;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (e < nd) {
      const int q = W.dn_pair[slot + e];
      if (q < np) {
        const double* x = W.ft + static_cast<size_t>(q) * kFtDoubles;
        v[0] = x[0]; v[1] = x[1]; v[2] = x[2];
        v[3] = x[6]; v[4] = x[7]; v[5] = x[8];
      }
    } else if (e < nd + nu) {
      const int q = r0 + (e - nd);
      if (q < np) {
        const double* x = W.ft + static_cast<size_t>(q) * kFtDoubles;
        v[0] = -x[0]; v[1] = -x[1]; v[2] = -x[2];
        v[3] = x[3]; v[4] = x[4]; v[5] = x[5];
      }
    }
    const int m = min(32, nd + nu - base);
    for (int l = 0; l < m; ++l) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        f[k] += __shfl_sync(0xffffffffu, v[k], l);
        t[k] += __shfl_sync(0xffffffffu, v[3 + k], l);
      }
    }
  }
  if (lane == 0) {
    for (int k = 0; k < 3; ++k) {
      force[3 * p + k] = f[k];
      torque[3 * p + k] = t[k];
    }
  }
}

}  // namespace

void launch_finalize(const Params& P, const Shapes& S, const Parts& D, const Lists& W, const double* vel,
                     double* pair_out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int need = (P.max_pairs + 63) / 64;
  const int grid = need < 4 * sms ? (need > 0 ? need : 1) : 4 * sms;
  k_finalize<<<grid, 64, 0, st>>>(P, S, D, W, vel, pair_out);
}

void launch_particle_sum(const Params& P, const Parts& D, const Lists& W, double* force, double* torque,
                         cudaStream_t st) {
  const int nb = (P.n + 3) / 4;   // four particles (warps) per block
  k_particle_sum<<<nb > 0 ? nb : 1, 128, 0, st>>>(P, D, W, force, torque);
}

}  // namespace gbc
