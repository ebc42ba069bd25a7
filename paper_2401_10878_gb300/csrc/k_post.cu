// Per-particle sums of the contact forces and torques (the pairs' force law
// runs in the node sweep's epilogue, force_law.cuh).
//
// Paper (arXiv:2401.10878):
//   Sec. 4.3.3  contact forces and torques are delivered to both particles.
#include <cfloat>

#include "contact_dev.cuh"

namespace gbc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// The sum of particle p's component c (one lane).
__device__ __forceinline__ void particle_sum(const Params& P, const Lists& W, int p, int c, double* __restrict__ force,
                                             double* __restrict__ torque) {
  const int* dp = W.dn_pair + static_cast<size_t>(p) * P.max_nbr;
  int pre[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) pre[u] = u < P.max_nbr ? dp[u] : 0;
  const int np = min(W.counters[0], P.max_pairs);
  const int nd = W.dn_count[p], nu = W.up_count[p], r0 = W.row_off[p];
  const int offj = c < 3 ? c : c + 3, offi = c;
  const long long flip_i = c < 3 ? static_cast<long long>(0x8000000000000000ULL) : 0LL;
  const int total = nd + nu;
  double acc = 0.0;
  for (int base = 0; base < total; base += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u;
      const bool isj = e < nd;
      int q = isj ? (base == 0 ? pre[u] : dp[e]) : (e < total ? r0 + (e - nd) : np);
      if (e < total) q = checked_index(W.err, q, np, -1);
      const bool ok = q >= 0 && q < np;
      const long long b = ok ? __double_as_longlong(W.ft[static_cast<size_t>(q) * kFtDoubles + (isj ? offj : offi)]) : 0LL;
      v[u] = __longlong_as_double(isj ? b : b ^ flip_i);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (base + u < total) acc += v[u];
  }
  if (c < 3) force[3 * p + c] = acc;
  else torque[3 * p + c - 3] = acc;
}

// K6: per particle and component (eight lanes per particle, six used), FP64
// adds in a fixed order: the pairs where the particle is j (by i), then the
// pairs where it is i (by j).  j receives +F and T_B, i receives -F and T_A.
// The first eight lower-partner pair indices are fetched together with the
// counts.
__global__ void __launch_bounds__(32) k_particle_sum(Params P, Parts D, Lists W, double* __restrict__ force,
                                                      double* __restrict__ torque) {
  pdl_begin();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    if (!W.publish) *W.err_host = *W.err;
    ++W.counters[kStepCounter];   // the contact history written this step is read by the next
  }
  // the cell list's bin counts start the next step at zero
  const int nbins = P.nbin[0] * P.nbin[1] * P.nbin[2];
  for (int b = t; b < nbins; b += gridDim.x * blockDim.x) W.bin_count[b] = 0;
  const int p = t >> 3, c = t & 7;
  if (p < P.n && c < 6) particle_sum(P, W, p, c, force, torque);
  // a host-buffer step that returns on its token: the step is complete when
  // every block's sums are stored, and the last block to finish mirrors the
  // error word and then publishes the host's token of this step (mapped host
  // memory), so the host can return without a stream synchronisation
  if (!W.publish) return;
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    __threadfence_system();
    const unsigned prev = atomicAdd(reinterpret_cast<unsigned*>(W.counters + kDoneCounter), 1u);
    if (prev == gridDim.x - 1) {
      W.counters[kDoneCounter] = 0;
      *reinterpret_cast<volatile int*>(W.err_host) = __ldcg(W.err);
      __threadfence_system();
      *reinterpret_cast<volatile int*>(W.err_host + 1) = __ldcg(W.counters + kTokenCounter);
    }
  }
}

}  // namespace

void launch_particle_sum(const Params& P, const Parts& D, const Lists& W, double* force, double* torque,
                         cudaStream_t st) {
  const int nb = (8 * P.n + 31) / 32;   // one-warp blocks (four particles each)
  launch_pdl(k_particle_sum, dim3(nb > 0 ? nb : 1), dim3(32), 0, st, P, D, W, force, torque);
}

}  // namespace gbc
