// Pseudofermion force (Supplement SI, Eqs. (force&CG) and (fermion_force)).
//
// With X = (M^dagger M)^{-1} phi and Y = M X,
//   dS_f/dtheta_{tau,b} = +2 Re[Y_{tau+1}^dagger dB_tau X_tau]     (tau < Ntau-1)
//   dS_f/dtheta_{tau,b} = -2 Re[Y_0^dagger dB_{Ntau-1} X_{Ntau-1}] (tau = Ntau-1),
// and dB_tau follows the product rule over the factors of B_tau = cB P_tau that
// contain bond b (one factor for family 1, two for families 2-4).
//
// One CTA per slice, independent of the others: Y_{tau+1} = X_{tau+1} -
// s_{tau+1} cB P_tau X_tau is formed from the slice's own forward sweep, so no
// separate apply of M is needed.  The sweep positions k = 1..7 of
// P = P(1) P(2) ... P(7) are then walked left to right with
//   u_k = P(k+1) ... P(7) X_tau          (recovered by stepping back with P(k)^{-1})
//   w_k = P(k-1)^dagger ... P(1)^dagger Y  (stepping forward; P(k)^dagger = P(k)),
// and at each position every bond of that family adds
//   2 cB Re[ w^dagger (dP(k)/dtheta_b) u ] = -2 cB Im[conj(w_i) U u_j - conj(w_j) conj(U) u_i].
// Only two slice buffers are live, so the kernel fits the same lattice sizes
// as the M^dagger M kernel.
#include "kernels.h"

namespace hqmc {

__constant__ static const int kFam[7] = {4, 3, 2, 1, 2, 3, 4};  // P(1) ... P(7)

__device__ __forceinline__ void force_slice(const Geo& g, double cB, double inv1, double inv2,
                                            const double2* __restrict__ U, const double2* __restrict__ X,
                                            double* __restrict__ dSf, int tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int V = g.V, N = g.Ntau;
  double2* u = reinterpret_cast<double2*>(smem_raw);
  double2* w = u + V;
  const int taup = (tau == N - 1) ? 0 : tau + 1;
  const double sigp = (taup == 0) ? -1.0 : 1.0;  // sign of the B term in row tau+1 of M
  const double sgn = (tau < N - 1) ? 1.0 : -1.0;
  const double2* Ut = U + (size_t)tau * V * 2;
  const size_t bt = (size_t)tau * V, bp = (size_t)taup * V;
  double2* out = reinterpret_cast<double2*>(dSf) + bt;  // (dS/dtheta_x, dS/dtheta_y) per site

  for (int s = threadIdx.x; s < V; s += blockDim.x) {
    u[s] = X[bt + s];
    out[s] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  apply_P(g, u, Ut);  // u = P X_tau
  for (int s = threadIdx.x; s < V; s += blockDim.x) w[s] = caxpy(X[bp + s], -sigp * cB, u[s]);  // Y_{tau+1}
  __syncthreads();
  // 1/(1 - |U|^2): family 1 carries tanh(a), the others tanh(a/2)
  auto inv_of = [&](int fam) { return fam == 1 ? inv1 : inv2; };
  factor_pass_inverse(g, kFam[0], u, Ut, inv_of(kFam[0]));  // u_1 = P(1)^{-1} P X_tau
  __syncthreads();

  const double coef = -2.0 * cB * sgn;
  const int nb = V >> 1;
#pragma unroll 1
  for (int k = 0; k < 7; ++k) {
    const int fam = kFam[k];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      int i, j, c;
      bond_of(g, fam, b, i, j, c);
      const double2 uu = __ldg(Ut + 2 * i + c);
      const double2 wi = w[i], wj = w[j], ui = u[i], uj = u[j];
      // val = conj(w_i) U u_j - conj(w_j) conj(U) u_i ; only Im(val) is needed.  Every
      // product-sum is written as an explicit fma so that the single-chain and the
      // batched kernel, which both inline this, round alike.
      const double2 Uuj = make_double2(fma(uu.x, uj.x, -__dmul_rn(uu.y, uj.y)), fma(uu.x, uj.y, __dmul_rn(uu.y, uj.x)));
      const double2 cUui = make_double2(fma(uu.x, ui.x, __dmul_rn(uu.y, ui.y)), fma(uu.x, ui.y, -__dmul_rn(uu.y, ui.x)));
      const double im = __dsub_rn(fma(wi.x, Uuj.y, -__dmul_rn(wi.y, Uuj.x)), fma(wj.x, cUui.y, -__dmul_rn(wj.y, cUui.x)));
      // bond b of a family is handled by the same thread at both of its positions
      double* o = reinterpret_cast<double*>(out + i) + c;
      *o = fma(coef, im, *o);
    }
    if (k == 6) break;
    __syncthreads();
    factor_pass(g, fam, w, Ut);                    // w_{k+1} = P(k) w_k
    factor_pass_inverse(g, kFam[k + 1], u, Ut, inv_of(kFam[k + 1]));  // u_{k+1} = P(k+1)^{-1} u_k
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024, 1)
force_kernel(Geo g, double cB, double inv1, double inv2, const double2* __restrict__ U,
             const double2* __restrict__ X, double* __restrict__ dSf) {
  force_slice(g, cB, inv1, inv2, U, X, dSf, blockIdx.x);
}

// The force of every chain of a batch: one CTA per (chain, slice) tile.
__global__ void __launch_bounds__(1024, 1) batch_force_kernel(const ChainDesc* __restrict__ descs,
                                                              const int2* __restrict__ tiles) {
  const int2 t = tiles[blockIdx.x];
  const ChainDesc& d = descs[t.x];
  force_slice(d.g, d.cB, d.inv1, d.inv2, d.U64, d.X, d.dSf, t.y);
}

cudaError_t launch_batch_force(const ChainDesc* d, const int2* tiles, int ntiles, int threads, size_t smem,
                               cudaStream_t s) {
  cudaError_t e = raise_smem_limit(batch_force_kernel, smem);
  if (e != cudaSuccess) return e;
  batch_force_kernel<<<ntiles, threads, smem, s>>>(d, tiles);
  return cudaGetLastError();
}

cudaError_t prepare_force(const SliceLaunch& sl) {
  return raise_smem_limit(force_kernel, 2 * sl.g.V * sizeof(double2));
}

cudaError_t launch_force(const SliceLaunch& sl, double cB, double t1, double t2, const double2* U, const double2* X,
                         double* dSf, cudaStream_t s) {
  force_kernel<<<sl.g.Ntau, sl.threads, 2 * sl.g.V * sizeof(double2), s>>>(sl.g, cB, 1.0 / (1.0 - t1 * t1),
                                                                          1.0 / (1.0 - t2 * t2), U, X, dSf);
  return cudaGetLastError();
}

}  // namespace hqmc
