// Fused application of M^dagger M, M and M^dagger (Methods, "Matrix-free
// representation of M^dagger M v"; matrix M of Eq. (M_alpha); checkerboard
// B of Eq. (eq24)).
//
// With B_tau = cB P_tau (see common.cuh) and z_tau = P_tau x_tau,
//   (M^dagger M x)_tau = x_tau - s_tau cB z_{tau-1} + cB P_tau (cB z_tau - s'_tau x_{tau+1}),
// s_0 = -1, s'_{Ntau-1} = -1, otherwise +1.  Each slice therefore needs two
// sweeps of P over its own data plus z_{tau-1} of the previous slice.
//
// Design: one CTA per slice; consecutive slices form a thread-block cluster.
// Every CTA computes z_tau in shared memory and publishes it; after a cluster
// barrier the CTA of slice tau reads z_{tau-1} from its left neighbour through
// distributed shared memory.  Only the first CTA of each cluster recomputes
// the halo z_{tau0-1} itself (overlapped with the barrier), so a cluster of C
// slices does 2C+1 sweeps instead of 3C.  All 7 factor passes of a sweep run
// on a slice held in shared memory; HBM sees each input once and the output
// once.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace hqmc {

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <class R, int MODE>
__device__ __forceinline__ C2<R> load_input(const MdagmArgs<R>& a, const C2<R>* p_old, size_t g, R beta,
                                            bool first) {
  if (MODE == MODE_CGDIR) {
    C2<R> rv = a.r[g];
    if (first) return rv;
    return caxpy(rv, beta, p_old[g]);
  }
  return a.x[g];
}

// Body of the fused kernel for the CTA that owns slice `tau` of the chain
// described by `a`; `slot` / `nslots` index its reduction partial (slot < nslots).
template <class R, int MODE, int MB>
__device__ __forceinline__ void mdagm_body(const MdagmArgs<R>& a, const int tau, const int slot, const int nslots) {
  using T = C2<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int V = a.g.V, N = a.g.Ntau;
  T* Z = reinterpret_cast<T*>(smem_raw);  // z_tau, read by the right neighbour
  T* W = Z + V;                           // work slice
  T* Y = W + V;                           // output accumulator
  __shared__ double red[32];
  __shared__ int s_flags;                 // bit 0: stop, bit 1: first iteration of a segment
  __shared__ R s_beta;
  __shared__ int s_k;

  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const bool active = tau < N;

  if (MODE == MODE_CGDIR) {
    cgdir_head<R>(a, slot == 0, s_flags, s_beta, s_k);  // every CTA reaches the same decision
    if (s_flags & 1) return;  // uniform over the whole grid: no cluster barrier is pending
  }
  if (MODE == MODE_RESID && a.gate != GATE_ALWAYS) {
    // this launch writes no CG state, so every CTA reads the same st->done
    if (threadIdx.x == 0) s_flags = gate_open(a.gate, *(volatile int*)&a.st->done) ? 0 : 1;
    __syncthreads();
    if (s_flags & 1) return;
  }
  const bool first = (MODE == MODE_CGDIR) && (s_flags & 2);
  const R beta = (MODE == MODE_CGDIR) ? s_beta : R(0);
  const C2<R>* p_old = nullptr;
  C2<R>* p_new = nullptr;
  if (MODE == MODE_CGDIR) {
    // select without indexing the parameter array (keeps it out of local memory)
    p_old = (s_k & 1) ? a.pbuf[1] : a.pbuf[0];
    p_new = (s_k & 1) ? a.pbuf[0] : a.pbuf[1];
  }
  const R cB = a.cB;
  const int NT = a.teff > 0 ? a.teff : (int)blockDim.x;  // stride of the site loops
  const int t0 = (int)threadIdx.x < NT ? (int)threadIdx.x : V;  // threads beyond NT take no sites
  const int taum = (tau == 0) ? N - 1 : tau - 1;
  const int taup = (tau == N - 1) ? 0 : tau + 1;
  const size_t base = (size_t)tau * V;

  constexpr int MBA = MB > 0 ? MB : 1;
  int ij[4][MBA];
  T uu[4][MBA];
  const T* Ut = a.U + base * 2;
  if constexpr (MB > 0) make_bonds(a.g, ij);
  if (active) {
    if constexpr (MB > 0) load_links(ij, Ut, uu);
    // rank 0 prefetches its halo input x_{tau-1}, the others x_{tau+1}
    const size_t bpre = (size_t)(rank == 0 ? taum : taup) * V;
    for (int s = t0; s < V; s += NT) {
      const T v = load_input<R, MODE>(a, p_old, base + s, beta, first);
      Z[s] = v;
      Y[s] = v;
      if (MODE == MODE_CGDIR) p_new[base + s] = v;
      W[s] = load_input<R, MODE>(a, p_old, bpre + s, beta, first);
    }
    __syncthreads();
    if constexpr (MB > 0) sweep(Z, ij, uu);  // z_tau = P_tau x_tau
    else apply_P(a.g, Z, Ut);
  }
  cluster_arrive();  // z_tau published

  const T* Zprev = W;
  if (rank == 0 && active) {
    // halo: z_{tau-1} = P_{tau-1} x_{tau-1} for the first slice of the cluster
    if constexpr (MB > 0) {
      load_links(ij, a.U + (size_t)taum * V * 2, uu);
      sweep(W, ij, uu);
      load_links(ij, Ut, uu);
    } else {
      apply_P(a.g, W, a.U + (size_t)taum * V * 2);
    }
  }
  cluster_wait();
  if (rank != 0) Zprev = cl.map_shared_rank(Z, rank - 1);

  double acc0 = 0.0, acc1 = 0.0;
  if (active) {
    const R sig = (tau == 0) ? R(-1) : R(1);
    const R sigp = (tau == N - 1) ? R(-1) : R(1);
    if (rank == 0) {
      const size_t bp = (size_t)taup * V;
      for (int s = t0; s < V; s += NT) {
        Y[s] = caxpy(Y[s], -sig * cB, W[s]);
        W[s] = caxpy(cscale(cB, Z[s]), -sigp, load_input<R, MODE>(a, p_old, bp + s, beta, first));
      }
    } else {
      for (int s = t0; s < V; s += NT) {
        Y[s] = caxpy(Y[s], -sig * cB, Zprev[s]);
        W[s] = caxpy(cscale(cB, Z[s]), -sigp, W[s]);
      }
    }
  }
  cluster_arrive();  // finished reading the neighbour's shared memory
  if (active) {
    __syncthreads();
    if constexpr (MB > 0) sweep(W, ij, uu);
    else apply_P(a.g, W, Ut);
    R accq = 0;  // CG direction: the thread's terms in the vector's precision (cdot_re_own)
    for (int s = t0; s < V; s += NT) {
      T q = caxpy(Y[s], cB, W[s]);
      if (MODE == MODE_APPLY) {
        a.y[base + s] = q;
      } else if (MODE == MODE_CGDIR) {
        a.y[base + s] = q;
        accq += cdot_re_own(p_new[base + s], q);
      } else {  // MODE_RESID (R = double): r = b - O x
        const double2 bv = a.b[base + s];
        const double2 rv = make_double2(bv.x - (double)q.x, bv.y - (double)q.y);
        if (a.r_out_fp32)
          reinterpret_cast<float2*>(a.r_out)[base + s] = make_float2((float)rv.x, (float)rv.y);
        else
          reinterpret_cast<double2*>(a.r_out)[base + s] = rv;
        acc0 += rv.x * rv.x + rv.y * rv.y;
        acc1 += bv.x * bv.x + bv.y * bv.y;
      }
    }
    if (MODE == MODE_CGDIR) acc0 = (double)accq;
  }
  if (MODE != MODE_APPLY) {
    const double t0 = block_sum(acc0, red);
    if (threadIdx.x == 0) a.part_out[slot] = t0;
    if (MODE == MODE_RESID) {
      const double t1 = block_sum(acc1, red);
      if (threadIdx.x == 0) a.part_out[nslots + slot] = t1;
    }
  }
  cluster_wait();  // keep z_tau alive until the right neighbour has read it
}

template <class R, int MODE, int MB>
__global__ void __launch_bounds__((SweepThreads<R, MB>::max), 1) mdagm_kernel(const MdagmArgs<R> a) {
  mdagm_body<R, MODE, MB>(a, blockIdx.x, blockIdx.x, gridDim.x);
}

// Many chains in one launch: CTA b serves cluster tile b / C of the tile table,
// i.e. slice tau0 + (b mod C) of chain `chain`.  Clusters never straddle two
// chains, so every chain sees exactly the decisions and partial sums of its own
// single-chain launch with the same cluster size.
template <class R, int MODE>
__global__ void __launch_bounds__(1024, 1) mdagm_batch_kernel(const MdagmArgs<R>* __restrict__ descs,
                                                              const int2* __restrict__ tiles, int C) {
  __shared__ MdagmArgs<R> a;
  const int2 tile = tiles[blockIdx.x / C];
  if (threadIdx.x == 0) a = descs[tile.x];
  __syncthreads();
  const int tau = tile.y + (int)(blockIdx.x % C);
  const int nslots = (a.g.Ntau + C - 1) / C * C;
  mdagm_body<R, MODE, 0>(a, tau, tau, nslots);
}

template <class R, int MODE>
static size_t mdagm_smem(const SliceLaunch& sl) {
  return (size_t)3 * sl.g.V * sizeof(C2<R>);
}

template <class R, int MODE, int MB>
static cudaError_t prepare_mb(const SliceLaunch& sl) {
  cudaError_t e = raise_smem_limit(mdagm_kernel<R, MODE, MB>, mdagm_smem<R, MODE>(sl));
  if (e != cudaSuccess) return e;
  if (sl.cluster > 8)
    e = cudaFuncSetAttribute(mdagm_kernel<R, MODE, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <class R, int MODE>
cudaError_t prepare_mdagm(const SliceLaunch& sl) {
  switch (sl.mb) {
    case 0: return prepare_mb<R, MODE, 0>(sl);
    case 1: return prepare_mb<R, MODE, 1>(sl);
    case 2: return prepare_mb<R, MODE, 2>(sl);
    case 3: return prepare_mb<R, MODE, 3>(sl);
    case 4: return prepare_mb<R, MODE, 4>(sl);
    default: return cudaErrorInvalidValue;
  }
}

template <class R, int MODE, int MB>
static cudaError_t launch_mb(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sl.grid);
  cfg.blockDim = dim3(sl.threads);
  cfg.dynamicSmemBytes = mdagm_smem<R, MODE>(sl);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sl.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mdagm_kernel<R, MODE, MB>, a);
}

template <class R, int MODE>
cudaError_t launch_mdagm(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s) {
  switch (sl.mb) {
    case 0: return launch_mb<R, MODE, 0>(sl, a, s);
    case 1: return launch_mb<R, MODE, 1>(sl, a, s);
    case 2: return launch_mb<R, MODE, 2>(sl, a, s);
    case 3: return launch_mb<R, MODE, 3>(sl, a, s);
    case 4: return launch_mb<R, MODE, 4>(sl, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MB>
static int max_active_clusters_mb(const SliceLaunch& sl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sl.grid);
  cfg.blockDim = dim3(sl.threads);
  cfg.dynamicSmemBytes = mdagm_smem<double, MODE_CGDIR>(sl);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sl.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)mdagm_kernel<double, MODE_CGDIR, MB>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

int mdagm_max_active_clusters(const SliceLaunch& sl) {
  switch (sl.mb) {
    case 0: return max_active_clusters_mb<0>(sl);
    case 1: return max_active_clusters_mb<1>(sl);
    case 2: return max_active_clusters_mb<2>(sl);
    case 3: return max_active_clusters_mb<3>(sl);
    case 4: return max_active_clusters_mb<4>(sl);
    default: return -1;
  }
}

// Clusters of C CTAs of the batched kernel the device can keep resident (<= 0: none).
int mdagm_batch_max_active_clusters(int C, int threads, size_t smem) {
  if (raise_smem_limit(mdagm_batch_kernel<double, MODE_CGDIR>, smem) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)mdagm_batch_kernel<double, MODE_CGDIR>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

template <class R, int MODE>
cudaError_t launch_mdagm_batch(const MdagmArgs<R>* descs, const int2* tiles, int ntiles, int C, int threads,
                               size_t smem, cudaStream_t s) {
  cudaError_t e = raise_smem_limit(mdagm_batch_kernel<R, MODE>, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ntiles * C);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mdagm_batch_kernel<R, MODE>, descs, tiles, C);
}
template cudaError_t launch_mdagm_batch<double, MODE_CGDIR>(const MdagmArgs<double>*, const int2*, int, int, int,
                                                            size_t, cudaStream_t);
template cudaError_t launch_mdagm_batch<double, MODE_RESID>(const MdagmArgs<double>*, const int2*, int, int, int,
                                                            size_t, cudaStream_t);

template cudaError_t launch_mdagm<double, MODE_APPLY>(const SliceLaunch&, const MdagmArgs<double>&, cudaStream_t);
template cudaError_t launch_mdagm<double, MODE_RESID>(const SliceLaunch&, const MdagmArgs<double>&, cudaStream_t);
template cudaError_t launch_mdagm<double, MODE_CGDIR>(const SliceLaunch&, const MdagmArgs<double>&, cudaStream_t);
template cudaError_t launch_mdagm<float, MODE_APPLY>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t launch_mdagm<float, MODE_CGDIR>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t prepare_mdagm<double, MODE_APPLY>(const SliceLaunch&);
template cudaError_t prepare_mdagm<double, MODE_RESID>(const SliceLaunch&);
template cudaError_t prepare_mdagm<double, MODE_CGDIR>(const SliceLaunch&);
template cudaError_t prepare_mdagm<float, MODE_APPLY>(const SliceLaunch&);
template cudaError_t prepare_mdagm<float, MODE_CGDIR>(const SliceLaunch&);

// ---------------------------------------------------------------------------
// y = M x:        y_tau = x_tau - s_tau  cB P_{tau-1} x_{tau-1}
// y = M^dagger x: y_tau = x_tau - s'_tau cB P_tau x_{tau+1}   (B Hermitian)
template <class R>
__device__ __forceinline__ void apply_M_slice(const Geo& g, R cB, const C2<R>* __restrict__ U,
                                              const C2<R>* __restrict__ x, C2<R>* __restrict__ y, int dagger,
                                              int tau) {
  using T = C2<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* W = reinterpret_cast<T*>(smem_raw);
  const int V = g.V, N = g.Ntau;
  int src, uslice;
  R sign;
  if (!dagger) {
    src = (tau == 0) ? N - 1 : tau - 1;
    uslice = src;
    sign = (tau == 0) ? R(1) : R(-1);
  } else {
    src = (tau == N - 1) ? 0 : tau + 1;
    uslice = tau;
    sign = (tau == N - 1) ? R(1) : R(-1);
  }
  const size_t bs = (size_t)src * V, bt = (size_t)tau * V;
  for (int s = threadIdx.x; s < V; s += blockDim.x) W[s] = x[bs + s];
  __syncthreads();
  apply_P(g, W, U + (size_t)uslice * V * 2);
  for (int s = threadIdx.x; s < V; s += blockDim.x) y[bt + s] = caxpy(x[bt + s], sign * cB, W[s]);
}

template <class R>
__global__ void __launch_bounds__(1024, 1)
apply_M_kernel(Geo g, R cB, const C2<R>* __restrict__ U, const C2<R>* __restrict__ x,
               C2<R>* __restrict__ y, int dagger) {
  apply_M_slice<R>(g, cB, U, x, y, dagger, blockIdx.x);
}

// phi = M^dagger R of every chain of a batch: one CTA per (chain, slice) tile.
__global__ void __launch_bounds__(1024, 1) batch_apply_Mdag_kernel(const ChainDesc* __restrict__ descs,
                                                                   const int2* __restrict__ tiles) {
  const int2 t = tiles[blockIdx.x];
  const ChainDesc& d = descs[t.x];
  apply_M_slice<double>(d.g, d.cB, d.U64, d.R, d.eta, 1, t.y);
}

cudaError_t launch_batch_apply_Mdag(const ChainDesc* d, const int2* tiles, int ntiles, int threads, size_t smem,
                                    cudaStream_t s) {
  cudaError_t e = raise_smem_limit(batch_apply_Mdag_kernel, smem);
  if (e != cudaSuccess) return e;
  batch_apply_Mdag_kernel<<<ntiles, threads, smem, s>>>(d, tiles);
  return cudaGetLastError();
}

template <class R>
cudaError_t prepare_apply_M(const SliceLaunch& sl) {
  return raise_smem_limit(apply_M_kernel<R>, sl.g.V * sizeof(C2<R>));
}

template <class R>
cudaError_t launch_apply_M(const SliceLaunch& sl, R cB, const C2<R>* U, const C2<R>* x, C2<R>* y,
                           int dagger, cudaStream_t s) {
  apply_M_kernel<R><<<sl.g.Ntau, sl.threads, sl.g.V * sizeof(C2<R>), s>>>(sl.g, cB, U, x, y, dagger);
  return cudaGetLastError();
}

template cudaError_t launch_apply_M<double>(const SliceLaunch&, double, const double2*, const double2*, double2*, int, cudaStream_t);
template cudaError_t launch_apply_M<float>(const SliceLaunch&, float, const float2*, const float2*, float2*, int, cudaStream_t);
template cudaError_t prepare_apply_M<double>(const SliceLaunch&);
template cudaError_t prepare_apply_M<float>(const SliceLaunch&);

}  // namespace hqmc
