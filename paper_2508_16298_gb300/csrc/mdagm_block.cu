// Register-blocked fused M^dagger M (Methods, "Matrix-free representation of
// M^dagger M v"; checkerboard of Eq. (eq24)).
//
// Same mathematics and cluster structure as mdagm.cu (one CTA per slice,
// z_{tau-1} = P_{tau-1} x_{tau-1} read from the left neighbour's shared memory),
// but each thread keeps a strip of the slice in registers (strip.cuh) and
// applies whole factors there.
//
// Links: FP32 computes U = t_f e^{i theta} from a float copy of theta wrapped
// to [-pi, pi) (8 bytes per site instead of 16 for a float link table);
// FP64 reads the precomputed complex-double link table.
#include <cooperative_groups.h>

#include "strip.cuh"

namespace cg = cooperative_groups;

namespace hqmc {

__device__ __forceinline__ void bcluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void bcluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <class R, int MODE>
__device__ __forceinline__ C2<R> bload(const MdagmArgs<R>& a, const C2<R>* p_old, size_t g, R beta, bool first) {
  if (MODE == MODE_CGDIR) {
    const C2<R> rv = a.r[g];
    if (first) return rv;
    return caxpy(rv, beta, p_old[g]);
  }
  return a.x[g];
}

template <class R, int NBY>
__device__ __forceinline__ void strip_links_for(const MdagmArgs<R>& a, const StripGeo& s, int slice,
                                                StripLinks<C2<R>, NBY>& k) {
  if constexpr (sizeof(R) == 4)
    load_strip_links<NBY>(s, a.th32 + (size_t)slice * a.g.V, (float)a.t1, (float)a.t2, k);
  else
    load_strip_links<NBY>(s, a.U + (size_t)slice * a.g.V * 2, k);
}

// Block sizes that leave room for the strip in registers.
template <class R, int NBY> struct BlockThreads {
  static constexpr int max = sizeof(R) == 8 ? 640 : (NBY == 1 ? 1024 : (NBY == 2 ? 512 : 384));
};

template <class R, int MODE, int NBY>
__global__ void __launch_bounds__((BlockThreads<R, NBY>::max), 1) mdagm_block_kernel(const MdagmArgs<R> a) {
  using T = C2<R>;
  constexpr int H = 2 * NBY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int V = a.g.V, N = a.g.Ntau, L = a.g.L;
  T* Zpub = reinterpret_cast<T*>(smem_raw);  // z_tau, read by the right neighbour
  T* Zh = Zpub + V;                           // rank 0: its own z_{tau-1}
  T* E0 = Zh + V;                             // exchange buffers
  T* E1 = E0 + V;
  __shared__ double red[32];
  __shared__ int s_flags;
  __shared__ R s_beta;
  __shared__ int s_k;

  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int tau = blockIdx.x;
  const bool active = tau < N;

  if (MODE == MODE_CGDIR) {
    cgdir_head<R>(a, blockIdx.x == 0, s_flags, s_beta, s_k);
    if (s_flags & 1) return;  // uniform over the whole grid: no cluster barrier is pending
  }
  const bool first = (MODE == MODE_CGDIR) && (s_flags & 2);
  const R beta = (MODE == MODE_CGDIR) ? s_beta : R(0);
  const T* p_old = nullptr;
  T* p_new = nullptr;
  if (MODE == MODE_CGDIR) {
    p_old = (s_k & 1) ? a.pbuf[1] : a.pbuf[0];
    p_new = (s_k & 1) ? a.pbuf[0] : a.pbuf[1];
  }
  const R cB = a.cB;
  const int taum = (tau == 0) ? N - 1 : tau - 1;
  const int taup = (tau == N - 1) ? 0 : tau + 1;
  const size_t bt = (size_t)tau * V, bp = (size_t)taup * V, bm = (size_t)taum * V;
  const StripGeo sg = strip_geo<NBY>(L);
  int eb = 0;

  T v[H][2], xn[H][2];
  StripLinks<T, NBY> lk;
  if (active) {
    strip_links_for<R, NBY>(a, sg, tau, lk);
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int s = y * L + (c ? sg.x1 : sg.x0);
        v[r][c] = bload<R, MODE>(a, p_old, bt + s, beta, first);
        if (MODE == MODE_CGDIR) p_new[bt + s] = v[r][c];
        xn[r][c] = bload<R, MODE>(a, p_old, bp + s, beta, first);
      }
    }
    strip_sweep(v, lk, sg, E0, E1, eb);  // z_tau
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
      Zpub[y * L + sg.x0] = v[r][0];
      Zpub[y * L + sg.x1] = v[r][1];
    }
  }
  bcluster_arrive();  // z_tau published

  if (rank == 0 && active) {
    // halo: z_{tau-1} for the first slice of the cluster
    strip_links_for<R, NBY>(a, sg, taum, lk);
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
      v[r][0] = bload<R, MODE>(a, p_old, bm + y * L + sg.x0, beta, first);
      v[r][1] = bload<R, MODE>(a, p_old, bm + y * L + sg.x1, beta, first);
    }
    strip_sweep(v, lk, sg, E0, E1, eb);
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
      Zh[y * L + sg.x0] = v[r][0];
      Zh[y * L + sg.x1] = v[r][1];
    }
    strip_links_for<R, NBY>(a, sg, tau, lk);
  }
  bcluster_wait();
  const T* Zprev = (rank == 0) ? Zh : cl.map_shared_rank(Zpub, rank - 1);

  R acc = 0;  // FP32: the thread's few terms in float (cdot_re_own)
  if (active) {
    const R sig = (tau == 0) ? R(-1) : R(1);
    const R sigp = (tau == N - 1) ? R(-1) : R(1);
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
      v[r][0] = caxpy(cscale(cB, Zpub[y * L + sg.x0]), -sigp, xn[r][0]);
      v[r][1] = caxpy(cscale(cB, Zpub[y * L + sg.x1]), -sigp, xn[r][1]);
    }
    strip_sweep(v, lk, sg, E0, E1, eb);  // P_tau (cB z_tau - s' x_{tau+1})
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int s = y * L + (c ? sg.x1 : sg.x0);
        const T xt = (MODE == MODE_CGDIR) ? p_new[bt + s] : a.x[bt + s];
        const T q = caxpy(caxpy(xt, -sig * cB, Zprev[s]), cB, v[r][c]);
        a.y[bt + s] = q;
        if (MODE == MODE_CGDIR) acc += cdot_re_own(xt, q);
      }
    }
  }
  bcluster_arrive();  // finished reading the neighbour's shared memory
  if (MODE == MODE_CGDIR) {
    const double t0 = block_sum((double)acc, red);
    if (threadIdx.x == 0) a.part_out[blockIdx.x] = t0;
  }
  bcluster_wait();  // keep z_tau alive until the right neighbour has read it
}

template <class R, int MODE, int NBY>
static cudaError_t block_prepare(const SliceLaunch& sl) {
  return raise_smem_limit(mdagm_block_kernel<R, MODE, NBY>, 4 * sl.g.V * sizeof(C2<R>));
}

template <class R, int MODE, int NBY>
static cudaError_t block_launch(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sl.grid);
  cfg.blockDim = dim3(sl.threads);
  cfg.dynamicSmemBytes = 4 * sl.g.V * sizeof(C2<R>);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sl.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mdagm_block_kernel<R, MODE, NBY>, a);
}

template <class R, int MODE>
cudaError_t prepare_mdagm_block(const SliceLaunch& sl) {
  switch (sl.nby) {
    case 1: return block_prepare<R, MODE, 1>(sl);
    case 2: return block_prepare<R, MODE, 2>(sl);
    case 3: return block_prepare<R, MODE, 3>(sl);
    default: return cudaErrorInvalidValue;
  }
}

template <class R, int MODE>
cudaError_t launch_mdagm_block(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s) {
  switch (sl.nby) {
    case 1: return block_launch<R, MODE, 1>(sl, a, s);
    case 2: return block_launch<R, MODE, 2>(sl, a, s);
    case 3: return block_launch<R, MODE, 3>(sl, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t prepare_mdagm_block<float, MODE_APPLY>(const SliceLaunch&);
template cudaError_t prepare_mdagm_block<float, MODE_CGDIR>(const SliceLaunch&);
template cudaError_t prepare_mdagm_block<double, MODE_APPLY>(const SliceLaunch&);
template cudaError_t prepare_mdagm_block<double, MODE_CGDIR>(const SliceLaunch&);

template <class R, int NBY>
static int block_clusters(const SliceLaunch& sl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(sl.grid);
  cfg.blockDim = dim3(sl.threads);
  cfg.dynamicSmemBytes = 4 * sl.g.V * sizeof(C2<R>);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sl.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)mdagm_block_kernel<R, MODE_CGDIR, NBY>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

int mdagm_block_max_active_clusters(const SliceLaunch& sl, int real_bytes) {
  if (real_bytes == 8) return sl.nby == 1 ? block_clusters<double, 1>(sl) : -1;
  switch (sl.nby) {
    case 1: return block_clusters<float, 1>(sl);
    case 2: return block_clusters<float, 2>(sl);
    case 3: return block_clusters<float, 3>(sl);
    default: return -1;
  }
}

int block_thread_cap(int real_bytes, int nby) {
  if (real_bytes == 8) return nby == 1 ? BlockThreads<double, 1>::max : 0;  // FP64 strips of 4 sites only
  return nby == 1 ? BlockThreads<float, 1>::max : nby == 2 ? BlockThreads<float, 2>::max : BlockThreads<float, 3>::max;
}
template cudaError_t launch_mdagm_block<float, MODE_APPLY>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t launch_mdagm_block<float, MODE_CGDIR>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t launch_mdagm_block<double, MODE_APPLY>(const SliceLaunch&, const MdagmArgs<double>&, cudaStream_t);
template cudaError_t launch_mdagm_block<double, MODE_CGDIR>(const SliceLaunch&, const MdagmArgs<double>&, cudaStream_t);

}  // namespace hqmc
