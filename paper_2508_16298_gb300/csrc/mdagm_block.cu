// Register-blocked fused M^dagger M (Methods, "Matrix-free representation of
// M^dagger M v"; checkerboard of Eq. (eq24)).
//
// Same mathematics and cluster structure as mdagm.cu (one CTA per slice,
// z_{tau-1} = P_{tau-1} x_{tau-1} read from the left neighbour's shared memory),
// but each thread keeps a 2 x H strip of the slice (H = 2*NBY rows) in
// registers and applies whole factors there:
//
//   "D" alignment: columns x0 = 2i+1, x1 = 2i+2, rows base+1 .. base+H
//                  -> the family-4 bonds (odd tail y) are internal;
//   "C" alignment: the same columns, rows base .. base+H-1
//                  -> families 3 (even tail y) and 2 (odd tail x) are internal.
//
// A sweep P = F4 F3 F2 F1 F2 F3 F4 (rightmost first) is then
//   F4 [D] | shift to C | F3 F2 [C] | F1 across columns | F2 F3 [C] | shift to D | F4 [D]
// where a shift moves the strip one row (only one row crosses to the
// neighbouring thread) and F1 exchanges the strip's sites with the left and
// right neighbours.  Three shared-memory exchanges and three barriers per
// sweep replace the seven full-slice passes of the generic kernel.
//
// Links: FP32 computes U = t_f e^{i theta} from a float copy of theta wrapped
// to [-pi, pi) (8 bytes per site instead of 16 for a float link table);
// FP64 reads the precomputed complex-double link table.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace hqmc {

__device__ __forceinline__ void bcluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void bcluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Link factors of one strip (tanh of the factor angle folded in).
template <class T, int NBY>
struct StripLinks {
  T u4[NBY][2];   // family 4: y-bonds with tail on D rows 0, 2, ... (odd y)
  T u3[NBY][2];   // family 3: y-bonds with tail on C rows 0, 2, ... (even y)
  T u2[2 * NBY];  // family 2: x-bond x0 -> x1 on every C row
  T u1l[2 * NBY]; // family 1: x-bond 2i -> x0 (this strip holds its head)
  T u1r[2 * NBY]; // family 1: x-bond x1 -> 2i+3 (this strip holds its tail)
};

// Per-thread geometry of the strip.
struct StripGeo {
  int L;
  int x0, x1;  // owned columns 2i+1, (2i+2) mod L
  int xl, xr;  // columns 2i and (2i+3) mod L of the family-1 partners
  int base;    // first C row (2*jj*NBY)
  int ytop;    // last D row (base + H) mod L
};

template <int NBY>
__device__ __forceinline__ StripGeo strip_geo(int L) {
  const int Lh = L >> 1;
  const int i = threadIdx.x % Lh, jj = threadIdx.x / Lh;
  StripGeo s;
  s.L = L;
  s.x0 = 2 * i + 1;
  s.x1 = (2 * i + 2 == L) ? 0 : 2 * i + 2;
  s.xl = 2 * i;
  s.xr = (2 * i + 3 >= L) ? 2 * i + 3 - L : 2 * i + 3;
  s.base = 2 * jj * NBY;
  const int top = s.base + 2 * NBY;
  s.ytop = (top >= L) ? top - L : top;
  return s;
}

__device__ __forceinline__ int drow(const StripGeo& s, int r, int H) { return r < H - 1 ? s.base + 1 + r : s.ytop; }

template <class T>
__device__ __forceinline__ T link_from_theta(float th, float t) {
  float sn, cs;
  __sincosf(th, &sn, &cs);
  return mk(t * cs, t * sn);
}

// FP32: from theta (float2 (theta_x, theta_y) per site, wrapped to [-pi, pi)).
template <int NBY>
__device__ __forceinline__ void load_strip_links(const StripGeo& s, const float2* __restrict__ th, float t1, float t2,
                                                 StripLinks<float2, NBY>& k) {
  constexpr int H = 2 * NBY;
  const int L = s.L;
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    const int yd = drow(s, 2 * b, H), yc = s.base + 2 * b;
    k.u4[b][0] = link_from_theta<float2>(__ldg(th + yd * L + s.x0).y, t2);
    k.u4[b][1] = link_from_theta<float2>(__ldg(th + yd * L + s.x1).y, t2);
    k.u3[b][0] = link_from_theta<float2>(__ldg(th + yc * L + s.x0).y, t2);
    k.u3[b][1] = link_from_theta<float2>(__ldg(th + yc * L + s.x1).y, t2);
  }
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int yc = s.base + r;
    k.u2[r] = link_from_theta<float2>(__ldg(th + yc * L + s.x0).x, t2);
    k.u1l[r] = link_from_theta<float2>(__ldg(th + yc * L + s.xl).x, t1);
    k.u1r[r] = link_from_theta<float2>(__ldg(th + yc * L + s.x1).x, t1);
  }
}

// FP64: from the link table (two complex links per site, t_f folded in).
template <int NBY>
__device__ __forceinline__ void load_strip_links(const StripGeo& s, const double2* __restrict__ U,
                                                 StripLinks<double2, NBY>& k) {
  constexpr int H = 2 * NBY;
  const int L = s.L;
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    const int yd = drow(s, 2 * b, H), yc = s.base + 2 * b;
    k.u4[b][0] = __ldg(U + 2 * (yd * L + s.x0) + 1);
    k.u4[b][1] = __ldg(U + 2 * (yd * L + s.x1) + 1);
    k.u3[b][0] = __ldg(U + 2 * (yc * L + s.x0) + 1);
    k.u3[b][1] = __ldg(U + 2 * (yc * L + s.x1) + 1);
  }
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int yc = s.base + r;
    k.u2[r] = __ldg(U + 2 * (yc * L + s.x0));
    k.u1l[r] = __ldg(U + 2 * (yc * L + s.xl));
    k.u1r[r] = __ldg(U + 2 * (yc * L + s.x1));
  }
}

// (vi, vj) <- (vi + u vj, vj + conj(u) vi)
template <class T>
__device__ __forceinline__ void bond2(T& vi, T& vj, const T& u) {
  const T a = vi, b = vj;
  vi = cfma(a, u, b);
  vj = cfmac(b, u, a);
}

// v <- P v on the strip; v is in D alignment on entry and exit.
template <class T, int NBY>
__device__ __forceinline__ void strip_sweep(T (&v)[2 * NBY][2], const StripLinks<T, NBY>& k, const StripGeo& s,
                                            T* __restrict__ E0, T* __restrict__ E1, int& eb) {
  constexpr int H = 2 * NBY;
  const int L = s.L;
  // F4 in D
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    bond2(v[2 * b][0], v[2 * b + 1][0], k.u4[b][0]);
    bond2(v[2 * b][1], v[2 * b + 1][1], k.u4[b][1]);
  }
  // D -> C: hand the last D row up, take C row 0 from the strip below
  {
    T* E = eb ? E1 : E0;
    eb ^= 1;
    E[s.ytop * L + s.x0] = v[H - 1][0];
    E[s.ytop * L + s.x1] = v[H - 1][1];
    __syncthreads();
#pragma unroll
    for (int r = H - 1; r > 0; --r) {
      v[r][0] = v[r - 1][0];
      v[r][1] = v[r - 1][1];
    }
    v[0][0] = E[s.base * L + s.x0];
    v[0][1] = E[s.base * L + s.x1];
  }
  // F3, F2 in C
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    bond2(v[2 * b][0], v[2 * b + 1][0], k.u3[b][0]);
    bond2(v[2 * b][1], v[2 * b + 1][1], k.u3[b][1]);
  }
#pragma unroll
  for (int r = 0; r < H; ++r) bond2(v[r][0], v[r][1], k.u2[r]);
  // F1 across columns: x0 is the head of (2i -> x0), x1 the tail of (x1 -> 2i+3)
  {
    T* E = eb ? E1 : E0;
    eb ^= 1;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      E[(s.base + r) * L + s.x0] = v[r][0];
      E[(s.base + r) * L + s.x1] = v[r][1];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const T pl = E[(s.base + r) * L + s.xl];
      const T pr = E[(s.base + r) * L + s.xr];
      v[r][0] = cfmac(v[r][0], k.u1l[r], pl);
      v[r][1] = cfma(v[r][1], k.u1r[r], pr);
    }
  }
  // F2, F3 in C
#pragma unroll
  for (int r = 0; r < H; ++r) bond2(v[r][0], v[r][1], k.u2[r]);
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    bond2(v[2 * b][0], v[2 * b + 1][0], k.u3[b][0]);
    bond2(v[2 * b][1], v[2 * b + 1][1], k.u3[b][1]);
  }
  // C -> D: hand C row 0 down, take the last D row from the strip above
  {
    T* E = eb ? E1 : E0;
    eb ^= 1;
    E[s.base * L + s.x0] = v[0][0];
    E[s.base * L + s.x1] = v[0][1];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < H - 1; ++r) {
      v[r][0] = v[r + 1][0];
      v[r][1] = v[r + 1][1];
    }
    v[H - 1][0] = E[s.ytop * L + s.x0];
    v[H - 1][1] = E[s.ytop * L + s.x1];
  }
  // F4 in D
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    bond2(v[2 * b][0], v[2 * b + 1][0], k.u4[b][0]);
    bond2(v[2 * b][1], v[2 * b + 1][1], k.u4[b][1]);
  }
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
    if (threadIdx.x < 32) {
      CgState* st = a.st;
      const int lane = threadIdx.x;
      const int done = *(volatile int*)&st->done;
      const int k = *(volatile int*)&st->k;
      const int seg = st->seg_start;
      int flags = 0;
      double beta = 0.0;
      int new_done = CG_RUNNING;
      if (done != CG_RUNNING) {
        flags = 1;
      } else if (k >= st->maxit) {
        flags = 1;
        new_done = CG_MAXIT;
      } else if (k == seg) {
        flags = 2;
      } else {
        const double rr = warp_sum_partials(a.part_in, a.n_part_in);
        if (!isfinite(rr)) {
          flags = 1;
          new_done = CG_NONFINITE;
        } else if (rr <= st->tol2bb) {
          flags = 1;
          new_done = CG_REC_CONVERGED;
        } else {
          beta = rr / st->rr[(k - 1) & 1];
        }
        if (blockIdx.x == 0 && lane == 0) st->rr[k & 1] = rr;
      }
      if (blockIdx.x == 0 && lane == 0) {
        if (new_done != CG_RUNNING) st->done = new_done;
        if (!(flags & 1)) st->k2 = k;
      }
      if (lane == 0) {
        s_flags = flags;
        s_beta = (R)beta;
        s_k = k;
      }
    }
    __syncthreads();
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

  double acc = 0.0;
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
        if (MODE == MODE_CGDIR) acc += cdot_re(xt, q);
      }
    }
  }
  bcluster_arrive();  // finished reading the neighbour's shared memory
  if (MODE == MODE_CGDIR) {
    const double t0 = block_sum(acc, red);
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
