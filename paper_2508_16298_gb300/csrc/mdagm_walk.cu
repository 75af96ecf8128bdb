// Persistent tau-walking fused M^dagger M in FP32 (Methods, "Matrix-free
// representation of M^dagger M v"; checkerboard of Eq. (eq24)).
//
// With B_tau = cB P_tau and z_tau = P_tau x_tau, row tau of M^dagger M is
//   y_tau = t_tau + cB P_tau w_tau,
//   t_tau = x_tau - s_tau cB z_{tau-1},   w_tau = cB z_tau - s'_tau x_{tau+1},
// (s_0 = -1 and s'_{Ntau-1} = -1 carry the antiperiodic wrap; all others +1).
// Each CTA owns a contiguous range [tb, te) of slices and walks it in order, so
// the z_{tau-1} that row tau needs is the one it computed in the previous
// step: a range of n slices costs 2n + 1 sweeps (one halo sweep at tb - 1) and
// no inter-CTA exchange.  The slice is held in register strips (strip.cuh).
//
// Memory: step j reads theta_j and the vector slices at j + 1 once, through a
// bulk asynchronous copy (cp.async.bulk, completion on an mbarrier) into a
// shared-memory stage.  Each thread copies what it needs out of the stage
// (its links and x_{j+1}), then one thread refills the stage for step j + 1
// while the block runs the two sweeps of step j, so HBM streams under the
// compute.  The vector read for the halo row tb - 1 is the only direct load.
// The first stage and the halo row are requested before the CG-direction head
// sums the previous kernels' partials, so that latency overlaps the copy.
//
// CG-direction mode forms p = r + beta p_old on the fly, writes p and q = O p,
// and accumulates <p, q> = Re sum_tau [<x_tau, t_tau> + cB <z_tau, w_tau>]
// (P is Hermitian, so <x, P w> = <P x, w>), one partial per CTA.
//
// Waits on the mbarrier are bounded (about one second of %globaltimer); on a
// timeout the block writes NaN into its outputs and sets the config's device
// error word, so the solve returns HQMC_ETIMEOUT instead of hanging.
#include "bulk.cuh"
#include "strip.cuh"

namespace hqmc {

// Block sizes that leave room for the strip in registers.
template <int NBY> struct WalkThreads {
  static constexpr int max = NBY == 1 ? 768 : (NBY == 2 ? 512 : 384);
};

int walk_thread_cap(int nby) {
  return nby == 1 ? WalkThreads<1>::max : nby == 2 ? WalkThreads<2>::max : nby == 3 ? WalkThreads<3>::max : 0;
}

// Shared memory: stage (theta + 1 or 2 vector slices), x_{j+1} copy, 2 exchange buffers.
size_t walk_smem_bytes(const Geo& g, int mode) {
  const int nv = mode == MODE_CGDIR ? 2 : 1;
  return (size_t)(1 + nv + 1 + 2) * g.V * sizeof(float2);
}

// MULTI: one launch over ms.nsys systems that share theta (launch_mdagm_walk_multi):
// CTA b walks slice range b / nsys of system b % nsys, so the CTAs resident at one
// time read the same theta slices, and each system's ranges are longer than in a
// one-system launch of the same grid (fewer halo sweeps per slice).
template <int MODE, int NBY, bool MULTI>
__global__ void __launch_bounds__(WalkThreads<NBY>::max, 1) mdagm_walk_kernel(const MdagmArgs<float> a,
                                                                                    const MultiStride ms) {
  using T = float2;
  constexpr int H = 2 * NBY;
  constexpr int NV = MODE == MODE_CGDIR ? 2 : 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int V = a.g.V, N = a.g.Ntau, L = a.g.L;
  float2* Sth = reinterpret_cast<float2*>(smem_raw);  // stage: theta_j
  T* Sv0 = Sth + V;                                   // stage: x_{j+1}, or r_{j+1}
  T* Sv1 = Sv0 + V;                                   // stage (CG direction): p_old_{j+1}
  T* X1 = Sv0 + NV * V;                               // x_{j+1}, each thread's own sites (slot-major)
  T* E0 = X1 + V;                                     // exchange buffers
  T* E1 = E0 + V;
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[32];
  __shared__ int s_flags;
  __shared__ float s_beta;
  __shared__ int s_k;

  // This CTA's system and slice range (MULTI), else the launch's only system.
  const int sys = MULTI ? (int)(blockIdx.x % (unsigned)ms.nsys) : 0;
  const int rng = MULTI ? (int)(blockIdx.x / (unsigned)ms.nsys) : (int)blockIdx.x;
  const int G = MULTI ? (int)(gridDim.x / (unsigned)ms.nsys) : gridDim.x;
  const size_t voff = MULTI ? (size_t)sys * (size_t)ms.vstride : 0;
  const size_t poff = MULTI ? (size_t)sys * (size_t)ms.pstride : 0;
  CgState* const st = MULTI ? a.st + sys : a.st;
#define WALK_Y (MULTI ? a.y + voff : a.y)

  // The direction buffers follow the iteration count k, which no kernel changes
  // while this one runs (the update kernel advances it): iteration k reads
  // pbuf[k & 1] and writes pbuf[(k + 1) & 1].  Read here, before the head.
  const int k0 = MODE == MODE_CGDIR ? *(volatile const int*)&st->k : 0;
  const T* p_old = nullptr;
  T* p_new = nullptr;
  if (MODE == MODE_CGDIR) {
    p_old = ((k0 & 1) ? a.pbuf[1] : a.pbuf[0]) + voff;
    p_new = ((k0 & 1) ? a.pbuf[0] : a.pbuf[1]) + voff;
  }
  const T* vsrc = (MODE == MODE_CGDIR ? a.r : a.x) + voff;

  const int tb = MULTI ? (int)((long long)rng * N / G) : (int)((long long)blockIdx.x * N / G);
  const int te = MULTI ? (int)((long long)(rng + 1) * N / G) : (int)((long long)(blockIdx.x + 1) * N / G);
  auto wrap = [N](int j) { return j < 0 ? j + N : (j >= N ? j - N : j); };

  // The stage always carries p_old in CG-direction mode (ignored on the first
  // iteration of a segment), so its size does not wait for the head.
  const uint32_t slice_bytes = (uint32_t)V * (uint32_t)sizeof(T);
  const uint32_t stage_bytes = slice_bytes * (MODE == MODE_CGDIR ? 3 : 2);
  auto issue = [&](int j) {  // stage of step j: theta_j and the vectors of slice j + 1
    const size_t sj = (size_t)wrap(j) * V, sn = (size_t)wrap(j + 1) * V;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&bar, stage_bytes);
    bulk_load(Sth, a.th32 + sj, slice_bytes, &bar);
    bulk_load(Sv0, vsrc + sn, slice_bytes, &bar);
    if (MODE == MODE_CGDIR) bulk_load(Sv1, p_old + sn, slice_bytes, &bar);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    issue(tb - 1);
  }

  const StripGeo sg = strip_geo<NBY>(L);
  T v[H][2], t[H][2];
  {  // x_{tb-1}, the halo row: r (or x) and p_old requested before the head
    const size_t base = (size_t)wrap(tb - 1) * V;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const size_t gi = base + y * L + (c ? sg.x1 : sg.x0);
        v[r][c] = vsrc[gi];
        if (MODE == MODE_CGDIR) t[r][c] = p_old[gi];
      }
    }
  }
  if (MODE == MODE_CGDIR) {
    cgdir_head_at<float>(a, rng == 0, s_flags, s_beta, s_k, st, a.part_in + poff,
                         a.part_rz ? a.part_rz + poff : nullptr, a.part_cross ? a.part_cross + poff : nullptr);
    if (s_flags & 1) {  // uniform over the grid; the stage in flight lands before the block exits
      if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0);
      return;
    }
  }
  const bool first = (MODE == MODE_CGDIR) && (s_flags & 2);
  const float beta = (MODE == MODE_CGDIR) ? s_beta : 0.f;
  if (MODE == MODE_CGDIR && !first) {  // p of the halo row, formed exactly as its owner forms it
#pragma unroll
    for (int r = 0; r < H; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) v[r][c] = caxpy(v[r][c], beta, t[r][c]);
  }
  const float cB = a.cB;
  const float t1 = (float)a.t1, t2 = (float)a.t2;
  int eb = 0;
  StripLinks<T, NBY> lk;
  double acc = 0.0;
  __syncthreads();  // the mbarrier is initialised before anyone waits on it

  uint32_t parity = 0;
  bool ok = true;
  // The stage is copied out cooperatively in slice order: thread (jj, i) of the
  // Lh x S block takes the 16-byte pair of columns (2i, 2i+1) in rows jj + m S
  // (m < H), conflict-free, and writes each site into the X1 slot of its owner:
  // column 2i is column x1 of thread i - 1 (of thread Lh - 1 for i = 0), column
  // 2i + 1 is column x0 of thread i, and row y is D row r of strip jo with
  // y - 1 = jo H + r (mod L).  In CG-direction mode the pass forms p = r + beta p_old
  // and writes p_new for the block's own slices.
  for (int j = tb - 1; j < te; ++j) {
    ok = ok && mbar_wait_bounded(&bar, parity);
    parity ^= 1;
    __syncthreads();  // every thread has read its X1 slots of the previous step
    if (ok) {
      float4* pn = reinterpret_cast<float4*>(p_new + (size_t)wrap(j + 1) * V);
      const float4* r4 = reinterpret_cast<const float4*>(Sv0);
      const float4* o4 = reinterpret_cast<const float4*>(Sv1);
      const bool own = j + 1 < te;
      const int Lh = sg.Lh, S = L / H, y0 = sg.base / H;  // this thread: column pair sg.i of rows y0 + m S
#pragma unroll 1
      for (int m = 0; m < H; ++m) {
        const int y = y0 + m * S;
        const int e = y * Lh + sg.i;
        float4 v = r4[e];
        if (MODE == MODE_CGDIR) {
          if (!first) {
            const float4 o = o4[e];
            v = make_float4(fmaf(beta, o.x, v.x), fmaf(beta, o.y, v.y), fmaf(beta, o.z, v.z), fmaf(beta, o.w, v.w));
          }
          if (own) pn[e] = v;
        }
        const int yp = (y == 0) ? L - 1 : y - 1;
        const int jo = yp / H, r = yp - jo * H;
        X1[(2 * r + 1) * blockDim.x + jo * Lh + sg.il] = make_float2(v.x, v.y);  // column 2i
        X1[(2 * r) * blockDim.x + jo * Lh + sg.i] = make_float2(v.z, v.w);       // column 2i + 1
      }
      load_strip_links_smem<NBY>(sg, Sth, t1, t2, lk);
    }
    if (!__syncthreads_and(ok)) {  // uniform: every thread leaves together
      ok = false;
      break;
    }
    if (threadIdx.x == 0 && j + 1 < te) issue(j + 1);

    float accj = 0.f;  // this step's terms, in float (cdot_re_own)
    if (MODE == MODE_CGDIR && j >= tb) {
#pragma unroll
      for (int r = 0; r < H; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) accj += cdot_re_own(v[r][c], t[r][c]);
    }
    strip_sweep(v, lk, sg, E0, E1, eb);  // z_j
    const float sn = (wrap(j + 1) == 0) ? -1.f : 1.f;  // s_{j+1}
    if (j < tb) {  // halo step: only t_{tb} is needed
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const int y = drow(sg, r, H);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const T xn = X1[(2 * r + c) * blockDim.x + threadIdx.x];
          t[r][c] = caxpy(xn, -sn * cB, v[r][c]);
          v[r][c] = xn;
        }
      }
      continue;
    }
    const float sp = (wrap(j) == N - 1) ? -1.f : 1.f;  // s'_j
    T tn[H][2];
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T xn = X1[(2 * r + c) * blockDim.x + threadIdx.x];
        const T w = caxpy(cscale(cB, v[r][c]), -sp, xn);
        if (MODE == MODE_CGDIR) accj += cB * cdot_re_own(v[r][c], w);
        tn[r][c] = caxpy(xn, -sn * cB, v[r][c]);
        v[r][c] = w;
      }
    }
    strip_sweep(v, lk, sg, E0, E1, eb);  // P_j w_j
    const size_t bj = (size_t)wrap(j) * V;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int y = drow(sg, r, H);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int s = y * L + (c ? sg.x1 : sg.x0);
        WALK_Y[bj + s] = caxpy(t[r][c], cB, v[r][c]);
        t[r][c] = tn[r][c];
        v[r][c] = X1[(2 * r + c) * blockDim.x + threadIdx.x];
      }
    }
    acc += (double)accj;
  }

  if (!ok) {
    // A stage never arrived: poison this block's outputs so the caller sees a
    // non-finite result, then give the copy in flight a bounded chance to land.
    const T nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    for (int j = tb; j < te; ++j)
      for (int s = threadIdx.x; s < V; s += blockDim.x) WALK_Y[(size_t)j * V + s] = nan2;
    acc = __longlong_as_double(0x7ff8000000000000ll);
    if (a.err && threadIdx.x == 0) atomicExch(a.err, 1);  // the host reports HQMC_ETIMEOUT
    mbar_wait_bounded(&bar, parity ^ 1);
  }
  if (MODE == MODE_CGDIR) {
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) a.part_out[poff + rng] = tot;
  }
#undef WALK_Y
}

template <int MODE, int NBY, bool MULTI = false>
static cudaError_t walk_launch(const SliceLaunch& sl, const MdagmArgs<float>& a, cudaStream_t s,
                               const MultiStride ms = MultiStride{1, 0, 0}) {
  const size_t smem = walk_smem_bytes(sl.g, MODE);
  const int grid = MULTI ? sl.grid * ms.nsys : sl.grid;
  mdagm_walk_kernel<MODE, NBY, MULTI><<<grid, sl.threads, smem, s>>>(a, ms);
  return cudaGetLastError();
}

template <int MODE, int NBY, bool MULTI = false>
static cudaError_t walk_prepare(const SliceLaunch& sl) {
  return raise_smem_limit(mdagm_walk_kernel<MODE, NBY, MULTI>, walk_smem_bytes(sl.g, MODE));
}

template <int MODE>
cudaError_t launch_mdagm_walk(const SliceLaunch& sl, const MdagmArgs<float>& a, cudaStream_t s) {
  if (sl.grid < 1 || sl.grid > sl.g.Ntau) return cudaErrorInvalidValue;
  switch (sl.nby) {
    case 1: return walk_launch<MODE, 1>(sl, a, s);
    case 2: return walk_launch<MODE, 2>(sl, a, s);
    case 3: return walk_launch<MODE, 3>(sl, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
cudaError_t prepare_mdagm_walk(const SliceLaunch& sl) {
  switch (sl.nby) {
    case 1: return walk_prepare<MODE, 1>(sl);
    case 2: return walk_prepare<MODE, 2>(sl);
    case 3: return walk_prepare<MODE, 3>(sl);
    default: return cudaErrorInvalidValue;
  }
}

// CTAs of this shape the device keeps resident per SM (0: none fit).
int mdagm_walk_blocks_per_sm(const SliceLaunch& sl) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const size_t smem = walk_smem_bytes(sl.g, MODE_CGDIR);
  switch (sl.nby) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 1, false>, sl.threads, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 2, false>, sl.threads, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 3, false>, sl.threads, smem); break;
    default: break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Multi-system CG-direction launch: sl.grid slice ranges per system, a.nsys systems.
cudaError_t launch_mdagm_walk_multi(const SliceLaunch& sl, const MdagmArgs<float>& a, const MultiStride& ms,
                                    cudaStream_t s) {
  if (sl.grid < 1 || sl.grid > sl.g.Ntau || ms.nsys < 1 || (long long)sl.grid * ms.nsys > (1ll << 30))
    return cudaErrorInvalidValue;
  switch (sl.nby) {
    case 1: return walk_launch<MODE_CGDIR, 1, true>(sl, a, s, ms);
    case 2: return walk_launch<MODE_CGDIR, 2, true>(sl, a, s, ms);
    case 3: return walk_launch<MODE_CGDIR, 3, true>(sl, a, s, ms);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_mdagm_walk_multi(const SliceLaunch& sl) {
  switch (sl.nby) {
    case 1: return walk_prepare<MODE_CGDIR, 1, true>(sl);
    case 2: return walk_prepare<MODE_CGDIR, 2, true>(sl);
    case 3: return walk_prepare<MODE_CGDIR, 3, true>(sl);
    default: return cudaErrorInvalidValue;
  }
}

// CTAs of the multi-system kernel the device keeps resident per SM (0: none fit).
int mdagm_walk_multi_blocks_per_sm(const SliceLaunch& sl) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const size_t smem = walk_smem_bytes(sl.g, MODE_CGDIR);
  switch (sl.nby) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 1, true>, sl.threads, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 2, true>, sl.threads, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mdagm_walk_kernel<MODE_CGDIR, 3, true>, sl.threads, smem); break;
    default: break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template cudaError_t launch_mdagm_walk<MODE_APPLY>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t launch_mdagm_walk<MODE_CGDIR>(const SliceLaunch&, const MdagmArgs<float>&, cudaStream_t);
template cudaError_t prepare_mdagm_walk<MODE_APPLY>(const SliceLaunch&);
template cudaError_t prepare_mdagm_walk<MODE_CGDIR>(const SliceLaunch&);

}  // namespace hqmc
