// Element-wise and reduction kernels of the HQMC path: link tables, the CG
// vector update (Eq. (pCG)), residual bookkeeping, leapfrog kicks and drifts
// (Eq. (leapfrog)), the Hamiltonian terms of Eq. (H_hmc) and the Gaussian
// draws of HQMC step (i).
#include "kernels.h"

namespace hqmc {

static inline int ew_blocks(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Link tables: U[site][c] = t_f e^{i theta}, t1 = tanh(a) for x-bonds with even
// tail x (family 1, the merged middle factor), t2 = tanh(a/2) for all others.
__device__ __forceinline__ void links_site(const Geo& g, const double* __restrict__ theta, double t1, double t2,
                                           double2* __restrict__ U64, float2* __restrict__ U32,
                                           float2* __restrict__ th32, long long i);

__global__ void links_kernel(Geo g, const double* __restrict__ theta, double t1, double t2,
                             double2* __restrict__ U64, float2* __restrict__ U32, float2* __restrict__ th32,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    links_site(g, theta, t1, t2, U64, U32, th32, i);
}

__device__ __forceinline__ void links_site(const Geo& g, const double* __restrict__ theta, double t1, double t2,
                                           double2* __restrict__ U64, float2* __restrict__ U32,
                                           float2* __restrict__ th32, long long i) {
  {
    const int s = (int)(i % g.V);
    const int x = s % g.L;
    const double2 th = reinterpret_cast<const double2*>(theta)[i];
    if (U64 || U32) {  // FP64 sincos is costly on this GPU: only when a link table is wanted
      double sx, cx, sy, cy;
      sincos(th.x, &sx, &cx);
      sincos(th.y, &sy, &cy);
      const double tx = (x & 1) ? t2 : t1;
      const double2 ux = make_double2(tx * cx, tx * sx);
      const double2 uy = make_double2(t2 * cy, t2 * sy);
      if (U64) {
        U64[2 * i] = ux;
        U64[2 * i + 1] = uy;
      }
      if (U32) {
        U32[2 * i] = make_float2((float)ux.x, (float)ux.y);
        U32[2 * i + 1] = make_float2((float)uy.x, (float)uy.y);
      }
    }
    if (th32) {
      // 2 pi periodicity of the links: wrap before rounding to float (any
      // representative of theta mod 2 pi gives the same link)
      const double w = 6.283185307179586, iw = 0.15915494309189535;
      th32[i] = make_float2((float)(th.x - w * rint(th.x * iw)), (float)(th.y - w * rint(th.y * iw)));
    }
  }
}

cudaError_t launch_links(const Geo& g, const double* theta, double t1, double t2, double2* U64,
                         float2* U32, float2* th32, cudaStream_t s) {
  const long long n = (long long)g.V * g.Ntau;
  links_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(g, theta, t1, t2, U64, U32, th32, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CG update: alpha = <r,r>/<p,Op>; x += alpha p; r -= alpha Op; partial <r,r>.
// Body of the CG update for block j of nblocks serving one chain.
// voff: element offset added to every vector access (one system of several stored
// back to back; 0 otherwise).
template <class R>
__device__ __forceinline__ void cg_update_body(const UpdArgs<R>& u, const int j, const int nblocks,
                                               const size_t voff = 0) {
  __shared__ double red[32];
  __shared__ int s_stop;
  __shared__ double s_alpha;
  __shared__ int s_k;
  CgState* st = u.st;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int done = *(volatile int*)&st->done;
    int stop = 0;
    double alpha = 0.0;
    if (done != CG_RUNNING) {
      stop = 1;
    } else {
      const int k = st->k2;
      const double pq = warp_sum_partials(u.part_pq, u.n_pq);
      const double rr = st->rr[k & 1];
      if (!isfinite(pq) || !(pq > 0.0)) {
        stop = 1;
        if (j == 0 && lane == 0) st->done = isfinite(pq) ? CG_BREAKDOWN : CG_NONFINITE;
      } else {
        alpha = rr / pq;
        if (j == 0 && lane == 0) {
          st->pq_last = pq;
          st->alpha_last = alpha;
        }
      }
    }
    if (lane == 0) {
      s_stop = stop;
      s_alpha = alpha;
      s_k = st->k2;
    }
  }
  __syncthreads();
  if (s_stop) return;
  const R alpha = (R)s_alpha;
  const C2<R>* __restrict__ p = ((s_k + 1) & 1) ? u.p1 : u.p0;
  R acc = 0;  // FP32: a thread's few terms in float (cdot_re_own)
  for (long long i = j * (long long)blockDim.x + threadIdx.x; i < u.n; i += (long long)nblocks * blockDim.x) {
    const C2<R> pv = p[voff + i];
    C2<R> rv = caxpy(u.r[voff + i], -alpha, u.q[voff + i]);
    u.r[voff + i] = rv;
    if (u.x_is_double) {
      double2* xd = reinterpret_cast<double2*>(u.x);
      xd[voff + i] = caxpy(xd[voff + i], (double)alpha, make_double2(pv.x, pv.y));
    } else {
      float2* xf = reinterpret_cast<float2*>(u.x);
      xf[voff + i] = caxpy(xf[voff + i], (float)alpha, make_float2(pv.x, pv.y));
    }
    acc += cdot_re_own(rv, rv);
  }
  const double t = block_sum((double)acc, red);
  if (threadIdx.x == 0) {
    u.part_rr[j] = t;
    if (j == 0) st->k = st->k2 + 1;
  }
}

template <class R>
__global__ void __launch_bounds__(256) cg_update_kernel(const UpdArgs<R> u) {
  cg_update_body<R>(u, blockIdx.x, gridDim.x);
}

// Many chains in one launch: block b serves (chain, local block) = blocks[b];
// each chain keeps the block count and element mapping of its own launch.
template <class R>
__global__ void __launch_bounds__(256) cg_update_batch_kernel(const UpdArgs<R>* __restrict__ descs,
                                                             const int2* __restrict__ blocks,
                                                             const int* __restrict__ nblocks) {
  const int2 b = blocks[blockIdx.x];
  cg_update_body<R>(descs[b.x], b.y, nblocks[b.x]);
}

template <class R>
cudaError_t launch_cg_update(long long n, int grid, void* x, int x_is_double, C2<R>* r,
                             C2<R>* const pbuf[2], const C2<R>* q, const double* part_pq, int n_pq,
                             double* part_rr, CgState* st, cudaStream_t s) {
  UpdArgs<R> u{n, x, x_is_double, r, pbuf[0], pbuf[1], q, part_pq, n_pq, part_rr, st};
  cg_update_kernel<R><<<grid, 256, 0, s>>>(u);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_batch(const void* descs, const int2* blocks, const int* nblocks, int total_blocks,
                                   cudaStream_t s) {
  cg_update_batch_kernel<double><<<total_blocks, 256, 0, s>>>((const UpdArgs<double>*)descs, blocks, nblocks);
  return cudaGetLastError();
}

// Systems stored back to back (FP32 mixed solve): block (j, k) is block j of system
// k, whose vectors start k vstride elements, partials k pstride doubles and state k
// states after system 0's.  The vector pointers stay system 0's (kernel parameters)
// with the offset added at each access, so the element loop reads no descriptor and
// holds no extra pointers.
__global__ void __launch_bounds__(256) cg_update_multi_kernel(const UpdArgs<float> base, long long vstride,
                                                              int pstride) {
  const size_t k = blockIdx.y;
  UpdArgs<float> u = base;
  u.part_pq = base.part_pq + k * pstride;
  u.part_rr = base.part_rr + k * pstride;
  u.st = base.st + k;
  cg_update_body<float>(u, blockIdx.x, gridDim.x, k * (size_t)vstride);
}

cudaError_t launch_cg_update_multi(const UpdArgs<float>& base, long long vstride, int pstride, int nsys,
                                   int blocks_per_system, cudaStream_t s) {
  if (nsys < 1 || nsys > 65535 || blocks_per_system < 1 || base.x_is_double) return cudaErrorInvalidValue;
  cg_update_multi_kernel<<<dim3(blocks_per_system, nsys), 256, 0, s>>>(base, vstride, pstride);
  return cudaGetLastError();
}

int cg_update_multi_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cg_update_multi_kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
template cudaError_t launch_cg_update<double>(long long, int, void*, int, double2*, double2* const[2],
                                              const double2*, const double*, int, double*, CgState*,
                                              cudaStream_t);
template cudaError_t launch_cg_update<float>(long long, int, void*, int, float2*, float2* const[2],
                                             const float2*, const double*, int, double*, CgState*,
                                             cudaStream_t);

// ---------------------------------------------------------------------------
// Residual bookkeeping after r = b - O x (partials: <r,r> then <b,b>).
//  START:    new solve; sets bb, tol2bb, k = seg_start = 0, rr[0].
//  RESTART:  new recurrence segment from the true residual (FP64 solver).
//  RELIABLE: keep the search direction; hand <r,r> to the next direction step
//            through the update-kernel partial slots (mixed solver).
//  REPORT:   only report ||r||/||b|| (final check after maxit).
__global__ void resid_finalize_kernel(const double* __restrict__ part, int n, int mode, double tol,
                                      int maxit, double* __restrict__ part_rr_out, int n_rr_out,
                                      CgState* st, double* report, int gate) {
  __shared__ int s_open;
  if (threadIdx.x == 0) s_open = gate_open(gate, *(volatile int*)&st->done);
  __syncthreads();
  if (!s_open) return;
  const double rr = warp_sum_partials(part, n);
  const double bb = warp_sum_partials(part + n, n);
  if (mode == FIN_RELIABLE)
    for (int k = 1 + threadIdx.x; k < n_rr_out; k += blockDim.x) part_rr_out[k] = 0.0;
  if (threadIdx.x != 0) return;
  if (report) {
    report[0] = rr;
    report[1] = bb;
  }
  if (mode == FIN_START) {
    st->bb = bb;
    st->tol2bb = tol * tol * bb;
    st->k = 0;
    st->k2 = 0;
    st->seg_start = 0;
    st->maxit = maxit;
    st->rr[0] = rr;
    st->rr[1] = rr;
    st->pq_last = 0.0;
    st->alpha_last = 0.0;
    st->loops = 0;
    st->n_rel = 0;
    st->loop_cap = (maxit > (1 << 29) ? (1 << 30) : 2 * maxit) + 64;
    if (!isfinite(rr) || !isfinite(bb)) st->done = CG_NONFINITE;
    else if (bb == 0.0 || rr <= st->tol2bb) st->done = CG_CONVERGED;
    else if (maxit <= 0) st->done = CG_MAXIT;
    else st->done = CG_RUNNING;
  } else if (mode == FIN_RESTART || mode == FIN_RELIABLE) {
    const int k = st->k;
    if (mode == FIN_RESTART) {
      st->seg_start = k;
      st->rr[k & 1] = rr;
    } else {
      part_rr_out[0] = rr;
    }
    bool stalled = false;
    if (mode == FIN_RELIABLE) {
      const int nr = st->n_rel;
      stalled = nr >= 8 && rr > 0.25 * st->rr_rel[nr & 7];
      st->rr_rel[nr & 7] = rr;
      st->n_rel = nr + 1;
    }
    // the iteration budget is the one set at the start of the solve
    if (!isfinite(rr)) st->done = CG_NONFINITE;
    else if (rr <= st->tol2bb) st->done = CG_CONVERGED;
    else if (k >= st->maxit) st->done = CG_MAXIT;
    else if (stalled) st->done = CG_STAGNATED;
    else st->done = CG_RUNNING;
  }
}

cudaError_t launch_resid_finalize(const double* part, int n, int mode, double tol, int maxit,
                                  double* part_rr_out, int n_rr_out, CgState* st, double* report,
                                  int gate, cudaStream_t s) {
  resid_finalize_kernel<<<1, 256, 0, s>>>(part, n, mode, tol, maxit, part_rr_out, n_rr_out, st, report, gate);
  return cudaGetLastError();
}

// One block per chain; the same bookkeeping as resid_finalize_kernel.
__global__ void resid_finalize_batch_kernel(const FinArgs* __restrict__ descs, int mode, double tol, int maxit,
                                            int gate) {
  const FinArgs f = descs[blockIdx.x];
  __shared__ int s_open;
  if (threadIdx.x == 0) s_open = gate_open(gate, *(volatile int*)&f.st->done);
  __syncthreads();
  if (!s_open) return;
  const double rr = warp_sum_partials(f.part, f.n);
  const double bb = warp_sum_partials(f.part + f.n, f.n);
  if (mode == FIN_RELIABLE)
    for (int k = 1 + threadIdx.x; k < f.n_rr_out; k += blockDim.x) f.part_rr_out[k] = 0.0;
  if (threadIdx.x != 0) return;
  CgState* st = f.st;
  if (f.report) {
    f.report[0] = rr;
    f.report[1] = bb;
  }
  if (mode == FIN_START) {
    st->bb = bb;
    st->tol2bb = tol * tol * bb;
    st->k = 0;
    st->k2 = 0;
    st->seg_start = 0;
    st->maxit = maxit;
    st->rr[0] = rr;
    st->rr[1] = rr;
    st->pq_last = 0.0;
    st->alpha_last = 0.0;
    st->loops = 0;
    st->n_rel = 0;
    st->loop_cap = (maxit > (1 << 29) ? (1 << 30) : 2 * maxit) + 64;
    if (!isfinite(rr) || !isfinite(bb)) st->done = CG_NONFINITE;
    else if (bb == 0.0 || rr <= st->tol2bb) st->done = CG_CONVERGED;
    else if (maxit <= 0) st->done = CG_MAXIT;
    else st->done = CG_RUNNING;
  } else if (mode == FIN_RESTART) {
    const int k = st->k;
    st->seg_start = k;
    st->rr[k & 1] = rr;
    if (!isfinite(rr)) st->done = CG_NONFINITE;
    else if (rr <= st->tol2bb) st->done = CG_CONVERGED;
    else if (k >= st->maxit) st->done = CG_MAXIT;
    else st->done = CG_RUNNING;
  } else if (mode == FIN_RELIABLE) {  // mixed solver: as resid_finalize_kernel
    const int k = st->k;
    f.part_rr_out[0] = rr;
    const int nr = st->n_rel;
    const bool stalled = nr >= 8 && rr > 0.25 * st->rr_rel[nr & 7];
    st->rr_rel[nr & 7] = rr;
    st->n_rel = nr + 1;
    if (!isfinite(rr)) st->done = CG_NONFINITE;
    else if (rr <= st->tol2bb) st->done = CG_CONVERGED;
    else if (k >= st->maxit) st->done = CG_MAXIT;
    else if (stalled) st->done = CG_STAGNATED;
    else st->done = CG_RUNNING;
  }
}

cudaError_t launch_resid_finalize_batch(const void* descs, int nchains, int mode, double tol, int maxit, int gate,
                                        cudaStream_t s) {
  resid_finalize_batch_kernel<<<nchains, 32, 0, s>>>((const FinArgs*)descs, mode, tol, maxit, gate);
  return cudaGetLastError();
}

// WHILE condition over many chains: continue while any chain is still active.
__global__ void loop_condition_batch_kernel(CgState* const* states, int nchains, cudaGraphConditionalHandle h,
                                            unsigned long long* bodies) {
  if (bodies) *bodies += 1;  // loop bodies run (launch accounting of a trajectory graph)
  bool cont = false;
  for (int c = 0; c < nchains; ++c) {
    CgState* st = states[c];
    const int d = st->done;
    const int loops = st->loops + 1;
    st->loops = loops;
    bool run = d == CG_RUNNING || d == CG_REC_CONVERGED;
    if (run && loops >= st->loop_cap) {
      st->done = CG_MAXIT;
      run = false;
    }
    cont = cont || run;
  }
  cudaGraphSetConditional(h, cont ? 1u : 0u);
}

cudaError_t launch_loop_condition_batch(CgState* const* states, int nchains, cudaGraphConditionalHandle h,
                                        cudaStream_t s, unsigned long long* bodies) {
  loop_condition_batch_kernel<<<1, 1, 0, s>>>(states, nchains, h, bodies);
  return cudaGetLastError();
}

__global__ void loop_condition_kernel(CgState* st, cudaGraphConditionalHandle h) {
  int d = st->done;
  const int loops = st->loops + 1;
  st->loops = loops;
  bool cont = d == CG_RUNNING || d == CG_REC_CONVERGED;
  if (cont && loops >= st->loop_cap) {
    st->done = CG_MAXIT;
    cont = false;
  }
  cudaGraphSetConditional(h, cont ? 1u : 0u);
}

cudaError_t launch_loop_condition(CgState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  loop_condition_kernel<<<1, 1, 0, s>>>(st, h);
  return cudaGetLastError();
}

// Flexible CG (Notay's FCG with one kept direction, i.e. the Polak-Ribiere form):
// the two dot products of the direction's beta after a variable preconditioner
// z = P_k(r), summed per thread in float like the other FP32 reductions.
__global__ void __launch_bounds__(256) fcg_dots_kernel(long long n, const float2* __restrict__ r,
                                                       const float2* __restrict__ r_old, const float2* __restrict__ z,
                                                       double* __restrict__ part_rz, double* __restrict__ part_cross,
                                                       const CgState* st) {
  __shared__ double red[32];
  if (st && *(volatile const int*)&st->done != CG_RUNNING) return;  // uniform: the next head skips too
  float a = 0.f, b = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 zv = z[i];
    a += cdot_re_own(r[i], zv);
    b += cdot_re_own(r_old[i], zv);
  }
  double t = block_sum((double)a, red);
  if (threadIdx.x == 0) part_rz[blockIdx.x] = t;
  t = block_sum((double)b, red);
  if (threadIdx.x == 0) part_cross[blockIdx.x] = t;
}

cudaError_t launch_fcg_dots(long long n, const float2* r, const float2* r_old, const float2* z, int grid,
                            double* part_rz, double* part_cross, const CgState* st, cudaStream_t s) {
  fcg_dots_kernel<<<grid, 256, 0, s>>>(n, r, r_old, z, part_rz, part_cross, st);
  return cudaGetLastError();
}

__global__ void accumulate_correction_kernel(long long n, double2* __restrict__ x, float2* __restrict__ xh,
                                             const CgState* st, int gate) {
  if (st && !gate_open(gate, *(volatile const int*)&st->done)) return;  // st is not written here
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 d = xh[i];
    const double2 xv = x[i];
    x[i] = make_double2(xv.x + (double)d.x, xv.y + (double)d.y);
    xh[i] = make_float2(0.f, 0.f);
  }
}

cudaError_t launch_accumulate_correction(long long n, double2* x, float2* xh, const CgState* st, int gate,
                                         cudaStream_t s) {
  accumulate_correction_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(n, x, xh, st, gate);
  return cudaGetLastError();
}

// nsys systems back to back: blockIdx.y is the system.
__global__ void accumulate_correction_multi_kernel(long long n, double2* __restrict__ x, float2* __restrict__ xh,
                                                   const CgState* st, int gate) {
  const size_t off = (size_t)blockIdx.y * (size_t)n;
  if (st && !gate_open(gate, *(volatile const int*)&st[blockIdx.y].done)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 d = xh[off + i];
    const double2 xv = x[off + i];
    x[off + i] = make_double2(xv.x + (double)d.x, xv.y + (double)d.y);
    xh[off + i] = make_float2(0.f, 0.f);
  }
}

cudaError_t launch_accumulate_correction_multi(long long n, int nsys, double2* x, float2* xh, const CgState* st,
                                               int gate, cudaStream_t s) {
  if (nsys < 1 || nsys > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ew_blocks(n, 256, 1024), (unsigned)nsys);
  accumulate_correction_multi_kernel<<<grid, 256, 0, s>>>(n, x, xh, st, gate);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bosonic force (Results, Eq. (eq3) and the compact action beside it, with
// S = dtau sum_tau L_B):  dS_B/dtheta_{tau,b} = cK [f'(theta_tau - theta_{tau-1})
// - f'(theta_{tau+1} - theta_tau)] with f' = sin (compact) or 2d (non-compact),
// plus the plaquette term K dtau d/dtheta sum cos(curl theta).
__device__ __forceinline__ double curl_at(const double* th, int L, int x, int y) {
  const int xp = (x + 1 == L) ? 0 : x + 1, yp = (y + 1 == L) ? 0 : y + 1;
  return th[2 * (x + L * y)] + th[2 * (xp + L * y) + 1] - th[2 * (x + L * yp)] - th[2 * (x + L * y) + 1];
}

__device__ __forceinline__ double fprime(double d, int noncompact) { return noncompact ? 2.0 * d : sin(d); }

// One thread per (site, chunk of kFinishChunk slices), walking its chunk in tau:
// the term f'(theta_{tau+1} - theta_tau) of slice tau is the f'(theta_tau' -
// theta_{tau'-1}) of slice tau' = tau + 1, so it is evaluated once and carried
// (the same operands in the same order: results identical to evaluating it twice).
constexpr int kFinishChunk = 32;

__device__ __forceinline__ void force_finish_unit(const Geo& g, const BosonParams& bp, const double* __restrict__ theta,
                                                  const double* __restrict__ dSf, double* __restrict__ F, long long k);

__global__ void force_finish_kernel(Geo g, BosonParams bp, const double* __restrict__ theta,
                                    const double* __restrict__ dSf, double* __restrict__ F, int nchunk) {
  const long long nt = (long long)g.V * nchunk;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nt;
       k += (long long)gridDim.x * blockDim.x)
    force_finish_unit(g, bp, theta, dSf, F, k);
}

// One (site, chunk of kFinishChunk slices) unit of the force's bosonic part.
__device__ __forceinline__ void force_finish_unit(const Geo& g, const BosonParams& bp, const double* __restrict__ theta,
                                                  const double* __restrict__ dSf, double* __restrict__ F, long long k) {
  {
    const int ch = (int)(k / g.V);
    const int s = (int)(k - (long long)ch * g.V);
    const int x = s % g.L, y = s / g.L;
    const int t0 = ch * kFinishChunk, t1 = min(g.Ntau, t0 + kFinishChunk);
    const int tm0 = (t0 == 0) ? g.Ntau - 1 : t0 - 1;
    const double2 thm = reinterpret_cast<const double2*>(theta + (size_t)tm0 * g.V * 2)[s];
    double2 th = reinterpret_cast<const double2*>(theta + (size_t)t0 * g.V * 2)[s];
    double dprev[2] = {fprime(th.x - thm.x, bp.noncompact), fprime(th.y - thm.y, bp.noncompact)};
    for (int tau = t0; tau < t1; ++tau) {
      const int tp = (tau + 1 == g.Ntau) ? 0 : tau + 1;
      const double2 thp = reinterpret_cast<const double2*>(theta + (size_t)tp * g.V * 2)[s];
      const double dnext[2] = {fprime(thp.x - th.x, bp.noncompact), fprime(thp.y - th.y, bp.noncompact)};
      // rounding written out (products rounded, no fused multiply-add) so that the
      // single-chain and the batched kernel that inline this give identical bits
      double dB[2] = {__dmul_rn(bp.cK, dprev[0] - dnext[0]), __dmul_rn(bp.cK, dprev[1] - dnext[1])};
      if (bp.Kdtau != 0.0) {
        const double* ths = theta + (size_t)tau * g.V * 2;
        const int xm = (x == 0) ? g.L - 1 : x - 1, ym = (y == 0) ? g.L - 1 : y - 1;
        const double s00 = sin(curl_at(ths, g.L, x, y));
        dB[0] = __dadd_rn(dB[0], __dadd_rn(__dmul_rn(-bp.Kdtau, s00),
                                            __dmul_rn(bp.Kdtau, sin(curl_at(ths, g.L, x, ym)))));
        dB[1] = __dadd_rn(dB[1], __dsub_rn(__dmul_rn(bp.Kdtau, s00),
                                            __dmul_rn(bp.Kdtau, sin(curl_at(ths, g.L, xm, y)))));
      }
      const size_t i = (size_t)tau * g.V + s;
      const double2 f = reinterpret_cast<const double2*>(dSf)[i];
      reinterpret_cast<double2*>(F)[i] = make_double2(__dsub_rn(-f.x, dB[0]), __dsub_rn(-f.y, dB[1]));
      dprev[0] = dnext[0];
      dprev[1] = dnext[1];
      th = thp;
    }
  }
}

cudaError_t launch_force_finish(const Geo& g, const BosonParams& bp, const double* theta,
                                const double* dSf, double* F, cudaStream_t s) {
  const int nchunk = (g.Ntau + kFinishChunk - 1) / kFinishChunk;
  const long long n = (long long)g.V * nchunk;
  force_finish_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(g, bp, theta, dSf, F, nchunk);
  return cudaGetLastError();
}

__global__ void kick_kernel(long long nb, double* __restrict__ p, const double* __restrict__ F, double h) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(F[i], h, p[i]);
}

__global__ void kick_drift_kernel(long long nb, double* __restrict__ p, double* __restrict__ theta,
                                  const double* __restrict__ F, double h, double dt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
       i += (long long)gridDim.x * blockDim.x) {
    const double pn = fma(F[i], h, p[i]);  // fused as in the batched kernel
    p[i] = pn;
    theta[i] = fma(2.0 * pn, dt, theta[i]);
  }
}

cudaError_t launch_kick(long long nb, double* p, const double* F, double h, cudaStream_t s) {
  kick_kernel<<<ew_blocks(nb, 256, 4096), 256, 0, s>>>(nb, p, F, h);
  return cudaGetLastError();
}

cudaError_t launch_kick_drift(long long nb, double* p, double* theta, const double* F, double h,
                              double dt, cudaStream_t s) {
  kick_drift_kernel<<<ew_blocks(nb, 256, 4096), 256, 0, s>>>(nb, p, theta, F, h, dt);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Hamiltonian terms: S_B(theta), sum p^2, Re <a, b>.  Per-block partials, then
// one block sums them in a fixed order.
// Partials of block j of nb (the same element grouping for a chain alone or in a batch).
__device__ __forceinline__ void action_partials_block(const Geo& g, const BosonParams& bp,
                                                      const double* __restrict__ theta, const double* __restrict__ p,
                                                      const double2* __restrict__ a, const double2* __restrict__ b,
                                                      double* __restrict__ part, int j, int nb) {
  __shared__ double red[32];
  const long long n = (long long)g.V * g.Ntau;
  double kin = 0.0, pot = 0.0, pp = 0.0, ab = 0.0;
  for (long long i = j * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) {
    const int tau = (int)(i / g.V);
    const int s = (int)(i - (long long)tau * g.V);
    const int tp = (tau + 1 == g.Ntau) ? 0 : tau + 1;
    const double* th = theta + (size_t)tau * g.V * 2;
    const double* thp = theta + (size_t)tp * g.V * 2;
    for (int c = 0; c < 2; ++c) {
      const double d = thp[2 * s + c] - th[2 * s + c];
      kin += bp.noncompact ? __dmul_rn(d, d) : 1.0 - cos(d);
    }
    if (bp.Kdtau != 0.0) pot += cos(curl_at(th, g.L, s % g.L, s / g.L));
    if (p) {
      const double2 pv = reinterpret_cast<const double2*>(p)[i];
      pp += cdot_re(pv, pv);
    }
    if (a && b) ab += cdot_re(a[i], b[i]);
  }
  double t;
  t = block_sum(kin, red);
  if (threadIdx.x == 0) part[4 * j + 0] = t;
  t = block_sum(pot, red);
  if (threadIdx.x == 0) part[4 * j + 1] = t;
  t = block_sum(pp, red);
  if (threadIdx.x == 0) part[4 * j + 2] = t;
  t = block_sum(ab, red);
  if (threadIdx.x == 0) part[4 * j + 3] = t;
}

__global__ void action_partials_kernel(Geo g, BosonParams bp, const double* __restrict__ theta,
                                       const double* __restrict__ p, const double2* __restrict__ a,
                                       const double2* __restrict__ b, double* __restrict__ part) {
  action_partials_block(g, bp, theta, p, a, b, part, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void action_finalize_warp(const BosonParams& bp, const double* __restrict__ part, int nblk,
                                                     double* __restrict__ terms);

__global__ void action_finalize_kernel(BosonParams bp, const double* __restrict__ part, int nblk,
                                       double* __restrict__ terms) {
  action_finalize_warp(bp, part, nblk, terms);
}

__device__ __forceinline__ void action_finalize_warp(const BosonParams& bp, const double* __restrict__ part, int nblk,
                                                     double* __restrict__ terms) {
  double s[4];
  for (int c = 0; c < 4; ++c) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 32) acc += part[4 * k + c];
    acc = warp_sum(acc);
    s[c] = __shfl_sync(0xffffffffu, acc, 0);
  }
  if (threadIdx.x == 0) {
    terms[0] = __dadd_rn(__dmul_rn(bp.cK, s[0]), __dmul_rn(bp.Kdtau, s[1]));
    terms[1] = s[2];
    terms[2] = s[3];
  }
}

cudaError_t launch_action_terms(const Geo& g, const BosonParams& bp, const double* theta,
                                const double* p, const double2* a, const double2* b, int grid,
                                double* part, double* terms, cudaStream_t s) {
  action_partials_kernel<<<grid, 256, 0, s>>>(g, bp, theta, p, a, b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  action_finalize_kernel<<<1, 32, 0, s>>>(bp, part, grid, terms);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011): 10 rounds of two 32x32->64 products
// with the round constants below and a Weyl key schedule.
struct U4 {
  uint32_t v[4];
};

__host__ __device__ inline U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.v[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.v[2];
    U4 o;
    o.v[0] = (uint32_t)(p1 >> 32) ^ c.v[1] ^ k0;
    o.v[1] = (uint32_t)p1;
    o.v[2] = (uint32_t)(p0 >> 32) ^ c.v[3] ^ k1;
    o.v[3] = (uint32_t)p0;
    c = o;
  }
  return c;
}

__host__ __device__ inline double u53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ inline void gauss_pair(uint64_t seed, uint32_t stream, uint64_t counter, uint32_t elem,
                                  double* g0, double* g1) {
  U4 c = {{elem, stream, (uint32_t)counter, (uint32_t)(counter >> 32)}};
  const U4 w = philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double ua = u53(w.v[0], w.v[1]);
  const double ub = u53(w.v[2], w.v[3]);
  const double r = sqrt(-2.0 * log(1.0 - ua));
  double sn, cs;
  sincos(2.0 * 3.141592653589793 * ub, &sn, &cs);
  *g0 = r * cs;
  *g1 = r * sn;
}

// p ~ N(0, 1/2) per bond (stream 0) and R ~ CN(0, 1) per site (stream 1) at site i.
__device__ __forceinline__ void draw_site(uint64_t seed, uint64_t counter, double* __restrict__ p,
                                          double2* __restrict__ R, long long i) {
  const double h = 0.70710678118654752440;  // sqrt(1/2)
  double g0, g1;
  if (p) {
    gauss_pair(seed, 0u, counter, (uint32_t)i, &g0, &g1);
    reinterpret_cast<double2*>(p)[i] = make_double2(g0 * h, g1 * h);
  }
  if (R) {
    gauss_pair(seed, 1u, counter, (uint32_t)i, &g0, &g1);
    R[i] = make_double2(g0 * h, g1 * h);
  }
}

__global__ void draw_kernel(long long n, uint64_t seed, uint64_t counter, double* __restrict__ p,
                            double2* __restrict__ R) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    draw_site(seed, counter, p, R, i);
}

cudaError_t launch_draw(long long n_sites, uint64_t seed, uint64_t counter, double* p, double2* R,
                        cudaStream_t s) {
  draw_kernel<<<ew_blocks(n_sites, 256, 4096), 256, 0, s>>>(n_sites, seed, counter, p, R);
  return cudaGetLastError();
}

// v ~ CN(0, 1) per site from Philox stream `stream` at traj_counter `counter`.
__global__ void draw_vector_kernel(long long n, uint64_t seed, uint32_t stream, uint64_t counter,
                                   double2* __restrict__ v) {
  const double h = 0.70710678118654752440;  // sqrt(1/2)
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double g0, g1;
    gauss_pair(seed, stream, counter, (uint32_t)i, &g0, &g1);
    v[i] = make_double2(g0 * h, g1 * h);
  }
}

cudaError_t launch_draw_vector(long long n_sites, uint64_t seed, uint32_t stream, uint64_t counter, double2* v,
                               cudaStream_t s) {
  draw_vector_kernel<<<ew_blocks(n_sites, 256, 4096), 256, 0, s>>>(n_sites, seed, stream, counter, v);
  return cudaGetLastError();
}

// r = phi - y with y from an FP32 apply (FP64 result).
__global__ void resid_from_fp32_kernel(long long n, const double2* __restrict__ phi, const float2* __restrict__ y,
                                       double2* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 p = phi[i];
    const float2 v = y[i];
    r[i] = make_double2(p.x - (double)v.x, p.y - (double)v.y);
  }
}

cudaError_t launch_resid_from_fp32(long long n, const double2* phi, const float2* y, double2* r, cudaStream_t s) {
  resid_from_fp32_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(n, phi, y, r);
  return cudaGetLastError();
}

// <a, b> = sum conj(a_i) b_i (complex), as per-block partials in a fixed order
// and one warp that sums them: out[0] = Re, out[1] = Im.
__global__ void cdot_partials_kernel(long long n, const double2* __restrict__ a, const double2* __restrict__ b,
                                     double* __restrict__ part) {
  __shared__ double red[32];
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  double t = block_sum(re, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x] = t;
  t = block_sum(im, red);
  if (threadIdx.x == 0) part[2 * blockIdx.x + 1] = t;
}

__global__ void cdot_finalize_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  for (int c = 0; c < 2; ++c) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 32) acc += part[2 * k + c];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) out[c] = acc;
  }
}

// <X_i, b> for i < k, X_i = X + i * stride: partials (grid per vector), then one warp
// per vector sums them in a fixed order into out[2 i], out[2 i + 1] (re, im).
__global__ void cdot_many_partials_kernel(long long n, const double2* __restrict__ X, long long stride,
                                          const double2* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[32];
  const double2* a = X + (size_t)blockIdx.y * stride;
  double re = 0.0, im = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    re += fma(x.x, y.x, __dmul_rn(x.y, y.y));
    im += fma(x.x, y.y, -__dmul_rn(x.y, y.x));
  }
  const size_t o = 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
  double t = block_sum(re, red);
  if (threadIdx.x == 0) part[o] = t;
  t = block_sum(im, red);
  if (threadIdx.x == 0) part[o + 1] = t;
}

__global__ void cdot_many_finalize_kernel(const double* __restrict__ part, int grid, double* __restrict__ out) {
  const double* p = part + 2 * (size_t)blockIdx.x * grid;
  for (int c = 0; c < 2; ++c) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < grid; k += 32) acc += p[2 * k + c];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) out[2 * blockIdx.x + c] = acc;
  }
}

cudaError_t launch_cdot_many(long long n, const double2* X, long long stride, int k, const double2* b, int grid,
                             double* part, double* out, cudaStream_t s) {
  cdot_many_partials_kernel<<<dim3(grid, k), 256, 0, s>>>(n, X, stride, b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cdot_many_finalize_kernel<<<k, 32, 0, s>>>(part, grid, out);
  return cudaGetLastError();
}

// y += c x (complex c).
__global__ void caxpy_kernel(long long n, double cr, double ci, const double2* __restrict__ x, double2* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i], w = y[i];
    y[i] = make_double2(fma(cr, v.x, fma(-ci, v.y, w.x)), fma(cr, v.y, fma(ci, v.x, w.y)));
  }
}

// y *= a (real a), in place.
__global__ void dscale_kernel(long long n, double a, double2* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 w = y[i];
    y[i] = make_double2(a * w.x, a * w.y);
  }
}

cudaError_t launch_dscale(long long n, double a, double2* y, cudaStream_t s) {
  dscale_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(n, a, y);
  return cudaGetLastError();
}

cudaError_t launch_caxpy(long long n, double cr, double ci, const double2* x, double2* y, cudaStream_t s) {
  caxpy_kernel<<<ew_blocks(n, 256, 4096), 256, 0, s>>>(n, cr, ci, x, y);
  return cudaGetLastError();
}

cudaError_t launch_cdot(long long n, const double2* a, const double2* b, int grid, double* part, double* out,
                        cudaStream_t s) {
  cdot_partials_kernel<<<grid, 256, 0, s>>>(n, a, b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cdot_finalize_kernel<<<1, 32, 0, s>>>(part, grid, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 throughput probe: every thread runs 8 independent FMA chains, so the
// FP64 pipe, not latency, limits the rate.  Used only to measure the FP64
// roofline denominator of this device.
__global__ void fp64_probe_kernel(double* out, int iters, double a, double b) {
  double v0 = threadIdx.x * 1e-3, v1 = v0 + 1, v2 = v0 + 2, v3 = v0 + 3, v4 = v0 + 4, v5 = v0 + 5,
         v6 = v0 + 6, v7 = v0 + 7;
  for (int i = 0; i < iters; ++i) {
    v0 = fma(v0, a, b); v1 = fma(v1, a, b); v2 = fma(v2, a, b); v3 = fma(v3, a, b);
    v4 = fma(v4, a, b); v5 = fma(v5, a, b); v6 = fma(v6, a, b); v7 = fma(v7, a, b);
  }
  const double s = ((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7));
  if (s == 123.456) out[0] = s;  // keeps the chains live
}

cudaError_t launch_fp64_probe(int blocks, int threads, int iters, double* out, cudaStream_t s) {
  fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched trajectory kernels: every chain's element loop keeps the grouping of its
// own launch (block j of nb), so a batch reproduces single-chain runs bit for bit.
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t counter) {
  U4 c = {{0u, 2u, (uint32_t)counter, (uint32_t)(counter >> 32)}};
  const U4 w = philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return u53(w.v[0], w.v[1]);
}

__global__ void __launch_bounds__(256) batch_elementwise_kernel(const ChainDesc* __restrict__ descs,
                                                                const int4* __restrict__ tab, int op,
                                                                const uint64_t* __restrict__ counter) {
  const int4 e = tab[blockIdx.x];
  const ChainDesc& d = descs[e.x];
  if (op == BT_RESTORE && d.info->accepted) return;
  const long long n = d.n;
  const long long i0 = e.y * (long long)blockDim.x + threadIdx.x, step = (long long)e.z * blockDim.x;
  switch (op) {
    case BT_DRAW: {
      const uint64_t ctr = *counter;
      for (long long i = i0; i < n; i += step) draw_site(d.seed, ctr, d.p, d.R, i);
    } break;
    case BT_LINKS:
      for (long long i = i0; i < n; i += step) links_site(d.g, d.theta, d.t1, d.t2, d.U64, nullptr, nullptr, i);
      break;
    case BT_ZERO_X:
      for (long long i = i0; i < n; i += step) d.X[i] = make_double2(0.0, 0.0);
      break;
    case BT_SAVE:
      for (long long i = i0; i < 2 * n; i += step) d.th0[i] = d.theta[i];
      break;
    case BT_RESTORE:
      for (long long i = i0; i < 2 * n; i += step) d.theta[i] = d.th0[i];
      break;
    case BT_KICK_DRIFT: {  // p += F dt/2; theta += 2 p dt (as kick_drift_kernel)
      const double h = d.dt / 2, dt = d.dt;
      for (long long i = i0; i < 2 * n; i += step) {
        const double pn = fma(d.F[i], h, d.p[i]);
        d.p[i] = pn;
        d.theta[i] = fma(2.0 * pn, dt, d.theta[i]);
      }
    } break;
    default: {  // BT_KICK: p += F dt/2 (as kick_kernel)
      const double h = d.dt / 2;
      for (long long i = i0; i < 2 * n; i += step) d.p[i] = fma(d.F[i], h, d.p[i]);
    } break;
  }
}

cudaError_t launch_batch_elementwise(const ChainDesc* d, const int4* tab, int nblocks, int op, const uint64_t* counter,
                                     cudaStream_t s) {
  batch_elementwise_kernel<<<nblocks, 256, 0, s>>>(d, tab, op, counter);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) batch_action_partials_kernel(const ChainDesc* __restrict__ descs,
                                                                    const int4* __restrict__ tab, int which) {
  const int4 e = tab[blockIdx.x];
  const ChainDesc& d = descs[e.x];
  if (which == 0) action_partials_block(d.g, d.bp, d.theta, d.p, d.R, d.R, d.part_act, e.y, e.z);
  else action_partials_block(d.g, d.bp, d.theta, d.p, d.eta, d.X, d.part_act, e.y, e.z);
}

__global__ void batch_action_finalize_kernel(const ChainDesc* __restrict__ descs, int which) {
  const ChainDesc& d = descs[blockIdx.x];
  action_finalize_warp(d.bp, d.part_act, d.act_grid, d.terms + 3 * which);
}

cudaError_t launch_batch_action(const ChainDesc* d, const int4* tab, int nblocks, int nchains, int which,
                                cudaStream_t s) {
  batch_action_partials_kernel<<<nblocks, 256, 0, s>>>(d, tab, which);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_action_finalize_kernel<<<nchains, 32, 0, s>>>(d, which);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) batch_force_finish_kernel(const ChainDesc* __restrict__ descs,
                                                                 const int4* __restrict__ tab) {
  const int4 e = tab[blockIdx.x];
  const ChainDesc& d = descs[e.x];
  const long long nt = (long long)d.g.V * ((d.g.Ntau + kFinishChunk - 1) / kFinishChunk);
  for (long long k = e.y * (long long)blockDim.x + threadIdx.x; k < nt; k += (long long)e.z * blockDim.x)
    force_finish_unit(d.g, d.bp, d.theta, d.dSf, d.F, k);
}

cudaError_t launch_batch_force_finish(const ChainDesc* d, const int4* tab, int nblocks, cudaStream_t s) {
  batch_force_finish_kernel<<<nblocks, 256, 0, s>>>(d, tab);
  return cudaGetLastError();
}

__global__ void batch_info_init_kernel(const ChainDesc* __restrict__ descs, int nchains,
                                       const uint64_t* __restrict__ counter) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchains) return;
  const ChainDesc& d = descs[c];
  hqmc_traj_info t = {};
  t.u = philox_uniform(d.seed, *counter);
  *d.info = t;
}

cudaError_t launch_batch_info_init(const ChainDesc* d, int nchains, const uint64_t* counter, cudaStream_t s) {
  batch_info_init_kernel<<<(nchains + 63) / 64, 64, 0, s>>>(d, nchains, counter);
  return cudaGetLastError();
}

// After a batched solve: count it, add its iterations, keep the largest true
// residual and the worst status (the report holds the last true residual of a
// converged chain, or the residual recomputed for an unconverged one).
__global__ void batch_solve_close_kernel(const ChainDesc* __restrict__ descs, int nchains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchains) return;
  const ChainDesc& d = descs[c];
  hqmc_traj_info* t = d.info;
  const CgState* st = d.st;
  const int status = solve_status(st->done, false);
  t->cg_solves += 1;
  t->cg_iterations += st->k;
  const double res = st->bb > 0 ? sqrt(d.report[0] / st->bb) : 0.0;
  t->max_true_residual = fmax(t->max_true_residual, res);
  if (t->status == HQMC_OK) t->status = status;
}

cudaError_t launch_batch_solve_close(const ChainDesc* d, int nchains, cudaStream_t s) {
  batch_solve_close_kernel<<<(nchains + 63) / 64, 64, 0, s>>>(d, nchains);
  return cudaGetLastError();
}

// H0 = S_B + sum p^2 + R^dagger R, H1 = S_B + sum p^2 + phi^dagger X; accept iff u < e^{-(H1 - H0)}.
__global__ void batch_metropolis_kernel(const ChainDesc* __restrict__ descs, int nchains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchains) return;
  const ChainDesc& d = descs[c];
  hqmc_traj_info* t = d.info;
  const double* tm = d.terms;
  t->H0 = tm[0] + tm[1] + tm[2];
  t->H1 = tm[3] + tm[4] + tm[5];
  t->dH = t->H1 - t->H0;
  const bool fin = isfinite(t->dH);
  if (!fin && t->status == HQMC_OK) t->status = HQMC_ENONFINITE;
  const bool ok = t->status == HQMC_OK || t->status == HQMC_ENOTCONV;
  t->accepted = (ok && fin && t->u < exp(-t->dH)) ? 1 : 0;
}

cudaError_t launch_batch_metropolis(const ChainDesc* d, int nchains, cudaStream_t s) {
  batch_metropolis_kernel<<<(nchains + 63) / 64, 64, 0, s>>>(d, nchains);
  return cudaGetLastError();
}

void philox_uniform_host(uint64_t seed, uint64_t counter, double* u) {
  U4 c = {{0u, 2u, (uint32_t)counter, (uint32_t)(counter >> 32)}};
  const U4 w = philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  *u = u53(w.v[0], w.v[1]);
}

}  // namespace hqmc
