// Tau-line preconditioner (Methods, "CG method and preconditioner").
//
// Built once per config from the pi-flux field.  O's same-site part there is
// the tau-line matrix T = a - b (S + S^dagger) on every site: a is the diagonal
// of O, b = B_ss, and S the antiperiodic tau shift.  Its bulk Cholesky factor
// is L = sqrt(b/rho)(1 - rho S) with rho + 1/rho = a/b.  The Neumann series of
// L^{-1}, with entries below 1e-3 dropped, keeps the powers rho^m S^m,
// m <= W.  The preconditioner is
//   Otilde^{-1} r = (rho/b) F_W^dagger F_W r,   F_W = sum_{m=0}^{W} rho^m S^m,
// applied to every site's tau line independently.
//
// One kernel does both passes on a tile of 32 sites (one warp width, so a
// slice row of the tile is 256 B contiguous in FP32) by TC consecutive slices:
//   1. the block loads u on slices [t0 - W, t1 + W] of its sites into shared
//      memory, every load independent (coalesced rows);
//   2. forward:  x_tau = sum_m rho^m u~_{tau-m} for tau in [t0, t1 + W], each
//      warp a contiguous sub-range, as a sliding-window recursion
//      x_tau = rho x_{tau-1} + u~_tau - rho^{W+1} u~_{tau-W-1} started W slices
//      before its sub-range, into a second shared buffer;
//   3. backward: y_tau = sum_m rho^m x~_{tau+m} for tau in [t0, t1), the same
//      recursion in descending tau; z = (rho/b) y is written once, with the
//      partial sums of Re <r, z> for pCG (r = u is still in shared memory).
// u~ and x~ are the antiperiodic extensions (a sign flip per wrap); the halo
// rows are read again by the neighbouring tile, mostly from L2, so HBM sees
// one read of r and one write of z.
#include "kernels.h"

namespace hqmc {

namespace {

// Position of slice j (any integer) on the antiperiodic tau line: index j mod N
// and the sign (-1)^(wraps).
struct LinePos {
  int m;
  float sgn;
};

__device__ __forceinline__ LinePos line_pos(int j, int N) {
  int q = j / N, m = j - q * N;
  if (m < 0) {
    m += N;
    q -= 1;
  }
  return LinePos{m, (q & 1) ? -1.f : 1.f};
}

__device__ __forceinline__ bool line_gate(const CgState* st) {
  return st == nullptr || *(volatile const int*)&st->done == CG_RUNNING;
}

}  // namespace

constexpr int kLineSites = 32;  // sites per tile (one warp width)
constexpr int kLineWarps = 8;   // warps per block: independent recursion chains hide the FMA latency

// Slices per tile: FP32 128, FP64 64 (shared memory: both buffers of the tile).
template <class R> constexpr int line_tile_slices() { return sizeof(R) == 4 ? 128 : 64; }

size_t line_smem_bytes(int real_bytes, int W) {
  const int tc = real_bytes == 4 ? line_tile_slices<float>() : line_tile_slices<double>();
  return (size_t)((tc + 2 * W + 1) + (tc + W + 1)) * kLineSites * 2 * real_bytes;
}

// One tile (site block bx, slice block by of a gx-wide grid) of z = Otilde^{-1} u
// with its partial of <u, z> in part[by * gx + bx].
template <class R>
__device__ __forceinline__ void line_precond_tile(const Geo& g, const LineCoef& lc, const C2<R>* __restrict__ u,
                                                  C2<R>* __restrict__ z, double* __restrict__ part, int bx, int by,
                                                  int gx) {
  using T = C2<R>;
  constexpr int TC = line_tile_slices<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int N = g.Ntau, V = g.V, W = lc.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s0 = bx * kLineSites, s = s0 + lane;
  const bool site_ok = s < V;
  const int t0 = by * TC, t1 = min(N, t0 + TC), nt = t1 - t0;
  const int nu = nt + 2 * W + 1;  // rows of u: slices t0 - W .. t1 + W
  const int nx = nt + W + 1;      // rows of x: slices t0 .. t1 + W
  T* U = reinterpret_cast<T*>(smem_raw);
  T* X = U + (size_t)(TC + 2 * W + 1) * kLineSites;

  // 1. u rows into shared memory by asynchronous copies (all in flight at once),
  //    then the sign of the antiperiodic extension on the rows that wrapped
  LinePos p = line_pos(t0 - W + warp, N);  // stepped by kLineWarps rows below
  for (int row = warp; row < nu; row += kLineWarps) {
    T* dst = U + row * kLineSites + lane;
    if (site_ok) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
      const T* src = u + (size_t)p.m * V + s;
      if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
      else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
    } else {
      *dst = mk(R(0), R(0));
    }
    p.m += kLineWarps;
    while (p.m >= N) {
      p.m -= N;
      p.sgn = -p.sgn;
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  {  // rows before slice 0 or past slice N-1 carry the sign of their wraps
    LinePos q = line_pos(t0 - W + warp, N);
    for (int row = warp; row < nu; row += kLineWarps) {
      if (q.sgn < 0.f) {
        T* e = U + row * kLineSites + lane;
        *e = mk(-e->x, -e->y);
      }
      q.m += kLineWarps;
      while (q.m >= N) {
        q.m -= N;
        q.sgn = -q.sgn;
      }
    }
  }
  __syncthreads();
  const R rho = (R)lc.rho, rw = (R)lc.rhoW1, sc = (R)lc.scale;
  // 2. forward: rows of x split over the warps; U row of slice tau is tau - t0 + W
  {
    const int per = (nx + kLineWarps - 1) / kLineWarps;
    const int a = warp * per, b = min(nx, a + per);  // x rows [a, b): slices t0 + a ..
    if (a < b) {
      T acc = mk(R(0), R(0));
#pragma unroll 4
      for (int m = 0; m <= W; ++m) acc = caxpy(U[(a + m) * kLineSites + lane], rho, acc);  // slices t0+a-W .. t0+a
      X[a * kLineSites + lane] = acc;
#pragma unroll 4
      for (int i = a + 1; i < b; ++i) {
        acc = caxpy(caxpy(U[(i + W) * kLineSites + lane], rho, acc), -rw, U[(i - 1) * kLineSites + lane]);
        X[i * kLineSites + lane] = acc;
      }
    }
  }
  __syncthreads();
  // 3. backward over the tile's own slices, split over the warps
  R dot = 0;  // FP32: the thread's terms in float (cdot_re_own)
  {
    const int per = (nt + kLineWarps - 1) / kLineWarps;
    const int a = warp * per, b = min(nt, a + per);  // output rows [a, b)
    if (a < b) {
      T acc = mk(R(0), R(0));
#pragma unroll 4
      for (int m = W; m >= 0; --m) acc = caxpy(X[(b - 1 + m) * kLineSites + lane], rho, acc);
      for (int i = b - 1;; --i) {
        const T zv = cscale(sc, acc);
        if (site_ok) {
          z[(t0 + i) * V + s] = zv;
          dot += cdot_re_own(U[(i + W) * kLineSites + lane], zv);
        }
        if (i == a) break;
        acc = caxpy(caxpy(X[(i - 1) * kLineSites + lane], rho, acc), -rw, X[(i + W) * kLineSites + lane]);
      }
    }
  }
  if (part) {
    const double tot = block_sum((double)dot, red);
    if (threadIdx.x == 0) part[by * gx + bx] = tot;
  }
}

template <class R>
__global__ void __launch_bounds__(kLineSites* kLineWarps) line_precond_kernel(Geo g, LineCoef lc,
                                                                             const C2<R>* __restrict__ u,
                                                                             C2<R>* __restrict__ z,
                                                                             double* __restrict__ part,
                                                                             const CgState* st) {
  if (!line_gate(st)) return;  // uniform over the grid
  line_precond_tile<R>(g, lc, u, z, part, blockIdx.x, blockIdx.y, gridDim.x);
}

// Many chains in one launch: block b runs tile tiles[b] = (chain, bx, by) with
// that chain's descriptor, so each chain's tiles and partials are those of its
// own launch.
template <class R>
__global__ void __launch_bounds__(kLineSites* kLineWarps) line_precond_batch_kernel(
    const LineBatchDesc<R>* __restrict__ descs, const int4* __restrict__ tiles) {
  const int4 t = tiles[blockIdx.x];
  const LineBatchDesc<R> d = descs[t.x];
  if (!line_gate(d.st)) return;  // uniform over the block
  line_precond_tile<R>(d.g, d.lc, d.u, d.z, d.part, t.y, t.z, d.gx);
}

// Preconditioned CG, fused update and preconditioner (one launch per iteration
// after the direction step):
//   alpha = <r, z>_k / <p, O p> from the direction kernel's partials (stop on a
//   non-positive or non-finite <p, O p>, as the plain update does);
//   r <- r - alpha q and x <- x + alpha p on the tile's own slices;
//   z = Otilde^{-1} r on the updated r, with the partials of <r, r> (convergence)
//   and <r, z> (next step length).
// The tile loads r and q on its slices and halo, forms r - alpha q there (the
// halo rows with the same arithmetic as the tiles that own them), then runs the
// two recursions as line_precond_kernel does.  The updated r goes to a second
// buffer (r_out): a tile's halo rows are other tiles' own rows, so writing r in
// place would race with their loads; the caller alternates the two buffers.
// One HBM pass over r and q, x, p instead of the update's pass plus the
// preconditioner's re-read of r.
template <class R>
__global__ void __launch_bounds__(kLineSites* kLineWarps) line_update_kernel(Geo g, LineCoef lc, LineUpdArgs<R> a) {
  using T = C2<R>;
  constexpr int TC = line_tile_slices<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_stop;
  __shared__ double s_alpha;
  __shared__ int s_k;
  CgState* st = a.st;
  const bool block0 = blockIdx.x == 0 && blockIdx.y == 0;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int done = *(volatile int*)&st->done;
    int stop = 0;
    double alpha = 0.0;
    if (done != CG_RUNNING) {
      stop = 1;
    } else {
      const int k = st->k2;
      const double pq = warp_sum_partials(a.part_pq, a.n_pq);
      const double rz = st->rr[k & 1];
      if (!isfinite(pq) || !(pq > 0.0)) {
        stop = 1;
        if (block0 && lane == 0) st->done = isfinite(pq) ? CG_BREAKDOWN : CG_NONFINITE;
      } else {
        alpha = rz / pq;
        if (block0 && lane == 0) {
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
  if (s_stop) return;  // uniform over the grid
  const R alpha = (R)s_alpha;
  const T* __restrict__ pdir = ((s_k + 1) & 1) ? a.p1 : a.p0;

  const int N = g.Ntau, V = g.V, W = lc.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s0 = blockIdx.x * kLineSites, s = s0 + lane;
  const bool site_ok = s < V;
  const int t0 = blockIdx.y * TC, t1 = min(N, t0 + TC), nt = t1 - t0;
  const int nu = nt + 2 * W + 1;  // rows of u: slices t0 - W .. t1 + W
  const int nx = nt + W + 1;      // rows of x: slices t0 .. t1 + W
  T* U = reinterpret_cast<T*>(smem_raw);
  T* X = U + (size_t)(TC + 2 * W + 1) * kLineSites;  // q rows first, then the forward pass

  // 1. r and q rows (tile and halo) by asynchronous copies
  LinePos p = line_pos(t0 - W + warp, N);
  for (int row = warp; row < nu; row += kLineWarps) {
    T* du = U + row * kLineSites + lane;
    T* dq = X + row * kLineSites + lane;
    if (site_ok) {
      const size_t gi = (size_t)p.m * V + s;
      const unsigned su = (unsigned)__cvta_generic_to_shared(du), sq = (unsigned)__cvta_generic_to_shared(dq);
      if constexpr (sizeof(T) == 8) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(su), "l"(a.r_in + gi) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sq), "l"(a.q + gi) : "memory");
      } else {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(su), "l"(a.r_in + gi) : "memory");
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sq), "l"(a.q + gi) : "memory");
      }
    } else {
      *du = mk(R(0), R(0));
      *dq = mk(R(0), R(0));
    }
    p.m += kLineWarps;
    while (p.m >= N) {
      p.m -= N;
      p.sgn = -p.sgn;
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // 2. r - alpha q on every row (the update's own arithmetic), the sign of the
  //    antiperiodic extension on wrapped rows; own rows go back to r, and x moves
  R rr = 0;  // FP32: the thread's terms in float (cdot_re_own)
  {
    LinePos q = line_pos(t0 - W + warp, N);
    for (int row = warp; row < nu; row += kLineWarps) {
      T* e = U + row * kLineSites + lane;
      T v = caxpy(*e, -alpha, X[row * kLineSites + lane]);
      const int own = row - W;  // slice t0 + own
      if (own >= 0 && own < nt && site_ok) {
        a.r_out[(size_t)(t0 + own) * V + s] = v;
        rr += cdot_re_own(v, v);
      }
      if (q.sgn < 0.f) v = mk(-v.x, -v.y);
      *e = v;
      q.m += kLineWarps;
      while (q.m >= N) {
        q.m -= N;
        q.sgn = -q.sgn;
      }
    }
  }
  // 2b. x <- x + alpha p on the own slices: every load of the thread first, then
  //     the stores (loads and stores through the same pointers cannot be reordered
  //     by the compiler, and a loop of load-update-store would wait on every load)
  if (site_ok) {
    constexpr int MAXO = TC / kLineWarps;
    T xv[MAXO], pv[MAXO];
#pragma unroll
    for (int m = 0; m < MAXO; ++m) {
      const int o = warp + m * kLineWarps;
      if (o < nt) {
        const size_t gi = (size_t)(t0 + o) * V + s;
        xv[m] = a.x[gi];
        pv[m] = pdir[gi];
      }
    }
#pragma unroll
    for (int m = 0; m < MAXO; ++m) {
      const int o = warp + m * kLineWarps;
      if (o < nt) a.x[(size_t)(t0 + o) * V + s] = caxpy(xv[m], alpha, pv[m]);
    }
  }
  __syncthreads();
  const R rho = (R)lc.rho, rw = (R)lc.rhoW1, sc = (R)lc.scale;
  // 3. forward pass into X (the q rows are no longer needed)
  {
    const int per = (nx + kLineWarps - 1) / kLineWarps;
    const int a0 = warp * per, b0 = min(nx, a0 + per);
    if (a0 < b0) {
      T acc = mk(R(0), R(0));
#pragma unroll 4
      for (int m = 0; m <= W; ++m) acc = caxpy(U[(a0 + m) * kLineSites + lane], rho, acc);
      X[a0 * kLineSites + lane] = acc;
#pragma unroll 4
      for (int i = a0 + 1; i < b0; ++i) {
        acc = caxpy(caxpy(U[(i + W) * kLineSites + lane], rho, acc), -rw, U[(i - 1) * kLineSites + lane]);
        X[i * kLineSites + lane] = acc;
      }
    }
  }
  __syncthreads();
  // 4. backward pass: z and <r, z>
  R rz = 0;
  {
    const int per = (nt + kLineWarps - 1) / kLineWarps;
    const int a0 = warp * per, b0 = min(nt, a0 + per);
    if (a0 < b0) {
      T acc = mk(R(0), R(0));
#pragma unroll 4
      for (int m = W; m >= 0; --m) acc = caxpy(X[(b0 - 1 + m) * kLineSites + lane], rho, acc);
      for (int i = b0 - 1;; --i) {
        const T zv = cscale(sc, acc);
        if (site_ok) {
          a.z[(size_t)(t0 + i) * V + s] = zv;
          rz += cdot_re_own(U[(i + W) * kLineSites + lane], zv);
        }
        if (i == a0) break;
        acc = caxpy(caxpy(X[(i - 1) * kLineSites + lane], rho, acc), -rw, X[(i + W) * kLineSites + lane]);
      }
    }
  }
  const int slot = blockIdx.y * gridDim.x + blockIdx.x;
  double t = block_sum((double)rr, red);
  if (threadIdx.x == 0) a.part_rr[slot] = t;
  t = block_sum((double)rz, red);
  if (threadIdx.x == 0) {
    a.part_rz[slot] = t;
    if (block0) st->k = s_k + 1;
  }
}

template <class R>
cudaError_t prepare_line_update(int W) {
  return raise_smem_limit(line_update_kernel<R>, line_update_smem_bytes(sizeof(R), W));
}
template cudaError_t prepare_line_update<double>(int);
template cudaError_t prepare_line_update<float>(int);

size_t line_update_smem_bytes(int real_bytes, int W) {
  const int tc = real_bytes == 4 ? line_tile_slices<float>() : line_tile_slices<double>();
  return (size_t)2 * (tc + 2 * W + 1) * kLineSites * 2 * real_bytes;
}

template <class R>
cudaError_t launch_line_update(const Geo& g, const LineCoef& lc, const LineLaunch& ll, const LineUpdArgs<R>& a,
                               cudaStream_t s) {
  const dim3 grid(ll.gx, ll.gy);
  line_update_kernel<R><<<grid, ll.block, line_update_smem_bytes(sizeof(R), lc.W), s>>>(g, lc, a);
  return cudaGetLastError();
}
template cudaError_t launch_line_update<double>(const Geo&, const LineCoef&, const LineLaunch&,
                                                const LineUpdArgs<double>&, cudaStream_t);
template cudaError_t launch_line_update<float>(const Geo&, const LineCoef&, const LineLaunch&,
                                               const LineUpdArgs<float>&, cudaStream_t);

LineLaunch line_launch(const Geo& g, int real_bytes) {
  LineLaunch ll;
  ll.chunk = real_bytes == 4 ? line_tile_slices<float>() : line_tile_slices<double>();
  ll.block = kLineSites * kLineWarps;
  ll.gx = (g.V + kLineSites - 1) / kLineSites;
  ll.gy = (g.Ntau + ll.chunk - 1) / ll.chunk;
  return ll;
}

template <class R>
cudaError_t prepare_line_precond(int W) {
  return raise_smem_limit(line_precond_kernel<R>, line_smem_bytes(sizeof(R), W));
}
template cudaError_t prepare_line_precond<double>(int);
template cudaError_t prepare_line_precond<float>(int);

template <class R>
cudaError_t launch_line_precond(const Geo& g, const LineCoef& lc, const LineLaunch& ll, const C2<R>* r, C2<R>* z,
                                double* part_rz, const CgState* st, cudaStream_t s) {
  const dim3 grid(ll.gx, ll.gy);
  line_precond_kernel<R><<<grid, ll.block, line_smem_bytes(sizeof(R), lc.W), s>>>(g, lc, r, z, part_rz, st);
  return cudaGetLastError();
}

cudaError_t launch_line_precond_batch(const LineBatchDesc<double>* descs, const int4* tiles, int ntiles, int W,
                                     cudaStream_t s) {
  line_precond_batch_kernel<double><<<ntiles, kLineSites * kLineWarps, line_smem_bytes(8, W), s>>>(descs, tiles);
  return cudaGetLastError();
}

cudaError_t prepare_line_precond_batch(int W) {
  return raise_smem_limit(line_precond_batch_kernel<double>, line_smem_bytes(8, W));
}

template cudaError_t launch_line_precond<double>(const Geo&, const LineCoef&, const LineLaunch&, const double2*,
                                                 double2*, double*, const CgState*, cudaStream_t);
template cudaError_t launch_line_precond<float>(const Geo&, const LineCoef&, const LineLaunch&, const float2*,
                                                float2*, double*, const CgState*, cudaStream_t);

// theta_y(x, y) = pi (x mod 2), theta_x = 0 on every slice: the field the
// preconditioner's coefficients are taken at.
__global__ void pi_flux_kernel(Geo g, double* __restrict__ theta) {
  const long long n = (long long)g.V * g.Ntau;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % g.V);
    const int x = s % g.L;
    theta[2 * i] = 0.0;
    theta[2 * i + 1] = (x & 1) ? 3.141592653589793 : 0.0;
  }
}

cudaError_t launch_pi_flux(const Geo& g, double* theta, cudaStream_t s) {
  pi_flux_kernel<<<256, 256, 0, s>>>(g, theta);
  return cudaGetLastError();
}

}  // namespace hqmc
