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
// slice row of the tile is 256 B contiguous in FP32) by tc consecutive slices
// (tc chosen per config so that, where possible, all tiles are resident at once):
//   1. forward:  x_tau = sum_m rho^m u~_{tau-m} for tau in [t0, t1 + W], each
//      warp a contiguous sub-range, as a sliding-window recursion
//      x_tau = rho x_{tau-1} + u~_tau - rho^{W+1} u~_{tau-W-1} started W slices
//      before its sub-range.  u is read straight from global memory, one
//      coalesced row per warp load: a stream for the entering row and one for
//      the leaving row W+1 slices behind (an L1 hit), each keeping its slice
//      index and the sign of its wraps.  x goes to shared memory, the tile's
//      only buffer, so several tiles share an SM;
//   2. backward: y_tau = sum_m rho^m x~_{tau+m} for tau in [t0, t1), the same
//      recursion in descending tau; z = (rho/b) y is written once.
// pCG also needs Re <r, z>.  With z = (rho/b) F^dagger F r it equals
// (rho/b) ||F r||^2 = (rho/b) sum_tau |x_tau|^2, and the tiles' own slices
// [t0, t1) partition the line, so the forward pass sums |x_tau|^2 over them: no
// second read of r, and the sum is positive by construction.
// u~ and x~ are the antiperiodic extensions (a sign flip per wrap); the halo
// rows are read again by the neighbouring tile, mostly from L2, so HBM sees
// one read of r and one write of z.
#include "kernels.h"

#include <algorithm>
#include <vector>

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

// Slices per tile of the fused update-and-preconditioner kernel, and the
// separate kernel's default where no height fits all tiles at once: FP32 128, FP64 64.
template <class R> constexpr int line_tile_slices() { return sizeof(R) == 4 ? 128 : 64; }

// Shared memory of a tile of tc slices: x on slices t0 .. t1 + W.
size_t line_smem_bytes(int real_bytes, int W, int tc) { return (size_t)(tc + W + 1) * kLineSites * 2 * real_bytes; }

// Candidate heights of the separate kernel's tiles.  FP32: tc = ceil(N / k),
// 16 <= tc <= 256, with at least four tiles resident per SM and all tiles
// resident at once (one round), ordered by the recursion work per SM (each
// warp restarts both recursions W slices early: a fixed cost per tile); the
// first is the default, the autotuner times them.  FP64 is bound by the FP64
// FMA rate, so the work per slice decides: the tallest tc = ceil(N / k) <= 256
// that still gives every SM two tiles, else 64.
std::vector<int> line_chunk_candidates(const Geo& g, int real_bytes, int W, int num_sms, size_t smem_per_sm) {
  std::vector<std::pair<double, int>> c;
  const long gx = (g.V + kLineSites - 1) / kLineSites;
  if (real_bytes == 8) {
    for (int k = 1; k <= g.Ntau; ++k) {
      const int tc = (g.Ntau + k - 1) / k;
      if (tc > 256) continue;
      if (tc < 64) break;
      // one tile must fit a block's opt-in shared memory (227 KB) and the SM
      if (line_smem_bytes(real_bytes, W, tc) > std::min(smem_per_sm - 1024, (size_t)227 * 1024)) continue;
      if (gx * ((g.Ntau + tc - 1) / tc) >= 2L * num_sms) return {tc};
    }
    return {line_tile_slices<double>()};
  }
  {
    int last = 0;
    for (int k = 1; k <= g.Ntau; ++k) {
      const int tc = (g.Ntau + k - 1) / k;
      if (tc == last) continue;
      last = tc;
      if (tc > 256) continue;
      if (tc < 16) break;
      const long per_sm = std::min<long>(2048 / (kLineSites * kLineWarps),
                                         (long)(smem_per_sm / (line_smem_bytes(real_bytes, W, tc) + 1024)));
      const long tiles = gx * ((g.Ntau + tc - 1) / tc);
      if (per_sm < 4 || tiles > per_sm * num_sms) continue;
      const double work = (double)((tiles + num_sms - 1) / num_sms) * (2.0 * tc + W + 1 + 2.0 * kLineWarps * W);
      c.push_back({work, tc});
    }
  }
  std::sort(c.begin(), c.end());
  std::vector<int> out;
  for (const auto& e : c) out.push_back(e.second);
  const int dflt = real_bytes == 4 ? line_tile_slices<float>() : line_tile_slices<double>();
  if (std::find(out.begin(), out.end(), dflt) == out.end()) out.push_back(dflt);
  return out;
}

namespace {

// Rows of u for consecutive slices j, j+1, ... of one site: the element, and
// the sign of the antiperiodic extension, (-1)^(wraps of j).  WRAP = false: the
// caller guarantees every slice it reads lies in [0, N) (no index or sign work).
template <class R, bool WRAP>
struct LineStream {
  const C2<R>* p;
  int m;
  R sgn;
  __device__ __forceinline__ void start(const C2<R>* u, int j, int N, int V, int s) {
    if constexpr (WRAP) {
      const LinePos q = line_pos(j, N);
      m = q.m;
      sgn = (R)q.sgn;
      p = u + (size_t)m * V + s;
    } else {
      p = u + (size_t)j * V + s;
    }
  }
  __device__ __forceinline__ C2<R> get() const {
    const C2<R> v = __ldg(p);
    if constexpr (WRAP) return mk(sgn * v.x, sgn * v.y);
    return v;
  }
  __device__ __forceinline__ void next(int N, int V) {
    p += V;
    if constexpr (WRAP) {
      if (++m == N) {
        m = 0;
        p -= (size_t)N * V;
        sgn = -sgn;
      }
    }
  }
};

// Forward pass of one warp: x rows [a, b) (row i is slice t0 + i) into X, and
// the sum of |x|^2 over the rows below nt (the tile's own slices).  Loads are
// issued in batches of kLineBatch rows per stream ahead of the dependent FMAs.
constexpr int kLineBatch = 8;

template <class R, bool WRAP>
__device__ __forceinline__ void line_forward(const C2<R>* __restrict__ u, C2<R>* __restrict__ X, int a, int b,
                                             int t0, int nt, int N, int V, int W, int site, int lane, R rho, R rw,
                                             R& xx) {
  using T = C2<R>;
  LineStream<R, WRAP> in, out;
  in.start(u, t0 + a - W, N, V, site);  // slices t0+a-W .. t0+a for the first window
  out = in;
  T acc = mk(R(0), R(0));
  int m = 0;
  for (; m + kLineBatch <= W + 1; m += kLineBatch) {
    T v[kLineBatch];
#pragma unroll
    for (int k = 0; k < kLineBatch; ++k) {
      v[k] = in.get();
      in.next(N, V);
    }
#pragma unroll
    for (int k = 0; k < kLineBatch; ++k) acc = caxpy(v[k], rho, acc);
  }
  for (; m <= W; ++m) {
    acc = caxpy(in.get(), rho, acc);
    in.next(N, V);
  }
  X[a * kLineSites + lane] = acc;
  if (a < nt) xx += cdot_re_own(acc, acc);
  int i = a + 1;
  for (; i + kLineBatch <= b; i += kLineBatch) {
    T vi[kLineBatch], vo[kLineBatch];
#pragma unroll
    for (int k = 0; k < kLineBatch; ++k) {
      vi[k] = in.get();
      vo[k] = out.get();
      in.next(N, V);
      out.next(N, V);
    }
#pragma unroll
    for (int k = 0; k < kLineBatch; ++k) {
      acc = caxpy(caxpy(vi[k], rho, acc), -rw, vo[k]);  // enters slice t0+i+k, leaves t0+i+k-W-1
      X[(i + k) * kLineSites + lane] = acc;
      if (i + k < nt) xx += cdot_re_own(acc, acc);
    }
  }
  for (; i < b; ++i) {
    acc = caxpy(caxpy(in.get(), rho, acc), -rw, out.get());
    in.next(N, V);
    out.next(N, V);
    X[i * kLineSites + lane] = acc;
    if (i < nt) xx += cdot_re_own(acc, acc);
  }
}

}  // namespace

// One tile (site block bx, slice block by of a gx-wide grid) of z = Otilde^{-1} u
// with its partial of <u, z> in part[by * gx + bx].
template <class R>
__device__ __forceinline__ void line_precond_tile(const Geo& g, const LineCoef& lc, int tc,
                                                  const C2<R>* __restrict__ u, C2<R>* __restrict__ z,
                                                  double* __restrict__ part, int bx, int by, int gx) {
  using T = C2<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int N = g.Ntau, V = g.V, W = lc.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s0 = bx * kLineSites, s = s0 + lane;
  const bool site_ok = s < V;
  const int sr = site_ok ? s : V - 1;  // lanes past the last site read a valid one and store nothing
  const int t0 = by * tc, t1 = min(N, t0 + tc), nt = t1 - t0;
  const int nx = nt + W + 1;  // rows of x: slices t0 .. t1 + W
  T* X = reinterpret_cast<T*>(smem_raw);
  const R rho = (R)lc.rho, rw = (R)lc.rhoW1, sc = (R)lc.scale;
  R xx = 0;  // sum of |x_tau|^2 over this thread's own slices (FP32: in float, cdot_re_own)

  // The tile reads slices t0 - W .. t1 + W of its sites: request all of them
  // into L2 at once (128-byte lines), so that the recursions' dependent loads
  // meet L2 latency rather than DRAM latency.
  {
    const int lines_per_row = (min(kLineSites, V - s0) * (int)sizeof(T) + 127) / 128;
    const int nrow = nt + 2 * W + 1;
    for (int k = threadIdx.x; k < nrow * lines_per_row; k += blockDim.x) {
      const int row = k / lines_per_row, l = k - row * lines_per_row;
      const int j = t0 - W + row;
      const int m = ((unsigned)j < (unsigned)N) ? j : line_pos(j, N).m;
      const char* pl = reinterpret_cast<const char*>(u + (size_t)m * V + s0) + 128 * l;
      asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pl));
    }
  }

  // 1. forward: rows of x split over the warps; x row i is slice t0 + i
  {
    const int per = (nx + kLineWarps - 1) / kLineWarps;
    const int a = warp * per, b = min(nx, a + per);  // x rows [a, b)
    if (a < b) {
      // slices read: t0 + a - W .. t0 + b - 1
      if (t0 + a - W >= 0 && t0 + b - 1 < N)
        line_forward<R, false>(u, X, a, b, t0, nt, N, V, W, sr, lane, rho, rw, xx);
      else
        line_forward<R, true>(u, X, a, b, t0, nt, N, V, W, sr, lane, rho, rw, xx);
    }
  }
  __syncthreads();
  // 2. backward over the tile's own slices, split over the warps
  {
    const int per = (nt + kLineWarps - 1) / kLineWarps;
    const int a = warp * per, b = min(nt, a + per);  // output rows [a, b)
    if (a < b) {
      T acc = mk(R(0), R(0));
#pragma unroll 4
      for (int m = W; m >= 0; --m) acc = caxpy(X[(b - 1 + m) * kLineSites + lane], rho, acc);
      for (int i = b - 1;; --i) {
        if (site_ok) z[(size_t)(t0 + i) * V + s] = cscale(sc, acc);
        if (i == a) break;
        acc = caxpy(caxpy(X[(i - 1) * kLineSites + lane], rho, acc), -rw, X[(i + W) * kLineSites + lane]);
      }
    }
  }
  if (part) {
    const double tot = block_sum(site_ok ? (double)sc * (double)xx : 0.0, red);
    if (threadIdx.x == 0) part[by * gx + bx] = tot;
  }
}

template <class R>
__global__ void __launch_bounds__(kLineSites* kLineWarps) line_precond_kernel(Geo g, LineCoef lc, int tc,
                                                                             const C2<R>* __restrict__ u,
                                                                             C2<R>* __restrict__ z,
                                                                             double* __restrict__ part,
                                                                             const CgState* st) {
  if (!line_gate(st)) return;  // uniform over the grid
  line_precond_tile<R>(g, lc, tc, u, z, part, blockIdx.x, blockIdx.y, gridDim.x);
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
  line_precond_tile<R>(d.g, d.lc, d.tc, d.u, d.z, d.part, t.y, t.z, d.gx);
}

// Preconditioned CG, fused update and preconditioner (one launch per iteration
// after the direction step):
//   alpha = <r, z>_k / <p, O p> from the direction kernel's partials (stop on a
//   non-positive or non-finite <p, O p>, as the plain update does);
//   r <- r - alpha q and x <- x + alpha p on the tile's own slices;
//   z = Otilde^{-1} r on the updated r, with the partials of <r, r> (convergence)
//   and <r, z> (next step length).
// The tile stages r and q on its slices and halo in shared memory by cp.async
// (fixed tiles of line_tile_slices rows), forms r - alpha q there (the halo rows
// with the same arithmetic as the tiles that own them), then runs the same two
// recursions as line_precond_kernel over the staged rows; <r, z> is summed
// directly.  (A streaming form like line_precond_kernel's was slower here: it
// re-reads r and q for the leaving row.)  The updated r goes to a second
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

LineLaunch line_launch(const Geo& g, int chunk) {
  LineLaunch ll;
  ll.chunk = chunk;
  ll.block = kLineSites * kLineWarps;
  ll.gx = (g.V + kLineSites - 1) / kLineSites;
  ll.gy = (g.Ntau + ll.chunk - 1) / ll.chunk;
  return ll;
}

LineLaunch line_update_launch(const Geo& g, int real_bytes) {
  return line_launch(g, real_bytes == 4 ? line_tile_slices<float>() : line_tile_slices<double>());
}

template <class R>
cudaError_t prepare_line_precond(int W, int tc) {
  return raise_smem_limit(line_precond_kernel<R>, line_smem_bytes(sizeof(R), W, tc));
}
template cudaError_t prepare_line_precond<double>(int, int);
template cudaError_t prepare_line_precond<float>(int, int);

template <class R>
cudaError_t launch_line_precond(const Geo& g, const LineCoef& lc, const LineLaunch& ll, const C2<R>* r, C2<R>* z,
                                double* part_rz, const CgState* st, cudaStream_t s) {
  const dim3 grid(ll.gx, ll.gy);
  line_precond_kernel<R><<<grid, ll.block, line_smem_bytes(sizeof(R), lc.W, ll.chunk), s>>>(g, lc, ll.chunk, r, z,
                                                                                            part_rz, st);
  return cudaGetLastError();
}

cudaError_t launch_line_precond_batch(const LineBatchDesc<double>* descs, const int4* tiles, int ntiles, int W,
                                     int tc, cudaStream_t s) {
  line_precond_batch_kernel<double><<<ntiles, kLineSites * kLineWarps, line_smem_bytes(8, W, tc), s>>>(descs, tiles);
  return cudaGetLastError();
}

cudaError_t prepare_line_precond_batch(int W, int tc) {
  return raise_smem_limit(line_precond_batch_kernel<double>, line_smem_bytes(8, W, tc));
}

cudaError_t launch_line_precond_batch(const LineBatchDesc<float>* descs, const int4* tiles, int ntiles, int W,
                                     int tc, cudaStream_t s) {
  line_precond_batch_kernel<float><<<ntiles, kLineSites * kLineWarps, line_smem_bytes(4, W, tc), s>>>(descs, tiles);
  return cudaGetLastError();
}

cudaError_t prepare_line_precond_batch32(int W, int tc) {
  return raise_smem_limit(line_precond_batch_kernel<float>, line_smem_bytes(4, W, tc));
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
