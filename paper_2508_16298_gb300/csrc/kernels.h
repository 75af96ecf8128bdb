// Host-side launch interface of the HQMC kernels (internal to libhqmc).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace hqmc {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it: several configs of different sizes share the kernel in a process).
template <class F>
inline cudaError_t raise_smem_limit(F* kernel, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void*)kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch shape of the slice kernels: one CTA per imaginary-time slice, grouped
// into thread-block clusters of `cluster` consecutive slices.
struct SliceLaunch {
  Geo g;
  int threads;   // threads per CTA
  int cluster;   // CTAs per cluster (consecutive slices)
  int grid;      // CTAs, a multiple of cluster, >= Ntau
  int mb;        // bonds of each family per thread held in registers (1..4; 0: links from global)
  int nby;       // register-blocked kernel: 2x2 blocks stacked per thread strip (0: not used)
  int walk;      // 1: persistent tau-walking kernel (FP32): `grid` CTAs, each a contiguous range of slices
};

enum { MODE_APPLY = 0, MODE_RESID = 1, MODE_CGDIR = 2 };

template <class R>
struct MdagmArgs {
  Geo g;
  R cB;                    // cosh(a) cosh(a/2)^6
  const C2<R>* U;          // link table, two complex links per site
  const C2<R>* x;          // APPLY / RESID input
  C2<R>* y;                // APPLY output; CGDIR: q = O p
  const double2* b;        // RESID right-hand side (complex double)
  void* r_out;             // RESID residual b - O x (complex double, or float if r_out_fp32)
  int r_out_fp32;
  const C2<R>* r;          // CGDIR residual
  C2<R>* pbuf[2];          // CGDIR directions: iteration k reads pbuf[k&1], writes pbuf[(k+1)&1]
  const double* part_in;   // CGDIR: partials of <r, r> from the update kernel
  int n_part_in;
  double* part_out;        // per-CTA partials: CGDIR <p, Op>; RESID <r,r> then <b,b>
  CgState* st;
  int gate;                // RESID: GATE_* condition on st->done (GATE_ALWAYS needs no st)
  const float2* th32;      // register-blocked FP32 kernel: (theta_x, theta_y) per site, wrapped to [-pi, pi)
  double t1, t2;           // tanh(a), tanh(a/2)
  int teff;                // generic kernel: threads that take part in the site loops (0: the whole block);
                           // a batch sets each chain's own block size so sums group sites as in its own launch
  const double* part_rz;   // CGDIR, preconditioned CG: partials of <r, z> (z = Otilde^{-1} r; x/r read z)
  int n_part_rz;
  int* err;                // set to 1 by a kernel whose bounded device-side wait gave up (NULL: not recorded)
  const double* part_cross;  // CGDIR, flexible CG: partials of Re<r_old, z> (Polak-Ribiere beta), n_part_rz of them
};

// First step of a CG-direction launch (one warp): read the CG state, decide
// whether this iteration runs, and compute beta = <r,r>_k / <r,r>_{k-1} from
// the update kernel's partials.  The writer block records the outcome in the state.
// Preconditioned CG (a.part_rz set, Eq. (pCG)): <r,r> still decides
// convergence, while rz = <r, Otilde^{-1} r> takes its place in beta and, kept in
// st->rr, in the step length.
// s_flags: bit 0 = skip the launch (uniform over the grid), bit 1 = first
// iteration of a recurrence segment (p = r, or p = z).
// Partial sums of the head: four running sums per lane for the FP32 kernels (their
// other registers dominate, and the dependent FP64 additions are slow); the compact
// sum for the FP64 kernels, whose occupancy the extra registers would lower.
template <class R>
__device__ __forceinline__ double head_sum(const double* p, int n) {
  if constexpr (sizeof(R) == 4) return warp_sum_partials4(p, n);
  return warp_sum_partials(p, n);
}

// Where the head finds the CG state and the partial arrays: the launch's own
// (HeadOwn, read from the arguments where they are used) or those of one system
// of a multi-system launch (HeadAt).
template <class R>
struct HeadOwn {
  const MdagmArgs<R>& a;
  __device__ __forceinline__ CgState* st() const { return a.st; }
  __device__ __forceinline__ const double* part_in() const { return a.part_in; }
  __device__ __forceinline__ const double* part_rz() const { return a.part_rz; }
  __device__ __forceinline__ const double* part_cross() const { return a.part_cross; }
};
struct HeadAt {
  CgState* s;
  const double *pin, *prz, *pcr;
  __device__ __forceinline__ CgState* st() const { return s; }
  __device__ __forceinline__ const double* part_in() const { return pin; }
  __device__ __forceinline__ const double* part_rz() const { return prz; }
  __device__ __forceinline__ const double* part_cross() const { return pcr; }
};

template <class R, class P>
__device__ __forceinline__ void cgdir_head_impl(const MdagmArgs<R>& a, const P& ptr, bool writer, int& s_flags,
                                                R& s_beta, int& s_k) {
  if (threadIdx.x < 32) {
    CgState* st = ptr.st();
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
      if (ptr.part_rz()) {
        const double rz = head_sum<R>(ptr.part_rz(), a.n_part_rz);
        if (!isfinite(rz) || !(rz > 0.0)) {
          flags = 1;
          new_done = isfinite(rz) ? CG_BREAKDOWN : CG_NONFINITE;
        } else if (writer && lane == 0) {
          st->rr[k & 1] = rz;
        }
      }
    } else {
      const double rr = head_sum<R>(ptr.part_in(), a.n_part_in);
      const double rz = ptr.part_rz() ? head_sum<R>(ptr.part_rz(), a.n_part_rz) : rr;
      // flexible CG: beta = Re<z_k, r_k - r_{k-1}> / Re<z_{k-1}, r_{k-1}> (Polak-Ribiere)
      const double cross = ptr.part_cross() ? head_sum<R>(ptr.part_cross(), a.n_part_rz) : 0.0;
      if (!isfinite(rr) || !isfinite(rz) || !isfinite(cross)) {
        flags = 1;
        new_done = CG_NONFINITE;
      } else if (rr <= st->tol2bb) {
        flags = 1;
        new_done = CG_REC_CONVERGED;
      } else if (!(rz > 0.0)) {
        flags = 1;
        new_done = CG_BREAKDOWN;
      } else {
        beta = (rz - cross) / st->rr[(k - 1) & 1];
      }
      if (writer && lane == 0) {
        if (!ptr.part_rz()) {
          st->rr[k & 1] = rr;
        } else {
          st->rr_rec = rr;
          if (!(flags & 1)) st->rr[k & 1] = rz;
        }
      }
    }
    if (writer && lane == 0) {
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
}

template <class R>
__device__ __forceinline__ void cgdir_head(const MdagmArgs<R>& a, bool writer, int& s_flags, R& s_beta,
                                           int& s_k) {
  cgdir_head_impl<R>(a, HeadOwn<R>{a}, writer, s_flags, s_beta, s_k);
}

// The head of one system of a multi-system launch (its state and partials given).
template <class R>
__device__ __forceinline__ void cgdir_head_at(const MdagmArgs<R>& a, bool writer, int& s_flags, R& s_beta,
                                              int& s_k, CgState* st, const double* part_in, const double* part_rz,
                                              const double* part_cross) {
  cgdir_head_impl<R>(a, HeadAt{st, part_in, part_rz, part_cross}, writer, s_flags, s_beta, s_k);
}

// Fused M^dagger M (three modes).
template <class R, int MODE>
cudaError_t launch_mdagm(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s);
template <class R, int MODE>
cudaError_t prepare_mdagm(const SliceLaunch& sl);
// Clusters of sl.cluster CTAs the device can keep resident (<= 0: none / error).
int mdagm_max_active_clusters(const SliceLaunch& sl);

// Register-blocked fused M^dagger M (APPLY and CGDIR modes; sl.nby in 1..3).
template <class R, int MODE>
cudaError_t launch_mdagm_block(const SliceLaunch& sl, const MdagmArgs<R>& a, cudaStream_t s);
template <class R, int MODE>
cudaError_t prepare_mdagm_block(const SliceLaunch& sl);
// Largest block for a strip of nby 2x2 blocks in this precision (0: not available).
int block_thread_cap(int real_bytes, int nby);
int mdagm_block_max_active_clusters(const SliceLaunch& sl, int real_bytes);

// Persistent tau-walking fused M^dagger M in FP32 (APPLY and CGDIR modes;
// sl.nby in 1..3, sl.grid CTAs <= Ntau, one contiguous slice range each).
template <int MODE>
cudaError_t launch_mdagm_walk(const SliceLaunch& sl, const MdagmArgs<float>& a, cudaStream_t s);
template <int MODE>
cudaError_t prepare_mdagm_walk(const SliceLaunch& sl);
int walk_thread_cap(int nby);
size_t walk_smem_bytes(const Geo& g, int mode);
int mdagm_walk_blocks_per_sm(const SliceLaunch& sl);
// Multi-system tau-walking launch: nsys systems on one field; CTA b serves system
// b % nsys and slice range b / nsys.  System k's vectors (r or z, pbuf, y) start
// vstride elements after system k - 1's, its CG state is a.st[k], and its partial
// arrays (part_in, part_rz, part_out) start pstride doubles after system k - 1's.
struct MultiStride {
  int nsys;
  long long vstride;
  int pstride;
};
// CG-direction mode: sl.grid slice ranges per system, sl.grid * ms.nsys CTAs.
cudaError_t launch_mdagm_walk_multi(const SliceLaunch& sl, const MdagmArgs<float>& a, const MultiStride& ms,
                                    cudaStream_t s);
cudaError_t prepare_mdagm_walk_multi(const SliceLaunch& sl);
int mdagm_walk_multi_blocks_per_sm(const SliceLaunch& sl);

// Tau-line preconditioner (precond.cu): z = (rho/b) F_W^dagger F_W r per site.
struct LineCoef {
  double rho;    // bulk Cholesky ratio of the pi-flux tau-line matrix
  double rhoW1;  // rho^(W+1)
  double scale;  // rho / b
  int W;         // powers of rho S kept in the truncated Neumann series
};
struct LineLaunch {
  int chunk;  // slices per tile
  int block;  // threads per block
  int gx, gy; // grid: site tiles x slice tiles (gx * gy partials of <r, z>)
};
// Separate preconditioner kernel: tiles of `chunk` slices.
LineLaunch line_launch(const Geo& g, int chunk);
// Fused update-and-preconditioner kernel: its fixed tile height.
LineLaunch line_update_launch(const Geo& g, int real_bytes);
size_t line_smem_bytes(int real_bytes, int W, int tc);
std::vector<int> line_chunk_candidates(const Geo& g, int real_bytes, int W, int num_sms, size_t smem_per_sm);
template <class R>
cudaError_t prepare_line_precond(int W, int tc);
// z = Otilde^{-1} r and partials of <r, z>; gated on st->done == CG_RUNNING unless st is NULL.
template <class R>
cudaError_t launch_line_precond(const Geo& g, const LineCoef& lc, const LineLaunch& ll, const C2<R>* r, C2<R>* z,
                                double* part_rz, const CgState* st, cudaStream_t s);
cudaError_t launch_pi_flux(const Geo& g, double* theta, cudaStream_t s);

// Batched preconditioner: one launch over the tiles (chain, bx, by) of many chains.
template <class R>
struct LineBatchDesc {
  Geo g;
  LineCoef lc;
  const C2<R>* u;
  C2<R>* z;
  double* part;
  const CgState* st;
  int gx;  // the chain's own tile grid width (partial index by * gx + bx)
  int tc;  // slices per tile, as in the chain's own launch
};
cudaError_t launch_line_precond_batch(const LineBatchDesc<double>* descs, const int4* tiles, int ntiles, int W,
                                     int tc, cudaStream_t s);
cudaError_t prepare_line_precond_batch(int W, int tc);
// The same in FP32 (the systems of a multi-system mixed solve).
cudaError_t launch_line_precond_batch(const LineBatchDesc<float>* descs, const int4* tiles, int ntiles, int W,
                                     int tc, cudaStream_t s);
cudaError_t prepare_line_precond_batch32(int W, int tc);

// Preconditioned CG: the vector update fused with the preconditioner (precond.cu).
template <class R>
struct LineUpdArgs {
  C2<R>* x;               // iterate (FP64) or FP32 correction (mixed)
  const C2<R>* r_in;      // residual before the step (read with halos)
  C2<R>* r_out;           // residual after the step (a different buffer)
  const C2<R>* p0;        // directions: the one used is pbuf[(k2+1)&1]
  const C2<R>* p1;
  const C2<R>* q;         // O p
  C2<R>* z;               // Otilde^{-1} r (output)
  const double* part_pq;  // partials of <p, O p>
  int n_pq;
  double* part_rr;        // per-tile partials of <r, r> and <r, z>
  double* part_rz;
  CgState* st;
};
size_t line_update_smem_bytes(int real_bytes, int W);
template <class R>
cudaError_t prepare_line_update(int W);
template <class R>
cudaError_t launch_line_update(const Geo& g, const LineCoef& lc, const LineLaunch& ll, const LineUpdArgs<R>& a,
                               cudaStream_t s);

// Fused M^dagger M over many chains in one launch (generic kernel, links from
// memory): CTA b runs cluster tile b / C = (chain, first slice) of `tiles`.
template <class R, int MODE>
cudaError_t launch_mdagm_batch(const MdagmArgs<R>* descs, const int2* tiles, int ntiles, int C, int threads,
                               size_t smem, cudaStream_t s);
// Clusters of C CTAs (threads, smem each) of the batched FP64 kernel the device keeps resident.
int mdagm_batch_max_active_clusters(int C, int threads, size_t smem);

// y = M x or M^dagger x.
template <class R>
cudaError_t launch_apply_M(const SliceLaunch& sl, R cB, const C2<R>* U, const C2<R>* x, C2<R>* y,
                           int dagger, cudaStream_t s);
template <class R>
cudaError_t prepare_apply_M(const SliceLaunch& sl);

// Link tables U = t_f e^{i theta} (double and/or float), theta -> links.
// th32 (optional): theta as float, wrapped to [-pi, pi), for the FP32 register-blocked kernel.
cudaError_t launch_links(const Geo& g, const double* theta, double t1, double t2, double2* U64,
                         float2* U32, float2* th32, cudaStream_t s);

// CG update x += alpha p, r -= alpha q, partial <r,r>; MIXED: x is the float
// correction.  Reads alpha from the partials of <p, Op>.
// The direction used is pbuf[(k2+1)&1], the one the direction kernel wrote.
template <class R>
cudaError_t launch_cg_update(long long n, int grid, void* x, int x_is_double, C2<R>* r,
                             C2<R>* const pbuf[2], const C2<R>* q, const double* part_pq, int n_pq,
                             double* part_rr, CgState* st, cudaStream_t s);

// Arguments of the CG update for one chain.
template <class R>
struct UpdArgs {
  long long n;
  void* x;
  int x_is_double;
  C2<R>* r;
  C2<R>* p0;
  C2<R>* p1;
  const C2<R>* q;
  const double* part_pq;
  int n_pq;
  double* part_rr;
  CgState* st;
};

// Arguments of the residual bookkeeping for one chain.
struct FinArgs {
  const double* part;
  int n;
  double* part_rr_out;
  int n_rr_out;
  CgState* st;
  double* report;
};

// Batched CG update: descs is a device array of per-chain UpdArgs<double>;
// blocks[b] = (chain, local block), nblocks[chain].
cudaError_t launch_cg_update_batch(const void* descs, const int2* blocks, const int* nblocks, int total_blocks,
                                   cudaStream_t s);
// FP32 update of nsys systems stored back to back (base: system 0's arguments, a FP32
// correction x; system k's vectors at k vstride elements, its partials at k pstride,
// its state at base.st + k), blocks_per_system blocks each (= partials of <r, r>).
cudaError_t launch_cg_update_multi(const UpdArgs<float>& base, long long vstride, int pstride, int nsys,
                                   int blocks_per_system, cudaStream_t s);
int cg_update_multi_blocks_per_sm();

enum { FIN_START = 0, FIN_RESTART = 1, FIN_RELIABLE = 2, FIN_REPORT = 3 };


// Batched finalize (every FIN_* mode, as resid_finalize), one block per chain;
// descs: device array of FinArgs.
cudaError_t launch_resid_finalize_batch(const void* descs, int nchains, int mode, double tol, int maxit, int gate,
                                        cudaStream_t s);
// bodies (nullable): device counter of loop bodies, incremented once per body.
cudaError_t launch_loop_condition_batch(CgState* const* states, int nchains, cudaGraphConditionalHandle h,
                                        cudaStream_t s, unsigned long long* bodies = nullptr);
// Sums the RESID partials into the CG state.
cudaError_t launch_resid_finalize(const double* part, int n, int mode, double tol, int maxit,
                                  double* part_rr_out, int n_rr_out, CgState* st, double* report,
                                  int gate, cudaStream_t s);

// Flexible CG: partials of Re<r, z> and Re<r_old, z> (grid blocks each), skipped
// unless the solve is running.
cudaError_t launch_fcg_dots(long long n, const float2* r, const float2* r_old, const float2* z, int grid,
                            double* part_rz, double* part_cross, const CgState* st, cudaStream_t s);

// x64 += xh32; xh32 = 0 (gated on st->done unless st is NULL).
cudaError_t launch_accumulate_correction(long long n, double2* x, float2* xh, const CgState* st, int gate,
                                         cudaStream_t s);
// The same for nsys systems stored back to back (system k: x + k n, xh + k n, st + k).
cudaError_t launch_accumulate_correction_multi(long long n, int nsys, double2* x, float2* xh, const CgState* st,
                                               int gate, cudaStream_t s);

// Ends a device-side CG loop body: counts it and sets the WHILE condition to
// "still running", forcing CG_MAXIT once loop_cap bodies have run.
cudaError_t launch_loop_condition(CgState* st, cudaGraphConditionalHandle h, cudaStream_t s);

// Fermion force dS_f/dtheta given X (FP64).
cudaError_t launch_force(const SliceLaunch& sl, double cB, double t1, double t2, const double2* U, const double2* X,
                         double* dSf, cudaStream_t s);
cudaError_t prepare_force(const SliceLaunch& sl);

struct BosonParams {
  double cK;      // 1/(J dtau)
  double Kdtau;   // K * dtau
  int noncompact;
};
// F = -dSf - dS_B(theta).
cudaError_t launch_force_finish(const Geo& g, const BosonParams& bp, const double* theta,
                                const double* dSf, double* F, cudaStream_t s);
// p += h F
cudaError_t launch_kick(long long nb, double* p, const double* F, double h, cudaStream_t s);
// p += h F; theta += 2 dt p
cudaError_t launch_kick_drift(long long nb, double* p, double* theta, const double* F, double h,
                              double dt, cudaStream_t s);
// terms[0] = S_B, terms[1] = sum p^2, terms[2] = Re <a, b>  (device doubles)
cudaError_t launch_action_terms(const Geo& g, const BosonParams& bp, const double* theta,
                                const double* p, const double2* a, const double2* b, int grid,
                                double* part, double* terms, cudaStream_t s);
// Philox draws.
cudaError_t launch_draw(long long n_sites, uint64_t seed, uint64_t counter, double* p, double2* R,
                        cudaStream_t s);
void philox_uniform_host(uint64_t seed, uint64_t counter, double* u);
// v ~ CN(0, 1) per site from Philox stream `stream` (3: stochastic-estimation vectors).
cudaError_t launch_draw_vector(long long n_sites, uint64_t seed, uint32_t stream, uint64_t counter, double2* v,
                               cudaStream_t s);
// out[0] + i out[1] = <a, b> = sum conj(a_i) b_i; part holds 2 * grid doubles.
// r = phi - y, y from an FP32 apply (the learned guess's input residual).
cudaError_t launch_resid_from_fp32(long long n, const double2* phi, const float2* y, double2* r, cudaStream_t s);
cudaError_t launch_cdot(long long n, const double2* a, const double2* b, int grid, double* part, double* out,
                        cudaStream_t s);
// out[2 i], out[2 i + 1] = <X_i, b> (re, im) for X_i = X + i * stride, i < k; part holds 2 * grid * k doubles.
cudaError_t launch_cdot_many(long long n, const double2* X, long long stride, int k, const double2* b, int grid,
                             double* part, double* out, cudaStream_t s);
// y *= a (real), in place
cudaError_t launch_dscale(long long n, double a, double2* y, cudaStream_t s);
// y += (cr + i ci) x (x and y distinct)
cudaError_t launch_caxpy(long long n, double cr, double ci, const double2* x, double2* y, cudaStream_t s);
// FP64 FMA throughput probe (16 flops per thread per iteration).
cudaError_t launch_fp64_probe(int blocks, int threads, int iters, double* out, cudaStream_t s);

// Learned preconditioner (net.cu).  Weights are BF16 [7][cout][cin] per layer.
cudaError_t launch_net_layer(const Geo& g, const float2* th32, const void* W, int cin, int cout, const float2* in,
                             float2* out, cudaStream_t s);
// Inference layer with the weights passed by value from host memory ([7][cout][cin] FP32 values of
// the BF16 weights): the same arithmetic as launch_net_layer.
// st (nullable): skip the launch unless the solve is running (flexible CG).
// tensor_cores: the 16-channel activations are BF16 in the chunk layout (net.cu);
// 1 -> 16 runs on CUDA cores and rounds its output, 16 -> 16 and 16 -> 1 are
// BF16 mma.sync products with FP32 accumulation.  Otherwise every layer is FP32
// on CUDA cores with channel-planar activations.  Every layer of one pass must
// use the same setting.
cudaError_t launch_net_layer_host_weights(const Geo& g, const float2* th32, const float* w, int cin, int cout,
                                         const float2* in, float2* out, const CgState* st, cudaStream_t s,
                                         bool tensor_cores = false);
cudaError_t launch_net_wgrad(const Geo& g, const float2* th32, int cin, int cout, const float2* d, const float2* h,
                             double* partials, int nchunks, cudaStream_t s);
cudaError_t launch_net_loss(const float2* h, const double2* x, const double* xx, float2* d, double* part, int nblocks,
                            long long n, cudaStream_t s);
cudaError_t launch_net_adam(float* w, float* m, float* v, const double* partials, int nchunks, int nw, void* wb,
                            float lr, float b1, float b2, float c1, float c2, float eps, float scale, cudaStream_t s);
cudaError_t launch_net_adjoint_weights(const void* W, void* Wt, int cin, int cout, cudaStream_t s);
cudaError_t launch_net_convert(const void* in, void* out, int to_float, double scale, long long n, cudaStream_t s);

// ---- batched trajectories (one graph per trajectory of many chains) ----------
// One chain of a batch as the batched trajectory kernels see it (device array,
// rewritten before every trajectory: the field pointer, seed and dt may change).
struct ChainDesc {
  Geo g;
  BosonParams bp;
  double cB, t1, t2;
  double inv1, inv2;         // 1 / (1 - t1^2), 1 / (1 - t2^2), computed on the host as for a single chain
  long long n;               // sites
  double* theta;             // the caller's field (in/out)
  double* th0;               // the field at the start of the trajectory
  double* p;                 // momenta
  double2* R;                // pseudofermion draw
  double2* eta;              // phi = M^dagger R
  double2* X;                // CG solution (and initial guess)
  double* F;                 // total force
  double* dSf;               // fermion part
  double2* U64;              // link table
  double* part_act;          // action partials (4 per block)
  int act_grid;              // blocks of the chain's action reduction (as in its own launch)
  double* terms;             // H0 terms [0..2], H1 terms [3..5]
  const CgState* st;         // CG state of the chain's solves
  const double* report;      // true <r, r>, <phi, phi> of the last residual
  uint64_t seed;
  double dt;
  hqmc_traj_info* info;      // device copy of the chain's trajectory info
};
// Block tables of the batched kernels: int4 (chain, local block, blocks of that chain, 0).
enum { BT_DRAW = 0, BT_LINKS = 1, BT_ZERO_X = 2, BT_SAVE = 3, BT_RESTORE = 4, BT_KICK_DRIFT = 5, BT_KICK = 6 };
cudaError_t launch_batch_elementwise(const ChainDesc* d, const int4* tab, int nblocks, int op, const uint64_t* counter,
                                     cudaStream_t s);
// Hamiltonian terms of every chain: which = 0 (H0: p, R, R) or 1 (H1: p, eta, X), into terms[3 * which ...].
cudaError_t launch_batch_action(const ChainDesc* d, const int4* tab, int nblocks, int nchains, int which,
                                cudaStream_t s);
cudaError_t launch_batch_force_finish(const ChainDesc* d, const int4* tab, int nblocks, cudaStream_t s);
// Per-chain bookkeeping: info reset (with the Metropolis uniform), after each solve, and the Metropolis test.
cudaError_t launch_batch_info_init(const ChainDesc* d, int nchains, const uint64_t* counter, cudaStream_t s);
cudaError_t launch_batch_solve_close(const ChainDesc* d, int nchains, cudaStream_t s);
cudaError_t launch_batch_metropolis(const ChainDesc* d, int nchains, cudaStream_t s);
// eta = M^dagger R (FP64) and the fermion force, one CTA per (chain, slice) of `tiles`.
cudaError_t launch_batch_apply_Mdag(const ChainDesc* d, const int2* tiles, int ntiles, int threads, size_t smem,
                                    cudaStream_t s);
cudaError_t launch_batch_force(const ChainDesc* d, const int2* tiles, int ntiles, int threads, size_t smem,
                               cudaStream_t s);

}  // namespace hqmc
