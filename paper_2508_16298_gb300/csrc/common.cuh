// Device-side building blocks shared by the HQMC kernels (sm_103a).
//
// Storage conventions (see include/hqmc.h): slice-major vectors v[tau][y][x]
// of interleaved complex numbers; theta[tau][y][x][c]; site s = x + L*y.
//
// The checkerboard product of Eq. (eq24) is evaluated in a factored form:
// every family factor e^{alpha T_f} equals cosh(alpha) * (1 + tanh(alpha) T_f)
// because T_f^2 = 1 and every site belongs to exactly one bond of each family.
// Hence B = cB * P with the scalar cB = cosh(a) cosh(a/2)^6 and
//   P = (1 + t2 T4)(1 + t2 T3)(1 + t2 T2)(1 + t1 T1)(1 + t2 T2)(1 + t2 T3)(1 + t2 T4),
// t1 = tanh(a), t2 = tanh(a/2), a = dtau*t.  The per-bond link factor
// U = t_f e^{i theta} ("link table") is computed once per gauge field, so the
// inner sweep is two complex FMAs per bond endpoint:
//   v_i <- v_i + U v_j,   v_j <- v_j + conj(U) v_i.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "status.h"

namespace hqmc {

template <class R> struct CT;
template <> struct CT<double> { using T = double2; };
template <> struct CT<float> { using T = float2; };
template <class R> using C2 = typename CT<R>::T;

__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

// a + u * b
template <class T> __device__ __forceinline__ T cfma(T a, T u, T b) {
  return mk(fma(u.x, b.x, fma(-u.y, b.y, a.x)), fma(u.x, b.y, fma(u.y, b.x, a.y)));
}
// a + conj(u) * b
template <class T> __device__ __forceinline__ T cfmac(T a, T u, T b) {
  return mk(fma(u.x, b.x, fma(u.y, b.y, a.x)), fma(u.x, b.y, fma(-u.y, b.x, a.y)));
}
// a + s * b (s real)
template <class T, class R> __device__ __forceinline__ T caxpy(T a, R s, T b) {
  return mk(fma(s, b.x, a.x), fma(s, b.y, a.y));
}
template <class T, class R> __device__ __forceinline__ T cscale(R s, T b) { return mk(s * b.x, s * b.y); }
// Re(conj(a) * b), with its rounding written out (one product rounded, one fused)
// so that every kernel that inlines it rounds alike
template <class T> __device__ __forceinline__ double cdot_re(T a, T b) {
  return fma((double)a.x, (double)b.x, __dmul_rn((double)a.y, (double)b.y));
}
// Re(conj(a) * b) in the vector's own precision.  FP32 kernels sum a thread's
// few terms this way and promote once: FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU, so a per-site double accumulation
// would dominate an FP32 kernel.
__device__ __forceinline__ float cdot_re_own(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ double cdot_re_own(double2 a, double2 b) { return cdot_re(a, b); }

// Slice geometry.
struct Geo {
  int L;      // spatial extent (even)
  int V;      // L*L
  int half;   // L/2
  int Ntau;   // slices
};

// Bond number b in [0, V/2) of checkerboard family fam (1..4): tail site i,
// head site j and bond direction c.
__device__ __forceinline__ void bond_of(const Geo& g, int fam, int b, int& i, int& j, int& c) {
  if (fam <= 2) {
    int y = b / g.half;
    int x = 2 * (b - y * g.half) + (fam - 1);
    int xp = (x + 1 == g.L) ? 0 : x + 1;
    i = x + g.L * y;
    j = xp + g.L * y;
    c = 0;
  } else {
    int k = b / g.L;
    int x = b - k * g.L;
    int y = 2 * k + (fam - 3);
    int yp = (y + 1 == g.L) ? 0 : y + 1;
    i = x + g.L * y;
    j = x + g.L * yp;
    c = 1;
  }
}

// Factor order of P as applied to a vector: the rightmost factor first.
__constant__ static const int kApplyOrder[7] = {4, 3, 2, 1, 2, 3, 4};

// v <- (1 + U T_fam) v on one slice held in shared memory.  U points at the
// slice's link table (two complex links per site).  Caller synchronises.
template <class T>
__device__ __forceinline__ void factor_pass(const Geo& g, int fam, T* v, const T* __restrict__ U) {
  const int nb = g.V >> 1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int i, j, c;
    bond_of(g, fam, b, i, j, c);
    T u = __ldg(U + 2 * i + c);
    T vi = v[i], vj = v[j];
    v[i] = cfma(vi, u, vj);
    v[j] = cfmac(vj, u, vi);
  }
}

// v <- (1 + U T_fam)^{-1} v = (1 - U T_fam) v / (1 - |U|^2); used by the force
// sweep to step back through the factors without storing every partial product.
// |U| is the family's tanh factor t_f, so inv = 1/(1 - t_f^2) is one constant per
// family (the caller's), not a division per bond.
template <class T, class R>
__device__ __forceinline__ void factor_pass_inverse(const Geo& g, int fam, T* v, const T* __restrict__ U, R inv) {
  const int nb = g.V >> 1;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int i, j, c;
    bond_of(g, fam, b, i, j, c);
    T u = __ldg(U + 2 * i + c);
    T mu = mk(-u.x, -u.y);
    T vi = v[i], vj = v[j];
    T ni = cfma(vi, mu, vj);
    T nj = cfmac(vj, mu, vi);
    v[i] = cscale(inv, ni);
    v[j] = cscale(inv, nj);
  }
}

// v <- P v: seven factor passes with a block barrier after each.
template <class T>
__device__ __forceinline__ void apply_P(const Geo& g, T* v, const T* __restrict__ U) {
#pragma unroll 1
  for (int k = 0; k < 7; ++k) {
    factor_pass(g, kApplyOrder[6 - k], v, U);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Register-resident sweep.  A thread owns bonds b = threadIdx.x + m*blockDim.x
// (m < MB) of every family; their endpoint pairs (packed i | j << 16, valid
// for V < 32768) are slice-independent and their link factors are loaded once
// per slice, so the seven passes of a sweep touch only shared memory.
// Largest block that leaves enough registers for MB bonds per family (MB = 0:
// links are re-read from global memory in every pass instead).
template <class R, int MB> struct SweepThreads {
  static constexpr int max = MB == 0 ? 1024
                             : sizeof(R) == 8 ? (MB == 1 ? 1024 : 512)
                                              : (MB <= 2 ? 1024 : (MB == 3 ? 768 : 512));
};
__host__ __device__ constexpr int sweep_thread_cap(int bytes_per_real, int mb) {
  return mb == 0 ? 1024 : bytes_per_real == 8 ? (mb == 1 ? 1024 : 512) : (mb <= 2 ? 1024 : (mb == 3 ? 768 : 512));
}

template <int MB>
__device__ __forceinline__ void make_bonds(const Geo& g, int (&ij)[4][MB]) {
  const int nb = g.V >> 1;
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      const int b = threadIdx.x + m * blockDim.x;
      int i = 0, j = 0, c = 0;
      if (b < nb) bond_of(g, f + 1, b, i, j, c);
      ij[f][m] = (b < nb) ? (i | (j << 16)) : -1;
    }
}

template <class T, int MB>
__device__ __forceinline__ void load_links(const int (&ij)[4][MB], const T* __restrict__ U, T (&u)[4][MB]) {
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      T z = {};
      if (ij[f][m] >= 0) z = __ldg(U + 2 * (ij[f][m] & 0xffff) + (f >= 2 ? 1 : 0));
      u[f][m] = z;
    }
}

// v <- P v (factors applied rightmost first: families 4 3 2 1 2 3 4).
template <class T, int MB>
__device__ __forceinline__ void sweep(T* v, const int (&ij)[4][MB], const T (&u)[4][MB]) {
  constexpr int fam[7] = {3, 2, 1, 0, 1, 2, 3};
#pragma unroll
  for (int k = 0; k < 7; ++k) {
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      const int p = ij[fam[k]][m];
      if (p >= 0) {
        const int i = p & 0xffff, j = p >> 16;
        const T vi = v[i], vj = v[j];
        v[i] = cfma(vi, u[fam[k]][m], vj);
        v[j] = cfmac(vj, u[fam[k]][m], vi);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Deterministic reductions: a fixed tree per block and a fixed order over the
// per-block partials, so that every block of a consumer kernel that sums the
// same partials gets bit-identical totals.

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v; the result is valid in thread 0.  `scratch` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = (lane < nw) ? scratch[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// Sum of n partials by one warp in a fixed order; every lane returns the total.
__device__ __forceinline__ double warp_sum_partials(const double* p, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s += p[k];
  s = warp_sum(s);
  return __shfl_sync(0xffffffffu, s, 0);
}

// The same sum with four running sums per lane (elements lane + 32 j, j mod 4):
// the dependent FP64 additions (slow on this part) form chains a quarter as
// long, for a few more registers.  Used where hundreds of partials are summed
// at the start of a kernel whose other registers dominate.
__device__ __forceinline__ double warp_sum_partials4(const double* p, int n) {
  const int lane = threadIdx.x & 31;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = lane;
  for (; k + 96 < n; k += 128) {
    s0 += p[k];
    s1 += p[k + 32];
    s2 += p[k + 64];
    s3 += p[k + 96];
  }
  if (k < n) s0 += p[k];
  if (k + 32 < n) s1 += p[k + 32];
  if (k + 64 < n) s2 += p[k + 64];
  double s = (s0 + s1) + (s2 + s3);
  s = warp_sum(s);
  return __shfl_sync(0xffffffffu, s, 0);
}

// ---------------------------------------------------------------------------
// Device-resident CG state.  Every field is written by exactly one kernel
// launch and read by later launches, or written by block 0 into a slot that
// the other blocks of the same launch do not read.
struct CgState {
  double rr[2];      // <r, r> of the current and previous iteration (index k & 1)
  double bb;         // <phi, phi>
  double tol2bb;     // tol^2 <phi, phi>
  double pq_last;    // last <p, O p>
  double alpha_last; // last step length
  int k;             // iterations completed; read by the direction kernel
  int k2;            // copy of k for the update kernel
  int seg_start;     // first iteration of the current recurrence segment
  int maxit;
  int done;          // CG_* below
  int loops;         // loop bodies executed in this solve
  int loop_cap;      // hard bound on loop bodies (termination guard of the device-side loop)
  int n_rel;         // mixed solver: reliable updates done
  double rr_rel[8];  // mixed solver: true <r,r> at the last eight reliable updates (ring)
  double rr_rec;     // preconditioned CG: last recursive <r,r> (rr[] holds <r, Otilde^{-1} r> there)
};

// CG_* outcome codes: status.h.

// Gates of the kernels that close a loop body: run always, only after the
// recursive residual converged, or whenever the solve is still active.
enum { GATE_ALWAYS = 0, GATE_REC = 1, GATE_ACTIVE = 2, GATE_UNCONVERGED = 3 };

__device__ __forceinline__ bool gate_open(int gate, int done) {
  if (gate == GATE_ALWAYS) return true;
  if (gate == GATE_REC) return done == CG_REC_CONVERGED;
  if (gate == GATE_UNCONVERGED) return done != CG_CONVERGED;
  return done == CG_RUNNING || done == CG_REC_CONVERGED;
}

}  // namespace hqmc
