// Register strips of the fused M^dagger M kernels (mdagm_block.cu, mdagm_walk.cu).
//
// A thread keeps a 2 x H strip of a slice (H = 2*NBY rows) in registers and
// applies whole checkerboard factors of Eq. (eq24) there:
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
// right neighbours: three shared-memory exchanges and three barriers per sweep.
#pragma once

#include "kernels.h"

namespace hqmc {

// Link factors of one strip (tanh of the factor angle folded in).
template <class T, int NBY>
struct StripLinks {
  T u4[NBY][2];   // family 4: y-bonds with tail on D rows 0, 2, ... (odd y)
  T u3[NBY][2];   // family 3: y-bonds with tail on C rows 0, 2, ... (even y)
  T u2[2 * NBY];  // family 2: x-bond x0 -> x1 on every C row
  T u1l[2 * NBY]; // family 1: x-bond 2i -> x0 (this strip holds its head)
  T u1r[2 * NBY]; // family 1: x-bond x1 -> 2i+3 (this strip holds its tail)
};

// Per-thread geometry of the strip.  Thread t owns column pair i = t mod L/2
// of the strip row jj = t div (L/2).
//
// Exchange buffers are planar: the x0 columns (odd) of all strips form plane A,
// the x1 columns (even) plane B, each indexed y*(L/2) + i.  Neighbouring
// threads of a strip row then touch consecutive words (no bank conflicts),
// where the natural layout would put their 8-byte entries 16 bytes apart.
struct StripGeo {
  int L, Lh;
  int x0, x1;  // owned columns 2i+1, (2i+2) mod L
  int xl, xr;  // columns 2i and (2i+3) mod L of the family-1 partners
  int i, il, ir;  // own column pair, and those of the left / right neighbours (mod L/2)
  int hv;      // plane B offset in the exchange buffers: L*L/2
  int base;    // first C row (2*jj*NBY)
  int ytop;    // last D row (base + H) mod L
};

template <int NBY>
__device__ __forceinline__ StripGeo strip_geo(int L) {
  const int Lh = L >> 1;
  const int i = threadIdx.x % Lh, jj = threadIdx.x / Lh;
  StripGeo s;
  s.L = L;
  s.Lh = Lh;
  s.x0 = 2 * i + 1;
  s.x1 = (2 * i + 2 == L) ? 0 : 2 * i + 2;
  s.xl = 2 * i;
  s.xr = (2 * i + 3 >= L) ? 2 * i + 3 - L : 2 * i + 3;
  s.i = i;
  s.il = (i == 0) ? Lh - 1 : i - 1;
  s.ir = (i == Lh - 1) ? 0 : i + 1;
  s.hv = L * Lh;
  s.base = 2 * jj * NBY;
  const int top = s.base + 2 * NBY;
  s.ytop = (top >= L) ? top - L : top;
  return s;
}

// Planar exchange-buffer slots (see StripGeo): own x0 / x1 entries of row y,
// and the left partner's x1 (column 2i) / right partner's x0 (column 2i+3).
__device__ __forceinline__ int ex_x0(const StripGeo& s, int y) { return y * s.Lh + s.i; }
__device__ __forceinline__ int ex_x1(const StripGeo& s, int y) { return s.hv + y * s.Lh + s.i; }
__device__ __forceinline__ int ex_xl(const StripGeo& s, int y) { return s.hv + y * s.Lh + s.il; }
__device__ __forceinline__ int ex_xr(const StripGeo& s, int y) { return y * s.Lh + s.ir; }

__device__ __forceinline__ int drow(const StripGeo& s, int r, int H) { return r < H - 1 ? s.base + 1 + r : s.ytop; }

template <class T>
__device__ __forceinline__ T link_from_theta(float th, float t) {
  float sn, cs;
  __sincosf(th, &sn, &cs);
  return mk(t * cs, t * sn);
}

// t e^{i theta} for theta in [-pi, pi] on the FMA pipe, from the Taylor series of
// sin and cos at the half angle h = theta/2 (|h| <= pi/2; the omitted terms are
// below (pi/2)^13/13! = 6e-8 and (pi/2)^14/14! = 7e-9), then
// cos theta = (cos h - sin h)(cos h + sin h), sin theta = 2 sin h cos h.
// Links formed this way share the work of a step with __sincosf, whose MUFU
// pipe otherwise bounds the link phase.
__device__ __forceinline__ float2 link_from_theta_poly(float th, float t) {
  const float h = 0.5f * th, h2 = h * h;
  float sp = fmaf(h2, -1.f / 39916800.f, 1.f / 362880.f);
  sp = fmaf(h2, sp, -1.f / 5040.f);
  sp = fmaf(h2, sp, 1.f / 120.f);
  sp = fmaf(h2, sp, -1.f / 6.f);
  sp = fmaf(h2, sp, 1.f);
  const float sh = h * sp;
  float cp = fmaf(h2, 1.f / 479001600.f, -1.f / 3628800.f);
  cp = fmaf(h2, cp, 1.f / 40320.f);
  cp = fmaf(h2, cp, -1.f / 720.f);
  cp = fmaf(h2, cp, 1.f / 24.f);
  cp = fmaf(h2, cp, -0.5f);
  const float ch = fmaf(h2, cp, 1.f);
  return make_float2(t * ((ch - sh) * (ch + sh)), (2.f * t) * (sh * ch));
}

template <bool SMEM>
__device__ __forceinline__ float2 th_at(const float2* th, int i) {
  if constexpr (SMEM) return th[i];
  else return __ldg(th + i);
}

// FP32 links from a theta slice staged in shared memory.  Every link of the
// strip lies on a C row (base .. base+H-1) at column 2i, 2i+1 or (2i+2) mod L,
// so two aligned 16-byte reads per row, (2i, 2i+1) and (x1, x1+1), fetch them.
template <int NBY>
__device__ __forceinline__ void load_strip_links_smem(const StripGeo& s, const float2* __restrict__ th, float t1,
                                                      float t2, StripLinks<float2, NBY>& k) {
  constexpr int H = 2 * NBY;
  const int L = s.L;
  const float4* th4 = reinterpret_cast<const float4*>(th);
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int y = s.base + r;
    const float4 a = th4[(y * L + s.xl) >> 1];  // theta(2i), theta(x0)
    const float4 b = th4[(y * L + s.x1) >> 1];  // theta(x1), theta(x1 + 1)
    k.u2[r] = link_from_theta<float2>(a.z, t2);
    k.u1l[r] = link_from_theta_poly(a.x, t1);  // family 1 on the FMA pipe, the rest on MUFU
    k.u1r[r] = link_from_theta_poly(b.x, t1);
    if (r & 1) {  // D row base + r = drow(r - 1): family 4, tails on odd y
      k.u4[r >> 1][0] = link_from_theta<float2>(a.w, t2);
      k.u4[r >> 1][1] = link_from_theta<float2>(b.y, t2);
    } else {      // C row base + r: family 3, tails on even y
      k.u3[r >> 1][0] = link_from_theta<float2>(a.w, t2);
      k.u3[r >> 1][1] = link_from_theta<float2>(b.y, t2);
    }
  }
}

// FP32: from theta (float2 (theta_x, theta_y) per site, wrapped to [-pi, pi)),
// read from global memory or from a slice staged in shared memory.
template <int NBY, bool SMEM = false>
__device__ __forceinline__ void load_strip_links(const StripGeo& s, const float2* __restrict__ th, float t1, float t2,
                                                 StripLinks<float2, NBY>& k) {
  constexpr int H = 2 * NBY;
  const int L = s.L;
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    const int yd = drow(s, 2 * b, H), yc = s.base + 2 * b;
    k.u4[b][0] = link_from_theta<float2>(th_at<SMEM>(th, yd * L + s.x0).y, t2);
    k.u4[b][1] = link_from_theta<float2>(th_at<SMEM>(th, yd * L + s.x1).y, t2);
    k.u3[b][0] = link_from_theta<float2>(th_at<SMEM>(th, yc * L + s.x0).y, t2);
    k.u3[b][1] = link_from_theta<float2>(th_at<SMEM>(th, yc * L + s.x1).y, t2);
  }
#pragma unroll
  for (int r = 0; r < H; ++r) {
    const int yc = s.base + r;
    k.u2[r] = link_from_theta<float2>(th_at<SMEM>(th, yc * L + s.x0).x, t2);
    k.u1l[r] = link_from_theta<float2>(th_at<SMEM>(th, yc * L + s.xl).x, t1);
    k.u1r[r] = link_from_theta<float2>(th_at<SMEM>(th, yc * L + s.x1).x, t1);
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
    E[ex_x0(s, s.ytop)] = v[H - 1][0];
    E[ex_x1(s, s.ytop)] = v[H - 1][1];
    __syncthreads();
#pragma unroll
    for (int r = H - 1; r > 0; --r) {
      v[r][0] = v[r - 1][0];
      v[r][1] = v[r - 1][1];
    }
    v[0][0] = E[ex_x0(s, s.base)];
    v[0][1] = E[ex_x1(s, s.base)];
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
      E[ex_x0(s, s.base + r)] = v[r][0];
      E[ex_x1(s, s.base + r)] = v[r][1];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const T pl = E[ex_xl(s, s.base + r)];
      const T pr = E[ex_xr(s, s.base + r)];
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
    E[ex_x0(s, s.base)] = v[0][0];
    E[ex_x1(s, s.base)] = v[0][1];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < H - 1; ++r) {
      v[r][0] = v[r + 1][0];
      v[r][1] = v[r + 1][1];
    }
    v[H - 1][0] = E[ex_x0(s, s.ytop)];
    v[H - 1][1] = E[ex_x1(s, s.ytop)];
  }
  // F4 in D
#pragma unroll
  for (int b = 0; b < NBY; ++b) {
    bond2(v[2 * b][0], v[2 * b + 1][0], k.u4[b][0]);
    bond2(v[2 * b][1], v[2 * b + 1][1], k.u4[b][1]);
  }
}

}  // namespace hqmc
