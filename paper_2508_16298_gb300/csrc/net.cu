// Learned preconditioner: a small 3D periodic convolution network on the
// space-time lattice, gauge covariant and linear in its input, with BF16
// weights and FP32 arithmetic.
//
// Layer l maps C_in complex channels to C_out complex channels:
//   h'(x, c) = sum_{mu=0..6} sum_{c'} W[mu][c][c'] (T_mu h)(x, c')
// with the seven stencil directions mu = 0 (centre), 1/2 = +x/-x, 3/4 = +y/-y,
// 5/6 = +tau/-tau and the parallel transporters
//   (T_{+x} h)(x) = e^{i theta_x(x)} h(x + x^),  (T_{-x} h)(x) = e^{-i theta_x(x - x^)} h(x - x^)
// (y alike), and (T_{+-tau} h)(x) = s h(x +- tau^) with s = -1 across the
// antiperiodic tau boundary.  Real weights commute with the U(1) phases, so the
// net is covariant under theta_ij -> theta_ij + l_i - l_j, h -> e^{i l} h, and
// without activations it is a linear map r -> K(theta) r, which is what a
// (flexible) CG preconditioner must be.  T_mu^dagger = T_{mu-bar} (the
// opposite direction), so the backward pass is the same stencil with
// W'[mu-bar] = W[mu]^T.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hqmc {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// BF16 activations of the tensor-core inference path ("chunk layout"): site i
// holds its 16 complex channels in 64 bytes, four 16-byte chunks; chunk q packs
//   re(2q) re(2q+1) | re(2q+8) re(2q+9) | im(2q) im(2q+1) | im(2q+8) im(2q+9)
// (BF16 pairs, lower channel in the low half).  Chunk q of a site is exactly the
// B fragment of mma.m16n8k16 that lane (g, q) needs for column g (its real part
// in .x .y, its imaginary part in .z .w), and a warp's 16-byte loads of chunks
// 0..3 of 8 consecutive sites cover 512 contiguous bytes.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&p);
}

__device__ __forceinline__ void store_bf16_chunks(uint4* __restrict__ dst, const float2 (&acc)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    dst[q] = make_uint4(pack_bf16x2(acc[2 * q].x, acc[2 * q + 1].x), pack_bf16x2(acc[2 * q + 8].x, acc[2 * q + 9].x),
                        pack_bf16x2(acc[2 * q].y, acc[2 * q + 1].y), pack_bf16x2(acc[2 * q + 8].y, acc[2 * q + 9].y));
}

// Transport factor and neighbour index of direction mu at global site i.
__device__ __forceinline__ void net_neighbour(const Geo& g, const float2* __restrict__ th32, long long i, int mu,
                                              long long& j, float2& ph) {
  const int V = g.V, L = g.L;
  const int tau = (int)(i / V);
  const int s = (int)(i - (long long)tau * V);
  const int x = s % L, y = s / L;
  float sn, cs;
  switch (mu) {
    case 0:
      j = i;
      ph = make_float2(1.f, 0.f);
      break;
    case 1: {
      const int xp = (x + 1 == L) ? 0 : x + 1;
      j = (long long)tau * V + xp + L * y;
      __sincosf(__ldg(th32 + i).x, &sn, &cs);
      ph = make_float2(cs, sn);
    } break;
    case 2: {
      const int xm = (x == 0) ? L - 1 : x - 1;
      j = (long long)tau * V + xm + L * y;
      __sincosf(__ldg(th32 + j).x, &sn, &cs);
      ph = make_float2(cs, -sn);
    } break;
    case 3: {
      const int yp = (y + 1 == L) ? 0 : y + 1;
      j = (long long)tau * V + x + L * yp;
      __sincosf(__ldg(th32 + i).y, &sn, &cs);
      ph = make_float2(cs, sn);
    } break;
    case 4: {
      const int ym = (y == 0) ? L - 1 : y - 1;
      j = (long long)tau * V + x + L * ym;
      __sincosf(__ldg(th32 + j).y, &sn, &cs);
      ph = make_float2(cs, -sn);
    } break;
    case 5: {
      const int tp = (tau + 1 == g.Ntau) ? 0 : tau + 1;
      j = (long long)tp * V + s;
      ph = make_float2(tp == 0 ? -1.f : 1.f, 0.f);
    } break;
    default: {
      const int tm = (tau == 0) ? g.Ntau - 1 : tau - 1;
      j = (long long)tm * V + s;
      ph = make_float2(tau == 0 ? -1.f : 1.f, 0.f);
    } break;
  }
}

// One layer, one thread per site.  Weights [7][COUT][CIN] (BF16) are widened
// to FP32 in shared memory, transposed to [7][CIN][COUT] so that the COUT
// weights of one (mu, c') pair are one or more 16-byte broadcast reads.  Site
// coordinates are computed once per site in 32-bit arithmetic, and a
// neighbour's CIN channels are read as 16-byte pairs.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) net_layer_kernel(Geo g, const float2* __restrict__ th32,
                                                        const __nv_bfloat16* __restrict__ W,
                                                        const float2* __restrict__ in, float2* __restrict__ out,
                                                        long long n) {
  __shared__ __align__(16) float w[7 * COUT * CIN];
  for (int k = threadIdx.x; k < 7 * COUT * CIN; k += blockDim.x) {
    const int mu = k / (COUT * CIN), c = (k / CIN) % COUT, cp = k % CIN;
    w[(mu * CIN + cp) * COUT + c] = __bfloat162float(W[k]);
  }
  __syncthreads();
  const int V = g.V, L = g.L, N = g.Ntau;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)n; i += gridDim.x * blockDim.x) {
    const int tau = i / V, s = i - tau * V, y = s / L, x = s - y * L;
    const int base = tau * V;
    float2 acc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int mu = 0; mu < 7; ++mu) {
      int j = i;
      float2 ph = make_float2(1.f, 0.f);
      float sn, cs;
      if (mu == 1) {
        j = base + y * L + (x + 1 == L ? 0 : x + 1);
        __sincosf(__ldg(th32 + i).x, &sn, &cs);
        ph = make_float2(cs, sn);
      } else if (mu == 2) {
        j = base + y * L + (x == 0 ? L - 1 : x - 1);
        __sincosf(__ldg(th32 + j).x, &sn, &cs);
        ph = make_float2(cs, -sn);
      } else if (mu == 3) {
        j = base + (y + 1 == L ? 0 : y + 1) * L + x;
        __sincosf(__ldg(th32 + i).y, &sn, &cs);
        ph = make_float2(cs, sn);
      } else if (mu == 4) {
        j = base + (y == 0 ? L - 1 : y - 1) * L + x;
        __sincosf(__ldg(th32 + j).y, &sn, &cs);
        ph = make_float2(cs, -sn);
      } else if (mu == 5) {
        const int tp = tau + 1 == N ? 0 : tau + 1;
        j = tp * V + s;
        ph = make_float2(tp == 0 ? -1.f : 1.f, 0.f);
      } else if (mu == 6) {
        const int tm = tau == 0 ? N - 1 : tau - 1;
        j = tm * V + s;
        ph = make_float2(tau == 0 ? -1.f : 1.f, 0.f);
      }
      const float* wm = w + mu * CIN * COUT;
#pragma unroll
      for (int cp2 = 0; cp2 < (CIN + 1) / 2; ++cp2) {
        float2 hv[2];
        if constexpr (CIN % 2 == 0) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(in + (size_t)j * CIN) + cp2);
          hv[0] = make_float2(q.x, q.y);
          hv[1] = make_float2(q.z, q.w);
        } else {
          hv[0] = __ldg(in + (size_t)j * CIN + 2 * cp2);
          hv[1] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cp = 2 * cp2 + h;
          if (cp >= CIN) break;
          const float2 v = cmulf(ph, hv[h]);
          const float* wc = wm + cp * COUT;
          if constexpr (COUT % 4 == 0) {
#pragma unroll
            for (int c4 = 0; c4 < COUT / 4; ++c4) {
              const float4 wv = reinterpret_cast<const float4*>(wc)[c4];
              acc[4 * c4 + 0].x = fmaf(wv.x, v.x, acc[4 * c4 + 0].x);
              acc[4 * c4 + 0].y = fmaf(wv.x, v.y, acc[4 * c4 + 0].y);
              acc[4 * c4 + 1].x = fmaf(wv.y, v.x, acc[4 * c4 + 1].x);
              acc[4 * c4 + 1].y = fmaf(wv.y, v.y, acc[4 * c4 + 1].y);
              acc[4 * c4 + 2].x = fmaf(wv.z, v.x, acc[4 * c4 + 2].x);
              acc[4 * c4 + 2].y = fmaf(wv.z, v.y, acc[4 * c4 + 2].y);
              acc[4 * c4 + 3].x = fmaf(wv.w, v.x, acc[4 * c4 + 3].x);
              acc[4 * c4 + 3].y = fmaf(wv.w, v.y, acc[4 * c4 + 3].y);
            }
          } else {
#pragma unroll
            for (int c = 0; c < COUT; ++c) {
              acc[c].x = fmaf(wc[c], v.x, acc[c].x);
              acc[c].y = fmaf(wc[c], v.y, acc[c].y);
            }
          }
        }
      }
    }
    if constexpr (COUT % 2 == 0) {
      float4* o = reinterpret_cast<float4*>(out + (size_t)i * COUT);
#pragma unroll
      for (int c2 = 0; c2 < COUT / 2; ++c2) o[c2] = make_float4(acc[2 * c2].x, acc[2 * c2].y, acc[2 * c2 + 1].x, acc[2 * c2 + 1].y);
    } else {
#pragma unroll
      for (int c = 0; c < COUT; ++c) out[(size_t)i * COUT + c] = acc[c];
    }
  }
}

// Inference form of the same layer.  The weights arrive as a kernel parameter
// (constant bank), transposed to [7][CIN][COUT]; with the direction and channel
// loops fully unrolled every weight index is a compile-time constant, so each
// FMA reads its weight straight from the constant bank: no shared-memory fill,
// no weight loads and no waits on them.  The arithmetic and its order are those
// of net_layer_kernel.  Activations with several channels are channel-planar
// here (channel c of site i at c * n + i), so every warp load and store is one
// contiguous row of 32 sites; the site-major layout of the training kernels
// would spread a warp's 16-byte loads over 32 lines.  The inference path's
// intermediate buffers are its own; one channel is the same in both layouts.
template <int CIN, int COUT>
struct NetLayerW {
  float w[7][CIN][COUT];
};

// OUT_BF16 (1 -> 16 layer of the tensor-core path): the output is rounded to BF16
// and written in the chunk layout instead of channel-planar FP32.
template <int CIN, int COUT, bool OUT_BF16>
__global__ void __launch_bounds__(256) net_layer_cw_kernel(Geo g, const float2* __restrict__ th32,
                                                           const __grid_constant__ NetLayerW<CIN, COUT> W,
                                                           const float2* __restrict__ in, float2* __restrict__ out,
                                                           int n, const CgState* st) {
  if (st && *(volatile const int*)&st->done != CG_RUNNING) return;  // flexible CG: the solve has stopped
  const int V = g.V, L = g.L, N = g.Ntau;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int tau = i / V, s = i - tau * V, y = s / L, x = s - y * L;
    const int base = tau * V;
    float2 acc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int mu = 0; mu < 7; ++mu) {
      int j = i;
      float2 ph = make_float2(1.f, 0.f);
      float sn, cs;
      if (mu == 1) {
        j = base + y * L + (x + 1 == L ? 0 : x + 1);
        __sincosf(__ldg(th32 + i).x, &sn, &cs);
        ph = make_float2(cs, sn);
      } else if (mu == 2) {
        j = base + y * L + (x == 0 ? L - 1 : x - 1);
        __sincosf(__ldg(th32 + j).x, &sn, &cs);
        ph = make_float2(cs, -sn);
      } else if (mu == 3) {
        j = base + (y + 1 == L ? 0 : y + 1) * L + x;
        __sincosf(__ldg(th32 + i).y, &sn, &cs);
        ph = make_float2(cs, sn);
      } else if (mu == 4) {
        j = base + (y == 0 ? L - 1 : y - 1) * L + x;
        __sincosf(__ldg(th32 + j).y, &sn, &cs);
        ph = make_float2(cs, -sn);
      } else if (mu == 5) {
        const int tp = tau + 1 == N ? 0 : tau + 1;
        j = tp * V + s;
        ph = make_float2(tp == 0 ? -1.f : 1.f, 0.f);
      } else if (mu == 6) {
        const int tm = tau == 0 ? N - 1 : tau - 1;
        j = tm * V + s;
        ph = make_float2(tau == 0 ? -1.f : 1.f, 0.f);
      }
#pragma unroll
      for (int cp = 0; cp < CIN; ++cp) {
        const float2 v = cmulf(ph, __ldg(in + (size_t)cp * n + j));
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
          const float wv = W.w[mu][cp][c];
          acc[c].x = fmaf(wv, v.x, acc[c].x);
          acc[c].y = fmaf(wv, v.y, acc[c].y);
        }
      }
    }
    if constexpr (OUT_BF16 && COUT == 16) {
      store_bf16_chunks(reinterpret_cast<uint4*>(out) + (size_t)i * 4, acc);
    } else {
#pragma unroll
      for (int c = 0; c < COUT; ++c) out[(size_t)c * n + i] = acc[c];
    }
  }
}

// Tensor-core inference layer with 16 input channels (16 or 1 output channels),
// BF16 activations in the chunk layout.  The phase of a transport is the same
// for every channel, so it factors out of the channel contraction:
//   sum_c' W[mu][c][c'] (T_mu h)(x, c') = ph_mu(x) (W[mu] h(x + mu))(c).
// Per group of 8 consecutive sites and direction mu a warp forms the products
// U = W[mu] (16 x 16) H (16 x 8) of the raw neighbour activations, once for the
// real and once for the imaginary parts: mma.sync.m16n8k16 with BF16 operands and
// FP32 accumulation, the weight fragments of all seven directions held in
// registers (rows g, g+8, columns 2q, 2q+1, 2q+8, 2q+9 of W[mu] in lane (g, q)).
// The centre and +-tau terms have real phases (1, or the boundary sign, applied
// exactly to the BF16 operand) and accumulate in place; the +-x and +-y products
// are multiplied by their sites' phases in FP32 and added.  Lane (g, q) loads
// chunk q of site g's neighbour (its B fragment, 16 bytes) and owns output
// channels g and g+8 of sites 2q and 2q+1.  COUT = 16: two lanes swap half of
// their results so that each writes one 16-byte chunk (512 contiguous bytes per
// warp); COUT = 1 (weight rows 1..15 zero): lanes g = 0 write the FP32 output.
struct NetLayerBf16 {
  uint32_t w[7 * 16 * 8];  // [mu][c][c'/2]: BF16 pairs (even c' in the low half); rows c >= COUT zero
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int COUT>
__global__ void __launch_bounds__(256, 4) net_layer_tc_kernel(Geo g, const float2* __restrict__ th32,
                                                           const __grid_constant__ NetLayerBf16 W,
                                                           const uint4* __restrict__ in, void* __restrict__ out,
                                                           int n, const CgState* st) {
  if (st && *(volatile const int*)&st->done != CG_RUNNING) return;  // flexible CG: the solve has stopped
  // weights in shared memory, rows padded to 12 words: the fragment reads of a warp
  // (rows g, columns 2q..) hit 32 distinct banks, and no registers hold them
  __shared__ uint32_t ws[7 * 16 * 12];
  for (int k = threadIdx.x; k < 7 * 16 * 8; k += blockDim.x) ws[(k >> 3) * 12 + (k & 7)] = W.w[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  auto frag = [&](int mu) {
    const uint32_t* r0 = ws + (mu * 16 + gq) * 12 + tq;
    const uint32_t* r8 = r0 + 8 * 12;
    return make_uint4(r0[0], r8[0], r0[4], r8[4]);  // rows g, g+8 x columns 2q.., 2q+8..
  };
  const int V = g.V, L = g.L, N = g.Ntau;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int srcA = (2 * tq) << 2, srcB = (2 * tq + 1) << 2;  // lanes whose column is site 2q / 2q+1
  for (int i0 = warp * 8; i0 < n; i0 += nwarps * 8) {  // n is a multiple of 8 (L even)
    const int i = i0 + gq;  // this lane's column (B operand)
    const int tau = i / V, s = i - tau * V, y = s / L, x = s - y * L;
    const int base = tau * V;
    const int tp = tau + 1 == N ? 0 : tau + 1, tm = tau == 0 ? N - 1 : tau - 1;
    // the seven neighbours (centre, +x, -x, +y, -y, +tau, -tau) and the four link
    // angles, all requested before any product so that their latencies overlap
    int j[7];
    j[0] = i;
    j[1] = base + y * L + (x + 1 == L ? 0 : x + 1);
    j[2] = base + y * L + (x == 0 ? L - 1 : x - 1);
    j[3] = base + (y + 1 == L ? 0 : y + 1) * L + x;
    j[4] = base + (y == 0 ? L - 1 : y - 1) * L + x;
    j[5] = tp * V + s;
    j[6] = tm * V + s;
    uint4 b[7];
#pragma unroll
    for (int mu = 0; mu < 7; ++mu) b[mu] = __ldg(in + (size_t)j[mu] * 4 + tq);
    const float thx_p = __ldg(th32 + i).x, thx_m = __ldg(th32 + j[2]).x;
    const float thy_p = __ldg(th32 + i).y, thy_m = __ldg(th32 + j[4]).y;
    // accumulators: [0] (channel g, site 2q), [1] (g, 2q+1), [2] (g+8, 2q), [3] (g+8, 2q+1)
    float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
    // centre and +-tau: real phases; the antiperiodic sign flips the BF16 sign bits (exact)
    const uint32_t s5 = tp == 0 ? 0x80008000u : 0u, s6 = tau == 0 ? 0x80008000u : 0u;
#pragma unroll
    for (int mu = 0; mu < 7; mu += (mu == 0 ? 5 : 1)) {  // 0, 5, 6
      const uint4 f = frag(mu);
      const uint32_t a4[4] = {f.x, f.y, f.z, f.w};
      const uint32_t sg = mu == 5 ? s5 : mu == 6 ? s6 : 0u;
      mma_bf16_16816(dr, a4, b[mu].x ^ sg, b[mu].y ^ sg);
      mma_bf16_16816(di, a4, b[mu].z ^ sg, b[mu].w ^ sg);
    }
    // +-x, +-y: the products times their sites' phases (ph = e^{+i theta} forward,
    // e^{-i theta(neighbour)} backward), the phases from the lanes owning the sites
#pragma unroll
    for (int mu = 1; mu <= 4; ++mu) {
      float sn, cs;
      __sincosf(mu == 1 ? thx_p : mu == 2 ? thx_m : mu == 3 ? thy_p : thy_m, &sn, &cs);
      const float phx = cs, phy = (mu & 1) ? sn : -sn;
      float ur[4] = {0.f, 0.f, 0.f, 0.f}, ui[4] = {0.f, 0.f, 0.f, 0.f};
      const uint4 f = frag(mu);
      const uint32_t a4[4] = {f.x, f.y, f.z, f.w};
      mma_bf16_16816(ur, a4, b[mu].x, b[mu].y);
      mma_bf16_16816(ui, a4, b[mu].z, b[mu].w);
      const float ax = __shfl_sync(0xffffffffu, phx, srcA), ay = __shfl_sync(0xffffffffu, phy, srcA);
      const float bx = __shfl_sync(0xffffffffu, phx, srcB), by = __shfl_sync(0xffffffffu, phy, srcB);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float px = (e & 1) ? bx : ax, py = (e & 1) ? by : ay;
        dr[e] = fmaf(px, ur[e], fmaf(-py, ui[e], dr[e]));
        di[e] = fmaf(px, ui[e], fmaf(py, ur[e], di[e]));
      }
    }
    if constexpr (COUT == 16) {
      // lane (g, q) keeps site 2q + (g & 1) and swaps the other site's values with lane g ^ 1
      const bool odd = gq & 1;
      const uint32_t keep_r = odd ? pack_bf16x2(dr[1], dr[3]) : pack_bf16x2(dr[0], dr[2]);  // channels g, g+8
      const uint32_t keep_i = odd ? pack_bf16x2(di[1], di[3]) : pack_bf16x2(di[0], di[2]);
      const uint32_t send_r = odd ? pack_bf16x2(dr[0], dr[2]) : pack_bf16x2(dr[1], dr[3]);
      const uint32_t send_i = odd ? pack_bf16x2(di[0], di[2]) : pack_bf16x2(di[1], di[3]);
      const uint32_t recv_r = __shfl_xor_sync(0xffffffffu, send_r, 4);
      const uint32_t recv_i = __shfl_xor_sync(0xffffffffu, send_i, 4);
      // chunk g/2 of the kept site: channels 2c, 2c+1 (lo/hi) from the even and odd lane
      const uint32_t lo_r = odd ? recv_r : keep_r, hi_r = odd ? keep_r : recv_r;
      const uint32_t lo_i = odd ? recv_i : keep_i, hi_i = odd ? keep_i : recv_i;
      const uint4 c = make_uint4((lo_r & 0xffffu) | (hi_r << 16), (lo_r >> 16) | (hi_r & 0xffff0000u),
                                 (lo_i & 0xffffu) | (hi_i << 16), (lo_i >> 16) | (hi_i & 0xffff0000u));
      reinterpret_cast<uint4*>(out)[(size_t)(i0 + 2 * tq + (odd ? 1 : 0)) * 4 + (gq >> 1)] = c;
    } else {
      if (gq == 0)
        *reinterpret_cast<float4*>(reinterpret_cast<float2*>(out) + i0 + 2 * tq) =
            make_float4(dr[0], di[0], dr[1], di[1]);
    }
  }
}

template <int CIN, int COUT, bool OUT_BF16 = false>
static cudaError_t layer_cw(const Geo& g, const float2* th32, const float* w, const float2* in, float2* out,
                            int n, int nb, const CgState* st, cudaStream_t s) {
  NetLayerW<CIN, COUT> W;
  for (int mu = 0; mu < 7; ++mu)
    for (int c = 0; c < COUT; ++c)
      for (int cp = 0; cp < CIN; ++cp) W.w[mu][cp][c] = w[(mu * COUT + c) * CIN + cp];
  net_layer_cw_kernel<CIN, COUT, OUT_BF16><<<nb, 256, 0, s>>>(g, th32, W, in, out, n, st);
  return cudaGetLastError();
}

// Weight gradient: G[mu][c][c'] = sum_x Re(conj(d(x, c)) (T_mu h)(x, c')), a
// reduction over the sites of seven 16 x 16 (at most) products.  Block b owns a
// contiguous chunk of sites and walks it in tiles of WG_TILE sites: the tile's
// d rows are staged in shared memory once, then for each direction mu the
// transported neighbour rows (T_mu h) are staged and every thread adds the
// tile's contribution to the weight entry (c, c') it owns (the threads of a warp
// read one or two d rows, broadcast, and 16 consecutive h entries: no bank
// conflicts).  Per tile the FP32 sums go into FP64 accumulators, and each
// block writes one partial per entry: partials[b][mu][c][c'].
constexpr int WG_TILE = 64;

template <int CIN, int COUT>
__global__ void __launch_bounds__(256) net_wgrad_kernel(Geo g, const float2* __restrict__ th32,
                                                        const float2* __restrict__ d, const float2* __restrict__ h,
                                                        double* __restrict__ partials, int n, int chunk) {
  constexpr int E = CIN * COUT;  // weight entries per direction (<= 256)
  __shared__ float2 Ds[WG_TILE * COUT];
  __shared__ float2 Hs[WG_TILE * CIN];
  const int t = threadIdx.x;
  const int c = t / CIN, cp = t - (t / CIN) * CIN;  // the entry this thread owns (t < E)
  double accd[7];
#pragma unroll
  for (int mu = 0; mu < 7; ++mu) accd[mu] = 0.0;
  const int i0 = blockIdx.x * chunk;
  const int i1 = min(n, i0 + chunk);
  const int V = g.V, L = g.L, N = g.Ntau;
  for (int tb = i0; tb < i1; tb += WG_TILE) {
    const int cnt = min(WG_TILE, i1 - tb);
    for (int k = t; k < WG_TILE * COUT; k += blockDim.x) {
      const int sl = k / COUT;
      Ds[k] = sl < cnt ? d[(size_t)tb * COUT + k] : make_float2(0.f, 0.f);
    }
#pragma unroll 1
    for (int mu = 0; mu < 7; ++mu) {
      for (int k = t; k < WG_TILE * CIN; k += blockDim.x) {
        const int sl = k / CIN, ch = k - sl * CIN;
        float2 v = make_float2(0.f, 0.f);
        if (sl < cnt) {
          const int i = tb + sl;
          const int tau = i / V, s = i - tau * V, y = s / L, x = s - y * L, base = tau * V;
          int j = i;
          float2 ph = make_float2(1.f, 0.f);
          float sn, cs;
          if (mu == 1) {
            j = base + y * L + (x + 1 == L ? 0 : x + 1);
            __sincosf(__ldg(th32 + i).x, &sn, &cs);
            ph = make_float2(cs, sn);
          } else if (mu == 2) {
            j = base + y * L + (x == 0 ? L - 1 : x - 1);
            __sincosf(__ldg(th32 + j).x, &sn, &cs);
            ph = make_float2(cs, -sn);
          } else if (mu == 3) {
            j = base + (y + 1 == L ? 0 : y + 1) * L + x;
            __sincosf(__ldg(th32 + i).y, &sn, &cs);
            ph = make_float2(cs, sn);
          } else if (mu == 4) {
            j = base + (y == 0 ? L - 1 : y - 1) * L + x;
            __sincosf(__ldg(th32 + j).y, &sn, &cs);
            ph = make_float2(cs, -sn);
          } else if (mu == 5) {
            const int tp = tau + 1 == N ? 0 : tau + 1;
            j = tp * V + s;
            ph = make_float2(tp == 0 ? -1.f : 1.f, 0.f);
          } else if (mu == 6) {
            const int tm = tau == 0 ? N - 1 : tau - 1;
            j = tm * V + s;
            ph = make_float2(tau == 0 ? -1.f : 1.f, 0.f);
          }
          v = cmulf(ph, __ldg(h + (size_t)j * CIN + ch));
        }
        Hs[k] = v;
      }
      __syncthreads();  // Ds (first direction) and Hs complete
      if (t < E) {
        float acc = 0.f;
#pragma unroll 8
        for (int sl = 0; sl < WG_TILE; ++sl) {
          const float2 dd = Ds[sl * COUT + c], hv = Hs[sl * CIN + cp];
          acc = fmaf(dd.x, hv.x, fmaf(dd.y, hv.y, acc));
        }
        accd[mu] += (double)acc;
      }
      __syncthreads();  // Hs (and, after the last direction, Ds) may be overwritten
    }
  }
  if (t < E) {
#pragma unroll
    for (int mu = 0; mu < 7; ++mu) partials[(size_t)blockIdx.x * (7 * E) + mu * E + t] = accd[mu];
  }
}

// loss = ||h - x||^2 / ||x||^2 (partials) and d = 2 (h - x) / ||x||^2; *xx = ||x||^2
__global__ void net_loss_kernel(const float2* __restrict__ h, const double2* __restrict__ x, const double* xx,
                                float2* __restrict__ d, double* __restrict__ part, long long n) {
  __shared__ double red[32];
  const double inv_xx = 1.0 / *xx;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ex = (double)h[i].x - x[i].x, ey = (double)h[i].y - x[i].y;
    acc += ex * ex + ey * ey;
    d[i] = make_float2((float)(2.0 * ex * inv_xx), (float)(2.0 * ey * inv_xx));
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t * inv_xx;
}

// Adam on the FP32 master weights; writes the BF16 copy used by the layers.
__global__ void net_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                const double* __restrict__ partials, int nchunks, int nw, __nv_bfloat16* __restrict__ wb,
                                float lr, float b1, float b2, float c1, float c2, float eps, float scale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nw) return;
  double gs = 0.0;
  for (int k = 0; k < nchunks; ++k) gs += partials[(long long)k * nw + e];
  const float gr = (float)gs * scale;
  const float mm = b1 * m[e] + (1.f - b1) * gr;
  const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
  m[e] = mm;
  v[e] = vv;
  const float wn = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  w[e] = wn;
  wb[e] = __float2bfloat16(wn);
}

// W'[mu-bar][c'][c] = W[mu][c][c'] for the backward stencil.
__global__ void net_adjoint_weights_kernel(const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ Wt,
                                           int cin, int cout) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 7 * cin * cout) return;
  const int mu = e / (cout * cin);
  const int c = (e / cin) % cout;
  const int cp = e % cin;
  const int mubar = mu == 0 ? 0 : (mu & 1) ? mu + 1 : mu - 1;
  Wt[(mubar * cin + cp) * cout + c] = W[e];
}

// complex double <-> complex float with a scale
__global__ void net_to_float_kernel(const double2* __restrict__ a, float2* __restrict__ b, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)(a[i].x * s), (float)(a[i].y * s));
}
__global__ void net_to_double_kernel(const float2* __restrict__ a, double2* __restrict__ b, double s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = make_double2((double)a[i].x * s, (double)a[i].y * s);
}

static inline int blocks_for(long long n, int t) {
  long long b = (n + t - 1) / t;
  return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

cudaError_t launch_net_layer(const Geo& g, const float2* th32, const void* W, int cin, int cout, const float2* in,
                             float2* out, cudaStream_t s) {
  const long long n = (long long)g.V * g.Ntau;
  const __nv_bfloat16* w = (const __nv_bfloat16*)W;
  const int nb = blocks_for(n, 256);
  if (cin == 1 && cout == 16) net_layer_kernel<1, 16><<<nb, 256, 0, s>>>(g, th32, w, in, out, n);
  else if (cin == 16 && cout == 16) net_layer_kernel<16, 16><<<nb, 256, 0, s>>>(g, th32, w, in, out, n);
  else if (cin == 16 && cout == 1) net_layer_kernel<16, 1><<<nb, 256, 0, s>>>(g, th32, w, in, out, n);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_net_layer_host_weights(const Geo& g, const float2* th32, const float* w, int cin, int cout,
                                         const float2* in, float2* out, const CgState* st, cudaStream_t s,
                                         bool tensor_cores) {
  const int n = g.V * g.Ntau;
  const int nb = blocks_for(n, 256);
  if (tensor_cores) {  // 16-channel activations in BF16 chunks: in (16 -> *) / out (* -> 16)
    if (n % 8 != 0) return cudaErrorInvalidValue;
    if (cin == 1 && cout == 16) return layer_cw<1, 16, true>(g, th32, w, in, out, n, nb, st, s);
    if (cin != 16 || (cout != 16 && cout != 1)) return cudaErrorInvalidValue;
    NetLayerBf16 W{};  // the weights are BF16 values: the conversion is exact; rows >= cout stay zero
    for (int mu = 0; mu < 7; ++mu)
      for (int c = 0; c < cout; ++c)
        for (int p = 0; p < 8; ++p) {
          const float* wr = w + ((size_t)mu * cout + c) * 16;
          const __nv_bfloat162 v = __floats2bfloat162_rn(wr[2 * p], wr[2 * p + 1]);
          W.w[(mu * 16 + c) * 8 + p] = *reinterpret_cast<const uint32_t*>(&v);
        }
    const int groups = n / 8;  // one warp per group of 8 sites, 8 warps per block
    const uint4* in4 = reinterpret_cast<const uint4*>(in);
    if (cout == 16) net_layer_tc_kernel<16><<<blocks_for(groups, 8), 256, 0, s>>>(g, th32, W, in4, out, n, st);
    else net_layer_tc_kernel<1><<<blocks_for(groups, 8), 256, 0, s>>>(g, th32, W, in4, out, n, st);
    return cudaGetLastError();
  }
  if (cin == 1 && cout == 16) return layer_cw<1, 16>(g, th32, w, in, out, n, nb, st, s);
  if (cin == 16 && cout == 16) return layer_cw<16, 16>(g, th32, w, in, out, n, nb, st, s);
  if (cin == 16 && cout == 1) return layer_cw<16, 1>(g, th32, w, in, out, n, nb, st, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_net_wgrad(const Geo& g, const float2* th32, int cin, int cout, const float2* d, const float2* h,
                             double* partials, int nchunks, cudaStream_t s) {
  const int n = g.V * g.Ntau;
  const int chunk = (n + nchunks - 1) / nchunks;
  if (cin == 1 && cout == 16) net_wgrad_kernel<1, 16><<<nchunks, 256, 0, s>>>(g, th32, d, h, partials, n, chunk);
  else if (cin == 16 && cout == 16) net_wgrad_kernel<16, 16><<<nchunks, 256, 0, s>>>(g, th32, d, h, partials, n, chunk);
  else if (cin == 16 && cout == 1) net_wgrad_kernel<16, 1><<<nchunks, 256, 0, s>>>(g, th32, d, h, partials, n, chunk);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_net_loss(const float2* h, const double2* x, const double* xx, float2* d, double* part, int nblocks,
                            long long n, cudaStream_t s) {
  net_loss_kernel<<<nblocks, 256, 0, s>>>(h, x, xx, d, part, n);
  return cudaGetLastError();
}

cudaError_t launch_net_adam(float* w, float* m, float* v, const double* partials, int nchunks, int nw, void* wb,
                            float lr, float b1, float b2, float c1, float c2, float eps, float scale, cudaStream_t s) {
  net_adam_kernel<<<(nw + 255) / 256, 256, 0, s>>>(w, m, v, partials, nchunks, nw, (__nv_bfloat16*)wb, lr, b1, b2, c1,
                                                  c2, eps, scale);
  return cudaGetLastError();
}

cudaError_t launch_net_adjoint_weights(const void* W, void* Wt, int cin, int cout, cudaStream_t s) {
  const int ne = 7 * cin * cout;
  net_adjoint_weights_kernel<<<(ne + 255) / 256, 256, 0, s>>>((const __nv_bfloat16*)W, (__nv_bfloat16*)Wt, cin, cout);
  return cudaGetLastError();
}

cudaError_t launch_net_convert(const void* in, void* out, int to_float, double scale, long long n, cudaStream_t s) {
  if (to_float)
    net_to_float_kernel<<<blocks_for(n, 256), 256, 0, s>>>((const double2*)in, (float2*)out, scale, n);
  else
    net_to_double_kernel<<<blocks_for(n, 256), 256, 0, s>>>((const float2*)in, (double2*)out, scale, n);
  return cudaGetLastError();
}

}  // namespace hqmc
