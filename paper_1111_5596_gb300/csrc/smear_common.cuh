// Device helpers shared by the smearing kernels: element loads/stores for
// FP32 and BF16 storage, complex multiply-accumulate, and link loads with
// reconstruct-12 decompression.
#pragma once

#include "qdpg_internal.h"

namespace qdpg {
namespace smear_dev {

enum LinkMode { L_F32 = 0, L_F32_R12 = 1, L_BF16 = 2, L_BF16_R12 = 3 };

__device__ __forceinline__ float2 ld2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat162* p) {
  __nv_bfloat162 v = *p;
  return __bfloat1622float2(v);
}
__device__ __forceinline__ void st2(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st2(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

// a * b with a fixed rounding sequence (no compiler-chosen contraction), so
// every kernel reconstructs reconstruct-12 links bit-identically.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
// Load link U_mu at element offset `off` (= t*ncl*V3 + s3) into m[9].
template <int LMODE>
__device__ __forceinline__ void load_link(const void* U, long long off, int V3, int mu, float2 m[9]) {
  if (LMODE == L_F32 || LMODE == L_BF16) {
    constexpr int ncl = 36;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      if (LMODE == L_F32)
        m[e] = ld2(static_cast<const float2*>(U) + off + (long long)(mu * 9 + e) * V3);
      else
        m[e] = ld2(static_cast<const __nv_bfloat162*>(U) + off + (long long)(mu * 9 + e) * V3);
    }
    (void)ncl;
  } else {
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      if (LMODE == L_F32_R12)
        m[e] = ld2(static_cast<const float2*>(U) + off + (long long)(mu * 6 + e) * V3);
      else
        m[e] = ld2(static_cast<const __nv_bfloat162*>(U) + off + (long long)(mu * 6 + e) * V3);
    }
    // row2[b] = conj(row0[b1] row1[b2] - row0[b2] row1[b1]), (b, b1, b2) cyclic
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
      float2 c = cmul(m[b1], m[3 + b2]);
      float2 d = cmul(m[b2], m[3 + b1]);
      m[6 + b] = make_float2(c.x - d.x, -(c.y - d.y));
    }
  }
}

// ---- packed FP32 pair arithmetic (fma.rn.f32x2, sm_100 and later) ----------
//
// A complex number lives in one 64-bit register pair (re, im).  With
// L = (Lr, Li) and psi = (pr, pi):
//   L (.) psi        = (Lr pr, Li pi)      -> re part  Lr pr - Li pi
//   L (.) swap(psi)  = (Lr pi, Li pr)      -> im part  Lr pi + Li pr
// so a complex multiply-accumulate is two packed FMAs into two pair
// accumulators P and Q, and the product's (re, im) = (P.x - P.y, Q.x + Q.y).
// Backward links enter conjugated, conj(U) = (Ur, -Ui), which turns the
// U^dag hop into the same two packed FMAs with the same final combination.

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float x, float y) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 unpack2(u64 r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ u64 pack2(float2 v) { return pack2(v.x, v.y); }
__device__ __forceinline__ u64 swap2(u64 r) {
  const float2 v = unpack2(r);
  return pack2(v.y, v.x);
}
// d = a (.) b + c, two lanes, round to nearest
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Links of one site as pairs, multiplied by kappa once per site:
// f[i][a*3+q] = kappa U_i(x)[a][q] and b[i][a*3+q] = kappa conj(U_i(x - i)[q][a])
// (the backward hop's matrix).
struct SiteLinks {
  u64 f[3][9];
  u64 b[3][9];
};

__device__ __forceinline__ void make_site_links(const float2 Uf[3][9], const float2 Ub[3][9], float kappa,
                                                SiteLinks& L) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        L.f[i][a * 3 + q] = pack2(kappa * Uf[i][a * 3 + q].x, kappa * Uf[i][a * 3 + q].y);
        L.b[i][a * 3 + q] = pack2(kappa * Ub[i][q * 3 + a].x, -(kappa * Ub[i][q * 3 + a].y));
      }
}

// Products of one half of the hop (M = the forward or the conjugated
// backward links, n[i][q] the matching neighbour values) accumulated into
// the pairs P[a] (real part P.x - P.y) and Q[a] (imaginary part Q.x + Q.y).
__device__ __forceinline__ void hop_accumulate(const u64 M[3][9], const u64 n[3][3], u64 P[3], u64 Q[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u64 sw[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) sw[q] = swap2(n[i][q]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        P[a] = fma2(M[i][a * 3 + q], n[i][q], P[a]);
        Q[a] = fma2(M[i][a * 3 + q], sw[q], Q[a]);
      }
  }
}

// One colour vector of one site: out[a] = c[a] + sum_i
//   [ kappa U_i(x) psi(x+i) + (kappa U_i(x-i))^dag psi(x-i) ][a]
// from neighbour values nf[i][q] = psi(x+i)[q], nb[i][q] = psi(x-i)[q] and
// kappa-scaled links.  The centre value seeds the accumulators (P = (c.x, 0),
// Q = (0, c.y)); forward products go in first, then backward ones.  Every
// kernel uses this sequence, so their results agree bit for bit.
__device__ __forceinline__ void hop_vector(const SiteLinks& L, const u64 nf[3][3], const u64 nb[3][3],
                                           const float2 c[3], float2 out[3]) {
  u64 P[3], Q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P[a] = pack2(c[a].x, 0.f);
    Q[a] = pack2(0.f, c[a].y);
  }
  hop_accumulate(L.f, nf, P, Q);
  hop_accumulate(L.b, nb, P, Q);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 p = unpack2(P[a]), qv = unpack2(Q[a]);
    out[a] = make_float2(p.x - p.y, qv.x + qv.y);
  }
}

}  // namespace smear_dev
}  // namespace qdpg
