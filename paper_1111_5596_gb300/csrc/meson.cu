// Meson two-point functions: the mesonic part of the paper's hadron-spectrum
// stage (Sec. 5, Fig. 4 "HAD").
//
//   C_j(t, p) = sum_{x in t} exp(-i p.(x - x0))
//               tr[ Gamma_snk S1(x) Gamma_src^dag g5 S2(x)^dag g5 ]
//
// Every DeGrand-Rossi basis element is a signed permutation whose
// permutation is an XOR with a 2-bit mask (row r has its one nonzero in
// column r ^ m).  Writing A = Gamma_snk (mask ma) and B = Gamma_src^dag
// (mask mb), the trace collapses to
//
//   c_j(x) = sum_{alpha, beta} w_j(alpha, beta) Q_{ma,mb}(alpha, beta)
//   Q_{ma,mb}(alpha, beta) = sum_{d, b} S1[alpha d][beta b] conj(S2[(alpha^ma) d][(beta^mb) b])
//   w_j(alpha, beta) = A[alpha^ma][alpha] B[beta][beta^mb] g5[beta^mb] g5[alpha^ma]
//
// so channels that share a mask pair share the 16 colour contractions Q and
// differ only in the unit-modulus weights w.  The sixteen mesons
// Gamma_snk = Gamma_src = Gamma(n) use only four mask pairs: 64 colour
// contractions (576 complex MACs) per site for all sixteen.
//
// A thread owns one site.  Site values are FP32; the timeslice/momentum sums
// are FP64: warp shuffle, then shared memory across warps, then one FP64
// atomic per block and value.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gamma_host.h"
#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"
#include "tmap.h"

namespace qdpg {

namespace {

using namespace gamma_host;

constexpr int kMesonThreads = 128;
constexpr int kMaxPassCh = 16;
constexpr int kMaxMom = 64;

struct MesonPass {
  int nq;                        // distinct (ma, mb) pairs, 1..4
  int ma[4], mb[4];
  int nch;                       // channels, 1..16
  int q_of[kMaxPassCh];          // pair index of each channel
  int out_row[kMaxPassCh];       // channel index in the output
  float2 w[kMaxPassCh][16];      // weight of Q_q[alpha*4 + beta]
  int jlo[4], jhi[4];            // channels of pair q: jlo[q] <= j < jhi[q] (grouped by pair)
  int mlo[4], mhi[4];            // channels whose two masks are both m (orbit kernel): mlo[m] <= j < mhi[m]
  unsigned long long wre[kMaxPassCh][16];  // (w.x, w.x) and (w.y, w.y) as packed FP32 pairs
  unsigned long long wim[kMaxPassCh][16];
};

struct Moms {
  int n;
  int origin[3];                 // origin along the three non-decay directions
  int k[kMaxMom][3];             // integer momenta
  bool zero_only;                // single momentum (0,0,0): no phases
};

__device__ __forceinline__ float2 ld2(const float2* p) { return __ldg(p); }
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
// d = a (.) b + c, two FP32 lanes, round to nearest
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 lds_pair_st(const float2* p) { return *reinterpret_cast<const u64*>(p); }
__device__ __forceinline__ u64 lds_pair_st(const __nv_bfloat162* p) {
  const float2 v = __bfloat1622float2(*p);
  return pack2(v.x, v.y);
}
__device__ __forceinline__ u64 lds_pair_st(const __half2* p) {
  const float2 v = __half22float2(*p);
  return pack2(v.x, v.y);
}
__device__ __forceinline__ float2 lds_elem(const float2* p) { return *p; }
__device__ __forceinline__ float2 lds_elem(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ float2 ld2(const __nv_bfloat162* p) {
  __nv_bfloat162 v = *p;
  return __bfloat1622float2(v);
}

// Element loaders of one site's propagator: component-major (F32, BF16)
// and site-major float16 (qdpg.h); comp folds to a constant when unrolled.
template <typename PsiT>
struct SoASite {
  const PsiT* p;
  int V3;
  __device__ SoASite(const PsiT* S, int t, int s3, int V3_) : p(S + (long long)t * 144 * V3_ + s3), V3(V3_) {}
  __device__ __forceinline__ float2 operator()(int comp) const { return ld2(p + (long long)comp * V3); }
};
// Float16 propagators are site-major, so a thread's own site is 576 strided
// bytes: the block's sites are first staged in shared memory with coalesced
// 16-byte loads, kF16Stride words per site (odd: conflict-free reads).
constexpr int kF16Stride = 145;
// Loaders of one site's float16 propagator: staged in shared memory (the
// site's 145-word slot, vector groups 48 words apart) or in global memory.
__device__ __forceinline__ float2 f16_word(uint32_t w) { return __half22float2(*reinterpret_cast<const __half2*>(&w)); }
__device__ __forceinline__ int f16_site_word(int comp) {  // vector group * 48 + word within the group
  const int sc = comp / 12, sp = comp % 12, sv = sc / 3, c = sc % 3;
  const int v = sv * 12 + sp;
  return (v >> 4) * 48 + (v & 15) * 3 + c;
}
struct F16Staged {
  const uint32_t* p;
  __device__ F16Staged(const uint32_t* slot) : p(slot) {}
  __device__ __forceinline__ float2 operator()(int comp) const { return f16_word(p[f16_site_word(comp)]); }
};
struct F16Global {
  const uint32_t* p;
  long long gs;  // words between vector groups
  __device__ F16Global(const uint32_t* S, int t, int s3, int V3)
      : p(S + ((long long)t * 3 * V3 + s3) * 48), gs((long long)V3 * 48) {}
  __device__ __forceinline__ float2 operator()(int comp) const {
    const int w = f16_site_word(comp);
    return f16_word(__ldg(p + (w / 48) * gs + w % 48));
  }
};

// Stage words of sites s0 .. s0+127 (all three vector groups) of timeslice t.
__device__ __forceinline__ void stage_f16(uint32_t* dst, const __half2* S, int t, int s0, int V3) {
  const int nsite = min(kMesonThreads, V3 - s0);
#pragma unroll
  for (int vg = 0; vg < 3; ++vg) {
    const uint4* src = reinterpret_cast<const uint4*>(S + ((long long)(t * 3 + vg) * V3 + s0) * 48);
    for (int q = threadIdx.x; q < nsite * 12; q += kMesonThreads) {
      const uint4 v = src[q];
      const int i = q / 12, w = (q % 12) * 4;
      uint32_t* d = dst + i * kF16Stride + vg * 48 + w;
      d[0] = v.x;
      d[1] = v.y;
      d[2] = v.z;
      d[3] = v.w;
    }
  }
}

// s + e = a + b exactly (Knuth's TwoSum, six FP32 additions; the compiler
// must not reassociate them, which CUDA does not do without fast-math).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  const float x = __fadd_rn(a, b);
  const float bv = __fsub_rn(x, a);
  const float av = __fsub_rn(x, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  s = x;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// SITES: write each channel's site value c_j(x) to sites[row(j)][t][x]
// (complex FP32) instead of reducing it.
template <int NQ, typename PsiT, bool SITES, bool SAME>
__global__ void __launch_bounds__(kMesonThreads) meson_kernel(const PsiT* __restrict__ S1, const PsiT* __restrict__ S2,
                                                              Geom g, MesonPass P, Moms M, double* __restrict__ out,
                                                              float2* __restrict__ sites, const ScaleRecord* rec1,
                                                              const ScaleRecord* rec2, int site_scale) {
  extern __shared__ double2 red[];  // [warp][nch * n_mom]
  const int s3 = blockIdx.x * kMesonThreads + threadIdx.x;
  const int t = blockIdx.y;
  const bool live = s3 < g.V3;
  const int V3 = g.V3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = P.nch * M.n;

  float2 Q[NQ][16];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int k = 0; k < 16; ++k) Q[q][k] = make_float2(0.f, 0.f);

  // the value is the stored number times 2^exp per field
  const int scale_exp = rec1 ? rec1->exp + rec2->exp : 0;
  constexpr bool kF16 = std::is_same<PsiT, __half2>::value;
  // float16: S2 (re-read by every mask pair) is staged in shared memory for
  // the block's sites; S1 is read once per value, from the staged copy when
  // S1 = S2 (SAME) and from global memory otherwise
  uint32_t* st = reinterpret_cast<uint32_t*>(red + (SITES ? 0 : (kMesonThreads / 32) * nv));
  if constexpr (kF16) {
    stage_f16(st, reinterpret_cast<const __half2*>(S2), t, blockIdx.x * kMesonThreads, V3);
    __syncthreads();
  }
  auto contract = [&](const auto& p1, const auto& p2) {
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        float2 a[9];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int b = 0; b < 3; ++b) a[d * 3 + b] = p1((al * 3 + d) * 12 + be * 3 + b);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int al2 = al ^ P.ma[q], be2 = be ^ P.mb[q];
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
              const float2 y = p2((al2 * 3 + d) * 12 + be2 * 3 + b);
              const float2 x = a[d * 3 + b];
              // acc += x * conj(y)
              acc.x = fmaf(x.x, y.x, acc.x);
              acc.x = fmaf(x.y, y.y, acc.x);
              acc.y = fmaf(x.y, y.x, acc.y);
              acc.y = fmaf(-x.x, y.y, acc.y);
            }
          Q[q][al * 4 + be] = acc;
        }
      }
  };
  if (live) {
    if constexpr (kF16) {
      const F16Staged p2(st + threadIdx.x * kF16Stride);
      if constexpr (SAME)
        contract(p2, p2);
      else
        contract(F16Global(reinterpret_cast<const uint32_t*>(S1), t, s3, V3), p2);
    } else {
      contract(SoASite<PsiT>(S1, t, s3, V3), SoASite<PsiT>(S2, t, s3, V3));
    }
  }

  // exp(-i p.(x - x0)) needs the three non-decay coordinates
  int c0 = 0, c1 = 0, c2 = 0;
  if (!M.zero_only && live) {
    c0 = s3 % g.sL[0];
    c1 = (s3 / g.sL[0]) % g.sL[1];
    c2 = s3 / (g.sL[0] * g.sL[1]);
  }

#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    for (int j = 0; j < P.nch; ++j) {
      if (P.q_of[j] != q) continue;
      float2 c = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 w = P.w[j][k];
        c.x = fmaf(w.x, Q[q][k].x, c.x);
        c.x = fmaf(-w.y, Q[q][k].y, c.x);
        c.y = fmaf(w.x, Q[q][k].y, c.y);
        c.y = fmaf(w.y, Q[q][k].x, c.y);
      }
      if constexpr (SITES) {
        if (live)
          sites[((long long)P.out_row[j] * g.Nt + t) * V3 + s3] =
              (scale_exp && site_scale) ? make_float2(ldexpf(c.x, scale_exp), ldexpf(c.y, scale_exp)) : c;
      } else {
        for (int m = 0; m < M.n; ++m) {
          float2 v = c;
          if (!M.zero_only) {
            // phase index: sum_k n_k (x_k - o_k) V3/L_k  (mod V3), exact in integers
            long long num = (long long)M.k[m][0] * (((c0 - M.origin[0]) % g.sL[0] + g.sL[0]) % g.sL[0]) * (V3 / g.sL[0]) +
                            (long long)M.k[m][1] * (((c1 - M.origin[1]) % g.sL[1] + g.sL[1]) % g.sL[1]) * (V3 / g.sL[1]) +
                            (long long)M.k[m][2] * (((c2 - M.origin[2]) % g.sL[2] + g.sL[2]) % g.sL[2]) * (V3 / g.sL[2]);
            num %= V3;
            if (num < 0) num += V3;
            float sn, cs;
            sincospif(2.0f * (float)num / (float)V3, &sn, &cs);
            // v = c * (cs - i sn)
            v = make_float2(c.x * cs + c.y * sn, c.y * cs - c.x * sn);
          }
          double re = live ? (double)v.x : 0.0;
          double im = live ? (double)v.y : 0.0;
          re = warp_sum(re);
          im = warp_sum(im);
          if (lane == 0) red[warp * nv + j * M.n + m] = make_double2(re, im);
        }
      }
    }
  }
  if constexpr (SITES) return;
  __syncthreads();
  const int nwarps = kMesonThreads / 32;
  for (int i = threadIdx.x; i < nv; i += kMesonThreads) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      re += red[w * nv + i].x;
      im += red[w * nv + i].y;
    }
    const int j = i / M.n, m = i % M.n;
    const long long o = ((long long)P.out_row[j] * M.n + m) * g.Nt + t;
    atomicAdd(out + 2 * o, ldexp(re, scale_exp));
    atomicAdd(out + 2 * o + 1, ldexp(im, scale_exp));
  }
}


// ---- staged kernel (component-major F32 / BF16 propagators) -----------------
//
// A block owns kStSites consecutive sites of one timeslice.  S2, which every
// mask pair re-reads, is staged once in shared memory by one tensor-map copy
// (box: the block's sites x the 144 components, [comp][site] in shared
// memory, so a warp's 32 sites of one component are 256 consecutive bytes);
// S1 is read once per element (from the staged copy when S1 = S2).  Two
// threads share a site: thread half h forms the colour contractions of sink
// spins 2h and 2h+1, and the channel values, linear in Q, are sums of the
// two halves' partial values (added in the timeslice sums, or through shared
// memory for site values).
constexpr int kStSites = 64;
constexpr int kStThreads = 2 * kStSites;

template <int NQ, typename PsiT, bool SITES, bool SAME>
__global__ void __launch_bounds__(kStThreads) meson_staged_kernel(const __grid_constant__ CUtensorMap map2,
                                                                  const PsiT* __restrict__ S1, Geom g, MesonPass P,
                                                                  Moms M, double* __restrict__ out,
                                                                  float2* __restrict__ sites, const ScaleRecord* rec1,
                                                                  const ScaleRecord* rec2, int site_scale,
                                                                  double2* __restrict__ partial, unsigned int* status,
                                                                  long long timeout_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PsiT* st = reinterpret_cast<PsiT*>(smem_raw);                         // [144][kStSites]
  constexpr uint32_t kStageBytes = 144u * kStSites * sizeof(PsiT);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kStageBytes);
  float2* cval = reinterpret_cast<float2*>(smem_raw + kStageBytes + 16);   // [nch][kStSites] channel values
  float2* phase = cval + kMaxPassCh * kStSites;                           // [n_mom][kStSites] cos, sin
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int site = tid & (kStSites - 1), h = tid / kStSites;
  const int s0 = blockIdx.x * kStSites, t = blockIdx.y;
  const int s3 = s0 + site;
  const bool live = s3 < g.V3;
  const int V3 = g.V3;
  const uint32_t bar_a = ptx::smem_addr(bar);

  if (tid == 0) {
    ptx::mbar_init(bar_a, 1);
    ptx::fence_mbar_init();
    ptx::mbar_arrive_expect_tx(bar_a, kStageBytes);
    ptx::tensor_g2s_2d(ptx::smem_addr(st), &map2, s0, t * 144, bar_a);
  }
  __syncthreads();
  const bool ok = ptx::mbar_wait_bounded(bar_a, 0, timeout_ns);
  if (!__syncthreads_and(ok ? 1 : 0)) {
    // the copy did not complete in time: record it, give the copy one more
    // bounded wait so that it is not in flight when the block exits
    if (tid == 0) {
      atomicOr(status, kStatusFullWait);
      if (!ptx::mbar_wait_bounded(bar_a, 0, timeout_ns)) atomicOr(status, kStatusDrain);
    }
    return;
  }

  const int scale_exp = rec1 ? rec1->exp + rec2->exp : 0;
  const PsiT* s1g = S1 + (long long)t * 144 * V3 + s3;
  auto p1 = [&](int comp) -> float2 {
    if constexpr (SAME) return lds_elem(st + comp * kStSites + site);
    else return ld2(s1g + (long long)comp * V3);
  };
  auto p2 = [&](int comp) -> float2 { return lds_elem(st + comp * kStSites + site); };

  // Q_q(alpha, beta) for alpha = 2h + i (index i*4 + beta) as packed pairs:
  // with x = S1 element and y = S2 element, x conj(y) = (P.x + P.y, R.x + R.y)
  // for P = (x.x, x.y) (.) y and R = (x.y, -x.x) (.) y: two fma.rn.f32x2 per
  // complex multiply-accumulate, y used as loaded.
  u64 Qp[NQ][8], Qr[NQ][8];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      const int al = 2 * h + i;
      u64 xa[9], xr[9];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float2 x = live ? p1((al * 3 + d) * 12 + be * 3 + b) : make_float2(0.f, 0.f);
          xa[d * 3 + b] = pack2(x.x, x.y);
          xr[d * 3 + b] = pack2(x.y, -x.x);
        }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int base = ((al ^ P.ma[q]) * 3) * 12 + (be ^ P.mb[q]) * 3;
        u64 pa = 0ull, ra = 0ull;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const u64 y = live ? lds_pair_st(st + (base + d * 12 + b) * kStSites + site) : 0ull;
            pa = fma2(xa[d * 3 + b], y, pa);
            ra = fma2(xr[d * 3 + b], y, ra);
          }
        Qp[q][i * 4 + be] = pa;
        Qr[q][i * 4 + be] = ra;
      }
    }
  // Q as (re, im) pairs and i Q = (-im, re), for the weighted channel sums
  u64 Qz[NQ][8], Qi[NQ][8];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float2 a = unpack2(Qp[q][k]), b = unpack2(Qr[q][k]);
      const float re = a.x + a.y, im = b.x + b.y;
      Qz[q][k] = pack2(re, im);
      Qi[q][k] = pack2(-im, re);
    }
  // this half's part of channel j: sum_k (w.x, w.x) (.) Q + (w.y, w.y) (.) iQ
  auto part_of = [&](int q, int j) -> float2 {
    u64 c = 0ull;
    for (int qq = 0; qq < NQ; ++qq) {
      if (qq != q) continue;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        c = fma2(P.wre[j][8 * h + k], Qz[qq][k], c);
        c = fma2(P.wim[j][8 * h + k], Qi[qq][k], c);
      }
    }
    return unpack2(c);
  };
  // the upper half's parts go through shared memory; the lower half adds its
  // own and stores the channel value (cval[j][site], or the site output)
  if (h == 1) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      for (int j = P.jlo[q]; j < P.jhi[q]; ++j) cval[j * kStSites + site] = part_of(q, j);
  }
  __syncthreads();
  if (h == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      for (int j = P.jlo[q]; j < P.jhi[q]; ++j) {
        const float2 mine = part_of(q, j), o = cval[j * kStSites + site];
        const float2 c = live ? make_float2(mine.x + o.x, mine.y + o.y) : make_float2(0.f, 0.f);
        if constexpr (SITES) {
          if (live)
            sites[((long long)P.out_row[j] * g.Nt + t) * V3 + s3] =
                (scale_exp && site_scale) ? make_float2(ldexpf(c.x, scale_exp), ldexpf(c.y, scale_exp)) : c;
        } else {
          cval[j * kStSites + site] = c;
        }
      }
  } else if (!SITES && !M.zero_only) {
    // phases exp(-i p.(x - x0)) of the block's sites, one momentum per pass of the upper half
    int c0 = 0, c1 = 0, c2 = 0;
    if (live) {
      c0 = s3 % g.sL[0];
      c1 = (s3 / g.sL[0]) % g.sL[1];
      c2 = s3 / (g.sL[0] * g.sL[1]);
    }
    for (int m = 0; m < M.n; ++m) {
      // phase index: sum_k n_k (x_k - o_k) V3/L_k  (mod V3), exact in integers
      long long num = (long long)M.k[m][0] * (((c0 - M.origin[0]) % g.sL[0] + g.sL[0]) % g.sL[0]) * (V3 / g.sL[0]) +
                      (long long)M.k[m][1] * (((c1 - M.origin[1]) % g.sL[1] + g.sL[1]) % g.sL[1]) * (V3 / g.sL[1]) +
                      (long long)M.k[m][2] * (((c2 - M.origin[2]) % g.sL[2] + g.sL[2]) % g.sL[2]) * (V3 / g.sL[2]);
      num %= V3;
      if (num < 0) num += V3;
      float sn, cs;
      sincospif(2.0f * (float)num / (float)V3, &sn, &cs);
      phase[m * kStSites + site] = make_float2(cs, sn);
    }
  }
  if constexpr (SITES) return;
  __syncthreads();
  // sums over the block's sites of c_j(x) exp(-i p_m.(x - x0)): warp w takes
  // values w, w + 4, ...; each lane adds two sites, then a butterfly in
  // two-float arithmetic (hi + lo, error-free sums), FP64 only for the
  // block's one atomic per value
  const int nv = P.nch * M.n;
  for (int v = warp; v < nv; v += kStThreads / 32) {
    const int j = v / M.n, m = v % M.n;
    float2 a = cval[j * kStSites + lane], b = cval[j * kStSites + lane + 32];
    if (!M.zero_only) {
      const float2 pa = phase[m * kStSites + lane], pb = phase[m * kStSites + lane + 32];
      a = make_float2(a.x * pa.x + a.y * pa.y, a.y * pa.x - a.x * pa.y);  // c (cs - i sn)
      b = make_float2(b.x * pb.x + b.y * pb.y, b.y * pb.x - b.x * pb.y);
    }
    float2 hi, lo;
    two_sum(a.x, b.x, hi.x, lo.x);
    two_sum(a.y, b.y, hi.y, lo.y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float hx = __shfl_xor_sync(0xffffffffu, hi.x, o), lx = __shfl_xor_sync(0xffffffffu, lo.x, o);
      const float hy = __shfl_xor_sync(0xffffffffu, hi.y, o), ly = __shfl_xor_sync(0xffffffffu, lo.y, o);
      float ex, ey;
      two_sum(hi.x, hx, hi.x, ex);
      two_sum(hi.y, hy, hi.y, ey);
      lo.x = lo.x + lx + ex;
      lo.y = lo.y + ly + ey;
    }
    if (lane == 0)  // this block's part of the sum; meson_fold_kernel adds the blocks in order
      partial[((long long)t * gridDim.x + blockIdx.x) * nv + v] = make_double2((double)hi.x + (double)lo.x,
                                                                               (double)hi.y + (double)lo.y);
  }
}

// out[value][t] = 2^exp * sum over the blocks of timeslice t of their partial
// sums (fixed order: the result does not depend on scheduling).
__global__ void __launch_bounds__(128) meson_fold_kernel(const double2* __restrict__ partial, int nbx, MesonPass P,
                                                         int n_mom, int Nt, double* __restrict__ out,
                                                         const ScaleRecord* rec1, const ScaleRecord* rec2) {
  __shared__ double2 red[4];
  const int v = blockIdx.x, t = blockIdx.y, nv = P.nch * n_mom;
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nbx; b += 128) {
    const double2 x = partial[((long long)t * nbx + b) * nv + v];
    re += x.x;
    im += x.y;
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(re, im);
  __syncthreads();
  if (threadIdx.x == 0) {
    re = red[0].x + red[1].x + red[2].x + red[3].x;
    im = red[0].y + red[1].y + red[2].y + red[3].y;
    const int scale_exp = rec1 ? rec1->exp + rec2->exp : 0;
    const int j = v / n_mom, m = v % n_mom;
    const long long o = ((long long)P.out_row[j] * n_mom + m) * Nt + t;
    out[2 * o] = ldexp(re, scale_exp);
    out[2 * o + 1] = ldexp(im, scale_exp);
  }
}


// ---- orbit kernel: channels whose two masks are equal (ma == mb) -------------
//
// With ma = mb = m for every channel (the sixteen mesons Gamma_snk =
// Gamma_src = Gamma(n) are of this kind: Gamma^dag permutes like Gamma), the
// spin positions (alpha, beta) split into four orbits by d = alpha ^ beta,
// and Q_m(alpha, alpha ^ d) pairs S1's block at (alpha, alpha ^ d) with S2's
// block at (alpha ^ m, alpha ^ m ^ d), which lies in the same orbit.  A
// thread owns (site, orbit d) for one first propagator: it keeps the orbit's
// four 3x3 colour blocks of S_a in registers and streams the same orbit's
// four blocks of each S_b once, each element serving all four masks.  The
// four orbit threads of a site add their parts of each channel value through
// shared memory.  One block stages OK_NP propagators for OK_S sites of one
// timeslice with one tensor-map copy each (box: OK_S sites x 144
// components, [comp][site] in shared memory).
//
// Pairs: first propagators ia in [0, NA) (staged index A[ia]) with second
// propagators ib in [0, NB) (staged index B[ib]); site values of pair
// (ia, ib) and channel j go to row rows[j] + (ia * NB + ib) * row_step.
constexpr int kOrbMaxProps = 8;

struct OrbitSet {
  int np;                          // staged propagators
  int na, nb;                      // first and second propagators in use (<= NA, NB)
  int A[kOrbMaxProps], B[kOrbMaxProps];
  int row_step;                    // SITES rows per pair (multi-propagator use)
  int t0;                          // first timeslice of the launch (blockIdx.y = t - t0)
  int nt_out;                      // timeslices of the site-value buffer
  CUtensorMap map[kOrbMaxProps];   // staged propagators, box OK_S sites x 144 components
};

template <int NA, int NB, int OK_S, typename PsiT, bool SITES, bool SAME = false>
__global__ void __launch_bounds__(OK_S * 4 * NA) meson_orbit_kernel(const __grid_constant__ OrbitSet O, Geom g,
                                                                     MesonPass P, Moms M, float2* __restrict__ sites,
                                                                     const ScaleRecord* rec1, const ScaleRecord* rec2,
                                                                     int site_scale, double2* __restrict__ partial,
                                                                     unsigned int* status, long long timeout_ns) {
  constexpr int kThreads = OK_S * 4 * NA;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // F32/BF16: [prop][144 comps][OK_S sites]; float16 (site-major fields):
  // [prop][3 vector groups][OK_S sites][48 words]
  constexpr bool kF16 = std::is_same<PsiT, __half2>::value;
  // a float16 self pair is converted once into FP32 rows of one site's 144
  // components (padded to 145: a warp's column reads hit distinct banks)
  constexpr bool kF16T = kF16 && SAME && NA == 1;
  PsiT* st = reinterpret_cast<PsiT*>(smem_raw);
  constexpr uint32_t kPropBytes = 144u * OK_S * sizeof(PsiT);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + (size_t)O.np * kPropBytes);
  float2* cpart = reinterpret_cast<float2*>(bar + 2);     // [4 orbits][kMaxPassCh][NA][OK_S] orbit parts
  float2* tr = cpart + 4 * NA * kMaxPassCh * OK_S;        // [OK_S][145] (float16 self pair)
  float2* phase = tr + (kF16T ? OK_S * 145 : 0);          // [n_mom][OK_S] (reducing form)
  const int tid = threadIdx.x;
  // warp-uniform orbit: thread = ((d * NA) + ia) * OK_S + site
  const int site = tid % OK_S, ia = (tid / OK_S) % NA, d = tid / (OK_S * NA);
  const int s0 = blockIdx.x * OK_S, t = blockIdx.y;  // t: timeslice O.t0 + t of the lattice
  const bool act = ia < O.na;                         // threads of an unused first propagator idle
  const int s3 = s0 + site;
  const bool live = s3 < g.V3;
  const int V3 = g.V3;
  const uint32_t bar_a = ptx::smem_addr(bar);

  if (tid == 0) {
    ptx::mbar_init(bar_a, 1);
    ptx::fence_mbar_init();
    ptx::mbar_arrive_expect_tx(bar_a, (uint32_t)O.np * kPropBytes);
    for (int i = 0; i < O.np; ++i) {
      if constexpr (kF16)
        ptx::tensor_g2s_3d(ptx::smem_addr(smem_raw + (size_t)i * kPropBytes), &O.map[i], 0, s0, (O.t0 + t) * 3,
                           bar_a);
      else
        ptx::tensor_g2s_2d(ptx::smem_addr(smem_raw + (size_t)i * kPropBytes), &O.map[i], s0, (O.t0 + t) * 144, bar_a);
    }
  }
  __syncthreads();
  const bool ok = ptx::mbar_wait_bounded(bar_a, 0, timeout_ns);
  if (!__syncthreads_and(ok ? 1 : 0)) {
    if (tid == 0) {
      atomicOr(status, kStatusFullWait);
      if (!ptx::mbar_wait_bounded(bar_a, 0, timeout_ns)) atomicOr(status, kStatusDrain);
    }
    return;
  }
  if constexpr (kF16T) {
    // [3 vector groups][OK_S sites][48 words] -> [site][component], FP32;
    // word w of group vg is vector v = 16 vg + w / 3, sink colour w % 3
    const uint32_t* L = reinterpret_cast<const uint32_t*>(smem_raw);
    for (int idx = tid; idx < 3 * OK_S * 48; idx += kThreads) {
      const int vg = idx / (OK_S * 48), r = idx - vg * (OK_S * 48), ss = r / 48, w = r - ss * 48;
      const int v = vg * 16 + w / 3, c = w % 3;
      tr[ss * 145 + ((v / 12) * 3 + c) * 12 + v % 12] = f16_word(L[idx]);
    }
    __syncthreads();
  }
  // element (comp) of staged propagator i at this thread's site
  auto elem = [&](int i, int comp) -> u64 {
    if constexpr (kF16T) {
      (void)i;
      return lds_pair_st(tr + site * 145 + comp);
    } else if constexpr (kF16) {
      const int w = f16_site_word(comp);  // vector group * 48 + word
      return lds_pair_st(st + (size_t)i * 144 * OK_S + ((w / 48) * OK_S + site) * 48 + w % 48);
    } else {
      return lds_pair_st(st + ((size_t)i * 144 + comp) * OK_S + site);
    }
  };
  // component of (spin row al, spin column be, colour row c, colour column e)
  auto comp_of = [](int al, int be, int c, int e) { return (al * 3 + c) * 12 + be * 3 + e; };

  if constexpr (!SITES) {
    // phases of the block's sites for the momentum sums, read after the
    // barrier that follows the orbit parts
    if (d == 1 && !M.zero_only) {
      int c0 = 0, c1 = 0, c2 = 0;
      if (live) {
        c0 = s3 % g.sL[0];
        c1 = (s3 / g.sL[0]) % g.sL[1];
        c2 = s3 / (g.sL[0] * g.sL[1]);
      }
      for (int m = 0; m < M.n; ++m) {
        long long num = (long long)M.k[m][0] * (((c0 - M.origin[0]) % g.sL[0] + g.sL[0]) % g.sL[0]) * (V3 / g.sL[0]) +
                        (long long)M.k[m][1] * (((c1 - M.origin[1]) % g.sL[1] + g.sL[1]) % g.sL[1]) * (V3 / g.sL[1]) +
                        (long long)M.k[m][2] * (((c2 - M.origin[2]) % g.sL[2] + g.sL[2]) % g.sL[2]) * (V3 / g.sL[2]);
        num %= V3;
        if (num < 0) num += V3;
        float sn, cs;
        sincospif(2.0f * (float)num / (float)V3, &sn, &cs);
        phase[m * OK_S + site] = make_float2(cs, sn);
      }
    }
  }
  // this thread's orbit blocks of S_a: x[al][c*3+e] at (al, al ^ d)
  u64 x[4][9];
  const int pa = O.A[act ? ia : 0];
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int k = 0; k < 9; ++k) x[al][k] = elem(pa, comp_of(al, al ^ d, k / 3, k % 3));

  for (int ib = 0; ib < O.nb; ++ib) {
    const int pb = O.B[ib];
    // Q as (re, im) and i Q = (-im, re)
    u64 Qz[4][4], Qi[4][4];
    if constexpr (SAME) {
      // S2 = S1: S2's orbit blocks are this thread's x, and
      // Q_m(al ^ m, .) = conj(Q_m(al, .)): |x|^2 sums for m = 0 and one
      // product per pair {al, al ^ m} (al the smaller) for m = 1, 2, 3
      (void)pb;
      u64 P0[4], Pp[3][2], Rp[3][2];
#pragma unroll
      for (int al = 0; al < 4; ++al) P0[al] = 0ull;
#pragma unroll
      for (int m = 1; m < 4; ++m) Pp[m - 1][0] = Pp[m - 1][1] = Rp[m - 1][0] = Rp[m - 1][1] = 0ull;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        u64 xs[4];
#pragma unroll
        for (int b = 1; b < 4; ++b) {
          const float2 v = unpack2(x[b][k]);
          xs[b] = pack2(v.y, v.x);
        }
#pragma unroll
        for (int al = 0; al < 4; ++al) P0[al] = fma2(x[al][k], x[al][k], P0[al]);
#pragma unroll
        for (int m = 1; m < 4; ++m)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            // the pair's smaller member: m = 1: 0, 2; m = 2: 0, 1; m = 3: 0, 1
            const int lo = m == 1 ? 2 * q : q, hi = lo ^ m;
            Pp[m - 1][q] = fma2(x[lo][k], x[hi][k], Pp[m - 1][q]);
            Rp[m - 1][q] = fma2(x[lo][k], xs[hi], Rp[m - 1][q]);
          }
      }
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        const float2 a = unpack2(P0[al]);
        const float re = a.x + a.y;
        Qz[al][0] = pack2(re, 0.f);
        Qi[al][0] = pack2(0.f, re);
      }
#pragma unroll
      for (int m = 1; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int lo = m == 1 ? 2 * q : q, hi = lo ^ m;
          const float2 a = unpack2(Pp[m - 1][q]), b = unpack2(Rp[m - 1][q]);
          const float re = a.x + a.y, im = b.y - b.x;
          Qz[lo][m] = pack2(re, im);
          Qi[lo][m] = pack2(-im, re);
          Qz[hi][m] = pack2(re, -im);
          Qi[hi][m] = pack2(im, re);
        }
    } else {
    // Pm[al][m] and Rm[al][m]: packed parts of Q_m(al, al ^ d) = sum x conj(y)
    // for mask m = 0..3 (all four; every index compile-time), re = P.x + P.y,
    // im = R.y - R.x
    u64 Pm[4][4], Rm[4][4];
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int m = 0; m < 4; ++m) Pm[al][m] = Rm[al][m] = 0ull;
#pragma unroll
    for (int be = 0; be < 4; ++be) {  // S_b's orbit block at (be, be ^ d)
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const u64 y = live ? elem(pb, comp_of(be, be ^ d, k / 3, k % 3)) : 0ull;
        const float2 yv = unpack2(y);
        const u64 ys = pack2(yv.y, yv.x);
#pragma unroll
        for (int m = 0; m < 4; ++m) {  // S1 block (al, al ^ d) pairs with S2 block (al ^ m, al ^ m ^ d)
          const int al = be ^ m;
          Pm[al][m] = fma2(x[al][k], y, Pm[al][m]);
          Rm[al][m] = fma2(x[al][k], ys, Rm[al][m]);
        }
      }
    }
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 a = unpack2(Pm[al][m]), b = unpack2(Rm[al][m]);
        const float re = a.x + a.y, im = b.y - b.x;
        Qz[al][m] = pack2(re, im);
        Qi[al][m] = pack2(-im, re);
      }
    }
    // this orbit's part of every channel: sum_al w_j(al, al ^ d) Q_m(al, al ^ d)
    // for the channels j of mask m (host-grouped: P.mlo[m] <= j < P.mhi[m])
    if (act) {
#pragma unroll
      for (int m = 0; m < 4; ++m)
        for (int j = P.mlo[m]; j < P.mhi[m]; ++j) {
          u64 c = 0ull;
#pragma unroll
          for (int al = 0; al < 4; ++al) {
            const int k = al * 4 + (al ^ d);
            c = fma2(P.wre[j][k], Qz[al][m], c);
            c = fma2(P.wim[j][k], Qi[al][m], c);
          }
          cpart[((d * kMaxPassCh + j) * NA + ia) * OK_S + site] = unpack2(c);  // a warp's lanes: contiguous
        }
    }
    __syncthreads();
    if constexpr (SITES) {
      // the four orbits' parts of each (first propagator, channel, site), shared by all threads
      const int scale_exp = rec1 ? rec1->exp + rec2->exp : 0;
      for (int u = tid; u < P.nch * NA * OK_S; u += kThreads) {
        const int us = u % OK_S, ua = (u / OK_S) % NA, uj = u / (OK_S * NA);
        if (ua >= O.na) continue;
        float2 c = make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const float2 v = cpart[((o * kMaxPassCh + uj) * NA + ua) * OK_S + us];
          c.x += v.x;
          c.y += v.y;
        }
        const int us3 = s0 + us;
        if (us3 < V3) {
          const long long row = (long long)P.out_row[uj] + (long long)(ua * O.nb + ib) * O.row_step;
          sites[(row * O.nt_out + t) * V3 + us3] =
              (scale_exp && site_scale) ? make_float2(ldexpf(c.x, scale_exp), ldexpf(c.y, scale_exp)) : c;
        }
      }
    } else {
      // timeslice/momentum sums of the block's sites (NA = NB = 1): thread
      // (channel tid / TPC, sites 4 (tid % TPC) .. +3) adds the four
      // orbits' parts of its sites, multiplies them by the phases and sums
      // them in two-float arithmetic; the channel's TPC = OK_S / 4 lanes
      // finish each sum with a butterfly
      constexpr int TPC = OK_S / 4;
      static_assert(SITES || (NA == 1 && OK_S % 4 == 0 && TPC <= 32 && (TPC & (TPC - 1)) == 0),
                    "the reducing form takes one pair and 4 sites per lane, a power-of-two lanes per channel");
      const int uj = tid / TPC, g4 = (tid % TPC) * 4;
      const int nv = P.nch * M.n;
      float2 cs[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float2 c = make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const float2 v = cpart[(o * kMaxPassCh + uj) * OK_S + g4 + q];
          c.x += v.x;
          c.y += v.y;
        }
        cs[q] = (uj < P.nch && s0 + g4 + q < V3) ? c : make_float2(0.f, 0.f);
      }
      for (int m = 0; m < M.n; ++m) {
        float2 hi = make_float2(0.f, 0.f), lo = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float2 a = cs[q];
          if (!M.zero_only) {
            const float2 pa2 = phase[m * OK_S + g4 + q];
            a = make_float2(a.x * pa2.x + a.y * pa2.y, a.y * pa2.x - a.x * pa2.y);  // c (cs - i sn)
          }
          float ex, ey;
          two_sum(hi.x, a.x, hi.x, ex);
          two_sum(hi.y, a.y, hi.y, ey);
          lo.x += ex;
          lo.y += ey;
        }
#pragma unroll
        for (int o = TPC / 2; o > 0; o >>= 1) {
          const float hx = __shfl_xor_sync(0xffffffffu, hi.x, o), lx = __shfl_xor_sync(0xffffffffu, lo.x, o);
          const float hy = __shfl_xor_sync(0xffffffffu, hi.y, o), ly = __shfl_xor_sync(0xffffffffu, lo.y, o);
          float ex, ey;
          two_sum(hi.x, hx, hi.x, ex);
          two_sum(hi.y, hy, hi.y, ey);
          lo.x = lo.x + lx + ex;
          lo.y = lo.y + ly + ey;
        }
        if (tid % TPC == 0 && uj < P.nch)
          partial[((long long)t * gridDim.x + blockIdx.x) * nv + uj * M.n + m] =
              make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
      }
    }
    __syncthreads();  // cpart is reused by the next second propagator
  }
}


// The orbit kernel for one pass of one pair (S1, S2), or QDPG_ERR_UNSUPPORTED
// where it does not apply (a channel with different masks, two different
// float16 propagators, a component row not a multiple of 16 bytes, no
// tensor-map support).
// Sites per block, for site-value output and for the reducing form (32 each:
// measured faster than 16-site blocks at 16^3x32 and 24^3x48).
constexpr int kOrbitSitesS = 32;
constexpr int kOrbitSitesR = 32;

int launch_orbit_pass(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                      float2* sites, cudaStream_t s, int site_scale) {
  const int kS = sites ? kOrbitSitesS : kOrbitSitesR;
  const Geom& g = S1->g;
  const bool bf = S1->prec == QDPG_BF16;
  const bool h16 = S1->prec == QDPG_F16;
  const bool same = S1->data == S2->data;
  if (S1->prec != QDPG_F32 && !bf && !(h16 && same)) return QDPG_ERR_UNSUPPORTED;  // float16: self pairs
  for (int q = 0; q < P.nq; ++q)
    if (P.ma[q] != P.mb[q]) return QDPG_ERR_UNSUPPORTED;
  const int esize = (bf || h16) ? 4 : 8;
  if (!h16 && ((long long)g.V3 * esize) % 16 != 0) return QDPG_ERR_UNSUPPORTED;
  OrbitSet O{};
  O.np = same ? 1 : 2;
  O.na = O.nb = 1;
  O.A[0] = 0;
  O.B[0] = same ? 0 : 1;
  O.row_step = 0;
  O.t0 = 0;
  O.nt_out = g.Nt;
  const qdpg_field* staged[2] = {S1, S2};
  // F32/BF16: (site; component row) boxes of kS x 144; float16: (word; site;
  // timeslice-vector-group) boxes of 48 x kS x 3
  for (int i = 0; i < O.np; ++i)
    if (reinterpret_cast<uintptr_t>(staged[i]->data) % 16 != 0 ||
        !(h16 ? encode_map_3d(&O.map[i], staged[i]->data, 4, 48, (uint64_t)g.V3, (uint64_t)g.Nt * 3, 48 * 4,
                              (uint64_t)g.V3 * 48 * 4, 48, kS, 3)
              : encode_map_2d(&O.map[i], staged[i]->data, esize, (uint64_t)g.V3, (uint64_t)g.Nt * 144,
                              (uint64_t)g.V3 * esize, kS, 144)))
      return QDPG_ERR_UNSUPPORTED;
  unsigned int* status = device_status_word();
  if (!status) return QDPG_ERR_UNSUPPORTED;
  const size_t smem = (size_t)O.np * 144 * kS * esize + 16 + (size_t)4 * kMaxPassCh * kS * sizeof(float2) +
                      (h16 ? (size_t)kS * 145 * sizeof(float2) : 0) + (size_t)M.n * kS * sizeof(float2);
  dim3 grid((g.V3 + kS - 1) / kS, g.Nt);
  void* partial = nullptr;
  if (!sites) {
    const int arc = dev_alloc(&partial, sizeof(double2) * (size_t)grid.x * g.Nt * P.nch * M.n, s,
                              "meson_2pt partial sums");
    if (arc != QDPG_OK) return arc;
  }
  ProfScope prof("meson_2pt", s);
  cudaError_t e = cudaSuccess;
#define QDPG_ORBIT(T, SITES)                                                                                   \
  do {                                                                                                         \
    constexpr int KS = SITES ? kOrbitSitesS : kOrbitSitesR;                                                    \
    auto k = same ? meson_orbit_kernel<1, 1, KS, T, SITES, true> : meson_orbit_kernel<1, 1, KS, T, SITES>;     \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
    if (e == cudaSuccess)                                                                                      \
      k<<<grid, kS * 4, smem, s>>>(O, g, P, M, sites, S1->rec, S2->rec, site_scale,                            \
                                   static_cast<double2*>(partial), status, wait_timeout_ns());                  \
  } while (0)
  if (h16) {
    if (sites) QDPG_ORBIT(__half2, true);
    else QDPG_ORBIT(__half2, false);
  } else if (bf) {
    if (sites) QDPG_ORBIT(__nv_bfloat162, true);
    else QDPG_ORBIT(__nv_bfloat162, false);
  } else {
    if (sites) QDPG_ORBIT(float2, true);
    else QDPG_ORBIT(float2, false);
  }
#undef QDPG_ORBIT
  if (e != cudaSuccess) {
    dev_free(partial, s);
    return fail(QDPG_ERR_CUDA, "meson_2pt: smem attribute: %s", cudaGetErrorString(e));
  }
  int rc = check_launch("meson_2pt");
  if (rc == QDPG_OK && !sites) {
    meson_fold_kernel<<<dim3(P.nch * M.n, g.Nt), 128, 0, s>>>(static_cast<const double2*>(partial), (int)grid.x, P,
                                                              M.n, g.Nt, out, S1->rec, S2->rec);
    rc = check_launch("meson_2pt fold");
  }
  dev_free(partial, s);
  return rc;
}

// The staged kernel for one pass, or QDPG_ERR_UNSUPPORTED where it does not
// apply (float16's site-major layout; a component row of the timeslice not a
// multiple of 16 bytes; no tensor-map support).
int launch_staged_pass(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                       float2* sites, cudaStream_t s, int site_scale) {
  const Geom& g = S1->g;
  const bool bf = S1->prec == QDPG_BF16;
  if (S1->prec != QDPG_F32 && !bf) return QDPG_ERR_UNSUPPORTED;
  const int esize = bf ? 4 : 8;
  if (((long long)g.V3 * esize) % 16 != 0 || reinterpret_cast<uintptr_t>(S2->data) % 16 != 0) return QDPG_ERR_UNSUPPORTED;
  CUtensorMap map;
  if (!encode_map_2d(&map, S2->data, esize, (uint64_t)g.V3, (uint64_t)g.Nt * 144, (uint64_t)g.V3 * esize, kStSites,
                     144))
    return QDPG_ERR_UNSUPPORTED;
  unsigned int* status = device_status_word();
  if (!status) return QDPG_ERR_UNSUPPORTED;
  const bool same = S1->data == S2->data;
  const size_t stage = (size_t)144 * kStSites * esize;
  const size_t smem = stage + 16 + (size_t)(kMaxPassCh + M.n) * kStSites * sizeof(float2);
  dim3 grid((g.V3 + kStSites - 1) / kStSites, g.Nt);
  // per-block partial sums of the timeslice/momentum values (no atomics:
  // hundreds of blocks per timeslice would serialise on the same outputs)
  void* partial = nullptr;
  if (!sites) {
    const int arc = dev_alloc(&partial, sizeof(double2) * (size_t)grid.x * g.Nt * P.nch * M.n, s,
                              "meson_2pt partial sums");
    if (arc != QDPG_OK) return arc;
  }
  ProfScope prof("meson_2pt", s);
  cudaError_t e = cudaSuccess;
#define QDPG_STAGED(NQ, T, SITES, SAME)                                                                        \
  do {                                                                                                         \
    auto k = meson_staged_kernel<NQ, T, SITES, SAME>;                                                          \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
    if (e == cudaSuccess)                                                                                      \
      k<<<grid, kStThreads, smem, s>>>(map, static_cast<const T*>(S1->data), g, P, M, out, sites, S1->rec,     \
                                       S2->rec, site_scale, static_cast<double2*>(partial), status,            \
                                       wait_timeout_ns());                                                     \
  } while (0)
#define QDPG_STAGED_T(NQ, T)                                  \
  do {                                                        \
    if (sites && same) QDPG_STAGED(NQ, T, true, true);        \
    else if (sites) QDPG_STAGED(NQ, T, true, false);          \
    else if (same) QDPG_STAGED(NQ, T, false, true);           \
    else QDPG_STAGED(NQ, T, false, false);                    \
  } while (0)
#define QDPG_STAGED_NQ(NQ)                                    \
  do {                                                        \
    if (bf) QDPG_STAGED_T(NQ, __nv_bfloat162);                \
    else QDPG_STAGED_T(NQ, float2);                           \
  } while (0)
  switch (P.nq) {
    case 1: QDPG_STAGED_NQ(1); break;
    case 2: QDPG_STAGED_NQ(2); break;
    case 3: QDPG_STAGED_NQ(3); break;
    default: QDPG_STAGED_NQ(4); break;
  }
#undef QDPG_STAGED_NQ
#undef QDPG_STAGED_T
#undef QDPG_STAGED
  if (e != cudaSuccess) {
    dev_free(partial, s);
    return fail(QDPG_ERR_CUDA, "meson_2pt: smem attribute: %s", cudaGetErrorString(e));
  }
  int rc = check_launch("meson_2pt");
  if (rc == QDPG_OK && !sites) {
    meson_fold_kernel<<<dim3(P.nch * M.n, g.Nt), 128, 0, s>>>(static_cast<const double2*>(partial), (int)grid.x, P,
                                                              M.n, g.Nt, out, S1->rec, S2->rec);
    rc = check_launch("meson_2pt fold");
  }
  dev_free(partial, s);
  return rc;
}

struct Channel {
  int row, ma, mb;
  float2 w[16];
};

// (lo, hi) FP32 pair as the 64-bit register image fma.rn.f32x2 takes (lo in the low word).
inline unsigned long long pack_host(float lo, float hi) {
  unsigned int a, b;
  memcpy(&a, &lo, 4);
  memcpy(&b, &hi, 4);
  return (unsigned long long)a | ((unsigned long long)b << 32);
}

int launch_pass(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                float2* sites, cudaStream_t s, int site_scale = 1) {
  const Geom& g = S1->g;
  const int form = debug_meson_form();  // 0: best available, 1: staged, 2: global reads
  if (form == 0) {
    const int rc = launch_orbit_pass(P, M, S1, S2, out, sites, s, site_scale);
    if (rc != QDPG_ERR_UNSUPPORTED) return rc;
  }
  if (form <= 1) {
    const int rc = launch_staged_pass(P, M, S1, S2, out, sites, s, site_scale);
    if (rc != QDPG_ERR_UNSUPPORTED) return rc;
  }
  dim3 grid((g.V3 + kMesonThreads - 1) / kMesonThreads, g.Nt);
  size_t smem = sites ? 0 : (size_t)(kMesonThreads / 32) * P.nch * M.n * sizeof(double2);
  const bool bf = S1->prec == QDPG_BF16;
  const bool h16 = S1->prec == QDPG_F16;
  const bool same = S1->data == S2->data;
  if (h16) smem += (size_t)kMesonThreads * kF16Stride * sizeof(uint32_t);  // staged S2
  ProfScope prof("meson_2pt", s);
#define QDPG_MESON_KERNEL(NQ, T, SITES, SAME)                                                          \
  do {                                                                                                 \
    auto k = meson_kernel<NQ, T, SITES, SAME>;                                                         \
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k<<<grid, kMesonThreads, smem, s>>>(static_cast<const T*>(S1->data), static_cast<const T*>(S2->data), g, P, M, \
                                        out, sites, S1->rec, S2->rec, site_scale);                     \
  } while (0)
#define QDPG_MESON_LAUNCH(NQ)                                                  \
  do {                                                                         \
    if (bf) {                                                                  \
      if (sites) QDPG_MESON_KERNEL(NQ, __nv_bfloat162, true, false);           \
      else QDPG_MESON_KERNEL(NQ, __nv_bfloat162, false, false);                \
    } else if (h16) {                                                          \
      if (sites && same) QDPG_MESON_KERNEL(NQ, __half2, true, true);           \
      else if (sites) QDPG_MESON_KERNEL(NQ, __half2, true, false);             \
      else if (same) QDPG_MESON_KERNEL(NQ, __half2, false, true);              \
      else QDPG_MESON_KERNEL(NQ, __half2, false, false);                       \
    } else {                                                                   \
      if (sites) QDPG_MESON_KERNEL(NQ, float2, true, false);                   \
      else QDPG_MESON_KERNEL(NQ, float2, false, false);                        \
    }                                                                          \
  } while (0)
  switch (P.nq) {
    case 1: QDPG_MESON_LAUNCH(1); break;
    case 2: QDPG_MESON_LAUNCH(2); break;
    case 3: QDPG_MESON_LAUNCH(3); break;
    default: QDPG_MESON_LAUNCH(4); break;
  }
#undef QDPG_MESON_LAUNCH
#undef QDPG_MESON_KERNEL
  return check_launch("meson_2pt");
}

}  // namespace

}  // namespace qdpg

using namespace qdpg;

namespace qdpg {
namespace {


// Channel masks and weights (the XOR-mask form of the trace, see the top of
// this file), sorted by mask pair.
int build_channels(const int* gamma_snk, const int* gamma_src, int n_chan, std::vector<Channel>& sorted,
                   const char* who) {
  static const int g5[4] = {1, 1, -1, -1};
  std::vector<Channel> chans;
  for (int j = 0; j < n_chan; ++j) {
    if (gamma_snk[j] < 0 || gamma_snk[j] > 15 || gamma_src[j] < 0 || gamma_src[j] > 15)
      return fail(QDPG_ERR_ARG, "%s: gamma index outside 0..15 in channel %d", who, j);
    Mat4 A = Gamma(gamma_snk[j]);
    Mat4 B = dagger(Gamma(gamma_src[j]));
    Channel c{};
    c.row = j;
    c.ma = xor_mask(A);
    c.mb = xor_mask(B);
    if (c.ma < 0 || c.mb < 0) return fail(QDPG_ERR_ARG, "%s: internal gamma table error", who);
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        CInt w = A.m[al ^ c.ma][al] * B.m[be][be ^ c.mb];
        const int sgn = g5[be ^ c.mb] * g5[al ^ c.ma];
        c.w[al * 4 + be] = make_float2((float)(sgn * w.re), (float)(sgn * w.im));
      }
    chans.push_back(c);
  }
  sorted.clear();
  for (int pair = 0; pair < 16; ++pair)
    for (const Channel& c : chans)
      if (c.ma * 4 + c.mb == pair) sorted.push_back(c);
  return QDPG_OK;
}

// Add channel c to pass P (pair index q); channels of one pair stay contiguous.
void add_channel(MesonPass& P, int q, const Channel& c) {
  P.q_of[P.nch] = q;
  P.out_row[P.nch] = c.row;
  for (int k = 0; k < 16; ++k) {
    P.w[P.nch][k] = c.w[k];
    P.wre[P.nch][k] = pack_host(c.w[k].x, c.w[k].x);
    P.wim[P.nch][k] = pack_host(c.w[k].y, c.w[k].y);
  }
  ++P.nch;
  if (P.jhi[q] == 0) P.jlo[q] = P.nch - 1;
  P.jhi[q] = P.nch;
  if (c.ma == c.mb) {  // channels arrive sorted by mask pair: those of (m, m) are contiguous
    if (P.mhi[c.ma] == 0) P.mlo[c.ma] = P.nch - 1;
    P.mhi[c.ma] = P.nch;
  }
}

// Shared by the reducing entry point (out_dev) and the site-value one (sites).
int meson_common(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src, int n_chan,
                 const int* moms, int n_mom, const int origin[4], double* out_dev, float2* sites, void* stream) {
  if (!S1 || !S2 || !gamma_snk || !gamma_src || !moms || (!out_dev && !sites))
    return fail(QDPG_ERR_ARG, "meson_2pt: null argument");
  if (S1->kind != QDPG_PROPAGATOR || S2->kind != QDPG_PROPAGATOR)
    return fail(QDPG_ERR_SHAPE, "meson_2pt: S1 and S2 must be propagators");
  if ((S1->prec != QDPG_F32 && S1->prec != QDPG_BF16 && S1->prec != QDPG_F16) || S2->prec != S1->prec)
    return fail(QDPG_ERR_DTYPE, "meson_2pt: S1 and S2 must share F32, BF16 or F16 storage");
  for (int mu = 0; mu < 4; ++mu)
    if (S1->g.L[mu] != S2->g.L[mu] || S1->g.jd != S2->g.jd) return fail(QDPG_ERR_SHAPE, "meson_2pt: lattices differ");
  if (n_chan < 1 || n_chan > 256) return fail(QDPG_ERR_ARG, "meson_2pt: n_chan %d outside 1..256", n_chan);
  if (n_mom < 1 || n_mom > kMaxMom) return fail(QDPG_ERR_ARG, "meson_2pt: n_mom %d outside 1..%d", n_mom, kMaxMom);
  const Geom& g = S1->g;

  Moms M{};
  M.n = n_mom;
  M.zero_only = (n_mom == 1 && moms[0] == 0 && moms[1] == 0 && moms[2] == 0);
  for (int k = 0; k < 3; ++k) M.origin[k] = origin ? origin[g.sd[k]] : 0;
  for (int m = 0; m < n_mom; ++m)
    for (int k = 0; k < 3; ++k) M.k[m][k] = moms[3 * m + k];

  // channels grouped by mask pair, then packed into passes of <= 4 pairs and <= 16 channels
  std::vector<Channel> sorted;
  const int crc = build_channels(gamma_snk, gamma_src, n_chan, sorted, "meson_2pt");
  if (crc != QDPG_OK) return crc;

  cudaStream_t s = as_stream(stream);
  if (!sites) {
    cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * (size_t)n_chan * n_mom * g.Nt, s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "meson_2pt: memset: %s", cudaGetErrorString(e));
  }

  // Many momenta: the pass's site values (unscaled, pass-local rows) go to a
  // temporary buffer and the tensor cores project them; the fields' scale is
  // applied to the FP64 sums there.  Each channel's block of the output
  // (n_mom x Nt) is then copied into place.
  const bool tensor_proj = !sites && n_mom >= kTensorProjMinMom;
  std::vector<int> mom_flat(3 * (size_t)n_mom);
  for (int i = 0; i < 3 * n_mom; ++i) mom_flat[i] = moms[i];
  MesonPass P{};
  auto flush = [&]() -> int {
    if (P.nch == 0) return QDPG_OK;
    int rc = QDPG_OK;
    if (!tensor_proj) {
      rc = launch_pass(P, M, S1, S2, out_dev, sites, s);
    } else {
      MesonPass L = P;
      for (int j = 0; j < L.nch; ++j) L.out_row[j] = j;
      const size_t site_bytes = sizeof(float2) * (size_t)L.nch * g.Nt * g.V3;
      const size_t out_bytes = sizeof(double) * 2 * (size_t)L.nch * n_mom * g.Nt;
      void* tsites = nullptr;
      void* tout = nullptr;
      int arc = dev_alloc(&tsites, site_bytes, s, "meson_2pt site values");
      if (arc == QDPG_OK) arc = dev_alloc(&tout, out_bytes, s, "meson_2pt projected sums");
      if (arc != QDPG_OK) {
        dev_free(tsites, s);
        return arc;
      }
      rc = launch_pass(L, M, S1, S2, nullptr, static_cast<float2*>(tsites), s, 0);
      if (rc == QDPG_OK)
        rc = launch_momproj(g, tsites, L.nch, mom_flat.data(), n_mom, origin, static_cast<double*>(tout), S1->rec, 1,
                            S2->rec, 1, s);
      const size_t blk = sizeof(double) * 2 * (size_t)n_mom * g.Nt;
      for (int j = 0; j < L.nch && rc == QDPG_OK; ++j) {
        cudaError_t e = cudaMemcpyAsync(reinterpret_cast<char*>(out_dev) + blk * P.out_row[j],
                                        static_cast<char*>(tout) + blk * j, blk, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) rc = fail(QDPG_ERR_CUDA, "meson_2pt: copy: %s", cudaGetErrorString(e));
      }
      dev_free(tsites, s);
      dev_free(tout, s);
    }
    P = MesonPass{};
    return rc;
  };
  for (const Channel& c : sorted) {
    int q = -1;
    for (int i = 0; i < P.nq; ++i)
      if (P.ma[i] == c.ma && P.mb[i] == c.mb) q = i;
    if ((q < 0 && P.nq == 4) || P.nch == kMaxPassCh) {
      int rc = flush();
      if (rc) return rc;
      q = -1;
    }
    if (q < 0) {
      q = P.nq++;
      P.ma[q] = c.ma;
      P.mb[q] = c.mb;
    }
    add_channel(P, q, c);  // channels arrive grouped by mask pair
  }
  return flush();
}

}  // namespace
}  // namespace qdpg

extern "C" {

int qdpg_meson_2pt(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src, int n_chan,
                   const int* moms, int n_mom, const int origin[4], double* out_dev, void* stream) {
  if (!out_dev) return fail(QDPG_ERR_ARG, "meson_2pt: null argument");
  return meson_common(S1, S2, gamma_snk, gamma_src, n_chan, moms, n_mom, origin, out_dev, nullptr, stream);
}

int qdpg_meson_sites(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src, int n_chan,
                     void* sites_dev, void* stream) {
  if (!sites_dev) return fail(QDPG_ERR_ARG, "meson_sites: null argument");
  if (reinterpret_cast<uintptr_t>(sites_dev) % 8) return fail(QDPG_ERR_ARG, "meson_sites: buffer not 8-byte aligned");
  static const int zero[3] = {0, 0, 0};
  return meson_common(S1, S2, gamma_snk, gamma_src, n_chan, zero, 1, nullptr, nullptr,
                      static_cast<float2*>(sites_dev), stream);
}

}  // extern "C"

// ---- all pairs of a set of propagators -------------------------------------

namespace qdpg {
namespace {

struct RecTable {
  const ScaleRecord* r[kOrbMaxProps];
};
// exp[(a * n + b) * n_chan + c] = exp_a + exp_b: the scale of pair (a, b)'s sums
__global__ void pair_exp_kernel_t(RecTable R, int n, int n_chan, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n * n_chan) return;
  const int pair = i / n_chan, a = pair / n, b = pair % n;
  out[i] = R.r[a]->exp + R.r[b]->exp;
}

}  // namespace
}  // namespace qdpg

extern "C" int qdpg_meson_2pt_multi(const qdpg_field_t* props, int n_props, const int* gamma_snk,
                                    const int* gamma_src, int n_chan, const int* moms, int n_mom, const int origin[4],
                                    double* out_dev, void* stream) {
  constexpr int kS = 4;  // sites per block: 4 sites x 4 orbits x 8 first propagators = 128 threads
  if (!props || !gamma_snk || !gamma_src || !moms || !out_dev) return fail(QDPG_ERR_ARG, "meson_2pt_multi: null argument");
  if (n_props < 1 || n_props > kOrbMaxProps)
    return fail(QDPG_ERR_ARG, "meson_2pt_multi: n_props %d outside 1..%d", n_props, kOrbMaxProps);
  for (int i = 0; i < n_props; ++i) {
    const qdpg_field* f = props[i];
    if (!f) return fail(QDPG_ERR_ARG, "meson_2pt_multi: null propagator %d", i);
    if (f->kind != QDPG_PROPAGATOR) return fail(QDPG_ERR_SHAPE, "meson_2pt_multi: field %d is not a propagator", i);
    if (f->prec != QDPG_F32 && f->prec != QDPG_BF16 && f->prec != QDPG_F16)
      return fail(QDPG_ERR_DTYPE, "meson_2pt_multi: propagators must be F32, BF16 or F16 (field %d)", i);
    if (f->prec != props[0]->prec) return fail(QDPG_ERR_DTYPE, "meson_2pt_multi: propagators differ in storage");
    for (int mu = 0; mu < 4; ++mu)
      if (f->g.L[mu] != props[0]->g.L[mu] || f->g.jd != props[0]->g.jd)
        return fail(QDPG_ERR_SHAPE, "meson_2pt_multi: lattices differ");
  }
  if (n_chan < 1 || n_chan > kMaxPassCh)
    return fail(QDPG_ERR_ARG, "meson_2pt_multi: n_chan %d outside 1..%d", n_chan, kMaxPassCh);
  if (n_mom < 1 || n_mom > kMaxMom) return fail(QDPG_ERR_ARG, "meson_2pt_multi: n_mom %d outside 1..%d", n_mom, kMaxMom);
  std::vector<Channel> sorted;
  int rc = build_channels(gamma_snk, gamma_src, n_chan, sorted, "meson_2pt_multi");
  if (rc != QDPG_OK) return rc;
  MesonPass P{};
  for (const Channel& c : sorted) {
    if (c.ma != c.mb)
      return fail(QDPG_ERR_UNSUPPORTED, "meson_2pt_multi: channel %d has unequal masks (only Gamma_snk, Gamma_src "
                  "pairs that permute alike, such as Gamma_snk = Gamma_src)", c.row);
    int q = -1;
    for (int i = 0; i < P.nq; ++i)
      if (P.ma[i] == c.ma) q = i;
    if (q < 0) {
      q = P.nq++;
      P.ma[q] = P.mb[q] = c.ma;
    }
    add_channel(P, q, c);
  }
  const Geom& g = props[0]->g;
  const bool bf = props[0]->prec == QDPG_BF16;
  const bool h16 = props[0]->prec == QDPG_F16;
  const int esize = bf || h16 ? 4 : 8;
  if (!h16 && ((long long)g.V3 * esize) % 16 != 0)
    return fail(QDPG_ERR_UNSUPPORTED, "meson_2pt_multi: a timeslice's component row must be a multiple of 16 bytes");
  OrbitSet O{};
  O.np = O.na = O.nb = n_props;
  O.row_step = n_chan;
  RecTable R{};
  for (int i = 0; i < n_props; ++i) {
    O.A[i] = O.B[i] = i;
    R.r[i] = props[i]->rec;
    // F32/BF16: (site; component row) boxes of kS x 144; float16: (word; site;
    // timeslice-vector-group) boxes of 48 x kS x 3 (a site's 48 words of one group are contiguous)
    const bool mapped =
        reinterpret_cast<uintptr_t>(props[i]->data) % 16 == 0 &&
        (h16 ? encode_map_3d(&O.map[i], props[i]->data, 4, 48, (uint64_t)g.V3, (uint64_t)g.Nt * 3, 48 * 4,
                             (uint64_t)g.V3 * 48 * 4, 48, kS, 3)
             : encode_map_2d(&O.map[i], props[i]->data, esize, (uint64_t)g.V3, (uint64_t)g.Nt * 144,
                             (uint64_t)g.V3 * esize, kS, 144));
    if (!mapped) return fail(QDPG_ERR_UNSUPPORTED, "meson_2pt_multi: no tensor map for propagator %d", i);
  }
  unsigned int* status = device_status_word();
  if (!status) return fail(QDPG_ERR_CUDA, "meson_2pt_multi: no status word");
  Moms M{};
  M.n = 1;
  M.zero_only = true;
  cudaStream_t s = as_stream(stream);

  // timeslice batches: site values of all pairs and channels for up to 4 GiB
  const long long n_rows = (long long)n_props * n_props * n_chan;
  const size_t per_t = (size_t)n_rows * g.V3 * sizeof(float2);
  int T = (int)std::min<long long>(g.Nt, std::max<long long>(1, (4LL << 30) / (long long)per_t));
  void *sites = nullptr, *tout = nullptr, *cexp = nullptr;
  rc = dev_alloc(&sites, per_t * T, s, "meson_2pt_multi site values");
  if (rc == QDPG_OK) rc = dev_alloc(&tout, sizeof(double) * 2 * (size_t)n_rows * n_mom * T, s, "meson_2pt_multi sums");
  if (rc == QDPG_OK) rc = dev_alloc(&cexp, sizeof(int) * (size_t)n_rows, s, "meson_2pt_multi scales");
  if (rc == QDPG_OK) {
    pair_exp_kernel_t<<<(int)((n_rows + 127) / 128), 128, 0, s>>>(R, n_props, n_chan, static_cast<int*>(cexp));
    rc = check_launch("meson_2pt_multi scales");
  }
  const size_t smem = (size_t)n_props * 144 * kS * esize + 16 + (size_t)4 * kOrbMaxProps * kMaxPassCh * kS * sizeof(float2);
  std::vector<int> mom_flat(moms, moms + 3 * (size_t)n_mom);
  for (int t0 = 0; t0 < g.Nt && rc == QDPG_OK; t0 += T) {
    const int nt = std::min(T, g.Nt - t0);
    O.t0 = t0;
    O.nt_out = nt;
    dim3 grid((g.V3 + kS - 1) / kS, nt);
    cudaError_t e = cudaSuccess;
    {
      ProfScope prof("meson_2pt", s);
#define QDPG_MULTI(T_)                                                                                          \
  do {                                                                                                         \
    auto k = meson_orbit_kernel<kOrbMaxProps, kOrbMaxProps, kS, T_, true>;                                     \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
    if (e == cudaSuccess)                                                                                      \
      k<<<grid, kS * 4 * kOrbMaxProps, smem, s>>>(O, g, P, M, static_cast<float2*>(sites), nullptr, nullptr, 0, \
                                                  nullptr, status, wait_timeout_ns());                          \
  } while (0)
      if (h16) QDPG_MULTI(__half2);
      else if (bf) QDPG_MULTI(__nv_bfloat162);
      else QDPG_MULTI(float2);
#undef QDPG_MULTI
      if (e != cudaSuccess) rc = fail(QDPG_ERR_CUDA, "meson_2pt_multi: smem attribute: %s", cudaGetErrorString(e));
      else rc = check_launch("meson_2pt_multi");
    }
    if (rc != QDPG_OK) break;
    Geom gb = g;  // the batch as a lattice of nt timeslices for the projection's row layout
    gb.Nt = nt;
    gb.L[g.jd] = nt;
    gb.V = (long long)nt * g.V3;
    rc = launch_momproj(gb, sites, (int)n_rows, mom_flat.data(), n_mom, origin, static_cast<double*>(tout), nullptr,
                        0, nullptr, 0, s, static_cast<const int*>(cexp));
    if (rc != QDPG_OK) break;
    // tout[row][m][0..nt) -> out[row][m][t0..t0+nt)
    const cudaError_t ce = cudaMemcpy2DAsync(out_dev + 2 * (size_t)t0, sizeof(double) * 2 * g.Nt, tout,
                                             sizeof(double) * 2 * nt, sizeof(double) * 2 * nt,
                                             (size_t)n_rows * n_mom, cudaMemcpyDeviceToDevice, s);
    if (ce != cudaSuccess) rc = fail(QDPG_ERR_CUDA, "meson_2pt_multi: copy: %s", cudaGetErrorString(ce));
  }
  dev_free(sites, s);
  dev_free(tout, s);
  dev_free(cexp, s);
  return rc;
}
