// The global-read form of the meson contraction: one thread per site reading
// both propagators from global memory (float16 pairs of different
// propagators, and the reference form for tests).  The kernel template and
// its launcher for one storage type; meson_global_{f32,bf16,f16}.cu
// instantiate it, so that the three compile in parallel.
#pragma once

#include "meson_dev.cuh"

namespace qdpg {
namespace meson {

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

template <typename T>
int launch_global_t(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                    float2* sites, cudaStream_t s, int site_scale) {
  const Geom& g = S1->g;
  dim3 grid((g.V3 + kMesonThreads - 1) / kMesonThreads, g.Nt);
  size_t smem = sites ? 0 : (size_t)(kMesonThreads / 32) * P.nch * M.n * sizeof(double2);
  constexpr bool h16 = std::is_same<T, __half2>::value;
  const bool same = S1->data == S2->data;
  if (h16) smem += (size_t)kMesonThreads * kF16Stride * sizeof(uint32_t);  // staged S2
  ProfScope prof("meson_2pt", s);
#define QDPG_MESON_KERNEL(NQ, SITES, SAME)                                                             \
  do {                                                                                                 \
    auto k = meson_kernel<NQ, T, SITES, SAME>;                                                         \
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k<<<grid, kMesonThreads, smem, s>>>(static_cast<const T*>(S1->data), static_cast<const T*>(S2->data), g, P, M, \
                                        out, sites, S1->rec, S2->rec, site_scale);                     \
  } while (0)
#define QDPG_MESON_LAUNCH(NQ)                                                  \
  do {                                                                         \
    if constexpr (h16) {                                                       \
      if (sites && same) QDPG_MESON_KERNEL(NQ, true, true);                    \
      else if (sites) QDPG_MESON_KERNEL(NQ, true, false);                      \
      else if (same) QDPG_MESON_KERNEL(NQ, false, true);                       \
      else QDPG_MESON_KERNEL(NQ, false, false);                                \
    } else {                                                                   \
      if (sites) QDPG_MESON_KERNEL(NQ, true, false);                           \
      else QDPG_MESON_KERNEL(NQ, false, false);                                \
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

}  // namespace meson
}  // namespace qdpg
