// Definitions shared by the meson translation units (meson.cu: planning,
// entry points, the staged form and the fold; meson_orbit.cu: the orbit
// kernel; meson_global_*.cu: the global-read form): the pass plan, the
// momentum table, element loaders and the two-float and warp sums, and the
// launchers each unit provides to the others.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"
#include "tmap.h"

namespace qdpg {
namespace meson {

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

// Sites per block, for site-value output and for the reducing form (32 each:
// measured faster than 16-site blocks at 16^3x32 and 24^3x48).
constexpr int kOrbitSitesS = 32;
constexpr int kOrbitSitesR = 32;

// One pass (up to 16 channels) of one pair: the orbit kernel (meson_orbit.cu;
// QDPG_ERR_UNSUPPORTED where it does not apply) and the global-read kernel
// (meson_global_*.cu, by storage).  out: the pass's [channel][momentum][t] sums, or sites:
// its site values for the projection.
int launch_orbit_pass(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                      float2* sites, cudaStream_t s, int site_scale);
int launch_global_f32(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                      float2* sites, cudaStream_t s, int site_scale);
int launch_global_bf16(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                       float2* sites, cudaStream_t s, int site_scale);
int launch_global_f16(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                      float2* sites, cudaStream_t s, int site_scale);
inline int launch_global_pass(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2,
                              double* out, float2* sites, cudaStream_t s, int site_scale) {
  if (S1->prec == QDPG_F16) return launch_global_f16(P, M, S1, S2, out, sites, s, site_scale);
  if (S1->prec == QDPG_BF16) return launch_global_bf16(P, M, S1, S2, out, sites, s, site_scale);
  return launch_global_f32(P, M, S1, S2, out, sites, s, site_scale);
}
// The eight-propagator orbit kernel of qdpg_meson_2pt_multi over nitems
// blocks of kMultiSites sites (meson_orbit.cu); prec: the fields' storage.
constexpr int kMultiSites = 4;
int launch_orbit_multi(const OrbitSet& O, const Geom& g, const MesonPass& P, const Moms& M, float2* sites, int prec,
                       size_t smem, dim3 grid, cudaStream_t s, unsigned int* status);
// out[value][t] from the blocks' partial sums (meson.cu).
int launch_meson_fold(const double2* partial, int nbx, const MesonPass& P, int nmom, int Nt, double* out,
                      const ScaleRecord* r1, const ScaleRecord* r2, cudaStream_t s);

}  // namespace meson
}  // namespace qdpg
