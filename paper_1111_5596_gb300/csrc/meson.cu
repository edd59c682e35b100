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
// This file: the channel plan, the entry points, the staged form and the
// fold of the blocks' partial sums; the orbit form is in meson_orbit.cu and
// the global-read form in meson_global_*.cu (shared definitions in
// meson_dev.cuh).  Site values are FP32; a block's timeslice/momentum sums
// are two-float, folded over the blocks in FP64 in a fixed order.
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
#include "meson_dev.cuh"
namespace qdpg {

namespace meson {

using namespace gamma_host;

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

int launch_meson_fold(const double2* partial, int nbx, const MesonPass& P, int nmom, int Nt, double* out,
                      const ScaleRecord* r1, const ScaleRecord* r2, cudaStream_t s) {
  meson_fold_kernel<<<dim3(P.nch * nmom, Nt), 128, 0, s>>>(partial, nbx, P, nmom, Nt, out, r1, r2);
  return check_launch("meson_2pt fold");
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
  const int form = debug_meson_form();  // 0: best available, 1: staged, 2: global reads
  if (form == 0) {
    const int rc = launch_orbit_pass(P, M, S1, S2, out, sites, s, site_scale);
    if (rc != QDPG_ERR_UNSUPPORTED) return rc;
  }
  if (form <= 1) {
    const int rc = launch_staged_pass(P, M, S1, S2, out, sites, s, site_scale);
    if (rc != QDPG_ERR_UNSUPPORTED) return rc;
  }
  return launch_global_pass(P, M, S1, S2, out, sites, s, site_scale);
}

}  // namespace meson

}  // namespace qdpg

using namespace qdpg;

namespace qdpg {
namespace {

using namespace meson;
using namespace gamma_host;

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

using namespace meson;

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
  constexpr int kS = kMultiSites;  // sites per block: 4 sites x 4 orbits x 8 first propagators = 128 threads
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
    {
      ProfScope prof("meson_2pt", s);
      rc = launch_orbit_multi(O, g, P, M, static_cast<float2*>(sites), props[0]->prec, smem, grid, s, status);
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
