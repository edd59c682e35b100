// The orbit form of the meson contraction (channels whose two masks are
// equal): the kernel, its one-pair launcher and the eight-propagator launcher
// of qdpg_meson_2pt_multi.
#include "meson_dev.cuh"

namespace qdpg {
namespace meson {

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
  if (h16) {  // float16: self pairs only
    if (sites) {
      auto k = meson_orbit_kernel<1, 1, kOrbitSitesS, __half2, true, true>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k<<<grid, kOrbitSitesS * 4, smem, s>>>(O, g, P, M, sites, S1->rec, S2->rec, site_scale,
                                               static_cast<double2*>(partial), status, wait_timeout_ns());
    } else {
      auto k = meson_orbit_kernel<1, 1, kOrbitSitesR, __half2, false, true>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess)
        k<<<grid, kOrbitSitesR * 4, smem, s>>>(O, g, P, M, sites, S1->rec, S2->rec, site_scale,
                                               static_cast<double2*>(partial), status, wait_timeout_ns());
    }
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
    rc = launch_meson_fold(static_cast<const double2*>(partial), (int)grid.x, P, M.n, g.Nt, out, S1->rec, S2->rec, s);
  }
  dev_free(partial, s);
  return rc;
}

int launch_orbit_multi(const OrbitSet& O, const Geom& g, const MesonPass& P, const Moms& M, float2* sites, int prec,
                       size_t smem, dim3 grid, cudaStream_t s, unsigned int* status) {
  cudaError_t e = cudaSuccess;
#define QDPG_MULTI(T_)                                                                                          \
  do {                                                                                                         \
    auto k = meson_orbit_kernel<kOrbMaxProps, kOrbMaxProps, kMultiSites, T_, true>;                            \
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
    if (e == cudaSuccess)                                                                                      \
      k<<<grid, kMultiSites * 4 * kOrbMaxProps, smem, s>>>(O, g, P, M, sites, nullptr, nullptr, 0, nullptr,    \
                                                           status, wait_timeout_ns());                         \
  } while (0)
  if (prec == QDPG_F16) QDPG_MULTI(__half2);
  else if (prec == QDPG_BF16) QDPG_MULTI(__nv_bfloat162);
  else QDPG_MULTI(float2);
#undef QDPG_MULTI
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "meson_2pt_multi: smem attribute: %s", cudaGetErrorString(e));
  return check_launch("meson_2pt_multi");
}

}  // namespace meson
}  // namespace qdpg
