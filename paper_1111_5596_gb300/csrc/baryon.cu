// Baryon two-point functions: the baryonic part of the paper's hadron
// spectrum stage (Sec. 5, Fig. 4 "HAD").
//
//   C(t, p) = sum_{x in t} exp(-i p.(x - x0)) sum_{alpha alpha'} P_{alpha' alpha}
//             < chi_alpha(x) chibar_alpha'(x0) >,     P = (1 + parity g4) / 2,
//
// nucleon  chi = eps_abc (u_a^T C g5 d_b) u_c,   Delta++  chi = eps_abc (u_a^T C g3 u_b) u_c,
// conjugate operator with Gbar = g4 G^dag g4 and Grassmann order (c', b', a').
// Wick's theorem gives 2 (nucleon) or 6 (Delta) pairings of the quarks with
// the antiquarks; with the source colours c' = src0, b' = src1, a' = src2 each
// term is one of
//   T^{cc'} K0(S^{aa'}, S^{bb'}),  K0(X, S^{bb'}),  K1(S^{ab'}, X),  ...
// where T^{cc'} = tr(P S^{cc'}), X = S^{..} P S^{..} (4x4 spin), and
//   K0(A, B) = sum G_{rho sigma} Gbar_{sigma' rho'} A_{rho rho'} B_{sigma sigma'},
//   K1(A, B) = sum G_{rho sigma} Gbar_{sigma' rho'} A_{rho sigma'} B_{sigma rho'},
// each a 16-term sum because G and Gbar are signed permutations (XOR masks).
// The pairing signs come from the Grassmann order of the six fields.
//
// A block stages the two propagators of 32 consecutive sites of a timeslice
// in shared memory (coalesced loads); each warp then contracts one site at
// a time, its lanes splitting the 36 (eps, eps') colour terms x Wick terms.
// Site values are FP32; timeslice/momentum sums are FP64.
#include <cuda_fp16.h>

#include <vector>

#include "gamma_host.h"
#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {

namespace {

using namespace gamma_host;

constexpr int kSites = 32;       // sites per block
constexpr int kWarps = 8;
constexpr int kStride = 145;     // float2 per staged site (144 + 1 against bank conflicts)
constexpr int kMaxMomB = 64;

struct BaryonSpec {
  int nterms;        // 2 (nucleon) or 6 (Delta)
  int mG, mGb;       // XOR masks of G and Gbar
  float2 g[4];       // G[r][r ^ mG]
  float2 gb[4];      // Gbar[r][r ^ mGb]
  float par;         // parity of the projector
  int eps[36][7];    // a, b, c, a', b', c', eps_abc * eps_a'b'c'
};

struct BMoms {
  int n;
  int origin[3];
  int k[kMaxMomB][3];
  bool zero_only;
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ float2 ldb(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldb(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ float2 ldb(const __half2* p) { return __half22float2(*p); }
// Element (t, comp, s3) of a propagator: component-major (F32, BF16) or
// site-major float16 (qdpg.h).
template <typename PsiT>
__device__ __forceinline__ long long prop_off(int V3, int t, int comp, int s3) {
  return ((long long)t * 144 + comp) * V3 + s3;
}
template <>
__device__ __forceinline__ long long prop_off<__half2>(int V3, int t, int comp, int s3) {
  return f16_prop_index(V3, t, comp, s3);
}

// spin block S^{c c'}: element (al, alp) of the staged site
__device__ __forceinline__ void load_block(const float2* S, int c, int cp, float2 A[16]) {
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int alp = 0; alp < 4; ++alp) A[al * 4 + alp] = S[(al * 3 + c) * 12 + alp * 3 + cp];
}

// tr(P S^{cc'}) = (1/2) sum_al [S_{al al} + par S_{al, al^2}]
__device__ __forceinline__ float2 trace_P(const float2* S, int c, int cp, float par) {
  float2 t = make_float2(0.f, 0.f);
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    const float2 d = S[(al * 3 + c) * 12 + al * 3 + cp];
    const float2 o = S[(al * 3 + c) * 12 + (al ^ 2) * 3 + cp];
    t.x += 0.5f * (d.x + par * o.x);
    t.y += 0.5f * (d.y + par * o.y);
  }
  return t;
}

// X = A P B for 4x4 spin blocks: X_{r r'} = (1/2) sum_a A_{r a} (B_{a r'} + par B_{a^2, r'})
__device__ __forceinline__ void apb(const float2 A[16], const float2 B[16], float par, float2 X[16]) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float2 b = make_float2(0.5f * (B[a * 4 + rp].x + par * B[(a ^ 2) * 4 + rp].x),
                                     0.5f * (B[a * 4 + rp].y + par * B[(a ^ 2) * 4 + rp].y));
        acc = caddf(acc, cmulf(A[r * 4 + a], b));
      }
      X[r * 4 + rp] = acc;
    }
}

// K0(A, B) = sum_{rho, sigma'} g_rho gb_sigma' A_{rho, sigma'^mGb} B_{rho^mG, sigma'}
// K1(A, B) = sum_{rho, sigma'} g_rho gb_sigma' A_{rho, sigma'} B_{rho^mG, sigma'^mGb}
template <bool SWAP, int MG, int MGB>
__device__ __forceinline__ float2 kgg(const BaryonSpec& B, const float2 A[16], const float2 Bm[16]) {
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
      const float2 w = cmulf(B.g[r], B.gb[sp]);
      const float2 a = SWAP ? A[r * 4 + sp] : A[r * 4 + (sp ^ MGB)];
      const float2 b = SWAP ? Bm[(r ^ MG) * 4 + (sp ^ MGB)] : Bm[(r ^ MG) * 4 + sp];
      acc = caddf(acc, cmulf(w, cmulf(a, b)));
    }
  return acc;
}

// Masks of G = C g5 (nucleon) and C g3 (Delta); Gbar has the same mask.
template <int KIND>
struct Masks {
  static constexpr int mg = KIND == 0 ? 1 : 3;
};

// One Wick term of one colour combination; u = S_u, d = S_d (staged site).
template <int KIND>
__device__ __forceinline__ float2 baryon_term(const BaryonSpec& B, const float2* u, const float2* d, int combo, int term) {
  constexpr int MG = Masks<KIND>::mg;
  const int a = B.eps[combo][0], b = B.eps[combo][1], c = B.eps[combo][2];
  const int ap = B.eps[combo][3], bp = B.eps[combo][4], cp = B.eps[combo][5];
  const float sgn_eps = (float)B.eps[combo][6];
  float2 P1[16], P2[16], X[16];
  float2 v;
  float sgn;
  if (KIND == 0) {  // nucleon: u_a d_b u_c
    if (term == 0) {  // pairing (2,1,0): +T^{cc'} K0(u^{aa'}, d^{bb'})
      load_block(u, a, ap, P1);
      load_block(d, b, bp, P2);
      v = cmulf(trace_P(u, c, cp, B.par), kgg<false, MG, MG>(B, P1, P2));
      sgn = 1.f;
    } else {  // pairing (0,1,2): -K0(u^{ac'} P u^{ca'}, d^{bb'})
      load_block(u, a, cp, P1);
      load_block(u, c, ap, P2);
      apb(P1, P2, B.par, X);
      load_block(d, b, bp, P2);
      v = kgg<false, MG, MG>(B, X, P2);
      sgn = -1.f;
    }
  } else {  // Delta: u_a u_b u_c
    switch (term) {
      case 0:  // (2,1,0) +: T^{cc'} K0(u^{aa'}, u^{bb'})
        load_block(u, a, ap, P1);
        load_block(u, b, bp, P2);
        v = cmulf(trace_P(u, c, cp, B.par), kgg<false, MG, MG>(B, P1, P2));
        sgn = 1.f;
        break;
      case 1:  // (0,1,2) -: K0(u^{ac'} P u^{ca'}, u^{bb'})
        load_block(u, a, cp, P1);
        load_block(u, c, ap, P2);
        apb(P1, P2, B.par, X);
        load_block(u, b, bp, P2);
        v = kgg<false, MG, MG>(B, X, P2);
        sgn = -1.f;
        break;
      case 2:  // (1,0,2) +: K1(u^{ab'}, u^{bc'} P u^{ca'})
        load_block(u, b, cp, P1);
        load_block(u, c, ap, P2);
        apb(P1, P2, B.par, X);
        load_block(u, a, bp, P1);
        v = kgg<true, MG, MG>(B, P1, X);
        sgn = 1.f;
        break;
      case 3:  // (0,2,1) +: K1(u^{ac'} P u^{cb'}, u^{ba'})
        load_block(u, a, cp, P1);
        load_block(u, c, bp, P2);
        apb(P1, P2, B.par, X);
        load_block(u, b, ap, P1);
        v = kgg<true, MG, MG>(B, X, P1);
        sgn = 1.f;
        break;
      case 4:  // (2,0,1) -: K0(u^{aa'}, u^{bc'} P u^{cb'})
        load_block(u, b, cp, P1);
        load_block(u, c, bp, P2);
        apb(P1, P2, B.par, X);
        load_block(u, a, ap, P1);
        v = kgg<false, MG, MG>(B, P1, X);
        sgn = -1.f;
        break;
      default:  // (1,2,0) -: T^{cc'} K1(u^{ab'}, u^{ba'})
        load_block(u, a, bp, P1);
        load_block(u, b, ap, P2);
        v = cmulf(trace_P(u, c, cp, B.par), kgg<true, MG, MG>(B, P1, P2));
        sgn = -1.f;
        break;
    }
  }
  const float s = sgn * sgn_eps;
  return make_float2(s * v.x, s * v.y);
}

// SITES: write the site value to sites[t][x] (complex FP32) instead of reducing.
template <typename PsiT, int KIND, bool SITES>
__global__ void __launch_bounds__(kWarps * 32) baryon_kernel(const PsiT* __restrict__ Su, const PsiT* __restrict__ Sd,
                                                             Geom g, BaryonSpec B, BMoms M, double* __restrict__ out,
                                                             float2* __restrict__ sites, const ScaleRecord* ru,
                                                             const ScaleRecord* rd, int site_scale) {
  extern __shared__ float2 sm[];
  float2* su = sm;
  float2* sd = sm + kSites * kStride;
  double2* red = reinterpret_cast<double2*>(sm + 2 * kSites * kStride);  // [warp][n_mom]
  const int t = blockIdx.y;
  const int s0 = blockIdx.x * kSites;
  const int V3 = g.V3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // float16 storage: the value is the stored number times 2^exp (u, u, d)
  const int scale_exp = ru ? 2 * ru->exp + rd->exp : 0;

  // stage the two propagators of the block's sites ([site][comp], padded)
  for (int e = threadIdx.x; e < 144 * kSites; e += blockDim.x) {
    const int comp = e / kSites, i = e % kSites;
    const int s3 = s0 + i;
    float2 vu = make_float2(0.f, 0.f), vd = make_float2(0.f, 0.f);
    if (s3 < V3) {
      const long long off = prop_off<PsiT>(V3, t, comp, s3);
      vu = ldb(Su + off);
      vd = ldb(Sd + off);
    }
    su[i * kStride + comp] = vu;
    sd[i * kStride + comp] = vd;
  }
  for (int e = threadIdx.x; e < kWarps * M.n; e += blockDim.x) red[e] = make_double2(0.0, 0.0);
  __syncthreads();

  const int nwork = 36 * B.nterms;
  for (int i = warp; i < kSites; i += kWarps) {
    const int s3 = s0 + i;
    if (s3 >= V3) break;
    float2 acc = make_float2(0.f, 0.f);
    for (int wk = lane; wk < nwork; wk += 32)
      acc = caddf(acc, baryon_term<KIND>(B, su + i * kStride, sd + i * kStride, wk / B.nterms, wk % B.nterms));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
    }
    if constexpr (SITES) {
      if (lane == 0)
        sites[(long long)t * V3 + s3] =
            (scale_exp && site_scale) ? make_float2(ldexpf(acc.x, scale_exp), ldexpf(acc.y, scale_exp)) : acc;
      continue;
    }
    if (lane == 0) {
      int c0 = s3 % g.sL[0], c1 = (s3 / g.sL[0]) % g.sL[1], c2 = s3 / (g.sL[0] * g.sL[1]);
      for (int m = 0; m < M.n; ++m) {
        double re = acc.x, im = acc.y;
        if (!M.zero_only) {
          long long num = (long long)M.k[m][0] * (((c0 - M.origin[0]) % g.sL[0] + g.sL[0]) % g.sL[0]) * (V3 / g.sL[0]) +
                          (long long)M.k[m][1] * (((c1 - M.origin[1]) % g.sL[1] + g.sL[1]) % g.sL[1]) * (V3 / g.sL[1]) +
                          (long long)M.k[m][2] * (((c2 - M.origin[2]) % g.sL[2] + g.sL[2]) % g.sL[2]) * (V3 / g.sL[2]);
          num %= V3;
          if (num < 0) num += V3;
          float sn, cs;
          sincospif(2.0f * (float)num / (float)V3, &sn, &cs);
          re = (double)(acc.x * cs + acc.y * sn);
          im = (double)(acc.y * cs - acc.x * sn);
        }
        red[warp * M.n + m].x += re;
        red[warp * M.n + m].y += im;
      }
    }
  }
  if constexpr (SITES) return;
  __syncthreads();
  for (int m = threadIdx.x; m < M.n; m += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      re += red[w * M.n + m].x;
      im += red[w * M.n + m].y;
    }
    const long long o = (long long)m * g.Nt + t;
    atomicAdd(out + 2 * o, ldexp(re, scale_exp));
    atomicAdd(out + 2 * o + 1, ldexp(im, scale_exp));
  }
}

}  // namespace

}  // namespace qdpg

using namespace qdpg;

namespace {

int baryon_common(qdpg_field_t Su, qdpg_field_t Sd, int kind, int parity, const int* moms, int n_mom,
                  const int origin[4], double* out_dev, float2* sites, void* stream) {
  if (!Su || !moms || (!out_dev && !sites)) return fail(QDPG_ERR_ARG, "baryon_2pt: null argument");
  if (kind != 0 && kind != 1) return fail(QDPG_ERR_ARG, "baryon_2pt: kind %d is neither 0 (nucleon) nor 1 (Delta)", kind);
  if (parity != 1 && parity != -1) return fail(QDPG_ERR_ARG, "baryon_2pt: parity must be +1 or -1");
  if (!Sd) {
    if (kind == 0) return fail(QDPG_ERR_ARG, "baryon_2pt: the nucleon needs a d-quark propagator");
    Sd = Su;
  }
  if (Su->kind != QDPG_PROPAGATOR || Sd->kind != QDPG_PROPAGATOR)
    return fail(QDPG_ERR_SHAPE, "baryon_2pt: Su and Sd must be propagators");
  if ((Su->prec != QDPG_F32 && Su->prec != QDPG_BF16 && Su->prec != QDPG_F16) || Sd->prec != Su->prec)
    return fail(QDPG_ERR_DTYPE, "baryon_2pt: Su and Sd must share F32, BF16 or F16 storage");
  for (int mu = 0; mu < 4; ++mu)
    if (Su->g.L[mu] != Sd->g.L[mu] || Su->g.jd != Sd->g.jd) return fail(QDPG_ERR_SHAPE, "baryon_2pt: lattices differ");
  if (n_mom < 1 || n_mom > kMaxMomB) return fail(QDPG_ERR_ARG, "baryon_2pt: n_mom %d outside 1..%d", n_mom, kMaxMomB);
  const Geom& g = Su->g;

  BMoms M{};
  M.n = n_mom;
  M.zero_only = (n_mom == 1 && moms[0] == 0 && moms[1] == 0 && moms[2] == 0);
  for (int k = 0; k < 3; ++k) M.origin[k] = origin ? origin[g.sd[k]] : 0;
  for (int m = 0; m < n_mom; ++m)
    for (int k = 0; k < 3; ++k) M.k[m][k] = moms[3 * m + k];

  // G = C g5 (nucleon) or C g3 (Delta), Gbar = g4 G^dag g4
  const Mat4 Cm = charge_conj();
  const Mat4 G = mat_mul(Cm, kind == 0 ? Gamma(15) : basis_gamma(2));
  const Mat4 Gb = mat_mul(mat_mul(basis_gamma(3), dagger(G)), basis_gamma(3));
  BaryonSpec B{};
  B.nterms = kind == 0 ? 2 : 6;
  B.mG = xor_mask(G);
  B.mGb = xor_mask(Gb);
  if (B.mG != (kind == 0 ? 1 : 3) || B.mGb != B.mG) return fail(QDPG_ERR_ARG, "baryon_2pt: internal gamma table error");
  for (int r = 0; r < 4; ++r) {
    B.g[r] = make_float2((float)G.m[r][r ^ B.mG].re, (float)G.m[r][r ^ B.mG].im);
    B.gb[r] = make_float2((float)Gb.m[r][r ^ B.mGb].re, (float)Gb.m[r][r ^ B.mGb].im);
  }
  B.par = (float)parity;
  static const int perms[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  static const int psign[6] = {1, 1, 1, -1, -1, -1};
  int n = 0;
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q, ++n) {
      for (int k = 0; k < 3; ++k) {
        B.eps[n][k] = perms[p][k];
        B.eps[n][3 + k] = perms[q][k];
      }
      B.eps[n][6] = psign[p] * psign[q];
    }

  cudaStream_t s = as_stream(stream);
  // Many momenta: unscaled site values to a temporary buffer, projected on
  // the tensor cores with the fields' scale applied to the FP64 sums.
  const bool tensor_proj = !sites && n_mom >= kTensorProjMinMom;
  float2* ksites = sites;
  int site_scale = 1;
  if (tensor_proj) {
    void* t = nullptr;
    const int arc = dev_alloc(&t, sizeof(float2) * (size_t)g.Nt * g.V3, s, "baryon_2pt site values");
    if (arc != QDPG_OK) return arc;
    ksites = static_cast<float2*>(t);
    site_scale = 0;
  } else if (!sites) {
    cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * (size_t)n_mom * g.Nt, s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "baryon_2pt: memset: %s", cudaGetErrorString(e));
  }
  const size_t smem = sizeof(float2) * 2 * kSites * kStride + sizeof(double2) * kWarps * n_mom;
  dim3 grid((g.V3 + kSites - 1) / kSites, g.Nt);
  ProfScope prof("baryon_2pt", s);
#define QDPG_BARYON_LAUNCH(T, KIND)                                                                          \
  do {                                                                                                       \
    if (ksites) {                                                                                            \
      auto k = baryon_kernel<T, KIND, true>;                                                                 \
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
      k<<<grid, kWarps * 32, smem, s>>>(static_cast<const T*>(Su->data), static_cast<const T*>(Sd->data), g, B, \
                                        M, out_dev, ksites, Su->rec, Sd->rec, site_scale);                   \
    } else {                                                                                                 \
      auto k = baryon_kernel<T, KIND, false>;                                                                \
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
      k<<<grid, kWarps * 32, smem, s>>>(static_cast<const T*>(Su->data), static_cast<const T*>(Sd->data), g, B, \
                                        M, out_dev, ksites, Su->rec, Sd->rec, site_scale);                   \
    }                                                                                                        \
  } while (0)
  if (Su->prec == QDPG_BF16) {
    if (kind == 0) QDPG_BARYON_LAUNCH(__nv_bfloat162, 0);
    else QDPG_BARYON_LAUNCH(__nv_bfloat162, 1);
  } else if (Su->prec == QDPG_F16) {
    if (kind == 0) QDPG_BARYON_LAUNCH(__half2, 0);
    else QDPG_BARYON_LAUNCH(__half2, 1);
  } else {
    if (kind == 0) QDPG_BARYON_LAUNCH(float2, 0);
    else QDPG_BARYON_LAUNCH(float2, 1);
  }
#undef QDPG_BARYON_LAUNCH
  int rc = check_launch("baryon_2pt");
  if (tensor_proj) {
    std::vector<int> mom_flat(moms, moms + 3 * (size_t)n_mom);
    if (rc == QDPG_OK)
      rc = launch_momproj(g, ksites, 1, mom_flat.data(), n_mom, origin, out_dev, Su->rec, 2, Sd->rec, 1, s);
    dev_free(ksites, s);
  }
  return rc;
}

}  // namespace

extern "C" int qdpg_baryon_2pt(qdpg_field_t Su, qdpg_field_t Sd, int kind, int parity, const int* moms, int n_mom,
                               const int origin[4], double* out_dev, void* stream) {
  if (!out_dev) return fail(QDPG_ERR_ARG, "baryon_2pt: null argument");
  return baryon_common(Su, Sd, kind, parity, moms, n_mom, origin, out_dev, nullptr, stream);
}

extern "C" int qdpg_baryon_sites(qdpg_field_t Su, qdpg_field_t Sd, int kind, int parity, void* sites_dev,
                                 void* stream) {
  if (!sites_dev) return fail(QDPG_ERR_ARG, "baryon_sites: null argument");
  if (reinterpret_cast<uintptr_t>(sites_dev) % 8) return fail(QDPG_ERR_ARG, "baryon_sites: buffer not 8-byte aligned");
  static const int zero[3] = {0, 0, 0};
  return baryon_common(Su, Sd, kind, parity, zero, 1, nullptr, nullptr, static_cast<float2*>(sites_dev), stream);
}
