// Field setup kernels: canonical import/export, point source, shift.
//
// Source creation is the first stage of the paper's Chroma measurement
// (Sec. 5); shift is the nearest-neighbour primitive of QDP++ expressions
// (Sec. 1).  All kernels here are pure data movement.
#include <algorithm>
#include <type_traits>
#include <cuda_fp16.h>

#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {

namespace {

constexpr int kThreads = 256;
constexpr int kTileSites = 32;  // sites per tile of the propagator import (32 x 145 complex64 in shared memory)

inline int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 32;  // grid-stride beyond 32 CTAs per SM
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// ---- element conversion ------------------------------------------------------
__device__ __forceinline__ void store_elem(float2* p, double re, double im) {
  *p = make_float2(__double2float_rn(re), __double2float_rn(im));
}
__device__ __forceinline__ void store_elem(__nv_bfloat162* p, double re, double im) {
  __nv_bfloat162 v;
  v.x = __double2bfloat16(re);
  v.y = __double2bfloat16(im);
  *p = v;
}
__device__ __forceinline__ void store_elem(__half2* p, double re, double im) {
  *p = __halves2half2(__double2half(re), __double2half(im));
}
// From FP32 values: one rounding, the same as from the equal FP64 values,
// without FP64 arithmetic (slow on this GPU).
__device__ __forceinline__ void store_elem(float2* p, float re, float im) { *p = make_float2(re, im); }
__device__ __forceinline__ void store_elem(__nv_bfloat162* p, float re, float im) {
  *p = __floats2bfloat162_rn(re, im);
}
__device__ __forceinline__ void store_elem(__half2* p, float re, float im) { *p = __floats2half2_rn(re, im); }
__device__ __forceinline__ void load_elem(const __half2* p, double& re, double& im) {
  const float2 v = __half22float2(*p);
  re = v.x;
  im = v.y;
}
__device__ __forceinline__ void load_elem(const float2* p, double& re, double& im) {
  float2 v = *p;
  re = v.x;
  im = v.y;
}
__device__ __forceinline__ void load_elem(const __nv_bfloat162* p, double& re, double& im) {
  __nv_bfloat162 v = *p;
  re = __bfloat162float(v.x);
  im = __bfloat162float(v.y);
}

// Whole timeslices [t0, t0 + nt) of a field whose canonical data (in the
// buffer a kernel is given) starts at canonical site site0 and spans nsites
// sites per direction; the whole field is {0, Nt, 0, V}.  A chunk of fewer
// timeslices is contiguous in the canonical order when j_decay = 3.
struct Chunk {
  int t0, nt;
  long long site0, nsites;
};

// Canonical complex index of device component `comp` at canonical site `site`.
__device__ __forceinline__ long long canon_index(int kind, bool r12, int nc, long long V, long long site,
                                                 int comp) {
  if (kind == QDPG_GAUGE) {
    int per = r12 ? 6 : 9;
    int mu = comp / per, e = comp % per;  // rows 0,1 of a reconstruct-12 link keep entry a*3+b
    return ((long long)mu * V + site) * 9 + e;
  }
  return site * nc + comp;
}

template <typename Src, typename Dst>
__global__ void __launch_bounds__(kThreads) import_kernel(Dst* __restrict__ dst, const Src* __restrict__ src,
                                                          Geom g, int kind, bool r12, int nc, Chunk ck) {
  const long long total = (long long)ck.nt * nc * g.V3;
  Dst* d0 = dst + (long long)ck.t0 * nc * g.V3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int s3 = (int)(i % g.V3);
    long long r = i / g.V3;
    int comp = (int)(r % nc);
    int t = ck.t0 + (int)(r / nc);
    long long site = canon_site(g, t, s3) - ck.site0;
    int nc_canon = (kind == QDPG_GAUGE) ? 9 : nc;
    long long ci = canon_index(kind, r12, nc_canon, ck.nsites, site, comp);
    store_elem(d0 + i, (double)src[2 * ci], (double)src[2 * ci + 1]);
  }
}

// Thread per canonical complex entry; reconstructs row 2 of reconstruct-12 links.
template <typename Dev>
__global__ void __launch_bounds__(kThreads) export_kernel(double* __restrict__ out, const Dev* __restrict__ dev,
                                                          Geom g, int kind, bool r12, int nc,
                                                          const ScaleRecord* rec, Chunk ck) {
  const int e2 = rec ? rec->exp : 0;  // value = stored * 2^exp
  const int nc_canon = (kind == QDPG_GAUGE) ? 9 : nc;
  const long long nmu = (kind == QDPG_GAUGE) ? 4 : 1;
  const long long total = nmu * ck.nsites * nc_canon;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int e = (int)(i % nc_canon);
    long long r = i / nc_canon;
    long long site = ck.site0 + r % ck.nsites;
    int mu = (int)(r / ck.nsites);
    // canonical site -> (t, s3)
    int x[4];
    long long rr = site;
    for (int d = 0; d < 4; ++d) {
      x[d] = (int)(rr % g.L[d]);
      rr /= g.L[d];
    }
    int t = x[g.jd];
    int s3 = x[g.sd[0]] + g.sL[0] * (x[g.sd[1]] + g.sL[1] * x[g.sd[2]]);
    const Dev* base = dev + (long long)t * nc * g.V3 + s3;
    double re, im;
    if (kind == QDPG_GAUGE && r12) {
      int a = e / 3, b = e % 3;
      if (a < 2) {
        load_elem(base + (long long)(mu * 6 + e) * g.V3, re, im);
      } else {
        // row2 = (row0 x row1)^*
        int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
        double r0r[2], r0i[2], r1r[2], r1i[2];
        load_elem(base + (long long)(mu * 6 + b1) * g.V3, r0r[0], r0i[0]);
        load_elem(base + (long long)(mu * 6 + b2) * g.V3, r0r[1], r0i[1]);
        load_elem(base + (long long)(mu * 6 + 3 + b1) * g.V3, r1r[0], r1i[0]);
        load_elem(base + (long long)(mu * 6 + 3 + b2) * g.V3, r1r[1], r1i[1]);
        // c = r0[b1]*r1[b2] - r0[b2]*r1[b1]
        double cr = (r0r[0] * r1r[1] - r0i[0] * r1i[1]) - (r0r[1] * r1r[0] - r0i[1] * r1i[0]);
        double ci = (r0r[0] * r1i[1] + r0i[0] * r1r[1]) - (r0r[1] * r1i[0] + r0i[1] * r1r[0]);
        re = cr;
        im = -ci;
      }
    } else {
      int comp = (kind == QDPG_GAUGE) ? mu * 9 + e : e;
      load_elem(base + (long long)comp * g.V3, re, im);
    }
    out[2 * i] = ldexp(re, e2);
    out[2 * i + 1] = ldexp(im, e2);
  }
}

// Unit entries of a point source; the field was zeroed before.  Element
// (t, comp, s3) sits at t_off + comp*V3 with t_off = t*ncomp*V3 + s3.
template <typename Dev>
__global__ void point_kernel(Dev* __restrict__ f, long long t_off, int V3, int ncomp, int fermion_comp) {
  const int k = threadIdx.x;
  if (ncomp == 144) {
    if (k < 12) store_elem(f + t_off + (long long)(k * 13) * V3, 1.0, 0.0);  // comp (k,k) of the 12x12
  } else if (k == 0) {
    store_elem(f + t_off + (long long)fermion_comp * V3, 1.0, 0.0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) shift_kernel(T* __restrict__ dst, const T* __restrict__ src, Geom g,
                                                         int nc, int mu, int sign) {
  const long long total = g.V * nc;
  int k = -1;
  for (int d = 0; d < 3; ++d)
    if (g.sd[d] == mu) k = d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int s3 = (int)(i % g.V3);
    long long r = i / g.V3;
    int comp = (int)(r % nc);
    int t = (int)(r / nc);
    int t2 = t, s32 = s3;
    if (k < 0) {
      t2 = t + sign;
      t2 = t2 < 0 ? t2 + g.Nt : (t2 >= g.Nt ? t2 - g.Nt : t2);
    } else {
      int c[3];
      c[0] = s3 % g.sL[0];
      c[1] = (s3 / g.sL[0]) % g.sL[1];
      c[2] = s3 / (g.sL[0] * g.sL[1]);
      int v = c[k] + sign;
      c[k] = v < 0 ? v + g.sL[k] : (v >= g.sL[k] ? v - g.sL[k] : v);
      s32 = c[0] + g.sL[0] * (c[1] + g.sL[1] * c[2]);
    }
    dst[i] = src[((long long)t2 * nc + comp) * g.V3 + s32];
  }
}

// ---- float16 propagators: site-major layout with a power-of-two scale ---------
//
// The canonical component comp = (s*3 + c)*12 + s' * 3 + c' of device word
// i (decomposed as in f16_prop_index, qdpg_internal.h).
__device__ __forceinline__ void f16_word_decode(long long i, int V3, int& t, int& s3, int& comp) {
  const int w = (int)(i % 48);
  const long long r = i / 48;
  s3 = (int)(r % V3);
  const long long r2 = r / V3;
  const int vg = (int)(r2 % 3);
  t = (int)(r2 / 3);
  const int v = vg * 16 + w / 3, c = w % 3;
  const int s = v / 12, sp = v - 12 * s;
  comp = (s * 3 + c) * 12 + sp;
}

// Exponent e with m * 2^-e < 2^14 (0 for m = 0).
__device__ __forceinline__ int f16_exp_for(float m) {
  if (!(m > 0.f)) return 0;
  int ex;
  frexpf(m, &ex);  // m = f * 2^ex, f in [0.5, 1)
  return ex - 14;
}

template <typename Src>
__global__ void __launch_bounds__(kThreads) f16_max_kernel(const Src* __restrict__ src, long long n,
                                                           unsigned* __restrict__ out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<Src, float>::value)
      m = fmaxf(m, fabsf(src[i]));  // exact
    else
      m = fmaxf(m, __double2float_ru(fmax(fabs((double)src[i]), 0.0)));  // rounded up: still a bound
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

template <typename Src>
__global__ void __launch_bounds__(kThreads) f16_import_kernel(__half2* __restrict__ dst, const Src* __restrict__ src,
                                                              Geom g, ScaleRecord* rec, Chunk ck) {
  const float m = __uint_as_float(rec->tmpmax);
  const int e = f16_exp_for(m);
  const long long total = (long long)ck.nt * 144 * g.V3;
  const long long w0 = (long long)ck.t0 * 144 * g.V3;  // a timeslice's words are contiguous
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int t, s3, comp;
    f16_word_decode(w0 + i, g.V3, t, s3, comp);
    const long long ci = (canon_site(g, t, s3) - ck.site0) * 144 + comp;
    store_elem(dst + w0 + i, ldexp((double)src[2 * ci], -e), ldexp((double)src[2 * ci + 1], -e));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    rec->exp = e;
    rec->maxabs = ldexpf(m, -e) * (1.f + 1.f / 1024.f);  // bound after rounding to float16
  }
}

// Propagators and fermions (NC = 144 or 12 complex entries per site), by
// tiles of TS consecutive device sites of one timeslice: a block reads the
// tile's canonical entries (each site's NC numbers are contiguous) with
// coalesced loads into shared memory, rows padded by one entry so that
// column reads spread over the banks, and writes them in the device layout
// with coalesced stores: component planes for F32/BF16, site-major vector
// groups scaled by 2^-e for float16 (F16: e from the whole field's maximum,
// as f16_import_kernel).
template <typename Src, typename Dst, int NC, int TS, bool F16>
__global__ void __launch_bounds__(kThreads) import_tile_kernel(Dst* __restrict__ dst, const Src* __restrict__ src,
                                                               Geom g, Chunk ck, ScaleRecord* rec) {
  __shared__ Src sm[TS][NC + 1][2];
  __shared__ long long sbase[TS];
  const int ntile = (g.V3 + TS - 1) / TS;
  const long long ntot = (long long)ck.nt * ntile;
  int e = 0;
  float m = 0.f;
  if constexpr (F16) {
    m = __uint_as_float(rec->tmpmax);
    e = f16_exp_for(m);
  }
  for (long long tile = blockIdx.x; tile < ntot; tile += gridDim.x) {
    const int t = ck.t0 + (int)(tile / ntile);
    const int s0 = (int)(tile % ntile) * TS;
    const int ns = min(TS, g.V3 - s0);
    if (threadIdx.x < ns) sbase[threadIdx.x] = (canon_site(g, t, s0 + threadIdx.x) - ck.site0) * NC;
    __syncthreads();
    for (int i = threadIdx.x; i < ns * NC; i += kThreads) {
      const int si = i / NC, c = i - si * NC;
      const long long ci = sbase[si] + c;
      sm[si][c][0] = src[2 * ci];
      sm[si][c][1] = src[2 * ci + 1];
    }
    __syncthreads();
    if constexpr (!F16) {
      for (int i = threadIdx.x; i < NC * TS; i += kThreads) {
        const int c = i / TS, si = i - c * TS;
        if (si < ns) store_elem(dst + ((long long)t * NC + c) * g.V3 + s0 + si, sm[si][c][0], sm[si][c][1]);
      }
    } else {
      // word ((t*3 + vg)*V3 + s3)*48 + w, w = (v mod 16)*3 + colour (qdpg.h)
      for (int i = threadIdx.x; i < 3 * TS * 48; i += kThreads) {
        const int vg = i / (TS * 48), r = i - vg * (TS * 48), si = r / 48, w = r - si * 48;
        if (si >= ns) continue;
        const int v = vg * 16 + w / 3, cc = w % 3;
        const int comp = ((v / 12) * 3 + cc) * 12 + v % 12;
        Dst* o = dst + (((long long)t * 3 + vg) * g.V3 + s0 + si) * 48 + w;
        if constexpr (std::is_same<Src, float>::value)
          store_elem(o, ldexpf(sm[si][comp][0], -e), ldexpf(sm[si][comp][1], -e));  // exact scaling, one rounding
        else
          store_elem(o, ldexp(sm[si][comp][0], -e), ldexp(sm[si][comp][1], -e));
      }
    }
    __syncthreads();
  }
  if constexpr (F16) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      rec->exp = e;
      rec->maxabs = ldexpf(m, -e) * (1.f + 1.f / 1024.f);  // bound after rounding to float16
    }
  }
}

__global__ void __launch_bounds__(kThreads) f16_export_kernel(double* __restrict__ out, const __half2* __restrict__ dev,
                                                              Geom g, const ScaleRecord* rec, Chunk ck) {
  const int e = rec->exp;
  const long long total = (long long)ck.nt * 144 * g.V3;
  const long long w0 = (long long)ck.t0 * 144 * g.V3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int t, s3, comp;
    f16_word_decode(w0 + i, g.V3, t, s3, comp);
    const long long ci = (canon_site(g, t, s3) - ck.site0) * 144 + comp;
    double re, im;
    load_elem(dev + w0 + i, re, im);
    out[2 * ci] = ldexp(re, e);
    out[2 * ci + 1] = ldexp(im, e);
  }
}

// Unit entries of a point source at (t, s3); the data was zeroed before.
__global__ void f16_point_kernel(__half2* __restrict__ f, int V3, int t, int s3, ScaleRecord* rec) {
  const int k = threadIdx.x;
  if (k < 12) f[f16_prop_index(V3, t, k * 13, s3)] = __halves2half2(__float2half(1.f), __float2half(0.f));
  if (k == 0) {
    rec->exp = 0;
    rec->maxabs = 1.f;
  }
}

// dst(x) = src(x + sign mu_hat) on whole 48-word site blocks; copies the scale.
__global__ void __launch_bounds__(kThreads) f16_shift_kernel(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src,
                                                             Geom g, int mu, int sign, ScaleRecord* drec,
                                                             const ScaleRecord* srec) {
  const long long total = g.V * 144;
  int k = -1;
  for (int d = 0; d < 3; ++d)
    if (g.sd[d] == mu) k = d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(i % 48);
    const long long r = i / 48;
    const int s3 = (int)(r % g.V3);
    const long long r2 = r / g.V3;
    const int vg = (int)(r2 % 3);
    const int t = (int)(r2 / 3);
    int t2 = t, s32 = s3;
    if (k < 0) {
      t2 = t + sign;
      t2 = t2 < 0 ? t2 + g.Nt : (t2 >= g.Nt ? t2 - g.Nt : t2);
    } else {
      int c[3];
      c[0] = s3 % g.sL[0];
      c[1] = (s3 / g.sL[0]) % g.sL[1];
      c[2] = s3 / (g.sL[0] * g.sL[1]);
      const int v = c[k] + sign;
      c[k] = v < 0 ? v + g.sL[k] : (v >= g.sL[k] ? v - g.sL[k] : v);
      s32 = c[0] + g.sL[0] * (c[1] + g.sL[1] * c[2]);
    }
    dst[i] = src[(((long long)t2 * 3 + vg) * g.V3 + s32) * 48 + w];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    drec->exp = srec->exp;
    drec->maxabs = srec->maxabs;
  }
}

}  // namespace

}  // namespace qdpg

namespace qdpg {
namespace {

// Conversion of one chunk of canonical data (device memory) into dst's
// layout.  F16 propagators: pass 0 folds the chunk's largest magnitude into
// the scale record's scratch, pass 1 converts with the scale that the
// whole field's maximum fixes.
int import_chunk(qdpg_field_t dst, const void* canon_dev, int canon, const Chunk& ck, int f16_pass, cudaStream_t s) {
  const long long total = (long long)ck.nt * dst->ncomp * dst->g.V3;
  const bool r12 = is_r12(dst->prec);
  const int grid = grid_for(total);
  const bool f64 = canon == QDPG_CANON_F64;
  ProfScope prof("field_import", s);
  if (is_f16_prop(dst)) {
    auto* d = static_cast<__half2*>(dst->data);
    const long long nreal = 2 * ck.nsites * 144;
    if (f16_pass == 0) {
      if (f64)
        f16_max_kernel<<<grid_for(nreal), kThreads, 0, s>>>(static_cast<const double*>(canon_dev), nreal,
                                                            &dst->rec->tmpmax);
      else
        f16_max_kernel<<<grid_for(nreal), kThreads, 0, s>>>(static_cast<const float*>(canon_dev), nreal,
                                                            &dst->rec->tmpmax);
    } else {
      const long long tiles = (long long)ck.nt * ((dst->g.V3 + kTileSites - 1) / kTileSites);
      const int tgrid = (int)std::min<long long>(tiles, 152LL * 8);
      if (f64)
        import_tile_kernel<double, __half2, 144, kTileSites / 2, true>
            <<<tgrid, kThreads, 0, s>>>(d, static_cast<const double*>(canon_dev), dst->g, ck, dst->rec);
      else
        import_tile_kernel<float, __half2, 144, kTileSites, true>
            <<<tgrid, kThreads, 0, s>>>(d, static_cast<const float*>(canon_dev), dst->g, ck, dst->rec);
    }
    return check_launch("field_import");
  }
  if (dst->kind == QDPG_PROPAGATOR || dst->kind == QDPG_FERMION) {
    // tiles of consecutive sites through shared memory (16 sites for FP64
    // canonical data, whose rows are twice as long)
    const int TSf = dst->kind == QDPG_PROPAGATOR ? kTileSites : 4 * kTileSites;
    const long long tiles = (long long)ck.nt * ((dst->g.V3 + TSf - 1) / TSf);
    const int tgrid = (int)std::min<long long>(f64 ? 2 * tiles : tiles, 152LL * 8);
#define QDPG_TILE(DT, NC, TS)                                                                                    \
  do {                                                                                                           \
    auto* d = static_cast<DT*>(dst->data);                                                                       \
    if (f64)                                                                                                     \
      import_tile_kernel<double, DT, NC, (TS) / 2, false>                                                        \
          <<<tgrid, kThreads, 0, s>>>(d, static_cast<const double*>(canon_dev), dst->g, ck, nullptr);           \
    else                                                                                                         \
      import_tile_kernel<float, DT, NC, TS, false>                                                               \
          <<<tgrid, kThreads, 0, s>>>(d, static_cast<const float*>(canon_dev), dst->g, ck, nullptr);            \
  } while (0)
    const bool prop = dst->kind == QDPG_PROPAGATOR;
    if (is_bf16(dst->prec)) {
      if (prop) QDPG_TILE(__nv_bfloat162, 144, kTileSites);
      else QDPG_TILE(__nv_bfloat162, 12, 4 * kTileSites);
    } else {
      if (prop) QDPG_TILE(float2, 144, kTileSites);
      else QDPG_TILE(float2, 12, 4 * kTileSites);
    }
#undef QDPG_TILE
    return check_launch("field_import");
  }
#define QDPG_IMPORT(DT)                                                                                          \
  do {                                                                                                           \
    auto* d = static_cast<DT*>(dst->data);                                                                       \
    if (f64)                                                                                                     \
      import_kernel<double><<<grid, kThreads, 0, s>>>(d, static_cast<const double*>(canon_dev), dst->g, dst->kind, \
                                                      r12, dst->ncomp, ck);                                      \
    else                                                                                                         \
      import_kernel<float><<<grid, kThreads, 0, s>>>(d, static_cast<const float*>(canon_dev), dst->g, dst->kind,   \
                                                     r12, dst->ncomp, ck);                                       \
  } while (0)
  if (is_f16(dst->prec))
    QDPG_IMPORT(__half2);
  else if (is_bf16(dst->prec))
    QDPG_IMPORT(__nv_bfloat162);
  else
    QDPG_IMPORT(float2);
#undef QDPG_IMPORT
  return check_launch("field_import");
}

// Before the first chunk: clear the F16 maximum.  After the last: imported
// F32/BF16 values are unscaled, exp = 0 (F16 import kernels set their exp).
int import_begin(qdpg_field_t dst, cudaStream_t s) {
  if (!is_f16_prop(dst)) return QDPG_OK;
  const cudaError_t e = cudaMemsetAsync(&dst->rec->tmpmax, 0, sizeof(unsigned), s);
  return e == cudaSuccess ? QDPG_OK : fail(QDPG_ERR_CUDA, "field_import: memset: %s", cudaGetErrorString(e));
}
int import_end(qdpg_field_t dst, cudaStream_t s) {
  if (!dst->rec || is_f16_prop(dst)) return QDPG_OK;
  const cudaError_t e = cudaMemsetAsync(dst->rec, 0, 2 * sizeof(int), s);
  return e == cudaSuccess ? QDPG_OK : fail(QDPG_ERR_CUDA, "field_import: scale reset: %s", cudaGetErrorString(e));
}

int export_chunk(qdpg_field_t src, double* canon_dev, const Chunk& ck, cudaStream_t s) {
  const long long total = (src->kind == QDPG_GAUGE ? 4 * 9 : src->ncomp) * ck.nsites;
  const int grid = grid_for(total);
  const bool r12 = is_r12(src->prec);
  ProfScope prof("field_export", s);
  if (is_f16_prop(src))
    f16_export_kernel<<<grid, kThreads, 0, s>>>(canon_dev, static_cast<const __half2*>(src->data), src->g, src->rec,
                                                ck);
  else if (is_f16(src->prec))
    export_kernel<<<grid, kThreads, 0, s>>>(canon_dev, static_cast<const __half2*>(src->data), src->g, src->kind,
                                            r12, src->ncomp, src->rec, ck);
  else if (is_bf16(src->prec))
    export_kernel<<<grid, kThreads, 0, s>>>(canon_dev, static_cast<const __nv_bfloat162*>(src->data), src->g,
                                            src->kind, r12, src->ncomp, src->rec, ck);
  else
    export_kernel<<<grid, kThreads, 0, s>>>(canon_dev, static_cast<const float2*>(src->data), src->g, src->kind,
                                            r12, src->ncomp, src->rec, ck);
  return check_launch("field_export");
}

Chunk whole_field(const Geom& g) { return Chunk{0, g.Nt, 0, g.V}; }

// Complex numbers per site in the canonical layout (all four links of a gauge field).
long long canon_per_site(const qdpg_field* f) { return f->kind == QDPG_GAUGE ? 36 : f->ncomp; }

// Host transfers: chunks of whole timeslices of at most 256 MiB of
// canonical data (or the QDPG_DEBUG_STAGE_BYTES setting) when j_decay = 3,
// else the whole field.
int chunk_timeslices(const qdpg_field* f, size_t csize) {
  if (f->g.jd != 3) return f->g.Nt;
  const size_t per_t = (size_t)f->g.V3 * canon_per_site(f) * csize;
  const long long limit = debug_stage_bytes() > 0 ? debug_stage_bytes() : (256LL << 20);
  long long n = (long long)(limit / (long long)per_t);
  if (n < 1) n = 1;
  if (n > f->g.Nt) n = f->g.Nt;
  return (int)n;
}
Chunk chunk_at(const qdpg_field* f, int t0, int nt) {
  if (f->g.jd != 3) return whole_field(f->g);
  return Chunk{t0, nt, (long long)t0 * f->g.V3, (long long)nt * f->g.V3};
}

// Copy a chunk between the host canonical buffer and the staging buffer
// (one run per link direction for a gauge field).
int copy_chunk(const qdpg_field* f, void* stage, const void* host, const Chunk& ck, size_t csize, bool to_device,
               cudaStream_t s) {
  const int nmu = f->kind == QDPG_GAUGE ? 4 : 1;
  const long long per = f->kind == QDPG_GAUGE ? 9 : f->ncomp;  // complex numbers per site and direction
  const size_t run = (size_t)ck.nsites * per * csize;
  for (int mu = 0; mu < nmu; ++mu) {
    const size_t hoff = ((size_t)mu * f->g.V + ck.site0) * per * csize;
    char* dptr = static_cast<char*>(stage) + mu * run;
    const char* hptr = static_cast<const char*>(host) + hoff;
    const cudaError_t e = to_device ? cudaMemcpyAsync(dptr, hptr, run, cudaMemcpyHostToDevice, s)
                                    : cudaMemcpyAsync(const_cast<char*>(hptr), dptr, run, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "field host copy: %s", cudaGetErrorString(e));
  }
  return QDPG_OK;
}

}  // namespace
}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_field_import(qdpg_field_t dst, const void* canon_dev, int canon, void* stream) {
  if (!dst || !canon_dev) return fail(QDPG_ERR_ARG, "field_import: null argument");
  if (canon != QDPG_CANON_F64 && canon != QDPG_CANON_F32)
    return fail(QDPG_ERR_DTYPE, "field_import: canonical type %d unknown", canon);
  cudaStream_t s = as_stream(stream);
  const Chunk all = whole_field(dst->g);
  int rc = import_begin(dst, s);
  if (rc == QDPG_OK && is_f16_prop(dst)) rc = import_chunk(dst, canon_dev, canon, all, 0, s);
  if (rc == QDPG_OK) rc = import_chunk(dst, canon_dev, canon, all, 1, s);
  if (rc == QDPG_OK) rc = import_end(dst, s);
  return rc;
}

int qdpg_field_export(qdpg_field_t src, double* canon_dev, void* stream) {
  if (!src || !canon_dev) return fail(QDPG_ERR_ARG, "field_export: null argument");
  return export_chunk(src, canon_dev, whole_field(src->g), as_stream(stream));
}

int qdpg_field_import_host(qdpg_field_t dst, const void* host_canon, int canon, void* stream) {
  if (!dst || !host_canon) return fail(QDPG_ERR_ARG, "field_import_host: null argument");
  if (canon != QDPG_CANON_F64 && canon != QDPG_CANON_F32)
    return fail(QDPG_ERR_DTYPE, "field_import_host: canonical type %d unknown", canon);
  cudaStream_t s = as_stream(stream);
  const size_t csize = canon == QDPG_CANON_F64 ? 16 : 8;
  const int ntc = chunk_timeslices(dst, csize);
  void* stage = nullptr;
  int rc = dev_alloc(&stage, (size_t)ntc * dst->g.V3 * canon_per_site(dst) * csize, s, "field_import_host staging");
  if (rc != QDPG_OK) return rc;
  rc = import_begin(dst, s);
  for (int pass = is_f16_prop(dst) ? 0 : 1; pass <= 1 && rc == QDPG_OK; ++pass)
    for (int t0 = 0; t0 < dst->g.Nt && rc == QDPG_OK; t0 += ntc) {
      const Chunk ck = chunk_at(dst, t0, ntc < dst->g.Nt - t0 ? ntc : dst->g.Nt - t0);
      rc = copy_chunk(dst, stage, host_canon, ck, csize, true, s);
      if (rc == QDPG_OK) rc = import_chunk(dst, stage, canon, ck, pass, s);
      if (dst->g.jd != 3) break;  // one chunk: the whole field
    }
  if (rc == QDPG_OK) rc = import_end(dst, s);
  dev_free(stage, s);
  return rc;
}

int qdpg_field_export_host(qdpg_field_t src, double* host_canon, void* stream) {
  if (!src || !host_canon) return fail(QDPG_ERR_ARG, "field_export_host: null argument");
  cudaStream_t s = as_stream(stream);
  const size_t csize = 16;
  const int ntc = chunk_timeslices(src, csize);
  void* stage = nullptr;
  int rc = dev_alloc(&stage, (size_t)ntc * src->g.V3 * canon_per_site(src) * csize, s, "field_export_host staging");
  if (rc != QDPG_OK) return rc;
  for (int t0 = 0; t0 < src->g.Nt && rc == QDPG_OK; t0 += ntc) {
    const Chunk ck = chunk_at(src, t0, ntc < src->g.Nt - t0 ? ntc : src->g.Nt - t0);
    rc = export_chunk(src, static_cast<double*>(stage), ck, s);
    if (rc == QDPG_OK) rc = copy_chunk(src, stage, host_canon, ck, csize, false, s);
    if (src->g.jd != 3) break;
  }
  dev_free(stage, s);
  return rc;
}

int qdpg_point_source(qdpg_field_t f, const int x0[4], int spin_color, void* stream) {
  if (!f || !x0) return fail(QDPG_ERR_ARG, "point_source: null argument");
  if (f->kind != QDPG_PROPAGATOR && f->kind != QDPG_FERMION)
    return fail(QDPG_ERR_SHAPE, "point_source: field must be a propagator or fermion");
  if (f->prec != QDPG_F32 && f->prec != QDPG_BF16 && f->prec != QDPG_F16)
    return fail(QDPG_ERR_DTYPE, "point_source: storage must be F32, BF16 or F16");
  for (int mu = 0; mu < 4; ++mu)
    if (x0[mu] < 0 || x0[mu] >= f->g.L[mu]) return fail(QDPG_ERR_ARG, "point_source: x0[%d] outside lattice", mu);
  if (f->kind == QDPG_FERMION && (spin_color < 0 || spin_color > 11))
    return fail(QDPG_ERR_ARG, "point_source: spin_color %d outside 0..11", spin_color);
  cudaStream_t s = as_stream(stream);
  const Geom& g = f->g;
  if (is_f16_prop(f)) {
    cudaError_t e = cudaMemsetAsync(f->data, 0, f16_data_bytes(g.V), s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "point_source: memset: %s", cudaGetErrorString(e));
    const int t = x0[g.jd];
    const int s3 = x0[g.sd[0]] + g.sL[0] * (x0[g.sd[1]] + g.sL[1] * x0[g.sd[2]]);
    ProfScope prof("point_source", s);
    f16_point_kernel<<<1, 32, 0, s>>>(static_cast<__half2*>(f->data), g.V3, t, s3, f->rec);
    return check_launch("point_source");
  }
  size_t bytes = (size_t)g.V * f->ncomp * f->esize;
  cudaError_t e = cudaMemsetAsync(f->data, 0, bytes, s);
  if (e == cudaSuccess && f->rec) e = cudaMemsetAsync(f->rec, 0, 2 * sizeof(int), s);  // exp = 0
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "point_source: memset: %s", cudaGetErrorString(e));
  const int t = x0[g.jd];
  const int s3 = x0[g.sd[0]] + g.sL[0] * (x0[g.sd[1]] + g.sL[1] * x0[g.sd[2]]);
  const long long t_off = (long long)t * f->ncomp * g.V3 + s3;
  const int fc = (f->kind == QDPG_FERMION) ? spin_color : 0;
  ProfScope prof("point_source", s);
  if (f->prec == QDPG_BF16)
    point_kernel<<<1, 32, 0, s>>>(static_cast<__nv_bfloat162*>(f->data), t_off, g.V3, f->ncomp, fc);
  else
    point_kernel<<<1, 32, 0, s>>>(static_cast<float2*>(f->data), t_off, g.V3, f->ncomp, fc);
  return check_launch("point_source");
}

int qdpg_shift(qdpg_field_t dst, qdpg_field_t src, int sign, int mu, void* stream) {
  if (!dst || !src) return fail(QDPG_ERR_ARG, "shift: null argument");
  if (sign != 1 && sign != -1) return fail(QDPG_ERR_ARG, "shift: sign must be +1 or -1");
  if (mu < 0 || mu > 3) return fail(QDPG_ERR_ARG, "shift: mu %d outside 0..3", mu);
  if (dst->kind != src->kind || dst->prec != src->prec) return fail(QDPG_ERR_SHAPE, "shift: fields differ in kind/precision");
  for (int d = 0; d < 4; ++d)
    if (dst->g.L[d] != src->g.L[d] || dst->g.jd != src->g.jd) return fail(QDPG_ERR_SHAPE, "shift: lattices differ");
  if (dst->data == src->data) return fail(QDPG_ERR_ARG, "shift: dst and src alias");
  cudaStream_t s = as_stream(stream);
  const long long total = src->g.V * src->ncomp;
  const int grid = grid_for(total);
  ProfScope prof("shift", s);
  if (is_f16_prop(src))
    f16_shift_kernel<<<grid, kThreads, 0, s>>>(static_cast<uint32_t*>(dst->data),
                                               static_cast<const uint32_t*>(src->data), src->g, mu, sign, dst->rec,
                                               src->rec);
  else if (src->esize == 8)
    shift_kernel<<<grid, kThreads, 0, s>>>(static_cast<uint2*>(dst->data), static_cast<const uint2*>(src->data),
                                           src->g, src->ncomp, mu, sign);
  else
    shift_kernel<<<grid, kThreads, 0, s>>>(static_cast<uint32_t*>(dst->data),
                                           static_cast<const uint32_t*>(src->data), src->g, src->ncomp, mu, sign);
  const int rc = check_launch("shift");
  if (rc == QDPG_OK && dst->rec && !is_f16_prop(src)) {  // the float16 kernel copies its scale itself
    cudaError_t e = cudaMemcpyAsync(dst->rec, src->rec, 2 * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "shift: scale copy: %s", cudaGetErrorString(e));
  }
  return rc;
}

}  // extern "C"
