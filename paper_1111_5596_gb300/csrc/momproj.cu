// Momentum projection of site correlators on the tensor cores (the paper's
// HAD stage, Sec. 5, projected to integer momenta):
//
//   out[chan][m][t] = sum_x sites[chan][t][x] exp(-i p_m.(x - x0)),
//
// a complex GEMM (rows = chan*Nt + t) x (sites) x (momenta).  Written in real
// arithmetic as C[row][n] = sum_k A[row][k] B[k][n] with k = (site, re/im) and
// n = (momentum, re/im):
//   B[2x][2m] = cos,  B[2x+1][2m] = sin,  B[2x][2m+1] = -sin,  B[2x+1][2m+1] = cos
// for exp(-i theta) = cos - i sin, so that C[row][2m] = Re and C[row][2m+1] = Im.
//
// Each CTA owns 128 rows and a range of sites.  It stages 32 sites at a time
// in shared memory in the tensor cores' K-major core-matrix layout (8 rows x
// 16 bytes per core matrix), the phases generated on the fly, and one thread
// issues tcgen05.mma (kind::tf32, M = 128, N = 2*n_mom padded to 16) into a
// TMEM accumulator.  TF32 keeps 10 mantissa bits, so every operand is split
// into hi + lo parts and three products hi*hi + hi*lo + lo*hi are
// accumulated (relative error ~2^-21 per product).  The CTA's FP32 partial
// sum over its sites is read back with tcgen05.ld and added to the FP64
// output with atomics (FP64 only for the sums across CTAs).
#include <algorithm>

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {

namespace {

constexpr int kM = 128;            // rows per CTA (tensor-core M)
constexpr int kChunk = 32;         // sites per staged chunk
constexpr int kKt = 2 * kChunk;    // real K per chunk
constexpr int kMaxMomP = 64;       // N = 2*n_mom <= 128
constexpr int kTmemCols = 128;
constexpr int kMaxAccSites = 256;  // sites summed in one FP32 tensor-core accumulator

struct ProjArgs {
  const ScaleRecord* ra;  // optional field scales: the sums are multiplied by
  const ScaleRecord* rb;  // 2^(ca * ra->exp + cb * rb->exp) (null: 2^0)
  int ca, cb;
  int rows;           // n_chan * Nt
  int Nt, V3, nmom, npad, sites_per_cta;
  int sL[3];
  int origin[3];
  int k[kMaxMomP][3];
};

// byte offset of element (r, k) of a K-major tile with kKt columns
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (kKt / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  lo = v - hi;
}

__device__ __forceinline__ void put(unsigned char* hi_base, unsigned char* lo_base, int r, int k, float v) {
  float h, l;
  split_tf32(v, h, l);
  const uint32_t o = core_off(r, k);
  *reinterpret_cast<float*>(hi_base + o) = h;
  *reinterpret_cast<float*>(lo_base + o) = l;
}

__global__ void __launch_bounds__(128, 1) momproj_kernel(const float2* __restrict__ sites, ProjArgs P,
                                                         double* __restrict__ out, unsigned int* status,
                                                         long long timeout_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Ahi = smem;
  unsigned char* Alo = Ahi + kM * kKt * 4;
  unsigned char* Bhi = Alo + kM * kKt * 4;
  unsigned char* Blo = Bhi + P.npad * kKt * 4;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Blo + P.npad * kKt * 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kM;
  const int xb = blockIdx.y * P.sites_per_cta;
  const int xe = min(P.V3, xb + P.sites_per_cta);
  const uint32_t bar_a = ptx::smem_addr(bar);

  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(tslot), kTmemCols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    ptx::mbar_init(bar_a, 1);
    ptx::fence_mbar_init();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = ptx::idesc_tf32(kM, P.npad);

  uint32_t phase = 0;
  bool issued = false, ok = true;
  for (int x0 = xb; x0 < xe && ok; x0 += kChunk) {
    // A: 128 rows x 32 sites (complex) -> real K = 64
    for (int e = tid; e < kM * kChunk; e += blockDim.x) {
      const int r = e / kChunk, j = e % kChunk;
      const int row = row0 + r, x = x0 + j;
      float2 v = make_float2(0.f, 0.f);
      if (row < P.rows && x < xe) v = __ldg(sites + (size_t)row * P.V3 + x);
      put(Ahi, Alo, r, 2 * j, v.x);
      put(Ahi, Alo, r, 2 * j + 1, v.y);
    }
    // B: npad rows (2 per momentum) x real K = 64
    for (int e = tid; e < (P.npad / 2) * kChunk; e += blockDim.x) {
      const int m = e / kChunk, j = e % kChunk;
      const int x = x0 + j;
      float cs = 0.f, sn = 0.f;
      if (m < P.nmom && x < xe) {
        const int c0 = x % P.sL[0], c1 = (x / P.sL[0]) % P.sL[1], c2 = x / (P.sL[0] * P.sL[1]);
        long long num = (long long)P.k[m][0] * (((c0 - P.origin[0]) % P.sL[0] + P.sL[0]) % P.sL[0]) * (P.V3 / P.sL[0]) +
                        (long long)P.k[m][1] * (((c1 - P.origin[1]) % P.sL[1] + P.sL[1]) % P.sL[1]) * (P.V3 / P.sL[1]) +
                        (long long)P.k[m][2] * (((c2 - P.origin[2]) % P.sL[2] + P.sL[2]) % P.sL[2]) * (P.V3 / P.sL[2]);
        num %= P.V3;
        if (num < 0) num += P.V3;
        sincospif(2.0f * (float)num / (float)P.V3, &sn, &cs);
      }
      put(Bhi, Blo, 2 * m, 2 * j, cs);
      put(Bhi, Blo, 2 * m, 2 * j + 1, sn);
      put(Bhi, Blo, 2 * m + 1, 2 * j, -sn);
      put(Bhi, Blo, 2 * m + 1, 2 * j + 1, cs);
    }
    ptx::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      ptx::tc_fence_after();
      const uint32_t ah = ptx::smem_addr(Ahi), al = ptx::smem_addr(Alo);
      const uint32_t bh = ptx::smem_addr(Bhi), bl = ptx::smem_addr(Blo);
      const uint32_t sbo_a = kKt * 32, sbo_b = kKt * 32;
#pragma unroll 1
      for (int s = 0; s < kKt / 8; ++s) {
        const uint32_t off = s * 256;  // two core matrices along K per instruction
        const uint64_t dah = ptx::smem_desc_noswizzle(ah + off, 128, sbo_a);
        const uint64_t dal = ptx::smem_desc_noswizzle(al + off, 128, sbo_a);
        const uint64_t dbh = ptx::smem_desc_noswizzle(bh + off, 128, sbo_b);
        const uint64_t dbl = ptx::smem_desc_noswizzle(bl + off, 128, sbo_b);
        ptx::mma_tf32(tmem, dah, dbh, idesc, issued ? 1u : 0u);
        issued = true;
        ptx::mma_tf32(tmem, dah, dbl, idesc, 1u);
        ptx::mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      ptx::mma_commit(bar_a);
    }
    issued = true;
    // the staged operands are overwritten only after the tensor cores read them
    const bool done = ptx::mbar_wait_bounded(bar_a, phase, timeout_ns);
    phase ^= 1;
    ok = __syncthreads_and(done ? 1 : 0) != 0;
    ptx::tc_fence_after();
  }

  if (!ok) {
    if (tid == 0) atomicOr(status, kStatusFullWait);
  } else if (issued) {
    // epilogue: warp w owns TMEM lanes (rows) 32w..32w+31
    const int row = row0 + warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    const double scale = ldexp(1.0, (P.ra ? P.ca * P.ra->exp : 0) + (P.rb ? P.cb * P.rb->exp : 0));
    for (int c0 = 0; c0 < P.npad; c0 += 16) {
      float v[16];
      ptx::tmem_ld16(taddr + c0, v);
      if (row < P.rows) {
        const int chan = row / P.Nt, t = row % P.Nt;
#pragma unroll
        for (int i = 0; i < 16; i += 2) {
          const int m = (c0 + i) / 2;
          if (m < P.nmom) {
            const long long o = ((long long)chan * P.nmom + m) * P.Nt + t;
            atomicAdd(out + 2 * o, (double)v[i] * scale);
            atomicAdd(out + 2 * o + 1, (double)v[i + 1] * scale);
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

}  // namespace qdpg

using namespace qdpg;

namespace qdpg {

int launch_momproj(const Geom& g, const void* sites_dev, int n_chan, const int* moms, int n_mom, const int origin[4],
                   double* out_dev, const ScaleRecord* ra, int ca, const ScaleRecord* rb, int cb, cudaStream_t s) {
  if (n_chan < 1) return fail(QDPG_ERR_ARG, "momentum_project: n_chan %d < 1", n_chan);
  if (n_mom < 1 || n_mom > kMaxMomP) return fail(QDPG_ERR_ARG, "momentum_project: n_mom %d outside 1..%d", n_mom, kMaxMomP);
  if (reinterpret_cast<uintptr_t>(sites_dev) % 8) return fail(QDPG_ERR_ARG, "momentum_project: sites not 8-byte aligned");
  const long long rows = (long long)n_chan * g.Nt;
  if (rows > (1LL << 30)) return fail(QDPG_ERR_ARG, "momentum_project: too many rows");
  unsigned int* status = device_status_word();
  if (!status) return fail(QDPG_ERR_CUDA, "momentum_project: no status word");
  ProjArgs P{};
  P.ra = ra;
  P.rb = rb;
  P.ca = ca;
  P.cb = cb;
  P.rows = (int)rows;
  P.Nt = g.Nt;
  P.V3 = g.V3;
  P.nmom = n_mom;
  P.npad = ((2 * n_mom + 15) / 16) * 16;
  for (int k = 0; k < 3; ++k) {
    P.sL[k] = g.sL[k];
    P.origin[k] = origin ? origin[g.sd[k]] : 0;
  }
  for (int m = 0; m < n_mom; ++m)
    for (int k = 0; k < 3; ++k) P.k[m][k] = moms[3 * m + k];
  const int row_tiles = (int)((rows + kM - 1) / kM);
  // split the sites so that about two waves of CTAs run; at least 32 sites
  // each, and at most kMaxAccSites: the tensor-core accumulator is FP32, so
  // its depth bounds the rounding error; longer sums go through the FP64
  // atomics across CTAs
  int nsplit = std::max(1, std::min((g.V3 + kChunk - 1) / kChunk, (2 * 152 + row_tiles - 1) / row_tiles));
  nsplit = std::max(nsplit, (g.V3 + kMaxAccSites - 1) / kMaxAccSites);
  P.sites_per_cta = ((g.V3 + nsplit - 1) / nsplit + kChunk - 1) / kChunk * kChunk;
  nsplit = (g.V3 + P.sites_per_cta - 1) / P.sites_per_cta;
  const size_t smem = (size_t)2 * kM * kKt * 4 + (size_t)2 * P.npad * kKt * 4 + 16;

  cudaError_t e = cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * (size_t)rows * n_mom, s);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "momentum_project: memset: %s", cudaGetErrorString(e));
  e = cudaFuncSetAttribute(momproj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "momentum_project: smem attribute: %s", cudaGetErrorString(e));
  dim3 grid(row_tiles, nsplit);
  ProfScope prof("momentum_project", s);
  momproj_kernel<<<grid, 128, smem, s>>>(static_cast<const float2*>(sites_dev), P, out_dev, status,
                                         wait_timeout_ns());
  return check_launch("momentum_project");
}

}  // namespace qdpg

extern "C" int qdpg_momentum_project(qdpg_lattice_t lat, const void* sites_dev, int n_chan, const int* moms,
                                     int n_mom, const int origin[4], double* out_dev, void* stream) {
  if (!lat || !sites_dev || !moms || !out_dev) return fail(QDPG_ERR_ARG, "momentum_project: null argument");
  return launch_momproj(lat->g, sites_dev, n_chan, moms, n_mom, origin, out_dev, nullptr, 0, nullptr, 0,
                        as_stream(stream));
}
