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
// A CTA owns 128 rows and at most kMaxCtaSites sites, in chunks of kChunk
// sites staged in shared memory (two buffers: the threads stage chunk c + 1
// while the tensor cores work on chunk c) in the K-major core-matrix layout
// (8 rows x 16 bytes per core matrix).  Site values arrive as 16-byte loads
// (two sites of one row), the next chunk's loads in flight while the current
// chunk is split and stored, and each warp's stores fill whole 512-byte runs,
// so staging has no bank conflicts.  The phase operand is the same for every
// row tile: a first kernel writes it for all sites, already split into hi +
// lo in the shared-memory image of each chunk, and one bulk copy per chunk
// brings it in.  The phases are products of three per-direction tables,
// exp(-2 pi i j / L_k), so no angle is reduced per site.  One thread
// issues tcgen05.mma (kind::tf32, M = 128, N = 2*n_mom padded to 16) into a
// TMEM accumulator; TF32 keeps 10 mantissa bits, so every operand is split
// into hi + lo parts and three products hi*hi + hi*lo + lo*hi are
// accumulated (relative error ~2^-21 per product).  The CTA's FP32 sum over
// its sites (the accumulator depth, at most kMaxCtaSites, bounds its
// rounding) goes to a buffer of partial sums; a last kernel adds the CTAs'
// partial sums in a fixed order in two-float arithmetic (error-free FP32
// additions, FP64 once per output) and applies the fields' scale.
#include <algorithm>

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {

namespace {

constexpr int kM = 128;             // rows per CTA (tensor-core M)
constexpr int kChunk = 16;          // sites per staged chunk
constexpr int kKt = 2 * kChunk;     // real K per chunk
constexpr int kMaxMomP = 64;        // N = 2*n_mom <= 128
constexpr int kMaxCtaSites = 256;   // sites summed in one FP32 tensor-core accumulator
constexpr int kMaxL = 128;          // longest spatial extent of the phase tables

struct ProjArgs {
  int rows;           // n_chan * Nt
  int Nt, V3, nmom, npad;
  int sites_per_cta;  // multiple of kChunk
  int sL[3];
  int origin[3];
  int k[kMaxMomP][3];
};

// Byte offset of the core-matrix row holding k = 4*kc .. 4*kc+3 of row r in
// a K-major tile of kKt columns.
__device__ __forceinline__ uint32_t core_row(int r, int kc) {
  return (uint32_t)(((r >> 3) * (kKt / 4) + kc) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void split4(float4 v, float4& hi, float4& lo) {
  auto h = [](float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); };
  hi = make_float4(h(v.x), h(v.y), h(v.z), h(v.w));
  lo = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The phase operand of every chunk, in its shared-memory image: for chunk c,
// [hi | lo] x (npad rows x kKt K-major core matrices); rows 2m: (cos, sin),
// rows 2m+1: (-sin, cos) per site, zero beyond V3 and for the padding rows.
__global__ void __launch_bounds__(256) phase_tile_kernel(ProjArgs P, float4* __restrict__ tiles) {
  __shared__ float2 tab[3][kMaxL];  // exp(-2 pi i j / L_k)
  for (int i = threadIdx.x; i < 3 * kMaxL; i += 256) {
    const int k = i / kMaxL, j = i % kMaxL;
    float sn = 0.f, cs = 1.f;
    if (j < P.sL[k]) sincospif(2.0f * (float)j / (float)P.sL[k], &sn, &cs);
    tab[k][j] = make_float2(cs, -sn);
  }
  __syncthreads();
  // one thread per (chunk, row n, core-matrix column kc): two sites, one row
  const int per_chunk = P.npad * (kKt / 4);
  const long long total = (long long)((P.V3 + kChunk - 1) / kChunk) * per_chunk;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < total; i += (long long)gridDim.x * 256) {
    const int c = (int)(i / per_chunk), rem = (int)(i % per_chunk);
    const int n = rem / (kKt / 4), kc = rem % (kKt / 4), m = n >> 1;
    float2 ph[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (m < P.nmom) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int xs = c * kChunk + 2 * kc + e;
        if (xs < P.V3) {
          const int cc[3] = {xs % P.sL[0], (xs / P.sL[0]) % P.sL[1], xs / (P.sL[0] * P.sL[1])};
          float2 f = make_float2(1.f, 0.f);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int L = P.sL[k];
            const int d = ((cc[k] - P.origin[k]) % L + L) % L;
            const int j = ((P.k[m][k] * d) % L + L) % L;
            f = cmulf(f, tab[k][j]);
          }
          ph[e] = f;  // exp(-i p.(x - x0)) = (cos, -sin)
        }
      }
    }
    const float4 v = (n & 1) ? make_float4(ph[0].y, ph[0].x, ph[1].y, ph[1].x)
                             : make_float4(ph[0].x, -ph[0].y, ph[1].x, -ph[1].y);
    float4 hi, lo;
    split4(v, hi, lo);
    const size_t base = (size_t)c * 2 * per_chunk;  // float4 units: [hi tile][lo tile]
    const size_t o = core_row(n, kc) / 16;
    tiles[base + o] = hi;
    tiles[base + per_chunk + o] = lo;
  }
}

__global__ void __launch_bounds__(128) momproj_kernel(const float2* __restrict__ sites, ProjArgs P,
                                                      const float4* __restrict__ tiles, float* __restrict__ partial,
                                                      unsigned int* status, long long timeout_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t a_bytes = kM * kKt * 4, b_bytes = P.npad * kKt * 4;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;  // A hi, A lo, B hi, B lo
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);  // [2] tensor cores done, [2] B landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kM;
  const int xb = blockIdx.y * P.sites_per_cta;
  const int xe = min(P.V3, xb + P.sites_per_cta);
  const int nchunks = (xe - xb + kChunk - 1) / kChunk;
  const int tcols = P.npad <= 32 ? 32 : (P.npad <= 64 ? 64 : 128);

  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(tslot), tcols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) ptx::mbar_init(ptx::smem_addr(bar + i), 1);
    ptx::fence_mbar_init();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = ptx::idesc_tf32(kM, P.npad);

  // A of one chunk: this thread's 8 core-matrix rows (two sites each)
  constexpr int kAPer = (kM / 8) * (kKt / 4) / 4 / 4;  // warp tasks per warp
  float4 va[kAPer];
  auto load_a = [&](int c) {
    const int x0 = xb + c * kChunk;
#pragma unroll
    for (int i = 0; i < kAPer; ++i) {
      const int u = warp + 4 * i;
      const int rg = u / (kKt / 16), kc = (u % (kKt / 16)) * 4 + (lane >> 3);
      const int row = row0 + rg * 8 + (lane & 7), x = x0 + 2 * kc;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < P.rows) {
        const float2* src = sites + (size_t)row * P.V3 + x;
        if (x + 1 < xe && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
          v = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          if (x < xe) { const float2 a = __ldg(src); v.x = a.x; v.y = a.y; }
          if (x + 1 < xe) { const float2 b = __ldg(src + 1); v.z = b.x; v.w = b.y; }
        }
      }
      va[i] = v;
    }
  };
  if (nchunks > 0) load_a(0);
  if (tid == 0 && nchunks > 0) {  // B of chunk 0
    const uint32_t bb = ptx::smem_addr(smem + 2 * a_bytes);
    ptx::mbar_arrive_expect_tx(ptx::smem_addr(bar + 2), 2 * b_bytes);
    ptx::bulk_g2s(bb, tiles + (size_t)(xb / kChunk) * 2 * (b_bytes / 16), 2 * b_bytes, ptx::smem_addr(bar + 2));
  }

  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    unsigned char* st = smem + s * stage_bytes;
    // write this chunk's A (in registers) into stage s
#pragma unroll
    for (int i = 0; i < kAPer; ++i) {
      const int u = warp + 4 * i;
      const int rg = u / (kKt / 16), kc = (u % (kKt / 16)) * 4 + (lane >> 3);
      float4 hi, lo;
      split4(va[i], hi, lo);
      const uint32_t o = core_row(rg * 8 + (lane & 7), kc);
      *reinterpret_cast<float4*>(st + o) = hi;
      *reinterpret_cast<float4*>(st + a_bytes + o) = lo;
    }
    ptx::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      const bool bin = ptx::mbar_wait_bounded(ptx::smem_addr(bar + 2 + s), (c >> 1) & 1, timeout_ns);
      if (bin) {
        ptx::tc_fence_after();
        const uint32_t ah = ptx::smem_addr(st), al = ah + a_bytes, bh = al + a_bytes, bl = bh + b_bytes;
        const uint32_t sbo = (kKt / 4) * 128;
#pragma unroll
        for (int k = 0; k < kKt / 8; ++k) {
          const uint32_t off = k * 256;  // two core matrices along K per instruction
          const uint64_t dah = ptx::smem_desc_noswizzle(ah + off, 128, sbo);
          const uint64_t dal = ptx::smem_desc_noswizzle(al + off, 128, sbo);
          const uint64_t dbh = ptx::smem_desc_noswizzle(bh + off, 128, sbo);
          const uint64_t dbl = ptx::smem_desc_noswizzle(bl + off, 128, sbo);
          ptx::mma_tf32(tmem, dah, dbh, idesc, (c > 0 || k > 0) ? 1u : 0u);
          ptx::mma_tf32(tmem, dah, dbl, idesc, 1u);
          ptx::mma_tf32(tmem, dal, dbh, idesc, 1u);
        }
        ptx::mma_commit(ptx::smem_addr(bar + s));
      } else {
        atomicOr(status, kStatusFullWait);
      }
    }
    // next chunk: its loads go out before this thread waits for stage s ^ 1
    if (c + 1 < nchunks) load_a(c + 1);
    if (c >= 1) {  // the tensor cores have read chunk c - 1 from stage s ^ 1
      const bool done = ptx::mbar_wait_bounded(ptx::smem_addr(bar + (s ^ 1)), ((c - 1) >> 1) & 1, timeout_ns);
      if (!__syncthreads_and(done ? 1 : 0)) {
        ok = false;
        break;
      }
      ptx::tc_fence_after();
    }
    if (tid == 0 && c + 1 < nchunks) {  // B of chunk c + 1 into stage s ^ 1
      const uint32_t bb = ptx::smem_addr(smem + (s ^ 1) * stage_bytes + 2 * a_bytes);
      ptx::mbar_arrive_expect_tx(ptx::smem_addr(bar + 2 + (s ^ 1)), 2 * b_bytes);
      ptx::bulk_g2s(bb, tiles + (size_t)(xb / kChunk + c + 1) * 2 * (b_bytes / 16), 2 * b_bytes,
                    ptx::smem_addr(bar + 2 + (s ^ 1)));
    }
  }
  if (ok && nchunks > 0) {  // the last commit covers every MMA issued before it
    const int c = nchunks - 1;
    const bool done = ptx::mbar_wait_bounded(ptx::smem_addr(bar + (c & 1)), (c >> 1) & 1, timeout_ns);
    ok = __syncthreads_and(done ? 1 : 0) != 0;
    ptx::tc_fence_after();
  }
  if (!ok) {
    // a wait ran out: record it and give the outstanding copies and MMAs one
    // more bounded wait so that nothing writes this CTA's buffers after it exits
    if (tid == 0) {
      atomicOr(status, kStatusFullWait);
      for (int c = max(0, nchunks - 2); c < nchunks; ++c) {
        if (!ptx::mbar_wait_bounded(ptx::smem_addr(bar + 2 + (c & 1)), (c >> 1) & 1, timeout_ns))
          atomicOr(status, kStatusDrain);
        if (!ptx::mbar_wait_bounded(ptx::smem_addr(bar + (c & 1)), (c >> 1) & 1, timeout_ns))
          atomicOr(status, kStatusDrain);
      }
    }
  } else {
    // epilogue: warp w owns TMEM lanes (rows) 32w..32w+31; partial[split][col][row]
    const int row = row0 + warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    float* dst = partial + (size_t)blockIdx.y * P.npad * P.rows;
    for (int c0 = 0; c0 < P.npad; c0 += 16) {
      float v[16];
      if (nchunks > 0) {
        ptx::tmem_ld16(taddr + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
      if (row < P.rows) {
#pragma unroll
        for (int i = 0; i < 16; ++i) dst[(size_t)(c0 + i) * P.rows + row] = v[i];
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 0) ptx::tmem_dealloc(tmem, tcols);
}

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  const float x = __fadd_rn(a, b);
  const float bv = __fsub_rn(x, a);
  const float av = __fsub_rn(x, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  s = x;
}

// out[(chan * nmom + m) * Nt + t] = 2^e * sum over the site splits of the
// partial sums: one thread per output, consecutive threads on consecutive
// rows (coalesced reads of partial[split][col][row] and writes of out), the
// splits added in order in two-float arithmetic (hi + lo), FP64 once.
// Block (32 rows, momentum m): eight groups of 32 threads each add every
// eighth CTA's partial sums of their row in two-float arithmetic (a warp
// reads 32 consecutive rows of one partial), then the eight group sums of a
// row are added in group order.
__global__ void __launch_bounds__(256) momproj_fold_kernel(const float* __restrict__ partial, int nsplit, int rows,
                                                           int npad, int nmom, int Nt, double* __restrict__ out,
                                                           const ScaleRecord* ra, int ca, const ScaleRecord* rb,
                                                           int cb, const int* __restrict__ chan_exp) {
  __shared__ float4 acc[8][32];  // (hr, lr, hi, li) per group and row
  const int rl = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int row = blockIdx.x * 32 + rl, m = blockIdx.y;
  float hr = 0.f, lr = 0.f, hi = 0.f, li = 0.f;
  if (row < rows) {
    for (int sp = grp; sp < nsplit; sp += 8) {
      const float* p = partial + (size_t)sp * npad * rows;
      float e;
      two_sum(hr, p[(size_t)(2 * m) * rows + row], hr, e);
      lr += e;
      two_sum(hi, p[(size_t)(2 * m + 1) * rows + row], hi, e);
      li += e;
    }
  }
  acc[grp][rl] = make_float4(hr, lr, hi, li);
  __syncthreads();
  if (grp != 0 || row >= rows) return;
  for (int g = 1; g < 8; ++g) {
    const float4 v = acc[g][rl];
    float e;
    two_sum(hr, v.x, hr, e);
    lr += e + v.y;
    two_sum(hi, v.z, hi, e);
    li += e + v.w;
  }
  const int chan = row / Nt, t = row % Nt;
  const int ex = chan_exp ? chan_exp[chan] : (ra ? ca * ra->exp : 0) + (rb ? cb * rb->exp : 0);
  const long long o = ((long long)chan * nmom + m) * Nt + t;
  out[2 * o] = ldexp((double)hr + (double)lr, ex);
  out[2 * o + 1] = ldexp((double)hi + (double)li, ex);
}

}  // namespace

}  // namespace qdpg

using namespace qdpg;

namespace qdpg {

int launch_momproj(const Geom& g, const void* sites_dev, int n_chan, const int* moms, int n_mom, const int origin[4],
                   double* out_dev, const ScaleRecord* ra, int ca, const ScaleRecord* rb, int cb, cudaStream_t s,
                   const int* chan_exp) {
  if (n_chan < 1) return fail(QDPG_ERR_ARG, "momentum_project: n_chan %d < 1", n_chan);
  if (n_mom < 1 || n_mom > kMaxMomP) return fail(QDPG_ERR_ARG, "momentum_project: n_mom %d outside 1..%d", n_mom, kMaxMomP);
  if (reinterpret_cast<uintptr_t>(sites_dev) % 8) return fail(QDPG_ERR_ARG, "momentum_project: sites not 8-byte aligned");
  for (int k = 0; k < 3; ++k)
    if (g.sL[k] > kMaxL) return fail(QDPG_ERR_UNSUPPORTED, "momentum_project: spatial extent above %d", kMaxL);
  const long long rows = (long long)n_chan * g.Nt;
  if (rows > (1LL << 30)) return fail(QDPG_ERR_ARG, "momentum_project: too many rows");
  unsigned int* status = device_status_word();
  if (!status) return fail(QDPG_ERR_CUDA, "momentum_project: no status word");
  ProjArgs P{};
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
  const size_t stage_bytes = (size_t)2 * kM * kKt * 4 + (size_t)2 * P.npad * kKt * 4;
  const size_t smem = 2 * stage_bytes + 4 * sizeof(uint64_t) + 16;
  // split the sites among CTAs of at most kMaxCtaSites sites each (the
  // tensor-core accumulator is FP32 and its depth bounds the rounding error;
  // longer sums add up in the FP64 fold), choosing the number of full waves
  // of resident CTAs and the split that fills them with the fewest chunks
  // per CTA: a grid a little over one wave would run its remainder as a
  // second wave of full-length CTAs
  const int nchunk_all = (g.V3 + kChunk - 1) / kChunk;
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(momproj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, momproj_kernel, 128, smem) != cudaSuccess)
    return fail(QDPG_ERR_CUDA, "momentum_project: device query failed");
  const long long slots = std::max(1LL, (long long)nsm * std::max(1, per_sm));
  const int min_split = (g.V3 + kMaxCtaSites - 1) / kMaxCtaSites;
  int nsplit = std::max(1, min_split), best_cost = -1;
  for (int w = 1; w <= 64; ++w) {
    const int ns = (int)std::min<long long>(nchunk_all, slots * w / row_tiles);
    if (ns < min_split) continue;
    const int spc = (nchunk_all + ns - 1) / ns;                                   // chunks per CTA
    const int waves = (int)(((long long)row_tiles * ((nchunk_all + spc - 1) / spc) + slots - 1) / slots);
    const int cost = waves * (spc + 2);                                           // + pipeline fill per CTA
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      nsplit = ns;
    }
    if (ns == nchunk_all) break;
  }
  P.sites_per_cta = (nchunk_all + nsplit - 1) / nsplit * kChunk;
  nsplit = (g.V3 + P.sites_per_cta - 1) / P.sites_per_cta;
  const int nchunk_pad = (g.V3 + kChunk - 1) / kChunk;
  const size_t tile_bytes = (size_t)nchunk_pad * 2 * P.npad * kKt * 4;

  void* partial = nullptr;
  void* tiles = nullptr;
  int rc = dev_alloc(&partial, sizeof(float) * (size_t)nsplit * P.npad * rows, s, "momentum_project partial sums");
  if (rc == QDPG_OK) rc = dev_alloc(&tiles, tile_bytes, s, "momentum_project phase tiles");
  if (rc != QDPG_OK) {
    dev_free(partial, s);
    return rc;
  }
  {
    ProfScope prof("momentum_project", s);
    const long long ntask = (long long)nchunk_pad * P.npad * (kKt / 4);
    phase_tile_kernel<<<(int)std::min<long long>((ntask + 255) / 256, 152LL * 8), 256, 0, s>>>(
        P, static_cast<float4*>(tiles));
    rc = check_launch("momentum_project phases");
    if (rc == QDPG_OK) {
      momproj_kernel<<<dim3(row_tiles, nsplit), 128, smem, s>>>(static_cast<const float2*>(sites_dev), P,
                                                                  static_cast<const float4*>(tiles),
                                                                  static_cast<float*>(partial), status,
                                                                  wait_timeout_ns());
      rc = check_launch("momentum_project");
    }
    if (rc == QDPG_OK) {
      momproj_fold_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)n_mom), 256, 0, s>>>(static_cast<const float*>(partial), nsplit,
                                                                  (int)rows, P.npad, n_mom, g.Nt, out_dev, ra, ca,
                                                                  rb, cb, chan_exp);
      rc = check_launch("momentum_project fold");
    }
  }
  dev_free(tiles, s);
  dev_free(partial, s);
  return rc;
}

}  // namespace qdpg

extern "C" int qdpg_momentum_project(qdpg_lattice_t lat, const void* sites_dev, int n_chan, const int* moms,
                                     int n_mom, const int origin[4], double* out_dev, void* stream) {
  if (!lat || !sites_dev || !moms || !out_dev) return fail(QDPG_ERR_ARG, "momentum_project: null argument");
  return launch_momproj(lat->g, sites_dev, n_chan, moms, n_mom, origin, out_dev, nullptr, 0, nullptr, 0,
                        as_stream(stream));
}
