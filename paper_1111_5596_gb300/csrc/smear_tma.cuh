// Pipelined Gaussian-smearing hop (the paper's SRC/SNK stages, Sec. 5):
// kernel template shared by the per-precision translation units.
//
// Same operation as smear_hop_kernel in smear.cu,
//   psi'(x) = psi(x) + kappa * sum_{i} [ U_i(x) psi(x+i) + U_i(x-i)^dag psi(x-i) ],
// organised for GB300's memory system:
//
//  * a CTA owns a tile of k rows of one (t, z) plane; each consumer thread
//    owns one site and keeps its six links in registers for all 48 colour
//    vectors of the propagator (one link load per site per iteration);
//  * a producer warp streams, G colour vectors at a time, the three colour
//    planes of the tile plus its halo (rows y0-1 and y0+k of plane z unless
//    the tile is the whole plane, and the same k rows of planes z-1 and z+1,
//    all periodic) from HBM/L2 into shared memory with bulk asynchronous
//    copies (cp.async.bulk on the TMA engine), several stages ahead of the
//    consumers, so the bytes in flight per SM do not depend on registers;
//  * mbarriers hand stages between producer and consumers ("full" with a
//    transaction count, "empty" with one arrival per consumer warp); every
//    wait is bounded and a wait that runs out records a flag in the device
//    status word instead of hanging; the producer then drains its own copies
//    (bounded as well) before the CTA exits;
//  * for the common tile shapes (LX > 0) the plane width, rows and halo are
//    template constants, so every shared-memory operand is a register base
//    plus an immediate offset.
#pragma once

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"
#include "smear_common.cuh"

namespace qdpg {
namespace tma_smear {

using namespace smear_dev;

constexpr int kMaxStages = 16;
constexpr int kMaxConsumers = 256;
constexpr size_t kSmemBudget = 200 * 1024;  // bytes of stages per CTA

// Shared-memory loads of staged elements (plain loads: __ldg is global-only).
__device__ __forceinline__ float2 lds(const float2* p) { return *p; }
__device__ __forceinline__ float2 lds(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ u64 lds_pair(const float2* p) { return *reinterpret_cast<const u64*>(p); }
__device__ __forceinline__ u64 lds_pair(const __nv_bfloat162* p) { return pack2(__bfloat1622float2(*p)); }

struct TmaTile {
  int k;         // plane rows per tile
  int ntiles_y;  // Ly / k
  int cwarps;    // consumer warps
  int halo;      // 1: rows y0-1 and y0+k are staged; 0: the tile is a whole plane (y wraps inside it)
  int rowsA;     // rows of plane z per colour: k + 2*halo
  int rows;      // rows per colour in a stage: rowsA + k (plane z-1) + k (plane z+1)
  int stages;    // pipeline depth, 2..kMaxStages
  int G;         // colour vectors per stage
};

struct HopLaunch {
  const void* in;
  void* out;
  const void* U;
  Geom g;
  TmaTile tt;
  float kappa;
  unsigned int* status;
  long long timeout_ns;
  int drop_vec;
  cudaStream_t stream;
};

template <typename PsiT, int LMODE, int LX, int KR, int HALO, int G>
__global__ void __launch_bounds__(kMaxConsumers + 32, 1)
    smear_hop_tma_kernel(const PsiT* __restrict__ in, PsiT* __restrict__ out, const void* __restrict__ U, Geom g,
                         TmaTile tt, float kappa, unsigned int* status, long long timeout_ns, int drop_vec) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int COLS = 12;
  constexpr int NC = 12 * COLS;
  constexpr int NV = 4 * COLS;
  constexpr int NSTEP = NV / G;
  static_assert(COLS % G == 0, "G must divide the 12 source columns");
  constexpr int NCL = (LMODE == L_F32_R12 || LMODE == L_BF16_R12) ? 24 : 36;
  const int Lx = LX ? LX : g.sL[0];
  const int k = LX ? KR : tt.k;
  const int halo = LX ? HALO : tt.halo;
  const int rowsA = k + 2 * halo;
  const int rows = rowsA + 2 * k;
  const int Ly = g.sL[1], Lz = g.sL[2], V3 = g.V3;
  const int S = tt.stages;
  const int yb = blockIdx.x % tt.ntiles_y;
  const int z = blockIdx.x / tt.ntiles_y;
  const int t = blockIdx.y;
  const int y0 = yb * k;
  const int CS = rows * Lx;  // elements per colour region
  const int stage_elems = G * 3 * CS;
  const uint32_t stage_bytes = (uint32_t)stage_elems * sizeof(PsiT);
  PsiT* st = reinterpret_cast<PsiT*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * stage_bytes);
  const uint32_t full0 = ptx::smem_addr(bars);
  const uint32_t empty0 = ptx::smem_addr(bars + S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, tt.cwarps);
    }
    ptx::fence_mbar_init();
  }
  __syncthreads();

  if (warp == tt.cwarps) {
    // ---------------- producer warp ----------------
    const PsiT* base_t = in + (size_t)t * NC * V3;
    const int zm = (z - 1 + Lz) % Lz, zp = (z + 1) % Lz;
    const int ym = (y0 - 1 + Ly) % Ly, yp = (y0 + k) % Ly;
    const int npieces = halo ? 5 : 3;
    const int ncopies = G * 3 * npieces;

    int j = 0;
    for (int s = 0, n = 0; j < NSTEP; ++j) {
      if (n > 0) {
        const bool ok = ptx::mbar_wait_bounded(empty0 + 8 * s, (n - 1) & 1, timeout_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicOr(status, kStatusEmptyWait);
          break;
        }
      }
      if (j * G > drop_vec || j * G + G <= drop_vec) {  // test hook: skip the stage holding drop_vec
        if (lane == 0) ptx::mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
        __syncwarp();
        for (int cp = lane; cp < ncopies; cp += 32) {
          const int gg = cp / (3 * npieces), rem = cp % (3 * npieces);
          const int c = rem / npieces, piece = rem % npieces;
          int src_off, dst_row, nrows;
          if (halo) {
            switch (piece) {
              case 0: src_off = (z * Ly + ym) * Lx; dst_row = 0; nrows = 1; break;
              case 1: src_off = (z * Ly + y0) * Lx; dst_row = 1; nrows = k; break;
              case 2: src_off = (z * Ly + yp) * Lx; dst_row = k + 1; nrows = 1; break;
              case 3: src_off = (zm * Ly + y0) * Lx; dst_row = rowsA; nrows = k; break;
              default: src_off = (zp * Ly + y0) * Lx; dst_row = rowsA + k; nrows = k; break;
            }
          } else {
            switch (piece) {
              case 0: src_off = (z * Ly + y0) * Lx; dst_row = 0; nrows = k; break;
              case 1: src_off = (zm * Ly + y0) * Lx; dst_row = rowsA; nrows = k; break;
              default: src_off = (zp * Ly + y0) * Lx; dst_row = rowsA + k; nrows = k; break;
            }
          }
          const int v = j * G + gg;
          const int comp = (v / COLS) * 3 * COLS + c * COLS + (v % COLS);
          const PsiT* src = base_t + (size_t)comp * V3 + src_off;
          const uint32_t dst = ptx::smem_addr(st + (size_t)s * stage_elems + (gg * 3 + c) * CS + dst_row * Lx);
          ptx::bulk_g2s(dst, src, (uint32_t)(nrows * Lx) * sizeof(PsiT), full0 + 8 * s);
        }
      }
      if (++s == S) {
        s = 0;
        ++n;
      }
    }
    // Drain: every copy this warp issued (the last S stages) has landed
    // before the CTA may exit.
    if (lane == 0) {
      for (int u = (j > S ? j - S : 0); u < j; ++u)
        if ((u * G > drop_vec || u * G + G <= drop_vec) &&
            !ptx::mbar_wait_bounded(full0 + 8 * (u % S), (u / S) & 1, timeout_ns))
          atomicOr(status, kStatusDrain);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int ctid = threadIdx.x;
  const bool active = ctid < Lx * k;
  const int r = active ? ctid / Lx : 0;
  const int x = active ? ctid % Lx : 0;
  const int y = y0 + r;
  const int s3 = x + Lx * (y + Ly * z);

  float2 Uf[3][9], Ub[3][9];
  if (active) {
    const int xm = x == 0 ? Lx - 1 : x - 1;
    const int ymn = y == 0 ? Ly - 1 : y - 1;
    const int zmn = z == 0 ? Lz - 1 : z - 1;
    const int sb[3] = {xm + Lx * (y + Ly * z), x + Lx * (ymn + Ly * z), x + Lx * (y + Ly * zmn)};
    const long long lt = (long long)t * NCL * V3;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      load_link<LMODE>(U, lt + s3, V3, g.sd[i], Uf[i]);
      load_link<LMODE>(U, lt + sb[i], V3, g.sd[i], Ub[i]);
    }
  }
  // shared-memory offsets (elements, within a colour region) of the seven sites
  const int rc = r + halo;
  const int oc = rc * Lx + x;
  const int yp_row = halo ? r + 2 : (r + 1 == k ? 0 : r + 1);
  const int ym_row = halo ? r : (r == 0 ? k - 1 : r - 1);
  const int of[3] = {rc * Lx + (x + 1 == Lx ? 0 : x + 1), yp_row * Lx + x, (rowsA + k + r) * Lx + x};
  const int ob[3] = {rc * Lx + (x == 0 ? Lx - 1 : x - 1), ym_row * Lx + x, (rowsA + r) * Lx + x};
  PsiT* outp = out + (size_t)t * NC * V3 + s3;
  SiteLinks L;
  make_site_links(Uf, Ub, L);

  for (int j = 0, s = 0, n = 0; j < NSTEP; ++j) {
    const bool ok = ptx::mbar_wait_bounded(full0 + 8 * s, n & 1, timeout_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(status, kStatusFullWait);
      break;
    }
    if (active) {
      const PsiT* sp = st + (size_t)s * stage_elems;
      const int v0 = j * G;
      PsiT* po = outp + (size_t)((v0 / COLS) * 3 * COLS + (v0 % COLS)) * V3;
#pragma unroll
      for (int gg = 0; gg < G; ++gg) {
        const PsiT* sg = sp + gg * 3 * CS;
        u64 nf[3][3], nb[3][3];
        float2 c[3], o[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            nf[i][q] = lds_pair(sg + of[i] + q * CS);
            nb[i][q] = lds_pair(sg + ob[i] + q * CS);
          }
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a] = lds(sg + oc + a * CS);
        hop_vector(L, nf, nb, c, kappa, o);
#pragma unroll
        for (int a = 0; a < 3; ++a) st2(po + (gg + a * COLS) * V3, o[a]);
      }
    }
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(empty0 + 8 * s);
    if (++s == S) {
      s = 0;
      ++n;
    }
  }
}

template <typename PsiT, int LMODE, int LX, int KR, int HALO, int G>
int launch_tma_t(const HopLaunch& a) {
  const size_t stage_bytes = (size_t)G * 3 * a.tt.rows * a.g.sL[0] * sizeof(PsiT);
  const size_t smem = a.tt.stages * stage_bytes + 2 * a.tt.stages * sizeof(uint64_t);
  auto kern = smear_hop_tma_kernel<PsiT, LMODE, LX, KR, HALO, G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear: smem attribute: %s", cudaGetErrorString(e));
  dim3 grid(a.tt.ntiles_y * a.g.sL[2], a.g.Nt);
  dim3 block(32 * (a.tt.cwarps + 1));
  ProfScope prof("smear_hop", a.stream);
  kern<<<grid, block, smem, a.stream>>>(static_cast<const PsiT*>(a.in), static_cast<PsiT*>(a.out), a.U, a.g, a.tt,
                                        a.kappa, a.status, a.timeout_ns, a.drop_vec);
  return check_launch("gauss_smear hop (pipelined)");
}

// Tile shapes with compile-time instantiations: (Lx, rows, halo).
#define QDPG_TMA_FIXED_SHAPES(X) \
  X(16, 16, 0)                   \
  X(24, 8, 1)                    \
  X(48, 4, 1)                    \
  X(8, 8, 0)                     \
  X(12, 12, 0)

// Launch the instantiation for (PsiT, LMODE): a fixed tile shape if one
// matches, else the runtime-shape kernel.
template <typename PsiT, int LMODE>
int launch_tma_any(const HopLaunch& a) {
  const int Lx = a.g.sL[0];
  constexpr int G = 2;
#define QDPG_TMA_TRY(LXV, KV, HV) \
  if (Lx == LXV && a.tt.k == KV && a.tt.halo == HV) return launch_tma_t<PsiT, LMODE, LXV, KV, HV, G>(a);
  QDPG_TMA_FIXED_SHAPES(QDPG_TMA_TRY)
#undef QDPG_TMA_TRY
  return launch_tma_t<PsiT, LMODE, 0, 0, 0, G>(a);
}

int launch_tma_f32(int lprec, const HopLaunch& a);
int launch_tma_bf16(int lprec, const HopLaunch& a);

}  // namespace tma_smear
}  // namespace qdpg
