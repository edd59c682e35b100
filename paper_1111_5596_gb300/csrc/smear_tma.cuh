// Pipelined, persistent Gaussian-smearing hop (the paper's SRC/SNK stages,
// Sec. 5): kernel template shared by the per-precision translation units.
//
// Same operation as smear_hop_kernel in smear.cu,
//   psi'(x) = psi(x) + kappa * sum_{i} [ U_i(x) psi(x+i) + U_i(x-i)^dag psi(x-i) ],
// organised for GB300's memory system:
//
//  * work items are (tile, half of the 48 colour vectors); a tile is k rows
//    of one (t, z) plane; one CTA per SM (two for tiles of at most 128
//    sites) walks the items round-robin, so neighbouring planes are in
//    flight together and share their halo reads in L2;
//  * each consumer thread owns one site and keeps its six links in registers
//    for the item's 24 colour vectors;
//  * one producer warp streams, with asynchronous copies on the TMA engine,
//    first the links of the item's tile into a shared-memory link buffer
//    (cp.async.bulk), then G colour vectors per stage of the three colour
//    planes of the tile plus its halo (rows y0-1 and y0+k of plane z unless
//    the tile is a whole plane, and the same k rows of planes z-1 and z+1,
//    all periodic), each run of consecutive rows in one copy; a whole-plane
//    tile whose planes z-1..z+1 are consecutive in memory takes the whole
//    stage in one tensor-map copy (cp.async.bulk.tensor, a 4-D box); it runs
//    ahead of the consumers across item boundaries, so consumers never wait
//    on global loads.  A stage holds region (colour q, vector gg) at
//    (q * G + gg) * rows * Lx, rows in the order the copies deliver them;
//  * mbarriers hand stages and the link buffer between producer and
//    consumers ("full" with a transaction count, "empty" with one arrival per
//    consumer warp); every wait is bounded, and a wait that runs out records
//    a flag in the device status word instead of hanging; the producer then
//    drains its own copies (bounded as well) before the CTA exits;
//  * for the common tile shapes (LX > 0) the plane width, rows and halo are
//    template constants, so every shared-memory operand is a register base
//    plus an immediate offset;
//  * halo tiles of those shapes keep a stage row-major, element (row, colour
//    q, vector gg, x) at ((row * 3 + q) * G + gg) * Lx + x, so that boxes of
//    whole rows for all three colours and the stage's G vectors stack: a
//    stage is five tensor-map copies (rows y0-1, y0..y0+k-1 and y0+k of
//    plane z, the same k rows of planes z-1 and z+1) instead of one bulk
//    copy per row run, colour and vector.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)

#include <type_traits>

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"
#include "smear_common.cuh"

namespace qdpg {
namespace tma_smear {

using namespace smear_dev;

constexpr int kMaxStages = 16;
constexpr int kMaxConsumers = 288;
constexpr int kSplit = 2;  // work items per tile: colour vectors 0..23 and 24..47

// Shared-memory loads of staged elements (plain loads: __ldg is global-only).
__device__ __forceinline__ float2 lds(const float2* p) { return *p; }
__device__ __forceinline__ float2 lds(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ u64 lds_pair(const float2* p) { return *reinterpret_cast<const u64*>(p); }
__device__ __forceinline__ u64 lds_pair(const __nv_bfloat162* p) { return pack2(__bfloat1622float2(*p)); }

struct TmaTile {
  int k;          // plane rows per tile
  int ntiles_y;   // Ly / k
  int cwarps;     // consumer warps
  int halo;       // 1: rows y0-1 and y0+k are staged; 0: the tile is a whole plane (y wraps inside it)
  int rowsA;      // rows of plane z per colour: k + 2*halo
  int rows;       // rows per colour in a stage: rowsA + k (plane z-1) + k (plane z+1)
  int stages;     // pipeline depth, 2..kMaxStages
  int G;          // colour vectors per stage
  int nitems;     // tiles * kSplit
  int grid;       // persistent CTAs
  int smem;       // dynamic shared memory bytes
  int use_tmap;   // 1: whole-plane tiles stage planes z-1..z+1 with one tensor-map copy
  int use_rm;     // 1: halo tiles of a fixed shape stage row-major with tensor-map copies
};

// Jobs of one launch: same lattice and precisions, own fields and kappa.
// Work items are job-major: item i belongs to job i / TmaTile::nitems.
constexpr int kMaxJobs = 64;
struct JobPtrs {
  const void* in;
  void* out;
  const void* U;
  float kappa;
};
// tmap[i]: job i's input propagator as a 4-D tensor (x; row = y + Ly*z;
// the 12 colour vectors of a spin row; spin-row-colour + 12*t), for the
// whole-plane tiles' tensor-map copies (TmaTile::use_tmap); for row-major
// halo tiles (TmaTile::use_rm) the same tensor with the row outermost (x;
// vector; spin-row-colour + 12*t; row), boxes of k rows, and tmap_row[i] its
// one-row boxes.
struct JobTable {
  int njobs;
  JobPtrs j[kMaxJobs];
  CUtensorMap tmap[kMaxJobs];
  CUtensorMap tmap_row[kMaxJobs];
};

struct HopLaunch {
  JobTable jobs;
  Geom g;
  TmaTile tt;
  unsigned int* status;
  long long timeout_ns;
  int drop_stage;
  cudaStream_t stream;
};

template <int LMODE>
struct LinkTraits {
  static constexpr bool r12 = LMODE == L_F32_R12 || LMODE == L_BF16_R12;
  static constexpr int NE = r12 ? 6 : 9;  // stored entries per link
  static constexpr bool f32 = LMODE == L_F32 || LMODE == L_F32_R12;
  typedef typename std::conditional<f32, float2, __nv_bfloat162>::type T;
};

// Link buffer layout (elements of the link type), for a tile of k rows:
//   F[i][e][k*Lx]   forward links U_{sd_i}(x), entry e, rows y0..y0+k-1 of plane z
//   YH[e][Lx]       U_{sd_1} on row y0-1 of plane z (halo tiles only)
//   ZB[e][k*Lx]     U_{sd_2} on rows y0..y0+k-1 of plane z-1
__host__ __device__ inline int link_elems(int NE, int k, int Lx, int halo) {
  return 3 * NE * k * Lx + (halo ? NE * Lx : 0) + NE * k * Lx;
}

// Read one link (entries at p + e*stride) from the buffer; expand row 2 for
// reconstruct-12 storage.
template <int LMODE, typename LT>
__device__ __forceinline__ void link_from_smem(const LT* p, int stride, float2 m[9]) {
  constexpr int NE = LinkTraits<LMODE>::NE;
#pragma unroll
  for (int e = 0; e < NE; ++e) m[e] = lds(p + e * stride);
  if (LinkTraits<LMODE>::r12) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
      const float2 c = cmul(m[b1], m[3 + b2]);
      const float2 d = cmul(m[b2], m[3 + b1]);
      m[6 + b] = make_float2(c.x - d.x, -(c.y - d.y));
    }
  }
}

// Threads per CTA (consumer warps + the producer warp) and the CTAs per SM
// the register budget is sized for: tiles of at most 128 sites run two CTAs
// per SM.
template <int LX, int KR>
struct TileLaunch {
  static constexpr int threads = LX ? ((LX * KR + 31) / 32 + 1) * 32 : kMaxConsumers + 32;
  static constexpr int min_blocks = (LX && LX * KR <= 96) ? 3 : ((LX && LX * KR <= 128) ? 2 : 1);
};

// CTAs per SM a tile of `sites` sites is sized for (registers and shared memory).
inline int ctas_per_sm(int sites) { return sites <= 96 ? 3 : (sites <= 128 ? 2 : 1); }

struct ItemPos {
  int t, z, y0, part;
};

__device__ __forceinline__ ItemPos decode_item(int it, const TmaTile& tt, int Lz) {
  const int tile = it / kSplit;
  ItemPos p;
  p.part = it % kSplit;
  p.y0 = (tile % tt.ntiles_y) * tt.k;
  const int rest = tile / tt.ntiles_y;
  p.z = rest % Lz;
  p.t = rest / Lz;
  return p;
}

template <typename PsiT, int LMODE, int LX, int KR, int HALO, int G>
__global__ void __launch_bounds__(TileLaunch<LX, KR>::threads, TileLaunch<LX, KR>::min_blocks)
    smear_hop_tma_kernel(const __grid_constant__ JobTable J, Geom g, TmaTile tt, unsigned int* status,
                         long long timeout_ns, int drop_stage) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  typedef typename LinkTraits<LMODE>::T LT;
  constexpr int NE = LinkTraits<LMODE>::NE;
  constexpr int NCL = 4 * NE;
  constexpr int COLS = 12;
  constexpr int NC = 12 * COLS;
  constexpr int VPI = 4 * COLS / kSplit;  // colour vectors per item
  constexpr int SPI = VPI / G;            // stages per item
  static_assert(VPI % G == 0 && COLS % G == 0, "G must divide the vectors of an item and the 12 columns");
  const int Lx = LX ? LX : g.sL[0];
  const int k = LX ? KR : tt.k;
  const int halo = LX ? HALO : tt.halo;
  const int rowsA = k + 2 * halo;
  const int rows = rowsA + 2 * k;
  const int Ly = g.sL[1], Lz = g.sL[2], V3 = g.V3;
  const int S = tt.stages;
  const int kLx = k * Lx;
  const int CS = rows * Lx;  // elements per colour region of a stage
  const int stage_elems = G * 3 * CS;
  // stage strides (elements) of a row, a colour and a vector: region-major
  // ([q][gg][row][x]) or, for halo tiles of a fixed shape, row-major
  // ([row][q][gg][x])
  constexpr bool RM = LX > 0 && HALO == 1;
  const int RS = RM ? 3 * G * Lx : Lx, QS = RM ? G * Lx : G * CS, VS = RM ? Lx : CS;
  const uint32_t stage_bytes = (uint32_t)stage_elems * sizeof(PsiT);
  const int lel = link_elems(NE, k, Lx, halo);
  const uint32_t link_bytes = (uint32_t)lel * sizeof(LT);
  const int lk_YH = 3 * NE * kLx;
  const int lk_ZB = lk_YH + (halo ? NE * Lx : 0);
  PsiT* st = reinterpret_cast<PsiT*>(smem_raw);
  LT* lbuf = reinterpret_cast<LT*>(smem_raw + (size_t)S * stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * stage_bytes + link_bytes);
  const uint32_t full0 = ptx::smem_addr(bars);
  const uint32_t empty0 = ptx::smem_addr(bars + S);
  const uint32_t lfull = ptx::smem_addr(bars + 2 * S);
  const uint32_t lempty = ptx::smem_addr(bars + 2 * S + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, tt.cwarps);
    }
    ptx::mbar_init(lfull, 1);
    ptx::mbar_init(lempty, tt.cwarps);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  // The next hop may begin its own set-up while this one runs; its reads and
  // writes of the spinor buffers wait for this grid to complete.
  ptx::launch_dependents();

  if (warp == tt.cwarps) {
    // ---------------- producer warp ----------------
    const int nlcopies = 4 * NE + (halo ? NE : 0);
    int gstage = 0, nitem = 0, last_link = -1;
    int s = 0, n = 0;  // slot and round of stage gstage (gstage = n*S + s), kept without division
    bool failed = false;
    const int total = tt.nitems * J.njobs;
    for (int it = blockIdx.x; it < total && !failed; it += gridDim.x, ++nitem) {
      const int job = it / tt.nitems;
      const ItemPos p = decode_item(it - job * tt.nitems, tt, Lz);
      const int zm = (p.z - 1 + Lz) % Lz, zp = (p.z + 1) % Lz;
      const int ym = (p.y0 - 1 + Ly) % Ly, yp = (p.y0 + k) % Ly;
      // links of the tile, once the consumers hold the previous item's in registers
      if (nitem > 0) {
        const bool ok = ptx::mbar_wait_bounded(lempty, (nitem - 1) & 1, timeout_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicOr(status, kStatusEmptyWait);
          break;
        }
      }
      if (lane == 0) ptx::mbar_arrive_expect_tx(lfull, link_bytes);
      __syncwarp();
      const LT* Ut = static_cast<const LT*>(J.j[job].U) + (size_t)p.t * NCL * V3;
      for (int cp = lane; cp < nlcopies; cp += 32) {
        int comp, src_off, dst, n;
        if (cp < 3 * NE) {  // F[i][e]
          const int i = cp / NE, e = cp % NE;
          const int mu = i == 0 ? g.sd[0] : (i == 1 ? g.sd[1] : g.sd[2]);  // no dynamic index into the parameter
          comp = mu * NE + e;
          src_off = (p.z * Ly + p.y0) * Lx;
          dst = (i * NE + e) * kLx;
          n = kLx;
        } else if (cp < 4 * NE) {  // ZB[e]
          const int e = cp - 3 * NE;
          comp = g.sd[2] * NE + e;
          src_off = (zm * Ly + p.y0) * Lx;
          dst = lk_ZB + e * kLx;
          n = kLx;
        } else {  // YH[e]
          const int e = cp - 4 * NE;
          comp = g.sd[1] * NE + e;
          src_off = (p.z * Ly + ym) * Lx;
          dst = lk_YH + e * Lx;
          n = Lx;
        }
        ptx::bulk_g2s(ptx::smem_addr(lbuf + dst), Ut + (size_t)comp * V3 + src_off, (uint32_t)n * sizeof(LT), lfull);
      }
      last_link = nitem;
      // the item's colour vectors, G per stage
      // spinors are read (and, by the consumers, written) only after the
      // previous kernel in the stream has completed; links do not depend on it
      if (nitem == 0) ptx::wait_dependencies();
      const PsiT* base_t = static_cast<const PsiT*>(J.j[job].in) + (size_t)p.t * NC * V3;
      // Whole-plane tiles stage planes z-1, z, z+1 as rows 0..3k-1; where the
      // three planes are consecutive in memory one copy per colour moves them.
      // Halo tiles: rows y0-1 .. y0+k of plane z in one run unless the y halo
      // wraps (then two), rows y0 .. y0+k-1 of planes z-1 and z+1 one each.
      const bool ywrap_lo = p.y0 == 0, ywrap_hi = p.y0 + k == Ly;
      int npieces = ywrap_lo || ywrap_hi ? 4 : 3;
      if (!halo) npieces = Lz < 3 ? 3 : (p.z == 0 || p.z == Lz - 1 ? 2 : 1);
      const int ncopies = G * 3 * npieces;
      for (int j = 0; j < SPI; ++j, ++gstage, s = s + 1 == S ? 0 : s + 1, n += s == 0) {
        if (n > 0) {
          const bool ok = ptx::mbar_wait_bounded(empty0 + 8 * s, (n - 1) & 1, timeout_ns);
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicOr(status, kStatusEmptyWait);
            failed = true;
            break;
          }
        }
        if (gstage == drop_stage) continue;  // test hook: the waits for this stage run out
        if (lane == 0) ptx::mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
        __syncwarp();
        if constexpr (RM) {
          // rows y0-1 (0), y0..y0+k-1 (1..k), y0+k (k+1) of plane z, then
          // the k rows of planes z-1 and z+1: five boxes of all three colours
          // and the stage's G vectors
          if (lane < 5) {
            const int v = p.part * VPI + j * G;
            const int c1 = v % COLS, c2 = 3 * (v / COLS) + COLS * p.t;
            const int dst_row = lane == 0 ? 0 : (lane == 1 ? 1 : (lane == 2 ? k + 1 : (lane == 3 ? k + 2 : 2 * k + 2)));
            const int src_y = lane == 0 ? ym : (lane == 2 ? yp : p.y0);
            const int src_z = lane == 3 ? zm : (lane == 4 ? zp : p.z);
            const CUtensorMap* m = (lane == 0 || lane == 2) ? &J.tmap_row[job] : &J.tmap[job];
            ptx::tensor_g2s_4d(ptx::smem_addr(st + (size_t)s * stage_elems + (size_t)dst_row * RS), m, 0, c1, c2,
                               src_y + Ly * src_z, full0 + 8 * s);
          }
          continue;
        }
        if (tt.use_tmap && npieces == 1) {
          // one box: x, rows of planes z-1..z+1, the stage's G vectors, 3 colours
          const int v = p.part * VPI + j * G;
          if (lane == 0)
            ptx::tensor_g2s_4d(ptx::smem_addr(st + (size_t)s * stage_elems), &J.tmap[job], 0, zm * Ly, v % COLS,
                               3 * (v / COLS) + COLS * p.t, full0 + 8 * s);
          continue;
        }
        for (int cp = lane; cp < ncopies; cp += 32) {
          const int gg = cp / (3 * npieces), rem = cp % (3 * npieces);
          const int c = rem / npieces, piece = rem % npieces;
          int src_off, dst_row, nrows;
          if (halo) {
            const int pz = npieces == 3 ? piece + 1 : piece;  // 0, 1: plane z in two runs; 1 alone: one run
            if (pz == 0) {  // the run before the wrap
              src_off = (p.z * Ly + ym) * Lx; dst_row = 0; nrows = ywrap_lo ? 1 : k + 1;
            } else if (pz == 1) {
              if (npieces == 3) {
                src_off = (p.z * Ly + ym) * Lx; dst_row = 0; nrows = k + 2;
              } else if (ywrap_lo) {
                src_off = (p.z * Ly + p.y0) * Lx; dst_row = 1; nrows = k + 1;
              } else {
                src_off = (p.z * Ly + yp) * Lx; dst_row = k + 1; nrows = 1;
              }
            } else if (pz == 2) {
              src_off = (zm * Ly + p.y0) * Lx; dst_row = rowsA; nrows = k;
            } else {
              src_off = (zp * Ly + p.y0) * Lx; dst_row = rowsA + k; nrows = k;
            }
          } else if (npieces == 1) {  // planes z-1, z, z+1 in one run
            src_off = zm * Ly * Lx; dst_row = 0; nrows = 3 * k;
          } else if (npieces == 2) {  // z = 0: z-1 wraps; z = Lz-1: z+1 wraps
            const bool first = piece == 0;
            if (p.z == 0) {
              src_off = (first ? zm : p.z) * Ly * Lx; dst_row = first ? 0 : k; nrows = first ? k : 2 * k;
            } else {
              src_off = (first ? zm : zp) * Ly * Lx; dst_row = first ? 0 : 2 * k; nrows = first ? 2 * k : k;
            }
          } else {
            switch (piece) {
              case 0: src_off = zm * Ly * Lx; dst_row = 0; nrows = k; break;
              case 1: src_off = p.z * Ly * Lx; dst_row = k; nrows = k; break;
              default: src_off = zp * Ly * Lx; dst_row = 2 * k; nrows = k; break;
            }
          }
          const int v = p.part * VPI + j * G + gg;
          const int comp = (v / COLS) * 3 * COLS + c * COLS + (v % COLS);
          const PsiT* src = base_t + (size_t)comp * V3 + src_off;
          const uint32_t dst = ptx::smem_addr(st + (size_t)s * stage_elems + (c * G + gg) * CS + dst_row * Lx);
          ptx::bulk_g2s(dst, src, (uint32_t)(nrows * Lx) * sizeof(PsiT), full0 + 8 * s);
        }
      }
    }
    // Drain: every copy this warp issued (the last S stages and the last
    // link fill) has landed before the CTA may exit.
    if (lane == 0) {
      for (int u = (gstage > S ? gstage - S : 0); u < gstage; ++u)
        if (u != drop_stage && !ptx::mbar_wait_bounded(full0 + 8 * (u % S), (u / S) & 1, timeout_ns))
          atomicOr(status, kStatusDrain);
      if (last_link >= 0 && !ptx::mbar_wait_bounded(lfull, last_link & 1, timeout_ns)) atomicOr(status, kStatusDrain);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int ctid = threadIdx.x;
  const bool active = ctid < kLx;
  const int r = active ? ctid / Lx : 0;
  const int x = active ? ctid % Lx : 0;
  const int xm = x == 0 ? Lx - 1 : x - 1;
  // shared-memory offsets (elements, within a colour region) of the seven
  // sites; rows of plane z from bz, of planes z-1 and z+1 from bzm and bzp
  const int bz = halo ? 0 : k, bzm = halo ? rowsA : 0, bzp = halo ? rowsA + k : 2 * k;
  const int rc = bz + r + halo;
  const int oc = rc * RS + x;
  const int yp_row = bz + (halo ? r + 2 : (r + 1 == k ? 0 : r + 1));
  const int ym_row = bz + (halo ? r : (r == 0 ? k - 1 : r - 1));
  const int of[3] = {rc * RS + (x + 1 == Lx ? 0 : x + 1), yp_row * RS + x, (bzp + r) * RS + x};
  const int ob[3] = {rc * RS + xm, ym_row * RS + x, (bzm + r) * RS + x};
  // link-buffer offsets of this site's six links
  const int lf = r * Lx + x;
  const bool yh = halo && r == 0;
  const int lyb = yh ? lk_YH + x : NE * kLx + (r == 0 ? k - 1 : r - 1) * Lx + x;
  const int lyb_stride = yh ? Lx : kLx;

  int s = 0, n = 0, nitem = 0;  // slot and round of the current stage
  const int total = tt.nitems * J.njobs;
  for (int it = blockIdx.x; it < total; it += gridDim.x, ++nitem) {
    const int job = it / tt.nitems;
    const ItemPos p = decode_item(it - job * tt.nitems, tt, Lz);
    const float kappa = J.j[job].kappa;
    bool ok = ptx::mbar_wait_bounded(lfull, nitem & 1, timeout_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(status, kStatusFullWait);
      return;
    }
    SiteLinks L;
    if (active) {
      float2 Uf[3][9], Ub[3][9];
#pragma unroll
      for (int i = 0; i < 3; ++i) link_from_smem<LMODE>(lbuf + i * NE * kLx + lf, kLx, Uf[i]);
      link_from_smem<LMODE>(lbuf + r * Lx + xm, kLx, Ub[0]);
      link_from_smem<LMODE>(lbuf + lyb, lyb_stride, Ub[1]);
      link_from_smem<LMODE>(lbuf + lk_ZB + lf, kLx, Ub[2]);
      make_site_links(Uf, Ub, kappa, L);
    }
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(lempty);
    if (nitem == 0) ptx::wait_dependencies();  // before the first spinor store

    const int s3 = x + Lx * ((p.y0 + r) + Ly * p.z);
    PsiT* outp = static_cast<PsiT*>(J.j[job].out) + (size_t)p.t * NC * V3 + s3;
    for (int j = 0; j < SPI; ++j, s = s + 1 == S ? 0 : s + 1, n += s == 0) {
      ok = ptx::mbar_wait_bounded(full0 + 8 * s, n & 1, timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(status, kStatusFullWait);
        return;
      }
      if (active) {
        const PsiT* sp = st + (size_t)s * stage_elems;
        const int v0 = p.part * VPI + j * G;
        PsiT* po = outp + (size_t)((v0 / COLS) * 3 * COLS + (v0 % COLS)) * V3;
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
          const PsiT* sg = sp + gg * VS;  // colour q of vector gg
          u64 nf[3][3], nb[3][3];
          float2 c[3], o[3];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              nf[i][q] = lds_pair(sg + of[i] + q * QS);
              nb[i][q] = lds_pair(sg + ob[i] + q * QS);
            }
#pragma unroll
          for (int a = 0; a < 3; ++a) c[a] = lds(sg + oc + a * QS);
          hop_vector(L, nf, nb, c, o);
#pragma unroll
          for (int a = 0; a < 3; ++a) st2(po + (gg + a * COLS) * V3, o[a]);
        }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(empty0 + 8 * s);
    }
  }
}

// Shared memory of one CTA: stages, link buffer, barriers.
template <typename PsiT, typename LT>
inline size_t tma_smem_bytes(const TmaTile& tt, int Lx, int NE) {
  const size_t stage_bytes = (size_t)tt.G * 3 * tt.rows * Lx * sizeof(PsiT);
  const size_t lbytes = (size_t)link_elems(NE, tt.k, Lx, tt.halo) * sizeof(LT);
  return tt.stages * stage_bytes + lbytes + (2 * tt.stages + 2) * sizeof(uint64_t);
}

template <typename PsiT, int LMODE, int LX, int KR, int HALO, int G>
int launch_tma_t(const HopLaunch& a) {
  auto kern = smear_hop_tma_kernel<PsiT, LMODE, LX, KR, HALO, G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.tt.smem);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear: smem attribute: %s", cudaGetErrorString(e));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.tt.grid);
  cfg.blockDim = dim3(32 * (a.tt.cwarps + 1));
  cfg.dynamicSmemBytes = a.tt.smem;
  cfg.stream = a.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope prof("smear_hop", a.stream);
  e = cudaLaunchKernelEx(&cfg, kern, a.jobs, a.g, a.tt, a.status, a.timeout_ns, a.drop_stage);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear hop (pipelined): %s", cudaGetErrorString(e));
  return check_launch("gauss_smear hop (pipelined)");
}

// Tile shapes with compile-time instantiations: (Lx, rows, halo).
#define QDPG_TMA_FIXED_SHAPES(X) \
  X(16, 16, 0)                   \
  X(16, 8, 1)                    \
  X(24, 8, 1)                    \
  X(24, 4, 1)                    \
  X(48, 4, 1)                    \
  X(48, 2, 1)                    \
  X(24, 12, 1)                   \
  X(48, 6, 1)                    \
  X(8, 8, 0)                     \
  X(12, 12, 0)

// Launch the instantiation for (PsiT, LMODE): a fixed tile shape if one
// matches, else the runtime-shape kernel.
template <typename PsiT, int LMODE>
int launch_tma_any(const HopLaunch& a) {
  const int Lx = a.g.sL[0];
  constexpr int G = 2;
#define QDPG_TMA_TRY(LXV, KV, HV)                                                 \
  if (Lx == LXV && a.tt.k == KV && a.tt.halo == HV && (HV == 0 || a.tt.use_rm)) \
    return launch_tma_t<PsiT, LMODE, LXV, KV, HV, G>(a);
  QDPG_TMA_FIXED_SHAPES(QDPG_TMA_TRY)
#undef QDPG_TMA_TRY
  return launch_tma_t<PsiT, LMODE, 0, 0, 0, G>(a);
}

int launch_tma_f32(int lprec, const HopLaunch& a);
int launch_tma_bf16(int lprec, const HopLaunch& a);

}  // namespace tma_smear
}  // namespace qdpg
