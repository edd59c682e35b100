// Tensor-core Gaussian-smearing hop for float16 propagators (the paper's
// SRC/SNK stages, Sec. 5, in reduced-precision storage).
//
// One iteration  psi'(x) = psi(x) + kappa sum_i [U_i(x) psi(x+i) + U_i(x-i)^dag psi(x-i)]
// acts on the 48 colour vectors of every site with the same six 3x3 link
// matrices.  Written with real numbers, for one site and one group of 16
// vectors it is a small dense product
//
//     D (16 vectors x 6 outputs) = sum_i  A_i (16 x 12) . B_i (12 x 6),
//
// A_i = the (re, im) of the three colours of the forward and backward
// neighbours in direction i, B_i = the two links written as real 6x6 blocks.
// Each of the three directions is one mma.sync m16n8k16 (float16 inputs,
// FP32 accumulation): K = 16 holds the forward neighbour's six numbers, two
// zeros, the backward neighbour's six numbers and two zeros; N = 8 holds the
// six outputs and two zero columns.  The float16 inputs are exact in the
// products and every sum is FP32; the result psi + kappa D is formed in
// FP32 and rounded to float16 once per iteration.
//
// Layout (qdpg.h): a propagator is three groups of 16 vectors, each stored
// site-major with the 48 float16 pairs of a site contiguous, so the A
// fragments of a warp's lanes are 24 consecutive words of shared memory.
//
// Scale: the field is stored as value * 2^-exp.  Hop k of a smearing call
// reads the largest stored magnitude M_k from the propagator's scale record
// (slot k), picks the shift Delta so that the bound
// (sqrt 2 + 6 |kappa| sqrt 6) M_k 2^-Delta of the output stays below 2^15,
// writes psi' * 2^-Delta, records exp_{k+1} = exp_k + Delta and folds the
// output's largest magnitude into slot k+1 with an atomic maximum.
//
// Pipeline: as in the FP32 kernel (smear_tma.cuh), a persistent CTA walks
// work items (tile of k plane rows at (t, z)); one producer warp streams,
// with bulk asynchronous copies, the tile's links and then per stage one
// vector group of the tile, its y halo rows and the same rows of planes
// z -+ 1; sixteen consumer warps (the default; eight with the tuning
// setting) each own four sites of the tile (eight with eight warps) and keep
// their link fragments in registers for the item's three stages.  The
// producer also writes the item's position into shared memory before it
// signals the links, so the consumers do not decode item indices, and each
// consumer computes its sites' stage offsets once (the tile shape is fixed).
// Every wait is bounded and reports through the device status word.
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {
namespace mma_smear {

constexpr int kMaxTile = 64;                         // sites per tile
constexpr int kMaxStages = 8;
constexpr int kWords = 48;                           // float16 pairs per site and vector group
constexpr int kTab = 12;                             // ints per site in the offset table

struct Job {
  const uint32_t* in;
  uint32_t* out;
  const uint32_t* U;
  float kappa;
  ScaleRecord* rec;
};
struct JobTable {
  int njobs;
  Job j[kMaxF16Jobs];
};

struct Tile {
  int k, ntiles_y, halo, rowsA, rows, T;
  int stages, nitems, grid, smem;
  int ne;          // stored entries per link: 6 (reconstruct-12) or 9
  int ls, lsh;     // link entry strides (words) of the tile rows and of the y-halo row
  int link_words;  // words of the link buffer
};

// Link buffer: types 0..2 = forward links U_{sd_i} on the tile's sites,
// type 3 = U_{sd_2} on the same rows of plane z-1, then (halo tiles) the
// y-halo row U_{sd_1}(row y0-1); 9 entries per link, entry stride ls.
__host__ __device__ inline int yh_base(int ls) { return 4 * 9 * ls; }

__device__ __forceinline__ void mma16816(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float2 h2f(uint32_t w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float x, float y) {
  __half2 h = __floats2half2_rn(x, y);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float cmul_re(float2 a, float2 b) { return a.x * b.x - a.y * b.y; }
__device__ __forceinline__ float cmul_im(float2 a, float2 b) { return a.x * b.y + a.y * b.x; }

// Output shift Delta for input magnitude m: the bound on the output
// (sqrt 2 + 6 |kappa| sqrt 6) m, with 2^-8 of slack for float16 links
// whose rows are not exactly unit vectors, times 2^-Delta is below 2^15.
__device__ __forceinline__ int delta_for(float m, float kappa) {
  const float b = m * (1.41421356f + 14.6969385f * fabsf(kappa)) * (1.f + 1.f / 256.f);
  if (!(b > 0.f)) return 0;
  int ex;
  frexpf(b, &ex);  // b < 2^ex
  return ex - 15;
}

// Offset q (0 = own, 1/2 = +-x, 3/4 = +-y, 5/6 = +-z) of a site's packed table.
__device__ __forceinline__ uint32_t offw(const uint32_t pk[4], int q) {
  return (q & 1) ? (pk[q >> 1] >> 16) : (pk[q >> 1] & 0xFFFFu);
}

struct ItemPos {
  int job, t, z, y0;
};
__device__ __forceinline__ ItemPos decode(int it, const Tile& tt, int Lz) {
  ItemPos p;
  p.job = it / tt.nitems;
  int r = it - p.job * tt.nitems;
  p.y0 = (r % tt.ntiles_y) * tt.k;
  r /= tt.ntiles_y;
  p.z = r % Lz;
  p.t = r / Lz;
  return p;
}

// NE: stored entries per link; CW: consumer warps; SPW: sites per consumer
// warp (CW * SPW >= the tile's sites; sites beyond the tile are clamped
// copies whose results are not stored).
template <int NE, int CW, int SPW>
__global__ void __launch_bounds__((CW + 1) * 32, 1)
    smear_hop_mma_kernel(const __grid_constant__ JobTable J, Geom g, Tile tt, int iter, unsigned int* status,
                         long long timeout_ns) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int Lx = g.sL[0], Ly = g.sL[1], Lz = g.sL[2], V3 = g.V3;
  const int k = tt.k, halo = tt.halo, rowsA = tt.rowsA, T = tt.T, S = tt.stages, ls = tt.ls, lsh = tt.lsh;
  const int stage_words = tt.rows * Lx * kWords;
  const uint32_t stage_bytes = (uint32_t)stage_words * 4u;
  uint32_t* st = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* lb = st + (size_t)S * stage_words;
  int* tab = reinterpret_cast<int*>(lb + tt.link_words);
  uint64_t* bars = reinterpret_cast<uint64_t*>(tab + T * kTab);
  int* hdr = reinterpret_cast<int*>(bars + 2 * S + 4);  // job, t, z, y0 of the item whose links are staged
  const uint32_t full0 = ptx::smem_addr(bars);
  const uint32_t empty0 = ptx::smem_addr(bars + S);
  const uint32_t lfull = ptx::smem_addr(bars + 2 * S);
  const uint32_t lempty = ptx::smem_addr(bars + 2 * S + 1);
  const uint32_t xdone = ptx::smem_addr(bars + 2 * S + 2);  // reconstruct-12 expansion done
  constexpr int kConsumerWarps = CW;
  constexpr int kSPW = SPW;  // sites per consumer warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = tt.nitems * J.njobs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(full0 + 8 * s, 1);
      ptx::mbar_init(empty0 + 8 * s, kConsumerWarps);
    }
    ptx::mbar_init(lfull, 1);
    ptx::mbar_init(lempty, kConsumerWarps);
    ptx::mbar_init(xdone, kConsumerWarps);
    ptx::fence_mbar_init();
  }
  // per-site offsets: stage words of the site and its six neighbours, and
  // the link-buffer words of its three backward links
  for (int st_i = threadIdx.x; st_i < T; st_i += blockDim.x) {
    const int r = st_i / Lx, x = st_i - r * Lx;
    const int xp = x + 1 == Lx ? 0 : x + 1, xm = x == 0 ? Lx - 1 : x - 1;
    int* e = tab + st_i * kTab;
    e[0] = ((r + halo) * Lx + x) * kWords;
    e[1] = ((r + halo) * Lx + xp) * kWords;
    e[2] = ((r + halo) * Lx + xm) * kWords;
    e[3] = ((halo ? r + 2 : (r + 1 == k ? 0 : r + 1)) * Lx + x) * kWords;
    e[4] = ((halo ? r : (r == 0 ? k - 1 : r - 1)) * Lx + x) * kWords;
    e[5] = ((rowsA + k + r) * Lx + x) * kWords;
    e[6] = ((rowsA + r) * Lx + x) * kWords;
    e[7] = r * Lx + xm;  // type 0, stride ls
    const bool yh = halo && r == 0;
    e[8] = yh ? yh_base(ls) + x : 9 * ls + (r == 0 ? k - 1 : r - 1) * Lx + x;
    e[9] = yh ? lsh : ls;
    e[10] = 3 * 9 * ls + st_i;  // type 3 (z-backward), stride ls
    e[11] = 0;
  }
  __syncthreads();
  ptx::launch_dependents();

  if (warp == kConsumerWarps) {
    // ---------------- producer warp ----------------
    constexpr int NCL = 4 * NE;
    const int npieces = halo ? 5 : 3;
    const int nlcopies = 4 * NE + (halo ? NE : 0);
    const uint32_t link_bytes = (uint32_t)(4 * T + (halo ? Lx : 0)) * NE * 4u;
    int gstage = 0, nitem = 0, last_link = -1;
    int s = 0, n = 0;
    bool failed = false;
    for (int it = blockIdx.x; it < total && !failed; it += gridDim.x, ++nitem) {
      const ItemPos p = decode(it, tt, Lz);
      const int zm = p.z == 0 ? Lz - 1 : p.z - 1, zp = p.z + 1 == Lz ? 0 : p.z + 1;
      const int ym = p.y0 == 0 ? Ly - 1 : p.y0 - 1, yp = (p.y0 + k) % Ly;
      if (nitem > 0) {
        const bool ok = ptx::mbar_wait_bounded(lempty, (nitem - 1) & 1, timeout_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicOr(status, kStatusEmptyWait);
          break;
        }
      }
      if (lane == 0) {
        hdr[0] = p.job; hdr[1] = p.t; hdr[2] = p.z; hdr[3] = p.y0;
        ptx::mbar_arrive_expect_tx(lfull, link_bytes);
      }
      __syncwarp();
      const uint32_t* Ut = J.j[p.job].U + (size_t)p.t * NCL * V3;
      for (int cp = lane; cp < nlcopies; cp += 32) {
        int comp, src_off, dst, nsites;
        if (cp < 3 * NE) {
          const int i = cp / NE, e = cp - i * NE;
          const int mu = i == 0 ? g.sd[0] : (i == 1 ? g.sd[1] : g.sd[2]);
          comp = mu * NE + e;
          src_off = (p.z * Ly + p.y0) * Lx;
          dst = (i * 9 + e) * ls;
          nsites = T;
        } else if (cp < 4 * NE) {
          const int e = cp - 3 * NE;
          comp = g.sd[2] * NE + e;
          src_off = (zm * Ly + p.y0) * Lx;
          dst = (3 * 9 + e) * ls;
          nsites = T;
        } else {
          const int e = cp - 4 * NE;
          comp = g.sd[1] * NE + e;
          src_off = (p.z * Ly + ym) * Lx;
          dst = yh_base(ls) + e * lsh;
          nsites = Lx;
        }
        ptx::bulk_g2s(ptx::smem_addr(lb + dst), Ut + (size_t)comp * V3 + src_off, (uint32_t)nsites * 4u, lfull);
      }
      last_link = nitem;
      if (nitem == 0) ptx::wait_dependencies();  // spinors of the previous hop
      for (int vg = 0; vg < 3; ++vg, ++gstage, s = s + 1 == S ? 0 : s + 1, n += s == 0) {
        if (n > 0) {
          const bool ok = ptx::mbar_wait_bounded(empty0 + 8 * s, (n - 1) & 1, timeout_ns);
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicOr(status, kStatusEmptyWait);
            failed = true;
            break;
          }
        }
        if (lane == 0) ptx::mbar_arrive_expect_tx(full0 + 8 * s, stage_bytes);
        __syncwarp();
        // rows y0-1 .. y0+k of plane z in one run unless the y halo wraps
        // (then two), rows y0 .. y0+k-1 of planes z-1 and z+1 one each
        const bool wlo = p.y0 == 0, whi = p.y0 + k == Ly;
        const int np = halo ? (wlo || whi ? 4 : 3) : npieces;
        if (lane < np) {
          int z2, src_row, dst_row, nrows;
          if (halo) {
            const int pz = np == 3 ? lane + 1 : lane;  // 0, 1: plane z (1 alone: one run); 2: z-1; 3: z+1
            if (pz == 0) {
              z2 = p.z; src_row = ym; dst_row = 0; nrows = wlo ? 1 : k + 1;
            } else if (pz == 1) {
              z2 = p.z;
              if (np == 3) {
                src_row = ym; dst_row = 0; nrows = k + 2;
              } else if (wlo) {
                src_row = p.y0; dst_row = 1; nrows = k + 1;
              } else {
                src_row = yp; dst_row = k + 1; nrows = 1;
              }
            } else if (pz == 2) {
              z2 = zm; src_row = p.y0; dst_row = rowsA; nrows = k;
            } else {
              z2 = zp; src_row = p.y0; dst_row = rowsA + k; nrows = k;
            }
          } else {
            z2 = lane == 0 ? p.z : (lane == 1 ? zm : zp);
            src_row = p.y0;
            nrows = k;
            dst_row = lane == 0 ? 0 : (lane == 1 ? rowsA : rowsA + k);
          }
          const uint32_t* src = J.j[p.job].in + (((size_t)p.t * 3 + vg) * V3 + (size_t)(z2 * Ly + src_row) * Lx) * kWords;
          const uint32_t dst = ptx::smem_addr(st + (size_t)s * stage_words + (size_t)dst_row * Lx * kWords);
          ptx::bulk_g2s(dst, src, (uint32_t)(nrows * Lx * kWords) * 4u, full0 + 8 * s);
        }
      }
    }
    if (lane == 0) {
      for (int u = (gstage > S ? gstage - S : 0); u < gstage; ++u)
        if (!ptx::mbar_wait_bounded(full0 + 8 * (u % S), (u / S) & 1, timeout_ns)) atomicOr(status, kStatusDrain);
      if (last_link >= 0 && !ptx::mbar_wait_bounded(lfull, last_link & 1, timeout_ns)) atomicOr(status, kStatusDrain);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  // Lane (g8, j) holds rows g8 and g8+8 (vectors) and the k pair of colour
  // j of the A fragments, and column n = g8 (output colour g8/2, re or im)
  // of B.  Lanes j = 3 cover the zero-padded k entries: they read colour 2
  // (finite data) against B rows that are zero; lanes g8 >= 6 cover the
  // zero output columns.  So every lane runs the same straight-line code.
  const int g8 = lane >> 2, j = lane & 3;
  const int jj = j < 3 ? j : 2;
  const int a_out = g8 >> 1, part = g8 & 1;
  const int a_c = a_out < 3 ? a_out : 2;
  const bool bvalid = g8 < 6 && j < 3;
  const bool store_lane = j < 3;
  const int lo = g8 * 3 + jj;  // word of (vector g8, colour jj) in a site block
  // this warp's sites: warp, warp + 8, ...; nsw of them (clamped copies pad to pairs)
  const int nsw = (T - warp + kConsumerWarps - 1) / kConsumerWarps;
  ptx::wait_dependencies();  // the previous hop's spinors and scale slots

  // per site: stage offsets (own, +-x, +-y, +-z), the same for every item
  // (below 2^16 words: two per register)
  uint32_t off[kSPW][4];
#pragma unroll
  for (int si = 0; si < kSPW; ++si) {
    int sti = warp + si * kConsumerWarps;
    sti = sti < T ? sti : T - 1;
    const int* e = tab + sti * kTab;
#pragma unroll
    for (int q = 0; q < 4; ++q) off[si][q] = (uint32_t)e[2 * q] | (q < 3 ? (uint32_t)e[2 * q + 1] << 16 : 0u);
  }
  int cur_job = -1;
  float sc = 1.f, kap = 0.f, mx = 0.f;
  int s = 0, n = 0, nitem = 0;
  for (int it = blockIdx.x; it < total; it += gridDim.x, ++nitem) {
    bool ok = ptx::mbar_wait_bounded(lfull, nitem & 1, timeout_ns);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicOr(status, kStatusFullWait);
      return;
    }
    ItemPos p;
    p.job = hdr[0]; p.t = hdr[1]; p.z = hdr[2]; p.y0 = hdr[3];
    if (p.job != cur_job) {
      if (cur_job >= 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && mx > 0.f) atomicMax(reinterpret_cast<unsigned*>(&J.j[cur_job].rec->cmax[iter + 1]),
                                             __float_as_uint(mx));
      }
      cur_job = p.job;
      mx = 0.f;
      const ScaleRecord* rec = J.j[p.job].rec;
      kap = J.j[p.job].kappa;
      const int d = delta_for(rec->cmax[iter], kap);
      sc = ldexpf(1.f, -d);
      if (it == p.job * tt.nitems && threadIdx.x == 0) J.j[p.job].rec->cexp[iter + 1] = rec->cexp[iter] + d;
    }
    if (NE == 6) {
      // reconstruct row 2 of every staged link: row2 = (row0 x row1)^*
      const int nl = 4 * T + (halo ? Lx : 0);
      for (int l = threadIdx.x; l < nl; l += kConsumerWarps * 32) {
        uint32_t* b = l < 4 * T ? lb + (l / T) * 9 * ls + (l % T) : lb + yh_base(ls) + (l - 4 * T);
        const int stride = l < 4 * T ? ls : lsh;
        float2 r0[3], r1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          r0[c] = h2f(b[c * stride]);
          r1[c] = h2f(b[(3 + c) * stride]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
          const float re = cmul_re(r0[c1], r1[c2]) - cmul_re(r0[c2], r1[c1]);
          const float im = cmul_im(r0[c1], r1[c2]) - cmul_im(r0[c2], r1[c1]);
          b[(6 + c) * stride] = f2h(re, -im);
        }
      }
      // every warp's links are complete before any warp reads them
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(xdone);
      ok = ptx::mbar_wait_bounded(xdone, nitem & 1, timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(status, kStatusFullWait);
        return;
      }
    }
    // per site: link fragments B_i
    // (forward M = U: (Mr, -Mi) | (Mi, Mr); backward M = conj(U^T): (Ur, Ui) | (-Ui, Ur))
    uint32_t bf[kSPW][3][2];
#pragma unroll
    for (int si = 0; si < kSPW; ++si) {
      int sti = warp + si * kConsumerWarps;
      sti = sti < T ? sti : T - 1;
      const int* e = tab + sti * kTab;
      const int bs1 = e[9];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const uint32_t uf = lb[(i * 9 + a_c * 3 + jj) * ls + sti];
        const int bq = i == 0 ? e[7] : (i == 1 ? e[8] : e[10]);
        const uint32_t ub = lb[bq + (jj * 3 + a_c) * (i == 1 ? bs1 : ls)];
        const uint32_t ufs = __byte_perm(uf, 0u, 0x1032), ubs = __byte_perm(ub, 0u, 0x1032);
        const uint32_t b0 = part == 0 ? (uf ^ 0x80000000u) : ufs;
        const uint32_t b1 = part == 0 ? ub : (ubs ^ 0x00008000u);
        bf[si][i][0] = bvalid ? b0 : 0u;
        bf[si][i][1] = bvalid ? b1 : 0u;
      }
    }
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(lempty);

    const int item_base = Lx * (p.y0 + Ly * p.z);  // s3 of the tile's first site
    for (int vg = 0; vg < 3; ++vg, s = s + 1 == S ? 0 : s + 1, n += s == 0) {
      ok = ptx::mbar_wait_bounded(full0 + 8 * s, n & 1, timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(status, kStatusFullWait);
        return;
      }
      const uint32_t* sb = st + (size_t)s * stage_words + lo;
      uint32_t* outv = J.j[p.job].out + (((size_t)p.t * 3 + vg) * V3 + item_base) * kWords + lo;
#pragma unroll
      for (int si = 0; si < kSPW; si += 2) {
        if (si < nsw) {
          float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const uint32_t* fa = sb + offw(off[si], 1 + 2 * i);
            const uint32_t* ba = sb + offw(off[si], 2 + 2 * i);
            const uint32_t* fb = sb + offw(off[si + 1], 1 + 2 * i);
            const uint32_t* bb = sb + offw(off[si + 1], 2 + 2 * i);
            mma16816(d0, fa[0], fa[24], ba[0], ba[24], bf[si][i][0], bf[si][i][1]);
            mma16816(d1, fb[0], fb[24], bb[0], bb[24], bf[si + 1][i][0], bf[si + 1][i][1]);
          }
          // psi + kappa D in FP32, then the exact power-of-two rescale
          auto finish = [&](const float (&d)[4], uint32_t pk0, int sti) {
            const uint32_t* own = sb + (pk0 & 0xFFFFu);
            const float2 c0 = h2f(own[0]), c1 = h2f(own[24]);
            const float o0 = sc * fmaf(kap, d[0], c0.x), o1 = sc * fmaf(kap, d[1], c0.y);
            const float o2 = sc * fmaf(kap, d[2], c1.x), o3 = sc * fmaf(kap, d[3], c1.y);
            if (store_lane && sti < T) {
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(o0), fabsf(o1)), fmaxf(fabsf(o2), fabsf(o3))));
              uint32_t* po = outv + (size_t)sti * kWords;
              po[0] = f2h(o0, o1);
              po[24] = f2h(o2, o3);
            }
          };
          finish(d0, off[si][0], warp + si * kConsumerWarps);
          finish(d1, off[si + 1][0], warp + (si + 1) * kConsumerWarps);
        }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(empty0 + 8 * s);
    }
  }
  if (cur_job >= 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.f)
      atomicMax(reinterpret_cast<unsigned*>(&J.j[cur_job].rec->cmax[iter + 1]), __float_as_uint(mx));
  }
}

// Slot 0 of each job's record = the field's scale; slots 1..n zeroed.
struct RecTable {
  int njobs;
  ScaleRecord* rec[kMaxF16Jobs];
  int n_iter[kMaxF16Jobs];
};
__global__ void scale_init_kernel(const __grid_constant__ RecTable R) {
  ScaleRecord* rec = R.rec[blockIdx.x];
  const int n = R.n_iter[blockIdx.x];
  for (int i = threadIdx.x + 1; i <= n; i += blockDim.x) rec->cmax[i] = 0.f;
  if (threadIdx.x == 0) {
    rec->cmax[0] = rec->maxabs;
    rec->cexp[0] = rec->exp;
  }
}
// The field's scale after n iterations.
__global__ void scale_final_kernel(const __grid_constant__ RecTable R) {
  ScaleRecord* rec = R.rec[blockIdx.x];
  const int n = R.n_iter[blockIdx.x];
  if (threadIdx.x == 0) {
    rec->exp = rec->cexp[n];
    rec->maxabs = rec->cmax[n];
  }
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// Tile: the largest divisor k of Ly with k*Lx <= 64; pipeline depth from
// what shared memory leaves.
bool pick_tile(const Geom& g, int ne, int njobs, Tile& tt) {
  const int Lx = g.sL[0], Ly = g.sL[1];
  if (Lx % 4 != 0 || Lx > kMaxTile) return false;
  int best = 0;
  for (int k = 1; k <= Ly; ++k)
    if (Ly % k == 0 && Lx * k <= kMaxTile) best = k;
  if (best == 0) return false;
  tt.k = best;
  tt.ntiles_y = Ly / best;
  tt.halo = best == Ly ? 0 : 1;
  tt.rowsA = best + 2 * tt.halo;
  tt.rows = tt.rowsA + 2 * best;
  tt.T = Lx * best;
  tt.ne = ne;
  tt.ls = (tt.T + 4 + 3) / 4 * 4;
  tt.lsh = (Lx + 4 + 3) / 4 * 4;
  tt.link_words = 4 * 9 * tt.ls + (tt.halo ? 9 * tt.lsh : 0);
  const size_t stage_bytes = (size_t)tt.rows * Lx * kWords * 4;
  const size_t fixed = (size_t)tt.link_words * 4 + (size_t)tt.T * kTab * 4;
  const size_t budget = 225 * 1024;
  const size_t bar_bytes = (2 * kMaxStages + 4) * 8 + 16;
  if (fixed + 2 * stage_bytes + bar_bytes > budget) return false;
  int S = (int)((budget - fixed - bar_bytes) / stage_bytes);
  if (S > kMaxStages) S = kMaxStages;
  tt.stages = S;
  tt.smem = (int)(S * stage_bytes + fixed + (2 * S + 4) * 8 + 16);
  tt.nitems = tt.ntiles_y * g.sL[2] * g.Nt;
  const int nsm = sm_count();
  if (nsm <= 0) return false;
  const int total = tt.nitems * njobs;
  tt.grid = total < nsm ? total : nsm;
  return true;
}

template <int NE, int CW, int SPW>
int launch_t(const JobTable& J, const Geom& g, const Tile& tt, int iter, cudaStream_t s) {
  auto kern = smear_hop_mma_kernel<NE, CW, SPW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tt.smem);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear (f16): smem attribute: %s", cudaGetErrorString(e));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tt.grid);
  cfg.blockDim = dim3((CW + 1) * 32);
  cfg.dynamicSmemBytes = tt.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  unsigned int* status = device_status_word();
  if (!status) return fail(QDPG_ERR_CUDA, "gauss_smear (f16): no device status word");
  ProfScope prof("smear_hop_f16", s);
  e = cudaLaunchKernelEx(&cfg, kern, J, g, tt, iter, status, wait_timeout_ns());
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear (f16) hop: %s", cudaGetErrorString(e));
  return check_launch("gauss_smear (f16) hop");
}

}  // namespace mma_smear

bool f16_hop_supported(const Geom& g) {
  mma_smear::Tile tt;
  return mma_smear::pick_tile(g, 9, 1, tt);
}

int launch_hop_f16(const F16HopJob* jobs, int njobs, int lprec, const Geom& g, int iter, cudaStream_t s) {
  using namespace mma_smear;
  if (njobs < 1 || njobs > kMaxF16Jobs) return fail(QDPG_ERR_ARG, "gauss_smear (f16): %d jobs", njobs);
  if (lprec != QDPG_F16 && lprec != QDPG_F16_R12)
    return fail(QDPG_ERR_DTYPE, "gauss_smear (f16): links must be F16 or F16_R12");
  if (iter < 0 || iter >= kScaleSlots - 1) return fail(QDPG_ERR_ARG, "gauss_smear (f16): iteration %d", iter);
  const int ne = lprec == QDPG_F16_R12 ? 6 : 9;
  Tile tt;
  if (!pick_tile(g, ne, njobs, tt))
    return fail(QDPG_ERR_UNSUPPORTED,
                "gauss_smear (f16): lattice not served (first spatial extent must be a multiple of 4, at most 64)");
  JobTable J;
  J.njobs = njobs;
  for (int i = 0; i < njobs; ++i)
    J.j[i] = Job{static_cast<const uint32_t*>(jobs[i].in), static_cast<uint32_t*>(jobs[i].out),
                 static_cast<const uint32_t*>(jobs[i].U), jobs[i].kappa, jobs[i].rec};
  if (debug_f16_warps() == 8)
    return ne == 6 ? launch_t<6, 8, 8>(J, g, tt, iter, s) : launch_t<9, 8, 8>(J, g, tt, iter, s);
  // 48-site tiles (x extent 24 or 48): twelve consumer warps of four sites
  // each, rather than sixteen of which a quarter compute clamped copies
  if (tt.T == 48) return ne == 6 ? launch_t<6, 12, 4>(J, g, tt, iter, s) : launch_t<9, 12, 4>(J, g, tt, iter, s);
  return ne == 6 ? launch_t<6, 16, 4>(J, g, tt, iter, s) : launch_t<9, 16, 4>(J, g, tt, iter, s);
}

int f16_scale_init(ScaleRecord* const* recs, const int* n_iter, int njobs, cudaStream_t s) {
  using namespace mma_smear;
  if (njobs < 1 || njobs > kMaxF16Jobs) return fail(QDPG_ERR_ARG, "gauss_smear (f16): %d jobs", njobs);
  RecTable R;
  R.njobs = njobs;
  for (int i = 0; i < njobs; ++i) {
    R.rec[i] = recs[i];
    R.n_iter[i] = n_iter[i];
  }
  scale_init_kernel<<<njobs, 128, 0, s>>>(R);
  return check_launch("gauss_smear (f16) scale init");
}

int f16_scale_final(ScaleRecord* const* recs, const int* n_iter, int njobs, cudaStream_t s) {
  using namespace mma_smear;
  if (njobs < 1 || njobs > kMaxF16Jobs) return fail(QDPG_ERR_ARG, "gauss_smear (f16): %d jobs", njobs);
  RecTable R;
  R.njobs = njobs;
  for (int i = 0; i < njobs; ++i) {
    R.rec[i] = recs[i];
    R.n_iter[i] = n_iter[i];
  }
  scale_final_kernel<<<njobs, 32, 0, s>>>(R);
  return check_launch("gauss_smear (f16) scale final");
}

}  // namespace qdpg
