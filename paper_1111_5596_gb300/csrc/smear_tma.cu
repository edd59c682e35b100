// Dispatcher of the pipelined smearing hop (kernel in smear_tma.cuh): tile
// choice and the hand-off to the per-precision instantiations.
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "smear_tma.cuh"
#include "tmap.h"

namespace qdpg {

namespace {

using tma_smear::TmaTile;

constexpr int kG = 2;  // colour vectors per pipeline stage

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cached[dev] = n;
  }
  return cached[dev];
}

// Tile of k plane rows: the largest divisor k of Ly with Lx*k <= max_consumers;
// pipeline depth from what shared memory leaves after the link buffer.
bool pick_tile(const Geom& g, int esize, int link_esize, int link_ne, int max_consumers, int stages, int grid_mode,
               int njobs, TmaTile& tt) {
  const int Lx = g.sL[0], Ly = g.sL[1];
  if ((Lx * esize) % 16 != 0 || (Lx * link_esize) % 16 != 0) return false;
  int best = 0;
  for (int k = 1; k <= Ly; ++k)
    if (Ly % k == 0 && Lx * k <= max_consumers) best = k;
  if (best == 0) return false;
  tt.k = best;
  tt.ntiles_y = Ly / best;
  tt.cwarps = (Lx * best + 31) / 32;
  tt.halo = best == Ly ? 0 : 1;
  tt.rowsA = best + 2 * tt.halo;
  tt.rows = tt.rowsA + 2 * best;
  tt.G = kG;
  const size_t stage_bytes = (size_t)kG * 3 * tt.rows * Lx * esize;
  const size_t link_bytes = (size_t)tma_smear::link_elems(link_ne, best, Lx, tt.halo) * link_esize;
  // small tiles leave room for two or three CTAs on the SM
  const int per_sm = tma_smear::ctas_per_sm(Lx * best);
  const size_t budget = (size_t)(222 / per_sm) * 1024;
  if (link_bytes + 2 * stage_bytes > budget) return false;
  int S = stages > 0 ? stages : (int)((budget - link_bytes) / stage_bytes);
  if (S > tma_smear::kMaxStages) S = tma_smear::kMaxStages;
  if (S < 2) return false;
  tt.stages = S;
  tt.smem = (int)(S * stage_bytes + link_bytes + (2 * S + 2) * sizeof(uint64_t));
  if (tt.smem > 227 * 1024) return false;
  tt.nitems = tt.ntiles_y * g.sL[2] * g.Nt * tma_smear::kSplit;
  const int nsm = sm_count();
  if (nsm <= 0) return false;
  // persistent: one resident wave of CTAs walks the items; otherwise one CTA per item
  const int total = tt.nitems * njobs;
  tt.grid = (grid_mode == 1 || total < nsm * per_sm) ? total : nsm * per_sm;
  return true;
}

// Default tile width: whole 16x16 planes; on wide planes (Lx >= 24) tiles
// of up to 288 sites for FP32 propagators (one CTA of nine consumer warps
// per SM) and of up to 128 for BF16 (several CTAs per SM), the faster
// choices measured on GB300.
int default_consumers(const Geom& g, int psi_prec) {
  if (g.sL[0] < 24) return 256;
  return psi_prec == QDPG_F32 ? 288 : 128;
}


// ---- launch configuration and the autotuning table ---------------------------

struct TileCfg {
  int consumers;  // most sites per tile
  int grid_mode;  // 0 persistent, 1 one CTA per item
  int stages;     // 0: as many as fit
};

struct TuneKey {
  int L[4], jd, psi, link;
  bool operator<(const TuneKey& o) const {
    return std::tie(L[0], L[1], L[2], L[3], jd, psi, link) <
           std::tie(o.L[0], o.L[1], o.L[2], o.L[3], o.jd, o.psi, o.link);
  }
};

std::mutex g_tune_mu;
std::map<TuneKey, std::pair<TileCfg, float>> g_tune;  // config and its measured microseconds per hop

TuneKey key_of(const Geom& g, int psi_prec, int lprec) {
  TuneKey k;
  for (int mu = 0; mu < 4; ++mu) k.L[mu] = g.L[mu];
  k.jd = g.jd;
  k.psi = psi_prec;
  k.link = lprec;
  return k;
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (the library links the runtime only).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

bool encode_map_2d(CUtensorMap* m, const void* base, int esize, uint64_t dim0, uint64_t dim1, uint64_t row_bytes,
                   uint32_t box0, uint32_t box1) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || (esize != 4 && esize != 8)) return false;
  const cuuint64_t dims[2] = {dim0, dim1};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_map_3d(CUtensorMap* m, const void* base, int esize, uint64_t dim0, uint64_t dim1, uint64_t dim2,
                   uint64_t stride1, uint64_t stride2, uint32_t box0, uint32_t box1, uint32_t box2) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || (esize != 4 && esize != 8)) return false;
  const cuuint64_t dims[3] = {dim0, dim1, dim2};
  const cuuint64_t strides[2] = {stride1, stride2};
  const cuuint32_t box[3] = {box0, box1, box2};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// The input propagator of one job as the 4-D tensor of the whole-plane
// tensor-map copies: (x; row = y + Ly*z; the 12 colour vectors of a spin
// row, stride V3; spin-row-colour + 12*t, stride 12*V3), box (Lx, 3k rows
// = planes z-1..z+1, G vectors, 3 colours) = one stage.
bool encode_psi_map(CUtensorMap* m, const void* in, const Geom& g, int esize, int k, int G) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t Lx = g.sL[0], V3 = g.V3;
  const cuuint64_t dims[4] = {Lx, (cuuint64_t)g.sL[1] * g.sL[2], 12, 12 * (cuuint64_t)g.Nt};
  const cuuint64_t strides[3] = {Lx * esize, V3 * esize, 12 * V3 * esize};
  const cuuint32_t box[4] = {(cuuint32_t)Lx, (cuuint32_t)(3 * k), (cuuint32_t)G, 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
            const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same tensor with the row outermost, for row-major halo-tile stages:
// dims (x; the 12 colour vectors of a spin row, stride V3; spin-row-colour +
// 12*t, stride 12*V3; row = y + Ly*z, stride Lx), box (Lx, G vectors, 3
// colours, `rows` rows), which lands in shared memory as [row][colour]
// [vector][x].
bool encode_psi_rm_map(CUtensorMap* m, const void* in, const Geom& g, int esize, int rows, int G) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t Lx = g.sL[0], V3 = g.V3;
  const cuuint64_t dims[4] = {Lx, 12, 12 * (cuuint64_t)g.Nt, (cuuint64_t)g.sL[1] * g.sL[2]};
  const cuuint64_t strides[3] = {V3 * esize, 12 * V3 * esize, Lx * esize};
  const cuuint32_t box[4] = {(cuuint32_t)Lx, (cuuint32_t)G, 3, (cuuint32_t)rows};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
            const_cast<void*>(in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The configuration a launch uses: explicit tuning settings first, then the
// autotuning table, then the defaults.
TileCfg current_cfg(const Geom& g, int psi_prec, int lprec) {
  TileCfg c{debug_tile_consumers(), debug_tile_grid(), debug_tile_stages()};
  const bool explicit_cfg = c.consumers || c.grid_mode || c.stages;
  if (!explicit_cfg) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key_of(g, psi_prec, lprec));
    if (it != g_tune.end()) return it->second.first;
  }
  if (!c.consumers) c.consumers = default_consumers(g, psi_prec);
  return c;
}

int launch_hop_tma_cfg(const tma_smear::JobPtrs* jobs, int njobs, int lprec, int psi_prec, const Geom& g,
                       cudaStream_t s, const TileCfg& cfg) {
  if (njobs < 1 || njobs > tma_smear::kMaxJobs) return QDPG_ERR_UNSUPPORTED;
  if ((psi_prec != QDPG_F32 && psi_prec != QDPG_BF16) || is_f16(lprec)) return QDPG_ERR_UNSUPPORTED;
  const bool bf = psi_prec == QDPG_BF16;
  tma_smear::HopLaunch a;
  const bool lr12 = lprec == QDPG_F32_R12 || lprec == QDPG_BF16_R12;
  const int lesize = (lprec == QDPG_F32 || lprec == QDPG_F32_R12) ? 8 : 4;
  if (!pick_tile(g, bf ? 4 : 8, lesize, lr12 ? 6 : 9, cfg.consumers, cfg.stages, cfg.grid_mode, njobs, a.tt))
    return QDPG_ERR_UNSUPPORTED;
  a.status = device_status_word();
  if (!a.status) return QDPG_ERR_UNSUPPORTED;
  a.jobs.njobs = njobs;
  for (int i = 0; i < njobs; ++i) a.jobs.j[i] = jobs[i];
  // whole-plane tiles whose stages are one box: tensor-map copies where
  // planes z-1..z+1 are consecutive (1 <= z <= Lz-2)
  const int esize = bf ? 4 : 8;
  const size_t stage_bytes = (size_t)a.tt.G * 3 * a.tt.rows * g.sL[0] * esize;
  a.tt.use_tmap = !debug_tensor_copy_off() && !a.tt.halo && g.sL[2] >= 3 && 3 * a.tt.k <= 256 && g.sL[0] <= 256 &&
                  stage_bytes % 128 == 0;
  for (int i = 0; i < njobs && a.tt.use_tmap; ++i)
    if (reinterpret_cast<uintptr_t>(jobs[i].in) % 16 != 0 ||
        !encode_psi_map(&a.jobs.tmap[i], jobs[i].in, g, esize, a.tt.k, a.tt.G))
      a.tt.use_tmap = 0;
  // halo tiles: row-major stages from five tensor-map copies (the fixed-shape
  // kernels; a row of a stage must start on a 128-byte boundary)
  a.tt.use_rm = !debug_tensor_copy_off() && a.tt.halo && a.tt.k <= 256 && g.sL[0] <= 256 &&
                ((size_t)3 * a.tt.G * g.sL[0] * esize) % 128 == 0;
  for (int i = 0; i < njobs && a.tt.use_rm; ++i)
    if (reinterpret_cast<uintptr_t>(jobs[i].in) % 16 != 0 ||
        !encode_psi_rm_map(&a.jobs.tmap[i], jobs[i].in, g, esize, a.tt.k, a.tt.G) ||
        !encode_psi_rm_map(&a.jobs.tmap_row[i], jobs[i].in, g, esize, 1, a.tt.G))
      a.tt.use_rm = 0;
  a.g = g;
  a.timeout_ns = wait_timeout_ns();
  a.drop_stage = debug_drop_vector();
  a.stream = s;
  return bf ? tma_smear::launch_tma_bf16(lprec, a) : tma_smear::launch_tma_f32(lprec, a);
}

int launch_one(const void* in, void* out, const void* U, int lprec, int psi_prec, const Geom& g, float kappa,
               cudaStream_t s, const TileCfg& cfg) {
  tma_smear::JobPtrs j{in, out, U, kappa};
  return launch_hop_tma_cfg(&j, 1, lprec, psi_prec, g, s, cfg);
}

bool tma_eligible(int cols, const Geom& g, const int hop_mu[3]) {
  if (cols != 12) return false;
  for (int i = 0; i < 3; ++i)
    if (hop_mu[i] != g.sd[i]) return false;
  return true;
}

}  // namespace

int launch_hop_tma(const void* in, void* out, const void* U, int lprec, int psi_prec, int cols, const Geom& g,
                   const int hop_mu[3], float kappa, cudaStream_t s) {
  if (!tma_eligible(cols, g, hop_mu)) return QDPG_ERR_UNSUPPORTED;
  return launch_one(in, out, U, lprec, psi_prec, g, kappa, s, current_cfg(g, psi_prec, lprec));
}

int launch_hop_tma_batch(const void* const* in, void* const* out, const void* const* U, const float* kappa, int njobs,
                         int lprec, int psi_prec, const Geom& g, const int hop_mu[3], cudaStream_t s) {
  if (!tma_eligible(12, g, hop_mu)) return QDPG_ERR_UNSUPPORTED;
  tma_smear::JobPtrs jobs[tma_smear::kMaxJobs];
  if (njobs > tma_smear::kMaxJobs) return QDPG_ERR_UNSUPPORTED;
  for (int i = 0; i < njobs; ++i) jobs[i] = tma_smear::JobPtrs{in[i], out[i], U[i], kappa[i]};
  return launch_hop_tma_cfg(jobs, njobs, lprec, psi_prec, g, s, current_cfg(g, psi_prec, lprec));
}

}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_tune_smear(qdpg_field_t U, qdpg_field_t psi, qdpg_field_t scratch, int j_decay, int reps, void* stream) {
  if (!U || !psi || !scratch) return fail(QDPG_ERR_ARG, "tune_smear: null field");
  if (U->kind != QDPG_GAUGE || psi->kind != QDPG_PROPAGATOR || scratch->kind != psi->kind ||
      scratch->prec != psi->prec || scratch->data == psi->data)
    return fail(QDPG_ERR_SHAPE, "tune_smear: needs a gauge field, a propagator and a distinct scratch propagator");
  if (reps < 1 || reps > 1000) return fail(QDPG_ERR_ARG, "tune_smear: reps outside 1..1000");
  if ((psi->prec != QDPG_F32 && psi->prec != QDPG_BF16) || is_f16(U->prec))
    return fail(QDPG_ERR_UNSUPPORTED, "tune_smear: only the F32/BF16 pipelined kernel has tunable launch shapes");
  const Geom& g = psi->g;
  int hop_mu[3], k = 0;
  for (int mu = 0; mu < 4; ++mu)
    if (mu != j_decay) hop_mu[k++] = mu;
  if (j_decay < 0 || j_decay > 3 || !tma_eligible(12, g, hop_mu))
    return fail(QDPG_ERR_UNSUPPORTED, "tune_smear: the pipelined kernel does not serve this geometry");
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(QDPG_ERR_CUDA, "tune_smear: event creation failed");
  static const int consumer_opts[] = {288, 256, 192, 128, 96, 64, 48, 32};
  TileCfg best{0, 0, 0};
  float best_us = 0.f;
  int last_k = -1;
  int rc = QDPG_OK;
  for (int ci = 0; ci < 8 && rc == QDPG_OK; ++ci) {
    // skip widths that give the same tile as the previous one
    int kk = 0;
    for (int d = 1; d <= g.sL[1]; ++d)
      if (g.sL[1] % d == 0 && g.sL[0] * d <= consumer_opts[ci]) kk = d;
    if (kk == 0 || kk == last_k) continue;
    last_k = kk;
    for (int gm = 0; gm < 2 && rc == QDPG_OK; ++gm) {
      const TileCfg cfg{consumer_opts[ci], gm, 0};
      int r = launch_one(psi->data, scratch->data, U->data, U->prec, psi->prec, g, 0.1f, s, cfg);
      if (r == QDPG_ERR_UNSUPPORTED) continue;
      if (r != QDPG_OK) { rc = r; break; }
      cudaEventRecord(e0, s);
      for (int i = 0; i < reps && r == QDPG_OK; ++i)
        r = launch_one(psi->data, scratch->data, U->data, U->prec, psi->prec, g, 0.1f, s, cfg);
      cudaEventRecord(e1, s);
      if (r != QDPG_OK) { rc = r; break; }
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(QDPG_ERR_CUDA, "tune_smear: timing failed"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us = ms * 1e3f / reps;
      if (best_us == 0.f || us < best_us) {
        best_us = us;
        best = cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QDPG_OK) return rc;
  if (best_us == 0.f) return fail(QDPG_ERR_UNSUPPORTED, "tune_smear: no configuration ran");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key_of(g, psi->prec, U->prec)] = {best, best_us};
  return ok();
}

int qdpg_tune_query(qdpg_field_t U, qdpg_field_t psi, int* consumers, int* grid_mode, float* us_per_hop) {
  if (!U || !psi || !consumers || !grid_mode || !us_per_hop) return fail(QDPG_ERR_ARG, "tune_query: null argument");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key_of(psi->g, psi->prec, U->prec));
  if (it == g_tune.end()) return fail(QDPG_ERR_ARG, "tune_query: no tuned configuration for these fields");
  *consumers = it->second.first.consumers;
  *grid_mode = it->second.first.grid_mode;
  *us_per_hop = it->second.second;
  return ok();
}

int qdpg_tune_save(const char* path) {
  if (!path) return fail(QDPG_ERR_ARG, "tune_save: null path");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = fopen(path, "w");
  if (!f) return fail(QDPG_ERR_ARG, "tune_save: cannot open %s", path);
  fprintf(f, "# L0 L1 L2 L3 j_decay psi_prec link_prec consumers grid_mode stages us_per_hop\n");
  for (const auto& kv : g_tune) {
    const TuneKey& k = kv.first;
    const TileCfg& c = kv.second.first;
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.3f\n", k.L[0], k.L[1], k.L[2], k.L[3], k.jd, k.psi, k.link,
            c.consumers, c.grid_mode, c.stages, kv.second.second);
  }
  fclose(f);
  return ok();
}

int qdpg_tune_load(const char* path) {
  if (!path) return fail(QDPG_ERR_ARG, "tune_load: null path");
  FILE* f = fopen(path, "r");
  if (!f) return fail(QDPG_ERR_ARG, "tune_load: cannot open %s", path);
  char line[512];
  int n = 0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    TuneKey k;
    TileCfg c;
    float us = 0.f;
    if (sscanf(line, "%d %d %d %d %d %d %d %d %d %d %f", &k.L[0], &k.L[1], &k.L[2], &k.L[3], &k.jd, &k.psi,
               &k.link, &c.consumers, &c.grid_mode, &c.stages, &us) != 11)
      continue;
    if (c.consumers < 32 || c.consumers > tma_smear::kMaxConsumers || c.grid_mode < 0 || c.grid_mode > 1 || c.stages < 0 || c.stages > 16)
      continue;
    g_tune[k] = {c, us};
    ++n;
  }
  fclose(f);
  return n > 0 ? ok() : fail(QDPG_ERR_ARG, "tune_load: no valid entries in %s", path);
}

}  // extern "C"
