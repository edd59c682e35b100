// Dispatcher of the pipelined smearing hop (kernel in smear_tma.cuh): tile
// choice and the hand-off to the per-precision instantiations.
#include "smear_tma.cuh"

namespace qdpg {

namespace {

using tma_smear::TmaTile;

constexpr int kG = 2;  // colour vectors per pipeline stage

// Tile of k plane rows: the largest divisor k of Ly with Lx*k <= max_consumers.
bool pick_tile(const Geom& g, int esize, int max_consumers, int stages, TmaTile& tt) {
  const int Lx = g.sL[0], Ly = g.sL[1];
  if ((Lx * esize) % 16 != 0) return false;
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
  int S = stages > 0 ? stages : (int)(tma_smear::kSmemBudget / stage_bytes);
  if (S > tma_smear::kMaxStages) S = tma_smear::kMaxStages;
  if (S < 2 || S * stage_bytes + 16 * S > 227 * 1024) return false;
  tt.stages = S;
  return true;
}

// Default tile width: whole 16x16 planes; narrower tiles on wide planes,
// where smaller CTAs (several per SM) measured faster on GB300.
int default_consumers(const Geom& g) { return g.sL[0] >= 24 ? 128 : 256; }

}  // namespace

int launch_hop_tma(const void* in, void* out, const void* U, int lprec, int psi_prec, int cols, const Geom& g,
                   const int hop_mu[3], float kappa, cudaStream_t s) {
  if (cols != 12) return QDPG_ERR_UNSUPPORTED;
  for (int i = 0; i < 3; ++i)
    if (hop_mu[i] != g.sd[i]) return QDPG_ERR_UNSUPPORTED;
  const bool bf = psi_prec == QDPG_BF16;
  tma_smear::HopLaunch a;
  const int cons = debug_tile_consumers() > 0 ? debug_tile_consumers() : default_consumers(g);
  if (!pick_tile(g, bf ? 4 : 8, cons, debug_tile_stages(), a.tt)) return QDPG_ERR_UNSUPPORTED;
  a.status = device_status_word();
  if (!a.status) return QDPG_ERR_UNSUPPORTED;
  a.in = in;
  a.out = out;
  a.U = U;
  a.g = g;
  a.kappa = kappa;
  a.timeout_ns = wait_timeout_ns();
  a.drop_vec = debug_drop_vector();
  a.stream = s;
  return bf ? tma_smear::launch_tma_bf16(lprec, a) : tma_smear::launch_tma_f32(lprec, a);
}

}  // namespace qdpg
