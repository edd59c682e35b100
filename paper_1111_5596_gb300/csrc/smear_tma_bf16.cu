// Instantiations of the pipelined smearing hop for BF16 propagator storage.
#include "smear_tma.cuh"

namespace qdpg {
namespace tma_smear {

int launch_tma_bf16(int lprec, const HopLaunch& a) {
  switch (lprec) {
    case QDPG_BF16_R12: return launch_tma_any<__nv_bfloat162, L_BF16_R12>(a);
    case QDPG_BF16: return launch_tma_any<__nv_bfloat162, L_BF16>(a);
    case QDPG_F32: return launch_tma_t<__nv_bfloat162, L_F32, 0, 0, 0, 2>(a);
    case QDPG_F32_R12: return launch_tma_t<__nv_bfloat162, L_F32_R12, 0, 0, 0, 2>(a);
  }
  return QDPG_ERR_UNSUPPORTED;
}

}  // namespace tma_smear
}  // namespace qdpg
