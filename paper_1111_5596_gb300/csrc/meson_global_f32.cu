// The global-read meson kernels for F32 propagators.
#include "meson_global.cuh"

namespace qdpg {
namespace meson {

int launch_global_f32(const MesonPass& P, const Moms& M, const qdpg_field* S1, const qdpg_field* S2, double* out,
                       float2* sites, cudaStream_t s, int site_scale) {
  return launch_global_t<float2>(P, M, S1, S2, out, sites, s, site_scale);
}

}  // namespace meson
}  // namespace qdpg
