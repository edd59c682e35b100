// Gaussian (Wuppertal) smearing: the paper's SRC and SNK stages (Sec. 5,
// Fig. 4).  One iteration is the site-fused covariant hop
//
//   psi'(x) = psi(x) + kappa * sum_{i != j_decay} [ U_i(x) psi(x+i) + U_i(x-i)^dag psi(x-i) ]
//
// on every colour vector of the field (4 spins x 12 source columns for a
// propagator, 4 spins for a fermion).  A thread owns one site: it loads the
// six links it needs once (reconstructing row 2 for reconstruct-12 storage)
// and reuses them for all colour vectors of the site, so link traffic is
// paid once per site per iteration, not once per column.  Arithmetic is FP32
// for every storage precision.
#include <cmath>

#include "qdpg_internal.h"
#include "qdpg_profile.h"
#include "smear_common.cuh"

namespace qdpg {

namespace {

using namespace smear_dev;

constexpr int kSmearThreads = 128;

// Neighbour (t2, s3_2) of (t, coords c) one step along direction mu.
__device__ __forceinline__ void neighbour(const Geom& g, int t, const int c[3], int mu, int sign, int& t2, int& s32) {
  int cc[3] = {c[0], c[1], c[2]};
  t2 = t;
  if (mu == g.jd) {
    t2 = t + sign;
    t2 = t2 < 0 ? t2 + g.Nt : (t2 >= g.Nt ? t2 - g.Nt : t2);
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (g.sd[k] == mu) {
        int v = cc[k] + sign;
        cc[k] = v < 0 ? v + g.sL[k] : (v >= g.sL[k] ? v - g.sL[k] : v);
      }
  }
  s32 = cc[0] + g.sL[0] * (cc[1] + g.sL[1] * cc[2]);
}

struct HopDirs {
  int mu[3];
};

template <typename PsiT, int LMODE, int COLS>
__global__ void __launch_bounds__(kSmearThreads) smear_hop_kernel(const PsiT* __restrict__ in, PsiT* __restrict__ out,
                                                                   const void* __restrict__ U, Geom g, HopDirs hd,
                                                                   float kappa) {
  const int s3 = blockIdx.x * kSmearThreads + threadIdx.x;
  const int t = blockIdx.y;
  if (s3 >= g.V3) return;
  constexpr int NC = 12 * COLS;
  constexpr int NCL = (LMODE == L_F32_R12 || LMODE == L_BF16_R12) ? 24 : 36;
  const int V3 = g.V3;
  int c[3];
  c[0] = s3 % g.sL[0];
  c[1] = (s3 / g.sL[0]) % g.sL[1];
  c[2] = s3 / (g.sL[0] * g.sL[1]);

  float2 Uf[3][9], Ub[3][9];
  long long pf[3], pb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int mu = hd.mu[i];
    int tf, sf, tb, sb;
    neighbour(g, t, c, mu, +1, tf, sf);
    neighbour(g, t, c, mu, -1, tb, sb);
    pf[i] = (long long)tf * NC * V3 + sf;
    pb[i] = (long long)tb * NC * V3 + sb;
    load_link<LMODE>(U, (long long)t * NCL * V3 + s3, V3, mu, Uf[i]);
    load_link<LMODE>(U, (long long)tb * NCL * V3 + sb, V3, mu, Ub[i]);
  }
  const long long p0 = (long long)t * NC * V3 + s3;
  SiteLinks L;
  make_site_links(Uf, Ub, kappa, L);

#pragma unroll 1
  for (int v = 0; v < 4 * COLS; ++v) {
    const int cb = (v / COLS) * 3 * COLS + (v % COLS);  // comp of colour 0 of this vector
    u64 nf[3][3], nb[3][3];
    float2 c[3], o[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        nf[i][k] = pack2(ld2(in + pf[i] + (long long)(cb + k * COLS) * V3));
        nb[i][k] = pack2(ld2(in + pb[i] + (long long)(cb + k * COLS) * V3));
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = ld2(in + p0 + (long long)(cb + a * COLS) * V3);
    hop_vector(L, nf, nb, c, o);
#pragma unroll
    for (int a = 0; a < 3; ++a) st2(out + p0 + (long long)(cb + a * COLS) * V3, o[a]);
  }
}

template <typename PsiT, int LMODE>
int launch_hop_cols(const void* in, void* out, const void* U, const Geom& g, HopDirs hd, float kappa, int cols,
                    cudaStream_t s) {
  dim3 grid((g.V3 + kSmearThreads - 1) / kSmearThreads, g.Nt);
  ProfScope prof("smear_hop", s);
  if (cols == 12)
    smear_hop_kernel<PsiT, LMODE, 12><<<grid, kSmearThreads, 0, s>>>(static_cast<const PsiT*>(in),
                                                                    static_cast<PsiT*>(out), U, g, hd, kappa);
  else
    smear_hop_kernel<PsiT, LMODE, 1><<<grid, kSmearThreads, 0, s>>>(static_cast<const PsiT*>(in),
                                                                   static_cast<PsiT*>(out), U, g, hd, kappa);
  return check_launch("gauss_smear hop");
}

template <typename PsiT>
int launch_hop(const void* in, void* out, const void* U, int lprec, const Geom& g, HopDirs hd, float kappa, int cols,
               cudaStream_t s) {
  if (!debug_force_simple_hop()) {
    const int psi_prec = sizeof(PsiT) == 4 ? QDPG_BF16 : QDPG_F32;
    const int rc = launch_hop_tma(in, out, U, lprec, psi_prec, cols, g, hd.mu, kappa, s);
    if (rc != QDPG_ERR_UNSUPPORTED) return rc;
  }
  switch (lprec) {
    case QDPG_F32: return launch_hop_cols<PsiT, L_F32>(in, out, U, g, hd, kappa, cols, s);
    case QDPG_F32_R12: return launch_hop_cols<PsiT, L_F32_R12>(in, out, U, g, hd, kappa, cols, s);
    case QDPG_BF16: return launch_hop_cols<PsiT, L_BF16>(in, out, U, g, hd, kappa, cols, s);
    case QDPG_BF16_R12: return launch_hop_cols<PsiT, L_BF16_R12>(in, out, U, g, hd, kappa, cols, s);
  }
  return fail(QDPG_ERR_DTYPE, "gauss_smear: link precision %d", lprec);
}

// data *= 2^-shift (exact for normal numbers), one thread adds shift to exp.
template <typename T>
__global__ void __launch_bounds__(256) rescale_kernel(T* __restrict__ d, long long n, int shift, ScaleRecord* rec) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float2 v = ld2(d + i);
    st2(d + i, make_float2(ldexpf(v.x, -shift), ldexpf(v.y, -shift)));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rec->exp += shift;
}

bool same_lattice(const Geom& a, const Geom& b) {
  for (int mu = 0; mu < 4; ++mu)
    if (a.L[mu] != b.L[mu]) return false;
  return a.jd == b.jd;
}

// Float16 propagators: tensor-core hops with the per-iteration scale slots
// of psi's scale record (slot 0 = psi's scale, slot n = the result's).
int gauss_smear_f16(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay, qdpg_field_t scratch,
                    cudaStream_t s) {
  const Geom& g = psi->g;
  if (j_decay != g.jd)
    return fail(QDPG_ERR_UNSUPPORTED, "gauss_smear (f16): j_decay must be the lattice's decay direction");
  if (n_iter > QDPG_F16_MAX_ITER)
    return fail(QDPG_ERR_ARG, "gauss_smear (f16): at most %d iterations per call", QDPG_F16_MAX_ITER);
  if (!f16_hop_supported(g))
    return fail(QDPG_ERR_UNSUPPORTED,
                "gauss_smear (f16): lattice not served (first spatial extent must be a multiple of 4, at most 64)");
  const size_t bytes = f16_data_bytes(g.V);
  void* tmp = scratch ? scratch->data : nullptr;
  bool owned = false;
  if (!tmp) {
    const int rc = dev_alloc(&tmp, bytes, s, "gauss_smear scratch");
    if (rc != QDPG_OK) return rc;
    owned = true;
  }
  ScaleRecord* rec = psi->rec;
  int rc = f16_scale_init(&rec, &n_iter, 1, s);
  void* bufs[2] = {psi->data, tmp};
  for (int it = 0; it < n_iter && rc == QDPG_OK; ++it) {
    const F16HopJob job{bufs[it & 1], bufs[(it + 1) & 1], U->data, (float)kappa, rec};
    rc = launch_hop_f16(&job, 1, U->prec, g, it, s);
  }
  if (rc == QDPG_OK) rc = f16_scale_final(&rec, &n_iter, 1, s);
  if (rc == QDPG_OK && (n_iter & 1)) {
    cudaError_t e = cudaMemcpyAsync(psi->data, tmp, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) rc = fail(QDPG_ERR_CUDA, "gauss_smear: copy-back: %s", cudaGetErrorString(e));
  }
  if (owned) dev_free(tmp, s);
  return rc;
}

}  // namespace

RescalePlan rescale_plan(double kappa, int n_iter) {
  const double g = std::log2(1.0 + 6.0 * std::fabs(kappa));  // growth bound, bits per iteration
  RescalePlan p{0, 0};
  if (!(g > 0.0) || n_iter * g <= 40.0) return p;
  p.every = g >= 32.0 ? 1 : (int)std::floor(32.0 / g);
  p.shift = (int)std::floor(p.every * g);
  if (p.shift < 1) p.every = 0;
  return p;
}

int launch_rescale(void* data, int prec, long long nelem, int shift, ScaleRecord* rec, cudaStream_t s) {
  if (!rec) return fail(QDPG_ERR_ARG, "rescale: field has no scale record");
  long long blocks = (nelem + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (prec == QDPG_BF16)
    rescale_kernel<<<(int)blocks, 256, 0, s>>>(static_cast<__nv_bfloat162*>(data), nelem, shift, rec);
  else if (prec == QDPG_F32)
    rescale_kernel<<<(int)blocks, 256, 0, s>>>(static_cast<float2*>(data), nelem, shift, rec);
  else
    return fail(QDPG_ERR_DTYPE, "rescale: precision %d", prec);
  return check_launch("gauss_smear rescale");
}

// One hop psi -> out with whichever kernel serves the geometry (see launch_hop).
int launch_hop_any(const void* in, void* out, const void* U, int lprec, int psi_prec, int cols, const Geom& g,
                   const int hop_mu[3], float kappa, cudaStream_t s) {
  HopDirs hd;
  for (int i = 0; i < 3; ++i) hd.mu[i] = hop_mu[i];
  if (psi_prec == QDPG_BF16) return launch_hop<__nv_bfloat162>(in, out, U, lprec, g, hd, kappa, cols, s);
  return launch_hop<float2>(in, out, U, lprec, g, hd, kappa, cols, s);
}

// Argument checks shared by the smearing entry points.
int check_smear_args(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay, const char* who) {
  if (!U || !psi) return fail(QDPG_ERR_ARG, "%s: null field", who);
  if (U->kind != QDPG_GAUGE) return fail(QDPG_ERR_SHAPE, "%s: U must be a gauge field", who);
  if (psi->kind != QDPG_PROPAGATOR && psi->kind != QDPG_FERMION)
    return fail(QDPG_ERR_SHAPE, "%s: psi must be a propagator or fermion", who);
  if (psi->prec != QDPG_F32 && psi->prec != QDPG_BF16 && psi->prec != QDPG_F16)
    return fail(QDPG_ERR_DTYPE, "%s: psi storage must be F32, BF16 or F16", who);
  if (!same_lattice(U->g, psi->g)) return fail(QDPG_ERR_SHAPE, "%s: U and psi on different lattices", who);
  if ((psi->prec == QDPG_F16) != is_f16(U->prec))
    return fail(QDPG_ERR_DTYPE, "%s: F16 propagators go with F16/F16_R12 links and only with them", who);
  if (j_decay < 0 || j_decay > 3) return fail(QDPG_ERR_ARG, "%s: j_decay %d outside 0..3", who, j_decay);
  if (n_iter < 0) return fail(QDPG_ERR_ARG, "%s: negative iteration count", who);
  if (!(kappa == kappa) || kappa > 1e30 || kappa < -1e30) return fail(QDPG_ERR_ARG, "%s: kappa not finite", who);
  return QDPG_OK;
}

// n_iter FP32/BF16 hops of psi with tmp (a buffer of psi's data size) as
// the other half of the ping-pong pair, the power-of-two rescaling where the
// growth bound needs it, and the copy back into psi after an odd count.
int smear_loop(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay, void* tmp, cudaStream_t s,
               const char* who) {
  HopDirs hd;
  int k = 0;
  for (int mu = 0; mu < 4; ++mu)
    if (mu != j_decay) hd.mu[k++] = mu;
  const int cols = psi->kind == QDPG_PROPAGATOR ? 12 : 1;
  void* bufs[2] = {psi->data, tmp};
  int rc = QDPG_OK;
  const RescalePlan plan = rescale_plan((float)kappa, n_iter);  // the kernel's kappa
  for (int it = 0; it < n_iter && rc == QDPG_OK; ++it) {
    const void* in = bufs[it & 1];
    void* out = bufs[(it + 1) & 1];
    if (psi->prec == QDPG_BF16)
      rc = launch_hop<__nv_bfloat162>(in, out, U->data, U->prec, psi->g, hd, (float)kappa, cols, s);
    else
      rc = launch_hop<float2>(in, out, U->data, U->prec, psi->g, hd, (float)kappa, cols, s);
    if (rc == QDPG_OK && plan.every && (it + 1) % plan.every == 0)
      rc = launch_rescale(out, psi->prec, psi->g.V * psi->ncomp, plan.shift, psi->rec, s);
  }
  if (rc == QDPG_OK && (n_iter & 1)) {
    const cudaError_t e =
        cudaMemcpyAsync(psi->data, tmp, (size_t)psi->g.V * psi->ncomp * psi->esize, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) rc = fail(QDPG_ERR_CUDA, "%s: copy-back: %s", who, cudaGetErrorString(e));
  }
  return rc;
}

}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_gauss_smear(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay, qdpg_field_t scratch,
                     void* stream) {
  int rc = check_smear_args(U, psi, kappa, n_iter, j_decay, "gauss_smear");
  if (rc != QDPG_OK) return rc;
  if (scratch) {
    if (scratch->kind != psi->kind || scratch->prec != psi->prec || !same_lattice(scratch->g, psi->g))
      return fail(QDPG_ERR_SHAPE, "gauss_smear: scratch differs from psi in kind/precision/lattice");
    if (scratch->data == psi->data) return fail(QDPG_ERR_ARG, "gauss_smear: scratch aliases psi");
  }
  if (n_iter == 0) return ok();
  if (psi->prec == QDPG_F16) return gauss_smear_f16(U, psi, kappa, n_iter, j_decay, scratch, as_stream(stream));

  cudaStream_t s = as_stream(stream);
  void* tmp = scratch ? scratch->data : nullptr;
  bool owned = false;
  if (!tmp) {
    rc = dev_alloc(&tmp, (size_t)psi->g.V * psi->ncomp * psi->esize, s, "gauss_smear scratch");
    if (rc != QDPG_OK) return rc;
    owned = true;
  }
  rc = smear_loop(U, psi, kappa, n_iter, j_decay, tmp, s, "gauss_smear");
  if (owned) dev_free(tmp, s);
  return rc;
}

}  // extern "C"

// ---- smearing without any allocation ------------------------------------------
//
// Some callers cannot allocate device memory at the point where they smear: a
// host application whose own pool manager owns all device memory (the way
// the paper's QDP++ pool serves QUDA's allocations, Sec. 4.3), code that must
// not pay the implicit device synchronisation of cudaMalloc/cudaFree, or a
// process whose memory budget is fixed up front.  For them the ping-pong
// buffer lives in a static device array that the library owns, of fixed size
// kStaticScratchBytes; every GPU that loads the library holds it until exit.

#include <mutex>

namespace qdpg {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
int static_scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "gauss_smear_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(QDPG_ERR_UNSUPPORTED, "gauss_smear_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(QDPG_ERR_CUDA, "gauss_smear_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return QDPG_OK;
}

}  // namespace
}  // namespace qdpg

extern "C" int qdpg_gauss_smear_noalloc(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay,
                                        void* stream) {
  int rc = check_smear_args(U, psi, kappa, n_iter, j_decay, "gauss_smear_noalloc");
  if (rc != QDPG_OK) return rc;
  if (psi->prec != QDPG_F32 && psi->prec != QDPG_BF16)
    return fail(QDPG_ERR_DTYPE, "gauss_smear_noalloc: psi storage must be F32 or BF16");
  const size_t bytes = (size_t)psi->g.V * psi->ncomp * psi->esize;
  if (bytes > kStaticScratchBytes)
    return fail(QDPG_ERR_ARG, "gauss_smear_noalloc: field of %zu bytes exceeds the %zu-byte static scratch", bytes,
                kStaticScratchBytes);
  if (n_iter == 0) return ok();

  void* tmp = nullptr;
  rc = static_scratch_address(&tmp);
  if (rc) return rc;
  // The scratch is written in full by the first iteration before it is read,
  // so stale contents of an earlier call never leak into this one.
  return smear_loop(U, psi, kappa, n_iter, j_decay, tmp, as_stream(stream), "gauss_smear_noalloc");
}
