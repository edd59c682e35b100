// Internal declarations shared by the translation units of libqdpg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdarg>
#include <cstddef>
#include <cstdint>

#include "qdpg.h"

namespace qdpg {

// Geometry as kernels see it (passed by value).
struct Geom {
  int L[4];    // extents per direction
  int jd;      // decay direction of the storage layout
  int sd[3];   // the other three directions, increasing
  int sL[3];   // their extents (s3 = x[sd0] + sL0*(x[sd1] + sL1*x[sd2]))
  int Nt;      // L[jd]
  int V3;      // sL0*sL1*sL2
  long long V; // Nt*V3
};

}  // namespace qdpg

struct qdpg_lattice {
  qdpg::Geom g;
};

namespace qdpg {

// Scale record of a propagator or fermion (device memory, after the data).
// The field's value is stored * 2^exp.  For float16 propagators maxabs and
// the per-iteration slots cmax/cexp of one smearing call (hop k reads slot k
// and writes slot k+1) drive the rescaling; FP32/BF16 fields use exp only.
constexpr int kScaleSlots = QDPG_F16_MAX_ITER + 1;
struct ScaleRecord {
  int exp;            // value = stored * 2^exp
  float maxabs;       // bound on |re|, |im| of the stored numbers
  unsigned tmpmax;    // scratch of the import's max reduction (float bits)
  int pad[13];
  float cmax[kScaleSlots];
  int cexp[kScaleSlots];
};
static_assert(sizeof(ScaleRecord) <= QDPG_SCALE_RECORD_BYTES, "scale record too large");

// Word index of (t, comp, s3) in a QDPG_F16 propagator (see qdpg.h).
__host__ __device__ inline long long f16_prop_index(int V3, int t, int comp, int s3) {
  const int sc = comp / 12, sp = comp - 12 * sc;  // sink (s, c); source (s', c')
  const int s = sc / 3, c = sc - 3 * s;
  const int v = s * 12 + sp;
  return ((long long)(t * 3 + (v >> 4)) * V3 + s3) * 48 + (v & 15) * 3 + c;
}

// Propagators and fermions (every precision) carry a scale record after
// their data, at the data size rounded up to 256 bytes.
inline bool has_scale_record(int kind) { return kind == QDPG_PROPAGATOR || kind == QDPG_FERMION; }
inline size_t data_bytes_rounded(long long V, int ncomp, int esize) {
  return ((size_t)V * ncomp * esize + 255) / 256 * 256;
}
inline size_t f16_data_bytes(long long V) { return data_bytes_rounded(V, 144, 4); }

}  // namespace qdpg

struct qdpg_field {
  qdpg::Geom g;
  int kind;
  int prec;
  int ncomp;     // complex components per site in device storage
  int esize;     // bytes per complex element
  void* data;    // borrowed device pointer
  size_t bytes;  // size of the wrapped buffer
  qdpg::ScaleRecord* rec;  // F16 propagators: the scale record inside the buffer; else null
};

namespace qdpg {

// Error reporting: sets the thread-local message and returns `code`.
int fail(int code, const char* fmt, ...);
int ok();
// Checks cudaGetLastError after a launch; counts the launch.
int check_launch(const char* what);
void count_launches(uint64_t n);

int ncomp_of(int kind, int prec);
int esize_of(int prec);
bool is_r12(int prec);
bool is_bf16(int prec);
bool is_f16(int prec);
// A QDPG_F16 propagator: site-major layout with a scale record.
inline bool is_f16_prop(const qdpg_field* f) { return f->kind == QDPG_PROPAGATOR && f->prec == QDPG_F16; }

// Per-device status word (device address) for bounded-wait timeouts.
unsigned int* device_status_word();
long long wait_timeout_ns();
int debug_drop_vector();
bool debug_force_simple_hop();
int debug_tile_consumers();  // max consumer threads per pipelined tile, 0 = per-geometry default
int debug_tile_stages();     // pipeline depth, 0 = as many as fit the shared-memory budget
int debug_tile_grid();       // 0: persistent CTAs, 1: one CTA per work item
int debug_tensor_copy_off();  // 1: no tensor-map copies in the pipelined FP32/BF16 hop
int debug_f16_warps();       // consumer warps of the float16 smearing kernel, 0 = default
// Stream-ordered device allocation of the library's temporaries (every
// allocation goes through here): QDPG_ERR_NOMEM with a message naming
// `what` on failure, including failures forced by QDPG_DEBUG_FAIL_ALLOCS.
int dev_alloc(void** p, size_t bytes, cudaStream_t s, const char* what);
long long debug_stage_bytes();  // chunk bound of the host-buffer import/export, 0 = default
int debug_meson_form();         // meson kernel: 0 best available, 1 staged S2, 2 global reads
void dev_free(void* p, cudaStream_t s);
constexpr unsigned int kStatusFullWait = 1u;   // consumer gave up waiting for data
constexpr unsigned int kStatusEmptyWait = 2u;  // producer gave up waiting for a free stage
constexpr unsigned int kStatusDrain = 4u;      // producer gave up draining its own copies

// Pipelined (bulk-copy) smearing hop; returns QDPG_ERR_UNSUPPORTED when the
// geometry or precision does not fit it, so the caller can use another kernel.
int launch_hop_tma(const void* in, void* out, const void* U, int lprec, int psi_prec, int cols, const Geom& g,
                   const int hop_mu[3], float kappa, cudaStream_t s);
// One hop with whichever smearing kernel serves the geometry.
int launch_hop_any(const void* in, void* out, const void* U, int lprec, int psi_prec, int cols, const Geom& g,
                   const int hop_mu[3], float kappa, cudaStream_t s);
// One pipelined hop over several jobs on the same lattice and precisions
// (each job its own in/out/links/kappa); QDPG_ERR_UNSUPPORTED as above.
int launch_hop_tma_batch(const void* const* in, void* const* out, const void* const* U, const float* kappa, int njobs,
                         int lprec, int psi_prec, const Geom& g, const int hop_mu[3], cudaStream_t s);

// Tensor-core smearing hop of float16 propagators (smear_mma.cu): one hop
// of up to kMaxF16Jobs jobs on the same lattice and link precision (F16 or
// F16_R12); `iter` is the hop's index within the jobs' smearing call (it
// reads scale slot iter and writes slot iter + 1 of each job's record).
constexpr int kMaxF16Jobs = 64;
struct F16HopJob {
  const void* in;
  void* out;
  const void* U;
  float kappa;
  ScaleRecord* rec;
};
bool f16_hop_supported(const Geom& g);
int launch_hop_f16(const F16HopJob* jobs, int njobs, int lprec, const Geom& g, int iter, cudaStream_t s);
// Scale slots of a smearing call: slot 0 = the field's scale, slots 1..n
// cleared (init); the field's scale = slot n (final).
int f16_scale_init(ScaleRecord* const* recs, const int* n_iter, int njobs, cudaStream_t s);
int f16_scale_final(ScaleRecord* const* recs, const int* n_iter, int njobs, cudaStream_t s);

// FP32/BF16 smearing whose growth bound N log2(1 + 6|kappa|) exceeds 40 bits
// is rescaled by an exact power of two every `every` iterations (`shift`
// bits down, added to the field's exp); every = 0: no rescaling.
struct RescalePlan {
  int every, shift;
};
RescalePlan rescale_plan(double kappa, int n_iter);
// data *= 2^-shift elementwise (F32 or BF16 storage); rec->exp += shift.
int launch_rescale(void* data, int prec, long long nelem, int shift, ScaleRecord* rec, cudaStream_t s);

// Tensor-core momentum projection of site values (momproj.cu); the sums are
// multiplied by 2^(ca * ra->exp + cb * rb->exp) (null records: 2^0), or by
// 2^chan_exp[chan] per channel where chan_exp (device memory) is given.
int launch_momproj(const Geom& g, const void* sites_dev, int n_chan, const int* moms, int n_mom, const int origin[4],
                   double* out_dev, const ScaleRecord* ra, int ca, const ScaleRecord* rb, int cb, cudaStream_t s,
                   const int* chan_exp = nullptr);
// meson_2pt/baryon_2pt with at least this many momenta project on the tensor cores.
constexpr int kTensorProjMinMom = 8;

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Device-side helpers --------------------------------------------------------

// Canonical site index of (t, s3) on geometry g.
__host__ __device__ inline long long canon_site(const Geom& g, int t, int s3) {
  int x[4];
  x[g.jd] = t;
  int r = s3;
  x[g.sd[0]] = r % g.sL[0];
  r /= g.sL[0];
  x[g.sd[1]] = r % g.sL[1];
  x[g.sd[2]] = r / g.sL[1];
  return (long long)x[0] + (long long)g.L[0] * (x[1] + (long long)g.L[1] * (x[2] + (long long)g.L[2] * x[3]));
}

}  // namespace qdpg
