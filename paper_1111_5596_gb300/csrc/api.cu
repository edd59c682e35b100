// Host side of the C ABI: errors, lattice geometry, field headers.
#include <cstdio>
#include <cstring>
#include <new>

#include "qdpg_internal.h"

namespace qdpg {

namespace {
thread_local char g_msg[512] = "";
thread_local int g_code = QDPG_OK;
std::atomic<uint64_t> g_launches{0};
}  // namespace

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  g_code = code;
  return code;
}

int ok() { return QDPG_OK; }

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  count_launches(1);
  return QDPG_OK;
}

bool is_r12(int prec) { return prec == QDPG_F32_R12 || prec == QDPG_BF16_R12 || prec == QDPG_F16_R12; }
bool is_bf16(int prec) { return prec == QDPG_BF16 || prec == QDPG_BF16_R12; }
bool is_f16(int prec) { return prec == QDPG_F16 || prec == QDPG_F16_R12; }

int esize_of(int prec) {
  switch (prec) {
    case QDPG_F32:
    case QDPG_F32_R12: return 8;
    case QDPG_BF16:
    case QDPG_BF16_R12:
    case QDPG_F16:
    case QDPG_F16_R12: return 4;
    default: return 0;
  }
}

int ncomp_of(int kind, int prec) {
  if (prec < QDPG_F32 || prec > QDPG_F16_R12) return 0;
  if (is_r12(prec) && kind != QDPG_GAUGE) return 0;
  // float16 storage: propagators (scaled, site-major) and gauge links only
  if (prec == QDPG_F16 && kind != QDPG_PROPAGATOR && kind != QDPG_GAUGE) return 0;
  switch (kind) {
    case QDPG_COLOR_MATRIX: return 9;
    case QDPG_GAUGE: return is_r12(prec) ? 24 : 36;
    case QDPG_FERMION: return 12;
    case QDPG_PROPAGATOR: return 144;
    default: return 0;
  }
}

}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_version(void) { return 100; }

uint64_t qdpg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int qdpg_last_error(char* buf, size_t n) {
  if (buf && n) {
    strncpy(buf, g_msg, n - 1);
    buf[n - 1] = '\0';
  }
  return g_code;
}

int qdpg_lattice_create(const int dims[4], int j_decay, qdpg_lattice_t* out) {
  if (!dims || !out) return fail(QDPG_ERR_ARG, "lattice_create: null argument");
  if (j_decay < 0 || j_decay > 3) return fail(QDPG_ERR_ARG, "lattice_create: j_decay %d outside 0..3", j_decay);
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 1) return fail(QDPG_ERR_ARG, "lattice_create: dims[%d] = %d < 1", mu, dims[mu]);
    V *= dims[mu];
  }
  if (V >= (1LL << 31)) return fail(QDPG_ERR_ARG, "lattice_create: volume %lld too large", V);
  if (dims[j_decay] > 65535) return fail(QDPG_ERR_ARG, "lattice_create: more than 65535 timeslices");
  qdpg_lattice* lat = new (std::nothrow) qdpg_lattice;
  if (!lat) return fail(QDPG_ERR_NOMEM, "lattice_create: out of host memory");
  Geom& g = lat->g;
  for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
  g.jd = j_decay;
  int k = 0;
  for (int mu = 0; mu < 4; ++mu)
    if (mu != j_decay) {
      g.sd[k] = mu;
      g.sL[k] = dims[mu];
      ++k;
    }
  g.Nt = dims[j_decay];
  g.V3 = g.sL[0] * g.sL[1] * g.sL[2];
  g.V = V;
  *out = lat;
  return ok();
}

void qdpg_lattice_destroy(qdpg_lattice_t lat) { delete lat; }

size_t qdpg_field_bytes(qdpg_lattice_t lat, int kind, int prec) {
  if (!lat) return 0;
  int nc = ncomp_of(kind, prec);
  if (!nc) return 0;
  if (has_scale_record(kind)) return data_bytes_rounded(lat->g.V, nc, esize_of(prec)) + QDPG_SCALE_RECORD_BYTES;
  return (size_t)lat->g.V * (size_t)nc * (size_t)esize_of(prec);
}

int qdpg_field_wrap(qdpg_lattice_t lat, int kind, int prec, void* dev_ptr, size_t bytes,
                    qdpg_field_t* out) {
  if (!lat || !out) return fail(QDPG_ERR_ARG, "field_wrap: null argument");
  int nc = ncomp_of(kind, prec);
  if (!nc) return fail(QDPG_ERR_DTYPE, "field_wrap: precision %d not valid for kind %d", prec, kind);
  size_t need = qdpg_field_bytes(lat, kind, prec);
  if (!dev_ptr) return fail(QDPG_ERR_ARG, "field_wrap: null device pointer");
  if (bytes < need) return fail(QDPG_ERR_SHAPE, "field_wrap: buffer of %zu bytes < %zu needed", bytes, need);
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 16) return fail(QDPG_ERR_ARG, "field_wrap: pointer not 16-byte aligned");
  qdpg_field* f = new (std::nothrow) qdpg_field;
  if (!f) return fail(QDPG_ERR_NOMEM, "field_wrap: out of host memory");
  f->g = lat->g;
  f->kind = kind;
  f->prec = prec;
  f->ncomp = nc;
  f->esize = esize_of(prec);
  f->data = dev_ptr;
  f->bytes = bytes;
  f->rec = has_scale_record(kind) ? reinterpret_cast<ScaleRecord*>(static_cast<char*>(dev_ptr) +
                                                                    data_bytes_rounded(lat->g.V, nc, f->esize))
                                   : nullptr;
  *out = f;
  return ok();
}

void qdpg_field_release(qdpg_field_t f) { delete f; }

}  // extern "C"
