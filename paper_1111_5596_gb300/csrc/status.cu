// Device-side status word: kernels whose bounded waits give up record it here
// (never trap), and the host reads it back through qdpg_device_status.
#include <atomic>
#include <mutex>

#include "qdpg_internal.h"

namespace qdpg {

namespace {

static __device__ unsigned int g_device_status;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned int* g_ptr[kMaxDevices] = {};
long long g_timeout_ns = 1000000000LL;  // 1 s
int g_drop_vector = -1;
bool g_force_simple = false;
int g_tile_consumers = 0;  // 0: the library's default for the geometry
int g_tile_stages = 0;
int g_tile_grid = 0;
int g_f16_warps = 0;  // 0: the library's default (16)
int g_tensor_copy_off = 0;  // 1: the pipelined hop stages with bulk copies only
int g_fail_allocs = 0;      // the next this many device allocations fail (test hook)
long long g_stage_bytes = 0;  // host import/export chunk bound, 0 = default
int g_meson_form = 0;         // meson contraction kernel: 0 best available, 1 staged, 2 global reads
std::atomic<uint64_t> g_allocs{0};

}  // namespace

unsigned int* device_status_word() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    g_ptr[dev] = static_cast<unsigned int*>(p);
  }
  return g_ptr[dev];
}

long long wait_timeout_ns() { return g_timeout_ns; }
int debug_drop_vector() { return g_drop_vector; }
bool debug_force_simple_hop() { return g_force_simple; }
int debug_tile_consumers() { return g_tile_consumers; }
int debug_tile_stages() { return g_tile_stages; }
int debug_tile_grid() { return g_tile_grid; }
int debug_f16_warps() { return g_f16_warps; }
int debug_tensor_copy_off() { return g_tensor_copy_off; }
long long debug_stage_bytes() { return g_stage_bytes; }
int debug_meson_form() { return g_meson_form; }

// The library's memory pool on the current device, created on first use:
// its own stream-ordered pool (not the device's default one), which keeps up
// to kPoolKeepBytes of freed memory mapped between calls instead of handing
// it back at every synchronisation, so a repeated call does not map its
// temporaries anew.
constexpr uint64_t kPoolKeepBytes = uint64_t(4) << 30;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t lib_pool(cudaMemPool_t* out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s, const char* what) {
  *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_fail_allocs > 0) {
      --g_fail_allocs;
      return fail(QDPG_ERR_NOMEM, "%s: allocation of %zu bytes refused (test hook)", what, bytes);
    }
  }
  cudaMemPool_t pool = nullptr;
  cudaError_t e = lib_pool(&pool);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "%s: memory pool: %s", what, cudaGetErrorString(e));
  e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();  // the failed allocation leaves no sticky error
    return fail(QDPG_ERR_NOMEM, "%s: allocation of %zu bytes: %s", what, bytes, cudaGetErrorString(e));
  }
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return QDPG_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

}  // namespace qdpg

using namespace qdpg;

extern "C" {

uint64_t qdpg_device_alloc_count(void) { return g_allocs.load(std::memory_order_relaxed); }

int qdpg_device_pool_used(uint64_t* bytes) {
  if (!bytes) return fail(QDPG_ERR_ARG, "device_pool_used: null argument");
  cudaMemPool_t pool = nullptr;
  cudaError_t e = lib_pool(&pool);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, bytes);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "device_pool_used: %s", cudaGetErrorString(e));
  return ok();
}

int qdpg_device_status(void* stream) {
  unsigned int* w = device_status_word();
  if (!w) return fail(QDPG_ERR_CUDA, "device_status: no status word on this device");
  cudaStream_t s = as_stream(stream);
  unsigned int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, w, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "device_status: %s", cudaGetErrorString(e));
  if (h) {
    const unsigned int zero = 0;
    e = cudaMemcpyAsync(w, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "device_status: %s", cudaGetErrorString(e));
    return fail(QDPG_ERR_TIMEOUT, "device_status: a kernel's bounded wait gave up (flags 0x%x)", h);
  }
  return ok();
}

int qdpg_debug_set(int what, long long value) {
  std::lock_guard<std::mutex> lk(g_mu);
  switch (what) {
    case QDPG_DEBUG_WAIT_TIMEOUT_NS:
      if (value < 1000 || value > 60000000000LL) return fail(QDPG_ERR_ARG, "debug_set: timeout out of range");
      g_timeout_ns = value;
      return ok();
    case QDPG_DEBUG_DROP_STAGE:
      g_drop_vector = (int)value;
      return ok();
    case QDPG_DEBUG_FORCE_SIMPLE_HOP:
      g_force_simple = value != 0;
      return ok();
    case QDPG_TUNE_TILE_CONSUMERS:
      if (value != 0 && (value < 32 || value > 288))
        return fail(QDPG_ERR_ARG, "debug_set: tile consumers outside 32..288 (0 = default)");
      g_tile_consumers = (int)value;
      return ok();
    case QDPG_TUNE_STAGES:
      if (value != 0 && (value < 2 || value > 16)) return fail(QDPG_ERR_ARG, "debug_set: stages outside 2..16");
      g_tile_stages = (int)value;
      return ok();
    case QDPG_TUNE_F16_WARPS:
      if (value != 0 && value != 8 && value != 16) return fail(QDPG_ERR_ARG, "debug_set: f16 consumer warps must be 8 or 16");
      g_f16_warps = (int)value;
      return ok();
    case QDPG_TUNE_TENSOR_COPY:
      if (value < 0 || value > 1) return fail(QDPG_ERR_ARG, "debug_set: tensor-copy setting outside 0..1");
      g_tensor_copy_off = (int)value;
      return ok();
    case QDPG_DEBUG_STAGE_BYTES:
      if (value < 0 || value > (1LL << 40)) return fail(QDPG_ERR_ARG, "debug_set: staging bytes outside 0..2^40");
      g_stage_bytes = value;
      return ok();
    case QDPG_DEBUG_MESON_FORM:
      if (value < 0 || value > 2) return fail(QDPG_ERR_ARG, "debug_set: meson kernel form outside 0..2");
      g_meson_form = (int)value;
      return ok();
    case QDPG_DEBUG_FAIL_ALLOCS:
      if (value < 0 || value > 1000000) return fail(QDPG_ERR_ARG, "debug_set: failing allocations outside 0..1e6");
      g_fail_allocs = (int)value;
      return ok();
    case QDPG_TUNE_GRID:
      if (value < 0 || value > 1) return fail(QDPG_ERR_ARG, "debug_set: grid mode outside 0..1");
      g_tile_grid = (int)value;
      return ok();
  }
  return fail(QDPG_ERR_ARG, "debug_set: unknown setting %d", what);
}

}  // extern "C"
