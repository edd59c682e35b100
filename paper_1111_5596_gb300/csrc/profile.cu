// Kernel-level timing with CUDA events on the launching stream.
//
// When enabled, every library kernel launch is bracketed by a pair of
// events recorded on the stream it is launched on; qdpg_profile_query sums
// the elapsed times per kernel name.  This is how per-stage wall-clock times
// (the paper times SRC, SNK and HAD separately, Sec. 5) and per-kernel
// durations for roofline figures are obtained without a profiler.
#include <mutex>
#include <string>
#include <vector>

#include "qdpg_internal.h"
#include "qdpg_profile.h"

namespace qdpg {

namespace {

struct Record {
  std::string name;
  cudaEvent_t start, stop;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Record> g_recs;     // records of the current window
std::vector<cudaEvent_t> g_pool;  // recycled events

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t s) : active_(false), idx_(0), s_(s) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_recs.size() >= 65536) return;
  // Events recorded into a stream capture cannot be timed later: launches
  // captured into a graph are not profiled.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  Record r{name, take_event(), take_event()};
  if (!r.start || !r.stop) return;
  cudaEventRecord(r.start, s);
  idx_ = g_recs.size();
  g_recs.push_back(r);
  active_ = true;
}

ProfScope::~ProfScope() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx_ < g_recs.size()) cudaEventRecord(g_recs[idx_].stop, s_);
}

}  // namespace qdpg

using namespace qdpg;

extern "C" {

int qdpg_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return ok();
}

int qdpg_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Record& r : g_recs) {
    g_pool.push_back(r.start);
    g_pool.push_back(r.stop);
  }
  g_recs.clear();
  return ok();
}

int qdpg_profile_query(const char* name, double* total_ms, uint64_t* launches) {
  if (!name || !total_ms || !launches) return fail(QDPG_ERR_ARG, "profile_query: null argument");
  std::lock_guard<std::mutex> lk(g_mu);
  double tot = 0.0;
  uint64_t n = 0;
  for (Record& r : g_recs) {
    if (r.name != name) continue;
    cudaError_t e = cudaEventSynchronize(r.stop);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "profile_query: %s", cudaGetErrorString(e));
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, r.start, r.stop);
    if (e != cudaSuccess) return fail(QDPG_ERR_CUDA, "profile_query: %s", cudaGetErrorString(e));
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *launches = n;
  return ok();
}

}  // extern "C"
